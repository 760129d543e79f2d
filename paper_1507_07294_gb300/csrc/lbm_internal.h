// Host-side declarations shared by the C ABI and the kernel launchers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <string>

#include "lbm_device.cuh"

namespace lbm {

// Message returned by lbm_last_error(NULL) (per host thread).
void set_global_error(const std::string& msg);

// Upper bound on the number of per-block partial sums of the FP64 reduction.
constexpr int kReduceMaxParts = 1024;

// phi_ref: order parameter of the previous step (read by 16-bit storage); may equal phi.
cudaError_t launch_phi(const float* src, const float* phi_ref, float* phi, const Geometry& geo,
                       int pattern, cudaStream_t st);
cudaError_t launch_mu(const float* phi, float* mu, const Geometry& geo, const Physics& ph,
                      cudaStream_t st);
// The chemical-potential pass with a TMA-fetched halo brick; `map` describes phi as a
// 3D FP32 tensor (nx, ny, nz) with box (kTX + 8, kTY + 2, kTZ + 2).  Only for grids
// with mu_tma_shape_ok.  A block whose wait for its copy runs out after `polls` polls
// sets *err to 1 (default budget: mu_tma_default_polls()).
cudaError_t launch_mu_tma(const CUtensorMap& map, const float* phi, float* mu,
                          const Geometry& geo, const Physics& ph, int* err, long long polls,
                          cudaStream_t st);
long long mu_tma_default_polls();
bool mu_tma_shape_ok(const Geometry& geo);
// TMA box of the chemical-potential pass: (kTX + 8, kTY + 2, kTZ + 2)
constexpr unsigned kMuTmaBox[3] = {40, 10, 18};
// With err non-null and Geometry::stage set, the two-cell pass stages its stencils in
// shared memory by TMA bulk copies (k_collide2t), with a wait bounded by `polls` whose
// failure sets *err like launch_mu_tma.
cudaError_t launch_collide(const float* src, float* dst, const float* phi, const float* mu,
                           const Geometry& geo, const Physics& ph, int pattern, bool have_prev,
                           cudaStream_t st, int* err = nullptr, long long polls = 0);
// Grids whose rows k_collide2t can stage (nx of 64, 128 or 256).
bool stage_shape_ok(const Geometry& geo);
cudaError_t launch_che(const float* src, float* dst, const float* phi, const float* mu,
                       const Geometry& geo, const Physics& ph, int pattern, bool have_prev,
                       float tf, cudaStream_t st);
cudaError_t launch_fields(const float* src, const float* phi, const float* mu, float* out,
                          const Geometry& geo, const Physics& ph, int pattern, float tf,
                          cudaStream_t st);
cudaError_t launch_init(float* state, const float* phi, const float* mu, const float* u0,
                        const float* p0, const Geometry& geo, const Physics& ph, int pattern,
                        float tf, cudaStream_t st);
cudaError_t launch_gather(const float* src, const float* phi_ref, float* dense, const Geometry& geo,
                          int pattern, int slot, cudaStream_t st);
// All slots of `count` listed cells into out[slot * count + k] (cells checked by the
// caller to lie in [0, geo.n)).
cudaError_t launch_gather_at(const float* src, const float* phi_ref, const long long* cells,
                             long long count, float* out, const Geometry& geo, int pattern,
                             cudaStream_t st);
cudaError_t launch_scatter(float* state, const float* dense, const Geometry& geo, int pattern,
                           int slot, cudaStream_t st);
cudaError_t launch_convert(const double* in, float* out, int n, cudaStream_t st);
cudaError_t launch_widen(const float* in, double* out, int n, cudaStream_t st);
int reduce_parts(const Geometry& geo);
// Resident blocks per SM of k_collide (kernel 0), the order-parameter kernel (kernel 1:
// k_phi_rows with rows, else k_phi) or k_collide2 (kernel 3); 0 on error.
int resident_blocks_per_sm(int kernel, int storage, bool rows = false);
cudaError_t launch_reduce(const float* src, const float* phi, double* partial, double* out,
                          const Geometry& geo, int pattern, bool with_g, cudaStream_t st);
// Bytes of the tiled cell-state array for n cells.
inline size_t state_bytes(int n, int storage) {
  const int tb = storage == kF32 ? tile_bytes<kF32>() : tile_bytes<kF16>();
  return static_cast<size_t>((n + kTile - 1) / kTile) * tb;
}
// Warps of a one-cell-per-thread launch over n cells (one partial each in the fused sums).
int cell_warps(long long n);
// Stream-collide of the default model variant that also reduces the state it writes:
// per-warp partials into parts (5 x cell_warps(n) floats), then the fixed-order
// reduction through partial (5 x kReduceMaxParts) into out (5 doubles, as launch_reduce).
cudaError_t launch_collide_sums(const float* src, float* dst, const float* phi, const float* mu,
                                const Geometry& geo, const Physics& ph, int pattern,
                                bool have_prev, float* parts, double* partial, double* out,
                                cudaStream_t st, int* err = nullptr, long long polls = 0);

// The fixed-order FP64 reduction of the per-warp partials of the step sums (the tail of
// launch_collide_sums): parts -> partial -> out (5 doubles).
cudaError_t launch_step_sums_final(const float* parts, double* partial, double* out,
                                   const Geometry& geo, cudaStream_t st);

// Single-pass step (lbm_fused.cu): pattern AB, default model variant, grids with
// fused_shape_ok (nx a multiple of 32 with whole-tile rows, ny a multiple of 8).  phi_in
// and phi_out (distinct arrays) are read and written with 16-bit storage only.  `seg`
// planes per block column segment, `pf` L2 prefetch distance in planes (0: none).  With
// parts non-null the launch also reduces the state it writes, like launch_collide_sums.
bool fused_shape_ok(const Geometry& geo);
int fused_default_segment(const Geometry& geo, int sms);
cudaError_t launch_fused(const float* src, float* dst, const float* phi_in, float* phi_out,
                         const Geometry& geo, const Physics& ph, bool have_prev, int seg, int pf,
                         float* parts, double* partial, double* out, cudaStream_t st);

}  // namespace lbm
