// C ABI of the solver (declared in include/lbm.h): context life cycle, parameter
// mapping, allocation through the caller's allocator, and the launch sequence of one
// time step.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "lbm.h"
#include "lbm_capi_internal.h"
#include "lbm_internal.h"

struct lbm_ctx {
  lbm_grid grid{};
  lbm_params params{};
  lbm::Geometry geo{};
  lbm::Physics ph{};
  lbm_allocator alloc{};
  bool have_alloc = false;
  cudaStream_t stream = nullptr;

  // device memory
  float* pop[2] = {nullptr, nullptr};  // tiled cell state(s): 22 populations + phi u
  int cur = 0;             // array holding the current state (pattern AB)
  float* phi = nullptr;    // order parameter of the current step: phi_buf[phi_sel]
  // phi_buf[1] exists only with 16-bit storage on grids the single-pass step takes: that
  // step reads the previous step's phi (the shift of slot 0) from one array while it
  // writes the new phi into the other
  float* phi_buf[2] = {nullptr, nullptr};
  int phi_sel = 0;
  float* mu = nullptr;     // chemical potential of the current step
  float* stage = nullptr;  // 7 planes: field read-out (rho, p, u, phi, mu), state
                           // gather/scatter, initial u and p
  double* partial = nullptr;  // reduction partials
  double* red = nullptr;      // 5 reduction results; red[7] holds the device error word
  float* step_parts = nullptr;   // per-warp partials of the fused step sums (FP32 sums of
                                 // 32 cells and a count: exact in float)

  // TMA descriptors of phi_buf[0], phi_buf[1] for the chemical-potential pass (when the
  // grid allows it)
  CUtensorMap phi_map[2]{};
  bool have_phi_map = false;
  bool use_phi_map = true;
  long long tma_polls = -1;  // poll budget of the copy's wait; -1: the kernel default
  int row_tiles = 0;         // Geometry::row_tiles when LBM_TUNE_ROWS is on
  int pairs = 0;             // Geometry::pairs when LBM_TUNE_CELL_PAIRS is on
  int stage_rows = 0;        // Geometry::stage when LBM_TUNE_STENCIL_STAGE is on
  int prefetch_sums = 0;     // Geometry::prefetch_collide of the steps that sum their result

  // single-pass step (lbm_fused.cu): enabled, planes per segment (0: by grid size), L2
  // prefetch distance in planes
  bool use_fused = false;
  int fused_seg = 0;
  int fused_pf = 0;
  int sms = 0;

  // CUDA graphs of two consecutive steps, one per parity of the stored state (which
  // array is current, or the AA step parity, and which phi array is current), replayed
  // by lbm_step; captured on first use, dropped whenever a kernel argument changes
  // (tuning, prescribed velocity)
  cudaGraphExec_t pair_graph[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaStream_t capture_stream = nullptr;
  bool use_graphs = true;

  // interface-tracking mode (0: coupled): prescribed velocity kind, amplitude, period
  int vel_kind = 0;
  double vel_U = 0.0, vel_period = 1.0;

  long long step = 0;
  bool odd = false;        // parity of the stored populations (pattern AA)
  bool have_prev = false;  // phiu holds the previous step's phi u
  bool initialized = false;
  bool retired = false;    // a TMA copy may have outlived its block: no more launches

  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events[3];

  std::string err;
};

namespace {

thread_local std::string g_create_error;

lbm_status fail(lbm_ctx* ctx, lbm_status st, const std::string& msg) {
  if (ctx)
    ctx->err = msg;
  else
    g_create_error = msg;
  return st;
}

lbm_status fail_cuda(lbm_ctx* ctx, const char* what, cudaError_t e) {
  return fail(ctx, LBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LBM_CK(ctx, call)                                        \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return fail_cuda((ctx), #call, e_);   \
  } while (0)

void* dev_alloc(lbm_ctx* c, size_t bytes) {
  if (c->have_alloc) return c->alloc.alloc(bytes, c->alloc.user);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  return p;
}

void dev_free(lbm_ctx* c, void* p) {
  if (!p) return;
  if (c->have_alloc)
    c->alloc.free(p, c->alloc.user);
  else
    cudaFree(p);
}

bool rate_ok(double s) { return s > 0.0 && s < 2.0 && std::isfinite(s); }

// Multiplier and shift of the multiply-shift division by d (see lbm::FastDiv).
lbm::FastDiv make_fast_div(unsigned d) {
  unsigned l = 0;
  while ((1ull << l) < d) ++l;
  const unsigned long long m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
  return lbm::FastDiv{d, static_cast<unsigned>(m), l};
}

// Float copies of the derived parameters (Eqs. 2, 14, 19, 33).
lbm::Physics make_physics(const lbm_params& p) {
  lbm::Physics ph{};
  ph.rho_g = static_cast<float>(p.rho_g);
  ph.half_drho = static_cast<float>(0.5 * (p.rho_l - p.rho_g));
  ph.nu_g = static_cast<float>(p.nu_g);
  ph.nu_mid = static_cast<float>(0.5 * (p.nu_l + p.nu_g));
  ph.half_dnu = static_cast<float>(0.5 * (p.nu_l - p.nu_g));
  ph.mob = static_cast<float>(p.mobility);
  ph.kappa = static_cast<float>(3.0 * p.D * p.sigma / 8.0);
  ph.beta = static_cast<float>(3.0 * p.sigma / (4.0 * p.D));
  ph.A = static_cast<float>(p.A);
  ph.eta = static_cast<float>(p.mobility / (p.A * (1.0 / p.sf[1] - 0.5)));
  for (int a = 0; a < 3; ++a) ph.gacc[a] = static_cast<float>(p.g[a]);
  ph.rho_ref = (p.flags & LBM_FLAG_BUOYANCY) ? static_cast<float>(0.5 * (p.rho_l + p.rho_g)) : 0.0f;
  for (int k = 0; k < 7; ++k) {
    ph.sf_a[k] = static_cast<float>(p.sf[k] / lbm::norm7(k));
    ph.sf_b[k] = static_cast<float>((1.0 - 0.5 * p.sf[k]) / lbm::norm7(k));
  }
  for (int k = 0; k < 15; ++k) {
    ph.sg_a[k] = static_cast<float>(p.sg[k] / lbm::norm15(k));
    ph.sg_b[k] = static_cast<float>((1.0 - 0.5 * p.sg[k]) / lbm::norm15(k));
  }
  ph.srt_flow = (p.flags & LBM_FLAG_SRT_FLOW) ? 1 : 0;
  ph.d3q7_stencil = (p.flags & LBM_FLAG_D3Q7_STENCIL) ? 1 : 0;
  return ph;
}

lbm_status validate(const lbm_grid* g, const lbm_params* p) {
  if (!g || !p) return fail(nullptr, LBM_EINVAL, "grid and params must not be NULL");
  if (g->nx < 1 || g->ny < 1 || g->nz < 1)
    return fail(nullptr, LBM_EINVAL, "grid sizes must be >= 1");
  const long long n = static_cast<long long>(g->nx) * g->ny * g->nz;
  if (n >= (1LL << 31) - 64) return fail(nullptr, LBM_EINVAL, "grid has 2^31 cells or more");
  if (g->walls_z != 0 && g->walls_z != 1) return fail(nullptr, LBM_EINVAL, "walls_z must be 0 or 1");
  if (!(p->rho_l > 0 && p->rho_g > 0)) return fail(nullptr, LBM_EINVAL, "densities must be > 0");
  if (!(p->nu_l > 0 && p->nu_g > 0)) return fail(nullptr, LBM_EINVAL, "viscosities must be > 0");
  if (!(p->mobility >= 0 && std::isfinite(p->mobility)))
    return fail(nullptr, LBM_EINVAL, "mobility must be >= 0");
  if (!(p->D > 0 && std::isfinite(p->sigma))) return fail(nullptr, LBM_EINVAL, "D must be > 0");
  if (!(p->A > 0 && p->A < 1.0 / 3.0)) return fail(nullptr, LBM_EINVAL, "A must lie in (0, 1/3)");
  for (int k = 0; k < 7; ++k)
    if (!rate_ok(p->sf[k])) return fail(nullptr, LBM_EINVAL, "sf rates must lie in (0, 2)");
  for (int k = 0; k < 15; ++k)
    if ((k < 9 || k > 13) && !rate_ok(p->sg[k]))
      return fail(nullptr, LBM_EINVAL, "sg rates must lie in (0, 2)");
  if (!(p->sf[1] == p->sf[2] && p->sf[2] == p->sf[3]))
    return fail(nullptr, LBM_EINVAL, "Eq. 19 needs s_1 = s_2 = s_3");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(p->g[a])) return fail(nullptr, LBM_EINVAL, "g must be finite");
  if (p->flags & ~(LBM_FLAG_BUOYANCY | LBM_FLAG_SRT_FLOW | LBM_FLAG_D3Q7_STENCIL))
    return fail(nullptr, LBM_EINVAL, "unknown flag");
  if (p->storage != LBM_STORAGE_FP32 && p->storage != LBM_STORAGE_FP16 &&
      p->storage != LBM_STORAGE_BF16)
    return fail(nullptr, LBM_EINVAL, "unknown storage type");
  if (p->pattern != LBM_PATTERN_AB && p->pattern != LBM_PATTERN_AA)
    return fail(nullptr, LBM_EINVAL, "unknown population pattern");
  return LBM_OK;
}

void drop_graphs(lbm_ctx* c) {
  for (auto& g : c->pair_graph) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

void release(lbm_ctx* c) {
  drop_graphs(c);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  c->capture_stream = nullptr;
  for (auto& list : c->events)
    for (auto& pr : list) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  dev_free(c, c->pop[0]);
  dev_free(c, c->pop[1]);
  dev_free(c, c->phi_buf[0]);
  dev_free(c, c->phi_buf[1]);
  dev_free(c, c->mu);
  dev_free(c, c->stage);
  dev_free(c, c->partial);
  dev_free(c, c->red);
  dev_free(c, c->step_parts);
  c->pop[0] = c->pop[1] = c->phi = c->phi_buf[0] = c->phi_buf[1] = c->mu = c->stage = nullptr;
  c->partial = c->red = nullptr;
  c->step_parts = nullptr;
}

// Device error word (1: a bounded wait on a TMA copy ran out), kept in red[7].
int* error_word(lbm_ctx* c) { return reinterpret_cast<int*>(c->red + 7); }

// Reports and clears the error word, given a host copy of red[0..7].  Word 1: a bounded
// wait for a TMA copy ran out, the copy then landed and the block returned; the steps
// since are invalid but the context is usable.  Word 2: the copy had not landed when
// its block returned, so it may have written into shared memory the block no longer
// owned; the context is retired (every later launching call fails).
lbm_status take_device_error(lbm_ctx* c, const double* h) {
  int word = 0;
  std::memcpy(&word, h + 7, sizeof(word));
  if (word == 0) return LBM_OK;
  cudaMemsetAsync(c->red + 7, 0, sizeof(double), c->stream);
  if (word >= 2) {
    c->retired = true;
    return fail(c, LBM_ECUDA,
                "a TMA copy in the chemical-potential pass had not landed when its block "
                "returned; the context is retired (destroy it)");
  }
  return fail(c, LBM_ETIMEOUT,
              "a bounded wait for a TMA copy in the chemical-potential pass ran out; the "
              "affected steps are not valid");
}

// Refuses launches on a context that is not initialised or has been retired.
lbm_status check_ready(lbm_ctx* c, bool need_init = true) {
  if (c->retired) return fail(c, LBM_ECUDA, "context retired after a TMA copy outlived its block");
  if (need_init && !c->initialized)
    return fail(c, LBM_EINVAL, "lbm_init_phi or lbm_write_state first");
  return LBM_OK;
}

// The chemical-potential pass can fetch its halo bricks by TMA when whole bricks tile
// x and y, the box fits the grid, and phi starts on a 16-byte boundary.
bool encode_phi_map(lbm_ctx* c, int which) {
  const lbm::Geometry& g = c->geo;
  float* phi = c->phi_buf[which];
  if (!lbm::mu_tma_shape_ok(g) || g.nx < static_cast<int>(lbm::kMuTmaBox[0]) ||
      g.ny < static_cast<int>(lbm::kMuTmaBox[1]) || g.nz < static_cast<int>(lbm::kMuTmaBox[2]) ||
      reinterpret_cast<uintptr_t>(phi) % 16 != 0)
    return false;
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!encode) return false;
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(g.nx), static_cast<cuuint64_t>(g.ny),
                              static_cast<cuuint64_t>(g.nz)};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(g.nx) * 4,
                                 static_cast<cuuint64_t>(g.nx) * g.ny * 4};
  const cuuint32_t box[3] = {lbm::kMuTmaBox[0], lbm::kMuTmaBox[1], lbm::kMuTmaBox[2]};
  const cuuint32_t elem[3] = {1, 1, 1};
  return encode(&c->phi_map[which], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, phi, dims, strides, box, elem,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// Per-warp partials of the fused step sums: 5 floats per 32 cells.
size_t step_parts_bytes(long long n) {
  return static_cast<size_t>(lbm::cell_warps(n)) * 5 * sizeof(float);
}

// Whether a context of this grid and these parameters keeps a second phi array (16-bit
// storage on grids the single-pass step takes).
bool wants_phi_alt(const lbm_grid& g, const lbm_params& p) {
  return p.storage != LBM_STORAGE_FP32 && p.pattern == LBM_PATTERN_AB && g.nx % lbm::kTile == 0 &&
         g.ny % 8 == 0 && g.ny / 8 <= 65535 && g.nz <= 65535 &&
         static_cast<long long>(g.ny) * (g.nx / lbm::kTile) * lbm::tile_bytes<lbm::kF32>() <
             (1LL << 31);
}

// Whether the next step goes through the single-pass kernel.
bool fused_applies(const lbm_ctx* c) {
  return c->use_fused && c->vel_kind == LBM_VELOCITY_NONE && c->params.pattern == LBM_PATTERN_AB &&
         !(c->params.flags & (LBM_FLAG_SRT_FLOW | LBM_FLAG_D3Q7_STENCIL)) &&
         lbm::fused_shape_ok(c->geo) && (c->geo.storage == lbm::kF32 || c->phi_buf[1]);
}

int fused_segment(const lbm_ctx* c) {
  if (c->fused_seg > 0) return c->fused_seg < c->geo.nz ? c->fused_seg : c->geo.nz;
  return lbm::fused_default_segment(c->geo, c->sms);
}

// Pattern of the next step's reads of the current state.
int read_pattern(const lbm_ctx* c) {
  if (c->params.pattern == LBM_PATTERN_AB) return lbm::kAB;
  return c->odd ? lbm::kAAOdd : lbm::kAAEven;
}

float* cur_state(lbm_ctx* c) { return c->pop[c->cur]; }

// Time factor of the prescribed velocity at step t: cos(pi t / T) for the deformation
// field (Eq. 41), 1 otherwise; evaluated in double on the host.
float velocity_time_factor(const lbm_ctx* c, long long t) {
  if (c->vel_kind != LBM_VELOCITY_DEFORMATION) return 1.0f;
  return static_cast<float>(std::cos(3.14159265358979323846 * static_cast<double>(t) / c->vel_period));
}

template <typename F>
cudaError_t timed(lbm_ctx* c, int kernel, F&& launch) {
  if (!c->profiling) return launch();
  cudaEvent_t a, b;
  cudaError_t e = cudaEventCreate(&a);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&b);
  if (e != cudaSuccess) return e;
  cudaEventRecord(a, c->stream);
  e = launch();
  cudaEventRecord(b, c->stream);
  c->events[kernel].emplace_back(a, b);
  return e;
}

// The device address of a caller's host buffer when it is page-locked (cudaHostAlloc,
// cudaHostRegister, PyTorch's pinned tensors): kernels then read or store it directly
// over the host link; nullptr for pageable memory.
template <typename T>
T* device_view(T* host) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();  // a pointer CUDA does not know: clear the error it reported
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? static_cast<T*>(a.devicePointer) : nullptr;
}

// Widen an FP32 device plane to double into the caller's host buffer, asynchronous on
// the context's stream: straight into it when it is page-locked (the widening kernel
// stores over the host link), else on the device into wide (n doubles) and a copy.
// (Measured on a GB300 with its Grace host: copy-engine copies to host memory slow
// down with the number of kernel launches before them -- 12 to 45 ms for 537 MB after
// 1000 to 9000 steps, 2.8 ms when repeated -- while a kernel's stores into the same
// page-locked memory keep their ~190 GB/s.)
lbm_status plane_to_host(lbm_ctx* c, const float* dev, double* host, double* wide) {
  const size_t n = static_cast<size_t>(c->geo.n);
  if (double* view = device_view(host)) {
    LBM_CK(c, lbm::launch_widen(dev, view, c->geo.n, c->stream));
    return LBM_OK;
  }
  if (!wide) return fail(c, LBM_EINVAL, "read-out buffer changed from page-locked to pageable");
  LBM_CK(c, lbm::launch_widen(dev, wide, c->geo.n, c->stream));
  LBM_CK(c, cudaMemcpyAsync(host, wide, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return LBM_OK;
}

}  // namespace

void lbm::set_global_error(const std::string& msg) { g_create_error = msg; }

int lbm::ctx_storage(const lbm_ctx* c) { return c->geo.storage; }

bool lbm::ctx_batchable(const lbm_ctx* c, std::string* why) {
  const char* r = nullptr;
  if (!c->initialized)
    r = "not initialised";
  else if (c->retired)
    r = "retired after a TMA copy outlived its block";
  else if (c->params.pattern != LBM_PATTERN_AB)
    r = "batches need LBM_PATTERN_AB";
  else if (c->vel_kind != LBM_VELOCITY_NONE)
    r = "batches run the coupled model only";
  else if (c->params.flags & (LBM_FLAG_SRT_FLOW | LBM_FLAG_D3Q7_STENCIL))
    r = "batches run the default model variant only";
  if (r && why) *why = r;
  return r == nullptr;
}

bool lbm::ctx_have_prev(const lbm_ctx* c) { return c->have_prev; }

cudaStream_t lbm::ctx_stream(const lbm_ctx* c) { return c->stream; }

void lbm::ctx_describe(const lbm_ctx* c, lbm::Geometry* geo, lbm::Physics* ph, float** state0,
                       float** state1, float** phi, float** mu, int* parity) {
  *geo = c->geo;
  *ph = c->ph;
  *state0 = c->pop[0];
  *state1 = c->pop[1];
  *phi = c->phi;
  *mu = c->mu;
  *parity = c->cur;
}

void lbm::ctx_advance(lbm_ctx* c, int n) {
  c->cur = (c->cur + n) & 1;
  c->step += n;
  c->have_prev = true;
}

namespace {

// One time step; with sums_out the stream-collide pass also reduces the new state into
// sums_out (5 doubles on the device; coupled default variant only).
lbm_status step_once(lbm_ctx* c, double* sums_out) {
  const int pat = read_pattern(c);
  const float* src = cur_state(c);
  float* dst = c->params.pattern == LBM_PATTERN_AB ? c->pop[1 - c->cur] : c->pop[c->cur];
  if (fused_applies(c)) {
    float* phi_out = c->geo.storage != lbm::kF32 ? c->phi_buf[1 - c->phi_sel] : nullptr;
    LBM_CK(c, timed(c, 2, [&] {
             return lbm::launch_fused(src, dst, c->phi, phi_out, c->geo, c->ph, c->have_prev,
                                      fused_segment(c), c->fused_pf,
                                      sums_out ? c->step_parts : nullptr, c->partial, sums_out,
                                      c->stream);
           }));
    if (phi_out) {
      c->phi_sel = 1 - c->phi_sel;
      c->phi = c->phi_buf[c->phi_sel];
    }
    c->cur = 1 - c->cur;
    c->have_prev = true;
    ++c->step;
    return LBM_OK;
  }
  LBM_CK(c, timed(c, 0, [&] { return lbm::launch_phi(src, c->phi, c->phi, c->geo, pat, c->stream); }));
  LBM_CK(c, timed(c, 1, [&] {
           return c->have_phi_map && c->use_phi_map
                      ? lbm::launch_mu_tma(c->phi_map[c->phi_sel], c->phi, c->mu, c->geo, c->ph,
                                           error_word(c),
                                           c->tma_polls < 0 ? lbm::mu_tma_default_polls()
                                                            : c->tma_polls,
                                           c->stream)
                      : lbm::launch_mu(c->phi, c->mu, c->geo, c->ph, c->stream);
         }));
  const bool prev = c->have_prev;
  if (c->vel_kind == LBM_VELOCITY_NONE) {
    lbm::Geometry gs = c->geo;  // the summing kernel has its own best prefetch distance
    gs.prefetch_collide = c->prefetch_sums;
    LBM_CK(c, timed(c, 2, [&] {
             return sums_out ? lbm::launch_collide_sums(src, dst, c->phi, c->mu, gs, c->ph,
                                                         pat, prev, c->step_parts, c->partial,
                                                         sums_out, c->stream, error_word(c),
                                                         c->tma_polls < 0
                                                             ? lbm::mu_tma_default_polls()
                                                             : c->tma_polls)
                             : lbm::launch_collide(src, dst, c->phi, c->mu, c->geo, c->ph, pat,
                                                   prev, c->stream, error_word(c),
                                                   c->tma_polls < 0 ? lbm::mu_tma_default_polls()
                                                                    : c->tma_polls);
           }));
  } else {
    const float tf = velocity_time_factor(c, c->step);
    LBM_CK(c, timed(c, 2, [&] {
             return lbm::launch_che(src, dst, c->phi, c->mu, c->geo, c->ph, pat, prev, tf,
                                    c->stream);
           }));
  }
  if (c->params.pattern == LBM_PATTERN_AB)
    c->cur = 1 - c->cur;
  else
    c->odd = !c->odd;
  c->have_prev = true;
  ++c->step;
  return LBM_OK;
}

// Steps of the coupled model with a previous step and no per-kernel timing have fixed
// kernel arguments, so two of them can be captured once and replayed.
bool graphs_apply(const lbm_ctx* c) {
  return c->use_graphs && c->vel_kind == LBM_VELOCITY_NONE && !c->profiling && c->have_prev;
}

int pair_parity(const lbm_ctx* c) {
  return (c->params.pattern == LBM_PATTERN_AB ? c->cur : (c->odd ? 1 : 0)) | (c->phi_sel << 1);
}

// Captures two steps from the current parity into c->pair_graph[parity]; the context's
// bookkeeping (array parity, step count) is left as it was.
lbm_status capture_pair(lbm_ctx* c, int parity) {
  if (!c->capture_stream &&
      cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(c, LBM_ECUDA, "cudaStreamCreate failed (graph capture)");
  const int cur = c->cur, phi_sel = c->phi_sel;
  const bool odd = c->odd, have_prev = c->have_prev;
  const long long step = c->step;
  cudaStream_t stream = c->stream;
  c->stream = c->capture_stream;
  cudaError_t e = cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal);
  lbm_status st = LBM_OK;
  if (e == cudaSuccess) {
    st = step_once(c, nullptr);
    if (st == LBM_OK) st = step_once(c, nullptr);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = e == cudaSuccess ? cudaStreamEndCapture(c->capture_stream, &graph) : e;
  c->stream = stream;
  c->cur = cur;
  c->phi_sel = phi_sel;
  c->phi = c->phi_buf[phi_sel];
  c->odd = odd;
  c->have_prev = have_prev;
  c->step = step;
  if (st != LBM_OK || ec != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return st != LBM_OK ? st : fail_cuda(c, "graph capture", ec);
  }
  e = cudaGraphInstantiate(&c->pair_graph[parity], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    c->pair_graph[parity] = nullptr;
    return fail_cuda(c, "cudaGraphInstantiate", e);
  }
  return LBM_OK;
}

// Whether the last step of lbm_step_reduce can carry the sums (else a separate pass).
bool fused_sums(const lbm_ctx* c) {
  return c->vel_kind == LBM_VELOCITY_NONE &&
         !(c->params.flags & (LBM_FLAG_SRT_FLOW | LBM_FLAG_D3Q7_STENCIL));
}

}  // namespace

extern "C" {

lbm_status lbm_create(const lbm_grid* grid, const lbm_params* params, const lbm_allocator* alloc,
                      void* cuda_stream, lbm_ctx** out) {
  if (!out) return fail(nullptr, LBM_EINVAL, "out must not be NULL");
  *out = nullptr;
  lbm_status st = validate(grid, params);
  if (st != LBM_OK) return st;
  if (alloc && (!alloc->alloc || !alloc->free))
    return fail(nullptr, LBM_EINVAL, "allocator needs both alloc and free");

  lbm_ctx* c = new lbm_ctx();
  c->grid = *grid;
  c->params = *params;
  if (alloc) {
    c->alloc = *alloc;
    c->have_alloc = true;
  }
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  const long long n = static_cast<long long>(grid->nx) * grid->ny * grid->nz;
  c->geo.nx = grid->nx;
  c->geo.ny = grid->ny;
  c->geo.nz = grid->nz;
  c->geo.walls = grid->walls_z;
  c->geo.n = static_cast<int>(n);
  c->geo.plane = grid->nx * grid->ny;
  c->geo.stride = static_cast<size_t>((n + 63) / 64 * 64);  // 256-byte aligned planes
  c->geo.storage = params->storage;  // LBM_STORAGE_* numbers match lbm::Storage
  c->geo.div_nx = make_fast_div(static_cast<unsigned>(grid->nx));
  c->geo.div_ny = make_fast_div(static_cast<unsigned>(grid->ny));
  // whole-tile rows whose planes of tiles span < 2^31 bytes in the widest storage
  if (grid->nx % lbm::kTile == 0 &&
      static_cast<long long>(grid->ny) * (grid->nx / lbm::kTile) * lbm::tile_bytes<lbm::kF32>() <
          (1LL << 31))
    c->row_tiles = grid->nx / lbm::kTile;
  c->geo.row_tiles = c->row_tiles;
  // two cells per thread in the stream-collide (either pattern): cells x and x + 32 of a row
  if (grid->nx % (2 * lbm::kTile) == 0) c->pairs = 1;
  c->geo.pairs = c->pairs;
  if (c->pairs && lbm::stage_shape_ok(c->geo)) c->stage_rows = 1;
  // on by default with FP32 populations only: with 16-bit ones the pass is faster
  // loading its stencils per cell (the block waits for all its rows before computing)
  c->geo.stage = params->storage == LBM_STORAGE_FP32 ? c->stage_rows : 0;
  // L2 prefetch distances: one wave of resident blocks
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) {
      c->geo.prefetch_collide =
          sms * lbm::resident_blocks_per_sm(c->geo.pairs ? 3 : 0, c->geo.storage);
      c->prefetch_sums = c->geo.prefetch_collide;
      c->geo.prefetch_phi =
          sms * lbm::resident_blocks_per_sm(1, c->geo.storage, c->geo.row_tiles > 0);
    }
  }
  c->ph = make_physics(*params);
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      c->sms = 0;
  }

  const size_t plane = c->geo.stride * sizeof(float);
  const size_t state_bytes = lbm::state_bytes(c->geo.n, c->geo.storage);
  c->pop[0] = static_cast<float*>(dev_alloc(c, state_bytes));
  if (params->pattern == LBM_PATTERN_AB) c->pop[1] = static_cast<float*>(dev_alloc(c, state_bytes));
  c->phi = c->phi_buf[0] = static_cast<float*>(dev_alloc(c, plane));
  const bool need_alt = wants_phi_alt(*grid, *params);
  if (need_alt) c->phi_buf[1] = static_cast<float*>(dev_alloc(c, plane));
  c->mu = static_cast<float*>(dev_alloc(c, plane));
  c->stage = static_cast<float*>(dev_alloc(c, plane * 7));
  c->partial = static_cast<double*>(dev_alloc(c, sizeof(double) * 5 * lbm::kReduceMaxParts));
  c->red = static_cast<double*>(dev_alloc(c, sizeof(double) * 8));
  c->step_parts = static_cast<float*>(dev_alloc(c, step_parts_bytes(c->geo.n)));
  if (!c->pop[0] || (params->pattern == LBM_PATTERN_AB && !c->pop[1]) || !c->phi ||
      (need_alt && !c->phi_buf[1]) || !c->mu ||
      !c->stage || !c->partial || !c->red || !c->step_parts) {
    release(c);
    delete c;
    return fail(nullptr, LBM_ENOMEM, "device allocation failed");
  }
  cudaError_t e = cudaMemsetAsync(c->pop[0], 0, state_bytes, c->stream);
  if (e == cudaSuccess && c->pop[1]) e = cudaMemsetAsync(c->pop[1], 0, state_bytes, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->red, 0, sizeof(double) * 8, c->stream);
  c->have_phi_map = encode_phi_map(c, 0) && (!c->phi_buf[1] || encode_phi_map(c, 1));
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    release(c);
    delete c;
    return fail(nullptr, LBM_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  }
  *out = c;
  return LBM_OK;
}

lbm_status lbm_init_phi(lbm_ctx* c, const double* phi, const double* u, const double* p) {
  if (!c) return LBM_EINVAL;
  if (const lbm_status rs = check_ready(c, false); rs != LBM_OK) return rs;
  if (!phi) return fail(c, LBM_EINVAL, "phi must not be NULL");
  const size_t n = static_cast<size_t>(c->geo.n);
  const size_t s = c->geo.stride;
  // page-locked inputs are read by the narrowing kernel itself over the host link;
  // pageable ones are copied to a device buffer first
  const bool pageable = !device_view(phi) ||
                        (u && (!device_view(u) || !device_view(u + n) || !device_view(u + 2 * n))) ||
                        (p && !device_view(p));
  double* tmp = nullptr;
  if (pageable) {
    tmp = static_cast<double*>(dev_alloc(c, n * sizeof(double)));
    if (!tmp) return fail(c, LBM_ENOMEM, "device allocation failed (init staging)");
  }
  auto upload = [&](const double* host, float* dst) -> cudaError_t {
    if (const double* view = device_view(host)) return lbm::launch_convert(view, dst, c->geo.n, c->stream);
    cudaError_t e = cudaMemcpyAsync(tmp, host, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return e;
    return lbm::launch_convert(tmp, dst, c->geo.n, c->stream);
  };
  cudaError_t e = upload(phi, c->phi);
  if (e == cudaSuccess && u)
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) e = upload(u + a * n, c->stage + a * s);
  if (e == cudaSuccess && p) e = upload(p, c->stage + 3 * s);
  if (e == cudaSuccess) e = lbm::launch_mu(c->phi, c->mu, c->geo, c->ph, c->stream);
  c->cur = 0;
  c->odd = false;
  if (e == cudaSuccess)
    e = lbm::launch_init(cur_state(c), c->phi, c->mu, u ? c->stage : nullptr,
                         p ? c->stage + 3 * s : nullptr, c->geo, c->ph, read_pattern(c),
                         velocity_time_factor(c, 0), c->stream);
  const cudaError_t es = cudaStreamSynchronize(c->stream);
  if (tmp) dev_free(c, tmp);
  if (e != cudaSuccess) return fail_cuda(c, "lbm_init_phi", e);
  if (es != cudaSuccess) return fail_cuda(c, "lbm_init_phi", es);
  c->step = 0;
  c->have_prev = false;
  c->initialized = true;
  return LBM_OK;
}


lbm_status lbm_step(lbm_ctx* c, int n) {
  if (!c) return LBM_EINVAL;
  if (n < 0) return fail(c, LBM_EINVAL, "n must be >= 0");
  if (const lbm_status rs = check_ready(c); rs != LBM_OK) return rs;
  int it = 0;
  if (n >= 2 && c->use_graphs && c->vel_kind == LBM_VELOCITY_NONE && !c->profiling &&
      !c->have_prev) {
    // the first step after initialisation (d_t(phi u) = 0) is never replayed
    const lbm_status st = step_once(c, nullptr);
    if (st != LBM_OK) return st;
    ++it;
  }
  while (n - it >= 2 && graphs_apply(c)) {
    const int parity = pair_parity(c);
    if (!c->pair_graph[parity]) {
      const lbm_status st = capture_pair(c, parity);
      if (st != LBM_OK) return st;
    }
    LBM_CK(c, cudaGraphLaunch(c->pair_graph[parity], c->stream));
    c->step += 2;  // two steps leave the array parity as it was
    it += 2;
  }
  for (; it < n; ++it) {
    const lbm_status st = step_once(c, nullptr);
    if (st != LBM_OK) return st;
  }
  return LBM_OK;
}

lbm_status lbm_step_reduce_async(lbm_ctx* c, int n, double* out_dev) {
  if (!c) return LBM_EINVAL;
  if (n < 1) return fail(c, LBM_EINVAL, "n must be >= 1");
  if (!out_dev || reinterpret_cast<uintptr_t>(out_dev) % alignof(double) != 0)
    return fail(c, LBM_EINVAL, "out_dev must be a non-NULL, 8-byte aligned pointer");
  if (const lbm_status rs = check_ready(c); rs != LBM_OK) return rs;
  if (!fused_sums(c)) {
    const lbm_status st = lbm_step(c, n);
    return st != LBM_OK ? st : lbm_reduce_async(c, out_dev);
  }
  const lbm_status st = lbm_step(c, n - 1);
  return st != LBM_OK ? st : step_once(c, out_dev);
}

lbm_status lbm_step_reduce(lbm_ctx* c, int n, double* sum_phi, double mom[3]) {
  if (!c) return LBM_EINVAL;
  if (!sum_phi || !mom) return fail(c, LBM_EINVAL, "outputs must not be NULL");
  const lbm_status st = lbm_step_reduce_async(c, n, c->red);
  if (st != LBM_OK) return st;
  double h[8];
  LBM_CK(c, cudaMemcpyAsync(h, c->red, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  if (const lbm_status te = take_device_error(c, h); te != LBM_OK) return te;
  *sum_phi = h[0];
  mom[0] = h[1];
  mom[1] = h[2];
  mom[2] = h[3];
  if (h[4] > 0) return fail(c, LBM_EUNSTABLE, "non-finite phi or momentum in " +
                                                  std::to_string(static_cast<long long>(h[4])) + " cells");
  return LBM_OK;
}

lbm_status lbm_read_fields(lbm_ctx* c, unsigned mask, double* phi, double* rho, double* p,
                           double* u, double* mu) {
  if (!c) return LBM_EINVAL;
  if (const lbm_status rs = check_ready(c); rs != LBM_OK) return rs;
  if (((mask & LBM_FIELD_PHI) && !phi) || ((mask & LBM_FIELD_RHO) && !rho) ||
      ((mask & LBM_FIELD_P) && !p) || ((mask & LBM_FIELD_U) && !u) || ((mask & LBM_FIELD_MU) && !mu))
    return fail(c, LBM_EINVAL, "a selected field has a NULL buffer");
  // phi and mu of the current state into staging planes 5 and 6: the solver's own phi
  // array is the reference of the 16-bit slot 0 and must keep the previous step's phi.
  const size_t n = static_cast<size_t>(c->geo.n);
  const size_t s = c->geo.stride;
  float* phi_now = c->stage + 5 * s;
  float* mu_now = c->stage + 6 * s;
  LBM_CK(c, lbm::launch_phi(cur_state(c), c->phi, phi_now, c->geo, read_pattern(c), c->stream));
  LBM_CK(c, lbm::launch_mu(phi_now, mu_now, c->geo, c->ph, c->stream));
  if (mask & (LBM_FIELD_RHO | LBM_FIELD_P | LBM_FIELD_U))
    LBM_CK(c, lbm::launch_fields(cur_state(c), phi_now, mu_now, c->stage, c->geo, c->ph,
                                 read_pattern(c), velocity_time_factor(c, c->step), c->stream));
  const bool pageable = ((mask & LBM_FIELD_PHI) && !device_view(phi)) ||
                        ((mask & LBM_FIELD_MU) && !device_view(mu)) ||
                        ((mask & LBM_FIELD_RHO) && !device_view(rho)) ||
                        ((mask & LBM_FIELD_P) && !device_view(p)) ||
                        ((mask & LBM_FIELD_U) &&
                         (!device_view(u) || !device_view(u + n) || !device_view(u + 2 * n)));
  double* wide = nullptr;
  if (pageable) {
    wide = static_cast<double*>(dev_alloc(c, n * sizeof(double)));
    if (!wide) return fail(c, LBM_ENOMEM, "device allocation failed (read-out staging)");
  }
  lbm_status st = LBM_OK;
  if (mask & LBM_FIELD_PHI) st = plane_to_host(c, phi_now, phi, wide);
  if (st == LBM_OK && (mask & LBM_FIELD_MU)) st = plane_to_host(c, mu_now, mu, wide);
  if (st == LBM_OK && (mask & LBM_FIELD_RHO)) st = plane_to_host(c, c->stage, rho, wide);
  if (st == LBM_OK && (mask & LBM_FIELD_P)) st = plane_to_host(c, c->stage + s, p, wide);
  for (int a = 0; a < 3 && st == LBM_OK && (mask & LBM_FIELD_U); ++a)
    st = plane_to_host(c, c->stage + (2 + a) * s, u + a * n, wide);
  double h[8];
  if (st == LBM_OK)
    LBM_CK(c, cudaMemcpyAsync(h, c->red, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  const cudaError_t es = cudaStreamSynchronize(c->stream);
  if (wide) dev_free(c, wide);
  if (st != LBM_OK) return st;
  if (es != cudaSuccess) return fail_cuda(c, "lbm_read_fields", es);
  return take_device_error(c, h);
}

lbm_status lbm_reduce(lbm_ctx* c, double* sum_phi, double mom[3]) {
  if (!c) return LBM_EINVAL;
  if (!sum_phi || !mom) return fail(c, LBM_EINVAL, "outputs must not be NULL");
  if (const lbm_status rs = check_ready(c); rs != LBM_OK) return rs;
  float* phi_now = c->stage + 5 * c->geo.stride;
  LBM_CK(c, lbm::launch_phi(cur_state(c), c->phi, phi_now, c->geo, read_pattern(c), c->stream));
  LBM_CK(c, lbm::launch_reduce(cur_state(c), phi_now, c->partial, c->red, c->geo, read_pattern(c),
                               c->vel_kind == LBM_VELOCITY_NONE, c->stream));
  double h[8];
  LBM_CK(c, cudaMemcpyAsync(h, c->red, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  if (const lbm_status te = take_device_error(c, h); te != LBM_OK) return te;
  *sum_phi = h[0];
  mom[0] = h[1];
  mom[1] = h[2];
  mom[2] = h[3];
  if (h[4] > 0) return fail(c, LBM_EUNSTABLE, "non-finite phi or momentum in " +
                                                  std::to_string(static_cast<long long>(h[4])) + " cells");
  return LBM_OK;
}

lbm_status lbm_reduce_async(lbm_ctx* c, double* out_dev) {
  if (!c) return LBM_EINVAL;
  if (!out_dev || reinterpret_cast<uintptr_t>(out_dev) % alignof(double) != 0)
    return fail(c, LBM_EINVAL, "out_dev must be a non-NULL, 8-byte aligned pointer");
  if (const lbm_status rs = check_ready(c); rs != LBM_OK) return rs;
  float* phi_now = c->stage + 5 * c->geo.stride;
  LBM_CK(c, lbm::launch_phi(cur_state(c), c->phi, phi_now, c->geo, read_pattern(c), c->stream));
  LBM_CK(c, lbm::launch_reduce(cur_state(c), phi_now, c->partial, out_dev, c->geo,
                               read_pattern(c), c->vel_kind == LBM_VELOCITY_NONE, c->stream));
  return LBM_OK;
}

lbm_status lbm_read_state(lbm_ctx* c, float* f, float* g, float* phiu_prev, long long* step) {
  if (!c) return LBM_EINVAL;
  if (const lbm_status rs = check_ready(c); rs != LBM_OK) return rs;
  const size_t n = static_cast<size_t>(c->geo.n);
  for (int q = 0; q < lbm::kTileSlots; ++q) {
    float* dst = nullptr;
    if (q < 7)
      dst = f ? f + q * n : nullptr;
    else if (q < lbm::kSlots)
      dst = g ? g + (q - 7) * n : nullptr;
    else
      dst = (phiu_prev && c->have_prev) ? phiu_prev + (q - lbm::kSlotPhiu) * n : nullptr;
    if (!dst) continue;
    if (float* view = device_view(dst)) {  // page-locked: the gather stores into it
      LBM_CK(c, lbm::launch_gather(cur_state(c), c->phi, view, c->geo, read_pattern(c), q,
                                   c->stream));
      continue;
    }
    LBM_CK(c, lbm::launch_gather(cur_state(c), c->phi, c->stage, c->geo, read_pattern(c), q,
                                 c->stream));
    LBM_CK(c, cudaMemcpyAsync(dst, c->stage, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  }
  if (phiu_prev && !c->have_prev) std::memset(phiu_prev, 0, 3 * n * sizeof(float));
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  if (step) *step = c->step;
  return LBM_OK;
}

lbm_status lbm_read_state_at(lbm_ctx* c, const long long* cells, long long count, float* f,
                             float* g, float* phiu_prev, long long* step) {
  if (!c) return LBM_EINVAL;
  if (const lbm_status rs = check_ready(c); rs != LBM_OK) return rs;
  if (count < 0) return fail(c, LBM_EINVAL, "count must be >= 0");
  if (count > 0 && !cells) return fail(c, LBM_EINVAL, "cells must not be NULL");
  for (long long k = 0; k < count; ++k)
    if (cells[k] < 0 || cells[k] >= c->geo.n)
      return fail(c, LBM_EINVAL, "cell index " + std::to_string(cells[k]) + " outside the grid");
  if (count > 0 && (f || g || (phiu_prev && c->have_prev))) {
    const size_t idx_bytes = static_cast<size_t>(count) * sizeof(long long);
    const size_t out_floats = static_cast<size_t>(count) * lbm::kTileSlots;
    char* buf = static_cast<char*>(dev_alloc(c, idx_bytes + out_floats * sizeof(float)));
    if (!buf) return fail(c, LBM_ENOMEM, "device allocation failed (cell gather)");
    long long* d_cells = reinterpret_cast<long long*>(buf);
    float* d_out = reinterpret_cast<float*>(buf + idx_bytes);
    const size_t cnt = static_cast<size_t>(count);
    cudaError_t e = cudaMemcpyAsync(d_cells, cells, idx_bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
      e = lbm::launch_gather_at(cur_state(c), c->phi, d_cells, count, d_out, c->geo,
                                read_pattern(c), c->stream);
    if (e == cudaSuccess && f)
      e = cudaMemcpyAsync(f, d_out, 7 * cnt * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && g)
      e = cudaMemcpyAsync(g, d_out + 7 * cnt, 15 * cnt * sizeof(float), cudaMemcpyDeviceToHost,
                          c->stream);
    if (e == cudaSuccess && phiu_prev && c->have_prev)
      e = cudaMemcpyAsync(phiu_prev, d_out + lbm::kSlotPhiu * cnt, 3 * cnt * sizeof(float),
                          cudaMemcpyDeviceToHost, c->stream);
    const cudaError_t es = cudaStreamSynchronize(c->stream);
    dev_free(c, buf);
    if (e != cudaSuccess) return fail_cuda(c, "lbm_read_state_at", e);
    if (es != cudaSuccess) return fail_cuda(c, "lbm_read_state_at", es);
  }
  if (phiu_prev && !c->have_prev && count > 0)
    std::memset(phiu_prev, 0, 3 * static_cast<size_t>(count) * sizeof(float));
  if (step) *step = c->step;
  return LBM_OK;
}

lbm_status lbm_write_state(lbm_ctx* c, const float* f, const float* g, const float* phiu_prev,
                           long long step) {
  if (!c) return LBM_EINVAL;
  if (const lbm_status rs = check_ready(c, false); rs != LBM_OK) return rs;
  if (!f || !g) return fail(c, LBM_EINVAL, "f and g must not be NULL");
  if (step < 0) return fail(c, LBM_EINVAL, "step must be >= 0");
  const size_t n = static_cast<size_t>(c->geo.n);
  const bool prev = phiu_prev && step > 0;
  c->cur = 0;
  c->odd = false;
  for (int q = 0; q < lbm::kTileSlots; ++q) {
    const float* src = nullptr;
    if (q < 7)
      src = f + q * n;
    else if (q < lbm::kSlots)
      src = g + (q - 7) * n;
    else if (prev)
      src = phiu_prev + (q - lbm::kSlotPhiu) * n;
    if (!src) continue;
    if (q == 0 && c->geo.storage != LBM_STORAGE_FP32) {
      // 16-bit storage: f_0 becomes the reference phi, slot 0 holds f_0 - phi = 0
      LBM_CK(c, cudaMemcpyAsync(c->phi, src, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
      LBM_CK(c, cudaMemsetAsync(c->stage, 0, n * sizeof(float), c->stream));
    } else {
      LBM_CK(c, cudaMemcpyAsync(c->stage, src, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    }
    LBM_CK(c, lbm::launch_scatter(cur_state(c), c->stage, c->geo, read_pattern(c), q, c->stream));
  }
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  c->have_prev = prev;
  c->step = step;
  c->initialized = true;
  return LBM_OK;
}

lbm_status lbm_set_velocity(lbm_ctx* c, int kind, double U, double period) {
  if (!c) return LBM_EINVAL;
  if (kind < LBM_VELOCITY_NONE || kind > LBM_VELOCITY_DEFORMATION)
    return fail(c, LBM_EINVAL, "unknown velocity kind");
  if (!std::isfinite(U)) return fail(c, LBM_EINVAL, "U must be finite");
  if (kind == LBM_VELOCITY_DEFORMATION && !(period > 0 && std::isfinite(period)))
    return fail(c, LBM_EINVAL, "the deformation field needs a period > 0");
  cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  c->vel_kind = kind;
  c->vel_U = U;
  c->vel_period = kind == LBM_VELOCITY_DEFORMATION ? period : 1.0;
  c->ph.vel_kind = kind;
  c->ph.vel_U = static_cast<float>(U);
  return LBM_OK;
}

lbm_status lbm_set_tuning(lbm_ctx* c, int param, int value) {
  if (!c) return LBM_EINVAL;
  if (value < 0) return fail(c, LBM_EINVAL, "tuning values must be >= 0");
  switch (param) {
    case LBM_TUNE_PREFETCH_COLLIDE: c->geo.prefetch_collide = value; break;
    case LBM_TUNE_PREFETCH_PHI: c->geo.prefetch_phi = value; break;
    case LBM_TUNE_PREFETCH_COLLIDE_SUMS: c->prefetch_sums = value; break;
    case LBM_TUNE_MU_TMA:
      if (value > 1) return fail(c, LBM_EINVAL, "LBM_TUNE_MU_TMA takes 0 or 1");
      c->use_phi_map = value == 1;
      break;
    case LBM_TUNE_GRAPHS:
      if (value > 1) return fail(c, LBM_EINVAL, "LBM_TUNE_GRAPHS takes 0 or 1");
      c->use_graphs = value == 1;
      break;
    case LBM_TUNE_TMA_WAIT_POLLS: c->tma_polls = value; break;
    case LBM_TUNE_ROWS:
      if (value > 1) return fail(c, LBM_EINVAL, "LBM_TUNE_ROWS takes 0 or 1");
      c->geo.row_tiles = value == 1 ? c->row_tiles : 0;
      break;
    case LBM_TUNE_CELL_PAIRS:
      if (value > 1) return fail(c, LBM_EINVAL, "LBM_TUNE_CELL_PAIRS takes 0 or 1");
      c->geo.pairs = value == 1 ? c->pairs : 0;
      break;
    case LBM_TUNE_STENCIL_STAGE:
      if (value > 1) return fail(c, LBM_EINVAL, "LBM_TUNE_STENCIL_STAGE takes 0 or 1");
      c->geo.stage = value == 1 ? c->stage_rows : 0;
      break;
    case LBM_TUNE_FUSED:
      if (value > 1) return fail(c, LBM_EINVAL, "LBM_TUNE_FUSED takes 0 or 1");
      c->use_fused = value == 1;
      break;
    case LBM_TUNE_FUSED_SEGMENT:
      if (value > (1 << 20)) return fail(c, LBM_EINVAL, "LBM_TUNE_FUSED_SEGMENT out of range");
      c->fused_seg = value;
      break;
    case LBM_TUNE_FUSED_PREFETCH:
      if (value > 64) return fail(c, LBM_EINVAL, "LBM_TUNE_FUSED_PREFETCH takes 0..64");
      c->fused_pf = value;
      break;
    default: return fail(c, LBM_EINVAL, "unknown tuning parameter");
  }
  cudaStreamSynchronize(c->stream);  // a replay may still be running
  drop_graphs(c);                    // their kernel arguments may have changed
  return LBM_OK;
}

lbm_status lbm_get_tuning(const lbm_ctx* c, int param, int* value) {
  if (!c || !value) return LBM_EINVAL;
  switch (param) {
    case LBM_TUNE_PREFETCH_COLLIDE: *value = c->geo.prefetch_collide; return LBM_OK;
    case LBM_TUNE_PREFETCH_PHI: *value = c->geo.prefetch_phi; return LBM_OK;
    case LBM_TUNE_PREFETCH_COLLIDE_SUMS: *value = c->prefetch_sums; return LBM_OK;
    case LBM_TUNE_MU_TMA: *value = (c->have_phi_map && c->use_phi_map) ? 1 : 0; return LBM_OK;
    case LBM_TUNE_GRAPHS: *value = c->use_graphs ? 1 : 0; return LBM_OK;
    case LBM_TUNE_TMA_WAIT_POLLS:
      *value = static_cast<int>(c->tma_polls < 0 ? lbm::mu_tma_default_polls() : c->tma_polls);
      return LBM_OK;
    case LBM_TUNE_ROWS:
      *value = c->geo.row_tiles > 0 ? 1 : 0;
      return LBM_OK;
    case LBM_TUNE_CELL_PAIRS: *value = c->geo.pairs; return LBM_OK;
    case LBM_TUNE_STENCIL_STAGE: *value = (c->geo.pairs && c->geo.stage) ? 1 : 0; return LBM_OK;
    case LBM_TUNE_FUSED: *value = fused_applies(c) ? 1 : 0; return LBM_OK;
    case LBM_TUNE_FUSED_SEGMENT: *value = fused_segment(c); return LBM_OK;
    case LBM_TUNE_FUSED_PREFETCH: *value = c->fused_pf; return LBM_OK;
    default: return LBM_EINVAL;
  }
}

lbm_status lbm_get_step(const lbm_ctx* c, long long* step) {
  if (!c || !step) return LBM_EINVAL;
  *step = c->step;
  return LBM_OK;
}

lbm_status lbm_profile(lbm_ctx* c, int enable) {
  if (!c) return LBM_EINVAL;
  for (auto& list : c->events) {
    for (auto& pr : list) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    list.clear();
  }
  c->profiling = enable != 0;
  return LBM_OK;
}

lbm_status lbm_profile_read(lbm_ctx* c, int kernel, double* total_ms, long long* launches) {
  if (!c) return LBM_EINVAL;
  if (kernel < 0 || kernel > 2 || !total_ms || !launches)
    return fail(c, LBM_EINVAL, "kernel must be 0, 1 or 2 and outputs non-NULL");
  LBM_CK(c, cudaStreamSynchronize(c->stream));
  double total = 0.0;
  for (auto& pr : c->events[kernel]) {
    float ms = 0.0f;
    LBM_CK(c, cudaEventElapsedTime(&ms, pr.first, pr.second));
    total += ms;
  }
  *total_ms = total;
  *launches = static_cast<long long>(c->events[kernel].size());
  return LBM_OK;
}

lbm_status lbm_memory_bytes(const lbm_grid* grid, const lbm_params* params, size_t* bytes) {
  if (!bytes) return fail(nullptr, LBM_EINVAL, "bytes must not be NULL");
  const lbm_status st = validate(grid, params);
  if (st != LBM_OK) return st;
  const long long n = static_cast<long long>(grid->nx) * grid->ny * grid->nz;
  const size_t plane = static_cast<size_t>((n + 63) / 64 * 64) * sizeof(float);
  const size_t state = lbm::state_bytes(static_cast<int>(n), params->storage);
  *bytes = state * (params->pattern == LBM_PATTERN_AB ? 2 : 1) +
           plane * (wants_phi_alt(*grid, *params) ? 10 : 9) +
           sizeof(double) * (5 * lbm::kReduceMaxParts + 8) + step_parts_bytes(n);
  return LBM_OK;
}

lbm_status lbm_destroy(lbm_ctx* c) {
  if (!c) return LBM_EINVAL;
  cudaStreamSynchronize(c->stream);
  release(c);
  delete c;
  return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* c) {
  return c ? c->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
