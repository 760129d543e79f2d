// Host-side declarations shared by the C ABI and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

// Upper bound on the number of per-block partial sums of the FP64 reduction.
constexpr int kReduceMaxParts = 1024;

cudaError_t launch_phi(const float* pop, float* phi, const Geometry& geo, bool odd,
                       cudaStream_t st);
cudaError_t launch_mu(const float* phi, float* mu, const Geometry& geo, const Physics& ph,
                      cudaStream_t st);
cudaError_t launch_collide(float* pop, float* phiu, const float* phi, const float* mu,
                           const Geometry& geo, const Physics& ph, bool odd, bool have_prev,
                           cudaStream_t st);
cudaError_t launch_fields(const float* pop, const float* phi, const float* mu, float* out,
                          const Geometry& geo, const Physics& ph, bool odd, cudaStream_t st);
cudaError_t launch_init(float* pop, float* phiu, const float* phi, const float* mu,
                        const float* u0, const float* p0, const Geometry& geo,
                        const Physics& ph, cudaStream_t st);
cudaError_t launch_gather(const float* pop, float* dense, const Geometry& geo, bool odd,
                          int slot, cudaStream_t st);
cudaError_t launch_convert(const double* in, float* out, int n, cudaStream_t st);
int reduce_parts(const Geometry& geo);
cudaError_t launch_reduce(const float* pop, const float* phi, double* partial, double* out,
                          const Geometry& geo, bool odd, cudaStream_t st);

}  // namespace lbm
