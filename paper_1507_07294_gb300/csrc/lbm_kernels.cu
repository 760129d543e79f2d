// Kernels of the coupled D3Q7 + D3Q15 MRT multiphase update (Liang, Shi & Chai,
// arXiv:1507.07294, Sec. II) for sm_103a, and their host-side launchers.
//
// One time step is three grid passes; the data dependency radius is 2 (lap mu at x
// needs mu at x +- c_i, which needs phi at x +- 2 c_i):
//   k_phi      phi = sum_i f_i of the streamed populations (Eqs. 13, 16)
//   k_mu       mu = 4 beta phi (phi^2 - 1) - kappa lap phi (Eq. 2, Eq. 36)
//   k_collide  fused: pull f and g, stencils of phi and mu, forces, u and p, both MRT
//              collisions, d_t(phi u), push f+ and g+ (Eqs. 14-34)
// plus initialisation, field read-out, state gather/scatter and the FP64 reduction.
#include <cuda_runtime.h>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ void cell_coords(const Geometry& geo, int idx, int& x, int& y, int& z) {
  x = idx % geo.nx;
  const int r = idx / geo.nx;
  y = r % geo.ny;
  z = r / geo.ny;
}

// ------------------------------------------------------------------ k_phi ---------
template <bool ODD>
__global__ void __launch_bounds__(kBlock) k_phi(const float* __restrict__ pop,
                                                float* __restrict__ phi, Geometry geo) {
  const int idx = blockIdx.x * kBlock + threadIdx.x;
  if (idx >= geo.n) return;
  int x, y, z;
  cell_coords(geo, idx, x, y, z);
  const Nbr nb = make_nbr(geo, x, y, z);
  float f[7];
  load_f<ODD>(pop, geo.stride, idx, nb, f);
  phi[idx] = f[0] + ((f[1] + f[2]) + (f[3] + f[4]) + (f[5] + f[6]));
}

// ------------------------------------------------------------------- k_mu ---------
__global__ void __launch_bounds__(kBlock) k_mu(const float* __restrict__ phi,
                                               float* __restrict__ mu, Geometry geo,
                                               Physics ph) {
  const int idx = blockIdx.x * kBlock + threadIdx.x;
  if (idx >= geo.n) return;
  int x, y, z;
  cell_coords(geo, idx, x, y, z);
  const Nbr nb = make_nbr(geo, x, y, z);
  Stencil s;
  load_stencil(phi, idx, nb, s);
  mu[idx] = chemical_potential(ph, s.c, stencil_lap(s));
}

// -------------------------------------------------------------- k_collide ---------
template <bool ODD>
__global__ void __launch_bounds__(kBlock) k_collide(float* pop,
                                                    float* __restrict__ phiu,
                                                    const float* __restrict__ phi,
                                                    const float* __restrict__ mu,
                                                    Geometry geo, Physics ph, int have_prev) {
  const int idx = blockIdx.x * kBlock + threadIdx.x;
  if (idx >= geo.n) return;
  int x, y, z;
  cell_coords(geo, idx, x, y, z);
  const Nbr nb = make_nbr(geo, x, y, z);

  float grad_phi[3], lap_mu, phi_c, mu_c;
  {
    Stencil s;
    load_stencil(phi, idx, nb, s);
    stencil_grad(s, grad_phi);
    phi_c = s.c;
  }
  {
    Stencil s;
    load_stencil(mu, idx, nb, s);
    lap_mu = stencil_lap(s);
    mu_c = s.c;
  }

  float g[15];
  load_g<ODD>(pop, geo.stride, idx, nb, g);
  const Macro M = macroscopic(ph, g, phi_c, mu_c, grad_phi, lap_mu);
  const float lambda_visc = 1.0f / (3.0f * (ph.nu_mid + phi_c * ph.half_dnu) + 0.5f);
  collide_d3q15(ph, g, M, lambda_visc);
  store_g<ODD>(pop, geo.stride, idx, nb, g);

  // d_t(phi u) by the backward difference of Eq. 34
  float dphiu[3];
  const size_t s = geo.stride;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float cur = phi_c * M.u[a];
    dphiu[a] = have_prev ? cur - phiu[a * s + idx] : 0.0f;
    phiu[a * s + idx] = cur;
  }

  float f[7];
  load_f<ODD>(pop, geo.stride, idx, nb, f);
  collide_d3q7(ph, f, phi_c, mu_c, M.u, dphiu);
  store_f<ODD>(pop, geo.stride, idx, nb, f);
}

// --------------------------------------------------------------- k_fields ---------
// rho, p, u of the current populations into out[0..4] (rho, p, ux, uy, uz).
template <bool ODD>
__global__ void __launch_bounds__(kBlock) k_fields(const float* __restrict__ pop,
                                                   const float* __restrict__ phi,
                                                   const float* __restrict__ mu,
                                                   float* __restrict__ out, Geometry geo,
                                                   Physics ph) {
  const int idx = blockIdx.x * kBlock + threadIdx.x;
  if (idx >= geo.n) return;
  int x, y, z;
  cell_coords(geo, idx, x, y, z);
  const Nbr nb = make_nbr(geo, x, y, z);
  float grad_phi[3], lap_mu, phi_c, mu_c;
  {
    Stencil s;
    load_stencil(phi, idx, nb, s);
    stencil_grad(s, grad_phi);
    phi_c = s.c;
  }
  {
    Stencil s;
    load_stencil(mu, idx, nb, s);
    lap_mu = stencil_lap(s);
    mu_c = s.c;
  }
  float g[15];
  load_g<ODD>(pop, geo.stride, idx, nb, g);
  const Macro M = macroscopic(ph, g, phi_c, mu_c, grad_phi, lap_mu);
  const size_t s = geo.stride;
  out[0 * s + idx] = M.rho;
  out[1 * s + idx] = M.p;
  out[2 * s + idx] = M.u[0];
  out[3 * s + idx] = M.u[1];
  out[4 * s + idx] = M.u[2];
}

// ------------------------------------------------------------------ k_init --------
// f = f^eq (Eq. 5), g = g^eq (Eq. 21) in the even-step layout; phi u stored.
// u0 and p0 may be null (zero).
__global__ void __launch_bounds__(kBlock) k_init(float* __restrict__ pop,
                                                 float* __restrict__ phiu,
                                                 const float* __restrict__ phi,
                                                 const float* __restrict__ mu,
                                                 const float* __restrict__ u0,
                                                 const float* __restrict__ p0, Geometry geo,
                                                 Physics ph) {
  const int idx = blockIdx.x * kBlock + threadIdx.x;
  if (idx >= geo.n) return;
  const size_t s = geo.stride;
  const float ph_ = phi[idx], mu_ = mu[idx];
  float u[3] = {0.0f, 0.0f, 0.0f};
  if (u0) {
    u[0] = u0[idx];
    u[1] = u0[s + idx];
    u[2] = u0[2 * s + idx];
  }
  const float p = p0 ? p0[idx] : 0.0f;
  const float rho = ph.rho_g + (1.0f + ph_) * ph.half_drho;

  // D3Q7: omega_0 = 1 - 3A, omega_i = A/2, c_s^2 = A
  const float emu = ph.eta * mu_;
  const float hw = 0.5f * ph.A * emu;
  pop[0 * s + idx] = ph_ - 3.0f * ph.A * emu;
  const float jx = 0.5f * ph_ * u[0], jy = 0.5f * ph_ * u[1], jz = 0.5f * ph_ * u[2];
  pop[1 * s + idx] = hw + jx;
  pop[2 * s + idx] = hw - jx;
  pop[3 * s + idx] = hw + jy;
  pop[4 * s + idx] = hw - jy;
  pop[5 * s + idx] = hw + jz;
  pop[6 * s + idx] = hw - jz;

  // D3Q15: g_i = 3 p omega_i + rho omega_i (3 c.u + 9/2 (c.u)^2 - 3/2 u^2), g_0 -= 3p
  const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  constexpr int cx[15] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
  constexpr int cy[15] = {0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, -1, 1, -1, 1};
  constexpr int cz[15] = {0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1, -1, 1};
#pragma unroll
  for (int i = 0; i < 15; ++i) {
    const float w = i == 0 ? 2.0f / 9.0f : (i < 7 ? 1.0f / 9.0f : 1.0f / 72.0f);
    const float cu = cx[i] * u[0] + cy[i] * u[1] + cz[i] * u[2];
    float v = 3.0f * p * w + rho * w * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu);
    if (i == 0) v -= 3.0f * p;
    pop[(7 + i) * s + idx] = v;
  }
  phiu[0 * s + idx] = ph_ * u[0];
  phiu[1 * s + idx] = ph_ * u[1];
  phiu[2 * s + idx] = ph_ * u[2];
}

// -------------------------------------------------- state gather / scatter --------
// Population `slot` of the current (pre-collision) state to dense[idx].
template <bool ODD>
__global__ void __launch_bounds__(kBlock) k_gather(const float* __restrict__ pop,
                                                   float* __restrict__ dense, Geometry geo,
                                                   int slot) {
  const int idx = blockIdx.x * kBlock + threadIdx.x;
  if (idx >= geo.n) return;
  int x, y, z;
  cell_coords(geo, idx, x, y, z);
  const Nbr nb = make_nbr(geo, x, y, z);
  float v = 0.0f;
  if (slot < 7) {
    float f[7];
    load_f<ODD>(pop, geo.stride, idx, nb, f);
#pragma unroll
    for (int q = 0; q < 7; ++q)
      if (q == slot) v = f[q];
  } else {
    float g[15];
    load_g<ODD>(pop, geo.stride, idx, nb, g);
#pragma unroll
    for (int q = 0; q < 15; ++q)
      if (q == slot - 7) v = g[q];
  }
  dense[idx] = v;
}

__global__ void __launch_bounds__(kBlock) k_convert(const double* __restrict__ in,
                                                    float* __restrict__ out, int n) {
  const int idx = blockIdx.x * kBlock + threadIdx.x;
  if (idx < n) out[idx] = static_cast<float>(in[idx]);
}

// --------------------------------------------------------------- k_reduce ---------
// Pass 1: block b sums cells b, b + B, ... in FP64 (fixed order: grid-stride by block
// rows, then a fixed shuffle tree).  partial[b] = {sum phi, jx, jy, jz, non-finite}.
template <bool ODD>
__global__ void __launch_bounds__(kBlock) k_reduce_partial(const float* __restrict__ pop,
                                                           const float* __restrict__ phi,
                                                           double* __restrict__ partial,
                                                           Geometry geo) {
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int idx = blockIdx.x * kBlock + threadIdx.x; idx < geo.n; idx += gridDim.x * kBlock) {
    int x, y, z;
    cell_coords(geo, idx, x, y, z);
    const Nbr nb = make_nbr(geo, x, y, z);
    float g[15];
    load_g<ODD>(pop, geo.stride, idx, nb, g);
    const float d7 = g[7] - g[8], d9 = g[9] - g[10], d11 = g[11] - g[12], d13 = g[13] - g[14];
    const float jx = (g[1] - g[2]) + ((d7 + d9) + (d11 + d13));
    const float jy = (g[3] - g[4]) + ((d7 + d9) - (d11 + d13));
    const float jz = (g[5] - g[6]) + ((d7 - d9) + (d11 - d13));
    const float p = phi[idx];
    acc[0] += p;
    acc[1] += jx;
    acc[2] += jy;
    acc[3] += jz;
    if (!(isfinite(p) && isfinite(jx) && isfinite(jy) && isfinite(jz))) acc[4] += 1.0;
  }
  __shared__ double sh[kBlock / 32][5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    double v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double v = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) v += sh[w][threadIdx.x];
    partial[blockIdx.x * 5 + threadIdx.x] = v;
  }
}

// Pass 2: one block folds the partials in a fixed order.
__global__ void __launch_bounds__(kBlock) k_reduce_final(const double* __restrict__ partial,
                                                         int nparts, double* __restrict__ out) {
  __shared__ double sh[kBlock];
  for (int k = 0; k < 5; ++k) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nparts; b += kBlock) v += partial[b * 5 + k];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = sh[0];
    __syncthreads();
  }
}

inline unsigned blocks_for(int n) { return static_cast<unsigned>((n + kBlock - 1) / kBlock); }

}  // namespace

// ------------------------------------------------------------ host launchers ------
cudaError_t launch_phi(const float* pop, float* phi, const Geometry& geo, bool odd,
                       cudaStream_t st) {
  if (odd)
    k_phi<true><<<blocks_for(geo.n), kBlock, 0, st>>>(pop, phi, geo);
  else
    k_phi<false><<<blocks_for(geo.n), kBlock, 0, st>>>(pop, phi, geo);
  return cudaGetLastError();
}

cudaError_t launch_mu(const float* phi, float* mu, const Geometry& geo, const Physics& ph,
                      cudaStream_t st) {
  k_mu<<<blocks_for(geo.n), kBlock, 0, st>>>(phi, mu, geo, ph);
  return cudaGetLastError();
}

cudaError_t launch_collide(float* pop, float* phiu, const float* phi, const float* mu,
                           const Geometry& geo, const Physics& ph, bool odd, bool have_prev,
                           cudaStream_t st) {
  if (odd)
    k_collide<true><<<blocks_for(geo.n), kBlock, 0, st>>>(pop, phiu, phi, mu, geo, ph, have_prev);
  else
    k_collide<false><<<blocks_for(geo.n), kBlock, 0, st>>>(pop, phiu, phi, mu, geo, ph, have_prev);
  return cudaGetLastError();
}

cudaError_t launch_fields(const float* pop, const float* phi, const float* mu, float* out,
                          const Geometry& geo, const Physics& ph, bool odd, cudaStream_t st) {
  if (odd)
    k_fields<true><<<blocks_for(geo.n), kBlock, 0, st>>>(pop, phi, mu, out, geo, ph);
  else
    k_fields<false><<<blocks_for(geo.n), kBlock, 0, st>>>(pop, phi, mu, out, geo, ph);
  return cudaGetLastError();
}

cudaError_t launch_init(float* pop, float* phiu, const float* phi, const float* mu,
                        const float* u0, const float* p0, const Geometry& geo,
                        const Physics& ph, cudaStream_t st) {
  k_init<<<blocks_for(geo.n), kBlock, 0, st>>>(pop, phiu, phi, mu, u0, p0, geo, ph);
  return cudaGetLastError();
}

cudaError_t launch_gather(const float* pop, float* dense, const Geometry& geo, bool odd,
                          int slot, cudaStream_t st) {
  if (odd)
    k_gather<true><<<blocks_for(geo.n), kBlock, 0, st>>>(pop, dense, geo, slot);
  else
    k_gather<false><<<blocks_for(geo.n), kBlock, 0, st>>>(pop, dense, geo, slot);
  return cudaGetLastError();
}

cudaError_t launch_convert(const double* in, float* out, int n, cudaStream_t st) {
  k_convert<<<blocks_for(n), kBlock, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

int reduce_parts(const Geometry& geo) {
  const int b = static_cast<int>(blocks_for(geo.n));
  return b < kReduceMaxParts ? b : kReduceMaxParts;
}

cudaError_t launch_reduce(const float* pop, const float* phi, double* partial, double* out,
                          const Geometry& geo, bool odd, cudaStream_t st) {
  const int parts = reduce_parts(geo);
  if (odd)
    k_reduce_partial<true><<<parts, kBlock, 0, st>>>(pop, phi, partial, geo);
  else
    k_reduce_partial<false><<<parts, kBlock, 0, st>>>(pop, phi, partial, geo);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reduce_final<<<1, kBlock, 0, st>>>(partial, parts, out);
  return cudaGetLastError();
}

}  // namespace lbm
