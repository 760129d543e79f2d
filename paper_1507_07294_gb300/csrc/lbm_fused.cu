// Single-pass time step of the coupled D3Q7 + D3Q15 MRT update (Liang, Shi & Chai,
// arXiv:1507.07294, Sec. II): the order parameter (Eqs. 13, 16), the chemical potential
// (Eq. 2 with the Laplacian of Eq. 36) and the fused stream-collide (Eqs. 14-34) in one
// kernel, for the two-array pull pattern.
//
// The three-pass step (lbm_kernels.cu) reads the 7 f slots twice (once for phi, once
// for the collision) and moves phi and mu through global memory: 248 B per cell in
// FP32 against the 200 B of the state itself.  Here each block owns a 32 x 8 column of
// cells and marches up z.  At iteration L it
//   A. forms phi of plane L on the block's 36 x 12 cells plus a 2-cell halo from the
//      pulled f (the halo cells' f come from neighbouring blocks' tiles, mostly L2 hits),
//   B. forms mu of plane L - 1 on the 34 x 10 cells with a 1-cell halo from phi planes
//      L - 2 .. L (15-point stencil in shared memory),
//   C. collides plane L - 2 with the phi and mu stencils read from shared memory.
// phi and mu never reach global memory (16-bit storage excepted: it writes phi for the
// shift of slot 0, to a second array).  The pulled f of the block's own cells, read for
// phi in A, wait in shared memory for the collision two iterations later (re-reading
// them from global memory that late would miss L2), and the collision's g and phi u
// loads are issued at the top of the iteration, before A, so that their latency
// overlaps A and B.  The arithmetic of every value is the same code in the same order
// as in the three-pass kernels, so both paths give the same bits.
//
// The z range is cut into segments (one per blockIdx.z) so that the grid has enough
// blocks; a segment computes phi on 2 planes below and above it and mu on 1, which the
// neighbouring segments compute too.
#include <cuda_runtime.h>

#include "lbm_cells.cuh"
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kFX = kTile;              // cells per block row: one tile
constexpr int kFY = 8;                  // rows per block
constexpr int kFThreads = kFX * kFY;    // 256: one thread per cell of a plane
constexpr int kPW = kFX + 4, kPH = kFY + 4;  // phi region: 2-cell halo
constexpr int kMW = kFX + 2, kMH = kFY + 2;  // mu region: 1-cell halo
// Ring depths.  Iteration L writes phi(L) before its first barrier; the oldest plane
// still read is L - 3 (collision of L - 2), and plane L - 4 was last read by the
// collision of iteration L - 1, which has no barrier after it: hence 5 planes.  mu(L-1)
// is written after the first barrier of iteration L, which orders it after iteration
// L - 1's reads of mu(L - 4): 3 planes suffice.  The pulled f of plane L are written
// before the first barrier and read by the collision of iteration L + 2; the slot they
// overwrite, plane L - 4's, was last read in iteration L - 2: 4 planes.
constexpr int kPR = 5, kMR = 3, kFR = 4;

struct FusedSmem {
  float phi[kPR][kPH][kPW];
  float mu[kMR][kMH][kMW];
  float f[kFR][kQ7][kFY][kFX];
};

__device__ __forceinline__ int phi_slot(int p) { return (p + 10) % kPR; }  // p >= -3
__device__ __forceinline__ int mu_slot(int p) { return (p + 12) % kMR; }   // p >= -3
__device__ __forceinline__ int f_slot(int p) { return (p + 12) % kFR; }    // p >= -3

// Whether plane p of the marching index is a plane of the grid: between walls only
// 0..nz-1 are; with periodic z every p is (its image).
__device__ __forceinline__ bool plane_real(const Geometry& geo, int p) {
  return !geo.walls || (p >= 0 && p < geo.nz);
}

// Grid plane of marching index p (periodic image; p in range between walls).
__device__ __forceinline__ int plane_of(const Geometry& geo, int p) {
  if (geo.walls) return p;
  p %= geo.nz;
  return p < 0 ? p + geo.nz : p;
}

// Marching index whose ring slot holds the values a stencil wants at plane p: between
// walls the ghost of a plane beyond the wall is the adjacent fluid plane.
__device__ __forceinline__ int stencil_plane(const Geometry& geo, int p) {
  return geo.walls ? min(max(p, 0), geo.nz - 1) : p;
}

// phi at (x, y, z) from the pulled populations, the sum exactly as in phi_cell; the
// pulled values (f_0 before the 16-bit shift is undone) are left in f.
template <int S>
__device__ __forceinline__ float phi_at(const float* src, const float* phi_ref,
                                        const Geometry& geo, int x, int y, int z, float f[7]) {
  typedef Elem<S> E;
  const int xm = x == 0 ? geo.nx - 1 : x - 1, xp = x == geo.nx - 1 ? 0 : x + 1;
  const int dym = y == 0 ? (geo.ny - 1) * geo.nx : -geo.nx;
  const int dyp = y == geo.ny - 1 ? -(geo.ny - 1) * geo.nx : geo.nx;
  const int row = (z * geo.ny + y) * geo.nx;
  const int c = row + x;
  f[0] = E::get(*pop_ptr<S, 0>(src, c));
  f[1] = E::get(*pop_ptr<S, 1>(src, row + xm));
  f[2] = E::get(*pop_ptr<S, 2>(src, row + xp));
  f[3] = E::get(*pop_ptr<S, 3>(src, c + dym));
  f[4] = E::get(*pop_ptr<S, 4>(src, c + dyp));
  if (geo.walls && z == 0)
    f[5] = E::get(*pop_ptr<S, 6>(src, c));  // bounce-back at the bottom wall
  else
    f[5] = E::get(*pop_ptr<S, 5>(src, c + (z == 0 ? (geo.nz - 1) * geo.plane : -geo.plane)));
  if (geo.walls && z == geo.nz - 1)
    f[6] = E::get(*pop_ptr<S, 5>(src, c));  // bounce-back at the top wall
  else
    f[6] = E::get(*pop_ptr<S, 6>(src, c + (z == geo.nz - 1 ? -(geo.nz - 1) * geo.plane : geo.plane)));
  const float f0 = S != kF32 ? f[0] + phi_ref[c] : f[0];
  return f0 + ((f[1] + f[2]) + (f[3] + f[4]) + (f[5] + f[6]));
}

// 3 resident blocks per SM (80 registers); at 4 (64 registers) the 16-bit kernels spill.
template <int S>
constexpr int fused_min_blocks() {
  return 3;
}

// One launch = one time step.  Block (bx, by, bs): cells x0 = 32 bx .. x0 + 31,
// y0 = 8 by .. y0 + 7, z in [bs seg, min(nz, (bs + 1) seg)).  Thread t: lane tx = t % 32,
// row ty = t / 32.  phi_in / phi_out: order parameter of the previous / this step (16-bit
// storage only; unused in FP32).  With SUMS each warp leaves its tile's sums in parts.
// `pf` is the L2 prefetch distance in planes (0: none).
template <int S, bool SUMS>
__global__ void __launch_bounds__(kFThreads, fused_min_blocks<S>())
    k_fused(const float* src, float* dst, const float* phi_in, float* phi_out, Geometry geo,
            Physics ph, int have_prev, int seg, int pf, float* parts) {
  __shared__ FusedSmem sm;
  const int tx = threadIdx.x & (kFX - 1), ty = threadIdx.x >> kTileShift;
  const int x0 = blockIdx.x * kFX, y0 = blockIdx.y * kFY;
  const int z0 = blockIdx.z * seg;
  const int z1 = min(z0 + seg, geo.nz);
  const int nx = geo.nx, ny = geo.ny;
  auto wrap_x = [&](int x) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); };
  auto wrap_y = [&](int y) { y %= ny; return y < 0 ? y + ny : y; };

  // phi items of this thread: main items k = t and t + 256 (< 384) cover rows 0..11,
  // columns 2..33; edge items e = t - 128 in [0, 48) cover columns 0, 1, 34, 35
  const int t = threadIdx.x;
  const bool has_main2 = t + kFThreads < kPH * kFX;
  const int e = t - 128;
  const bool has_edge = e >= 0 && e < kPH * 4;
  const int edge_r = e >> 2, edge_c = (e & 3) < 2 ? (e & 3) : kPW - 4 + (e & 3);
  // mu items: main k = t and t + 256 (< 320) over rows 0..9, columns 1..32; edges
  // e2 = t - 64 in [0, 20) at columns 0 and 33
  const bool has_mu2 = t + kFThreads < kMH * kFX;
  const int e2 = t - 64;
  const bool has_mu_edge = e2 >= 0 && e2 < kMH * 2;

  for (int L = z0 - 2; L <= z1 + 1; ++L) {
    // L2 prefetch of the tiles this block streams pf planes ahead: each warp the whole
    // tile of its own row, warps 0..3 the f slots of the halo rows y0-2, y0-1, y0+8, y0+9
    if (pf > 0 && tx == 0) {
      const int pq = L + pf;
      if (pq <= z1 + 1 && plane_real(geo, pq)) {
        const int zq = plane_of(geo, pq);
        const int cell = (zq * ny + (y0 + ty)) * nx + x0;
        prefetch_l2(src + tile_floats<S>(cell), static_cast<unsigned>(tile_bytes<S>()));
        if (ty < 4) {
          const int yh = wrap_y(ty < 2 ? y0 - 2 + ty : y0 + kFY + ty - 2);
          const int ch = (zq * ny + yh) * nx + x0;
          prefetch_l2(src + tile_floats<S>(ch),
                      static_cast<unsigned>(kQ7 * kTile * sizeof(typename Elem<S>::T)));
        }
      }
    }
    // the collision's g and phi u (plane L - 2), loaded now so that they arrive during A
    // and B
    const int Zc = L - 2;
    const bool collide = Zc >= z0;
    const int cz = plane_of(geo, collide ? Zc : z0);
    const int idx = (cz * ny + (y0 + ty)) * nx + x0 + tx;
    const Nbr nb = make_nbr(geo, x0 + tx, y0 + ty, cz);
    float g[15], prev[3];
    if (collide) load_cell<kAB, S, false>(src, geo, idx, nb, g, nullptr, prev);
    // A. phi of plane L; the pulled f of the own cells go to the f ring for the
    // collision of plane L in iteration L + 2
    if (plane_real(geo, L)) {
      const int z = plane_of(geo, L);
      float(*P)[kPW] = sm.phi[phi_slot(L)];
      const bool own_plane = L >= z0 && L < z1;
      float fp[7];
      {
        const int r = ty;  // main item t: rows 0..7
        const float v = phi_at<S>(src, phi_in, geo, x0 + tx, wrap_y(y0 - 2 + r), z, fp);
        P[r][tx + 2] = v;
        if (own_plane && r >= 2) {
          if (S != kF32) phi_out[(z * ny + (y0 + r - 2)) * nx + x0 + tx] = v;
#pragma unroll
          for (int i = 0; i < kQ7; ++i) sm.f[f_slot(L)][i][r - 2][tx] = fp[i];
        }
      }
      if (has_main2) {
        const int r = ty + kFY;  // rows 8..11
        const float v = phi_at<S>(src, phi_in, geo, x0 + tx, wrap_y(y0 - 2 + r), z, fp);
        P[r][tx + 2] = v;
        if (own_plane && r < kFY + 2) {
          if (S != kF32) phi_out[(z * ny + (y0 + r - 2)) * nx + x0 + tx] = v;
#pragma unroll
          for (int i = 0; i < kQ7; ++i) sm.f[f_slot(L)][i][r - 2][tx] = fp[i];
        }
      }
      if (has_edge)
        P[edge_r][edge_c] = phi_at<S>(src, phi_in, geo, wrap_x(x0 - 2 + edge_c),
                                      wrap_y(y0 - 2 + edge_r), z, fp);
    }
    __syncthreads();
    // B. mu of plane L - 1 (the 15-point Laplacian exactly as in mu_columns)
    const int Q = L - 1;
    if (Q >= z0 - 1 && plane_real(geo, Q)) {
      const float(*P0)[kPW] = sm.phi[phi_slot(stencil_plane(geo, Q - 1))];
      const float(*P1)[kPW] = sm.phi[phi_slot(Q)];
      const float(*P2)[kPW] = sm.phi[phi_slot(stencil_plane(geo, Q + 1))];
      float(*Mq)[kMW] = sm.mu[mu_slot(Q)];
      // mu at mu-region (i, j) = phi-region (i + 1, j + 1)
      auto mu_item = [&](int i, int j) {
        const int a = i + 1, b = j + 1;
        const float c0 = P0[a][b], c1 = P1[a][b], c2 = P2[a][b];
        const float f1 = (P1[a][b - 1] + P1[a][b + 1]) + (P1[a - 1][b] + P1[a + 1][b]);
        const float d0 = (P0[a - 1][b - 1] + P0[a - 1][b + 1]) + (P0[a + 1][b - 1] + P0[a + 1][b + 1]);
        const float d2 = (P2[a - 1][b - 1] + P2[a - 1][b + 1]) + (P2[a + 1][b - 1] + P2[a + 1][b + 1]);
        const float lap = lap15_columns(c0, c1, c2, f1, d0, d2);
        Mq[i][j] = chemical_potential(ph, c1, lap);
      };
      mu_item(ty, tx + 1);
      if (has_mu2) mu_item(ty + kFY, tx + 1);
      if (has_mu_edge) mu_item(e2 >> 1, (e2 & 1) ? kMW - 1 : 0);
    }
    __syncthreads();
    // C. collision of plane L - 2
    if (collide) {
      const int zm = stencil_plane(geo, Zc - 1), zp = stencil_plane(geo, Zc + 1);
      float f[7];
#pragma unroll
      for (int i = 0; i < kQ7; ++i) f[i] = sm.f[f_slot(Zc)][i][ty][tx];
      auto stencils = [&] {
        CellStencils cs;
        {
          const float(*A0)[kPW] = sm.phi[phi_slot(zm)];
          const float(*A1)[kPW] = sm.phi[phi_slot(Zc)];
          const float(*A2)[kPW] = sm.phi[phi_slot(zp)];
          const int r = ty + 2, j = tx + 2;
          Stencil s;
          s.c = A1[r][j];
          s.xm = A1[r][j - 1];
          s.xp = A1[r][j + 1];
          s.ym = A1[r - 1][j];
          s.yp = A1[r + 1][j];
          s.zm = A0[r][j];
          s.zp = A2[r][j];
#pragma unroll
          for (int bb = 0; bb < 8; ++bb)
            s.k[bb] = ((bb & 4) ? A2 : A0)[r + ((bb & 2) ? 1 : -1)][j + ((bb & 1) ? 1 : -1)];
          stencil_grad(s, cs.grad_phi);
          cs.phi = s.c;
        }
        {
          const float(*B0)[kMW] = sm.mu[mu_slot(zm)];
          const float(*B1)[kMW] = sm.mu[mu_slot(Zc)];
          const float(*B2)[kMW] = sm.mu[mu_slot(zp)];
          const int r = ty + 1, j = tx + 1;
          Stencil s;
          s.c = B1[r][j];
          s.xm = B1[r][j - 1];
          s.xp = B1[r][j + 1];
          s.ym = B1[r - 1][j];
          s.yp = B1[r + 1][j];
          s.zm = B0[r][j];
          s.zp = B2[r][j];
#pragma unroll
          for (int bb = 0; bb < 8; ++bb)
            s.k[bb] = ((bb & 4) ? B2 : B0)[r + ((bb & 2) ? 1 : -1)][j + ((bb & 1) ? 1 : -1)];
          cs.lap_mu = stencil_lap(s);
          cs.mu = s.c;
        }
        return cs;
      };
      if (SUMS) {
        float s4[4];
        collide_loaded<kAB, 0, S, true>(dst, geo, ph, have_prev, idx, nb, g, f, prev, stencils, s4);
        const bool bad = !(isfinite(s4[0]) && isfinite(s4[1]) && isfinite(s4[2]) && isfinite(s4[3]));
        warp_sums_store(s4, bad, parts, idx & ~31);
      } else {
        collide_loaded<kAB, 0, S, false>(dst, geo, ph, have_prev, idx, nb, g, f, prev, stencils,
                                         nullptr);
      }
    }
  }
}

template <int S>
cudaError_t launch_fused_s(const float* src, float* dst, const float* phi_in, float* phi_out,
                           const Geometry& geo, const Physics& ph, bool have_prev, int seg,
                           int pf, float* parts, cudaStream_t st) {
  const dim3 grid(geo.nx / kFX, geo.ny / kFY, (geo.nz + seg - 1) / seg);
  const int prev = have_prev ? 1 : 0;
  if (parts)
    k_fused<S, true><<<grid, kFThreads, 0, st>>>(src, dst, phi_in, phi_out, geo, ph, prev, seg,
                                                 pf, parts);
  else
    k_fused<S, false><<<grid, kFThreads, 0, st>>>(src, dst, phi_in, phi_out, geo, ph, prev, seg,
                                                  pf, nullptr);
  return cudaGetLastError();
}

}  // namespace

// Whole blocks in x and y, and a grid whose y and z extents (ny / 8 and the segments,
// at least one plane each) stay within 65535.
bool fused_shape_ok(const Geometry& geo) {
  return geo.row_tiles > 0 && geo.nx % kFX == 0 && geo.ny % kFY == 0 && geo.ny / kFY <= 65535 &&
         geo.nz <= 65535;
}

int fused_default_segment(const Geometry& geo, int sms) {
  // about 4 waves of 3 blocks per SM, segments of 16 to 64 planes (a segment re-forms
  // phi on 4 and mu on 2 planes beyond its ends)
  const long long cols = static_cast<long long>(geo.nx / kFX) * (geo.ny / kFY);
  const long long want = 4LL * 3 * (sms > 0 ? sms : 152);
  long long seg = cols > 0 ? (static_cast<long long>(geo.nz) * cols + want - 1) / want : geo.nz;
  if (seg < 16) seg = 16;
  if (seg > 64) seg = 64;
  if (seg > geo.nz) seg = geo.nz;
  return static_cast<int>(seg);
}

cudaError_t launch_fused(const float* src, float* dst, const float* phi_in, float* phi_out,
                         const Geometry& geo, const Physics& ph, bool have_prev, int seg, int pf,
                         float* parts, double* partial, double* out, cudaStream_t st) {
  cudaError_t e;
  if (geo.storage == kF16)
    e = launch_fused_s<kF16>(src, dst, phi_in, phi_out, geo, ph, have_prev, seg, pf, parts, st);
  else if (geo.storage == kBF16)
    e = launch_fused_s<kBF16>(src, dst, phi_in, phi_out, geo, ph, have_prev, seg, pf, parts, st);
  else
    e = launch_fused_s<kF32>(src, dst, phi_in, phi_out, geo, ph, have_prev, seg, pf, parts, st);
  if (e != cudaSuccess || !parts) return e;
  return launch_step_sums_final(parts, partial, out, geo, st);
}

}  // namespace lbm
