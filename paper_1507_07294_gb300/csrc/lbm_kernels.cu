// Kernels of the coupled D3Q7 + D3Q15 MRT multiphase update (Liang, Shi & Chai,
// arXiv:1507.07294, Sec. II) for sm_103a, and their host-side launchers.
//
// One time step is three grid passes; the data dependency radius is 2 (lap mu at x
// needs mu at x +- c_i, which needs phi at x +- 2 c_i):
//   k_phi      phi = sum_i f_i of the streamed populations (Eqs. 13, 16); k_phi_rows
//              is the same pass for grids whose rows are whole tiles
//   k_mu       mu = 4 beta phi (phi^2 - 1) - kappa lap phi (Eq. 2, Eq. 36); k_mu_tma
//              fetches its halo bricks with TMA tensor copies
//   k_collide  fused: pull f and g, stencils of phi and mu, forces, u and p, both MRT
//              collisions, d_t(phi u), store f+ and g+ (Eqs. 14-34)
// plus k_collide_sums (k_collide that also sums the state it writes, for
// lbm_step_reduce), k_che (interface tracking with a prescribed velocity),
// initialisation, field read-out, state gather/scatter and the FP64 reduction.
// Every kernel is templated on the population storage pattern and type
// (lbm_device.cuh); the per-cell bodies live in lbm_cells.cuh, shared with the batched
// kernels.
#include <cuda.h>
#include <cuda_runtime.h>

#include "lbm_cells.cuh"
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

namespace {

// Latency hiding for the streaming kernels: thread 0 of block b prefetches into L2 the
// data of the cells of block b + dist, which a block of the next wave will stream in
// (dist = one wave: SMs x resident blocks per SM).  k_collide prefetches the whole cell
// state of those cells (all 25 slots) and their phi and mu; k_phi only the 7 f slots of
// each tile.
template <int S, bool ALL_SLOTS>
__device__ __forceinline__ void prefetch_ahead(const float* state, const float* phi, const float* mu,
                                               const Geometry& geo, int dist) {
  if (dist <= 0 || threadIdx.x != 0) return;
  prefetch_cells<S, ALL_SLOTS>(state, phi, mu, geo,
                               static_cast<long long>(blockIdx.x + dist) * kBlock);
}

// ------------------------------------------------------------------ k_phi ---------
// With 16-bit storage slot 0 holds f_0 - phi_ref, phi_ref the order parameter of the
// step that wrote it; phi_ref and phi may be the same array (each thread reads its own
// cell before writing it).
template <int P, int S>
__global__ void __launch_bounds__(kBlock) k_phi(const float* __restrict__ src,
                                                const float* phi_ref, float* phi, Geometry geo) {
  prefetch_ahead<S, false>(src, nullptr, nullptr, geo, geo.prefetch_phi);
  const int idx = blockIdx.x * kBlock + threadIdx.x;
  if (idx >= geo.n) return;
  phi_cell<P, S>(src, phi_ref, phi, geo, idx);
}

// ------------------------------------------------------------- k_phi_rows ---------
// k_phi on grids whose rows are whole tiles (Geometry::row_tiles > 0), for the pulls of
// pattern P (AB: slot i of x - c_i; the even in-place step: slot i of the cell itself;
// the odd one: slot opp(i) of x - c_i, across a wall slot i of the cell itself):
// each warp takes one tile (32 cells of a row) through kPhiRowsK consecutive planes, so
// the neighbour deltas and the coordinate bookkeeping are computed once per column
// rather than once per cell, and all loads of the column are issued before the first
// store (phi_ref may be phi itself: each cell's phi_ref is read before its own write).
// Block (bx, by): tiles 8 bx .. 8 bx + 7 of a plane, planes kPhiRowsK by onwards.  The
// sums are phi_cell's, in the same order, so the result is bitwise the same.  Lane 0 of
// each warp prefetches into L2 the 7 f slots of the tiles that the same warp of the
// block `ahead` rows of blocks further (blockIdx.y + ahead) will read; the launcher
// turns the prefetch distance geo.prefetch_phi, in blocks, into rows of blocks.
constexpr int kPhiRowsK = 2;

template <int S>
__device__ __forceinline__ void prefetch_rows_ahead(const float* src, const Geometry& geo, int tp,
                                                    int ahead) {
  if (ahead <= 0 || (threadIdx.x & (kTile - 1)) != 0) return;
  const int by = static_cast<int>(blockIdx.y) + ahead;
  if (by >= static_cast<int>(gridDim.y)) return;
  const int q = blockIdx.x * (kBlock / kTile) + (threadIdx.x >> kTileShift);
  if (q >= tp) return;
  constexpr int bytes = kQ7 * kTile * static_cast<int>(sizeof(typename Elem<S>::T));
  const int z1 = min(geo.nz, (by + 1) * kPhiRowsK);
  for (int z = by * kPhiRowsK; z < z1; ++z)
    prefetch_l2(reinterpret_cast<const char*>(src) + (static_cast<long long>(z) * tp + q) * tile_bytes<S>(),
                bytes);
}

template <int S, int P = kAB>
__global__ void __launch_bounds__(kBlock) k_phi_rows(const float* __restrict__ src,
                                                     const float* phi_ref, float* phi,
                                                     Geometry geo, int ahead) {
  typedef Elem<S> E;
  typedef typename E::T T;
  constexpr int EB = static_cast<int>(sizeof(T)), TB = tile_bytes<S>(), L = kTile - 1;
  constexpr int SL = kTile * EB;  // bytes of one slot of a tile
  const int tp = geo.plane >> kTileShift;  // tiles per plane
  prefetch_rows_ahead<S>(src, geo, tp, ahead);
  const int q = blockIdx.x * (kBlock / kTile) + (threadIdx.x >> kTileShift);
  if (q >= tp) return;
  const int lane = threadIdx.x & L, rt = geo.row_tiles, row = rt * TB;
  const int p = q * kTile + lane;  // cell within the plane
  const int y = fast_div(p, geo.div_nx);
  const int x = p - y * geo.nx;
  const int dxm = lane ? -EB : (x ? L * EB - TB : L * EB + (rt - 1) * TB);
  const int dxp = lane != L ? EB : (x != geo.nx - 1 ? TB - L * EB : -L * EB - (rt - 1) * TB);
  const int dym = y ? -row : (geo.ny - 1) * row;
  const int dyp = y != geo.ny - 1 ? row : -(geo.ny - 1) * row;
  const long long plane_b = static_cast<long long>(tp) * TB;
  const int z0 = blockIdx.y * kPhiRowsK;
  const int nk = min(kPhiRowsK, geo.nz - z0);
  const char* own = reinterpret_cast<const char*>(src) +
                    (static_cast<long long>(z0) * tp + q) * TB + lane * EB;
  const int cell0 = z0 * geo.plane + p;
  auto get = [](const char* a) { return E::get(*reinterpret_cast<const T*>(a)); };
  float f[kPhiRowsK][7], ref[kPhiRowsK];
#pragma unroll
  for (int k = 0; k < kPhiRowsK; ++k) {
    if (k < nk) {
      const int z = z0 + k;
      const char* o = own + k * plane_b;
      f[k][0] = get(o);
      if (P == kAAEven) {
#pragma unroll
        for (int i = 1; i < 7; ++i) f[k][i] = get(o + i * SL);
      } else if (P == kAAOdd) {
        // slot opp(i) of x - c_i: f_5 from slot 6 of z - 1, f_6 from slot 5 of z + 1;
        // across a wall each is the cell's own slot (5 and 6), one slot back and one
        // further
        const char* zm = z > 0 ? o - plane_b : (geo.walls ? o - SL : o + (geo.nz - 1) * plane_b);
        const char* zp = z < geo.nz - 1 ? o + plane_b
                                        : (geo.walls ? o + SL : o - (geo.nz - 1) * plane_b);
        f[k][1] = get(o + dxm + 2 * SL);
        f[k][2] = get(o + dxp + 1 * SL);
        f[k][3] = get(o + dym + 4 * SL);
        f[k][4] = get(o + dyp + 3 * SL);
        f[k][5] = get(zm + 6 * SL);
        f[k][6] = get(zp + 5 * SL);
      } else {
        // f_5 comes from z - 1 and f_6 from z + 1; across a wall each is the cell's own
        // opposite slot (6 and 5), i.e. one slot further and one slot back
        const char* zm = z > 0 ? o - plane_b : (geo.walls ? o + SL : o + (geo.nz - 1) * plane_b);
        const char* zp = z < geo.nz - 1 ? o + plane_b
                                        : (geo.walls ? o - SL : o - (geo.nz - 1) * plane_b);
        f[k][1] = get(o + dxm + 1 * SL);
        f[k][2] = get(o + dxp + 2 * SL);
        f[k][3] = get(o + dym + 3 * SL);
        f[k][4] = get(o + dyp + 4 * SL);
        f[k][5] = get(zm + 5 * SL);
        f[k][6] = get(zp + 6 * SL);
      }
      if (S != kF32) ref[k] = phi_ref[cell0 + k * geo.plane];
    }
  }
#pragma unroll
  for (int k = 0; k < kPhiRowsK; ++k) {
    if (k < nk) {
      if (S != kF32) f[k][0] += ref[k];
      phi[cell0 + k * geo.plane] =
          f[k][0] + ((f[k][1] + f[k][2]) + (f[k][3] + f[k][4]) + (f[k][5] + f[k][6]));
    }
  }
}

// ------------------------------------------------------------------- k_mu ---------
// k_mu covers the kTX x kTY x kTZ bricks with a three-dimensional grid, or, where there
// are more than 65535 bricks along y or z (the limit of a grid's y and z extents), with
// a one-dimensional grid over the bricks in the same order (x fastest, then y, then z),
// decoded here.  (k_mu_tma takes only grids of the first kind.)
__device__ __forceinline__ void brick_of(int nbx, int nby, int& bx, int& by, int& bz) {
  bx = blockIdx.x;
  by = blockIdx.y;
  bz = blockIdx.z;
  if (gridDim.y == 1 && gridDim.z == 1) {
    const int b = blockIdx.x, r = b / nbx;
    bx = b - r * nbx;
    bz = r / nby;
    by = r - bz * nby;
  }
}

template <bool D3Q7>
__global__ void __launch_bounds__(kTX* kTY) k_mu(const float* __restrict__ phi,
                                                 float* __restrict__ mu, Geometry geo,
                                                 Physics ph) {
  __shared__ float tile[kHZ][kHY][kHX];
  int bx, by, bz;
  brick_of((geo.nx + kTX - 1) / kTX, (geo.ny + kTY - 1) / kTY, bx, by, bz);
  mu_brick<D3Q7>(phi, mu, geo, ph, bx, by, bz, tile);
}

// ------------------------------------------------------------- k_mu_tma ---------
// The same pass with the halo brick fetched by one TMA tensor copy instead of plain
// loads: box kBX x kHY x kHZ of phi starting at (x0 - 4, y0 - 1, z0 - 1), so the
// innermost start coordinate stays a multiple of 4 floats (16 bytes); entries outside
// the grid arrive as zeros and are then replaced, on boundary bricks only, by their
// periodic image or wall ghost with plain loads.  Needs nx % 32 == 0 and ny % 8 == 0
// (whole bricks in x and y).  The wait on the copy's mbarrier is bounded: if it runs
// out (after `polls` polls; kMbarSpins by default), the block waits once more (bounded,
// kMbarSpins polls) for its copy and returns, setting *err to at least 1 if the copy
// landed in that second wait and to 2 if it did not.
constexpr int kBX = kTX + 8;  // 4 columns either side; the stencil uses columns 3 .. 36
constexpr int kMuThreads = kTX * kTY / 2;  // two rows of the brick per thread

// mu of the brick's columns as mu_columns computes them, with each thread taking two
// adjacent rows, i = 2 threadIdx.y + 1 and i + 1 of the halo tile, in paired FP32
// instructions: per plane the two columns' four rows i - 1 .. i + 2 are loaded once
// (12 shared-memory loads instead of 18), the in-plane x-pair sums h of those rows
// serve the face sum of one column and the diagonal sum of the other, and the rest of
// Eqs. 36 and 2 runs once for both cells.  Each lane's operations and their order are
// those of mu_columns, so mu is bitwise the same.
template <bool D3Q7>
__device__ __forceinline__ void mu_columns_pair(const float (*tile)[kHY][kBX],
                                                float* __restrict__ mu, const Geometry& geo,
                                                const Physics& ph, int x0, int y0, int z0) {
  typedef VOps<float2> O;
  const int lane = threadIdx.x, i = 2 * threadIdx.y + 1, j = lane + 4;
  const int x = x0 + lane, y = y0 + i - 1;  // the first row's cell; the second is y + 1
  // the planes' partial sums of the two columns: centres c, face sums f, corner sums d
  auto plane = [&](int l, float2& c, float2& f, float2& d) {
    const float(*t)[kBX] = tile[l];
    const float m0 = t[i - 1][j - 1], p0 = t[i - 1][j + 1], c0 = t[i - 1][j];
    const float m1 = t[i][j - 1], p1 = t[i][j + 1], c1 = t[i][j];
    const float m2 = t[i + 1][j - 1], p2 = t[i + 1][j + 1], c2 = t[i + 1][j];
    const float m3 = t[i + 2][j - 1], p3 = t[i + 2][j + 1], c3 = t[i + 2][j];
    const float2 h12 = O::add(make_float2(m1, m2), make_float2(p1, p2));
    const float2 h03 = O::add(make_float2(m0, m3), make_float2(p0, p3));
    c = make_float2(c1, c2);
    f = O::add(h12, O::add(make_float2(c0, c1), make_float2(c2, c3)));
    d = O::add(make_float2(h03.x, h12.x), make_float2(h12.y, h03.y));
  };
  float2 c0, f0, d0, c1, f1, d1;
  plane(0, c0, f0, d0);
  plane(1, c1, f1, d1);
  const int nl = min(kTZ, geo.nz - z0);
  float* out = mu + (static_cast<size_t>(z0) * geo.ny + y) * geo.nx + x;
  const size_t zstride = static_cast<size_t>(geo.plane);
  const float2 beta4 = O::k(4.0f * ph.beta), mkappa = O::k(-ph.kappa);
  for (int l = 1; l <= nl; ++l) {
    float2 c2, f2, d2;
    plane(l + 1, c2, f2, d2);
    const float2 faces = O::fma(O::k(-6.0f), c1, O::add(f1, O::add(c0, c2)));
    const float2 lap =
        D3Q7 ? faces
             : O::fma(O::k(2.0f / 3.0f), faces,
                      O::mul(O::k(1.0f / 12.0f), O::fma(O::k(-8.0f), c1, O::add(d0, d2))));
    const float2 m = O::fma(O::mul(beta4, c1), O::fma(c1, c1, O::k(-1.0f)), O::mul(mkappa, lap));
    float* o = out + (l - 1) * zstride;
    o[0] = m.x;
    o[geo.nx] = m.y;
    c0 = c1; f0 = f1; d0 = d1;
    c1 = c2; f1 = f2; d1 = d2;
  }
}

constexpr unsigned kMuBoxBytes = kBX * kHY * kHZ * 4;
constexpr long long kMbarSpins = 1 << 22;
static_assert(kMuTmaBox[0] == kBX && kMuTmaBox[1] == kHY && kMuTmaBox[2] == kHZ,
              "TMA box of the host descriptor");

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// true once phase `parity` of the mbarrier has completed; false after `polls` polls
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long long polls) {
  for (long long k = 0; k < polls; ++k) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <bool D3Q7>
__global__ void __launch_bounds__(kMuThreads, 7) k_mu_tma(const __grid_constant__ CUtensorMap map,
                                                     const float* __restrict__ phi,
                                                     float* __restrict__ mu, Geometry geo,
                                                     Physics ph, int* err, long long polls) {
  __shared__ alignas(128) float tile[kHZ][kHY][kBX];
  __shared__ alignas(8) unsigned long long bar_storage;
  const unsigned bar = smem_addr(&bar_storage);
  const int tid = threadIdx.y * kTX + threadIdx.x;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY, z0 = blockIdx.z * kTZ;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"(kMuBoxBytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(&tile[0][0][0])),
        "l"(reinterpret_cast<unsigned long long>(&map)), "r"(x0 - 4), "r"(y0 - 1), "r"(z0 - 1),
        "r"(bar)
        : "memory");
  }
  if (!__syncthreads_and(mbar_wait(bar, 0, polls))) {
    if (tid == 0) {
      // let the copy into this block's shared memory land; if even that bounded wait
      // runs out, the copy may still be writing when the block exits: word 2 tells the
      // host to retire the context (no further launches on it)
      atomicMax(err, mbar_wait(bar, 0, kMbarSpins) ? 1 : 2);
    }
    __syncthreads();
    return;
  }
  // periodic images and wall ghosts of the halo entries outside the grid
  const int nl = min(kTZ, geo.nz - z0);
  const bool xlo = x0 == 0, xhi = x0 + kTX >= geo.nx;
  const bool ylo = y0 == 0, yhi = y0 + kTY >= geo.ny;
  const bool zlo = z0 == 0, zhi = z0 + nl >= geo.nz;
  if (xlo || xhi || ylo || yhi || zlo || zhi) {
    auto fill = [&](int l, int i, int jj) {
      const int gx = wrap(x0 - 4 + jj, geo.nx, kBX);
      const int gy = wrap(y0 - 1 + i, geo.ny, kHY);
      const int gz = ghost_z(geo, z0 - 1 + l);
      tile[l][i][jj] = __ldg(phi + (static_cast<size_t>(gz) * geo.ny + gy) * geo.nx + gx);
    };
    const int nthreads = kMuThreads;
    // x faces: columns 3 and kTX + 4 of every row and plane
    for (int k = tid; k < 2 * kHZ * kHY; k += nthreads) {
      const int side = k / (kHZ * kHY), r = k - side * kHZ * kHY;
      if (side == 0 ? xlo : xhi) fill(r / kHY, r % kHY, side == 0 ? 3 : kTX + 4);
    }
    // y faces: rows 0 and kTY + 1, columns 3 .. kTX + 4, every plane
    for (int k = tid; k < 2 * kHZ * (kTX + 2); k += nthreads) {
      const int side = k / (kHZ * (kTX + 2)), r = k - side * kHZ * (kTX + 2);
      if (side == 0 ? ylo : yhi) fill(r / (kTX + 2), side == 0 ? 0 : kTY + 1, 3 + r % (kTX + 2));
    }
    // z faces: planes 0 and nl + 1, rows 0 .. kTY + 1, columns 3 .. kTX + 4
    for (int k = tid; k < 2 * kHY * (kTX + 2); k += nthreads) {
      const int side = k / (kHY * (kTX + 2)), r = k - side * kHY * (kTX + 2);
      if (side == 0 ? zlo : zhi) fill(side == 0 ? 0 : nl + 1, r / (kTX + 2), 3 + r % (kTX + 2));
    }
    __syncthreads();
  }
  mu_columns_pair<D3Q7>(tile, mu, geo, ph, x0, y0, z0);
}

// -------------------------------------------------------------- k_collide ---------

template <int P, int VAR, int S>
__global__ void __launch_bounds__(kBlock, collide_min_blocks<S>())
    k_collide(const float* src, float* dst, const float* __restrict__ phi,
              const float* __restrict__ mu, Geometry geo, Physics ph, int have_prev) {
  prefetch_ahead<S, true>(src, phi, mu, geo, geo.prefetch_collide);
  const int idx = blockIdx.x * kBlock + threadIdx.x;
  if (idx >= geo.n) return;
  collide_cell<P, VAR, S>(src, dst, phi, mu, geo, ph, have_prev, idx);
}

// k_collide with two cells per thread (collide_pair, the arithmetic in paired FP32
// instructions): block b takes cells 256 b .. 256 b + 255 as 4 pairs of adjacent tiles of
// one row; lane l of warp w the cells 256 b + 64 w + l and 256 b + 64 w + 32 + l.  Pattern
// P (two arrays, or either step of the in-place pattern) on grids with Geometry::pairs (n
// is then a multiple of 64, so a warp is wholly inside or outside the grid).  With SUMS
// each warp leaves the sums of its two tiles in parts, as k_collide_sums.
// 4 resident blocks of 128 threads (128 registers, no spills); at 5 the 16-bit kernels
// spill and run 17 % slower.
template <int S>
constexpr int collide2_min_blocks() {
  return 4;
}

template <int VAR, int S, bool SUMS, int P = kAB>
__global__ void __launch_bounds__(kBlock / 2, collide2_min_blocks<S>())
    k_collide2(const float* src, float* dst, const float* __restrict__ phi,
               const float* __restrict__ mu, Geometry geo, Physics ph, int have_prev,
               float* __restrict__ parts) {
  prefetch_ahead<S, true>(src, phi, mu, geo, geo.prefetch_collide);
  const int idx = blockIdx.x * kBlock + (threadIdx.x >> 5) * (2 * kTile) + (threadIdx.x & 31);
  if (idx >= geo.n) return;
  if (SUMS) {
    float s[8];
    collide_pair<VAR, S, true, P>(src, dst, phi, mu, geo, ph, have_prev, idx, s);
    const bool bad0 = !(isfinite(s[0]) && isfinite(s[1]) && isfinite(s[2]) && isfinite(s[3]));
    const bool bad1 = !(isfinite(s[4]) && isfinite(s[5]) && isfinite(s[6]) && isfinite(s[7]));
    warp_sums_store(s, bad0, parts, idx & ~31);
    warp_sums_store(s + 4, bad1, parts, (idx + kTile) & ~31);
  } else {
    collide_pair<VAR, S, false, P>(src, dst, phi, mu, geo, ph, have_prev, idx, nullptr);
  }
}

// k_collide2 with the phi and mu stencils staged in shared memory by TMA bulk copies
// (grids whose rows are 64, 128 or 256 cells: a block's 256 cells are R = 256 / nx whole
// rows).  For each of its rows and each of the 9 (dy, dz) neighbour rows the stencils
// use (walls: the ghost of a row beyond the wall is the row itself), thread 0 issues one
// `cp.async.bulk` of the whole row of phi and one of mu into shared memory (at most 72
// copies of nx floats, completing on one mbarrier), while every thread loads its two
// cells' populations; after the (bounded) wait the two x-halo values of each row are
// filled from the row itself (periodic x) and the cells read their 15-point stencils
// from shared memory: no stencil load instructions and no stencil registers in flight.
// The values are those load_stencil reads, so the state is bit-identical to k_collide2.
// A block whose wait runs out waits once more (bounded), sets *err as k_mu_tma does,
// and returns without touching the state.  With SUMS each warp leaves the sums of its
// two tiles in parts, as k_collide2.
constexpr int kStRowPad = 8;                            // floats: 4 before, 4 after a row
constexpr int kStFloats = 9 * 4 * (64 + kStRowPad);    // per field, max over nx = 64..256

__device__ __forceinline__ void bulk_row(unsigned dst, const float* src, unsigned bytes,
                                         unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

template <int VAR, int S, bool SUMS, int P = kAB>
__global__ void __launch_bounds__(kBlock / 2, collide2_min_blocks<S>())
    k_collide2t(const float* src, float* dst, const float* __restrict__ phi,
                const float* __restrict__ mu, Geometry geo, Physics ph, int have_prev, int* err,
                long long polls, float* __restrict__ parts) {
  __shared__ alignas(128) float st[2][kStFloats];
  __shared__ alignas(8) unsigned long long bar_storage;
  prefetch_ahead<S, true>(src, phi, mu, geo, geo.prefetch_collide);
  const unsigned bar = smem_addr(&bar_storage);
  const int nx = geo.nx, R = kBlock / nx, stride = nx + kStRowPad;
  const int b0 = blockIdx.x * kBlock;
  const int rows = min(R, (geo.n - b0) / nx);  // whole rows of this block
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const unsigned row_bytes = static_cast<unsigned>(nx) * 4u;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"(2u * 9u * static_cast<unsigned>(rows) * row_bytes)
                 : "memory");
    for (int r = 0; r < rows; ++r) {
      const int gr = b0 / nx + r;  // global row index: y + ny z
      const int z = gr / geo.ny, y = gr - z * geo.ny;
      for (int k = 0; k < 9; ++k) {
        const int dy = k % 3 - 1, dz = k / 3 - 1;
        const int yy = y + dy < 0 ? geo.ny - 1 : (y + dy >= geo.ny ? 0 : y + dy);
        int zz = z + dz;
        if (geo.walls)
          zz = (zz < 0 || zz >= geo.nz) ? z : zz;
        else
          zz = zz < 0 ? geo.nz - 1 : (zz >= geo.nz ? 0 : zz);
        const size_t row0 = (static_cast<size_t>(zz) * geo.ny + yy) * nx;
        const int off = (r * 9 + k) * stride + 4;
        bulk_row(smem_addr(&st[0][off]), phi + row0, row_bytes, bar);
        bulk_row(smem_addr(&st[1][off]), mu + row0, row_bytes, bar);
      }
    }
  }
  // the populations of the two cells, loaded while the copies fly
  const int idx = b0 + (threadIdx.x >> 5) * (2 * kTile) + (threadIdx.x & 31);
  const bool active = idx < geo.n;
  int x = 0, y = 0, z = 0;
  if (active) cell_coords(geo, idx, x, y, z);
  const Nbr na = make_nbr(geo, x, y, z), nb2 = make_nbr(geo, x + kTile, y, z);
  float ga[15], fa[7], pa[3], gb[15], fb[7], pb[3];
  if (active) {
    load_cell<P, S, true>(src, geo, idx, na, ga, fa, pa);
    load_cell<P, S, true>(src, geo, idx + kTile, nb2, gb, fb, pb);
  }
  __syncthreads();  // the barrier is initialised and armed before anyone polls it
  if (!__syncthreads_and(mbar_wait(bar, 0, polls))) {
    if (threadIdx.x == 0) atomicMax(err, mbar_wait(bar, 0, kMbarSpins) ? 1 : 2);
    __syncthreads();
    return;
  }
  // periodic x halo of every row copy: column -1 = nx - 1, column nx = 0
  for (int k = threadIdx.x; k < 2 * 9 * rows * 2; k += blockDim.x) {
    const int side = k & 1, rk = (k >> 1) % (9 * rows), f = (k >> 1) / (9 * rows);
    float* row = &st[f][rk * stride + 4];
    if (side)
      row[nx] = row[0];
    else
      row[-1] = row[nx - 1];
  }
  __syncthreads();
  // with SUMS every lane of a warp takes part in the warp sums; a warp is wholly inside
  // or outside the grid (n is a multiple of 64)
  if (!active) return;
  // stencil of the cell at x in block row r from the staged rows (k = 3 (dz + 1) + dy + 1)
  const int r = (idx - b0) / nx;
  auto stencil = [&](const float* a, int xc) {
    const float* base = a + r * 9 * stride + 4 + xc;
    auto row = [&](int dy, int dz) { return base + (3 * (dz + 1) + dy + 1) * stride; };
    Stencil s;
    s.c = row(0, 0)[0];
    s.xm = row(0, 0)[-1];
    s.xp = row(0, 0)[1];
    s.ym = row(-1, 0)[0];
    s.yp = row(1, 0)[0];
    s.zm = row(0, -1)[0];
    s.zp = row(0, 1)[0];
#pragma unroll
    for (int b = 0; b < 8; ++b)
      s.k[b] = row((b & 2) ? 1 : -1, (b & 4) ? 1 : -1)[(b & 1) ? 1 : -1];
    return s;
  };
  StencilV<float2> sp, sm;
  {
    const Stencil s0 = stencil(st[0], x), s1 = stencil(st[0], x + kTile);
    sp.c = make_float2(s0.c, s1.c);
    sp.xm = make_float2(s0.xm, s1.xm);
    sp.xp = make_float2(s0.xp, s1.xp);
    sp.ym = make_float2(s0.ym, s1.ym);
    sp.yp = make_float2(s0.yp, s1.yp);
    sp.zm = make_float2(s0.zm, s1.zm);
    sp.zp = make_float2(s0.zp, s1.zp);
#pragma unroll
    for (int b = 0; b < 8; ++b) sp.k[b] = make_float2(s0.k[b], s1.k[b]);
  }
  {
    const Stencil s0 = stencil(st[1], x), s1 = stencil(st[1], x + kTile);
    sm.c = make_float2(s0.c, s1.c);
    sm.xm = make_float2(s0.xm, s1.xm);
    sm.xp = make_float2(s0.xp, s1.xp);
    sm.ym = make_float2(s0.ym, s1.ym);
    sm.yp = make_float2(s0.yp, s1.yp);
    sm.zm = make_float2(s0.zm, s1.zm);
    sm.zp = make_float2(s0.zp, s1.zp);
#pragma unroll
    for (int b = 0; b < 8; ++b) sm.k[b] = make_float2(s0.k[b], s1.k[b]);
  }
  float2 g[15], f[7], prev[3], cur[3];
#pragma unroll
  for (int i = 0; i < 15; ++i) g[i] = make_float2(ga[i], gb[i]);
#pragma unroll
  for (int i = 0; i < 7; ++i) f[i] = make_float2(fa[i], fb[i]);
#pragma unroll
  for (int a = 0; a < 3; ++a) prev[a] = make_float2(pa[a], pb[a]);
  pair_compute<VAR, S>(ph, have_prev, g, f, prev, sp, sm, cur);
  if (SUMS) {
    float s4[8];
    pair_sums<S>(g, f, sp.c, na, 0, s4);
    pair_sums<S>(g, f, sp.c, nb2, 1, s4 + 4);
    const bool bad0 = !(isfinite(s4[0]) && isfinite(s4[1]) && isfinite(s4[2]) && isfinite(s4[3]));
    const bool bad1 = !(isfinite(s4[4]) && isfinite(s4[5]) && isfinite(s4[6]) && isfinite(s4[7]));
    warp_sums_store(s4, bad0, parts, idx & ~31);
    warp_sums_store(s4 + 4, bad1, parts, (idx + kTile) & ~31);
  }
  store_pair<P, S>(dst, geo, idx, na, nb2, g, f, cur);
}

// Fused stream-collide that also sums the state it writes (collide_cell with SUMS):
// each warp leaves 5 floats in parts[5 w ..] (w = its first cell / 32; warp_sums_store).
// The 32 cells of a warp are summed in FP32 by a fixed butterfly (FP64 throughput on
// this GPU is a small fraction of FP32, and no block barrier holds finished warps back);
// everything above in FP64, in a fixed order.
template <int P, int S>
__global__ void __launch_bounds__(kBlock, collide_min_blocks<S>())
    k_collide_sums(const float* src, float* dst, const float* __restrict__ phi,
                   const float* __restrict__ mu, Geometry geo, Physics ph, int have_prev,
                   float* __restrict__ parts) {
  prefetch_ahead<S, true>(src, phi, mu, geo, geo.prefetch_collide);
  const int idx = blockIdx.x * kBlock + threadIdx.x;
  if ((idx & ~31) >= geo.n) return;  // the whole warp lies beyond the grid
  float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  bool bad = false;
  if (idx < geo.n) {
    collide_cell<P, 0, S, true>(src, dst, phi, mu, geo, ph, have_prev, idx, s);
    bad = !(isfinite(s[0]) && isfinite(s[1]) && isfinite(s[2]) && isfinite(s[3]));
  }
  warp_sums_store(s, bad, parts, idx & ~31);
}

// ------------------------------------------------------------------ k_che ---------
// Interface tracking with a prescribed velocity (Sec. III A, B): only the D3Q7 lattice
// evolves (Eq. 4); u is analytic, so the flow lattice and the stencils of phi and mu
// are not needed.  tf is the time factor of the velocity field at this step.
template <int P, int S>
__global__ void __launch_bounds__(kBlock) k_che(const float* src, float* dst,
                                                const float* __restrict__ phi,
                                                const float* __restrict__ mu, Geometry geo,
                                                Physics ph, int have_prev, float tf) {
  const int idx = blockIdx.x * kBlock + threadIdx.x;
  if (idx >= geo.n) return;
  int x, y, z;
  cell_coords(geo, idx, x, y, z);
  const Nbr nb = make_nbr(geo, x, y, z);
  float f[7], prev[3];
  load_f<P, S>(src, idx, nb, f);
#pragma unroll
  for (int a = 0; a < 3; ++a) prev[a] = src[phiu_index<S>(idx, a)];
  const float phi_c = __ldg(phi + idx), mu_c = __ldg(mu + idx);
  float u[3];
  prescribed_velocity(ph, geo, x, y, z, tf, u);
  float dphiu[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float cur = __fmul_rn(phi_c, u[a]);
    dphiu[a] = have_prev ? __fsub_rn(cur, prev[a]) : 0.0f;
    dst[phiu_index<S>(idx, a)] = cur;
  }
  collide_d3q7<S != kF32>(ph, f, phi_c, mu_c, u, dphiu);
  store_f<P, S>(dst, idx, nb, f);
}

// --------------------------------------------------------------- k_fields ---------
// rho, p, u of the current populations into out[0..4] (rho, p, ux, uy, uz).
template <int P, int S>
__global__ void __launch_bounds__(kBlock) k_fields(const float* __restrict__ src,
                                                   const float* __restrict__ phi,
                                                   const float* __restrict__ mu,
                                                   float* __restrict__ out, Geometry geo,
                                                   Physics ph, float tf) {
  const int idx = blockIdx.x * kBlock + threadIdx.x;
  if (idx >= geo.n) return;
  int x, y, z;
  cell_coords(geo, idx, x, y, z);
  const size_t s = geo.stride;
  if (ph.vel_kind != kVelNone) {  // tracking mode: prescribed u, no pressure
    float u[3];
    prescribed_velocity(ph, geo, x, y, z, tf, u);
    out[0 * s + idx] = ph.rho_g + (1.0f + __ldg(phi + idx)) * ph.half_drho;
    out[1 * s + idx] = 0.0f;
    out[2 * s + idx] = u[0];
    out[3 * s + idx] = u[1];
    out[4 * s + idx] = u[2];
    return;
  }
  const Nbr nb = make_nbr(geo, x, y, z);
  const CellStencils cs = ph.d3q7_stencil ? cell_stencils<true>(phi, mu, idx, nb)
                                          : cell_stencils<false>(phi, mu, idx, nb);
  float g[15];
  load_g<P, S>(src, idx, nb, g);
  const Macro M = macroscopic(ph, moments15(g), cs.phi, cs.mu, cs.grad_phi, cs.lap_mu);
  out[0 * s + idx] = M.rho;
  out[1 * s + idx] = M.p;
  out[2 * s + idx] = M.u[0];
  out[3 * s + idx] = M.u[1];
  out[4 * s + idx] = M.u[2];
}

// ------------------------------------------------------------------ k_init --------
// Pre-collision populations f = f^eq (Eq. 5), g = g^eq (Eq. 21) placed for a step of
// pattern P; phi u stored in the own tile.  u0 (3 dense planes) and p0 may be null.
template <int P, int S>
__global__ void __launch_bounds__(kBlock) k_init(float* state, const float* __restrict__ phi,
                                                 const float* __restrict__ mu,
                                                 const float* __restrict__ u0,
                                                 const float* __restrict__ p0, Geometry geo,
                                                 Physics ph, float tf) {
  const int idx = blockIdx.x * kBlock + threadIdx.x;
  if (idx >= geo.n) return;
  int x, y, z;
  cell_coords(geo, idx, x, y, z);
  const Nbr nb = make_nbr(geo, x, y, z);
  const size_t s = geo.stride;
  const float ph_ = phi[idx], mu_ = mu[idx];
  float u[3] = {0.0f, 0.0f, 0.0f};
  if (ph.vel_kind != kVelNone) {
    prescribed_velocity(ph, geo, x, y, z, tf, u);
  } else if (u0) {
    u[0] = u0[idx];
    u[1] = u0[s + idx];
    u[2] = u0[2 * s + idx];
  }
  const float p = p0 ? p0[idx] : 0.0f;
  const float rho = ph.rho_g + (1.0f + ph_) * ph.half_drho;

  // D3Q7: omega_0 = 1 - 3A, omega_i = A/2, c_s^2 = A
  const float emu = ph.eta * mu_;
  const float hw = 0.5f * ph.A * emu;
  const float jx = 0.5f * ph_ * u[0], jy = 0.5f * ph_ * u[1], jz = 0.5f * ph_ * u[2];
  // 16-bit storage keeps f_0 - phi in slot 0
  const float f0 = S != kF32 ? -3.0f * ph.A * emu : ph_ - 3.0f * ph.A * emu;
  const float f[7] = {f0, hw + jx, hw - jx, hw + jy, hw - jy, hw + jz, hw - jz};
  place_f<P, S>(state, idx, nb, f);

  // D3Q15: g_i = 3 p omega_i + rho omega_i (3 c.u + 9/2 (c.u)^2 - 3/2 u^2), g_0 -= 3p
  const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  constexpr int cx[15] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
  constexpr int cy[15] = {0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, -1, 1, -1, 1};
  constexpr int cz[15] = {0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1, -1, 1};
  float g[15];
#pragma unroll
  for (int i = 0; i < 15; ++i) {
    const float w = i == 0 ? 2.0f / 9.0f : (i < 7 ? 1.0f / 9.0f : 1.0f / 72.0f);
    const float cu = cx[i] * u[0] + cy[i] * u[1] + cz[i] * u[2];
    g[i] = 3.0f * p * w + rho * w * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu);
  }
  g[0] -= 3.0f * p;
  place_g<P, S>(state, idx, nb, g);
  state[phiu_index<S>(idx, 0)] = ph_ * u[0];
  state[phiu_index<S>(idx, 1)] = ph_ * u[1];
  state[phiu_index<S>(idx, 2)] = ph_ * u[2];
}

// -------------------------------------------------- state gather / scatter --------
// Slot `slot` of cell idx of the current pre-collision state: populations through the
// pattern's addressing, phi u (slots 22..24) from the own tile; with 16-bit storage the
// reference phi added back to slot 0.
template <int P, int S>
__device__ __forceinline__ float state_value(const float* __restrict__ src,
                                             const float* __restrict__ phi_ref,
                                             const Geometry& geo, int idx, int slot) {
  int x, y, z;
  cell_coords(geo, idx, x, y, z);
  const Nbr nb = make_nbr(geo, x, y, z);
  float v = 0.0f;
  switch (slot) {
#define X(I, O, CX, CY, CZ) \
  case I:                   \
    v = pop_load<S, P, I, O, CX, CY, CZ>(src, idx, nb); \
    break;
    LBM_D3Q7_LIST(X)
#undef X
#define X(I, O, CX, CY, CZ) \
  case 7 + I:               \
    v = pop_load<S, P, 7 + I, 7 + O, CX, CY, CZ>(src, idx, nb); \
    break;
    LBM_D3Q15_LIST(X)
#undef X
    default:
      v = src[phiu_index<S>(idx, slot - kSlotPhiu)];
  }
  if (S != kF32 && slot == 0) v += phi_ref[idx];
  return v;
}

// Slot `slot` of every cell to dense[idx].
template <int P, int S>
__global__ void __launch_bounds__(kBlock) k_gather(const float* __restrict__ src,
                                                   const float* __restrict__ phi_ref,
                                                   float* __restrict__ dense, Geometry geo,
                                                   int slot) {
  const int idx = blockIdx.x * kBlock + threadIdx.x;
  if (idx >= geo.n) return;
  dense[idx] = state_value<P, S>(src, phi_ref, geo, idx, slot);
}

// All kTileSlots slots of `count` listed cells (indices checked against geo.n by the
// caller): out[q * count + k] = slot q of cell cells[k].
template <int P, int S>
__global__ void __launch_bounds__(kBlock) k_gather_at(const float* __restrict__ src,
                                                      const float* __restrict__ phi_ref,
                                                      const long long* __restrict__ cells,
                                                      long long count, float* __restrict__ out,
                                                      Geometry geo) {
  const long long items = count * kTileSlots;
  const long long stride = static_cast<long long>(gridDim.x) * kBlock;
  for (long long i = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x; i < items;
       i += stride) {
    const int q = static_cast<int>(i / count);
    const long long k = i - q * count;
    out[i] = state_value<P, S>(src, phi_ref, geo, static_cast<int>(cells[k]), q);
  }
}

// dense[idx] = pre-collision value of slot `slot` of cell idx, placed where a step of
// pattern P reads it (the inverse of k_gather).
// (With 16-bit storage the caller writes f_0 into the order-parameter array and
// scatters zeros into slot 0.)
template <int P, int S>
__global__ void __launch_bounds__(kBlock) k_scatter(float* state, const float* __restrict__ dense,
                                                    Geometry geo, int slot) {
  const int idx = blockIdx.x * kBlock + threadIdx.x;
  if (idx >= geo.n) return;
  int x, y, z;
  cell_coords(geo, idx, x, y, z);
  const Nbr nb = make_nbr(geo, x, y, z);
  const float v = dense[idx];
  switch (slot) {
#define X(I, O, CX, CY, CZ) \
  case I:                   \
    pop_place<S, P, I, O, CX, CY, CZ>(state, idx, nb, v); \
    break;
    LBM_D3Q7_LIST(X)
#undef X
#define X(I, O, CX, CY, CZ) \
  case 7 + I:               \
    pop_place<S, P, 7 + I, 7 + O, CX, CY, CZ>(state, idx, nb, v); \
    break;
    LBM_D3Q15_LIST(X)
#undef X
    default:
      state[phiu_index<S>(idx, slot - kSlotPhiu)] = v;
  }
}

__global__ void __launch_bounds__(kBlock) k_convert(const double* __restrict__ in,
                                                    float* __restrict__ out, int n) {
  const int idx = blockIdx.x * kBlock + threadIdx.x;
  if (idx < n) out[idx] = static_cast<float>(in[idx]);
}

__global__ void __launch_bounds__(kBlock) k_widen(const float* __restrict__ in,
                                                  double* __restrict__ out, int n) {
  const int idx = blockIdx.x * kBlock + threadIdx.x;
  if (idx < n) out[idx] = static_cast<double>(in[idx]);
}

// --------------------------------------------------------------- k_reduce ---------
// Pass 1: block b sums cells b*256 + t, then strides by the grid, in FP64 (fixed
// order: grid-stride rows, then a fixed shuffle tree).
// partial[b] = {sum phi, jx, jy, jz, non-finite count}.
// with_g = 0 (tracking mode, no flow lattice): the momentum sums are zero.
template <int P, int S>
__global__ void __launch_bounds__(kBlock) k_reduce_partial(const float* __restrict__ src,
                                                           const float* __restrict__ phi,
                                                           double* __restrict__ partial,
                                                           Geometry geo, int with_g) {
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  // 64-bit loop index: geo.n < 2^31, but the last stride (up to kReduceMaxParts blocks)
  // could pass INT_MAX; idx itself is < geo.n inside the loop.
  const long long stride = static_cast<long long>(gridDim.x) * kBlock;
  for (long long i = static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x; i < geo.n; i += stride) {
    const int idx = static_cast<int>(i);
    float jx = 0.0f, jy = 0.0f, jz = 0.0f;
    if (with_g) {
      int x, y, z;
      cell_coords(geo, idx, x, y, z);
      const Nbr nb = make_nbr(geo, x, y, z);
      float g[15];
      load_g<P, S>(src, idx, nb, g);
      const float d7 = g[7] - g[8], d9 = g[9] - g[10], d11 = g[11] - g[12], d13 = g[13] - g[14];
      jx = (g[1] - g[2]) + ((d7 + d9) + (d11 + d13));
      jy = (g[3] - g[4]) + ((d7 + d9) - (d11 + d13));
      jz = (g[5] - g[6]) + ((d7 - d9) + (d11 - d13));
    }
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

// Block b sums parts [b chunk, (b + 1) chunk) (5 floats each) in FP64, in a fixed order.
__global__ void __launch_bounds__(kBlock) k_reduce_chunks(const float* __restrict__ parts,
                                                          int nparts, int chunk,
                                                          double* __restrict__ out) {
  __shared__ double sh[kBlock];
  const int b0 = blockIdx.x * chunk;
  const int b1 = min(nparts, b0 + chunk);
  for (int k = 0; k < 5; ++k) {
    double v = 0.0;
    for (int b = b0 + threadIdx.x; b < b1; b += kBlock) v += parts[b * 5 + k];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x * 5 + k] = sh[0];
    __syncthreads();
  }
}

// Blocks of kBlock threads covering n cells; 64-bit so that n + kBlock - 1 cannot wrap
// for n up to 2^31 - 1.
inline unsigned blocks_for(long long n) { return static_cast<unsigned>((n + kBlock - 1) / kBlock); }

// Host-side dispatch of a kernel template over the pattern (FP32 storage) or the
// 16-bit storage types (pattern AB only).
#define LBM_DISPATCH_P(pattern, KERNEL, S, ...)                        \
  {                                                                    \
    if ((pattern) == kAB)                                              \
      KERNEL<kAB, S><<<blocks_, kBlock, 0, st>>>(__VA_ARGS__);         \
    else if ((pattern) == kAAEven)                                     \
      KERNEL<kAAEven, S><<<blocks_, kBlock, 0, st>>>(__VA_ARGS__);     \
    else                                                               \
      KERNEL<kAAOdd, S><<<blocks_, kBlock, 0, st>>>(__VA_ARGS__);      \
  }

#define LBM_DISPATCH(geo, pattern, KERNEL, ...)                        \
  do {                                                                 \
    const unsigned blocks_ = blocks_for((geo).n);                      \
    if ((geo).storage == kF16)                                         \
      LBM_DISPATCH_P(pattern, KERNEL, kF16, __VA_ARGS__)               \
    else if ((geo).storage == kBF16)                                   \
      LBM_DISPATCH_P(pattern, KERNEL, kBF16, __VA_ARGS__)              \
    else                                                               \
      LBM_DISPATCH_P(pattern, KERNEL, kF32, __VA_ARGS__)               \
  } while (0)

}  // namespace

// ------------------------------------------------------------ host launchers ------
cudaError_t launch_phi(const float* src, const float* phi_ref, float* phi, const Geometry& geo,
                       int pattern, cudaStream_t st) {
  const int tp = geo.plane / kTile;
  const int chunks = (geo.nz + kPhiRowsK - 1) / kPhiRowsK;
  if (geo.row_tiles > 0 && chunks <= 65535) {
    const dim3 grid((tp + kBlock / kTile - 1) / (kBlock / kTile), chunks);
    const int ahead = geo.prefetch_phi > 0
                          ? static_cast<int>((geo.prefetch_phi + grid.x - 1) / grid.x)
                          : 0;
#define LBM_PHI_ROWS(S)                                                                   \
  if (pattern == kAAEven)                                                                 \
    k_phi_rows<S, kAAEven><<<grid, kBlock, 0, st>>>(src, phi_ref, phi, geo, ahead);       \
  else if (pattern == kAAOdd)                                                             \
    k_phi_rows<S, kAAOdd><<<grid, kBlock, 0, st>>>(src, phi_ref, phi, geo, ahead);        \
  else                                                                                    \
    k_phi_rows<S, kAB><<<grid, kBlock, 0, st>>>(src, phi_ref, phi, geo, ahead);
    if (geo.storage == kF16) {
      LBM_PHI_ROWS(kF16)
    } else if (geo.storage == kBF16) {
      LBM_PHI_ROWS(kBF16)
    } else {
      LBM_PHI_ROWS(kF32)
    }
#undef LBM_PHI_ROWS
    return cudaGetLastError();
  }
  LBM_DISPATCH(geo, pattern, k_phi, src, phi_ref, phi, geo);
  return cudaGetLastError();
}

long long mu_tma_default_polls() { return kMbarSpins; }

// Grid of the k_mu launch over nbx x nby x nbz bricks (brick_of).
static dim3 brick_grid(int nbx, int nby, int nbz) {
  if (nby <= 65535 && nbz <= 65535) return dim3(nbx, nby, nbz);
  return dim3(static_cast<unsigned>(static_cast<long long>(nbx) * nby * nbz));
}

cudaError_t launch_mu_tma(const CUtensorMap& map, const float* phi, float* mu,
                          const Geometry& geo, const Physics& ph, int* err, long long polls,
                          cudaStream_t st) {
  const dim3 grid(geo.nx / kTX, geo.ny / kTY, (geo.nz + kTZ - 1) / kTZ);
  if (ph.d3q7_stencil)
    k_mu_tma<true><<<grid, dim3(kTX, kTY / 2), 0, st>>>(map, phi, mu, geo, ph, err, polls);
  else
    k_mu_tma<false><<<grid, dim3(kTX, kTY / 2), 0, st>>>(map, phi, mu, geo, ph, err, polls);
  return cudaGetLastError();
}

// Whole bricks in x and y, and a three-dimensional grid of them (at most 65535 bricks
// along y and z); other grids take k_mu.
bool mu_tma_shape_ok(const Geometry& geo) {
  return geo.nx % kTX == 0 && geo.ny % kTY == 0 && geo.ny / kTY <= 65535 &&
         (geo.nz + kTZ - 1) / kTZ <= 65535;
}

cudaError_t launch_mu(const float* phi, float* mu, const Geometry& geo, const Physics& ph,
                      cudaStream_t st) {
  const dim3 grid = brick_grid((geo.nx + kTX - 1) / kTX, (geo.ny + kTY - 1) / kTY,
                               (geo.nz + kTZ - 1) / kTZ);
  if (ph.d3q7_stencil)
    k_mu<true><<<grid, dim3(kTX, kTY), 0, st>>>(phi, mu, geo, ph);
  else
    k_mu<false><<<grid, dim3(kTX, kTY), 0, st>>>(phi, mu, geo, ph);
  return cudaGetLastError();
}

template <int VAR>
void collide_variant(const float* src, float* dst, const float* phi, const float* mu,
                     const Geometry& geo, const Physics& ph, int pattern, int prev, int* err,
                     long long polls, cudaStream_t st) {
  const unsigned blocks = blocks_for(geo.n);
#define LBM_COLLIDE_P(S)                                                                    \
  {                                                                                         \
    if (pattern == kAB && geo.pairs && geo.stage && err)                                    \
      k_collide2t<VAR, S, false><<<blocks, kBlock / 2, 0, st>>>(src, dst, phi, mu, geo, ph,   \
                                                               prev, err, polls, nullptr);  \
    else if (pattern == kAAEven && geo.pairs && geo.stage && err)                           \
      k_collide2t<VAR, S, false, kAAEven><<<blocks, kBlock / 2, 0, st>>>(                   \
          src, dst, phi, mu, geo, ph, prev, err, polls, nullptr);                           \
    else if (pattern == kAAOdd && geo.pairs && geo.stage && err)                            \
      k_collide2t<VAR, S, false, kAAOdd><<<blocks, kBlock / 2, 0, st>>>(                    \
          src, dst, phi, mu, geo, ph, prev, err, polls, nullptr);                           \
    else if (pattern == kAB && geo.pairs)                                                   \
      k_collide2<VAR, S, false><<<blocks, kBlock / 2, 0, st>>>(src, dst, phi, mu, geo, ph,     \
                                                               prev, nullptr);              \
    else if (pattern == kAB)                                                                \
      k_collide<kAB, VAR, S><<<blocks, kBlock, 0, st>>>(src, dst, phi, mu, geo, ph, prev);     \
    else if (pattern == kAAEven && geo.pairs)                                               \
      k_collide2<VAR, S, false, kAAEven><<<blocks, kBlock / 2, 0, st>>>(                    \
          src, dst, phi, mu, geo, ph, prev, nullptr);                                       \
    else if (pattern == kAAOdd && geo.pairs)                                                \
      k_collide2<VAR, S, false, kAAOdd><<<blocks, kBlock / 2, 0, st>>>(                     \
          src, dst, phi, mu, geo, ph, prev, nullptr);                                       \
    else if (pattern == kAAEven)                                                            \
      k_collide<kAAEven, VAR, S><<<blocks, kBlock, 0, st>>>(src, dst, phi, mu, geo, ph, prev); \
    else                                                                                    \
      k_collide<kAAOdd, VAR, S><<<blocks, kBlock, 0, st>>>(src, dst, phi, mu, geo, ph, prev);  \
  }
  if (geo.storage == kF16)
    LBM_COLLIDE_P(kF16)
  else if (geo.storage == kBF16)
    LBM_COLLIDE_P(kBF16)
  else
    LBM_COLLIDE_P(kF32)
#undef LBM_COLLIDE_P
}

cudaError_t launch_collide(const float* src, float* dst, const float* phi, const float* mu,
                           const Geometry& geo, const Physics& ph, int pattern, bool have_prev,
                           cudaStream_t st, int* err, long long polls) {
  const int prev = have_prev ? 1 : 0;
  const int var = (ph.srt_flow ? kVarSrtFlow : 0) | (ph.d3q7_stencil ? kVarD3Q7 : 0);
  switch (var) {
    case 0: collide_variant<0>(src, dst, phi, mu, geo, ph, pattern, prev, err, polls, st); break;
    case kVarSrtFlow:
      collide_variant<kVarSrtFlow>(src, dst, phi, mu, geo, ph, pattern, prev, err, polls, st);
      break;
    case kVarD3Q7:
      collide_variant<kVarD3Q7>(src, dst, phi, mu, geo, ph, pattern, prev, err, polls, st);
      break;
    default:
      collide_variant<kVarSrtFlow | kVarD3Q7>(src, dst, phi, mu, geo, ph, pattern, prev, err,
                                              polls, st);
  }
  return cudaGetLastError();
}

bool stage_shape_ok(const Geometry& geo) {
  return geo.nx == 64 || geo.nx == 128 || geo.nx == 256;
}

int cell_warps(long long n) { return static_cast<int>((n + 31) / 32); }

cudaError_t launch_collide_sums(const float* src, float* dst, const float* phi, const float* mu,
                                const Geometry& geo, const Physics& ph, int pattern,
                                bool have_prev, float* parts, double* partial, double* out,
                                cudaStream_t st, int* err, long long polls) {
  const int prev = have_prev ? 1 : 0;
  if (pattern == kAB && geo.pairs && geo.stage && err) {
    const unsigned blocks = blocks_for(geo.n);
    if (geo.storage == kF16)
      k_collide2t<0, kF16, true><<<blocks, kBlock / 2, 0, st>>>(src, dst, phi, mu, geo, ph, prev, err, polls, parts);
    else if (geo.storage == kBF16)
      k_collide2t<0, kBF16, true><<<blocks, kBlock / 2, 0, st>>>(src, dst, phi, mu, geo, ph, prev, err, polls, parts);
    else
      k_collide2t<0, kF32, true><<<blocks, kBlock / 2, 0, st>>>(src, dst, phi, mu, geo, ph, prev, err, polls, parts);
  } else if (pattern == kAB && geo.pairs) {
    const unsigned blocks = blocks_for(geo.n);
    if (geo.storage == kF16)
      k_collide2<0, kF16, true><<<blocks, kBlock / 2, 0, st>>>(src, dst, phi, mu, geo, ph, prev, parts);
    else if (geo.storage == kBF16)
      k_collide2<0, kBF16, true><<<blocks, kBlock / 2, 0, st>>>(src, dst, phi, mu, geo, ph, prev, parts);
    else
      k_collide2<0, kF32, true><<<blocks, kBlock / 2, 0, st>>>(src, dst, phi, mu, geo, ph, prev, parts);
  } else if ((pattern == kAAEven || pattern == kAAOdd) && geo.pairs) {
    const unsigned blocks = blocks_for(geo.n);
    const bool staged = geo.stage && err;
#define LBM_SUMS_AA(S)                                                                        \
  if (pattern == kAAEven && staged)                                                           \
    k_collide2t<0, S, true, kAAEven><<<blocks, kBlock / 2, 0, st>>>(src, dst, phi, mu, geo,    \
                                                                    ph, prev, err, polls,      \
                                                                    parts);                    \
  else if (staged)                                                                            \
    k_collide2t<0, S, true, kAAOdd><<<blocks, kBlock / 2, 0, st>>>(src, dst, phi, mu, geo, ph, \
                                                                   prev, err, polls, parts);  \
  else if (pattern == kAAEven)                                                                \
    k_collide2<0, S, true, kAAEven><<<blocks, kBlock / 2, 0, st>>>(src, dst, phi, mu, geo, ph, \
                                                                   prev, parts);              \
  else                                                                                        \
    k_collide2<0, S, true, kAAOdd><<<blocks, kBlock / 2, 0, st>>>(src, dst, phi, mu, geo, ph,  \
                                                                  prev, parts);
    if (geo.storage == kF16) {
      LBM_SUMS_AA(kF16)
    } else if (geo.storage == kBF16) {
      LBM_SUMS_AA(kBF16)
    } else {
      LBM_SUMS_AA(kF32)
    }
#undef LBM_SUMS_AA
  } else {
    LBM_DISPATCH(geo, pattern, k_collide_sums, src, dst, phi, mu, geo, ph, prev, parts);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_step_sums_final(parts, partial, out, geo, st);
}

cudaError_t launch_step_sums_final(const float* parts, double* partial, double* out,
                                   const Geometry& geo, cudaStream_t st) {
  const int nparts = cell_warps(geo.n);
  const int groups = nparts < kReduceMaxParts ? nparts : kReduceMaxParts;
  const int chunk = (nparts + groups - 1) / groups;
  k_reduce_chunks<<<groups, kBlock, 0, st>>>(parts, nparts, chunk, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reduce_final<<<1, kBlock, 0, st>>>(partial, groups, out);
  return cudaGetLastError();
}

cudaError_t launch_che(const float* src, float* dst, const float* phi, const float* mu,
                       const Geometry& geo, const Physics& ph, int pattern, bool have_prev,
                       float tf, cudaStream_t st) {
  LBM_DISPATCH(geo, pattern, k_che, src, dst, phi, mu, geo, ph, have_prev ? 1 : 0, tf);
  return cudaGetLastError();
}

cudaError_t launch_fields(const float* src, const float* phi, const float* mu, float* out,
                          const Geometry& geo, const Physics& ph, int pattern, float tf,
                          cudaStream_t st) {
  LBM_DISPATCH(geo, pattern, k_fields, src, phi, mu, out, geo, ph, tf);
  return cudaGetLastError();
}

cudaError_t launch_init(float* state, const float* phi, const float* mu, const float* u0,
                        const float* p0, const Geometry& geo, const Physics& ph, int pattern,
                        float tf, cudaStream_t st) {
  LBM_DISPATCH(geo, pattern, k_init, state, phi, mu, u0, p0, geo, ph, tf);
  return cudaGetLastError();
}

cudaError_t launch_gather(const float* src, const float* phi_ref, float* dense, const Geometry& geo,
                          int pattern, int slot, cudaStream_t st) {
  LBM_DISPATCH(geo, pattern, k_gather, src, phi_ref, dense, geo, slot);
  return cudaGetLastError();
}

cudaError_t launch_gather_at(const float* src, const float* phi_ref, const long long* cells,
                             long long count, float* out, const Geometry& geo, int pattern,
                             cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const long long items = count * kTileSlots;
  const long long need = (items + kBlock - 1) / kBlock;
  do {
    const unsigned blocks_ = static_cast<unsigned>(need < 4096 ? need : 4096);
    if (geo.storage == kF16)
      LBM_DISPATCH_P(pattern, k_gather_at, kF16, src, phi_ref, cells, count, out, geo)
    else if (geo.storage == kBF16)
      LBM_DISPATCH_P(pattern, k_gather_at, kBF16, src, phi_ref, cells, count, out, geo)
    else
      LBM_DISPATCH_P(pattern, k_gather_at, kF32, src, phi_ref, cells, count, out, geo)
  } while (0);
  return cudaGetLastError();
}

cudaError_t launch_scatter(float* state, const float* dense, const Geometry& geo, int pattern,
                           int slot, cudaStream_t st) {
  LBM_DISPATCH(geo, pattern, k_scatter, state, dense, geo, slot);
  return cudaGetLastError();
}

cudaError_t launch_convert(const double* in, float* out, int n, cudaStream_t st) {
  k_convert<<<blocks_for(n), kBlock, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_widen(const float* in, double* out, int n, cudaStream_t st) {
  k_widen<<<blocks_for(n), kBlock, 0, st>>>(in, out, n);
  return cudaGetLastError();
}

int resident_blocks_per_sm(int kernel, int storage, bool rows) {
  int blocks = 0;
  cudaError_t e;
  if (kernel == 1 && rows)
    e = storage == kF16    ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_phi_rows<kF16>, kBlock, 0)
        : storage == kBF16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_phi_rows<kBF16>, kBlock, 0)
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_phi_rows<kF32>, kBlock, 0);
  else if (kernel == 3)
    e = storage == kF16    ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_collide2<0, kF16, false>, kBlock / 2, 0)
        : storage == kBF16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_collide2<0, kBF16, false>, kBlock / 2, 0)
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_collide2<0, kF32, false>, kBlock / 2, 0);
  else if (kernel == 0)
    e = storage == kF16    ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_collide<kAB, 0, kF16>, kBlock, 0)
        : storage == kBF16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_collide<kAB, 0, kBF16>, kBlock, 0)
                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_collide<kAB, 0, kF32>, kBlock, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_phi<kAB, kF32>, kBlock, 0);
  return e == cudaSuccess ? blocks : 0;
}

int reduce_parts(const Geometry& geo) {
  const int b = static_cast<int>(blocks_for(geo.n));
  return b < kReduceMaxParts ? b : kReduceMaxParts;
}

cudaError_t launch_reduce(const float* src, const float* phi, double* partial, double* out,
                          const Geometry& geo, int pattern, bool with_g, cudaStream_t st) {
  const int parts = reduce_parts(geo);
  const int wg = with_g ? 1 : 0;
  const unsigned blocks_ = static_cast<unsigned>(parts);
  if (geo.storage == kF16)
    LBM_DISPATCH_P(pattern, k_reduce_partial, kF16, src, phi, partial, geo, wg)
  else if (geo.storage == kBF16)
    LBM_DISPATCH_P(pattern, k_reduce_partial, kBF16, src, phi, partial, geo, wg)
  else
    LBM_DISPATCH_P(pattern, k_reduce_partial, kF32, src, phi, partial, geo, wg)
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reduce_final<<<1, kBlock, 0, st>>>(partial, parts, out);
  return cudaGetLastError();
}

}  // namespace lbm
