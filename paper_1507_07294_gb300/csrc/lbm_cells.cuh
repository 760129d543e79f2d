// Per-cell and per-brick bodies of the three step passes, shared by the single-run
// kernels (lbm_kernels.cu) and the batched kernels that advance many runs in one launch
// (lbm_batch.cu).  See lbm_kernels.cu for what each pass computes.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

constexpr int kBlock = 256;

// Resident blocks per SM the stream-collide kernels are compiled for: 3 (80 registers)
// with FP32 storage, which is DRAM-bound; 4 (64 registers) with 16-bit storage, which
// is bound by instruction issue and gains more from the extra warps than it loses to
// the tighter register budget.
template <int S>
constexpr int collide_min_blocks() {
  return S == kF32 ? 3 : 4;
}

// Bulk prefetch of [p, p + bytes) into L2 (a hint: no completion to wait for).  p must be
// 16-byte aligned and bytes a multiple of 16.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// L2 prefetch, by the calling thread, of what a block streams for the kBlock cells that
// start at cell `first` (a multiple of kBlock): with ALL_SLOTS the whole cell state (all
// 25 slots) and phi and mu of those cells, else the 7 f slots of each tile.  Ranges are
// clipped to the arrays.
template <int S, bool ALL_SLOTS>
__device__ __forceinline__ void prefetch_cells(const float* state, const float* phi,
                                               const float* mu, const Geometry& geo,
                                               long long first) {
  if (first < 0 || first >= geo.n) return;
  const long long cells = min(static_cast<long long>(kBlock), geo.n - first);
  // kBlock is a multiple of kTile, so `first` starts a tile
  const int tiles = static_cast<int>((cells + kTile - 1) / kTile);
  const float* t0 = state + tile_floats<S>(static_cast<int>(first));
  if (ALL_SLOTS) {
    prefetch_l2(t0, static_cast<unsigned>(tiles * tile_bytes<S>()));
    const unsigned bytes = static_cast<unsigned>(cells * sizeof(float)) & ~15u;
    if (bytes) {
      prefetch_l2(phi + first, bytes);
      prefetch_l2(mu + first, bytes);
    }
  } else {
    for (int t = 0; t < tiles; ++t)
      prefetch_l2(t0 + t * (tile_bytes<S>() / 4),
                  static_cast<unsigned>(kQ7 * kTile * sizeof(typename Elem<S>::T)));
  }
}

__device__ __forceinline__ void cell_coords(const Geometry& geo, int idx, int& x, int& y, int& z) {
  const int r = fast_div(idx, geo.div_nx);
  x = idx - r * geo.nx;
  z = fast_div(r, geo.div_ny);
  y = r - z * geo.ny;
}


// ------------------------------------------------- pull addressing on tile rows -------
// When every row of the grid is a whole number of tiles (nx a multiple of kTile), the
// tile of cell (x + dx, y + dy, z + dz) is the own tile moved by whole rows and planes
// of tiles, and only the x step can leave the tile (lanes 0 and 31).  The byte address
// of a pulled population is then z[dz] + (x[dx] + y[dy]) + slot offset, the periodic
// images folded into the per-thread deltas: a few integer operations per distinct
// source cell instead of a tile mapping per load.  Used for cells off the walls (the
// bounce-back links keep the general loaders), by the two-array pulls and by the odd
// steps of the in-place pattern; Geometry::row_tiles is 0 where the layout does not
// allow it.
struct RowPull {
  const char* z[3];  // own slot-0 address moved by dz = -1, 0, +1 planes
  int x[3], y[3];    // byte deltas of dx, dy = -1, 0, +1
};

// From the neighbour offsets: with whole-tile rows the y and z offsets are multiples of
// kTile cells, i.e. whole tiles of tile_bytes / kTile bytes per cell; only lanes 0 and
// 31 step into another tile in x (the previous or next one, or across the periodic
// image of the row).
template <int S>
__device__ __forceinline__ RowPull row_pull(const float* src, const Nbr& nb, int idx) {
  constexpr int EB = static_cast<int>(sizeof(typename Elem<S>::T));
  constexpr int TB = tile_bytes<S>(), TBC = TB / kTile, L = kTile - 1;
  static_assert(TB % kTile == 0, "tile bytes per cell");
  const int lane = idx & L;
  RowPull r;
  r.x[0] = lane ? -EB : (((nb.xm + 1) >> kTileShift) - 1) * TB + L * EB;
  r.x[1] = 0;
  r.x[2] = lane != L ? EB : (((nb.xp - 1) >> kTileShift) + 1) * TB - L * EB;
  r.y[0] = nb.ym * TBC;
  r.y[1] = 0;
  r.y[2] = nb.yp * TBC;
  r.z[1] = reinterpret_cast<const char*>(src) + static_cast<long long>(idx >> kTileShift) * TB +
           lane * EB;
  r.z[0] = r.z[1] + static_cast<long long>(nb.zm) * TBC;
  r.z[2] = r.z[1] + static_cast<long long>(nb.zp) * TBC;
  return r;
}

// Value of slot SLOT of the cell at offset (DX, DY, DZ).
template <int S, int SLOT, int DX, int DY, int DZ>
__device__ __forceinline__ float row_load(const RowPull& r) {
  typedef typename Elem<S>::T T;
  const char* p = r.z[DZ + 1] + (r.x[DX + 1] + r.y[DY + 1]);
  return Elem<S>::get(*reinterpret_cast<const T*>(p + SLOT * kTile * static_cast<int>(sizeof(T))));
}

// Store v into slot SLOT of the cell at offset (DX, DY, DZ).
template <int S, int SLOT, int DX, int DY, int DZ>
__device__ __forceinline__ void row_store(const RowPull& r, float v) {
  typedef typename Elem<S>::T T;
  char* p = const_cast<char*>(r.z[DZ + 1]) + (r.x[DX + 1] + r.y[DY + 1]);
  *reinterpret_cast<T*>(p + SLOT * kTile * static_cast<int>(sizeof(T))) = Elem<S>::put(v);
}

// The loaders of pattern P (load_f, load_g) for a cell off the walls: AB pulls slot i
// of x - c_i; the odd step of the in-place pattern reads slot opp(i) of x - c_i.
template <int P, int S>
__device__ __forceinline__ void row_load_f(const RowPull& r, float f[7]) {
#define X(I, O, CX, CY, CZ) f[I] = row_load<S, P == kAAOdd ? O : I, -CX, -CY, -CZ>(r);
  LBM_D3Q7_LIST(X)
#undef X
}

template <int P, int S>
__device__ __forceinline__ void row_load_g(const RowPull& r, float g[15]) {
#define X(I, O, CX, CY, CZ) g[I] = row_load<S, 7 + (P == kAAOdd ? O : I), -CX, -CY, -CZ>(r);
  LBM_D3Q15_LIST(X)
#undef X
}

// The odd step of the in-place pattern writes f_i+ to slot i of x + c_i (store_f,
// store_g for a cell off the walls).
template <int S>
__device__ __forceinline__ void row_store_f_odd(const RowPull& r, const float f[7]) {
#define X(I, O, CX, CY, CZ) row_store<S, I, CX, CY, CZ>(r, f[I]);
  LBM_D3Q7_LIST(X)
#undef X
}

template <int S>
__device__ __forceinline__ void row_store_g_odd(const RowPull& r, const float g[15]) {
#define X(I, O, CX, CY, CZ) row_store<S, 7 + I, CX, CY, CZ>(r, g[I]);
  LBM_D3Q15_LIST(X)
#undef X
}

// Whether pattern P addresses this cell's neighbours by rows of tiles: two-array pulls
// and the odd in-place step, on grids of whole-tile rows, off the walls.
template <int P>
__device__ __forceinline__ bool use_rows(const Geometry& geo, const Nbr& nb) {
  return (P == kAB || P == kAAOdd) && geo.row_tiles && !(nb.wlo || nb.whi);
}

// ---------------------------------------------------------- order parameter -------
// phi = sum_i f_i of the streamed populations (Eqs. 13, 16).  With 16-bit storage slot
// 0 holds f_0 - phi_ref, phi_ref the order parameter of the step that wrote it;
// phi_ref and phi may be the same array (each thread reads its own cell first).
template <int P, int S>
__device__ __forceinline__ void phi_cell(const float* src, const float* phi_ref, float* phi,
                                         const Geometry& geo, int idx) {
  int x, y, z;
  cell_coords(geo, idx, x, y, z);
  const Nbr nb = make_nbr(geo, x, y, z);
  float f[7];
  if (use_rows<P>(geo, nb))
    row_load_f<P, S>(row_pull<S>(src, nb, idx), f);
  else
    load_f<P, S>(src, idx, nb, f);
  if (S != kF32) f[0] += phi_ref[idx];
  phi[idx] = f[0] + ((f[1] + f[2]) + (f[3] + f[4]) + (f[5] + f[6]));
}

// ------------------------------------------------------- chemical potential -------
// Shared-memory tiling of the 15-point stencil: a block of kTX x kTY threads computes a
// kTX x kTY x kTZ brick of cells from one load of the brick plus a one-cell halo, so
// each phi value is read from global memory (kTX+2)(kTY+2)(kTZ+2)/(kTX kTY kTZ) = 1.5
// times instead of 15 times.  The halo is loaded row by row (one address computation
// per row of kTX + 2 values), and each thread walks its column in z keeping, per plane,
// the centre, the sum of the 4 in-plane face neighbours and the sum of the 4 in-plane
// diagonal neighbours, so every plane is summed once for the three cells that use it.
constexpr int kTX = 32, kTY = 8, kTZ = 16;
constexpr int kHX = kTX + 2, kHY = kTY + 2, kHZ = kTZ + 2;

// v mod n for v in [-1, n + span): a compare and add when n >= span, else a modulo.
__device__ __forceinline__ int wrap(int v, int n, int span) {
  if (n >= span) return v < 0 ? v + n : (v >= n ? v - n : v);
  v %= n;
  return v < 0 ? v + n : v;
}

// mu of the kTX x kTY columns of brick (x0, y0, z0) from a halo tile already in shared
// memory: tile[l][i][jj] holds phi at (x0 - XOFF + jj, y0 - 1 + i, z0 - 1 + l) with
// ghosts and periodic images filled in.  Threads outside the grid return.
template <bool D3Q7, int HX, int XOFF>
__device__ __forceinline__ void mu_columns(const float (*tile)[kHY][HX], float* __restrict__ mu,
                                           const Geometry& geo, const Physics& ph, int x0, int y0,
                                           int z0) {
  const int lane = threadIdx.x, warp = threadIdx.y;
  const int x = x0 + lane, y = y0 + warp;
  if (x >= geo.nx || y >= geo.ny) return;
  const int i = warp + 1, j = lane + XOFF;
  // per-plane partial sums of column (i, j): centre, faces, diagonals
  auto plane = [&](int l, float& c, float& f, float& d) {
    c = tile[l][i][j];
    f = (tile[l][i][j - 1] + tile[l][i][j + 1]) + (tile[l][i - 1][j] + tile[l][i + 1][j]);
    d = (tile[l][i - 1][j - 1] + tile[l][i - 1][j + 1]) + (tile[l][i + 1][j - 1] + tile[l][i + 1][j + 1]);
  };
  float c0, f0, d0, c1, f1, d1;
  plane(0, c0, f0, d0);
  plane(1, c1, f1, d1);
  const int nl = min(kTZ, geo.nz - z0);
  float* out = mu + (static_cast<size_t>(z0) * geo.ny + y) * geo.nx + x;
  const size_t zstride = static_cast<size_t>(geo.plane);
  for (int l = 1; l <= nl; ++l) {
    float c2, f2, d2;
    plane(l + 1, c2, f2, d2);
    // Eq. 36 on the D3Q15 stencil: 2/3 (faces - 6 c) + 1/12 (corners - 8 c); with the
    // D3Q7 weights: faces - 6 c
    const float lap = D3Q7 ? lap7_columns(c0, c1, c2, f1) : lap15_columns(c0, c1, c2, f1, d0, d2);
    out[(l - 1) * zstride] = chemical_potential(ph, c1, lap);
    c0 = c1; f0 = f1; d0 = d1;
    c1 = c2; f1 = f2; d1 = d2;
  }
}

// Source z of halo plane zz: clamped to the fluid between walls (the stencil ghost is
// the adjacent node), wrapped when periodic.
__device__ __forceinline__ int ghost_z(const Geometry& geo, int zz) {
  return geo.walls ? min(max(zz, 0), geo.nz - 1) : wrap(zz, geo.nz, kHZ);
}

// mu = 4 beta phi (phi^2 - 1) - kappa lap phi (Eq. 2) for brick (bx, by, bz) of the grid;
// called by all kTX x kTY threads of a block, `tile` in shared memory, loaded here with
// plain loads.  The only barrier is the one after the tile load; threads outside the
// grid return after it, so a caller that reuses `tile` for another brick must
// synchronise the block first.
template <bool D3Q7>
__device__ __forceinline__ void mu_brick(const float* __restrict__ phi, float* __restrict__ mu,
                                         const Geometry& geo, const Physics& ph, int bx, int by,
                                         int bz, float (*tile)[kHY][kHX]) {
  const int x0 = bx * kTX, y0 = by * kTY, z0 = bz * kTZ;
  const int lane = threadIdx.x, warp = threadIdx.y;
  // columns of the halo brick this lane loads: j = lane and, for lanes 0-1, j = 32 + lane
  const int gx_a = wrap(x0 - 1 + lane, geo.nx, kHX);
  const int gx_b = wrap(x0 - 1 + kTX + (lane & 1), geo.nx, kHX);
  for (int r = warp; r < kHZ * kHY; r += kTY) {
    const int l = r / kHY, i = r - l * kHY;
    const int gy = wrap(y0 - 1 + i, geo.ny, kHY);
    const int gz = ghost_z(geo, z0 - 1 + l);
    const float* row = phi + (static_cast<size_t>(gz) * geo.ny + gy) * geo.nx;
    tile[l][i][lane] = __ldg(row + gx_a);
    if (lane < 2) tile[l][i][kTX + lane] = __ldg(row + gx_b);
  }
  __syncthreads();
  mu_columns<D3Q7, kHX, 1>(tile, mu, geo, ph, x0, y0, z0);
}

// ------------------------------------------------------ fused stream-collide -------
// Stencil quantities of one cell: grad phi (Eq. 35), lap mu (Eq. 36), centre values.
struct CellStencils {
  float grad_phi[3], lap_mu, phi, mu;
};

template <bool D3Q7 = false>
__device__ __forceinline__ CellStencils cell_stencils(const float* __restrict__ phi,
                                                      const float* __restrict__ mu, int idx,
                                                      const Nbr& nb) {
  CellStencils cs;
  {
    Stencil s;
    load_stencil(phi, idx, nb, s);
    if (D3Q7)
      stencil_grad7(s, cs.grad_phi);
    else
      stencil_grad(s, cs.grad_phi);
    cs.phi = s.c;
  }
  {
    Stencil s;
    load_stencil(mu, idx, nb, s);
    cs.lap_mu = D3Q7 ? stencil_lap7(s) : stencil_lap(s);
    cs.mu = s.c;
  }
  return cs;
}


// Pull f and g, stencils of phi and mu, forces, u and p, both MRT collisions,
// d_t(phi u), store f+ and g+ (Eqs. 14-34).  src and dst are the same array for the
// in-place patterns.  All 25 cell-state loads are issued first so that they are in
// flight together with the stencil loads.
// With SUMS, sums[0..3] receive the cell's contributions to the global sums of the state
// after this step (as lbm_reduce defines them): streaming only permutes post-collision
// values, and a population that meets a wall re-enters its own cell with the opposite
// velocity, so sum phi = sum of all post-collision f, and the lattice momentum = sum of
// c_i g_i with c_i negated for the populations that bounce.  Each value is taken as the
// next step will read it back from storage (16-bit rounding, the slot-0 shift undone).
// The cell-state reads of the stream-collide body: the pulled g (and, with LOAD_F, f) of
// pattern P and phi u of the previous step.
template <int P, int S, bool LOAD_F>
__device__ __forceinline__ void load_cell(const float* src, const Geometry& geo, int idx,
                                          const Nbr& nb, float g[15], float f[7], float prev[3]) {
  if (use_rows<P>(geo, nb)) {
    const RowPull r = row_pull<S>(src, nb, idx);
    row_load_g<P, S>(r, g);
    if (LOAD_F) row_load_f<P, S>(r, f);
  } else {
    load_g<P, S>(src, idx, nb, g);
    if (LOAD_F) load_f<P, S>(src, idx, nb, f);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) prev[a] = src[phiu_index<S>(idx, a)];
}

// collide_loaded is the body for a cell whose populations are loaded; `stencils()`
// returns its CellStencils (from the global phi and mu arrays in collide_cell, from
// shared-memory planes in the fused single-pass kernel).  The values it is given are
// the only inputs that differ between the two, so both give the same bits.
template <int P, int VAR, int S, bool SUMS, typename StencilFn>
__device__ __forceinline__ void collide_loaded(float* dst, const Geometry& geo, const Physics& ph,
                                               int have_prev, int idx, const Nbr& nb,
                                               float g[15], float f[7], const float prev[3],
                                               StencilFn stencils, float* sums) {
  const CellStencils cs = stencils();
  const Moments15 mo = moments15(g);
  const Macro M = macroscopic(ph, mo, cs.phi, cs.mu, cs.grad_phi, cs.lap_mu);
  const float lambda_visc = viscous_rate(ph, cs.phi);
  collide_d3q15<(VAR & kVarSrtFlow) != 0>(ph, g, mo, M, lambda_visc);
  if (SUMS) {
    typedef Elem<S> E;
    float v[15];
#pragma unroll
    for (int i = 0; i < 15; ++i) v[i] = E::get(E::put(g[i]));
    // sum c_i v_i (corners (1,1,1), (1,1,-1), (1,-1,1), (1,-1,-1) and their opposites)
    const float a7 = v[7] - v[8], a9 = v[9] - v[10], a11 = v[11] - v[12], a13 = v[13] - v[14];
    float jx = (v[1] - v[2]) + ((a7 + a9) + (a11 + a13));
    float jy = (v[3] - v[4]) + ((a7 + a9) - (a11 + a13));
    float jz = (v[5] - v[6]) + ((a7 - a9) + (a11 - a13));
    if (nb.wlo || nb.whi) {
      // populations leaving through a wall come back reversed: take 2 c_i v_i off
#define X(I, O, CX, CY, CZ)                                    \
  if ((CZ > 0 && nb.whi) || (CZ < 0 && nb.wlo)) {              \
    jx -= 2.0f * CX * v[I];                                    \
    jy -= 2.0f * CY * v[I];                                    \
    jz -= 2.0f * CZ * v[I];                                    \
  }
      LBM_D3Q15_LIST(X)
#undef X
    }
    sums[1] = jx;
    sums[2] = jy;
    sums[3] = jz;
  }
  if (P == kAAOdd && use_rows<P>(geo, nb))
    row_store_g_odd<S>(row_pull<S>(dst, nb, idx), g);
  else
    store_g<P, S>(dst, idx, nb, g);

  // d_t(phi u) by the backward difference of Eq. 34; phi u lives in the own tile
  float dphiu[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float cur = __fmul_rn(cs.phi, M.u[a]);
    dphiu[a] = have_prev ? __fsub_rn(cur, prev[a]) : 0.0f;
    dst[phiu_index<S>(idx, a)] = cur;
  }

  collide_d3q7<S != kF32>(ph, f, cs.phi, cs.mu, M.u, dphiu);
  if (SUMS) {
    typedef Elem<S> E;
    float f0 = E::get(E::put(f[0]));
    if (S != kF32) f0 += cs.phi;  // slot 0 holds f_0 - phi
    sums[0] = f0 + ((E::get(E::put(f[1])) + E::get(E::put(f[2]))) +
                    (E::get(E::put(f[3])) + E::get(E::put(f[4]))) +
                    (E::get(E::put(f[5])) + E::get(E::put(f[6]))));
  }
  if (P == kAAOdd && use_rows<P>(geo, nb))
    row_store_f_odd<S>(row_pull<S>(dst, nb, idx), f);
  else
    store_f<P, S>(dst, idx, nb, f);
}

template <int P, int VAR, int S, bool SUMS, typename StencilFn>
__device__ __forceinline__ void collide_cell_at(const float* src, float* dst, const Geometry& geo,
                                                const Physics& ph, int have_prev, int idx,
                                                const Nbr& nb, StencilFn stencils, float* sums) {
  float g[15], f[7], prev[3];
  load_cell<P, S, true>(src, geo, idx, nb, g, f, prev);
  collide_loaded<P, VAR, S, SUMS>(dst, geo, ph, have_prev, idx, nb, g, f, prev, stencils, sums);
}

template <int P, int VAR, int S, bool SUMS = false>
__device__ __forceinline__ void collide_cell(const float* src, float* dst,
                                             const float* __restrict__ phi,
                                             const float* __restrict__ mu, const Geometry& geo,
                                             const Physics& ph, int have_prev, int idx,
                                             float* sums = nullptr) {
  int x, y, z;
  cell_coords(geo, idx, x, y, z);
  const Nbr nb = make_nbr(geo, x, y, z);
  collide_cell_at<P, VAR, S, SUMS>(
      src, dst, geo, ph, have_prev, idx, nb,
      [&] { return cell_stencils<(VAR & kVarD3Q7) != 0>(phi, mu, idx, nb); }, sums);
}

// ------------------------------------------- two cells per thread, paired FP32 -------
// The arithmetic of the stream-collide body for two cells, one in each lane of float2
// (the generic per-cell math with V = float2): g and f hold the pulled populations (f[0]
// unused with 16-bit storage), prev the phi u of the previous step, sp and sm the phi
// and mu stencils.  On return g and f hold the post-collision populations (with 16-bit
// storage f[0] = f_0+ - phi) and cur the new phi u.  Per lane the operations are those
// of the one-cell body, so each cell gets the same bits.
template <int VAR, int S>
__device__ __forceinline__ void pair_compute(const Physics& ph, int have_prev, float2 g[15],
                                             float2 f[7], const float2 prev[3],
                                             const StencilV<float2>& sp,
                                             const StencilV<float2>& sm, float2 cur[3]) {
  typedef VOps<float2> O;
  constexpr bool D3Q7 = (VAR & kVarD3Q7) != 0;
  float2 grad_phi[3];
  if (D3Q7)
    stencil_grad7(sp, grad_phi);
  else
    stencil_grad(sp, grad_phi);
  const float2 lap_mu = D3Q7 ? stencil_lap7(sm) : stencil_lap(sm);
  const float2 phc = sp.c, muc = sm.c;
  const Moments15V<float2> mo = moments15(g);
  const MacroV<float2> M = macroscopic(ph, mo, phc, muc, grad_phi, lap_mu);
  const float2 lambda_visc = viscous_rate(ph, phc);
  collide_d3q15<(VAR & kVarSrtFlow) != 0>(ph, g, mo, M, lambda_visc);
  // d_t(phi u) by the backward difference of Eq. 34
  float2 dphiu[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cur[a] = O::mul(phc, M.u[a]);
    dphiu[a] = have_prev ? O::sub(cur[a], prev[a]) : make_float2(0.0f, 0.0f);
  }
  collide_d3q7<S != kF32>(ph, f, phc, muc, M.u, dphiu);
}

// Both stencils of one scalar field for cells idx and idx + kTile, packed per lane.
__device__ __forceinline__ StencilV<float2> pair_stencil(const float* __restrict__ a, int idx0,
                                                         const Nbr& n0, int idx1, const Nbr& n1) {
  Stencil s0, s1;
  load_stencil(a, idx0, n0, s0);
  load_stencil(a, idx1, n1, s1);
  StencilV<float2> sp;
  sp.c = make_float2(s0.c, s1.c);
  sp.xm = make_float2(s0.xm, s1.xm);
  sp.xp = make_float2(s0.xp, s1.xp);
  sp.ym = make_float2(s0.ym, s1.ym);
  sp.yp = make_float2(s0.yp, s1.yp);
  sp.zm = make_float2(s0.zm, s1.zm);
  sp.zp = make_float2(s0.zp, s1.zp);
#pragma unroll
  for (int k = 0; k < 8; ++k) sp.k[k] = make_float2(s0.k[k], s1.k[k]);
  return sp;
}

// Post-collision sums of one cell (lane c of the pair) as collide_loaded forms them:
// sum phi and the lattice momentum with the wall reversal, each value as the next step
// reads it back from storage.
template <int S>
__device__ __forceinline__ void pair_sums(const float2 g[15], const float2 f[7], float2 phc,
                                          const Nbr& nb, int c, float* sums) {
  typedef Elem<S> E;
  float v[15];
#pragma unroll
  for (int i = 0; i < 15; ++i) v[i] = E::get(E::put(c ? g[i].y : g[i].x));
  const float a7 = v[7] - v[8], a9 = v[9] - v[10], a11 = v[11] - v[12], a13 = v[13] - v[14];
  float jx = (v[1] - v[2]) + ((a7 + a9) + (a11 + a13));
  float jy = (v[3] - v[4]) + ((a7 + a9) - (a11 + a13));
  float jz = (v[5] - v[6]) + ((a7 - a9) + (a11 - a13));
  if (nb.wlo || nb.whi) {
#define X(I, O_, CX, CY, CZ)                                   \
  if ((CZ > 0 && nb.whi) || (CZ < 0 && nb.wlo)) {              \
    jx -= 2.0f * CX * v[I];                                    \
    jy -= 2.0f * CY * v[I];                                    \
    jz -= 2.0f * CZ * v[I];                                    \
  }
    LBM_D3Q15_LIST(X)
#undef X
  }
  sums[1] = jx;
  sums[2] = jy;
  sums[3] = jz;
  float fc[7];
#pragma unroll
  for (int i = 0; i < 7; ++i) fc[i] = c ? f[i].y : f[i].x;
  float f0 = E::get(E::put(fc[0]));
  if (S != kF32) f0 += c ? phc.y : phc.x;  // slot 0 holds f_0 - phi
  sums[0] = f0 + ((E::get(E::put(fc[1])) + E::get(E::put(fc[2]))) +
                  (E::get(E::put(fc[3])) + E::get(E::put(fc[4]))) +
                  (E::get(E::put(fc[5])) + E::get(E::put(fc[6]))));
}

// The stores of a pair's post-collision state (cells idx and idx + kTile) with pattern P:
// g, phi u and f; the odd in-place step writes the neighbours' slots, by rows off the
// walls, as collide_loaded does.
template <int P, int S>
__device__ __forceinline__ void store_pair(float* dst, const Geometry& geo, int idx,
                                           const Nbr& na, const Nbr& nb2, const float2 g[15],
                                           const float2 f[7], const float2 cur[3]) {
  const int idx2 = idx + kTile;
  auto put_g = [&](int i, const Nbr& nb, const float* v) {
    if (P == kAAOdd && use_rows<P>(geo, nb))
      row_store_g_odd<S>(row_pull<S>(dst, nb, i), v);
    else
      store_g<P, S>(dst, i, nb, v);
  };
  auto put_f = [&](int i, const Nbr& nb, const float* v) {
    if (P == kAAOdd && use_rows<P>(geo, nb))
      row_store_f_odd<S>(row_pull<S>(dst, nb, i), v);
    else
      store_f<P, S>(dst, i, nb, v);
  };
  float a[15], b[15];
#pragma unroll
  for (int i = 0; i < 15; ++i) {
    a[i] = g[i].x;
    b[i] = g[i].y;
  }
  put_g(idx, na, a);
  put_g(idx2, nb2, b);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dst[phiu_index<S>(idx, k)] = cur[k].x;
    dst[phiu_index<S>(idx2, k)] = cur[k].y;
  }
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    a[i] = f[i].x;
    b[i] = f[i].y;
  }
  put_f(idx, na, a);
  put_f(idx2, nb2, b);
}

// The stream-collide body for cells idx and idx + kTile (the same lane of two adjacent
// tiles of one row) with pattern P: loads and stores per cell, the arithmetic once for
// both (pair_compute).  Both cells are loaded before either is stored, so the in-place
// patterns (src == dst) stay race-free as in collide_cell.  With SUMS, sums[0..3] and
// sums[4..7] receive the two cells' contributions (as collide_loaded).
template <int VAR, int S, bool SUMS, int P = kAB>
__device__ __forceinline__ void collide_pair(const float* src, float* dst,
                                             const float* __restrict__ phi,
                                             const float* __restrict__ mu, const Geometry& geo,
                                             const Physics& ph, int have_prev, int idx,
                                             float* sums) {
  int x, y, z;
  cell_coords(geo, idx, x, y, z);
  const int idx2 = idx + kTile;
  const Nbr na = make_nbr(geo, x, y, z), nb2 = make_nbr(geo, x + kTile, y, z);
  float ga[15], fa[7], pa[3], gb[15], fb[7], pb[3];
  load_cell<P, S, true>(src, geo, idx, na, ga, fa, pa);
  load_cell<P, S, true>(src, geo, idx2, nb2, gb, fb, pb);
  const StencilV<float2> sp = pair_stencil(phi, idx, na, idx2, nb2);
  const StencilV<float2> sm = pair_stencil(mu, idx, na, idx2, nb2);
  float2 g[15], f[7], prev[3], cur[3];
#pragma unroll
  for (int i = 0; i < 15; ++i) g[i] = make_float2(ga[i], gb[i]);
#pragma unroll
  for (int i = 0; i < 7; ++i) f[i] = make_float2(fa[i], fb[i]);
#pragma unroll
  for (int a = 0; a < 3; ++a) prev[a] = make_float2(pa[a], pb[a]);
  pair_compute<VAR, S>(ph, have_prev, g, f, prev, sp, sm, cur);
  if (SUMS) {
    pair_sums<S>(g, f, sp.c, na, 0, sums);
    pair_sums<S>(g, f, sp.c, nb2, 1, sums + 4);
  }
  store_pair<P, S>(dst, geo, idx, na, nb2, g, f, cur);
}

// Sums of the fused step sums over the 32 cells of a warp, stored as 5 floats at
// parts[5 w] (w = the warp's first cell / 32): sum phi, momentum x, y, z (FP32 sums)
// and the count of cells with a non-finite contribution (exact in float); the
// reduction over warps that follows is FP64.  The four sums take 6 shuffles instead of
// 20: across lane bit 4 a lane keeps two values and hands its partner the other two,
// across bit 3 one of those, so that lane l then carries value 2 (l >> 4 & 1) +
// (l >> 3 & 1) over 4 lanes; three butterfly levels over bits 2..0 complete each sum in
// its group of 8 lanes.  All 32 lanes must call it.
__device__ __forceinline__ void warp_sums_store(const float s[4], bool bad, float* parts,
                                                long long first_cell) {
  const unsigned nbad = __popc(__ballot_sync(0xffffffffu, bad));
  const unsigned lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8;
  const float keep0 = b4 ? s[2] : s[0], keep1 = b4 ? s[3] : s[1];
  const float give0 = b4 ? s[0] : s[2], give1 = b4 ? s[1] : s[3];
  const float a0 = keep0 + __shfl_xor_sync(0xffffffffu, give0, 16);
  const float a1 = keep1 + __shfl_xor_sync(0xffffffffu, give1, 16);
  float v = (b3 ? a1 : a0) + __shfl_xor_sync(0xffffffffu, b3 ? a0 : a1, 8);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  float* out = parts + static_cast<size_t>(first_cell >> 5) * 5;
  if ((lane & 7) == 0) out[lane >> 3] = v;
  if (lane == 0) out[4] = static_cast<float>(nbad);
}

}  // namespace lbm
