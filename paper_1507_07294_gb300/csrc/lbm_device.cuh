// Device-side building blocks of the coupled D3Q7 + D3Q15 MRT update (Liang, Shi &
// Chai, arXiv:1507.07294, Sec. II).  Everything here runs in FP32 on the CUDA cores:
// the per-cell moment transforms are small, sparse and memory-bound, so they are
// written as add trees over the orthogonal rows of M (Eq. 9) and Gamma (Eq. 25)
// rather than as dense products.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstddef>
#include <cstdint>

namespace lbm {

// ---------------------------------------------------------------------------------
// Parameters passed by value to every kernel (kept in the constant bank).
// ---------------------------------------------------------------------------------
// Division of a non-negative int by a fixed divisor d >= 1 with one high multiply, an
// add and a shift (Granlund & Montgomery, "Division by invariant integers using
// multiplication", 1994): with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (umulhi(m, n) + n) >> l for all 0 <= n < 2^31.
struct FastDiv {
  unsigned d, m, l;
};

struct Geometry {
  int nx, ny, nz;
  int walls;       // 1: halfway bounce-back at z = 0 and z = nz
  int n;           // cells, < 2^31
  int plane;       // nx * ny
  size_t stride;   // elements between consecutive planes of dense per-cell arrays
  FastDiv div_nx, div_ny;
  int prefetch_collide;  // L2 prefetch distance of k_collide in blocks (0: none)
  int prefetch_phi;      // same for k_phi
  int storage;           // population storage type (Storage); selects the kernel instance
  int row_tiles;         // nx / kTile when rows are whole tiles and a plane of tiles spans
                         // < 2^31 bytes (pull addressing of RowPull), else 0
};

__device__ __forceinline__ int fast_div(int n, const FastDiv& f) {
  const unsigned long long t =
      static_cast<unsigned long long>(__umulhi(f.m, static_cast<unsigned>(n))) + static_cast<unsigned>(n);
  return static_cast<int>(t >> f.l);
}

struct Physics {
  float rho_g;       // Eq. 14: rho = rho_g + (1 + phi) * half_drho
  float half_drho;   // (rho_l - rho_g) / 2
  float nu_g, half_dnu, nu_mid;  // nu(phi) = nu_mid + phi * half_dnu
  float mob;         // mobility (Eq. 1)
  float kappa, beta; // Eq. 2
  float eta, A;      // Eqs. 5, 8, 19
  float gacc[3];     // body acceleration
  float rho_ref;     // G = (rho - rho_ref) g; 0 for the plain weight
  // Relaxation rates divided by the squared norms of the moment rows (norm7, norm15):
  // sf_a[k] = s_k / |M_k|^2 and sf_b[k] = (1 - s_k / 2) / |M_k|^2 for S^f (Eq. 10);
  // sg_a, sg_b the same for S^g (Eq. 26), entries 9..13 unused (viscous, per cell).
  float sf_a[7], sf_b[7];
  float sg_a[15], sg_b[15];
  int vel_kind;      // 0: coupled; else the prescribed velocity field (VelocityKind)
  float vel_U;       // its amplitude U
  int srt_flow;      // 1: every D3Q15 rate is the viscous one (single relaxation time)
  int d3q7_stencil;  // 1: Eqs. 35-36 with the D3Q7 weights (7-point central differences)
};

// Squared norms of the rows of M (Eq. 9) and Gamma (Eq. 25): both sets of rows are
// orthogonal, so M^{-1} = M^T diag(1 / |M_k|^2) and likewise for Gamma.
//   |M_k|^2     = 7, 2, 2, 2, 42, 12, 4
//   |Gamma_k|^2 = 15, 18, 360, 10, 40, 10, 40, 10, 40, 12, 4, 8, 8, 8, 8
__host__ __device__ constexpr float norm7(int k) {
  return k == 0 ? 7.0f : (k <= 3 ? 2.0f : (k == 4 ? 42.0f : (k == 5 ? 12.0f : 4.0f)));
}
__host__ __device__ constexpr float norm15(int k) {
  return k == 0 ? 15.0f
       : k == 1 ? 18.0f
       : k == 2 ? 360.0f
       : k <= 8 ? ((k & 1) ? 10.0f : 40.0f)
       : k == 9 ? 12.0f
       : k == 10 ? 4.0f
                 : 8.0f;
}

// Compile-time model variants of the step kernels (bit set): kVarSrtFlow, kVarD3Q7.
constexpr int kVarSrtFlow = 1;
constexpr int kVarD3Q7 = 2;

// Prescribed velocity fields of the interface-tracking mode (Sec. III A, B).
enum VelocityKind { kVelNone = 0, kVelUniform = 1, kVelRotation = 2, kVelDeformation = 3 };

// Population q of the D3Q7 set lives at slot q (0..6), population i of the D3Q15
// set at slot 7 + i, and the three components of phi u of the previous step at slots
// 22..24.  Velocity orders: Eq. 6 and Eq. 23.  In both orders the opposite of i > 0 is
// i + 1 for odd i and i - 1 for even i.
constexpr int kQ7 = 7;
constexpr int kQ15 = 15;
constexpr int kSlots = kQ7 + kQ15;    // populations
constexpr int kSlotPhiu = kSlots;     // first phi u slot
constexpr int kTileSlots = kSlots + 3;

// Cell-state layout: tiles of kTile consecutive cells (x fastest); a tile stores its
// 25 slots one after another, kTile values each: the 22 populations in the storage
// type (FP32, FP16 or BF16), then the 3 phi u components in FP32 (3.2 KB per tile in
// FP32, 1.75 KB with 16-bit populations).  A warp's own-cell accesses therefore fall
// in one small block of memory instead of 25 arrays a whole grid apart, which keeps
// the number of pages a warp touches small.
constexpr int kTile = 32;
constexpr int kTileShift = 5;

// Population storage types.  With 16-bit storage, slot 0 holds f_0 - phi (phi of the
// step that wrote it, kept in the order-parameter array) instead of f_0 ~ phi ~ +-1,
// which 16 bits would round to ~1e-3; all arithmetic stays FP32.
enum Storage { kF32 = 0, kF16 = 1, kBF16 = 2 };

template <int S>
struct Elem;
template <>
struct Elem<kF32> {
  typedef float T;
  static __device__ __forceinline__ float get(T v) { return v; }
  static __device__ __forceinline__ T put(float v) { return v; }
};
template <>
struct Elem<kF16> {
  typedef __half T;
  static __device__ __forceinline__ float get(T v) { return __half2float(v); }
  static __device__ __forceinline__ T put(float v) { return __float2half_rn(v); }
};
template <>
struct Elem<kBF16> {
  typedef __nv_bfloat16 T;
  static __device__ __forceinline__ float get(T v) { return __bfloat162float(v); }
  static __device__ __forceinline__ T put(float v) { return __float2bfloat16_rn(v); }
};

template <int S>
__host__ __device__ constexpr int tile_bytes() {
  return kSlots * kTile * static_cast<int>(sizeof(typename Elem<S>::T)) + 3 * kTile * 4;
}

// Start of the tile holding cell i (as a float pointer: tiles are 16-byte multiples).
template <int S>
__device__ __forceinline__ size_t tile_floats(int i) {
  return static_cast<size_t>(i >> kTileShift) * (tile_bytes<S>() / 4);
}

template <int S, int SLOT>
__device__ __forceinline__ typename Elem<S>::T* pop_ptr(float* state, int i) {
  typedef typename Elem<S>::T T;
  return reinterpret_cast<T*>(state + tile_floats<S>(i)) + SLOT * kTile + (i & (kTile - 1));
}

template <int S, int SLOT>
__device__ __forceinline__ const typename Elem<S>::T* pop_ptr(const float* state, int i) {
  typedef typename Elem<S>::T T;
  return reinterpret_cast<const T*>(state + tile_floats<S>(i)) + SLOT * kTile + (i & (kTile - 1));
}

// phi u component a of cell i
template <int S>
__device__ __forceinline__ size_t phiu_index(int i, int a) {
  return tile_floats<S>(i) + (kSlots * kTile * sizeof(typename Elem<S>::T)) / 4 + a * kTile +
         (i & (kTile - 1));
}

// ---------------------------------------------------------------------------------
// Neighbour offsets of one cell.  x and y wrap; z wraps or, between walls, the
// stencil ghost of an out-of-range node is the node itself (offset 0).
// ---------------------------------------------------------------------------------
struct Nbr {
  int xm, xp, ym, yp, zm, zp;  // element offsets to x-1, x+1, ...
  bool wlo, whi;               // cell touches the bottom / top wall
};

__device__ __forceinline__ Nbr make_nbr(const Geometry& geo, int x, int y, int z) {
  Nbr nb;
  nb.xm = (x == 0) ? geo.nx - 1 : -1;
  nb.xp = (x == geo.nx - 1) ? -(geo.nx - 1) : 1;
  nb.ym = (y == 0) ? (geo.ny - 1) * geo.nx : -geo.nx;
  nb.yp = (y == geo.ny - 1) ? -(geo.ny - 1) * geo.nx : geo.nx;
  if (geo.walls) {
    nb.wlo = (z == 0);
    nb.whi = (z == geo.nz - 1);
    nb.zm = nb.wlo ? 0 : -geo.plane;
    nb.zp = nb.whi ? 0 : geo.plane;
  } else {
    nb.wlo = nb.whi = false;
    nb.zm = (z == 0) ? (geo.nz - 1) * geo.plane : -geo.plane;
    nb.zp = (z == geo.nz - 1) ? -(geo.nz - 1) * geo.plane : geo.plane;
  }
  return nb;
}

template <int CX, int CY, int CZ>
__device__ __forceinline__ int offset(const Nbr& nb) {
  return (CX > 0 ? nb.xp : (CX < 0 ? nb.xm : 0)) + (CY > 0 ? nb.yp : (CY < 0 ? nb.ym : 0)) +
         (CZ > 0 ? nb.zp : (CZ < 0 ? nb.zm : 0));
}

// ---------------------------------------------------------------------------------
// Population storage patterns.  A step reads the pre-collision populations of each
// cell, collides, and stores the post-collision ones so that the next step finds its
// pre-collision values.
//
// kAB (two arrays, "pull"): the current array holds post-collision values of the
//   previous step, slot (i, y) = f_i^+(y).  A step reads f_i(x) = f_i^+(x - c_i) from
//   slot (i, x - c_i) of the current array and writes f_i^+(x) to slot (i, x) of the
//   other array; the arrays then swap roles.  A link whose source x - c_i lies beyond
//   a wall is closed by bounce-back: f_i(x) = f_opp(i)^+(x), slot (opp(i), x).
// kAAEven / kAAOdd (one array, in place, half the memory): even steps read slot
//   (i, x) and write to slot (opp(i), x); odd steps read f_i(x) from slot
//   (opp(i), x - c_i) and write to slot (i, x + c_i), where the next even step finds
//   it.  Each cell reads and writes the same set of slots, so the update is race-free
//   in place.  Across a wall an odd step reads slot (i, x) and writes slot (opp(i), x).
//   On GB300 the odd step, whose reads and writes both land on neighbours' lines in
//   the array being updated, moves data markedly slower than the two-array pattern.
//
// The pointers carry no __restrict__: the in-place pattern loads and then stores the
// same slots through one array, and those loads must stay ahead of the stores.
// ---------------------------------------------------------------------------------
enum Pattern { kAB = 0, kAAEven = 1, kAAOdd = 2 };

template <int S, int P, int SLOT, int SLOT_OPP, int CX, int CY, int CZ>
__device__ __forceinline__ float pop_load(const float* a, int idx, const Nbr& nb) {
  typedef Elem<S> E;
  if (P == kAAEven) return E::get(*pop_ptr<S, SLOT>(a, idx));
  const bool wall = (CZ > 0 && nb.wlo) || (CZ < 0 && nb.whi);
  if (P == kAAOdd) {
    if (wall) return E::get(*pop_ptr<S, SLOT>(a, idx));
    return E::get(*pop_ptr<S, SLOT_OPP>(a, idx + offset<-CX, -CY, -CZ>(nb)));
  }
  if (wall) return E::get(*pop_ptr<S, SLOT_OPP>(a, idx));
  return E::get(*pop_ptr<S, SLOT>(a, idx + offset<-CX, -CY, -CZ>(nb)));
}

// Store the post-collision value of direction SLOT of cell idx.
template <int S, int P, int SLOT, int SLOT_OPP, int CX, int CY, int CZ>
__device__ __forceinline__ void pop_store(float* a, int idx, const Nbr& nb, float v) {
  typedef Elem<S> E;
  if (P == kAB) {
    *pop_ptr<S, SLOT>(a, idx) = E::put(v);
  } else if (P == kAAEven) {
    *pop_ptr<S, SLOT_OPP>(a, idx) = E::put(v);
  } else {
    const bool wall = (CZ > 0 && nb.whi) || (CZ < 0 && nb.wlo);
    if (wall)
      *pop_ptr<S, SLOT_OPP>(a, idx) = E::put(v);
    else
      *pop_ptr<S, SLOT>(a, idx + offset<CX, CY, CZ>(nb)) = E::put(v);
  }
}

// Place the PRE-collision value of direction SLOT of cell idx where a step of pattern
// P reads it (inverse of pop_load): used to write initial and restored states.
template <int S, int P, int SLOT, int SLOT_OPP, int CX, int CY, int CZ>
__device__ __forceinline__ void pop_place(float* a, int idx, const Nbr& nb, float v) {
  typedef Elem<S> E;
  if (P == kAAEven) {
    *pop_ptr<S, SLOT>(a, idx) = E::put(v);
    return;
  }
  const bool wall = (CZ > 0 && nb.wlo) || (CZ < 0 && nb.whi);
  if (P == kAAOdd) {
    if (wall)
      *pop_ptr<S, SLOT>(a, idx) = E::put(v);
    else
      *pop_ptr<S, SLOT_OPP>(a, idx + offset<-CX, -CY, -CZ>(nb)) = E::put(v);
    return;
  }
  if (wall)
    *pop_ptr<S, SLOT_OPP>(a, idx) = E::put(v);
  else
    *pop_ptr<S, SLOT>(a, idx + offset<-CX, -CY, -CZ>(nb)) = E::put(v);
}

// D3Q7 velocities (Eq. 6) as template arguments: slot, opposite slot, c.
#define LBM_D3Q7_LIST(X) \
  X(0, 0, 0, 0, 0)       \
  X(1, 2, 1, 0, 0)       \
  X(2, 1, -1, 0, 0)      \
  X(3, 4, 0, 1, 0)       \
  X(4, 3, 0, -1, 0)      \
  X(5, 6, 0, 0, 1)       \
  X(6, 5, 0, 0, -1)

// D3Q15 velocities (Eq. 23): index i, opposite, c.
#define LBM_D3Q15_LIST(X) \
  X(0, 0, 0, 0, 0)        \
  X(1, 2, 1, 0, 0)        \
  X(2, 1, -1, 0, 0)       \
  X(3, 4, 0, 1, 0)        \
  X(4, 3, 0, -1, 0)       \
  X(5, 6, 0, 0, 1)        \
  X(6, 5, 0, 0, -1)       \
  X(7, 8, 1, 1, 1)        \
  X(8, 7, -1, -1, -1)     \
  X(9, 10, 1, 1, -1)      \
  X(10, 9, -1, -1, 1)     \
  X(11, 12, 1, -1, 1)     \
  X(12, 11, -1, 1, -1)    \
  X(13, 14, 1, -1, -1)    \
  X(14, 13, -1, 1, 1)

template <int P, int S = kF32>
__device__ __forceinline__ void load_f(const float* a, int idx, const Nbr& nb, float f[7]) {
#define X(I, O, CX, CY, CZ) f[I] = pop_load<S, P, I, O, CX, CY, CZ>(a, idx, nb);
  LBM_D3Q7_LIST(X)
#undef X
}

template <int P, int S = kF32>
__device__ __forceinline__ void store_f(float* a, int idx, const Nbr& nb, const float f[7]) {
#define X(I, O, CX, CY, CZ) pop_store<S, P, I, O, CX, CY, CZ>(a, idx, nb, f[I]);
  LBM_D3Q7_LIST(X)
#undef X
}

template <int P, int S = kF32>
__device__ __forceinline__ void place_f(float* a, int idx, const Nbr& nb, const float f[7]) {
#define X(I, O, CX, CY, CZ) pop_place<S, P, I, O, CX, CY, CZ>(a, idx, nb, f[I]);
  LBM_D3Q7_LIST(X)
#undef X
}

template <int P, int S = kF32>
__device__ __forceinline__ void load_g(const float* a, int idx, const Nbr& nb, float g[15]) {
#define X(I, O, CX, CY, CZ) g[I] = pop_load<S, P, 7 + I, 7 + O, CX, CY, CZ>(a, idx, nb);
  LBM_D3Q15_LIST(X)
#undef X
}

template <int P, int S = kF32>
__device__ __forceinline__ void store_g(float* a, int idx, const Nbr& nb, const float g[15]) {
#define X(I, O, CX, CY, CZ) pop_store<S, P, 7 + I, 7 + O, CX, CY, CZ>(a, idx, nb, g[I]);
  LBM_D3Q15_LIST(X)
#undef X
}

template <int P, int S = kF32>
__device__ __forceinline__ void place_g(float* a, int idx, const Nbr& nb, const float g[15]) {
#define X(I, O, CX, CY, CZ) pop_place<S, P, 7 + I, 7 + O, CX, CY, CZ>(a, idx, nb, g[I]);
  LBM_D3Q15_LIST(X)
#undef X
}

// ---------------------------------------------------------------------------------
// Paired FP32 arithmetic.  Blackwell issues two FP32 additions, products or fused
// multiply-adds as one instruction (__fadd2_rn, __fmul2_rn, __ffma2_rn), each lane
// rounded exactly like the scalar operation.  The per-cell transforms below pair
// operations of the same form on independent values (mirrored population pairs, x and
// y components), which cuts the instructions the stream-collide kernel issues.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ float2 pr(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as b * (-1) + a: the product is exact, so each lane rounds like a - b
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// ---------------------------------------------------------------------------------
// Isotropic difference schemes on the 15-point D3Q15 stencil (Eqs. 35-36 with the
// flow-lattice weights 1/9 (faces), 1/72 (corners) and c_s^2 = 1/3):
//   grad chi = 1/3 (face differences) + 1/24 (corner differences)
//   lap chi  = 2/3 sum_faces (chi_n - chi) + 1/12 sum_corners (chi_n - chi)
// ---------------------------------------------------------------------------------
struct Stencil {
  float c;                      // centre
  float xm, xp, ym, yp, zm, zp; // faces
  float k[8];                   // corners, k[(sz > 0) * 4 + (sy > 0) * 2 + (sx > 0)]
};

__device__ __forceinline__ void load_stencil(const float* __restrict__ a, int idx, const Nbr& nb,
                                             Stencil& s) {
  s.c = __ldg(a + idx);
  s.xm = __ldg(a + idx + nb.xm);
  s.xp = __ldg(a + idx + nb.xp);
  s.ym = __ldg(a + idx + nb.ym);
  s.yp = __ldg(a + idx + nb.yp);
  s.zm = __ldg(a + idx + nb.zm);
  s.zp = __ldg(a + idx + nb.zp);
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int ox = (b & 1) ? nb.xp : nb.xm;
    const int oy = (b & 2) ? nb.yp : nb.ym;
    const int oz = (b & 4) ? nb.zp : nb.zm;
    s.k[b] = __ldg(a + idx + ox + oy + oz);
  }
}

// The same schemes with the D3Q7 weights (omega_i / c_s^2 = 1/2 for every A): plain
// central differences on the 6 faces.
__device__ __forceinline__ float stencil_lap7(const Stencil& s) {
  return ((s.xm + s.xp) + (s.ym + s.yp) + (s.zm + s.zp)) - 6.0f * s.c;
}

__device__ __forceinline__ void stencil_grad7(const Stencil& s, float g[3]) {
  g[0] = 0.5f * (s.xp - s.xm);
  g[1] = 0.5f * (s.yp - s.ym);
  g[2] = 0.5f * (s.zp - s.zm);
}

__device__ __forceinline__ float stencil_lap(const Stencil& s) {
  const float2 fxy = padd(pr(s.xm, s.ym), pr(s.xp, s.yp));
  const float faces = (fxy.x + fxy.y) + (s.zm + s.zp);
  // (k0 + k1 + k4 + k5, k2 + k3 + k6 + k7)
  const float2 c = padd(padd(pr(s.k[0], s.k[2]), pr(s.k[1], s.k[3])),
                        padd(pr(s.k[4], s.k[6]), pr(s.k[5], s.k[7])));
  const float corners = c.x + c.y;
  return (2.0f / 3.0f) * (faces - 6.0f * s.c) + (1.0f / 12.0f) * (corners - 8.0f * s.c);
}

// Corner sums sum_corners c_a chi: the x differences and x sums of the four (y, z)
// rows of corners, paired as (y-, y+) per z plane, then combined along y and z.
__device__ __forceinline__ void stencil_grad(const Stencil& s, float g[3]) {
  const float2 lo0 = pr(s.k[0], s.k[2]), hi0 = pr(s.k[1], s.k[3]);  // z- plane: x-, x+
  const float2 lo1 = pr(s.k[4], s.k[6]), hi1 = pr(s.k[5], s.k[7]);  // z+ plane
  const float2 dx = padd(psub(hi0, lo0), psub(hi1, lo1));  // x differences, (y-, y+)
  const float2 sx0 = padd(hi0, lo0), sx1 = padd(hi1, lo1);  // x sums, (y-, y+) per plane
  const float2 sy = padd(sx0, sx1);                          // (y- total, y+ total)
  const float2 sz = psub(sx1, sx0);                          // z+ minus z-, (y-, y+)
  const float kx = dx.x + dx.y, ky = sy.y - sy.x, kz = sz.x + sz.y;
  const float2 gxy = pfma(pr(1.0f / 24.0f, 1.0f / 24.0f), pr(kx, ky),
                          pmul(pr(1.0f / 3.0f, 1.0f / 3.0f), psub(pr(s.xp, s.yp), pr(s.xm, s.ym))));
  g[0] = gxy.x;
  g[1] = gxy.y;
  g[2] = (1.0f / 3.0f) * (s.zp - s.zm) + (1.0f / 24.0f) * kz;
}

// u(x, t) of the interface-tracking tests at node (x, y, z) (nodes at integer
// coordinates of a periodic box); tf is the time factor (cos(pi t / T) for the
// deformation field, 1 otherwise).
//   uniform:     (U, 0, 0)
//   rotation:    Eq. 37, v = -Omega (z - N/2), w = Omega (y - N/2), Omega = U pi / N, N = ny
//   deformation: Eq. 41 with L = nx.
__device__ __forceinline__ void prescribed_velocity(const Physics& ph, const Geometry& geo, int x,
                                                    int y, int z, float tf, float u[3]) {
  const float U = ph.vel_U;
  if (ph.vel_kind == kVelUniform) {
    u[0] = U;
    u[1] = 0.0f;
    u[2] = 0.0f;
  } else if (ph.vel_kind == kVelRotation) {
    const float omega = U * 3.14159265358979f / static_cast<float>(geo.ny);
    const float c = 0.5f * static_cast<float>(geo.ny);
    u[0] = 0.0f;
    u[1] = -omega * (static_cast<float>(z) - c);
    u[2] = omega * (static_cast<float>(y) - c);
  } else {
    const float inv_l = 1.0f / static_cast<float>(geo.nx);
    const float ax = static_cast<float>(x) * inv_l, ay = static_cast<float>(y) * inv_l,
                az = static_cast<float>(z) * inv_l;
    const float sx = sinpif(ax), sy = sinpif(ay), sz = sinpif(az);
    const float s2x = sinpif(2.0f * ax), s2y = sinpif(2.0f * ay), s2z = sinpif(2.0f * az);
    u[0] = 2.0f * U * sx * sx * s2y * s2z * tf;
    u[1] = -U * s2x * sy * sy * s2z * tf;
    u[2] = -U * s2x * s2y * sz * sz * tf;
  }
}

// mu = 4 beta phi (phi^2 - 1) - kappa lap phi (Eq. 2).
__device__ __forceinline__ float chemical_potential(const Physics& ph, float phi, float lap_phi) {
  return 4.0f * ph.beta * phi * (phi * phi - 1.0f) - ph.kappa * lap_phi;
}

// ---------------------------------------------------------------------------------
// Macroscopic state of one cell from its D3Q15 populations and the stencils.
// ---------------------------------------------------------------------------------
struct Macro {
  float rho, p;
  float u[3];
  float grad_rho[3];
  float F[3];  // F_s + F_a + G
};

// Moments of the D3Q15 populations (rows of Gamma, Eq. 25) and sum_{i != 0} g_i.
struct Moments15 {
  float m[15];
  float moving;
};

// The opposite pairs are taken as butterflies, two at a time: (1, 3) with (2, 4) gives
// the x and y axes; the corners pair by c_y, (7, 9) | (8, 10) for c_y = +1 and
// (11, 13) | (12, 14) for c_y = -1, and two more butterfly levels give their moments.
__device__ __forceinline__ Moments15 moments15(const float g[15]) {
  Moments15 r;
  const float2 A = pr(g[1], g[3]), B = pr(g[2], g[4]);
  const float2 s_xy = padd(A, B), d_xy = psub(A, B);  // (sx, sy), (dx, dy)
  const float sz = g[5] + g[6], dz = g[5] - g[6];
  const float2 c1 = pr(g[7], g[9]), c2 = pr(g[8], g[10]);
  const float2 c3 = pr(g[11], g[13]), c4 = pr(g[12], g[14]);
  const float2 sa_ = padd(c1, c2), da = psub(c1, c2);  // (s7, s9), (d7, d9)
  const float2 sb = padd(c3, c4), db = psub(c3, c4);   // (s11, s13), (d11, d13)
  const float2 sp = padd(sa_, sb), sm = psub(sa_, sb);  // (s7 + s11, s9 + s13), (s7 - s11, s9 - s13)
  const float2 dp = padd(da, db), dm = psub(da, db);    // likewise for d
  const float C = sp.x + sp.y;                          // sum over the 8 corners
  const float2 Cxy = pr(dp.x + dp.y, dm.x + dm.y);      // sum c_x g, sum c_y g over corners
  const float Cz = dp.x - dp.y;
  const float sa = s_xy.x + s_xy.y + sz;
  r.moving = sa + C;
  r.m[0] = g[0] + sa + C;
  r.m[1] = -2.0f * g[0] - sa + C;
  r.m[2] = 16.0f * g[0] - 4.0f * sa + C;
  const float2 m35 = padd(d_xy, Cxy), m46 = pfma(pr(-4.0f, -4.0f), d_xy, Cxy);
  r.m[3] = m35.x;
  r.m[4] = m46.x;
  r.m[5] = m35.y;
  r.m[6] = m46.y;
  r.m[7] = dz + Cz;
  r.m[8] = -4.0f * dz + Cz;
  r.m[9] = 2.0f * s_xy.x - s_xy.y - sz;
  r.m[10] = s_xy.y - sz;
  r.m[11] = sm.x + sm.y;  // c_x c_y
  r.m[12] = sm.x - sm.y;  // c_y c_z
  r.m[13] = sp.x - sp.y;  // c_x c_z
  r.m[14] = dm.x - dm.y;  // c_x c_y c_z
  return r;
}

// Eqs. 14, 29, 30 and the forces of Eq. 28, from the moments of the populations.
__device__ __forceinline__ Macro macroscopic(const Physics& ph, const Moments15& mo, float phi,
                                             float mu, const float grad_phi[3], float lap_mu) {
  Macro m;
  m.rho = ph.rho_g + (1.0f + phi) * ph.half_drho;
  // lattice momentum sum_i c_i g_i and sum_{i != 0} g_i
  const float jx = mo.m[3], jy = mo.m[5], jz = mo.m[7];
  const float sum_moving = mo.moving;
  float Fsg[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    m.grad_rho[a] = ph.half_drho * grad_phi[a];
    Fsg[a] = mu * grad_phi[a] + (m.rho - ph.rho_ref) * ph.gacc[a];  // F_s + G
  }
  const float fa = ph.half_drho * ph.mob * lap_mu;  // F_a = fa * u
  const float inv = __fdividef(1.0f, m.rho - 0.5f * fa);
  m.u[0] = (jx + 0.5f * Fsg[0]) * inv;
  m.u[1] = (jy + 0.5f * Fsg[1]) * inv;
  m.u[2] = (jz + 0.5f * Fsg[2]) * inv;
  const float uu = m.u[0] * m.u[0] + m.u[1] * m.u[1] + m.u[2] * m.u[2];
  const float udr = m.u[0] * m.grad_rho[0] + m.u[1] * m.grad_rho[1] + m.u[2] * m.grad_rho[2];
  // c_s^2/(1 - omega_0) = 3/7; rho s_0(u) = -rho u^2 / 3
  m.p = (3.0f / 7.0f) * (sum_moving + 0.5f * udr - m.rho * uu * (1.0f / 3.0f));
#pragma unroll
  for (int a = 0; a < 3; ++a) m.F[a] = Fsg[a] + fa * m.u[a];
  return m;
}

// ---------------------------------------------------------------------------------
// D3Q15 MRT collision in moment space (Eqs. 20, 26, 31, 32):
//   m+ = m - S (m - m^eq) + (I - S/2) mT,   g+ = Gamma^{-1} m+
// written as g+ = g - Gamma^{-1} Delta with Delta = S (m - m^eq) - (I - S/2) mT, so
// that the small correction is what passes through the FP32 back-transform.
// Gamma^{-1} = Gamma^T diag(1/|row_k|^2), |row|^2 = 15,18,360,10,40,10,40,10,40,12,4,8,8,8,8.
// ---------------------------------------------------------------------------------
template <bool SRT = false>
__device__ __forceinline__ void collide_d3q15(const Physics& ph, float g[15], const Moments15& mo,
                                              const Macro& M, float lambda_visc) {
  const float* m = mo.m;

  // equilibrium moments, Eq. 31 (c = 1)
  const float rho = M.rho, p = M.p, ux = M.u[0], uy = M.u[1], uz = M.u[2];
  const float uu = ux * ux + uy * uy + uz * uz;
  float meq[15];
  meq[0] = 0.0f;
  meq[1] = 3.0f * p + rho * uu;
  meq[2] = -(45.0f * p + 5.0f * rho * uu);
  meq[3] = rho * ux;
  meq[4] = (-7.0f / 3.0f) * rho * ux;
  meq[5] = rho * uy;
  meq[6] = (-7.0f / 3.0f) * rho * uy;
  meq[7] = rho * uz;
  meq[8] = (-7.0f / 3.0f) * rho * uz;
  meq[9] = rho * (2.0f * ux * ux - uy * uy - uz * uz);
  meq[10] = rho * (uy * uy - uz * uz);
  meq[11] = rho * ux * uy;
  meq[12] = rho * uy * uz;
  meq[13] = rho * ux * uz;
  meq[14] = 0.0f;

  // forcing moments, Eq. 32 (c = 1, X = c_s^2 grad rho)
  const float Xx = M.grad_rho[0] * (1.0f / 3.0f), Xy = M.grad_rho[1] * (1.0f / 3.0f),
              Xz = M.grad_rho[2] * (1.0f / 3.0f);
  const float Fx = M.F[0], Fy = M.F[1], Fz = M.F[2];
  const float Yx = Xx + Fx, Yy = Xy + Fy, Yz = Xz + Fz;
  const float udX = ux * Xx + uy * Xy + uz * Xz;
  const float udF = ux * Fx + uy * Fy + uz * Fz;
  float mT[15];
  mT[0] = 3.0f * udX;  // u . grad rho
  mT[1] = -udX + 2.0f * udF;
  mT[2] = -(7.0f * udX + 10.0f * udF);
  mT[3] = Fx;
  mT[4] = (-7.0f / 3.0f) * Fx;
  mT[5] = Fy;
  mT[6] = (-7.0f / 3.0f) * Fy;
  mT[7] = Fz;
  mT[8] = (-7.0f / 3.0f) * Fz;
  mT[9] = 4.0f * ux * Yx - 2.0f * uy * Yy - 2.0f * uz * Yz;
  mT[10] = 2.0f * uy * Yy - 2.0f * uz * Yz;
  mT[11] = ux * Yy + uy * Yx;
  mT[12] = uy * Yz + uz * Yy;
  mT[13] = ux * Yz + uz * Yx;
  mT[14] = 0.0f;

  // Delta_k / |row_k|^2; the fixed rates come divided by the norms
  float a[15];
  const float keep_visc = 1.0f - 0.5f * lambda_visc;
#pragma unroll
  for (int k = 0; k < 15; ++k) {
    if (SRT || (k >= 9 && k <= 13))
      a[k] = (lambda_visc * (m[k] - meq[k]) - keep_visc * mT[k]) * (1.0f / norm15(k));
    else
      a[k] = ph.sg_a[k] * (m[k] - meq[k]) - ph.sg_b[k] * mT[k];
  }

  // back transform: g_i -= sum_k Gamma_ki a_k
  const float e_axis = a[0] - a[1] - 4.0f * a[2];
  g[0] -= a[0] - 2.0f * a[1] + 16.0f * a[2];
  {
    // axis v: g(+v) -= e_v + o_v, g(-v) -= e_v - o_v; x and y paired, then z
    const float2 o_xy = pfma(pr(-4.0f, -4.0f), pr(a[4], a[6]), pr(a[3], a[5]));
    const float2 e_xy = pr(e_axis + 2.0f * a[9], e_axis - a[9] + a[10]);
    const float2 gp = psub(pr(g[1], g[3]), padd(e_xy, o_xy));
    const float2 gm = psub(pr(g[2], g[4]), psub(e_xy, o_xy));
    g[1] = gp.x;
    g[3] = gp.y;
    g[2] = gm.x;
    g[4] = gm.y;
    const float oz = a[7] - 4.0f * a[8], ez = e_axis - a[9] - a[10];
    g[5] -= ez + oz;
    g[6] -= ez - oz;
  }
  {
    // corner v = (vx, vy, vz): g(+v) -= even + odd, g(-v) -= even - odd, with
    // even = e0 + vx vy a11 + vy vz a12 + vx vz a13 and odd = vx px + vy py + vz pz +
    // vx vy vz a14.  The corners with vx = 1 pair as (vz = +1, vz = -1): (7, 9) for
    // vy = +1, (11, 13) for vy = -1; then
    //   even = (e0 + vz a13) + vy (a11 + vz a12),  odd = (px + vz pz) + vy (py + vz a14)
    const float e0 = a[0] + a[1] + a[2];
    const float px = a[3] + a[4], py = a[5] + a[6], pz = a[7] + a[8];
    const float2 P = pr(e0 + a[13], e0 - a[13]), Q = pr(a[11] + a[12], a[11] - a[12]);
    const float2 R = pr(px + pz, px - pz), T = pr(py + a[14], py - a[14]);
    const float2 e_up = padd(P, Q), e_dn = psub(P, Q);  // vy = +1, -1
    const float2 o_up = padd(R, T), o_dn = psub(R, T);
    const float2 g79 = psub(pr(g[7], g[9]), padd(e_up, o_up));
    const float2 g810 = psub(pr(g[8], g[10]), psub(e_up, o_up));
    const float2 g1113 = psub(pr(g[11], g[13]), padd(e_dn, o_dn));
    const float2 g1214 = psub(pr(g[12], g[14]), psub(e_dn, o_dn));
    g[7] = g79.x;
    g[9] = g79.y;
    g[8] = g810.x;
    g[10] = g810.y;
    g[11] = g1113.x;
    g[13] = g1113.y;
    g[12] = g1214.x;
    g[14] = g1214.y;
  }
}

// ---------------------------------------------------------------------------------
// D3Q7 MRT collision in moment space (Eqs. 15, 17, 18):
//   m+ = m - S (m - m^eq) + (I - S/2) mR,   f+ = M^{-1} m+
// again applied as f+ = f - M^{-1} Delta; |row|^2 of M = 7, 2, 2, 2, 42, 12, 4.
// ---------------------------------------------------------------------------------
// With SHIFT0 (16-bit storage) f[0] is not read: f_0 = phi - sum_{i>0} f_i, so
// m_0 = phi and m_4 = 6 phi - 7 sum_{i>0} f_i; on return f[0] holds f_0^+ - phi.
// Every scalar product and sum here is written with an explicit rounding intrinsic
// (__fmul_rn, __fadd_rn, __fsub_rn, __fmaf_rn), which the compiler never contracts or
// splits, so the result is the same bits in every kernel that inlines it (left to
// itself, the compiler fused different multiply-add pairs in different kernels).
template <bool SHIFT0 = false>
__device__ __forceinline__ void collide_d3q7(const Physics& ph, float f[7], float phi, float mu,
                                             const float u[3], const float dphiu[3]) {
  // x and y opposite pairs as paired butterflies, (1, 3) with (2, 4)
  const float2 fp = pr(f[1], f[3]), fm = pr(f[2], f[4]);
  const float2 s_xy = padd(fp, fm), d_xy = psub(fp, fm);
  const float sz = __fadd_rn(f[5], f[6]);
  const float smov = __fadd_rn(__fadd_rn(s_xy.x, s_xy.y), sz);
  float m[7];
  m[0] = SHIFT0 ? phi : __fadd_rn(f[0], smov);
  m[1] = d_xy.x;
  m[2] = d_xy.y;
  m[3] = __fsub_rn(f[5], f[6]);
  m[4] = SHIFT0 ? __fmaf_rn(6.0f, phi, __fmul_rn(-7.0f, smov)) : __fmaf_rn(6.0f, f[0], -smov);
  m[5] = __fsub_rn(__fmaf_rn(2.0f, s_xy.x, -s_xy.y), sz);
  m[6] = __fsub_rn(s_xy.y, sz);
  // m - m^eq (Eq. 17); rows 0, 5, 6 have m^eq = phi, 0, 0
  const float k4 = __fmul_rn(__fmul_rn(21.0f, ph.A), ph.eta);
  float d[7];
  d[0] = __fsub_rn(m[0], phi);
  d[1] = __fsub_rn(m[1], __fmul_rn(phi, u[0]));
  d[2] = __fsub_rn(m[2], __fmul_rn(phi, u[1]));
  d[3] = __fsub_rn(m[3], __fmul_rn(phi, u[2]));
  d[4] = __fsub_rn(m[4], __fmaf_rn(-k4, mu, __fmul_rn(6.0f, phi)));
  d[5] = m[5];
  d[6] = m[6];
  // b_k = [s_k (m_k - m_k^eq) - (1 - s_k/2) mR_k] / |M_k|^2 with mR of Eq. 18
  float b[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    if (k >= 1 && k <= 3)
      b[k] = __fmaf_rn(ph.sf_a[k], d[k], __fmul_rn(-ph.sf_b[k], dphiu[k - 1]));
    else
      b[k] = __fmul_rn(ph.sf_a[k], d[k]);
  }
  const float e = __fsub_rn(b[0], b[4]);
  const float c0 = __fmaf_rn(6.0f, b[4], b[0]);
  if (SHIFT0)
    f[0] = -__fadd_rn(smov, c0);
  else
    f[0] = __fsub_rn(f[0], c0);
  const float2 e_xy = pr(__fmaf_rn(2.0f, b[5], e), __fadd_rn(__fsub_rn(e, b[5]), b[6]));
  const float2 b12 = pr(b[1], b[2]);
  const float2 up = psub(fp, padd(e_xy, b12)), dn = psub(fm, psub(e_xy, b12));
  f[1] = up.x;
  f[3] = up.y;
  f[2] = dn.x;
  f[4] = dn.y;
  const float ez = __fsub_rn(__fsub_rn(e, b[5]), b[6]);
  f[5] = __fsub_rn(f[5], __fadd_rn(ez, b[3]));
  f[6] = __fsub_rn(f[6], __fsub_rn(ez, b[3]));
}

}  // namespace lbm
