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
  int pairs;             // 1: the stream-collide takes two cells per thread (k_collide2,
                         // either pattern; needs nx a multiple of 2 kTile)
  int stage;             // 1: k_collide2 stages the phi and mu stencils in shared memory
                         // by TMA bulk copies (k_collide2t; needs pairs and nx of 64,
                         // 128 or 256)
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
// Per-cell arithmetic, generic over the lane type V: float for one cell per thread,
// float2 for two cells per thread (one in each lane, the paired FP32 instructions
// __fadd2_rn, __fmul2_rn, __ffma2_rn doing both cells at once).  Every sum, product
// and fused multiply-add is written with an explicit rounding intrinsic, which the
// compiler never contracts or splits; each lane of a paired instruction rounds like
// the scalar one.  So a cell's values are the same bits whichever kernel, lane type or
// number of cells per thread computes them.
// ---------------------------------------------------------------------------------
template <typename V>
struct VOps;

template <>
struct VOps<float> {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  static __device__ __forceinline__ float neg(float a) { return -a; }
  static __device__ __forceinline__ float k(float a) { return a; }
  static __device__ __forceinline__ float rcp(float a) { return __fdividef(1.0f, a); }
};

template <>
struct VOps<float2> {
  static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
  // a - b as b * (-1) + a: the product is exact, so each lane rounds like a - b
  static __device__ __forceinline__ float2 sub(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
  }
  static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
  static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) {
    return __ffma2_rn(a, b, c);
  }
  static __device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
  static __device__ __forceinline__ float2 k(float a) { return make_float2(a, a); }
  static __device__ __forceinline__ float2 rcp(float2 a) {
    return make_float2(__fdividef(1.0f, a.x), __fdividef(1.0f, a.y));
  }
};

// Stencil of one scalar field around the cell(s): centre, 6 faces, 8 corners.
template <typename V>
struct StencilV {
  V c;                    // centre
  V xm, xp, ym, yp, zm, zp;  // faces
  V k[8];                 // corners, k[(sz > 0) * 4 + (sy > 0) * 2 + (sx > 0)]
};
typedef StencilV<float> Stencil;

// The difference schemes with the D3Q7 weights (omega_i / c_s^2 = 1/2 for every A):
// plain central differences on the 6 faces.
template <typename V>
__device__ __forceinline__ V stencil_lap7(const StencilV<V>& s) {
  typedef VOps<V> O;
  const V faces = O::add(O::add(O::add(s.xm, s.xp), O::add(s.ym, s.yp)), O::add(s.zm, s.zp));
  return O::fma(O::k(-6.0f), s.c, faces);
}

template <typename V>
__device__ __forceinline__ void stencil_grad7(const StencilV<V>& s, V g[3]) {
  typedef VOps<V> O;
  g[0] = O::mul(O::k(0.5f), O::sub(s.xp, s.xm));
  g[1] = O::mul(O::k(0.5f), O::sub(s.yp, s.ym));
  g[2] = O::mul(O::k(0.5f), O::sub(s.zp, s.zm));
}

// Isotropic difference schemes on the 15-point D3Q15 stencil (Eqs. 35-36 with the
// flow-lattice weights 1/9 (faces), 1/72 (corners) and c_s^2 = 1/3):
//   lap chi  = 2/3 sum_faces (chi_n - chi) + 1/12 sum_corners (chi_n - chi)
//   grad chi = 1/3 (face differences) + 1/24 (corner differences)
template <typename V>
__device__ __forceinline__ V stencil_lap(const StencilV<V>& s) {
  typedef VOps<V> O;
  const V faces = O::add(O::add(O::add(s.xm, s.xp), O::add(s.ym, s.yp)), O::add(s.zm, s.zp));
  const V corners = O::add(O::add(O::add(s.k[0], s.k[1]), O::add(s.k[4], s.k[5])),
                           O::add(O::add(s.k[2], s.k[3]), O::add(s.k[6], s.k[7])));
  return O::fma(O::k(2.0f / 3.0f), O::fma(O::k(-6.0f), s.c, faces),
                O::mul(O::k(1.0f / 12.0f), O::fma(O::k(-8.0f), s.c, corners)));
}

// Corner sums sum_corners c_a chi from the x differences and x sums of the four (y, z)
// rows of corners.
template <typename V>
__device__ __forceinline__ void stencil_grad(const StencilV<V>& s, V g[3]) {
  typedef VOps<V> O;
  // rows of corners: (z-, y-) = k0, k1; (z-, y+) = k2, k3; (z+, y-) = k4, k5; (z+, y+) = k6, k7
  const V dx0 = O::sub(s.k[1], s.k[0]), dx1 = O::sub(s.k[3], s.k[2]);
  const V dx2 = O::sub(s.k[5], s.k[4]), dx3 = O::sub(s.k[7], s.k[6]);
  const V sx0 = O::add(s.k[1], s.k[0]), sx1 = O::add(s.k[3], s.k[2]);
  const V sx2 = O::add(s.k[5], s.k[4]), sx3 = O::add(s.k[7], s.k[6]);
  const V kx = O::add(O::add(dx0, dx2), O::add(dx1, dx3));
  const V ky = O::sub(O::add(sx1, sx3), O::add(sx0, sx2));
  const V kz = O::add(O::sub(sx2, sx0), O::sub(sx3, sx1));
  const V third = O::k(1.0f / 3.0f), w = O::k(1.0f / 24.0f);
  g[0] = O::fma(w, kx, O::mul(third, O::sub(s.xp, s.xm)));
  g[1] = O::fma(w, ky, O::mul(third, O::sub(s.yp, s.ym)));
  g[2] = O::fma(w, kz, O::mul(third, O::sub(s.zp, s.zm)));
}

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
  return __fmaf_rn(__fmul_rn(4.0f * ph.beta, phi), __fmaf_rn(phi, phi, -1.0f),
                   __fmul_rn(-ph.kappa, lap_phi));
}

// The 15-point Laplacian of Eq. 36 at a node from per-plane partial sums of its column:
// centres c0, c1, c2 of the planes below, at and above the node, the sum f1 of the 4
// in-plane face neighbours at the node's plane, and the sums d0, d2 of the 4 in-plane
// diagonal neighbours of the planes below and above (the stencil's corners):
//   2/3 (faces - 6 c1) + 1/12 (corners - 8 c1)
__device__ __forceinline__ float lap15_columns(float c0, float c1, float c2, float f1, float d0,
                                               float d2) {
  return __fmaf_rn(2.0f / 3.0f, __fmaf_rn(-6.0f, c1, __fadd_rn(f1, __fadd_rn(c0, c2))),
                   __fmul_rn(1.0f / 12.0f, __fmaf_rn(-8.0f, c1, __fadd_rn(d0, d2))));
}

// The same with the D3Q7 weights: faces - 6 c1.
__device__ __forceinline__ float lap7_columns(float c0, float c1, float c2, float f1) {
  return __fmaf_rn(-6.0f, c1, __fadd_rn(f1, __fadd_rn(c0, c2)));
}

// ---------------------------------------------------------------------------------
// Macroscopic state of the cell(s) from the D3Q15 populations and the stencils.
// ---------------------------------------------------------------------------------
template <typename V>
struct MacroV {
  V rho, p;
  V u[3];
  V grad_rho[3];
  V F[3];  // F_s + F_a + G
};
typedef MacroV<float> Macro;

// Moments of the D3Q15 populations (rows of Gamma, Eq. 25) and sum_{i != 0} g_i.
template <typename V>
struct Moments15V {
  V m[15];
  V moving;
};
typedef Moments15V<float> Moments15;

// Opposite pairs as butterflies: axis sums and differences, the corners paired by
// opposites and then by the sign of c_y.
template <typename V>
__device__ __forceinline__ Moments15V<V> moments15(const V g[15]) {
  typedef VOps<V> O;
  Moments15V<V> r;
  const V sx = O::add(g[1], g[2]), dx = O::sub(g[1], g[2]);
  const V sy = O::add(g[3], g[4]), dy = O::sub(g[3], g[4]);
  const V sz = O::add(g[5], g[6]), dz = O::sub(g[5], g[6]);
  const V s7 = O::add(g[7], g[8]), d7 = O::sub(g[7], g[8]);
  const V s9 = O::add(g[9], g[10]), d9 = O::sub(g[9], g[10]);
  const V s11 = O::add(g[11], g[12]), d11 = O::sub(g[11], g[12]);
  const V s13 = O::add(g[13], g[14]), d13 = O::sub(g[13], g[14]);
  const V spx = O::add(s7, s11), spy = O::add(s9, s13);  // c_y = +1 corners paired with c_y = -1
  const V smx = O::sub(s7, s11), smy = O::sub(s9, s13);
  const V dpx = O::add(d7, d11), dpy = O::add(d9, d13);
  const V dmx = O::sub(d7, d11), dmy = O::sub(d9, d13);
  const V C = O::add(spx, spy);   // sum over the 8 corners
  const V Cx = O::add(dpx, dpy);  // sum c_x g over the corners
  const V Cy = O::add(dmx, dmy);  // sum c_y g
  const V Cz = O::sub(dpx, dpy);  // sum c_z g
  const V sa = O::add(O::add(sx, sy), sz);
  r.moving = O::add(sa, C);
  r.m[0] = O::add(O::add(g[0], sa), C);
  r.m[1] = O::add(O::fma(O::k(-2.0f), g[0], O::neg(sa)), C);
  r.m[2] = O::add(O::fma(O::k(16.0f), g[0], O::mul(O::k(-4.0f), sa)), C);
  r.m[3] = O::add(dx, Cx);
  r.m[4] = O::fma(O::k(-4.0f), dx, Cx);
  r.m[5] = O::add(dy, Cy);
  r.m[6] = O::fma(O::k(-4.0f), dy, Cy);
  r.m[7] = O::add(dz, Cz);
  r.m[8] = O::fma(O::k(-4.0f), dz, Cz);
  r.m[9] = O::sub(O::fma(O::k(2.0f), sx, O::neg(sy)), sz);
  r.m[10] = O::sub(sy, sz);
  r.m[11] = O::add(smx, smy);  // c_x c_y
  r.m[12] = O::sub(smx, smy);  // c_y c_z
  r.m[13] = O::sub(spx, spy);  // c_x c_z
  r.m[14] = O::sub(dmx, dmy);  // c_x c_y c_z
  return r;
}

// Eqs. 14, 29, 30 and the forces of Eq. 28, from the moments of the populations.
template <typename V>
__device__ __forceinline__ MacroV<V> macroscopic(const Physics& ph, const Moments15V<V>& mo, V phi,
                                                 V mu, const V grad_phi[3], V lap_mu) {
  typedef VOps<V> O;
  MacroV<V> m;
  m.rho = O::fma(O::add(O::k(1.0f), phi), O::k(ph.half_drho), O::k(ph.rho_g));
  const V j[3] = {mo.m[3], mo.m[5], mo.m[7]};  // lattice momentum sum_i c_i g_i
  const V wrho = O::sub(m.rho, O::k(ph.rho_ref));
  V Fsg[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    m.grad_rho[a] = O::mul(O::k(ph.half_drho), grad_phi[a]);
    Fsg[a] = O::fma(mu, grad_phi[a], O::mul(wrho, O::k(ph.gacc[a])));  // F_s + G
  }
  const V fa = O::mul(O::k(ph.half_drho * ph.mob), lap_mu);  // F_a = fa * u
  const V inv = O::rcp(O::fma(O::k(-0.5f), fa, m.rho));
#pragma unroll
  for (int a = 0; a < 3; ++a) m.u[a] = O::mul(O::fma(O::k(0.5f), Fsg[a], j[a]), inv);
  const V uu = O::fma(m.u[0], m.u[0], O::fma(m.u[1], m.u[1], O::mul(m.u[2], m.u[2])));
  const V udr = O::fma(m.u[0], m.grad_rho[0],
                       O::fma(m.u[1], m.grad_rho[1], O::mul(m.u[2], m.grad_rho[2])));
  // c_s^2/(1 - omega_0) = 3/7; rho s_0(u) = -rho u^2 / 3
  m.p = O::mul(O::k(3.0f / 7.0f),
               O::fma(O::k(-1.0f / 3.0f), O::mul(m.rho, uu), O::fma(O::k(0.5f), udr, mo.moving)));
#pragma unroll
  for (int a = 0; a < 3; ++a) m.F[a] = O::fma(fa, m.u[a], Fsg[a]);
  return m;
}

// lambda_9..13 = 1 / tau_g with nu = c_s^2 (tau_g - 1/2) (Eq. 33), nu linear in phi.
template <typename V>
__device__ __forceinline__ V viscous_rate(const Physics& ph, V phi) {
  typedef VOps<V> O;
  return O::rcp(O::fma(O::k(3.0f), O::fma(phi, O::k(ph.half_dnu), O::k(ph.nu_mid)), O::k(0.5f)));
}

// ---------------------------------------------------------------------------------
// D3Q15 MRT collision in moment space (Eqs. 20, 26, 31, 32):
//   m+ = m - S (m - m^eq) + (I - S/2) mT,   g+ = Gamma^{-1} m+
// written as g+ = g - Gamma^{-1} Delta with Delta = S (m - m^eq) - (I - S/2) mT, so
// that the small correction is what passes through the FP32 back-transform.
// Gamma^{-1} = Gamma^T diag(1/|row_k|^2), |row|^2 = 15,18,360,10,40,10,40,10,40,12,4,8,8,8,8.
// ---------------------------------------------------------------------------------
template <bool SRT, typename V>
__device__ __forceinline__ void collide_d3q15(const Physics& ph, V g[15], const Moments15V<V>& mo,
                                              const MacroV<V>& M, V lambda_visc) {
  typedef VOps<V> O;
  const V* m = mo.m;
  const V rho = M.rho, p = M.p, ux = M.u[0], uy = M.u[1], uz = M.u[2];
  const V uxx = O::mul(ux, ux), uyy = O::mul(uy, uy), uzz = O::mul(uz, uz);
  const V ruu = O::mul(rho, O::add(O::add(uxx, uyy), uzz));
  const V rux = O::mul(rho, ux), ruy = O::mul(rho, uy), ruz = O::mul(rho, uz);
  // equilibrium moments, Eq. 31 (c = 1); rows 0 and 14 are 0
  V meq[15];
  meq[1] = O::fma(O::k(3.0f), p, ruu);
  meq[2] = O::neg(O::fma(O::k(45.0f), p, O::mul(O::k(5.0f), ruu)));
  meq[3] = rux;
  meq[4] = O::mul(O::k(-7.0f / 3.0f), rux);
  meq[5] = ruy;
  meq[6] = O::mul(O::k(-7.0f / 3.0f), ruy);
  meq[7] = ruz;
  meq[8] = O::mul(O::k(-7.0f / 3.0f), ruz);
  meq[9] = O::mul(rho, O::sub(O::fma(O::k(2.0f), uxx, O::neg(uyy)), uzz));
  meq[10] = O::mul(rho, O::sub(uyy, uzz));
  meq[11] = O::mul(rux, uy);
  meq[12] = O::mul(ruy, uz);
  meq[13] = O::mul(rux, uz);

  // forcing moments, Eq. 32 (c = 1, X = c_s^2 grad rho, Y = X + F)
  const V third = O::k(1.0f / 3.0f);
  const V Xx = O::mul(M.grad_rho[0], third), Xy = O::mul(M.grad_rho[1], third),
          Xz = O::mul(M.grad_rho[2], third);
  const V Fx = M.F[0], Fy = M.F[1], Fz = M.F[2];
  const V Yx = O::add(Xx, Fx), Yy = O::add(Xy, Fy), Yz = O::add(Xz, Fz);
  const V udX = O::fma(ux, Xx, O::fma(uy, Xy, O::mul(uz, Xz)));
  const V udF = O::fma(ux, Fx, O::fma(uy, Fy, O::mul(uz, Fz)));
  const V uYx = O::mul(ux, Yx), uYy = O::mul(uy, Yy), uYz = O::mul(uz, Yz);
  V mT[15];
  mT[0] = O::mul(O::k(3.0f), udX);  // u . grad rho
  mT[1] = O::fma(O::k(2.0f), udF, O::neg(udX));
  mT[2] = O::neg(O::fma(O::k(7.0f), udX, O::mul(O::k(10.0f), udF)));
  mT[3] = Fx;
  mT[4] = O::mul(O::k(-7.0f / 3.0f), Fx);
  mT[5] = Fy;
  mT[6] = O::mul(O::k(-7.0f / 3.0f), Fy);
  mT[7] = Fz;
  mT[8] = O::mul(O::k(-7.0f / 3.0f), Fz);
  mT[9] = O::fma(O::k(4.0f), uYx, O::mul(O::k(-2.0f), O::add(uYy, uYz)));
  mT[10] = O::mul(O::k(2.0f), O::sub(uYy, uYz));
  mT[11] = O::fma(ux, Yy, O::mul(uy, Yx));
  mT[12] = O::fma(uy, Yz, O::mul(uz, Yy));
  mT[13] = O::fma(ux, Yz, O::mul(uz, Yx));

  // Delta_k / |row_k|^2; the fixed rates come divided by the norms
  V a[15];
  const V keep = O::fma(O::k(-0.5f), lambda_visc, O::k(1.0f));
#pragma unroll
  for (int k = 0; k < 15; ++k) {
    const V d = (k == 0 || k == 14) ? m[k] : O::sub(m[k], meq[k]);
    const bool visc = SRT || (k >= 9 && k <= 13);
    if (k == 14) {
      a[k] = visc ? O::mul(O::mul(lambda_visc, d), O::k(1.0f / norm15(k)))
                  : O::mul(O::k(ph.sg_a[k]), d);
    } else if (visc) {
      a[k] = O::mul(O::fma(lambda_visc, d, O::mul(O::neg(keep), mT[k])), O::k(1.0f / norm15(k)));
    } else {
      a[k] = O::fma(O::k(ph.sg_a[k]), d, O::mul(O::k(-ph.sg_b[k]), mT[k]));
    }
  }

  // back transform: g_i -= sum_k Gamma_ki a_k
  const V e_axis = O::fma(O::k(-4.0f), a[2], O::sub(a[0], a[1]));
  g[0] = O::sub(g[0], O::fma(O::k(16.0f), a[2], O::fma(O::k(-2.0f), a[1], a[0])));
  {
    // axis v: g(+v) -= e_v + o_v, g(-v) -= e_v - o_v
    const V ox = O::fma(O::k(-4.0f), a[4], a[3]), oy = O::fma(O::k(-4.0f), a[6], a[5]);
    const V oz = O::fma(O::k(-4.0f), a[8], a[7]);
    const V ex = O::fma(O::k(2.0f), a[9], e_axis);
    const V em = O::sub(e_axis, a[9]);
    const V ey = O::add(em, a[10]), ez = O::sub(em, a[10]);
    g[1] = O::sub(g[1], O::add(ex, ox));
    g[2] = O::sub(g[2], O::sub(ex, ox));
    g[3] = O::sub(g[3], O::add(ey, oy));
    g[4] = O::sub(g[4], O::sub(ey, oy));
    g[5] = O::sub(g[5], O::add(ez, oz));
    g[6] = O::sub(g[6], O::sub(ez, oz));
  }
  {
    // corner v = (vx, vy, vz): g(+v) -= even + odd, g(-v) -= even - odd, with
    // even = e0 + vx vy a11 + vy vz a12 + vx vz a13 and odd = vx px + vy py + vz pz +
    // vx vy vz a14.  For the corners with vx = 1:
    //   even = (e0 + vz a13) + vy (a11 + vz a12),  odd = (px + vz pz) + vy (py + vz a14)
    const V e0 = O::add(O::add(a[0], a[1]), a[2]);
    const V px = O::add(a[3], a[4]), py = O::add(a[5], a[6]), pz = O::add(a[7], a[8]);
    const V Pp = O::add(e0, a[13]), Pm = O::sub(e0, a[13]);        // vz = +1, -1
    const V Qp = O::add(a[11], a[12]), Qm = O::sub(a[11], a[12]);
    const V Rp = O::add(px, pz), Rm = O::sub(px, pz);
    const V Tp = O::add(py, a[14]), Tm = O::sub(py, a[14]);
    const V eu7 = O::add(Pp, Qp), eu9 = O::add(Pm, Qm);  // vy = +1
    const V ed11 = O::sub(Pp, Qp), ed13 = O::sub(Pm, Qm);  // vy = -1
    const V ou7 = O::add(Rp, Tp), ou9 = O::add(Rm, Tm);
    const V od11 = O::sub(Rp, Tp), od13 = O::sub(Rm, Tm);
    g[7] = O::sub(g[7], O::add(eu7, ou7));
    g[8] = O::sub(g[8], O::sub(eu7, ou7));
    g[9] = O::sub(g[9], O::add(eu9, ou9));
    g[10] = O::sub(g[10], O::sub(eu9, ou9));
    g[11] = O::sub(g[11], O::add(ed11, od11));
    g[12] = O::sub(g[12], O::sub(ed11, od11));
    g[13] = O::sub(g[13], O::add(ed13, od13));
    g[14] = O::sub(g[14], O::sub(ed13, od13));
  }
}

// ---------------------------------------------------------------------------------
// D3Q7 MRT collision in moment space (Eqs. 15, 17, 18):
//   m+ = m - S (m - m^eq) + (I - S/2) mR,   f+ = M^{-1} m+
// again applied as f+ = f - M^{-1} Delta; |row|^2 of M = 7, 2, 2, 2, 42, 12, 4.
// With SHIFT0 (16-bit storage) f[0] is not read: f_0 = phi - sum_{i>0} f_i, so
// m_0 = phi and m_4 = 6 phi - 7 sum_{i>0} f_i; on return f[0] holds f_0^+ - phi.
// ---------------------------------------------------------------------------------
template <bool SHIFT0, typename V>
__device__ __forceinline__ void collide_d3q7(const Physics& ph, V f[7], V phi, V mu, const V u[3],
                                             const V dphiu[3]) {
  typedef VOps<V> O;
  const V sx = O::add(f[1], f[2]), dx = O::sub(f[1], f[2]);
  const V sy = O::add(f[3], f[4]), dy = O::sub(f[3], f[4]);
  const V sz = O::add(f[5], f[6]);
  const V smov = O::add(O::add(sx, sy), sz);
  V m[7];
  m[0] = SHIFT0 ? phi : O::add(f[0], smov);
  m[1] = dx;
  m[2] = dy;
  m[3] = O::sub(f[5], f[6]);
  m[4] = SHIFT0 ? O::fma(O::k(6.0f), phi, O::mul(O::k(-7.0f), smov))
                : O::fma(O::k(6.0f), f[0], O::neg(smov));
  m[5] = O::sub(O::fma(O::k(2.0f), sx, O::neg(sy)), sz);
  m[6] = O::sub(sy, sz);
  // m - m^eq (Eq. 17); rows 5, 6 have m^eq = 0
  const float k4 = __fmul_rn(__fmul_rn(21.0f, ph.A), ph.eta);
  V d[7];
  d[0] = O::sub(m[0], phi);
  d[1] = O::sub(m[1], O::mul(phi, u[0]));
  d[2] = O::sub(m[2], O::mul(phi, u[1]));
  d[3] = O::sub(m[3], O::mul(phi, u[2]));
  d[4] = O::sub(m[4], O::fma(O::k(-k4), mu, O::mul(O::k(6.0f), phi)));
  d[5] = m[5];
  d[6] = m[6];
  // b_k = [s_k (m_k - m_k^eq) - (1 - s_k/2) mR_k] / |M_k|^2 with mR of Eq. 18
  V b[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    if (k >= 1 && k <= 3)
      b[k] = O::fma(O::k(ph.sf_a[k]), d[k], O::mul(O::k(-ph.sf_b[k]), dphiu[k - 1]));
    else
      b[k] = O::mul(O::k(ph.sf_a[k]), d[k]);
  }
  const V e = O::sub(b[0], b[4]);
  const V c0 = O::fma(O::k(6.0f), b[4], b[0]);
  f[0] = SHIFT0 ? O::neg(O::add(smov, c0)) : O::sub(f[0], c0);
  const V ex = O::fma(O::k(2.0f), b[5], e);
  const V em = O::sub(e, b[5]);
  const V ey = O::add(em, b[6]), ez = O::sub(em, b[6]);
  f[1] = O::sub(f[1], O::add(ex, b[1]));
  f[2] = O::sub(f[2], O::sub(ex, b[1]));
  f[3] = O::sub(f[3], O::add(ey, b[2]));
  f[4] = O::sub(f[4], O::sub(ey, b[2]));
  f[5] = O::sub(f[5], O::add(ez, b[3]));
  f[6] = O::sub(f[6], O::sub(ez, b[3]));
}

}  // namespace lbm
