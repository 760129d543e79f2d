// Batched execution: many runs of different sizes advanced together, one launch per
// pass for all of them.
//
// A batch step of n time steps launches, n times, the three passes (order parameter,
// chemical potential, fused stream-collide) each ONCE for every run of the batch.  The
// runs' descriptors (geometry, physics, array pointers, parity) sit in a device table;
// each pass's blocks take (run, block-of-that-run) work items from it -- a persistent
// grid striding over the items, or one block per item -- so runs of uneven size share
// the launch and small runs no longer pay a launch each.  Because the kernels read the
// run set from the table, the 3n launches of a batch step are captured once into a CUDA
// graph per launch shape and replayed for any run set with that shape: between replays
// the host only rewrites the table.  Runs of at least a set size (they fill the GPU
// alone, and the single-run kernels read their parameters from the constant bank rather
// than shared memory) can instead take their own launches on their own streams, which
// then overlap the shared ones.  The per-cell arithmetic is the same device code as the
// single-run kernels (lbm_cells.cuh), so results are bit-identical to lbm_step's.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_capi_internal.h"
#include "lbm_cells.cuh"
#include "lbm_internal.h"

namespace lbm {

constexpr int kMaxBatchRuns = 256;

struct RunDesc {
  Geometry geo;
  Physics ph;
  float* state[2];  // the two population arrays (pattern AB)
  float* phi;
  float* mu;
  int parity;     // state[parity] holds the current state at batch step 0
  int have_prev;  // 1: every batched run has taken its first step
  int pad[2];
};

struct BatchTable {
  int nruns;
  int total_cells;   // items of the order-parameter and stream-collide passes
  int total_bricks;  // items of the chemical-potential pass
  int cell_first[kMaxBatchRuns + 1];   // first item of run r (prefix sums)
  int brick_first[kMaxBatchRuns + 1];
  RunDesc runs[kMaxBatchRuns];
};

namespace {

// Largest r with first[r] <= item (first[0] = 0, first[nruns] = total); `first` is the
// block's shared-memory copy of the prefix sums.
__device__ __forceinline__ int find_run(const int* first, int nruns, int item) {
  int lo = 0, hi = nruns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// The block's threads copy the nruns + 1 prefix sums into shared memory once, so that
// each block's run lookups are a binary search in shared memory rather than a chain of
// dependent global loads; the caller synchronises before the first lookup (seek does).
__device__ __forceinline__ void load_firsts(const int* __restrict__ first, int nruns, int* s_first) {
  for (int k = threadIdx.x + threadIdx.y * blockDim.x; k <= nruns; k += blockDim.x * blockDim.y)
    s_first[k] = __ldg(first + k);
}

// The block's threads copy run r's descriptor into shared memory.
__device__ __forceinline__ void load_desc(const BatchTable* __restrict__ t, int r, RunDesc& sd) {
  constexpr int words = sizeof(RunDesc) / 4;
  const int* src = reinterpret_cast<const int*>(&t->runs[r]);
  int* dst = reinterpret_cast<int*>(&sd);
  for (int k = threadIdx.x + threadIdx.y * blockDim.x; k < words; k += blockDim.x * blockDim.y)
    dst[k] = __ldg(src + k);
}

// A block's items increase, so its run changes rarely: the descriptor in shared memory
// is reloaded only when an item belongs to another run than the previous one.  Every
// thread of the block takes the same branch (the condition depends on the item only).
struct RunCursor {
  int r = -1;      // run whose descriptor is in shared memory
  int first = 0;   // its first item
  int end = 0;     // one past its last item
};

__device__ __forceinline__ void seek(const BatchTable* __restrict__ t, const int* s_first,
                                     int nruns, int item, RunCursor& c, RunDesc& sd) {
  if (item < c.end) return;
  __syncthreads();  // the block is done with the previous descriptor (and s_first is loaded)
  const int r = find_run(s_first, nruns, item);
  load_desc(t, r, sd);
  __syncthreads();
  c.r = r;
  c.first = s_first[r];
  c.end = s_first[r + 1];
}

// Work items are blocks of kBlock cells (order parameter, stream-collide) or bricks
// (chemical potential).  A launch either has fewer blocks than items and strides over
// them (persistent), or one block per item.  `dist` > 0: thread 0 prefetches into L2
// the data of item + dist when it belongs to the same run (for a persistent launch,
// dist = gridDim.x is the block's own next item).
template <int S>
__global__ void __launch_bounds__(kBlock) kb_phi(const BatchTable* __restrict__ t, int step,
                                                 int dist) {
  __shared__ RunDesc sd;
  __shared__ int s_first[kMaxBatchRuns + 1];
  const int nitems = t->total_cells, nruns = t->nruns;
  if (blockIdx.x < nitems) load_firsts(t->cell_first, nruns, s_first);
  RunCursor c;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    seek(t, s_first, nruns, item, c, sd);
    const float* src = sd.state[(sd.parity + step) & 1];
    if (threadIdx.x == 0 && dist > 0 && item + dist < c.end)
      prefetch_cells<S, false>(src, nullptr, nullptr, sd.geo,
                               static_cast<long long>(item + dist - c.first) * kBlock);
    const int idx = (item - c.first) * kBlock + threadIdx.x;
    if (idx < sd.geo.n) phi_cell<kAB, S>(src, sd.phi, sd.phi, sd.geo, idx);
  }
}

__global__ void __launch_bounds__(kTX* kTY) kb_mu(const BatchTable* __restrict__ t, int step) {
  __shared__ RunDesc sd;
  __shared__ float tile[kHZ][kHY][kHX];
  __shared__ int s_first[kMaxBatchRuns + 1];
  const int nitems = t->total_bricks, nruns = t->nruns;
  if (blockIdx.x < nitems) load_firsts(t->brick_first, nruns, s_first);
  RunCursor c;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    seek(t, s_first, nruns, item, c, sd);
    const int local = item - c.first;
    const int nbx = (sd.geo.nx + kTX - 1) / kTX, nby = (sd.geo.ny + kTY - 1) / kTY;
    const int bx = local % nbx, rest = local / nbx;
    mu_brick<false>(sd.phi, sd.mu, sd.geo, sd.ph, bx, rest % nby, rest / nby, tile);
    __syncthreads();  // the next brick reuses the tile
  }
}

// Blocks of kBlock / 2 threads take items of kBlock cells: two cells per thread, in the
// two lanes of paired instructions (collide_pair: cells x and x + 32 of a row) for runs
// whose rows are pairs of tiles (Geometry::pairs), else one after the other with the
// one-cell body (cells i and i + kBlock / 2 of the item).  Bit-identical either way.
template <int S>
__global__ void __launch_bounds__(kBlock / 2, 4) kb_collide(
    const BatchTable* __restrict__ t, int step, int dist) {
  __shared__ RunDesc sd;
  __shared__ int s_first[kMaxBatchRuns + 1];
  const int nitems = t->total_cells, nruns = t->nruns;
  if (blockIdx.x < nitems) load_firsts(t->cell_first, nruns, s_first);
  RunCursor c;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    seek(t, s_first, nruns, item, c, sd);
    const float* src = sd.state[(sd.parity + step) & 1];
    if (threadIdx.x == 0 && dist > 0 && item + dist < c.end)
      prefetch_cells<S, true>(src, sd.phi, sd.mu, sd.geo,
                              static_cast<long long>(item + dist - c.first) * kBlock);
    float* dst = sd.state[(sd.parity + step + 1) & 1];
    const int base = (item - c.first) * kBlock;
    if (sd.geo.pairs) {
      const int idx = base + (threadIdx.x >> 5) * (2 * kTile) + (threadIdx.x & 31);
      if (idx < sd.geo.n)
        collide_pair<0, S, false>(src, dst, sd.phi, sd.mu, sd.geo, sd.ph, sd.have_prev, idx,
                                  nullptr);
    } else {
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int idx = base + h * (kBlock / 2) + threadIdx.x;
        if (idx < sd.geo.n)
          collide_cell<kAB, 0, S>(src, dst, sd.phi, sd.mu, sd.geo, sd.ph, sd.have_prev, idx);
      }
    }
  }
}

int bricks_of(const Geometry& g) {
  return ((g.nx + kTX - 1) / kTX) * ((g.ny + kTY - 1) / kTY) * ((g.nz + kTZ - 1) / kTZ);
}

}  // namespace

}  // namespace lbm

struct lbm_batch {
  cudaStream_t stream = nullptr;
  bool own_stream = false;  // created here: graphs cannot be captured on the legacy stream
  lbm_allocator alloc{};
  bool have_alloc = false;
  lbm::BatchTable* table = nullptr;  // device
  std::vector<unsigned char> host;   // host image of the table
  int sms = 0;
  int resident[3] = {0, 0, 0};  // blocks per SM of each pass's kernel
  // blocks of the phi, mu, collide passes: > 0 persistent, 0 one block per item
  int grid[3] = {0, 0, 0};
  // prefetch distance in items of the phi and collide passes: -1 one wave (the launch's
  // blocks when persistent, else SMs x resident blocks), 0 off, > 0 that many items
  int dist[3] = {-1, 0, -1};
  // launch shapes of the graph being captured or replayed
  int launch_grid[3] = {0, 0, 0};
  int launch_dist[3] = {0, 0, 0};
  // runs of at least this many cells take their own launches; 0: every run shares
  long long split_cells = 0;
  int last_shared = 0;  // runs in the shared launches of the last batch step
  // instantiated graphs by (steps, storage, launch grids, launch distances)
  std::map<std::vector<int>, cudaGraphExec_t> graphs;
  cudaEvent_t done = nullptr;
  std::string err;
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status st, const std::string& msg) {
  if (b)
    b->err = msg;
  else
    lbm::set_global_error(msg);
  return st;
}

#define LBM_BCK(b, call)                                                                  \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return bfail((b), LBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

void drop_graphs(lbm_batch* b) {
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

cudaError_t launch_pass_kernels(lbm_batch* b, int storage, int steps) {
  const lbm::BatchTable* t = b->table;
  const int* g = b->launch_grid;
  const int* d = b->launch_dist;
  for (int s = 0; s < steps; ++s) {
    if (storage == LBM_STORAGE_FP16)
      lbm::kb_phi<lbm::kF16><<<g[0], lbm::kBlock, 0, b->stream>>>(t, s, d[0]);
    else if (storage == LBM_STORAGE_BF16)
      lbm::kb_phi<lbm::kBF16><<<g[0], lbm::kBlock, 0, b->stream>>>(t, s, d[0]);
    else
      lbm::kb_phi<lbm::kF32><<<g[0], lbm::kBlock, 0, b->stream>>>(t, s, d[0]);
    lbm::kb_mu<<<g[1], dim3(lbm::kTX, lbm::kTY), 0, b->stream>>>(t, s);
    if (storage == LBM_STORAGE_FP16)
      lbm::kb_collide<lbm::kF16><<<g[2], lbm::kBlock / 2, 0, b->stream>>>(t, s, d[2]);
    else if (storage == LBM_STORAGE_BF16)
      lbm::kb_collide<lbm::kBF16><<<g[2], lbm::kBlock / 2, 0, b->stream>>>(t, s, d[2]);
    else
      lbm::kb_collide<lbm::kF32><<<g[2], lbm::kBlock / 2, 0, b->stream>>>(t, s, d[2]);
  }
  return cudaGetLastError();
}

// Blocks of a one-block-per-item launch: the items rounded up (by at most 1/16) so that
// run sets of similar size share a graph; the extra blocks find no item and exit.
int round_items(int items) {
  int q = 64;
  while (q * 16 < items) q *= 2;
  return (items + q - 1) / q * q;
}

// Launch shapes of each pass for a table with the given item counts.
void plan_launch(lbm_batch* b, int cell_items, int brick_items) {
  const int items[3] = {cell_items, brick_items, cell_items};
  for (int p = 0; p < 3; ++p) {
    const bool persistent = b->grid[p] > 0;
    b->launch_grid[p] = persistent ? b->grid[p] : round_items(items[p]);
    int d = b->dist[p];
    if (d < 0) d = persistent ? b->grid[p] : b->sms * b->resident[p];
    b->launch_dist[p] = p == 1 ? 0 : d;
  }
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(const lbm_allocator* alloc, void* cuda_stream, lbm_batch** out) {
  if (!out) return bfail(nullptr, LBM_EINVAL, "out must not be NULL");
  *out = nullptr;
  if (alloc && (!alloc->alloc || !alloc->free))
    return bfail(nullptr, LBM_EINVAL, "allocator needs both alloc and free");
  lbm_batch* b = new lbm_batch();
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  if (!b->stream) {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return bfail(nullptr, LBM_ECUDA, "cudaStreamCreate failed");
    }
    b->own_stream = true;
  }
  if (alloc) {
    b->alloc = *alloc;
    b->have_alloc = true;
  }
  void* p = nullptr;
  if (b->have_alloc)
    p = b->alloc.alloc(sizeof(lbm::BatchTable), b->alloc.user);
  else if (cudaMalloc(&p, sizeof(lbm::BatchTable)) != cudaSuccess)
    p = nullptr;
  if (!p) {
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return bfail(nullptr, LBM_ENOMEM, "device allocation failed (batch table)");
  }
  b->table = static_cast<lbm::BatchTable*>(p);
  b->host.assign(sizeof(lbm::BatchTable), 0);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->resident[0], lbm::kb_phi<lbm::kF32>,
                                                lbm::kBlock, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->resident[1], lbm::kb_mu, lbm::kTX * lbm::kTY,
                                                0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->resident[2], lbm::kb_collide<lbm::kF32>,
                                                lbm::kBlock / 2, 0);
  for (int p = 0; p < 3; ++p) b->resident[p] = std::max(b->resident[p], 1);
  b->grid[0] = b->sms * 8;
  b->grid[1] = b->sms * 6;
  b->grid[2] = 0;
  if (cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess) {
    lbm_batch_destroy(b);
    return bfail(nullptr, LBM_ECUDA, "cudaEventCreate failed");
  }
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_set_grid(lbm_batch* b, int pass, int blocks) {
  if (!b) return LBM_EINVAL;
  if (pass < 0 || pass > 2 || blocks < 0 || blocks > (1 << 24))
    return bfail(b, LBM_EINVAL, "pass must be 0..2 and blocks in 0..2^24");
  b->grid[pass] = blocks;
  return LBM_OK;
}

lbm_status lbm_batch_get_grid(const lbm_batch* b, int pass, int* blocks) {
  if (!b || !blocks || pass < 0 || pass > 2) return LBM_EINVAL;
  *blocks = b->grid[pass];
  return LBM_OK;
}

lbm_status lbm_batch_set_split(lbm_batch* b, long long cells) {
  if (!b) return LBM_EINVAL;
  if (cells < 0) return bfail(b, LBM_EINVAL, "cells must be >= 0");
  b->split_cells = cells;
  return LBM_OK;
}

lbm_status lbm_batch_get_split(const lbm_batch* b, long long* cells) {
  if (!b || !cells) return LBM_EINVAL;
  *cells = b->split_cells;
  return LBM_OK;
}

lbm_status lbm_batch_set_prefetch(lbm_batch* b, int pass, int items) {
  if (!b) return LBM_EINVAL;
  if ((pass != 0 && pass != 2) || items < -1 || items > (1 << 24))
    return bfail(b, LBM_EINVAL, "pass must be 0 or 2 and items in -1..2^24");
  b->dist[pass] = items;
  return LBM_OK;
}

lbm_status lbm_batch_get_prefetch(const lbm_batch* b, int pass, int* items) {
  if (!b || !items || (pass != 0 && pass != 2)) return LBM_EINVAL;
  *items = b->dist[pass];
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, lbm_ctx* const* runs, int nruns, int nsteps) {
  if (!b) return LBM_EINVAL;
  if (!runs || nruns < 1 || nruns > lbm::kMaxBatchRuns)
    return bfail(b, LBM_EINVAL, "need 1.." + std::to_string(lbm::kMaxBatchRuns) + " runs");
  if (nsteps < 0) return bfail(b, LBM_EINVAL, "nsteps must be >= 0");
  if (nsteps == 0) return LBM_OK;
  const int storage = lbm::ctx_storage(runs[0]);
  for (int r = 0; r < nruns; ++r) {
    if (!runs[r]) return bfail(b, LBM_EINVAL, "NULL run");
    for (int q = 0; q < r; ++q)
      if (runs[q] == runs[r]) return bfail(b, LBM_EINVAL, "a run appears twice");
    std::string why;
    if (!lbm::ctx_batchable(runs[r], &why)) return bfail(b, LBM_EINVAL, "run " + std::to_string(r) + ": " + why);
    if (lbm::ctx_storage(runs[r]) != storage)
      return bfail(b, LBM_EINVAL, "all runs of a batch need the same storage type");
  }
  // the first step after initialisation (d_t(phi u) = 0) is taken with lbm_step
  for (int r = 0; r < nruns; ++r)
    if (!lbm::ctx_have_prev(runs[r]))
      return bfail(b, LBM_EINVAL, "run " + std::to_string(r) +
                                      " has taken no step yet: take the first with lbm_step");
  // runs of at least split_cells cells fill the GPU by themselves: they take their own
  // launches (lbm_step on their own streams), which then overlap the shared launches
  std::vector<lbm_ctx*> shared, own;
  for (int r = 0; r < nruns; ++r) {
    lbm::Geometry g;
    lbm::Physics ph;
    float *s0, *s1, *phi, *mu;
    int parity;
    lbm::ctx_describe(runs[r], &g, &ph, &s0, &s1, &phi, &mu, &parity);
    (b->split_cells > 0 && g.n >= b->split_cells ? own : shared).push_back(runs[r]);
  }
  // table of the shared runs: prefix sums and descriptors
  lbm::BatchTable* h = reinterpret_cast<lbm::BatchTable*>(b->host.data());
  const int nshared = static_cast<int>(shared.size());
  h->nruns = nshared;
  h->cell_first[0] = 0;
  h->brick_first[0] = 0;
  long long cells = 0, bricks = 0;
  for (int r = 0; r < nshared; ++r) {
    lbm::RunDesc& d = h->runs[r];
    std::memset(&d, 0, sizeof(d));
    lbm::ctx_describe(shared[r], &d.geo, &d.ph, &d.state[0], &d.state[1], &d.phi, &d.mu, &d.parity);
    d.have_prev = 1;
    cells += (d.geo.n + lbm::kBlock - 1) / lbm::kBlock;
    bricks += lbm::bricks_of(d.geo);
    if (cells > (1LL << 30) || bricks > (1LL << 30)) return bfail(b, LBM_EINVAL, "batch too large");
    h->cell_first[r + 1] = static_cast<int>(cells);
    h->brick_first[r + 1] = static_cast<int>(bricks);
  }
  h->total_cells = static_cast<int>(cells);
  h->total_bricks = static_cast<int>(bricks);

  for (lbm_ctx* c : own) {
    const lbm_status st = lbm_step(c, nsteps);
    if (st != LBM_OK) return bfail(b, st, std::string("lbm_step: ") + lbm_last_error(c));
  }
  b->last_shared = nshared;
  if (nshared == 0) return LBM_OK;

  // order the shared launches after each shared run's pending work
  for (lbm_ctx* c : shared) {
    LBM_BCK(b, cudaEventRecord(b->done, lbm::ctx_stream(c)));
    LBM_BCK(b, cudaStreamWaitEvent(b->stream, b->done, 0));
  }
  const size_t bytes = offsetof(lbm::BatchTable, runs) + sizeof(lbm::RunDesc) * nshared;
  LBM_BCK(b, cudaMemcpyAsync(b->table, h, bytes, cudaMemcpyHostToDevice, b->stream));

  // one graph per launch shape, replayed for any run set that has it
  plan_launch(b, h->total_cells, h->total_bricks);
  const std::vector<int> key = {nsteps, storage, b->launch_grid[0], b->launch_grid[1],
                                b->launch_grid[2], b->launch_dist[0], b->launch_dist[2]};
  auto it = b->graphs.find(key);
  if (it == b->graphs.end()) {
    if (b->graphs.size() >= 64) drop_graphs(b);
    cudaGraph_t graph = nullptr;
    LBM_BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    const cudaError_t le = launch_pass_kernels(b, storage, nsteps);
    const cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
    if (le != cudaSuccess || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return bfail(b, LBM_ECUDA, std::string("graph capture: ") +
                                     cudaGetErrorString(le != cudaSuccess ? le : ce));
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return bfail(b, LBM_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
    it = b->graphs.emplace(key, exec).first;
  }
  LBM_BCK(b, cudaGraphLaunch(it->second, b->stream));
  // each shared run's later work waits for the batch
  LBM_BCK(b, cudaEventRecord(b->done, b->stream));
  for (lbm_ctx* c : shared) {
    LBM_BCK(b, cudaStreamWaitEvent(lbm::ctx_stream(c), b->done, 0));
    lbm::ctx_advance(c, nsteps);
  }
  return LBM_OK;
}

lbm_status lbm_batch_destroy(lbm_batch* b) {
  if (!b) return LBM_EINVAL;
  cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  if (b->done) cudaEventDestroy(b->done);
  if (b->table) {
    if (b->have_alloc)
      b->alloc.free(b->table, b->alloc.user);
    else
      cudaFree(b->table);
  }
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return LBM_OK;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : ""; }

}  // extern "C"
