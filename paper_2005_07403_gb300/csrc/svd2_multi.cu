// Many batches of the paper's method in one persistent launch:
// svd2_multi_plan_bytes / svd2_multi_prepare / svd2_multi_run.
//
// A parallel Kogbetliantz sweep (Sec. 1) produces one batch of 2x2 problems
// per step, and an application often holds several independent sweeps (or
// problems of different sizes and kinds) at once.  Launching one kernel per
// batch costs a launch and a tail of idle SMs per batch, which dominates for
// short batches.  Here the batches of a step are cut into tiles of
// block * mpt * unroll consecutive matrices; tile t of the concatenated tile
// sequence belongs to the batch whose tile prefix range holds it.  CTA c takes
// tiles c, c + grid, c + 2 grid, ... -- by default one CTA per tile, or a
// persistent grid of a given size: no atomics, no scratch memory, the same
// assignment on every launch, so the launch can be captured once in a CUDA
// graph and replayed every step.  Real and complex batches form
// two tile sequences, each walked by its own persistent kernel (launched one
// after the other), so each kernel carries only its own variant of the method
// and keeps its own register budget.  A third kernel, the fix-up pass,
// recomputes with the general arithmetic the matrices the fast arithmetic
// marked (it reads the plan's flag word and ends when there are none).
#include <cstddef>
#include <mutex>
#include <new>
#include <unordered_map>
#include <utility>

#include "svd2_common.cuh"
#include "svd2_fwd_impl.cuh"

namespace svd2 {

// Device copy of one batch descriptor (the public svd2_batch_desc, plus the
// first tile index of the batch in the concatenated tile sequence).
struct MultiBatch {
  int32_t kind;       // SVD2_KIND_D or SVD2_KIND_Z
  uint32_t flags;
  int64_t n;
  int64_t tile0;      // first tile of this batch
  const double *a[8];
  double *u[8];
  double *v[8];
  double *smax;
  double *smin;
  int32_t *s;
};

// Plan header, then nbatch MultiBatch records: the nreal real batches first,
// then the complex ones, each kind with its own tile sequence from 0.
struct MultiPlanHeader {
  int32_t nbatch;
  int32_t nreal;
  int32_t tile_matrices;   // matrices per tile = block * mpt * unroll
  int32_t block;
  int64_t tiles_real;
  int64_t tiles_cplx;
  int32_t mpt, unroll;
  unsigned long long redo;   // fix-up flag of the current run (zeroed before each run)
};
constexpr size_t kPlanHeader = 64;
static_assert(sizeof(MultiPlanHeader) <= kPlanHeader, "plan header");
constexpr size_t kRedoOffset = offsetof(MultiPlanHeader, redo);

// Matrix k of batch b from the loaded elements a: the fast arithmetic, the
// outputs stored; s = kRedoS and *bad set when the fast arithmetic cannot
// finish it.
template <bool CPLX>
__device__ __forceinline__ void multi_one(const MultiBatch &b, int64_t k, const double *a,
                                          unsigned &bad) {
  constexpr int NA = CPLX ? 8 : 4;
  double u[NA], v[NA], sx, sn;
  int32_t s;
  HotAr<double, CPLX> ar;
  svd2_one<double, CPLX>(ar, a, u, v, sx, sn, s);
  if (b.flags & SVD2_BACKSCALE) backscale(sx, sn, s);
  bad |= ar.bad;
#pragma unroll
  for (int e = 0; e < NA; ++e) {
    __stcs(b.u[e] + k, u[e]);
    __stcs(b.v[e] + k, v[e]);
  }
  __stcs(b.smax + k, sx);
  __stcs(b.smin + k, sn);
  __stcs(b.s + k, ar.bad ? kRedoS : s);
}

template <bool CPLX, int M>
__device__ __forceinline__ void multi_group(const MultiBatch &b, int64_t k0, int64_t n,
                                            unsigned long long *redo) {
  constexpr int NA = CPLX ? 8 : 4;
  unsigned bad = 0;
  if (k0 + M <= n) {
    double in[NA][M];
#pragma unroll
    for (int e = 0; e < NA; ++e) {
#pragma unroll
      for (int m = 0; m < M; ++m) in[e][m] = __ldcs(b.a[e] + k0 + m);
    }
#pragma unroll
    for (int m = 0; m < M; ++m) {
      double a[NA];
#pragma unroll
      for (int e = 0; e < NA; ++e) a[e] = in[e][m];
      multi_one<CPLX>(b, k0 + m, a, bad);
    }
  } else {
    for (int64_t k = k0; k < n; ++k) {   // ragged end of a batch
      double a[NA];
#pragma unroll
      for (int e = 0; e < NA; ++e) a[e] = b.a[e][k];
      multi_one<CPLX>(b, k, a, bad);
    }
  }
  if (bad) *redo = 1;
}

template <bool CPLX, int M, int UNR>
// (1024, 1): the 64-register budget of two 512-thread blocks per SM, stated so
// that 1024-thread blocks are admitted too.
__global__ void __launch_bounds__(1024, 1) multi_kernel(const unsigned char *plan) {
  const MultiPlanHeader &h = *reinterpret_cast<const MultiPlanHeader *>(plan);
  const MultiBatch *batches = reinterpret_cast<const MultiBatch *>(plan + kPlanHeader);
  const int b_end = CPLX ? h.nbatch : h.nreal;
  const int64_t total = CPLX ? h.tiles_cplx : h.tiles_real;
  const int64_t per_tile = (int64_t)blockDim.x * M * UNR;
  if (h.tile_matrices != per_tile) return;   // launched with another shape than planned
  auto *redo = reinterpret_cast<unsigned long long *>(const_cast<unsigned char *>(plan) + kRedoOffset);
  // The record of the block's current batch, in shared memory: the threads
  // read its pointers where they use them instead of holding all of them in
  // registers across the method.  Every thread of the block walks the same
  // tiles, so the batch changes for all of them at once (uniform barriers).
  __shared__ MultiBatch sb;
  static_assert(sizeof(MultiBatch) % 8 == 0 && sizeof(MultiBatch) / 8 <= 32, "record copy");
  const int b_begin = CPLX ? h.nreal : 0;
  int bi = b_begin;   // batch of the current tile; a block's tiles only increase
  int cur = -1;
  for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
    if (cur < 0) {   // the block's first tile: the last batch with tile0 <= t
      int lo = b_begin, hi = b_end - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (batches[mid].tile0 <= t) lo = mid; else hi = mid - 1;
      }
      bi = lo;
    }
    while (bi + 1 < b_end && batches[bi + 1].tile0 <= t) ++bi;
    if (bi != cur) {
      __syncthreads();            // the previous record is no longer read
      if (threadIdx.x < sizeof(MultiBatch) / 8)
        reinterpret_cast<uint64_t *>(&sb)[threadIdx.x] =
            reinterpret_cast<const uint64_t *>(&batches[bi])[threadIdx.x];
      __syncthreads();
      cur = bi;
    }
    const MultiBatch &b = sb;
    const int64_t base = (t - b.tile0) * per_tile;
#pragma unroll
    for (int r = 0; r < UNR; ++r) {
      const int64_t k0 = base + ((int64_t)r * blockDim.x + threadIdx.x) * M;
      if (k0 < b.n) multi_group<CPLX, M>(b, k0, b.n, redo);
    }
  }
}

// Fix-up pass after both persistent kernels: when the run flagged any
// matrix, every matrix with s = kRedoS is recomputed with the general
// arithmetic; otherwise one word is read.
__global__ void __launch_bounds__(256) multi_fix_kernel(const unsigned char *plan) {
  const MultiPlanHeader &h = *reinterpret_cast<const MultiPlanHeader *>(plan);
  if (h.redo == 0) return;
  const MultiBatch *batches = reinterpret_cast<const MultiBatch *>(plan + kPlanHeader);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int bi = 0; bi < h.nbatch; ++bi) {
    const MultiBatch &b = batches[bi];
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < b.n; k += stride) {
      if (b.s[k] != kRedoS) continue;
      if (b.kind == SVD2_KIND_Z)
        exact_one<double, true>(b.a, b.u, b.v, b.smax, b.smin, b.s, b.flags, k);
      else
        exact_one<double, false>(b.a, b.u, b.v, b.smax, b.smin, b.s, b.flags, k);
    }
  }
}

using MultiKernel = void (*)(const unsigned char *);

template <bool CPLX>
static MultiKernel pick_multi(int mpt, int unroll) {
  if (mpt == 1 && unroll == 1) return multi_kernel<CPLX, 1, 1>;
  if (mpt == 1 && unroll == 2) return multi_kernel<CPLX, 1, 2>;
  if (mpt == 2 && unroll == 1) return multi_kernel<CPLX, 2, 1>;
  if (mpt == 2 && unroll == 2) return multi_kernel<CPLX, 2, 2>;
  if (mpt == 4 && unroll == 1) return multi_kernel<CPLX, 4, 1>;
  if (mpt == 4 && unroll == 2) return multi_kernel<CPLX, 4, 2>;
  return nullptr;
}

}  // namespace svd2

using namespace svd2;

// Tile counts of the plans prepared in this process (real, complex) and their
// tile size (matrices per tile), keyed by the plan's device address: grid 0
// launches one block per tile, and a launch shape with another tile size is
// rejected.
struct PlanTiles {
  int64_t real, cplx, per_tile;
};
static std::mutex g_tiles_mu;
static std::unordered_map<const void *, PlanTiles> g_tiles;

extern "C" size_t svd2_multi_plan_bytes(int32_t nbatch) {
  if (nbatch < 0) return 0;
  return kPlanHeader + (size_t)nbatch * sizeof(MultiBatch);
}

extern "C" int svd2_multi_prepare(const svd2_batch_desc *descs, int32_t nbatch, int block,
                                  int mpt, int unroll, void *plan, size_t plan_bytes,
                                  int64_t *total_tiles) {
  if (nbatch < 0 || !plan || (nbatch > 0 && !descs)) return SVD2_EINVAL;
  if (block < 32 || block > 1024 || block % 32 || !pick_multi<false>(mpt, unroll)) return SVD2_EINVAL;
  if (plan_bytes < svd2_multi_plan_bytes(nbatch) || !aligned(plan, 16)) return SVD2_EINVAL;
  const int64_t per_tile = (int64_t)block * mpt * unroll;
  unsigned char *host = new (std::nothrow) unsigned char[svd2_multi_plan_bytes(nbatch)];
  if (!host) return SVD2_ENOMEM;
  MultiPlanHeader h{};
  h.nbatch = nbatch;
  h.tile_matrices = (int32_t)per_tile;
  h.block = block;
  h.mpt = mpt;
  h.unroll = unroll;
  int64_t tiles_of[2] = {0, 0};
  int32_t nreal = 0;
  for (int32_t i = 0; i < nbatch; ++i) nreal += descs[i].kind == SVD2_KIND_Z ? 0 : 1;
  int32_t slot_of[2] = {0, nreal};   // next record of each kind
  MultiBatch *mb = reinterpret_cast<MultiBatch *>(host + kPlanHeader);
  for (int32_t i = 0; i < nbatch; ++i) {
    const svd2_batch_desc &d = descs[i];
    const int kz = d.kind == SVD2_KIND_Z ? 1 : 0;
    int64_t &tiles = tiles_of[kz];
    const int na = d.kind == SVD2_KIND_Z ? 8 : 4;
    if ((d.kind != SVD2_KIND_D && d.kind != SVD2_KIND_Z) || d.n < 0 ||
        (d.flags & ~SVD2_BACKSCALE)) {
      delete[] host;
      return SVD2_EINVAL;
    }
    MultiBatch b{};
    b.kind = d.kind;
    b.flags = d.flags;
    b.n = d.n;
    b.tile0 = tiles;
    for (int e = 0; e < 8; ++e) {
      b.a[e] = e < na ? static_cast<const double *>(d.a[e]) : nullptr;
      b.u[e] = e < na ? static_cast<double *>(d.u[e]) : nullptr;
      b.v[e] = e < na ? static_cast<double *>(d.v[e]) : nullptr;
      if (e < na && d.n > 0 && (!b.a[e] || !b.u[e] || !b.v[e])) {
        delete[] host;
        return SVD2_EINVAL;
      }
    }
    b.smax = static_cast<double *>(d.smax);
    b.smin = static_cast<double *>(d.smin);
    b.s = d.s;
    if (d.n > 0 && (!b.smax || !b.smin || !b.s)) {
      delete[] host;
      return SVD2_EINVAL;
    }
    mb[slot_of[kz]++] = b;
    tiles += (d.n + per_tile - 1) / per_tile;
  }
  h.nreal = nreal;
  h.tiles_real = tiles_of[0];
  h.tiles_cplx = tiles_of[1];
  std::memcpy(host, &h, sizeof(h));
  const cudaError_t e = cudaMemcpy(plan, host, svd2_multi_plan_bytes(nbatch),
                                   cudaMemcpyHostToDevice);
  delete[] host;
  if (e != cudaSuccess) return record_cuda_error(e);
  if (total_tiles) *total_tiles = tiles_of[0] + tiles_of[1];
  {
    std::lock_guard<std::mutex> g(g_tiles_mu);
    g_tiles[plan] = {tiles_of[0], tiles_of[1], per_tile};
  }
  return SVD2_OK;
}

// Blocks of one kind's launch.  grid > 0: that many blocks walking the tiles
// round-robin.  grid 0: one block per tile when the plan's tile count is
// known here (measured fastest on GB300: the method's long unrolled body
// stays in the instruction cache while the warps of young blocks run
// together, where those of long-lived blocks drift apart and stall on
// instruction fetch), otherwise one resident wave.
static int multi_grid(MultiKernel k, int block, int grid, int64_t tiles, int *out) {
  if (grid == 0 && tiles >= 0) {
    const int64_t g = tiles > 0 ? tiles : 1;
    grid = (int)(g < 0x7fffffffLL ? g : 0x7fffffffLL);
  } else if (grid == 0) {
    int resident = 0;
    SVD2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k, block, 0));
    grid = sm_count() * (resident > 0 ? resident : 1);
  }
  *out = grid;
  return SVD2_OK;
}

// The real-batch kernel, then the complex-batch kernel, on one stream.
static int multi_launch(const void *plan, int block, int mpt, int unroll, int grid,
                        cudaStream_t st) {
  const MultiKernel kr = pick_multi<false>(mpt, unroll), kz = pick_multi<true>(mpt, unroll);
  if (!kr || !kz || block < 32 || block > 1024 || block % 32 || grid < 0) return SVD2_EINVAL;
  int64_t tr = -1, tz = -1;
  {
    std::lock_guard<std::mutex> g(g_tiles_mu);
    auto it = g_tiles.find(plan);
    if (it != g_tiles.end()) {
      // the kernels process nothing with another tile size than the plan's
      if ((int64_t)block * mpt * unroll != it->second.per_tile) return SVD2_EINVAL;
      tr = it->second.real;
      tz = it->second.cplx;
    }
  }
  int gr = 0, gz = 0;
  int rc = multi_grid(kr, block, grid, tr, &gr);
  if (rc == SVD2_OK) rc = multi_grid(kz, block, grid, tz, &gz);
  if (rc != SVD2_OK) return rc;
  const auto *pl = static_cast<const unsigned char *>(plan);
  SVD2_CUDA_TRY(cudaMemsetAsync(const_cast<unsigned char *>(pl) + kRedoOffset, 0,
                                sizeof(unsigned long long), st));
  kr<<<gr, block, 0, st>>>(pl);
  SVD2_CUDA_TRY(cudaGetLastError());
  kz<<<gz, block, 0, st>>>(pl);
  SVD2_CUDA_TRY(cudaGetLastError());
  multi_fix_kernel<<<sm_count() * 4, 256, 0, st>>>(pl);
  SVD2_CUDA_TRY(cudaGetLastError());
  return SVD2_OK;
}

extern "C" int svd2_multi_run(const void *plan, int block, int mpt, int unroll, int grid,
                              svd2_stream_t stream) {
  if (!plan || !aligned(plan, 16)) return SVD2_EINVAL;
  return multi_launch(plan, block, mpt, unroll, grid, (cudaStream_t)stream);
}

// The persistent launches captured once into an executable CUDA graph, for
// replay at every step (the plan's batch pointers stay fixed while the data
// in them changes).
extern "C" int svd2_multi_graph_create(const void *plan, int block, int mpt, int unroll, int grid,
                                       void **graph_exec) {
  if (!graph_exec || !plan || !aligned(plan, 16)) return SVD2_EINVAL;
  if (!pick_multi<false>(mpt, unroll) || block < 32 || block > 1024 || block % 32 || grid < 0)
    return SVD2_EINVAL;
  cudaStream_t cs = nullptr;
  SVD2_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int rc = SVD2_OK;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rc = multi_launch(plan, block, mpt, unroll, grid, cs);
    e = cudaStreamEndCapture(cs, &graph);
  }
  if (e == cudaSuccess && rc == SVD2_OK) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (rc != SVD2_OK) return rc;
  if (e != cudaSuccess) return record_cuda_error(e);
  *graph_exec = exec;
  return SVD2_OK;
}

extern "C" int svd2_graph_launch(void *graph_exec, svd2_stream_t stream) {
  if (!graph_exec) return SVD2_EINVAL;
  SVD2_CUDA_TRY(cudaGraphLaunch(static_cast<cudaGraphExec_t>(graph_exec), (cudaStream_t)stream));
  return SVD2_OK;
}

extern "C" int svd2_graph_destroy(void *graph_exec) {
  if (!graph_exec) return SVD2_EINVAL;
  SVD2_CUDA_TRY(cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(graph_exec)));
  return SVD2_OK;
}
