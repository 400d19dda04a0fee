// Many batches of the paper's method in one persistent launch:
// svd2_multi_plan_bytes / svd2_multi_prepare / svd2_multi_run.
//
// A parallel Kogbetliantz sweep (Sec. 1) produces one batch of 2x2 problems
// per step, and an application often holds several independent sweeps (or
// problems of different sizes and kinds) at once.  Launching one kernel per
// batch costs a launch and a tail of idle SMs per batch, which dominates for
// short batches.  Here the batches of a step are cut into tiles of
// block * mpt * unroll consecutive matrices; tile t of the concatenated tile
// sequence belongs to the batch whose tile prefix range holds it.  A grid of
// (SMs x resident blocks) CTAs walks the tiles in a fixed round-robin order,
// CTA c taking tiles c, c + grid, c + 2 grid, ...: no atomics, no scratch
// memory, the same assignment on every launch, so the launch can be captured
// once in a CUDA graph and replayed every step.  A tile's kind (real or
// complex double) is uniform over the CTA, so the branch between the two
// method variants never diverges inside a warp.
#include <new>

#include "svd2_common.cuh"
#include "svd2_math.cuh"

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

// Plan header, then nbatch MultiBatch records.
struct MultiPlanHeader {
  int32_t nbatch;
  int32_t tile_matrices;   // matrices per tile = block * mpt * unroll
  int64_t total_tiles;
  int32_t block, mpt, unroll, pad;
};
constexpr size_t kPlanHeader = 64;

template <bool CPLX, int M>
__device__ __forceinline__ void multi_group(const MultiBatch &b, int64_t k0, int64_t n) {
  constexpr int NA = CPLX ? 8 : 4;
  if (k0 + M <= n) {
    double in[NA][M];
#pragma unroll
    for (int e = 0; e < NA; ++e) {
#pragma unroll
      for (int m = 0; m < M; ++m) in[e][m] = __ldcs(b.a[e] + k0 + m);
    }
#pragma unroll
    for (int m = 0; m < M; ++m) {
      double a[NA], u[NA], v[NA], sx, sn;
      int32_t s;
      int piv;
#pragma unroll
      for (int e = 0; e < NA; ++e) a[e] = in[e][m];
      if constexpr (CPLX)
        svd2_cplx<double>(a, u, v, sx, sn, s, piv);
      else
        svd2_real<double>(a, u, v, sx, sn, s, piv);
      if (b.flags & SVD2_BACKSCALE) {
        if (s != kZeroS) {
          sx = scalef(sx, -s);
          sn = scalef(sn, -s);
        }
        s = 0;
      }
#pragma unroll
      for (int e = 0; e < NA; ++e) {
        __stcs(b.u[e] + k0 + m, u[e]);
        __stcs(b.v[e] + k0 + m, v[e]);
      }
      __stcs(b.smax + k0 + m, sx);
      __stcs(b.smin + k0 + m, sn);
      __stcs(b.s + k0 + m, s);
    }
  } else {
    for (int64_t k = k0; k < n; ++k) {   // ragged end of a batch
      double a[NA], u[NA], v[NA], sx, sn;
      int32_t s;
      int piv;
#pragma unroll
      for (int e = 0; e < NA; ++e) a[e] = b.a[e][k];
      if constexpr (CPLX)
        svd2_cplx<double>(a, u, v, sx, sn, s, piv);
      else
        svd2_real<double>(a, u, v, sx, sn, s, piv);
      if (b.flags & SVD2_BACKSCALE) {
        if (s != kZeroS) {
          sx = scalef(sx, -s);
          sn = scalef(sn, -s);
        }
        s = 0;
      }
#pragma unroll
      for (int e = 0; e < NA; ++e) {
        b.u[e][k] = u[e];
        b.v[e][k] = v[e];
      }
      b.smax[k] = sx;
      b.smin[k] = sn;
      b.s[k] = s;
    }
  }
}

template <int M, int UNR>
__global__ void __launch_bounds__(512) multi_kernel(const unsigned char *plan) {
  const MultiPlanHeader &h = *reinterpret_cast<const MultiPlanHeader *>(plan);
  const MultiBatch *batches = reinterpret_cast<const MultiBatch *>(plan + kPlanHeader);
  const int nbatch = h.nbatch;
  const int64_t total = h.total_tiles;
  const int64_t per_tile = (int64_t)blockDim.x * M * UNR;
  if (h.tile_matrices != per_tile) return;   // launched with another shape than planned
  int bi = 0;   // batch of the current tile; tiles only increase, so walk forward
  for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
    while (bi + 1 < nbatch && batches[bi + 1].tile0 <= t) ++bi;
    const MultiBatch &b = batches[bi];
    const int64_t base = (t - b.tile0) * per_tile;
#pragma unroll
    for (int r = 0; r < UNR; ++r) {
      const int64_t k0 = base + ((int64_t)r * blockDim.x + threadIdx.x) * M;
      if (k0 < b.n) {
        if (b.kind == SVD2_KIND_Z)
          multi_group<true, M>(b, k0, b.n);
        else
          multi_group<false, M>(b, k0, b.n);
      }
    }
  }
}

using MultiKernel = void (*)(const unsigned char *);

static MultiKernel pick_multi(int mpt, int unroll) {
  if (mpt == 1 && unroll == 1) return multi_kernel<1, 1>;
  if (mpt == 1 && unroll == 2) return multi_kernel<1, 2>;
  if (mpt == 2 && unroll == 1) return multi_kernel<2, 1>;
  if (mpt == 2 && unroll == 2) return multi_kernel<2, 2>;
  return nullptr;
}

}  // namespace svd2

using namespace svd2;

extern "C" size_t svd2_multi_plan_bytes(int32_t nbatch) {
  if (nbatch < 0) return 0;
  return kPlanHeader + (size_t)nbatch * sizeof(MultiBatch);
}

extern "C" int svd2_multi_prepare(const svd2_batch_desc *descs, int32_t nbatch, int block,
                                  int mpt, int unroll, void *plan, size_t plan_bytes,
                                  int64_t *total_tiles) {
  if (nbatch < 0 || !plan || (nbatch > 0 && !descs)) return SVD2_EINVAL;
  if (block < 32 || block > 512 || block % 32 || !pick_multi(mpt, unroll)) return SVD2_EINVAL;
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
  int64_t tiles = 0;
  MultiBatch *mb = reinterpret_cast<MultiBatch *>(host + kPlanHeader);
  for (int32_t i = 0; i < nbatch; ++i) {
    const svd2_batch_desc &d = descs[i];
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
    mb[i] = b;
    tiles += (d.n + per_tile - 1) / per_tile;
  }
  h.total_tiles = tiles;
  std::memcpy(host, &h, sizeof(h));
  const cudaError_t e = cudaMemcpy(plan, host, svd2_multi_plan_bytes(nbatch),
                                   cudaMemcpyHostToDevice);
  delete[] host;
  if (e != cudaSuccess) return record_cuda_error(e);
  if (total_tiles) *total_tiles = tiles;
  return SVD2_OK;
}

static int multi_grid(MultiKernel k, int block, int grid, int *out) {
  if (grid == 0) {
    int resident = 0;
    SVD2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k, block, 0));
    grid = sm_count() * (resident > 0 ? resident : 1);
  }
  *out = grid;
  return SVD2_OK;
}

extern "C" int svd2_multi_run(const void *plan, int block, int mpt, int unroll, int grid,
                              svd2_stream_t stream) {
  if (!plan || !aligned(plan, 16)) return SVD2_EINVAL;
  MultiKernel k = pick_multi(mpt, unroll);
  if (!k || block < 32 || block > 512 || block % 32 || grid < 0) return SVD2_EINVAL;
  int g = 0;
  const int rc = multi_grid(k, block, grid, &g);
  if (rc != SVD2_OK) return rc;
  k<<<g, block, 0, (cudaStream_t)stream>>>(static_cast<const unsigned char *>(plan));
  SVD2_CUDA_TRY(cudaGetLastError());
  return SVD2_OK;
}

// The persistent launch captured once into an executable CUDA graph, for
// replay at every step (the plan's batch pointers stay fixed while the data
// in them changes).
extern "C" int svd2_multi_graph_create(const void *plan, int block, int mpt, int unroll, int grid,
                                       void **graph_exec) {
  if (!graph_exec || !plan || !aligned(plan, 16)) return SVD2_EINVAL;
  MultiKernel k = pick_multi(mpt, unroll);
  if (!k || block < 32 || block > 512 || block % 32 || grid < 0) return SVD2_EINVAL;
  int g = 0;
  int rc = multi_grid(k, block, grid, &g);
  if (rc != SVD2_OK) return rc;
  cudaStream_t cs = nullptr;
  SVD2_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    k<<<g, block, 0, cs>>>(static_cast<const unsigned char *>(plan));
    const cudaError_t el = cudaGetLastError();
    e = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = el;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
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
