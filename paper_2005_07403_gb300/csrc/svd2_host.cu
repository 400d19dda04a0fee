// svd2_batch_host: the forward forms on batches held in HOST memory.
//
// When every array is page-locked (pinned) host memory, which kernels can
// address directly under unified addressing, the forward kernel runs on the
// host arrays themselves: inputs and outputs cross the host link once, with
// no staging (on GB300 the link carries ~250 GB/s in both directions
// together, whether copy engines or kernels drive it, and the direct form
// saves the staging).  Otherwise the batch is cut into chunks that flow
// through a three-stage pipeline on
// three streams -- host-to-device copies of a chunk's input arrays, the forward
// kernel, device-to-host copies of its outputs -- double-buffered in device
// staging memory, so the copies of one chunk overlap the kernel of the next
// and the copies in the other direction (the host link is full duplex).  The
// caller's stream is made to wait for the last chunk, so the call behaves like
// an asynchronous operation on that stream.  Host arrays should be pinned
// (page-locked) for the copies to overlap; pageable memory works but
// serialises the copies.
//
// The staging buffers and streams are created on first use per device and
// kept until the process exits; host-pipeline calls are serialised within the
// process.
#include <mutex>

#include "svd2_common.cuh"

namespace {

struct Stage {
  void *buf[2] = {nullptr, nullptr};
  size_t bytes = 0;                      // per slot
  cudaStream_t st[3] = {nullptr, nullptr, nullptr};   // h2d, compute, d2h
  cudaEvent_t in_ready[2] = {}, computed[2] = {}, out_done[2] = {};
  cudaEvent_t start = nullptr;           // the caller's stream at the call
  bool init = false;
};

std::mutex g_mu;
Stage g_stage[64];

int setup(Stage &S, size_t slot_bytes) {
  if (!S.init) {
    for (auto &s : S.st) SVD2_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
      SVD2_CUDA_TRY(cudaEventCreateWithFlags(&S.in_ready[b], cudaEventDisableTiming));
      SVD2_CUDA_TRY(cudaEventCreateWithFlags(&S.computed[b], cudaEventDisableTiming));
      SVD2_CUDA_TRY(cudaEventCreateWithFlags(&S.out_done[b], cudaEventDisableTiming));
    }
    SVD2_CUDA_TRY(cudaEventCreateWithFlags(&S.start, cudaEventDisableTiming));
    S.init = true;
  }
  if (S.bytes < slot_bytes) {
    // a previous call's copies may still use the old buffers
    for (auto &s : S.st) SVD2_CUDA_TRY(cudaStreamSynchronize(s));
    for (auto &p : S.buf) {
      if (p) SVD2_CUDA_TRY(cudaFree(p));
      p = nullptr;
    }
    S.bytes = 0;
    for (auto &p : S.buf) SVD2_CUDA_TRY(cudaMalloc(&p, slot_bytes));
    S.bytes = slot_bytes;
  }
  return SVD2_OK;
}

int launch(int op, int64_t n, const void *const *A, void *const *U, void *const *V, void *smax,
           void *smin, int32_t *s, uint32_t flags, cudaStream_t st) {
  const auto stream = (svd2_stream_t)st;
  switch (op) {
    case 0:
      return svd2_batch_d(n, (const double *const *)A, (double *const *)U, (double *const *)V,
                          (double *)smax, (double *)smin, s, flags, stream);
    case 1:
      return svd2_batch_z(n, (const double *const *)A, (double *const *)U, (double *const *)V,
                          (double *)smax, (double *)smin, s, flags, stream);
    case 2:
      return svd2_batch_s(n, (const float *const *)A, (float *const *)U, (float *const *)V,
                          (float *)smax, (float *)smin, s, flags, stream);
    case svd2::kOpSTan64:
      return svd2_batch_s_tan64(n, (const float *const *)A, (float *const *)U,
                                (float *const *)V, (float *)smax, (float *)smin, s,
                                SVD2_TAN64_TAU_LOG2, flags, nullptr, stream);
    default:
      return svd2_batch_c(n, (const float *const *)A, (float *const *)U, (float *const *)V,
                          (float *)smax, (float *)smin, s, flags, stream);
  }
}

// True when p is page-locked host memory that kernels can address at the same
// pointer value (cudaHostAlloc / cudaMallocHost / cudaHostRegister memory under
// unified addressing); false for pageable memory, device memory or an error.
bool kernel_addressable_host(const void *p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();   // clear the error of an unknown pointer
    return false;
  }
  return at.type == cudaMemoryTypeHost && at.devicePointer == p && at.hostPointer == p;
}

}  // namespace

using namespace svd2;

extern "C" int svd2_batch_host(int op, int64_t n, const void *const *A, void *const *U,
                               void *const *V, void *smax, void *smin, int32_t *s,
                               uint32_t flags, int64_t chunk, svd2_stream_t stream) {
  if (op < 0 || op >= kNumOps || n < 0 || chunk < 0 || (flags & ~(SVD2_BACKSCALE | SVD2_SINE)))
    return SVD2_EINVAL;
  if (n == 0) return SVD2_OK;
  const int na = (op == kOpZ || op == kOpC) ? 8 : 4;
  const size_t es = (op == kOpD || op == kOpZ) ? 8 : 4;
  if (!A || !U || !V || !smax || !smin || !s) return SVD2_EINVAL;
  for (int e = 0; e < na; ++e)
    if (!A[e] || !U[e] || !V[e]) return SVD2_EINVAL;
  // every array page-locked: the kernel reads and writes them directly over the
  // host link (no staging copies; measured faster than the copy pipeline)
  bool direct = kernel_addressable_host(smax) && kernel_addressable_host(smin) &&
                kernel_addressable_host(s);
  for (int e = 0; e < na && direct; ++e)
    direct = kernel_addressable_host(A[e]) && kernel_addressable_host(U[e]) &&
             kernel_addressable_host(V[e]);
  if (direct) return launch(op, n, A, U, V, smax, smin, s, flags, (cudaStream_t)stream);
  if (chunk == 0) chunk = int64_t(1) << 21;
  chunk = (chunk + 63) / 64 * 64;                 // keeps every sub-array 256-byte aligned
  const int64_t c = n < chunk ? n : chunk;
  // slot layout: A[na], U[na], V[na], smax, smin (each c elements of es bytes), s (c int32)
  const size_t arr = (size_t)c * es;
  const size_t slot = arr * (3 * na + 2) + (size_t)c * sizeof(int32_t);
  int dev = 0;
  SVD2_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return SVD2_EINVAL;
  std::lock_guard<std::mutex> g(g_mu);
  Stage &S = g_stage[dev];
  int rc = setup(S, slot);
  if (rc != SVD2_OK) return rc;
  const cudaStream_t caller = (cudaStream_t)stream;
  // the pipeline starts after the caller's prior work (calls are serialised
  // by g_mu, so one event per device serves every call)
  SVD2_CUDA_TRY(cudaEventRecord(S.start, caller));
  SVD2_CUDA_TRY(cudaStreamWaitEvent(S.st[0], S.start, 0));
  // ... and after the previous call's chunks have left both slots
  for (int b = 0; b < 2; ++b) SVD2_CUDA_TRY(cudaStreamWaitEvent(S.st[0], S.out_done[b], 0));
  const int64_t nchunks = (n + c - 1) / c;
  for (int64_t i = 0; i < nchunks; ++i) {
    const int b = (int)(i & 1);
    const int64_t off = i * c;
    const int64_t m = (n - off < c) ? (n - off) : c;
    auto *base = static_cast<unsigned char *>(S.buf[b]);
    void *dA[8], *dU[8], *dV[8];
    for (int e = 0; e < na; ++e) {
      dA[e] = base + arr * e;
      dU[e] = base + arr * (na + e);
      dV[e] = base + arr * (2 * na + e);
    }
    void *dsx = base + arr * (3 * na), *dsn = base + arr * (3 * na + 1);
    auto *ds = reinterpret_cast<int32_t *>(base + arr * (3 * na + 2));
    // stage 1: inputs of chunk i, once chunk i - 2 has left this slot
    if (i >= 2) SVD2_CUDA_TRY(cudaStreamWaitEvent(S.st[0], S.out_done[b], 0));
    for (int e = 0; e < na; ++e)
      SVD2_CUDA_TRY(cudaMemcpyAsync(dA[e], static_cast<const unsigned char *>(A[e]) + off * es,
                                    (size_t)m * es, cudaMemcpyHostToDevice, S.st[0]));
    SVD2_CUDA_TRY(cudaEventRecord(S.in_ready[b], S.st[0]));
    // stage 2: the kernel
    SVD2_CUDA_TRY(cudaStreamWaitEvent(S.st[1], S.in_ready[b], 0));
    if (i >= 2) SVD2_CUDA_TRY(cudaStreamWaitEvent(S.st[1], S.out_done[b], 0));
    rc = launch(op, m, dA, dU, dV, dsx, dsn, ds, flags, S.st[1]);
    if (rc != SVD2_OK) return rc;
    SVD2_CUDA_TRY(cudaEventRecord(S.computed[b], S.st[1]));
    // stage 3: outputs of chunk i
    SVD2_CUDA_TRY(cudaStreamWaitEvent(S.st[2], S.computed[b], 0));
    for (int e = 0; e < na; ++e) {
      SVD2_CUDA_TRY(cudaMemcpyAsync(static_cast<unsigned char *>(U[e]) + off * es, dU[e],
                                    (size_t)m * es, cudaMemcpyDeviceToHost, S.st[2]));
      SVD2_CUDA_TRY(cudaMemcpyAsync(static_cast<unsigned char *>(V[e]) + off * es, dV[e],
                                    (size_t)m * es, cudaMemcpyDeviceToHost, S.st[2]));
    }
    SVD2_CUDA_TRY(cudaMemcpyAsync(static_cast<unsigned char *>(smax) + off * es, dsx,
                                  (size_t)m * es, cudaMemcpyDeviceToHost, S.st[2]));
    SVD2_CUDA_TRY(cudaMemcpyAsync(static_cast<unsigned char *>(smin) + off * es, dsn,
                                  (size_t)m * es, cudaMemcpyDeviceToHost, S.st[2]));
    SVD2_CUDA_TRY(cudaMemcpyAsync(s + off, ds, (size_t)m * sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, S.st[2]));
    SVD2_CUDA_TRY(cudaEventRecord(S.out_done[b], S.st[2]));
  }
  // the caller's stream continues once every output has arrived
  SVD2_CUDA_TRY(cudaStreamWaitEvent(caller, S.out_done[(nchunks - 1) & 1], 0));
  if (nchunks >= 2) SVD2_CUDA_TRY(cudaStreamWaitEvent(caller, S.out_done[nchunks & 1], 0));
  return SVD2_OK;
}
