// svd2_batch_s_rerun_noalloc: the FP32 form with FP64 re-run for callers that
// cannot allocate device memory.
//
// The re-run form needs scratch memory: the call's re-run count, the flag of
// its fix-up pass and the index list of the matrices to re-run (4 bytes per
// matrix).  svd2_batch_s_rerun takes that scratch from the caller.  Some
// callers cannot provide it: an application whose device memory
// is entirely owned by another allocator (a framework's caching pool, or a host
// program that hands this library only the input and output buffers), or code
// that must not call cudaMalloc once it is running (cudaMalloc may synchronise
// the device, which a latency-bound loop or a system with a fixed start-up
// memory budget cannot accept).  This entry point keeps its scratch in the
// fixed array below instead, which the CUDA runtime places in device memory
// when the library is loaded: every device that loads the library holds
// kScratchBytes (about 4 MiB) until the process exits.
//
// Set-up: the first call on a device, with that device current, looks up the
// array's device address with cudaGetSymbolAddress (no allocation) and caches
// it; make that first call before any stream capture.  The cached address
// holds while the device's context lives: after cudaDeviceReset the module may
// be loaded again at another address, so the entry point must not be used
// across a device reset.  In host code the array's
// name is only a host-side stand-in, so the kernels always receive the looked-up
// address.  All calls on a device share the one array: the count, the flag and
// the list length are cleared at the start of each call, and calls whose
// work can overlap on the GPU -- on different streams without ordering between
// them -- race on it and must not be made.
#include <mutex>

#include "svd2_common.cuh"

namespace {

constexpr int64_t kMaxN = SVD2_NOALLOC_MAX_N;
// layout of the re-run workspace: 256 header bytes (counters), then one uint32
// index per matrix
constexpr size_t kScratchBytes = 256 + (size_t)kMaxN * sizeof(uint32_t);

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[64] = {nullptr};

// Device address of g_scratch on the current device (looked up once per device).
int scratch_address(void **addr) {
  int dev = 0;
  SVD2_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return SVD2_EINVAL;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return svd2::record_cuda_error(e);
    g_scratch_addr[dev] = p;
  }
  *addr = g_scratch_addr[dev];
  return SVD2_OK;
}

}  // namespace

extern "C" int svd2_batch_s_rerun_noalloc(int64_t n, const float *const A[4], float *const U[4],
                                          float *const V[4], float *smax, float *smin, int32_t *s,
                                          int tau_log2, uint32_t flags, svd2_stream_t stream) {
  if (n < 0) return SVD2_EINVAL;
  if (n > kMaxN) return SVD2_ETOOBIG;
  if (n == 0) return SVD2_OK;
  void *scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != SVD2_OK) return rc;
  return svd2_batch_s_rerun(n, A, U, V, smax, smin, s, tau_log2, flags, scratch, kScratchBytes,
                            stream);
}
