// Host-side plumbing shared by the library's translation units: error
// recording, device properties, launch shapes and the vector memory helpers of
// the streaming kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "svd2.h"

namespace svd2 {

// ------------------------------------------------------------ error state

int record_cuda_error(cudaError_t e);   // stores e for svd2_last_cuda_error, returns SVD2_ECUDA

#define SVD2_CUDA_TRY(call)                                  \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return ::svd2::record_cuda_error(e_); \
  } while (0)

// Number of SMs of the current device (cached per device).
int sm_count();
// A 256-byte block of device memory, zeroed in stream order on st, from the
// library's stream-ordered pool of the current device (per-call flags of the
// fast/fix-up kernel pair); flag_release returns it in stream order.
int flag_block(cudaStream_t st, void **p);
int flag_release(void *p, cudaStream_t st);

// ----------------------------------------------------------- launch shape

struct Launch {
  int block;    // threads per block
  int mpt;      // matrices per thread per load group
  int unroll;   // load groups in flight per thread
  int waves;    // grid = waves * SMs * resident blocks per SM (0: cover the work)
};

// op 4: the real FP32 form with the FP64 tangent step (its own launch shape)
enum Op { kOpD = 0, kOpZ = 1, kOpS = 2, kOpC = 3, kOpSTan64 = 4, kNumOps = 5 };
// Largest block size of op's batch kernel (its launch bounds): 1024 where the
// kernel is held to 64 registers anyway (FP64, complex, the tangent step),
// 512 for the plain real FP32 kernel, which may use up to 128.
inline int max_block(int op) { return op == kOpS ? 512 : 1024; }
Launch get_launch(int op);

// Grid size for `units` work items of `block` threads each, capped as above.
int64_t grid_for(int64_t units, const Launch &L, int resident_blocks_per_sm);

inline bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// ------------------------------------------------- vector loads and stores

// Load M consecutive elements of T starting at p (p aligned to min(16, M*sizeof(T))).
// Streaming (evict-first) cache policy: every input is read once.
template <typename T, int M>
__device__ __forceinline__ void load_vec(const T *p, T (&x)[M]) {
  constexpr int B = M * (int)sizeof(T);
  if constexpr (B >= 16) {
#pragma unroll
    for (int k = 0; k < B / 16; ++k) {
      const uint4 w = __ldcs(reinterpret_cast<const uint4 *>(p) + k);
      memcpy(&x[k * (16 / sizeof(T))], &w, 16);
    }
  } else if constexpr (B == 8) {
    const uint2 w = __ldcs(reinterpret_cast<const uint2 *>(p));
    memcpy(&x[0], &w, 8);
  } else {
    const unsigned w = __ldcs(reinterpret_cast<const unsigned *>(p));
    memcpy(&x[0], &w, 4);
  }
}

// Store M consecutive elements; streaming stores (written once, not re-read).
template <typename T, int M>
__device__ __forceinline__ void store_vec(T *p, const T (&x)[M]) {
  constexpr int B = M * (int)sizeof(T);
  if constexpr (B >= 16) {
#pragma unroll
    for (int k = 0; k < B / 16; ++k) {
      uint4 w;
      memcpy(&w, &x[k * (16 / sizeof(T))], 16);
      __stcs(reinterpret_cast<uint4 *>(p) + k, w);
    }
  } else if constexpr (B == 8) {
    uint2 w;
    memcpy(&w, &x[0], 8);
    __stcs(reinterpret_cast<uint2 *>(p), w);
  } else {
    unsigned w;
    memcpy(&w, &x[0], 4);
    __stcs(reinterpret_cast<unsigned *>(p), w);
  }
}

}  // namespace svd2
