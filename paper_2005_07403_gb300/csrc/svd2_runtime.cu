// Library runtime: per-thread error state, device-property cache, the
// process-wide launch-shape table, and the version string.
#include <mutex>

#include "svd2_common.cuh"

namespace svd2 {

static thread_local int g_last_cuda_error = 0;

int record_cuda_error(cudaError_t e) {
  g_last_cuda_error = (int)e;
  return SVD2_ECUDA;
}

int sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (!cache[dev]) {
    int c = 0;
    if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0)
      c = 152;
    cache[dev] = c;
  }
  return cache[dev];
}

// Defaults, from the autotuner on GB300 (n = 2^24 .. 2^26): the FP64 forms are
// bound by arithmetic and take one matrix per thread; the real FP32 form is
// bound by issue and HBM and takes 8-byte vectors with a capped grid.
static std::mutex g_launch_mu;
static Launch g_launch[kNumOps] = {
    {256, 1, 1, 0},   // d
    {512, 1, 1, 0},   // z
    {512, 2, 1, 4},   // s
    {256, 2, 1, 0},   // c
};

Launch get_launch(int op) {
  std::lock_guard<std::mutex> g(g_launch_mu);
  return g_launch[op];
}

int64_t grid_for(int64_t units, const Launch &L, int resident_blocks_per_sm) {
  int64_t need = (units + L.block - 1) / L.block;
  if (need < 1) need = 1;
  if (L.waves > 0) {
    const int64_t cap = (int64_t)L.waves * sm_count() * (resident_blocks_per_sm > 0 ? resident_blocks_per_sm : 1);
    if (need > cap) need = cap;
  }
  if (need > 0x7fffffffLL) need = 0x7fffffffLL;
  return need;
}

}  // namespace svd2

using namespace svd2;

extern "C" int svd2_set_launch(int op, int block, int mpt, int unroll, int waves) {
  if (op < 0 || op >= kNumOps) return SVD2_EINVAL;
  if (block < 32 || block > 512 || block % 32) return SVD2_EINVAL;
  if (mpt != 1 && mpt != 2 && mpt != 4) return SVD2_EINVAL;
  if (unroll != 1 && unroll != 2) return SVD2_EINVAL;
  if (waves < 0 || waves > 1024) return SVD2_EINVAL;
  std::lock_guard<std::mutex> g(g_launch_mu);
  g_launch[op] = Launch{block, mpt, unroll, waves};
  return SVD2_OK;
}

extern "C" int svd2_get_launch(int op, int *block, int *mpt, int *unroll, int *waves) {
  if (op < 0 || op >= kNumOps) return SVD2_EINVAL;
  const Launch L = get_launch(op);
  if (block) *block = L.block;
  if (mpt) *mpt = L.mpt;
  if (unroll) *unroll = L.unroll;
  if (waves) *waves = L.waves;
  return SVD2_OK;
}

extern "C" int svd2_last_cuda_error(void) { return g_last_cuda_error; }

extern "C" const char *svd2_version(void) { return "svd2-gb300 0.1 (sm_103a)"; }
