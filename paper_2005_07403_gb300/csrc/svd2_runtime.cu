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
    {1024, 4, 1, 2},  // s with the FP64 tangent step
};

Launch get_launch(int op) {
  std::lock_guard<std::mutex> g(g_launch_mu);
  return g_launch[op];
}

// One stream-ordered memory pool per device for the per-call flag blocks,
// created on first use and kept until the process exits; freed blocks stay in
// the pool (release threshold: never), so later calls do not allocate from
// the driver.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};

static int pool_of_current_device(cudaMemPool_t *out) {
  int dev = 0;
  SVD2_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return SVD2_EINVAL;
  std::lock_guard<std::mutex> g(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    SVD2_CUDA_TRY(cudaMemPoolCreate(&pool, &props));
    uint64_t keep = UINT64_MAX;
    SVD2_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    g_pool[dev] = pool;
  }
  *out = g_pool[dev];
  return SVD2_OK;
}

int flag_block(cudaStream_t st, void **p) {
  cudaMemPool_t pool = nullptr;
  const int rc = pool_of_current_device(&pool);
  if (rc != SVD2_OK) return rc;
  SVD2_CUDA_TRY(cudaMallocFromPoolAsync(p, 256, pool, st));
  SVD2_CUDA_TRY(cudaMemsetAsync(*p, 0, 256, st));
  return SVD2_OK;
}

int flag_release(void *p, cudaStream_t st) {
  SVD2_CUDA_TRY(cudaFreeAsync(p, st));
  return SVD2_OK;
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
  if (block < 32 || block > max_block(op) || block % 32) return SVD2_EINVAL;
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
