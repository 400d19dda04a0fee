// Autotuner of the launch shapes: svd2_autotune_fwd and svd2_multi_autotune.
//
// The best block size, matrices per thread (vector width of the loads) and
// number of load groups in flight depend on the form (the FP64 forms are bound
// by arithmetic, the FP32 ones by HBM), on the register count of each kernel
// instantiation and on the batch size.  The tuner times every candidate shape
// on the caller's own batch with CUDA events on the caller's stream and keeps
// the fastest (ties to the earlier candidate).
#include <cfloat>

#include "svd2_common.cuh"

namespace {

int call_fwd(int op, int64_t n, const void *const *A, void *const *U, void *const *V, void *smax,
             void *smin, int32_t *s, cudaStream_t st) {
  const auto stream = (svd2_stream_t)st;
  switch (op) {
    case 0:
      return svd2_batch_d(n, (const double *const *)A, (double *const *)U, (double *const *)V,
                          (double *)smax, (double *)smin, s, 0, stream);
    case 1:
      return svd2_batch_z(n, (const double *const *)A, (double *const *)U, (double *const *)V,
                          (double *)smax, (double *)smin, s, 0, stream);
    case 2:
      return svd2_batch_s(n, (const float *const *)A, (float *const *)U, (float *const *)V,
                          (float *)smax, (float *)smin, s, 0, stream);
    case 3:
      return svd2_batch_c(n, (const float *const *)A, (float *const *)U, (float *const *)V,
                          (float *)smax, (float *)smin, s, 0, stream);
    case svd2::kOpSTan64:
      return svd2_batch_s_tan64(n, (const float *const *)A, (float *const *)U,
                                (float *const *)V, (float *)smax, (float *)smin, s,
                                SVD2_TAN64_TAU_LOG2, 0, nullptr, stream);
    default:
      return SVD2_EINVAL;
  }
}

// Time `reps` calls of f after one warm-up call; *ms = milliseconds per call.
template <typename F>
int time_calls(F f, int reps, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, float *ms) {
  int rc = f();
  if (rc != SVD2_OK) return rc;
  SVD2_CUDA_TRY(cudaEventRecord(e0, st));
  for (int r = 0; r < reps; ++r) {
    rc = f();
    if (rc != SVD2_OK) return rc;
  }
  SVD2_CUDA_TRY(cudaEventRecord(e1, st));
  SVD2_CUDA_TRY(cudaEventSynchronize(e1));
  float t = 0;
  SVD2_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
  *ms = t / reps;
  return SVD2_OK;
}

struct Events {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaSuccess;
  Events() {
    err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
  }
  ~Events() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

}  // namespace

using namespace svd2;

extern "C" int svd2_autotune_fwd(int op, int64_t n, const void *const *A, void *const *U,
                                 void *const *V, void *smax, void *smin, int32_t *s, int reps,
                                 svd2_tune_result *best, svd2_stream_t stream) {
  if (op < 0 || op >= kNumOps || n <= 0 || reps < 1 || !best) return SVD2_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  Events ev;
  if (ev.err != cudaSuccess) return record_cuda_error(ev.err);
  const Launch saved = get_launch(op);
  // block sizes above the op's kernel limit are refused by set_launch and skipped
  static const int blocks[] = {64, 128, 256, 512, 1024};
  static const int mpts[] = {1, 2, 4};
  static const int unrolls[] = {1, 2};
  // grid: as the work needs (0), or 1, 2 or 4 resident waves (on the tangent-step
  // kernel 1 - 2 waves of 1024-thread blocks measured 0.6% above 4)
  static const int waves[] = {0, 1, 2, 4};
  svd2_tune_result b{0, 0, 0, 0, FLT_MAX};
  for (int bl : blocks)
    for (int m : mpts)
      for (int u : unrolls)
        for (int w : waves) {
          int rc = svd2_set_launch(op, bl, m, u, w);
          if (rc != SVD2_OK) continue;
          float ms = 0;
          rc = time_calls([&] { return call_fwd(op, n, A, U, V, smax, smin, s, st); }, reps, st,
                          ev.e0, ev.e1, &ms);
          if (rc != SVD2_OK) {
            svd2_set_launch(op, saved.block, saved.mpt, saved.unroll, saved.waves);
            return rc;
          }
          if (ms < b.ms) b = svd2_tune_result{bl, m, u, w, ms};
        }
  svd2_set_launch(op, b.block, b.mpt, b.unroll, b.waves);
  *best = b;
  return SVD2_OK;
}

extern "C" int svd2_multi_autotune(const svd2_batch_desc *descs, int32_t nbatch, void *plan,
                                   size_t plan_bytes, int reps, svd2_tune_result *best,
                                   svd2_stream_t stream) {
  if (nbatch < 0 || reps < 1 || !best) return SVD2_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  Events ev;
  if (ev.err != cudaSuccess) return record_cuda_error(ev.err);
  static const int blocks[] = {64, 128, 256, 512, 1024};
  static const int mpts[] = {1, 2, 4};
  static const int unrolls[] = {1, 2};
  svd2_tune_result b{0, 0, 0, 0, FLT_MAX};
  for (int bl : blocks)
    for (int m : mpts)
      for (int u : unrolls) {
        int rc = svd2_multi_prepare(descs, nbatch, bl, m, u, plan, plan_bytes, nullptr);
        if (rc != SVD2_OK) return rc;
        float ms = 0;
        rc = time_calls([&] { return svd2_multi_run(plan, bl, m, u, 0, stream); }, reps, st,
                        ev.e0, ev.e1, &ms);
        if (rc != SVD2_OK) return rc;
        if (ms < b.ms) b = svd2_tune_result{bl, m, u, 0, ms};
      }
  const int rc = svd2_multi_prepare(descs, nbatch, b.block, b.mpt, b.unroll, plan, plan_bytes,
                                    nullptr);
  if (rc != SVD2_OK) return rc;
  *best = b;
  return SVD2_OK;
}
