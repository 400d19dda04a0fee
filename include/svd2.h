/*
 * svd2.h -- C ABI of the GB300 (sm_103a) batched 2x2 SVD library.
 *
 * Computes, for n independent real or complex 2x2 matrices A, the SVD
 * A = U Sigma V^* by the method of V. Novakovic, "Batched computation of the
 * singular value decompositions of order two by the AVX-512 vectorization"
 * (arXiv 2005.07403): exact power-of-two scaling (Sec. 2.1, Eq. 2), the URV
 * factorization (Sec. 2.2, Eq. 4 - Eq. 11), the SVD of the non-negative upper
 * triangular middle factor (Sec. 2.3, Eq. 12 - Eq. 17) and the assembly of U
 * and V (Eq. 28, Eq. 29).  This is the annihilation step of one parallel
 * Kogbetliantz sweep (Sec. 1).
 *
 * Data layout (Sec. 3): the split layout.  Each matrix element has its own
 * contiguous array of n values, the real and imaginary parts of complex
 * elements in separate arrays.  Element arrays are passed as a HOST array of
 * DEVICE pointers, in the record order of Sec. 8:
 *   real    (4): a11, a21, a12, a22
 *   complex (8): Re a11, Im a11, Re a21, Im a21, Re a12, Im a12, Re a22, Im a22
 * U and V use the same order as A.  smax, smin and s are arrays of n values.
 * All device arrays are caller-owned (the library never frees them), must be
 * distinct from each other (outputs must not alias inputs or each other) and
 * may have any alignment of their element type; 16-byte aligned arrays take
 * vectorised loads and stores.
 *
 * Outputs (Sec. 2.3, Fig. 1): by default smax, smin hold the scaled singular
 * values Sigma' (sigma'_max >= sigma'_min >= 0, always finite for finite
 * input, Theorem 1) and s holds the scale exponent of Eq. 2, so that
 * Sigma = 2^-s Sigma'.  The zero matrix has s = SVD2_S_ZERO (the paper's
 * s = DBL_MAX).  With SVD2_BACKSCALE the library stores Sigma = 2^-s Sigma'
 * (correctly rounded; it may overflow or underflow, Sec. 2.3) and s = 0.
 *
 * Preconditions and errors: inputs must be finite (Sec. 1); non-finite input
 * gives unspecified values but never a fault or a hang.  All entry points are
 * asynchronous on the given stream (NULL = the legacy default stream) and
 * return SVD2_OK, or a negative code: SVD2_EINVAL for a bad argument (n < 0, a
 * NULL array with n > 0, unknown flags), SVD2_ECUDA when a CUDA call failed
 * (its cudaError_t is kept per thread for svd2_last_cuda_error()).  n == 0 is
 * a no-op.  Inputs are never modified.
 */
#ifndef SVD2_H
#define SVD2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; declared here so the header needs no CUDA headers. */
typedef struct CUstream_st *svd2_stream_t;

#define SVD2_OK 0
#define SVD2_EINVAL (-1)
#define SVD2_ECUDA (-2)
#define SVD2_ENOMEM (-3)
#define SVD2_ETOOBIG (-4)     /* n above the fixed capacity of an allocation-free entry point */

#define SVD2_S_ZERO INT32_MAX      /* s of the all-zero matrix (Eq. 2: s = DBL_MAX) */
#define SVD2_BACKSCALE 1u          /* store Sigma = 2^-s Sigma' and s = 0 (Fig. 1)  */
/* Assemble U by Eq. 31 -- from sin = cos tan of the angles (Sec. 7) -- in
 * place of the tangent form of Eq. 29 (the same matrix in exact arithmetic;
 * V, Sigma' and s are unchanged).  Accepted by svd2_batch_{d,z,s,c} and
 * svd2_batch_host (ops 0 - 3) only; other entry points return SVD2_EINVAL. */
#define SVD2_SINE 2u

/*
 * Real FP64: n matrices.  A[4], U[4], V[4] hold device pointers to n doubles
 * each; smax, smin: n doubles; s: n int32.  Sec. 2 with the real forms of
 * Eq. 10; every step is a correctly rounded IEEE double operation in the
 * paper's order, so the results are those of the step-by-step method.
 * Every batch form runs as two kernels on the stream: the batch kernel
 * finishes every matrix whose divisions, square roots and scaling stay in the
 * normal range on branch-free instruction sequences and marks the others; a
 * second kernel (which reads one flag word and ends when nothing was marked)
 * recomputes the marked ones (zero columns, subnormal entries, entries
 * spanning the exponent range) with the general sequences -- the same
 * correctly rounded results either way.  Each call takes a 256-byte flag block
 * from a stream-ordered memory pool that the library creates per device on
 * first use (it keeps what it allocates until the process exits).
 */
int svd2_batch_d(int64_t n, const double *const A[4], double *const U[4],
                 double *const V[4], double *smax, double *smin, int32_t *s,
                 uint32_t flags, svd2_stream_t stream);

/* Complex FP64 (complex128 split into real and imaginary parts): A[8], U[8],
 * V[8] of n doubles each.  Sec. 2, Eq. 1 - Eq. 29, Fig. 3 - Fig. 10. */
int svd2_batch_z(int64_t n, const double *const A[8], double *const U[8],
                 double *const V[8], double *smax, double *smin, int32_t *s,
                 uint32_t flags, svd2_stream_t stream);

/* Real FP32: the single-precision variant of Sec. 1 and Sec. 7 (FLT_*
 * constants, h = FLT_MAX_EXP - 3 = 125, tan(2 phi) bounded by sqrt(FLT_MAX)).
 * Two kernels and a flag block per call, as svd2_batch_d. */
int svd2_batch_s(int64_t n, const float *const A[4], float *const U[4],
                 float *const V[4], float *smax, float *smin, int32_t *s,
                 uint32_t flags, svd2_stream_t stream);

/* Complex FP32 (complex64 split into parts); as svd2_batch_z in single precision. */
int svd2_batch_c(int64_t n, const float *const A[8], float *const U[8],
                 float *const V[8], float *smax, float *smin, int32_t *s,
                 uint32_t flags, svd2_stream_t stream);

/*
 * Singular values only (the counterpart of LAPACK's xLAS2, named with xLASV2
 * at the start of Sec. 2): the method of svd2_batch_{d,z,s,c} without the
 * assembly of U and V (Eq. 28, Eq. 29) and without their stores.  smax, smin
 * and s receive exactly the values the full form stores (Sigma', s; with
 * SVD2_BACKSCALE, Sigma and s = 0).  A as for the full form; the per-matrix
 * traffic falls to 52 B (real FP64), 84 B (complex128), 28 B (real FP32),
 * 44 B (complex64).  Errors as above.
 */
int svd2_values_d(int64_t n, const double *const A[4], double *smax, double *smin,
                  int32_t *s, uint32_t flags, svd2_stream_t stream);
int svd2_values_z(int64_t n, const double *const A[8], double *smax, double *smin,
                  int32_t *s, uint32_t flags, svd2_stream_t stream);
int svd2_values_s(int64_t n, const float *const A[4], float *smax, float *smin,
                  int32_t *s, uint32_t flags, svd2_stream_t stream);
int svd2_values_c(int64_t n, const float *const A[8], float *smax, float *smin,
                  int32_t *s, uint32_t flags, svd2_stream_t stream);

/*
 * The interleaved layout: the n matrices as one row-major (n, 2, 2) array, each
 * matrix's entries contiguous -- the one-matrix-at-a-time data of the
 * pointwise routine x1svd2 (Sec. 4: the interface of Sec. 4 with S = 1), and
 * torch's layout for a batch of 2x2 real or complex matrices.  A, U, V: device pointers to n*4 values (real: a11 a12 a21
 * a22) or n*8 values (complex: Re a11, Im a11, Re a12, Im a12, Re a21, Im a21,
 * Re a22, Im a22); U and V in the same layout.  U and V both NULL: singular
 * values only; one NULL: SVD2_EINVAL.  smax, smin, s: n values each.  Results
 * bit-identical to the split-layout forms on the same matrices.  Errors as
 * above.
 */
int svd2_batch_interleaved_d(int64_t n, const double *A, double *U, double *V, double *smax,
                             double *smin, int32_t *s, uint32_t flags, svd2_stream_t stream);
int svd2_batch_interleaved_z(int64_t n, const double *A, double *U, double *V, double *smax,
                             double *smin, int32_t *s, uint32_t flags, svd2_stream_t stream);
int svd2_batch_interleaved_s(int64_t n, const float *A, float *U, float *V, float *smax,
                             float *smin, int32_t *s, uint32_t flags, svd2_stream_t stream);
int svd2_batch_interleaved_c(int64_t n, const float *A, float *U, float *V, float *smax,
                             float *smin, int32_t *s, uint32_t flags, svd2_stream_t stream);

/*
 * One parallel step of the Kogbetliantz method for the SVD of an m x m matrix
 * G (Sec. 1), m = 2n even.  pairs: device array of m int32, the pivot pairs
 * (p_0, q_0, p_1, q_1, ...), together a permutation of 0 .. m-1.  The step
 * gathers the n pivot blocks A^[k] (elements (p_k,p_k), (q_k,p_k), (p_k,q_k),
 * (q_k,q_k)), computes their SVDs by the method (with the back-scaling of
 * Fig. 1), and updates G in place from the left by (U^[k])^* on rows p_k, q_k
 * and from the right by V^[k] on columns p_k, q_k; the pivot blocks become
 * diag(sigma_max, sigma_min) with the off-diagonal pivot positions exactly 0.
 * G: device matrix, element (r, c) at G[r rs + c cs] -- column-major
 * (rs = 1, cs = leading dimension >= m) or row-major (cs = 1, rs >= m); for
 * z and c the elements are complex (real and imaginary part adjacent, as in
 * complex128/complex64 arrays), strides counted in complex elements.
 * workspace: device memory of svd2_kog_workspace_bytes(op, m) bytes (op:
 * 0 = d, 1 = z, 2 = s, 3 = c), 256-byte aligned, used by this call only; it
 * holds U, V, Sigma of the step and, at offset 0, the number of pairs skipped
 * because an index was outside 0 .. m-1 or p = q (svd2_kog_skipped; every
 * 2x2 block in the rows or the columns of a skipped pair is left untouched).  Pairs that repeat an index give
 * unspecified values (the blocks overlap) but never an out-of-range access.
 * Two kernels on `stream`.  Errors: SVD2_EINVAL for m odd or < 2, NULL
 * pointers, another layout, a small or misaligned workspace; SVD2_ECUDA.
 */
size_t svd2_kog_workspace_bytes(int op, int64_t m);
int svd2_kog_step_d(int64_t m, double *G, int64_t rs, int64_t cs, const int32_t *pairs,
                    void *workspace, size_t workspace_bytes, svd2_stream_t stream);
int svd2_kog_step_z(int64_t m, double *G, int64_t rs, int64_t cs, const int32_t *pairs,
                    void *workspace, size_t workspace_bytes, svd2_stream_t stream);
int svd2_kog_step_s(int64_t m, float *G, int64_t rs, int64_t cs, const int32_t *pairs,
                    void *workspace, size_t workspace_bytes, svd2_stream_t stream);
int svd2_kog_step_c(int64_t m, float *G, int64_t rs, int64_t cs, const int32_t *pairs,
                    void *workspace, size_t workspace_bytes, svd2_stream_t stream);
/* Pairs skipped by the last step that used `workspace`; synchronous. */
int svd2_kog_skipped(const void *workspace, int64_t *count);

/*
 * FP32 form with FP64 re-run.  The single-precision method (as svd2_batch_s /
 * svd2_batch_c) runs over all n matrices; every matrix whose scaled singular
 * values satisfy sigma'_min < 2^tau_log2 * sigma'_max (compared in float, the
 * product by the power of two being exact) is decomposed again by the
 * double-precision method on its exactly widened elements, and its float
 * outputs are replaced by the double results rounded to nearest float, with
 * sigma' on the float run's scale: sigma'_32 = RN(sigma'_64 * 2^(s32 - s64)).
 * s is the float run's exponent (h = 125).  The tangent and cosine
 * computations of Eq. 6 - Eq. 16 are where single precision loses the
 * small singular value of an ill-conditioned matrix (sigma'_min carries about
 * u * sigma'_max / sigma'_min relative error from r''_22, Fig. 8); a kept
 * matrix has sigma'_min / sigma'_max >= 2^tau_log2, bounding that error.
 * tau_log2 in [-100, 0]; the library's measured default is SVD2_RERUN_TAU_LOG2.
 * Four kernels on the stream: the single-precision batch kernel, which marks
 * the matrices to re-run; a compaction of their indices into the workspace;
 * the double-precision re-run of the listed matrices; the fix-up pass.
 * workspace: device memory of at least svd2_rerun_workspace_bytes(n) bytes
 * (256 bytes plus 4 per matrix for the index list),
 * 16-byte aligned, caller-owned, used by this call only (two calls sharing a
 * workspace must be ordered on one stream).  After the call completes, its
 * first 8 bytes hold the number of re-run matrices (uint64), see
 * svd2_rerun_count.  flags as for svd2_batch_s (SVD2_BACKSCALE applies Fig. 1
 * to the final float results).  Errors as above.
 */
#define SVD2_RERUN_TAU_LOG2 (-8)
size_t svd2_rerun_workspace_bytes(int64_t n);
int svd2_batch_s_rerun(int64_t n, const float *const A[4], float *const U[4],
                       float *const V[4], float *smax, float *smin, int32_t *s,
                       int tau_log2, uint32_t flags, void *workspace,
                       size_t workspace_bytes, svd2_stream_t stream);
int svd2_batch_c_rerun(int64_t n, const float *const A[8], float *const U[8],
                       float *const V[8], float *smax, float *smin, int32_t *s,
                       int tau_log2, uint32_t flags, void *workspace,
                       size_t workspace_bytes, svd2_stream_t stream);
/* Number of matrices re-run by the last call that used `workspace` (a device
 * pointer); synchronous: call it once that call has completed. */
int svd2_rerun_count(const void *workspace, int64_t *count);

/*
 * Real FP32 form with the FP64 tangent step.  The single-precision method (as
 * svd2_batch_s) runs over all n matrices, and where a matrix is
 * ill-conditioned one step of it runs in double precision: when
 * |r''_22| < 2^tau_log2 * r11 at Eq. 7 (compared in float; r''_22 / r11 is
 * within a factor of two of sigma_min / sigma_max, since r11 <= sigma_max <=
 * sqrt(2) r11 after the column pivoting of Fig. 5), the quotient
 * -tan(alpha) = a'''_21 / a'''_11 of Eq. 6 and the fma of Eq. 7 are evaluated
 * in double on the exactly widened a''' and
 * r''_22 = RN32(cos(alpha) * RN32(fma64(tan(alpha), a'''_12, a'''_22))).
 * Every other step stays in float.  In the real case the a''' are the
 * scaled entries with their signs changed, so they are exact in float and
 * the cancellation of Eq. 7 -- where single precision loses the small
 * singular value of an ill-conditioned matrix (Fig. 8) -- is the double
 * method's own.  Matrices that do not take the step get exactly the
 * svd2_batch_s results.  tau_log2 in [-100, 0]; SVD2_TAN64_TAU_LOG2 is the
 * library's measured default.  count: NULL, or a device uint64 to which the
 * call ADDS the number of matrices that took the step (zero it first).  One
 * kernel and the fix-up pass on the stream; no workspace.  Other arguments,
 * results and errors as svd2_batch_s (the paper reports no single-precision
 * results; Sec. 1 and Sec. 7 remark on single precision).
 */
#define SVD2_TAN64_TAU_LOG2 (-3)
int svd2_batch_s_tan64(int64_t n, const float *const A[4], float *const U[4],
                       float *const V[4], float *smax, float *smin, int32_t *s,
                       int tau_log2, uint32_t flags, unsigned long long *count,
                       svd2_stream_t stream);

/*
 * svd2_batch_s_rerun without a workspace argument, for callers that cannot
 * allocate device memory: an application whose device memory belongs to
 * another allocator (a framework's caching pool, or a host program that gives
 * this library only the input and output buffers), or code that must not call
 * cudaMalloc once running (cudaMalloc may synchronise the device, which a
 * latency-bound loop or a fixed start-up memory budget cannot accept).  The
 * paper has no counterpart; it is a deployment variant of the re-run form.
 * The scratch (sized by the workspace formula of svd2_batch_s_rerun for
 * SVD2_NOALLOC_MAX_N matrices) is a fixed array of about 4 MiB in
 * device memory, reserved on every device that loads the library until the
 * process exits; n is limited to SVD2_NOALLOC_MAX_N matrices (larger n returns
 * SVD2_ETOOBIG) -- split larger batches, or use svd2_batch_s_rerun.  The first
 * call on a device (with that device current) looks up the array's address;
 * make it before any stream capture.  The address is kept for the life of the
 * process, so the entry point must not be used on a device after
 * cudaDeviceReset (which may reload the library's device code elsewhere).  The call allocates nothing.  All calls
 * on one device share the array: calls whose GPU work may overlap (different
 * streams with no ordering between them) race and must not be made.
 * Arguments, results and other errors as svd2_batch_s_rerun.
 */
#define SVD2_NOALLOC_MAX_N (1 << 20)
int svd2_batch_s_rerun_noalloc(int64_t n, const float *const A[4], float *const U[4],
                               float *const V[4], float *smax, float *smin, int32_t *s,
                               int tau_log2, uint32_t flags, svd2_stream_t stream);

/*
 * Backward (adjoint) of the real 2x2 SVD, FP64 and FP32.  The paper defines
 * no backward; this is the differentiation form built on its forward.  For
 * A = U diag(s1, s2) V^T and a loss with gradients gU, gV (element order
 * u11, u21, u12, u22) and g1, g2, it writes
 *   gA = U M V^T,  M = [[g1, p - q], [-p - q, g2]],  J = U^T gU,  K = V^T gV,
 *   a = J12 - J21,  b = K12 - K21,  p = (a-b)/(2(s1+s2)),  q = (a+b)/(2(s1-s2)),
 * with 1/(s1 - s2) replaced by g / (s1 (g^2 + rel_delta^2)), g = (s1 - s2)/s1,
 * which equals it for g >> rel_delta and stays bounded as the singular values
 * meet (rel_delta >= 0; 0 disables the safeguard, except that s1 = s2, where
 * the formula reads 0/0, gives the safeguard's value at zero gap, 0).  s1, s2 are the singular
 * values themselves (back-scaled: a forward call with SVD2_BACKSCALE).  U, V,
 * s1, s2 as produced by svd2_batch_d / svd2_batch_s.  gU, gV may be NULL (and
 * their entries, g1, g2) to mean zero gradients.  Device arrays of n values,
 * asynchronous on stream; errors as above.
 */
int svd2_bwd_d(int64_t n, const double *const U[4], const double *const V[4],
               const double *s1, const double *s2, const double *const gU[4],
               const double *const gV[4], const double *g1, const double *g2,
               double *const gA[4], double rel_delta, svd2_stream_t stream);
int svd2_bwd_s(int64_t n, const float *const U[4], const float *const V[4],
               const float *s1, const float *s2, const float *const gU[4],
               const float *const gV[4], const float *g1, const float *g2,
               float *const gA[4], float rel_delta, svd2_stream_t stream);

/*
 * Backward of the complex 2x2 SVD, FP64 and FP32 (split layout, 8 arrays each
 * for U, V, gU, gV, gA: real and imaginary parts of u11, u21, u12, u22).
 * Gradients are dL/dRe + i dL/dIm (so the real and imaginary rows of gA are
 * the derivatives with respect to the real and imaginary rows of A).  For
 * A = U diag(s1, s2) V^*, J = U^* gU, K = V^* gV, a = J12 - conj(J21),
 * b = K12 - conj(K21), p, q as in svd2_bwd_d (complex now, same safeguard):
 *   gA = U M V^*,  M = [[g1 + i t1, p - q], [-conj(p) - conj(q), g2 + i t2]],
 *   t_i = (Im J_ii - Im K_ii) / (2 s_i)   (0 when s_i = 0).
 * The singular vectors are determined only up to the phase gauge
 * U, V -> U D, V D (D unitary diagonal); the t_i terms are exact for losses
 * invariant under it (then Im J_ii + Im K_ii = 0), the losses whose
 * derivative is defined.  For real data the result is svd2_bwd_d's.  The
 * paper defines no backward.  Arguments, NULL gradients and errors as
 * svd2_bwd_d.
 */
int svd2_bwd_z(int64_t n, const double *const U[8], const double *const V[8],
               const double *s1, const double *s2, const double *const gU[8],
               const double *const gV[8], const double *g1, const double *g2,
               double *const gA[8], double rel_delta, svd2_stream_t stream);
int svd2_bwd_c(int64_t n, const float *const U[8], const float *const V[8],
               const float *s1, const float *s2, const float *const gU[8],
               const float *const gV[8], const float *g1, const float *g2,
               float *const gA[8], float rel_delta, svd2_stream_t stream);

/*
 * Many batches in one launch (the batches of one or more parallel Kogbetliantz
 * steps, Sec. 1), real FP64 and complex FP64 mixed.  Each batch is described
 * as for svd2_batch_d / svd2_batch_z; the batches are cut into tiles of
 * block * mpt * unroll matrices and the grid walks the tiles in a fixed
 * round-robin order (no atomics, no scratch, deterministic; the results equal
 * those of one svd2_batch_d / svd2_batch_z call per batch).
 *
 * svd2_multi_plan_bytes(nbatch): device bytes of a plan for nbatch batches.
 * svd2_multi_prepare: writes the plan for this launch shape (block a multiple
 *   of 32 in 32..1024, mpt in {1, 2, 4}, unroll in {1, 2}) to the caller-owned
 *   device buffer `plan` (16-byte aligned) with a synchronous copy, and returns
 *   the tile count in *total_tiles (may be NULL).  descs is a host array.
 * svd2_multi_run: one launch per kind over the plan, then the fix-up pass
 *   over every batch (reads the plan's flag word and ends when nothing was
 *   marked), asynchronous on `stream`; block, mpt and unroll must be those of
 *   the plan: for a plan prepared in this process another tile size returns
 *   SVD2_EINVAL (a plan copied in from elsewhere is checked by the kernels,
 *   which then process nothing).  grid 0: one block per tile for a plan prepared in
 *   this process (the tile counts are remembered on the host; the fastest on
 *   GB300), else SMs x resident blocks; grid > 0: that many blocks, a
 *   persistent grid walking the tiles when it is at most the resident count.
 * svd2_multi_graph_create: the same launch captured into an executable CUDA
 *   graph (*graph_exec), replayed with svd2_graph_launch and freed with
 *   svd2_graph_destroy.  The plan and the batch arrays must stay allocated
 *   while the graph is used; their contents may change between replays.
 */
#define SVD2_KIND_D 0
#define SVD2_KIND_Z 1
typedef struct svd2_batch_desc {
  int32_t kind;        /* SVD2_KIND_D or SVD2_KIND_Z */
  uint32_t flags;      /* 0 or SVD2_BACKSCALE */
  int64_t n;           /* matrices in this batch */
  const void *a[8];    /* element arrays of A (4 used when real), record order */
  void *u[8];
  void *v[8];
  void *smax;
  void *smin;
  int32_t *s;
} svd2_batch_desc;
size_t svd2_multi_plan_bytes(int32_t nbatch);
int svd2_multi_prepare(const svd2_batch_desc *descs, int32_t nbatch, int block, int mpt,
                       int unroll, void *plan, size_t plan_bytes, int64_t *total_tiles);
int svd2_multi_run(const void *plan, int block, int mpt, int unroll, int grid,
                   svd2_stream_t stream);
int svd2_multi_graph_create(const void *plan, int block, int mpt, int unroll, int grid,
                            void **graph_exec);
int svd2_graph_launch(void *graph_exec, svd2_stream_t stream);
int svd2_graph_destroy(void *graph_exec);

/*
 * Autotuner.  svd2_autotune_fwd times the forward kernel of op (0 = d, 1 = z,
 * 2 = s, 3 = c, 4 = svd2_batch_s_tan64 at SVD2_TAN64_TAU_LOG2) on the caller's
 * batch (arguments as for svd2_batch_*) for every block in {64, 128, 256,
 * 512, 1024} that the op admits (see svd2_set_launch), mpt in {1, 2, 4},
 * unroll in {1, 2} and waves in {0, 1, 2, 4}, `reps` timed launches each after one
 * warm-up launch, sets the fastest as the op's launch shape and returns it
 * with its time per launch (ms).  svd2_multi_autotune does the same for the
 * multi-batch launch (block in {64, 128, 256, 512, 1024}, mpt in {1, 2, 4},
 * unroll in {1, 2}), leaving `plan` prepared for the winning shape.  Both synchronise the stream, write
 * the outputs (as a normal call would) and allocate nothing on the device.
 */
typedef struct svd2_tune_result {
  int block, mpt, unroll, waves;
  float ms;
} svd2_tune_result;
int svd2_autotune_fwd(int op, int64_t n, const void *const *A, void *const *U, void *const *V,
                      void *smax, void *smin, int32_t *s, int reps, svd2_tune_result *best,
                      svd2_stream_t stream);
int svd2_multi_autotune(const svd2_batch_desc *descs, int32_t nbatch, void *plan,
                        size_t plan_bytes, int reps, svd2_tune_result *best,
                        svd2_stream_t stream);

/*
 * The forward forms (op 0 = d, 1 = z, 2 = s, 3 = c, 4 = svd2_batch_s_tan64 at
 * SVD2_TAN64_TAU_LOG2) on a batch held in HOST
 * memory: A, U, V are host arrays of host element pointers, smax, smin, s host
 * arrays, in the layout above.  When every array is page-locked host memory
 * (cudaHostAlloc, cudaMallocHost, cudaHostRegister; checked with
 * cudaPointerGetAttributes), the kernel reads and writes the arrays directly
 * across the host link and `chunk` is unused.  Otherwise the batch is cut into chunks of `chunk`
 * matrices (0 = 2^21; rounded up to a multiple of 64) that are copied to the
 * device, decomposed and copied back through a double-buffered three-stream
 * pipeline, so the copies in both directions overlap the kernels.  The call is
 * asynchronous on `stream`: the stream waits for the last chunk's outputs, and
 * the host arrays must stay valid (and unmodified) until then.  Host memory
 * should be pinned for the copies to overlap.  The device staging buffers
 * (two chunks of inputs and outputs) and the pipeline's streams are created by
 * the first call on a device and kept until the process exits; calls are
 * serialised within the process.  Errors as above.
 */
int svd2_batch_host(int op, int64_t n, const void *const *A, void *const *U, void *const *V,
                    void *smax, void *smin, int32_t *s, uint32_t flags, int64_t chunk,
                    svd2_stream_t stream);

/*
 * Launch shape of the forward kernels.  op: 0 = d, 1 = z, 2 = s, 3 = c,
 * 4 = svd2_batch_s_tan64 (the tangent-step kernel has its own shape; the
 * re-run forms use those of ops 2 and 3).  block: threads per block (a
 * multiple of 32, 32..1024; 32..512 for op 2, whose kernel may use up to 128
 * registers per thread); mpt: matrices per
 * thread per load (1, 2 or 4); unroll: load groups in flight per thread (1 or
 * 2); waves: resident-grid multiples (grid = waves x SMs x resident blocks per
 * SM, capped by the work; 0 = as many blocks as the work needs).  The setting
 * is process-wide and applies to later calls.  Returns SVD2_EINVAL for an
 * unsupported shape.
 */
int svd2_set_launch(int op, int block, int mpt, int unroll, int waves);
int svd2_get_launch(int op, int *block, int *mpt, int *unroll, int *waves);

/*
 * Self-test of the library's double arithmetic.  The FP64 forms compute their
 * divisions and square roots on the integer and FP32 pipes, exactly rounded
 * to nearest even (on GB300 the hardware IEEE double division and square root
 * take ~10 slots each of the narrow FP64 pipe).  For i < n this writes
 * lib[i] = the library's result and hw[i] = the hardware instruction's
 * (op 0: x[i] / y[i]; op 1: sqrt(x[i]); op 2: x[i] rounded to float, stored
 * widened exactly; op 3: the float whose bit pattern is the low 32 bits of
 * x[i], widened to double -- the conversions of the FP32 form's FP64 re-run;
 * op 4: x[i] and y[i] rounded to float, then the double quotient of the two
 * floats completed from their float quotient, as the tangent step of
 * svd2_batch_s_tan64 computes it, NaN where its operands are outside the
 * routine's domain; y unused for ops 1-3).  All pointers are device arrays of
 * n doubles.  The two must agree bit for bit (NaNs: any NaN).
 */
int svd2_arith_check(int op, int64_t n, const double *x, const double *y, double *lib,
                     double *hw, svd2_stream_t stream);

/*
 * Self-test of the single-precision branch-free reciprocal, square root and
 * division (Markstein's method) against the hardware's correctly rounded
 * sequences (__frcp_rn, __fsqrt_rn, __fdiv_rn), on indices k in
 * [begin, begin + count): op 0: the reciprocal of the float with bit pattern
 * k; op 1: the square root of the float with bit pattern k; op 2: a / b for a,
 * b in [1, 2) with significands k >> 23 and k & 0x7fffff (k < 2^46); op 3: a /
 * b for the two floats of a counter-based random 64-bit pattern of k, counted
 * only where b is in [2^-125, 2^125] and a is zero or |a| >= 2^-102 with
 * |a / b| in [2^-125, 2^127].  result: device memory of 3 uint64, which the caller initialises to
 * {0, UINT64_MAX, 0}: [0] gains the mismatches, [1] becomes the smallest
 * mismatching k, [2] gains the cases checked.  Asynchronous on `stream`.
 */
int svd2_fp32_selfcheck(int op, uint64_t begin, uint64_t count, void *result,
                        svd2_stream_t stream);

/* The cudaError_t of the last failed CUDA call made by this thread (0 if none). */
int svd2_last_cuda_error(void);

/* Library version string. */
const char *svd2_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SVD2_H */
