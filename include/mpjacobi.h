/*
 * mpjacobi.h -- C ABI of the GB300 (sm_103a) mixed precision preconditioned
 * Jacobi eigensolver / SVD of Zhang & Bai, "A mixed precision preconditioned
 * Jacobi method for the symmetric eigenvalue problem" (arXiv 2211.03339).
 *
 * Conventions shared by every entry point
 *   - All matrix and vector pointers are DEVICE pointers (cudaMalloc'd or
 *     managed memory visible to the current device), owned by the caller.
 *     The library never frees caller memory.  Inputs are never modified.
 *   - Matrices are column-major FP64 with the stated leading dimension
 *     (ld >= rows).
 *   - work/work_bytes: optional caller-provided device workspace of at least
 *     the size the matching *_workspace_bytes() returns; when work == NULL the
 *     library allocates (and frees) it with cudaMallocAsync on `stream`.
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued on that stream.  The sweep loops read one device
 *     scalar per sweep (the convergence test), so the call returns after the
 *     solve has finished on the GPU.
 *   - stats: optional (may be NULL), filled on return.
 *   - Return value: MPJ_SUCCESS or one of the status codes below.  On
 *     MPJ_NOT_CONVERGED the outputs hold the last iterate.  On any other
 *     error the outputs are unspecified.
 *   - Thread safety: calls on different streams may run concurrently; the
 *     last-error string is per thread.
 *
 * Notation: u = 2^-53 (the paper's omega), upsilon = 2^-24 (Sec. 6).
 */
#ifndef MPJACOBI_H
#define MPJACOBI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MPJ_SUCCESS = 0,
    MPJ_BAD_ARG = 1,          /* n < 1, m < n, ld < rows, NULL pointer, tol <= 0 ... */
    MPJ_NONFINITE_INPUT = 2,  /* A holds NaN or Inf                                   */
    MPJ_NOT_CONVERGED = 3,    /* max_sweeps reached; outputs hold the last iterate     */
    MPJ_RANK_DEFICIENT = 4,   /* SVD: a zero column norm (Alg. 5.2 assumes rank n);
                                 MGS: a zero r_jj                                      */
    MPJ_CUDA_ERROR = 5,       /* a CUDA runtime call failed; see mpj_last_error()      */
    MPJ_NO_DEVICE = 6         /* no sm_103 device visible                              */
};

/* Per-call statistics.  JU (rotations) is reported in units of
 * N = n(n-1)/2 as in the paper's tables (Sec. 6). */
typedef struct mpj_stats {
    int    sweeps;             /* SP: high precision sweeps executed              */
    int    sweeps_stage1;      /* sweeps of the single precision step 1           */
    double rotations;          /* JU of the high precision sweeps, in units of N  */
    double rotations_stage1;   /* JU of step 1, in units of N                     */
    double off_T0;             /* EVD: ||off(T)||_F when the FP64 sweeps start    */
    double off_final;          /* EVD: ||off(T)||_F at return                     */
    double norm_A;             /* ||A||_F                                         */
    float  ms_stage[4];        /* GPU ms of step 1, step 2 (MGS), step 3, sweeps  */
    int    block;              /* block size b of the block-pair solves           */
    int    status;             /* same as the return value                        */
} mpj_stats;

/* Optional tuning knobs; pass NULL for the defaults (zero fields also mean
 * "default").  The library reads no environment variables: every switch of its
 * numerical path is a field of this struct, in effect for the one call that
 * receives it. */
typedef struct mpj_options {
    int    max_sweeps;         /* FP64 sweeps cap (default 40)                     */
    int    max_sweeps_stage1;  /* FP32 sweeps cap (default 40)                     */
    int    max_inner;          /* inner sweeps of each 2b x 2b block solve (default 1) */
    double tol_stage1;         /* step-1 stop: ||off(T32)||_F <= tol_stage1 ||A32||_F
                                  (default 2^-21, eight FP32 ulps)                 */
    double ju_ratio;           /* one-sided stop: sweep applies < ju_ratio*N rotations
                                  (default 2e-4, Sec. 6)                           */
    int    block;              /* block size b: 16 or 32 (0 = choose by n)         */
    int    flags;              /* MPJ_OPT_* bits: alternative paths for comparisons
                                  and studies (0 = the default path)               */
    int    stage1_tf32_terms;  /* TF32 products per rotation tile of the FP32 stage
                                  (b = 32): 3 = hi*hi + hi*lo + lo*hi (default,
                                  about FP32 accuracy), 1 = hi*hi only (about
                                  2^-11, a lower-precision step 1 in the sense of
                                  Sec. 6, Figs. 6.2-6.3)                           */
} mpj_options;

/* mpj_options.flags */
#define MPJ_OPT_SIMT_STAGE1   1   /* FP32 stage on the SIMT engine (no tensor cores)      */
#define MPJ_OPT_SIMT_SWEEPS   2   /* FP64 sweeps on the SIMT engine (double-float / FP64
                                     tile products instead of the tensor cores)           */
#define MPJ_OPT_FP64_PRODUCTS 4   /* congruence, MGS panel projections and C = A Q as FP64
                                     GEMMs instead of exactly split tensor-core products  */
#define MPJ_OPT_FULL_INNER    8   /* tensor-core FP64 sweeps: full tournament inside each
                                     block solve instead of the cross-pair schedule       */
#define MPJ_OPT_MGS_GLOBAL   16   /* MGS panels from global memory instead of the shared
                                     memory of a thread-block cluster                     */
#define MPJ_OPT_TRACE        32   /* per-sweep rotation counts and off-norms on stderr    */
#define MPJ_OPT_FP64_SOLVES  64   /* one-sided tensor-core sweeps: block solves keep the
                                     Gram matrix in FP64 (default: FP32 off-diagonal,
                                     FP64 diagonal and rotations, where the range allows)  */

/* ------------------------------------------------------------------------
 * Symmetric eigendecomposition A = V diag(Lambda) V^T.
 *
 * mpj_syevj_mp  -- Algorithm 4.1 (Sec. 4):
 *   step 1  [Z, Phi] = eig(A) in single precision (upsilon): FP32 block Jacobi
 *           of fl32(A) (any backward stable solver satisfies Lemma 2.2);
 *   step 2  Q = MGS(Z) in double precision (Lemma 2.1; blocked MGS);
 *   step 3  T = Q^T A Q, P = Q in double precision;
 *   step 4  cyclic Jacobi sweeps in double precision (Lemma 3.1 rotations,
 *           parallel round-robin block order) while ||off(T)||_F > tol ||A||_F.
 * mpj_syevj_plain -- Algorithm 3.2 (Sec. 3.1): step 4 alone from T = A, P = I.
 *
 *   A       n x n symmetric (only read; both triangles must hold the matrix)
 *   n       order, n >= 1;  lda >= n
 *   Lambda  n eigenvalues, ascending
 *   V       n x n eigenvectors (columns, matching Lambda), ldv >= n
 *   tol     relative stopping tolerance (> 0), e.g. n * 2^-53
 *   opts    NULL or tuning knobs
 * ------------------------------------------------------------------------ */
int mpj_syevj_mp(const double* A, int n, int lda, double* Lambda, double* V, int ldv,
                 double tol, const mpj_options* opts, mpj_stats* stats,
                 void* work, size_t work_bytes, void* stream);
int mpj_syevj_plain(const double* A, int n, int lda, double* Lambda, double* V, int ldv,
                    double tol, const mpj_options* opts, mpj_stats* stats,
                    void* work, size_t work_bytes, void* stream);
size_t mpj_syevj_workspace_bytes(int n);

/* ------------------------------------------------------------------------
 * Singular value decomposition A = U diag(Sigma) V^T, m >= n, rank n.
 *
 * mpj_gesvj_mp  -- Algorithm 5.2 (Sec. 5):
 *   step 1  right singular vectors Z of fl32(A) by one-sided FP32 block Jacobi;
 *   step 2  Q = MGS(Z) in double precision;
 *   step 3  C = A Q, V = Q in double precision;
 *   steps 4-10  one-sided cyclic Jacobi sweeps (Lemma 5.1) in double precision;
 *   steps 11-13 columns ordered by decreasing ||c_j||, sigma_j = ||c_j||,
 *           u_j = c_j / sigma_j.
 * mpj_gesvj_plain -- Algorithm 5.1 from C = A, V = I, then steps 11-13.
 *
 *   A       m x n (lda >= m), m >= n >= 1
 *   Sigma   n singular values, descending
 *   U       m x n left singular vectors (ldu >= m)
 *   V       n x n right singular vectors (ldv >= n)
 *   tol     a pair (i,j) is rotated while |c_i^T c_j| > tol ||c_i|| ||c_j||
 *           (e.g. 8 * 2^-53); a sweep that applies fewer than ju_ratio * N
 *           rotations ends the iteration (Sec. 6).  Once a sweep applies fewer
 *           than N rotations the inner products are accumulated with Dot2
 *           (compensated), so the cosines are accurate to working precision.
 * ------------------------------------------------------------------------ */
int mpj_gesvj_mp(const double* A, int m, int n, int lda, double* Sigma, double* U, int ldu,
                 double* V, int ldv, double tol, const mpj_options* opts, mpj_stats* stats,
                 void* work, size_t work_bytes, void* stream);
int mpj_gesvj_plain(const double* A, int m, int n, int lda, double* Sigma, double* U, int ldu,
                    double* V, int ldv, double tol, const mpj_options* opts, mpj_stats* stats,
                    void* work, size_t work_bytes, void* stream);
size_t mpj_gesvj_workspace_bytes(int m, int n);

/* ------------------------------------------------------------------------
 * Batched eigendecompositions: many independent symmetric matrices, each
 * solved by Algorithm 4.1 (method 1) or Algorithm 3.2 (method 0), in one
 * persistent kernel launch (one CTA per matrix at a time, atomic work queue,
 * largest matrices first).  Sizes 1 <= n_i <= 256.
 *
 * Packed layouts (device, column-major, ld n_i): A_i and V_i start at offset
 * sum_{j<i} n_j^2, Lambda_i (ascending) at sum_{j<i} n_j.
 *
 * mpj_batch_plan_create: ns is a HOST array of the count sizes.  Allocates the
 *   job list and one scratch slot per resident CTA (about 2.7 MB each; see
 *   mpj_batch_plan_info) on the current device; synchronous.
 * mpj_syevj_batched: enqueues one memset and one kernel on `stream`, performs
 *   no host synchronisation and no allocation (it may be captured in a CUDA
 *   graph).  tol: relative tolerance of every matrix (<= 0: n_i * 2^-53).
 *   status (optional, device, count ints): per-matrix MPJ_* code.
 *   sweeps (optional, device, count ints): FP64 sweeps + 1000 * FP32 sweeps.
 *   Runs of one plan must not overlap (they share the scratch and counter).
 * ------------------------------------------------------------------------ */
typedef struct mpj_batch_plan_s mpj_batch_plan;
typedef struct mpj_batch_tuning {
    int ctas_per_sm;        /* 1 or 2 (default 2)                               */
    int max_inner;          /* inner sweeps per block solve for n > 2b (def. 1)  */
    int block_large;        /* block size b for n > 64: 16 or 32 (default 32)    */
    int max_sweeps;         /* FP64 sweeps cap (default 40)                      */
    int max_sweeps_stage1;  /* FP32 sweeps cap (default 40)                      */
} mpj_batch_tuning;
int mpj_batch_plan_create(const int* ns, int count, int method, const mpj_batch_tuning* tuning,
                          mpj_batch_plan** plan);
int mpj_batch_plan_info(const mpj_batch_plan* plan, long long* a_elems, long long* lambda_elems,
                        int* ctas, size_t* scratch_bytes);
int mpj_syevj_batched(mpj_batch_plan* plan, const double* A, double* Lambda, double* V, double tol,
                      int* status, int* sweeps, void* stream);
void mpj_batch_plan_destroy(mpj_batch_plan* plan);

/* ------------------------------------------------------------------------
 * Reverse-mode derivative of A = V diag(Lambda) V^T for a batch of `batch`
 * symmetric n x n matrices (no counterpart in the paper; it lets training code
 * differentiate through the solver):
 *   A_bar = V (diag(Lambda_bar) + sym(F o (V^T V_bar))) V^T,
 *   F_ij = 1/(lambda_j - lambda_i) (i != j; a zero gap contributes 0),
 *   sym(X) = (X + X^T)/2; A_bar is exactly symmetric.
 * Layouts (device): Lambda, gLambda: batch x n; V, gV, gA: batch x (n x n)
 * column-major, ld n, contiguous.  gLambda or gV may be NULL (zero).  The
 * derivative is well defined only for distinct eigenvalues.
 * ------------------------------------------------------------------------ */
int mpj_syev_backward_batched(const double* Lambda, const double* V, const double* gLambda,
                              const double* gV, int n, int batch, double* gA,
                              void* work, size_t work_bytes, void* stream);
size_t mpj_syev_backward_workspace_bytes(int n, int batch);

/* ------------------------------------------------------------------------
 * Single steps of the pipeline, exposed for stage-wise checks.
 * ------------------------------------------------------------------------ */

/* Step 1 of Alg. 4.1: FP32 block Jacobi of fl32(A).  Z (n x n, ldz) receives the
 * eigenvectors widened exactly to FP64, ordered by ascending eigenvalue; D (n)
 * the FP32 eigenvalues widened to FP64. */
int mpj_stage1_syevj32(const double* A, int n, int lda, double* Z, int ldz, double* D,
                       const mpj_options* opts, mpj_stats* stats,
                       void* work, size_t work_bytes, void* stream);

/* Lemma 2.1 / step 2 of Alg. 4.1: modified Gram-Schmidt Z = Q R (m x n, m >= n) in
 * FP64, blocked: each 32-column panel is orthogonalised column by column (MGS)
 * by one thread-block cluster, then the trailing columns are projected against
 * the panel (two FP64 GEMMs).  For n >= 1024 the columns are first grouped in
 * 256-column panels, orthogonalised in order; the projections between those
 * panels are FP64 products on the tensor cores by exact splitting (error of the
 * order of an FP64 dot product's rounding).  R is not formed.  Returns
 * MPJ_RANK_DEFICIENT if some r_jj == 0. */
int mpj_mgs(const double* Z, int m, int n, int ldz, double* Q, int ldq,
            void* work, size_t work_bytes, void* stream);
size_t mpj_mgs_workspace_bytes(int m, int n);

/* mpj_mgs_noalloc -- the blocked MGS of mpj_mgs, with 32-column panels at every
 * size (the tensor-core projections between 256-column panels need scratch of
 * their own), for callers that cannot allocate device memory at call time:
 * for instance code running where an allocation could block on a device-wide
 * synchronisation or fail under memory pressure (a latency-critical loop), or
 * applications whose own memory manager owns all device memory and does not
 * allow allocations from libraries.  The paper has no counterpart.
 *   Z, m, n, ldz, Q, ldq, stream: as for mpj_mgs.  Nothing is allocated and
 *   nothing is freed (no cudaMalloc, cudaFree or allocating library routine).
 *   Scratch: a fixed device array of MPJ_MGS_NOALLOC_MAX_SCRATCH_DOUBLES
 *   doubles (8 MiB) compiled into the library.  A call needs
 *   32 * n * (1 + ceil(m / 256)) doubles of it (a square Z fits up to
 *   n = 2730); larger sizes are rejected with MPJ_BAD_ARG before any device
 *   work.
 *   The array is reserved on a GPU when the library's module is loaded there,
 *   which with CUDA's lazy module loading happens at the first call of the
 *   library on that GPU, and stays reserved until the process exits.  Make a
 *   first call (of this or any other entry point) in set-up code, before any
 *   stream capture, so that the reservation cannot fail later for lack of
 *   memory.  Each call looks up the array's address in the CUDA context that
 *   is current (a host-side query that allocates nothing).
 *   All calls share the one array, which keeps the previous call's contents:
 *   calls that may overlap on the GPU (different streams, or several host
 *   threads) race on it and must be serialised by the caller.
 *   Returns MPJ_RANK_DEFICIENT if some r_jj == 0; the call synchronises the
 *   stream (it reads that flag). */
#define MPJ_MGS_NOALLOC_MAX_SCRATCH_DOUBLES (1u << 20)
int mpj_mgs_noalloc(const double* Z, int m, int n, int ldz, double* Q, int ldq, void* stream);

/* Step 3 of Alg. 4.1: T = Q^T (A Q) in FP64 (A n x n symmetric, Q n x n).  The
 * upper triangle is computed and mirrored, so T is exactly symmetric.  Both
 * products run on the bf16 tensor cores by exact splitting (8 slices of 7 bits
 * per row of op(A) / column of op(B), power-of-two scaled); the error stays
 * within the bound of an FP64 product, |T - Q^T A Q| <= 2 gamma_n (2 + gamma_n)
 * |Q|^T |A| |Q| elementwise (Sec. 4).  n > 32768 uses FP64 GEMMs. */
int mpj_congruence(const double* A, int lda, const double* Q, int ldq, int n,
                   double* T, int ldt, void* work, size_t work_bytes, void* stream);
size_t mpj_congruence_workspace_bytes(int n);

/* Step 4 of Alg. 4.1 / Alg. 3.2 on a given symmetric T and start P (both n x n,
 * ld >= n): FP64 block-Jacobi sweeps in place while ||off(T)||_F > tol * normA.
 * T is overwritten by the final iterate (not sorted); P by P * prod(J). */
int mpj_sweeps(double* T, int ldt, double* P, int ldp, int n, double tol, double normA,
               const mpj_options* opts, mpj_stats* stats,
               void* work, size_t work_bytes, void* stream);
size_t mpj_sweeps_workspace_bytes(int n);

/* ------------------------------------------------------------------------
 * Diagnostics (no counterpart in the paper): every kernel launch of the
 * library is counted per kernel class; when profiling is enabled each launch
 * is also bracketed by CUDA events recorded on its own stream, and the
 * elapsed times are summed whenever the library synchronises.
 * ------------------------------------------------------------------------ */
void mpj_profile_enable(int on);
void mpj_profile_reset(void);
/* launches and summed event time (ms) of class kclass (0 <= kclass < classes) */
int mpj_profile_read(int kclass, long long* launches, double* total_ms);
/* Algorithmic bytes that the library itself counted for the launches of class
 * kclass since the last reset (0 for classes that count none): the one-pass
 * tile update of the FP32 step counts 3 x 64 x 64 x 4 bytes per off-diagonal
 * tile it updates (read once, written with its mirror); tiles whose two block
 * rotations are the identity are skipped and not counted. */
int mpj_profile_units(int kclass, double* bytes);
const char* mpj_profile_name(int kclass);
int mpj_profile_classes(void);
unsigned long long mpj_kernel_launches(void);   /* all classes, since load */

/* ------------------------------------------------------------------------ */
const char* mpj_status_string(int status);
const char* mpj_last_error(void);      /* last CUDA error text of this thread */
const char* mpj_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MPJACOBI_H */
