// internal.h -- host-side declarations shared by the translation units of
// libmpjacobi.so.  Not part of the public ABI (see include/mpjacobi.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstddef>
#include <cstdint>

#include "../../include/mpjacobi.h"

namespace mpj {

// ---------------------------------------------------------------- errors
void set_error(const char* where, cudaError_t e);
void set_error_msg(const char* msg);

#define MPJ_CUDA_TRY(expr)                                                    \
    do {                                                                      \
        cudaError_t _e = (expr);                                              \
        if (_e != cudaSuccess) { ::mpj::set_error(#expr, _e); return MPJ_CUDA_ERROR; } \
    } while (0)

#define MPJ_LAUNCH_CHECK(name)                                                \
    do {                                                                      \
        cudaError_t _e = cudaGetLastError();                                  \
        if (_e != cudaSuccess) { ::mpj::set_error(name, _e); return MPJ_CUDA_ERROR; } \
    } while (0)

#define MPJ_TRY(expr)                                                         \
    do { int _s = (expr); if (_s != MPJ_SUCCESS) return _s; } while (0)

// ---------------------------------------------------------------- workspace
// A bump allocator over one device buffer; every carve is 256-byte aligned.
struct Arena {
    char*  base = nullptr;
    size_t size = 0;
    size_t used = 0;
    template <class T>
    T* take(size_t count) {
        size_t off = (used + 255) & ~size_t(255);
        size_t bytes = count * sizeof(T);
        if (base == nullptr) { used = off + bytes; return nullptr; }   // sizing pass
        if (off + bytes > size) return nullptr;
        used = off + bytes;
        return reinterpret_cast<T*>(base + off);
    }
};

// Owns a workspace: either the caller's buffer or a stream-ordered allocation.
struct Workspace {
    void*        ptr = nullptr;
    bool         owned = false;
    cudaStream_t stream = nullptr;
    int acquire(void* caller, size_t caller_bytes, size_t need, cudaStream_t s);
    ~Workspace();
};

// Pinned host scratch for the per-sweep convergence read-back.
struct HostScratch {
    double*             d = nullptr;
    unsigned long long* u = nullptr;
    int init();
    ~HostScratch();
};

// A second stream for the V updates of the sweep engines.  Round g uses buffer
// set g & 1; the V update of round g runs on sv after the solve of round g
// (event `solved`), and the solve of round g + 2 -- which rewrites that set --
// waits for it (event `vdone`).  The destructor makes the main stream wait for
// every V update (and the main stream) before anything later on it reads V.
// The sweeps themselves run on `main`, a high-priority stream ordered after the
// caller's stream, and the V updates on the low-priority `sv`, so that SM slots
// freed by V tiles go to the next block solve (the critical path) first.
struct SideStream {
    cudaStream_t caller = nullptr, main = nullptr, sv = nullptr;
    cudaEvent_t solved[2] = {nullptr, nullptr}, vdone[2] = {nullptr, nullptr};
    cudaEvent_t start = nullptr, fin = nullptr;
    bool pending[2] = {false, false};
    int g = 0;
    int init(cudaStream_t s);
    int begin_round();          // returns the buffer set of this round, -1 on error
    int after_solve();          // V stream waits for this round's solve
    int after_v();              // marks this round's V update
    void end_round() { ++g; }
    ~SideStream();
};

// ---------------------------------------------------------------- per-call switches
// The path switches of mpj_options (flags, stage1_tf32_terms) for the call in
// progress on this thread: KnobScope sets them at the entry of a C-ABI call and
// restores the previous ones on return; without a scope they are the defaults.
struct Knobs {
    bool simt_stage1 = false;   // FP32 stage on the SIMT engine
    bool simt_sweeps = false;   // FP64 sweeps on the SIMT engine
    bool fp64_products = false; // FP64-pipe GEMMs instead of exactly split products
    bool full_inner = false;    // tensor-core FP64 sweeps: full inner tournament
    bool mgs_global = false;    // MGS panels from global memory
    bool trace = false;         // per-sweep trace on stderr
    bool fp64_solves = false;   // one-sided tensor-core solves: S kept in FP64
    int stage1_terms = 3;       // TF32 products per tile of the FP32 stage: 3 or 1
};
const Knobs& knobs();
struct KnobScope {
    Knobs saved;
    explicit KnobScope(const mpj_options* o);
    ~KnobScope();
};

// ---------------------------------------------------------------- profiling
// Kernel classes counted (and, when enabled, timed with CUDA events on the
// launching stream) by ProfScope; names in prof.cu.
enum ProfClass {
    PC_SOLVE2_F32 = 0, PC_APPLY2_F32, PC_SOLVE2_F64, PC_APPLY2_F64, PC_DGEMM, PC_MGS_PANEL,
    PC_MGS_PROJ, PC_GRAM1_F32, PC_SOLVE1_F32, PC_APPLY1_F32, PC_GRAM1_F64, PC_SOLVE1_F64,
    PC_APPLY1_F64, PC_AUX, PC_APPLY2V_F32, PC_APPLY2V_F64, PC_BATCHED, PC_TC1_F32, PC_TC2_F32,
    PC_OZ_SLICE, PC_OZ_GEMM, PC_TCV_F32, PC_TCP1_F64, PC_TCP2_F64, PC_TCV_F64, PC_GRAM_TC64,
    PC_TCC_F64, PC_TCV1_F64, PC_TILE_F32, kProfClasses
};
struct ProfScope {
    int cls;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    ProfScope(int cls, cudaStream_t s);
    ~ProfScope();
};
void prof_flush();
// Add algorithmic bytes to a class's work count (mpj_profile_units).
void prof_add_units(int cls, double bytes);
// Per-sweep trace on stderr (rotation counts, off-norms): MPJ_OPT_TRACE.
inline bool trace_on() { return knobs().trace; }
#define MPJ_PROF(cls, stream) ::mpj::ProfScope _mpj_prof_scope((cls), (stream))

// ---------------------------------------------------------------- shapes
inline int round_up(int x, int m) { return (x + m - 1) / m * m; }
int choose_block(int n, const mpj_options* o);

// ---------------------------------------------------------------- engines
// Two-sided block Jacobi (Alg. 3.2 / step 4 of Alg. 4.1, parallel round-robin
// block order) on a padded N x N symmetric matrix T (ld = N) and V (ld = N).
struct SweepResult {
    int    sweeps = 0;
    double rotations = 0;       // applied (non-skipped) rotations, absolute count
    double off_initial = 0;
    double off_final = 0;
    int    status = MPJ_SUCCESS;
};

template <class Real>
size_t twosided_workspace_bytes(int N, int B);
template <class Real>
int twosided_sweeps(Real* T, Real* V, int N, int n, int B, double tol_abs, double eps_skip,
                    int max_sweeps, int max_inner, void* work, cudaStream_t s, SweepResult* res);

// The FP32 engine of step 1 with the rotations applied on the tensor cores
// (tc_apply.cu): block size b = 32 (N a multiple of 64), T column-major N x N
// and symmetric, Vt = V^T column-major (V row-major).
size_t tc32_workspace_bytes(int N);
int twosided_sweeps_tc32(float* T, float* Vt, int N, int n, double tol_abs, double eps_skip, int max_sweeps,
                         int max_inner, void* work, cudaStream_t s, SweepResult* res);
// The FP64 engine with the rotations applied on the tensor cores by exact
// splitting (tc64_apply.cu): block size b = 32, T and V column-major N x N.
// The workspace holds the block rotations, their digit planes and the N x N
// scratch P of pass 1.  cross selects the cross-pair inner schedule.
size_t tc64_workspace_bytes(int N);
bool tc64_supported(int N, int B);
int twosided_sweeps_tc64(double* T, double* V, int N, int n, double tol_abs, double eps_skip, int max_sweeps,
                         int max_inner, int cross, void* work, cudaStream_t s, SweepResult* res);
// One-sided FP64 sweeps with the block Grams and rotations on the tensor cores
// (tc64_onesided.cu): b = 32, N a multiple of 64, m even, 128 <= m < 2^20.
bool onesided_tc64_supported(int m, int N, int B);
size_t onesided_tc64_workspace_bytes(int m, int N);
int onesided_sweeps_tc64(double* C, double* V, int m, int N, int n, double tol_rot, double ju_ratio,
                         int max_sweeps, int max_inner, void* work, cudaStream_t s, SweepResult* res);
// One-sided FP32 sweeps (step 1 of Alg. 5.2) with the block Grams and rotations
// on the TF32 tensor cores (tc_apply.cu): C (m x N) and V (N x N) row-major,
// b = 32, N a multiple of 64, m >= 128.  The block solves are the SIMT FP32
// solves of onesided.cu (solve1_f32_round).
bool onesided_tc32_supported(int m, int N, int B);
size_t onesided_tc32_workspace_bytes(int m, int N);
int onesided_sweeps_tc32(float* C, float* V, int m, int N, int n, double tol_rot, double ju_ratio,
                         int max_sweeps, int max_inner, void* work, cudaStream_t s, SweepResult* res);
int configure_solve1_f32();
int solve1_f32_round(const float* Ghi, const float* Glo, int nsplit, int K, float* Wbuf, double tol_rot,
                     int max_inner, int cross_round, unsigned long long* rot, cudaStream_t s);
// Row-major FP32 copy of A (m x n, padded with zero columns to N) and the squared
// column norms of a row-major C.
int copy_rowmajor_f32(const double* A, int lda, int m, int n, float* C, int N, cudaStream_t s);
int colnorms2_rowmajor_f32(const float* C, int m, int N, int n, double* nrm2, cudaStream_t s);
// Z[:, c] = V[:, perm[c]] (widened) from a row-major V.
int gather_z32_rowmajor(const float* Vt, int ld, const int* perm, int n, double* Z, int ldz,
                        cudaStream_t s);
// Inner schedule of the block solves (1: cross pairs, see inner_jacobi) of the
// FP32 stage, the SIMT FP64 engine and the tensor-core FP64 engine.
int cross_schedule(bool fp64, bool tc64);

// One-sided block Jacobi (Alg. 5.1 / steps 4-10 of Alg. 5.2) on C (m x N, ld = ldc)
// and V (N x N, ld = N).
template <class Real>
size_t onesided_workspace_bytes(int m, int N, int B);
template <class Real>
int onesided_sweeps(Real* C, int ldc, Real* V, int m, int N, int n, int B, double tol_rot,
                    double ju_ratio, int max_sweeps, int max_inner, void* work, cudaStream_t s,
                    SweepResult* res);

// FP64 GEMM: C = alpha * op(A) * op(B) + beta * C (column-major).  When
// upper_mirror is set, only tiles on or above the diagonal of the (square) C
// are computed and each result is also written to the mirrored position.
int dgemm(bool transA, bool transB, int M, int N, int K, double alpha, const double* A, int lda,
          const double* B, int ldb, double beta, double* C, int ldc, bool upper_mirror,
          cudaStream_t s);

int dgemm_batched(bool transA, bool transB, int M, int N, int K, double alpha, const double* A,
                  int lda, long long sA, const double* B, int ldb, long long sB, double beta,
                  double* C, int ldc, long long sC, int batch, bool upper_mirror, cudaStream_t s);

// FP64 products on the bf16 tensor cores by exact splitting (ozaki.cu).  An
// operand holds the 8 bf16 slice planes of `rows` rows of length K (row i of
// op(A), or column j of op(B)) and the binary exponent of each row.
struct OzOperand {
    __nv_bfloat16* planes;
    int* ex;
    int rows, K;
};
size_t oz_operand_bytes(int rows, int K);
int oz_operand(void* base, int rows, int K, OzOperand* op);
bool oz_supported(int M, int N, int K);
// Exactly split products unless MPJ_OPT_FP64_PRODUCTS keeps them on the FP64 pipe.
inline bool oz_enabled() { return !knobs().fp64_products; }
// Slice rows: row r is X[r * row_stride + k * k_stride], k < K (k_stride 1 or the
// rows of a column-major matrix, row_stride 1).
int oz_slice(const double* X, long long row_stride, long long k_stride, int rows, int K, OzOperand* op,
             cudaStream_t s);
// C (ld ldc) = alpha * A B^T-of-the-operands + beta C: C_ij = alpha sum_k opA(i,k) opB(k,j)
// + beta C_ij with A holding the rows of op(A) and B the columns of op(B).  With
// upper_mirror (square C) the upper triangle is mirrored onto the lower.  A
// timed-out tensor-core wait sets bit 2 of *d_flag.
int oz_gemm(const OzOperand& A, const OzOperand& B, double alpha, double beta, double* C, int ldc,
            bool upper_mirror, int* d_flag, cudaStream_t s);

// Blocked MGS (Lemma 2.1) in place on Q (m x n, ld = ldq).  Needs n x 32 doubles
// of workspace for the panel projections.
size_t mgs_workspace_bytes(int m, int n);
int mgs_inplace(double* Q, int m, int n, int ldq, void* work, int* d_flag, cudaStream_t s);
// The same with 256-column panels whose mutual projections run on the tensor
// cores (mgs.cu); ozW: oz_operand_bytes(n, m), ozS: mgs_panel_oz_bytes(m, n),
// Rbuf: 256 x n doubles.
size_t mgs_panel_oz_bytes(int m, int n);
int mgs_blocked_oz(double* Q, int m, int n, int ldq, void* work, int* d_flag, void* ozW, void* ozS,
                   double* Rbuf, cudaStream_t s);

// ---------------------------------------------------------------- helpers (kernels.cu)
int copy_pad_f64(const double* A, int lda, int rows, int cols, double* T, int ldt, int Rpad,
                 int Cpad, bool identity_pad, cudaStream_t s);
int copy_pad_f32(const double* A, int lda, int rows, int cols, float* T, int ldt, int Rpad,
                 int Cpad, bool identity_pad, cudaStream_t s);
int scale_pow2_f64(double* A, int ld, int rows, int cols, int e, cudaStream_t s);
int set_identity_f64(double* V, int ld, int rows, int cols, cudaStream_t s);
int set_identity_f32(float* V, int ld, int rows, int cols, cudaStream_t s);
int copy_f64(const double* src, int lds, int rows, int cols, double* dst, int ldd, cudaStream_t s);
int sumsq_f64(const double* A, int lda, int rows, int cols, double* partial, double* out,
              cudaStream_t s);
int offnorm2(const void* T, bool is_double, int ld, int n, double* partial, double* out,
             cudaStream_t s);
// ranks of keys (ascending or descending), ties broken by index; perm[rank] = i
int rank_sort(const double* keys, int stride, int n, bool descending, int* perm, cudaStream_t s);
int gather_vec(const double* in, const int* perm, int n, double* out, cudaStream_t s);
int diag_to_f64(const void* T, bool is_double, int ld, int n, double* d, cudaStream_t s);
int gather_eig(const double* T, int ldt, const double* Vw, int ldvw, const int* perm, int n,
               double* Lambda, double* V, int ldv, cudaStream_t s);
int gather_z32(const float* V32, int ld32, const int* perm, int n, double* Z, int ldz,
               cudaStream_t s);
int colnorms_f64(const double* C, int ldc, int m, int n, double* nrm, cudaStream_t s);
int colnorms2_f32(const float* C, int ldc, int m, int n, double* nrm2, cudaStream_t s);
int svd_post(const double* C, int ldc, const double* Vw, int ldvw, const double* nrm,
             const int* perm, int m, int n, double* Sigma, double* U, int ldu, double* V,
             int ldv, int* d_flag, cudaStream_t s);

}  // namespace mpj
