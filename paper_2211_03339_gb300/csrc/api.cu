// api.cu -- the C ABI (include/mpjacobi.h): argument checks, workspace layout
// and the order of the steps of Algorithms 3.2, 4.1, 5.1 and 5.2.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace mpj {
const char* last_error();
}

using namespace mpj;

namespace {

constexpr double kU = 1.1102230246251565e-16;    // 2^-53
constexpr double kUps = 5.9604644775390625e-08;  // 2^-24

struct Opts {
    int max_sweeps = 40, max_sweeps1 = 40, max_inner = 1, block = 0;
    double tol1 = 8 * kUps, ju_ratio = 2e-4;      // step-1 stop: 8 ulps of FP32 (see mpjacobi.h)
};

Opts read_opts(const mpj_options* o) {
    Opts r;
    if (o) {
        if (o->max_sweeps > 0) r.max_sweeps = o->max_sweeps;
        if (o->max_sweeps_stage1 > 0) r.max_sweeps1 = o->max_sweeps_stage1;
        if (o->max_inner > 0) r.max_inner = o->max_inner;
        if (o->tol_stage1 > 0) r.tol1 = o->tol_stage1;
        if (o->ju_ratio >= 0 && o->ju_ratio == o->ju_ratio && o->ju_ratio != 0) r.ju_ratio = o->ju_ratio;
        r.block = o->block;
    }
    return r;
}

int padded(int n, int B) {
    int M = 2 * B;
    int N = round_up(n, M);
    return N < M ? M : N;
}

// Stage timing with events on the caller's stream.
struct Timer {
    cudaEvent_t ev[6] = {};
    bool on = false;
    cudaStream_t s = nullptr;
    int init(bool enable, cudaStream_t st) {
        on = enable; s = st;
        if (!on) return MPJ_SUCCESS;
        for (auto& e : ev) MPJ_CUDA_TRY(cudaEventCreate(&e));
        return MPJ_SUCCESS;
    }
    void mark(int i) { if (on) cudaEventRecord(ev[i], s); }
    float ms(int a, int b) {
        if (!on) return 0.f;
        float t = 0.f;
        cudaEventSynchronize(ev[b]);
        cudaEventElapsedTime(&t, ev[a], ev[b]);
        return t;
    }
    ~Timer() { if (on) for (auto& e : ev) if (e) cudaEventDestroy(e); }
};

struct Scal {           // small device scratch shared by the drivers
    double* partial;    // 1024
    double* val;        // 8
    int* flag;          // 4
    int* perm;          // n
    double* d;          // n
};

int take_scal(Arena& a, int n, Scal& sc) {
    sc.partial = a.take<double>(1024);
    sc.val = a.take<double>(8);
    sc.flag = a.take<int>(4);
    sc.perm = a.take<int>((size_t)(n > 0 ? n : 1));
    sc.d = a.take<double>((size_t)(n > 0 ? n : 1));
    return (a.base && (!sc.partial || !sc.val || !sc.flag || !sc.perm || !sc.d)) ? MPJ_BAD_ARG : MPJ_SUCCESS;
}

int read_scalar(const double* dval, double* out, cudaStream_t s) {
    double h = 0;
    MPJ_CUDA_TRY(cudaMemcpyAsync(&h, dval, sizeof(double), cudaMemcpyDeviceToHost, s));
    MPJ_CUDA_TRY(cudaStreamSynchronize(s));
    *out = h;
    return MPJ_SUCCESS;
}

// Status flag of a driver: bit 1 rank deficiency (a zero column), bit 2 a
// tensor-core wait that timed out (reported as a CUDA error).
int read_flag(const int* dflag, int* out, cudaStream_t s) {
    int h = 0;
    MPJ_CUDA_TRY(cudaMemcpyAsync(&h, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    MPJ_CUDA_TRY(cudaStreamSynchronize(s));
    if (h & 2) { set_error_msg("tensor-core product: MMA or TMA wait timed out"); return MPJ_CUDA_ERROR; }
    *out = h & 1;
    return MPJ_SUCCESS;
}

// T = Q^T (A Q) with the upper triangle mirrored (T exactly symmetric), A
// symmetric; W (n x n) is scratch.  With the two operand buffers (oz_operand_bytes
// (n, n) each) both products run on the tensor cores by exact splitting
// (ozaki.cu); the slices of Q serve as the columns of Q in A Q and as the rows
// of Q^T in Q^T W.
int congruence_fp64(const double* A, int lda, const double* Q, int ldq, int n, double* W, double* T,
                    int ldt, void* oz1, void* oz2, int* d_flag, cudaStream_t s) {
    if (oz1 && oz2 && oz_enabled() && oz_supported(n, n, n)) {
        OzOperand oa, oq;
        MPJ_TRY(oz_operand(oz1, n, n, &oa));
        MPJ_TRY(oz_operand(oz2, n, n, &oq));
        MPJ_TRY(oz_slice(A, lda, 1, n, n, &oa, s));        // rows of A (= its columns)
        MPJ_TRY(oz_slice(Q, ldq, 1, n, n, &oq, s));        // columns of Q
        MPJ_TRY(oz_gemm(oa, oq, 1.0, 0.0, W, n, false, d_flag, s));
        MPJ_TRY(oz_slice(W, n, 1, n, n, &oa, s));          // columns of W
        MPJ_TRY(oz_gemm(oq, oa, 1.0, 0.0, T, ldt, true, d_flag, s));
        return MPJ_SUCCESS;
    }
    MPJ_TRY(dgemm(false, false, n, n, n, 1.0, A, lda, Q, ldq, 0.0, W, n, false, s));
    MPJ_TRY(dgemm(true, false, n, n, n, 1.0, Q, ldq, W, n, 0.0, T, ldt, true, s));
    return MPJ_SUCCESS;
}

int frob_norm(const double* A, int lda, int m, int n, const Scal& sc, double* out, cudaStream_t s) {
    MPJ_TRY(sumsq_f64(A, lda, m, n, sc.partial, sc.val, s));
    double ss;
    MPJ_TRY(read_scalar(sc.val, &ss, s));
    *out = sqrt(ss);
    return MPJ_SUCCESS;
}

size_t max2(size_t a, size_t b) { return a > b ? a : b; }

// ------------------------------------------------------------------ EVD layout
struct EvdBufs {
    double *T64, *V64, *Q, *Wt;
    float *T32, *V32;
    void* eng;
    void* mgsw;
    void *oz1, *oz2, *ozs;       // tensor-core operand slices (mp only)
    Scal sc;
};

size_t evd_engine_bytes(int N, int B) {
    size_t e = max2(twosided_workspace_bytes<double>(N, B), twosided_workspace_bytes<float>(N, B));
    return B == 32 ? max2(e, tc32_workspace_bytes(N)) : e;
}

int evd_layout(Arena& a, int n, int N, int B, bool mp, EvdBufs& b) {
    size_t NN = (size_t)N * N, nn = (size_t)n * n;
    b.T64 = a.take<double>(NN);
    b.V64 = a.take<double>(NN);
    b.Q = mp ? a.take<double>(nn) : nullptr;
    b.Wt = mp ? a.take<double>(nn) : nullptr;
    b.T32 = mp ? a.take<float>(NN) : nullptr;
    b.V32 = mp ? a.take<float>(NN) : nullptr;
    b.eng = a.take<char>(evd_engine_bytes(N, B));
    b.mgsw = mp ? a.take<char>(mgs_workspace_bytes(n, n)) : nullptr;
    b.oz1 = mp ? a.take<char>(oz_operand_bytes(n, n)) : nullptr;
    b.oz2 = mp ? a.take<char>(oz_operand_bytes(n, n)) : nullptr;
    b.ozs = mp ? a.take<char>(mgs_panel_oz_bytes(n, n)) : nullptr;
    MPJ_TRY(take_scal(a, n, b.sc));
    if (a.base && (!b.T64 || !b.V64 || !b.eng ||
                   (mp && (!b.Q || !b.Wt || !b.T32 || !b.V32 || !b.mgsw || !b.oz1 || !b.oz2 || !b.ozs))))
        return MPJ_BAD_ARG;
    return MPJ_SUCCESS;
}

size_t evd_bytes(int n, bool mp, const mpj_options* o) {
    int B = choose_block(n, o);
    int N = padded(n, B);
    Arena a;
    EvdBufs b;
    evd_layout(a, n, N, B, mp, b);
    return a.used + 512;
}

// FP32 step 1 of Alg. 4.1 into bufs (Z -> b.Q, ascending D -> b.sc.d).
int stage1_evd(const double* A, int lda, int n, int N, int B, double normA, const Opts& op,
               EvdBufs& b, SweepResult* r1, cudaStream_t s) {
    MPJ_TRY(copy_pad_f32(A, lda, n, n, b.T32, N, N, N, false, s));
    MPJ_TRY(set_identity_f32(b.V32, N, N, N, s));
    const bool tc = B == 32 && !knobs().simt_stage1;
    if (tc) {
        // tensor-core engine: V32 holds V row-major
        MPJ_TRY(twosided_sweeps_tc32(b.T32, b.V32, N, n, op.tol1 * normA, kUps, op.max_sweeps1, op.max_inner,
                                     b.eng, s, r1));
    } else {
        MPJ_TRY(twosided_sweeps<float>(b.T32, b.V32, N, n, B, op.tol1 * normA, kUps, op.max_sweeps1,
                                       op.max_inner, b.eng, s, r1));
    }
    MPJ_TRY(diag_to_f64(b.T32, false, N, n, b.sc.d, s));
    MPJ_TRY(rank_sort(b.sc.d, 1, n, false, b.sc.perm, s));
    if (tc) {
        MPJ_TRY(gather_z32_rowmajor(b.V32, N, b.sc.perm, n, b.Q, n, s));
    } else {
        MPJ_TRY(gather_z32(b.V32, N, b.sc.perm, n, b.Q, n, s));
    }
    return MPJ_SUCCESS;
}

int check_evd_args(const double* A, int n, int lda, const void* L, const void* V, int ldv,
                   double tol) {
    if (!A || !L || !V || n < 1 || lda < n || ldv < n || !(tol > 0) || !std::isfinite(tol)) {
        set_error_msg("invalid argument");
        return MPJ_BAD_ARG;
    }
    return MPJ_SUCCESS;
}

int syevj_impl(bool mp, const double* A, int n, int lda, double* Lambda, double* V, int ldv,
               double tol, const mpj_options* opts, mpj_stats* st, void* work, size_t work_bytes,
               void* stream) {
    KnobScope knob_scope(opts);
    if (st) memset(st, 0, sizeof(*st));
    MPJ_TRY(check_evd_args(A, n, lda, Lambda, V, ldv, tol));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Opts op = read_opts(opts);
    const int B = choose_block(n, opts);
    const int N = padded(n, B);
    Workspace ws;
    MPJ_TRY(ws.acquire(work, work_bytes, evd_bytes(n, mp, opts), s));
    Arena a;
    a.base = static_cast<char*>(ws.ptr);
    a.size = work ? work_bytes : evd_bytes(n, mp, opts);
    EvdBufs b;
    if (evd_layout(a, n, N, B, mp, b) != MPJ_SUCCESS) { set_error_msg("workspace layout"); return MPJ_BAD_ARG; }
    Timer tm;
    MPJ_TRY(tm.init(st != nullptr, s));
    tm.mark(0);
    double normA;
    MPJ_TRY(frob_norm(A, lda, n, n, b.sc, &normA, s));
    if (st) { st->norm_A = normA; st->block = B; }
    if (!std::isfinite(normA)) { if (st) st->status = MPJ_NONFINITE_INPUT; return MPJ_NONFINITE_INPUT; }

    SweepResult r1, r2;
    if (mp) {
        MPJ_TRY(stage1_evd(A, lda, n, N, B, normA, op, b, &r1, s));                       // step 1
        tm.mark(1);
        MPJ_CUDA_TRY(cudaMemsetAsync(b.sc.flag, 0, sizeof(int), s));
        if (n >= 1024 && oz_enabled() && oz_supported(n, n, n)) {                           // step 2
            MPJ_TRY(mgs_blocked_oz(b.Q, n, n, n, b.mgsw, b.sc.flag, b.oz1, b.ozs, b.Wt, s));
        } else {
            MPJ_TRY(mgs_inplace(b.Q, n, n, n, b.mgsw, b.sc.flag, s));
        }
        tm.mark(2);
        MPJ_CUDA_TRY(cudaMemsetAsync(b.T64, 0, sizeof(double) * (size_t)N * N, s));        // step 3
        MPJ_TRY(congruence_fp64(A, lda, b.Q, n, n, b.Wt, b.T64, N, b.oz1, b.oz2, b.sc.flag, s));
        MPJ_TRY(copy_pad_f64(b.Q, n, n, n, b.V64, N, N, N, true, s));                      // P = Q
        tm.mark(3);
        int fl = 0;
        MPJ_TRY(read_flag(b.sc.flag, &fl, s));
        if (fl) { if (st) st->status = MPJ_RANK_DEFICIENT; return MPJ_RANK_DEFICIENT; }
    } else {
        MPJ_TRY(copy_pad_f64(A, lda, n, n, b.T64, N, N, N, false, s));
        MPJ_TRY(set_identity_f64(b.V64, N, N, N, s));
        tm.mark(1); tm.mark(2); tm.mark(3);
    }
    MPJ_TRY(twosided_sweeps<double>(b.T64, b.V64, N, n, B, tol * normA, kU, op.max_sweeps,
                                    op.max_inner, b.eng, s, &r2));                          // step 4
    MPJ_TRY(diag_to_f64(b.T64, true, N, n, b.sc.d, s));
    MPJ_TRY(rank_sort(b.sc.d, 1, n, false, b.sc.perm, s));
    MPJ_TRY(gather_eig(b.T64, N, b.V64, N, b.sc.perm, n, Lambda, V, ldv, s));
    tm.mark(4);
    MPJ_CUDA_TRY(cudaStreamSynchronize(s));
    prof_flush();
    const double Np = 0.5 * (double)n * (double)(n - 1);
    if (st) {
        st->sweeps = r2.sweeps;
        st->sweeps_stage1 = r1.sweeps;
        st->rotations = Np > 0 ? r2.rotations / Np : 0.0;
        st->rotations_stage1 = Np > 0 ? r1.rotations / Np : 0.0;
        st->off_T0 = r2.off_initial;
        st->off_final = r2.off_final;
        st->ms_stage[0] = tm.ms(0, 1);
        st->ms_stage[1] = tm.ms(1, 2);
        st->ms_stage[2] = tm.ms(2, 3);
        st->ms_stage[3] = tm.ms(3, 4);
        st->status = r2.status;
    }
    return r2.status;
}

// ------------------------------------------------------------------ SVD layout
struct SvdBufs {
    double *C64, *V64, *Q;
    float *C32, *V32;
    void* eng;
    void* mgsw;
    void *ozA, *ozQ, *ozs;       // tensor-core operand slices (mp only): rows of A, Q, MGS panels
    double* Rbuf;                // 256 x n projections of the block MGS (mp only)
    double* nrm;
    Scal sc;
};

int svd_layout(Arena& a, int m, int n, int N, int B, bool mp, SvdBufs& b) {
    size_t mN = (size_t)m * N, NN = (size_t)N * N, nn = (size_t)n * n;
    b.C64 = a.take<double>(mN);
    b.V64 = a.take<double>(NN);
    b.Q = mp ? a.take<double>(nn) : nullptr;
    b.C32 = mp ? a.take<float>(mN) : nullptr;
    b.V32 = mp ? a.take<float>(NN) : nullptr;
    b.eng = a.take<char>(max2(max2(onesided_workspace_bytes<double>(m, N, B),
                                   onesided_workspace_bytes<float>(m, N, B)),
                              max2(onesided_tc64_supported(m, N, B) ? onesided_tc64_workspace_bytes(m, N) : 0,
                                   onesided_tc32_supported(m, N, B) ? onesided_tc32_workspace_bytes(m, N) : 0)));
    b.mgsw = mp ? a.take<char>(mgs_workspace_bytes(n, n)) : nullptr;
    b.ozA = mp ? a.take<char>(oz_operand_bytes(m, n)) : nullptr;
    b.ozQ = mp ? a.take<char>(oz_operand_bytes(n, n)) : nullptr;
    b.ozs = mp ? a.take<char>(mgs_panel_oz_bytes(n, n)) : nullptr;
    b.Rbuf = mp ? a.take<double>(256 * (size_t)n) : nullptr;
    b.nrm = a.take<double>((size_t)N);
    MPJ_TRY(take_scal(a, n, b.sc));
    if (a.base && (!b.C64 || !b.V64 || !b.eng || !b.nrm ||
                   (mp && (!b.Q || !b.C32 || !b.V32 || !b.mgsw || !b.ozA || !b.ozQ || !b.ozs || !b.Rbuf))))
        return MPJ_BAD_ARG;
    return MPJ_SUCCESS;
}

size_t svd_bytes(int m, int n, bool mp, const mpj_options* o) {
    int B = choose_block(n, o);
    int N = padded(n, B);
    Arena a;
    SvdBufs b;
    svd_layout(a, m, n, N, B, mp, b);
    return a.used + 512;
}

int gesvj_impl(bool mp, const double* A, int m, int n, int lda, double* Sigma, double* U, int ldu,
               double* V, int ldv, double tol, const mpj_options* opts, mpj_stats* st, void* work,
               size_t work_bytes, void* stream) {
    KnobScope knob_scope(opts);
    if (st) memset(st, 0, sizeof(*st));
    if (!A || !Sigma || !U || !V || n < 1 || m < n || lda < m || ldu < m || ldv < n || !(tol > 0) ||
        !std::isfinite(tol)) {
        set_error_msg("invalid argument");
        return MPJ_BAD_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Opts op = read_opts(opts);
    const int B = choose_block(n, opts);
    const int N = padded(n, B);
    Workspace ws;
    MPJ_TRY(ws.acquire(work, work_bytes, svd_bytes(m, n, mp, opts), s));
    Arena a;
    a.base = static_cast<char*>(ws.ptr);
    a.size = work ? work_bytes : svd_bytes(m, n, mp, opts);
    SvdBufs b;
    if (svd_layout(a, m, n, N, B, mp, b) != MPJ_SUCCESS) { set_error_msg("workspace layout"); return MPJ_BAD_ARG; }
    Timer tm;
    MPJ_TRY(tm.init(st != nullptr, s));
    tm.mark(0);
    double normA;
    MPJ_TRY(frob_norm(A, lda, m, n, b.sc, &normA, s));
    if (st) { st->norm_A = normA; st->block = B; }
    if (!std::isfinite(normA)) { if (st) st->status = MPJ_NONFINITE_INPUT; return MPJ_NONFINITE_INPUT; }
    MPJ_CUDA_TRY(cudaMemsetAsync(b.sc.flag, 0, sizeof(int), s));
    SweepResult r1, r2;
    if (mp) {
        // step 1: one-sided FP32 Jacobi of fl32(A); Z = right vectors ordered by decreasing ||c_j||
        if (!knobs().simt_stage1 && onesided_tc32_supported(m, N, B)) {
            // TF32 tensor cores: C and V row-major (the rotations' operands K-major)
            MPJ_TRY(copy_rowmajor_f32(A, lda, m, n, b.C32, N, s));
            MPJ_TRY(set_identity_f32(b.V32, N, N, N, s));
            MPJ_TRY(onesided_sweeps_tc32(b.C32, b.V32, m, N, n, sqrt((double)m) * kUps, op.ju_ratio,
                                         op.max_sweeps1, op.max_inner, b.eng, s, &r1));
            MPJ_TRY(colnorms2_rowmajor_f32(b.C32, m, N, n, b.sc.d, s));
            MPJ_TRY(rank_sort(b.sc.d, 1, n, true, b.sc.perm, s));
            MPJ_TRY(gather_z32_rowmajor(b.V32, N, b.sc.perm, n, b.Q, n, s));
        } else {
            MPJ_TRY(copy_pad_f32(A, lda, m, n, b.C32, m, m, N, false, s));
            MPJ_TRY(set_identity_f32(b.V32, N, N, N, s));
            MPJ_TRY(onesided_sweeps<float>(b.C32, m, b.V32, m, N, n, B, sqrt((double)m) * kUps,
                                           op.ju_ratio, op.max_sweeps1, op.max_inner, b.eng, s, &r1));
            MPJ_TRY(colnorms2_f32(b.C32, m, m, n, b.sc.d, s));
            MPJ_TRY(rank_sort(b.sc.d, 1, n, true, b.sc.perm, s));
            MPJ_TRY(gather_z32(b.V32, N, b.sc.perm, n, b.Q, n, s));
        }
        tm.mark(1);
        if (n >= 1024 && oz_enabled() && oz_supported(n, n, n)) {                           // step 2
            MPJ_TRY(mgs_blocked_oz(b.Q, n, n, n, b.mgsw, b.sc.flag, b.ozA, b.ozs, b.Rbuf, s));
        } else {
            MPJ_TRY(mgs_inplace(b.Q, n, n, n, b.mgsw, b.sc.flag, s));
        }
        tm.mark(2);
        MPJ_CUDA_TRY(cudaMemsetAsync(b.C64, 0, sizeof(double) * (size_t)m * N, s));        // step 3
        if (oz_enabled() && oz_supported(m, n, n)) {
            // C = A Q on the tensor cores by exact splitting: rows of A, columns of Q
            OzOperand oa, oq;
            MPJ_TRY(oz_operand(b.ozA, m, n, &oa));
            MPJ_TRY(oz_operand(b.ozQ, n, n, &oq));
            MPJ_TRY(oz_slice(A, 1, lda, m, n, &oa, s));
            MPJ_TRY(oz_slice(b.Q, n, 1, n, n, &oq, s));
            MPJ_TRY(oz_gemm(oa, oq, 1.0, 0.0, b.C64, m, false, b.sc.flag, s));
        } else {
            MPJ_TRY(dgemm(false, false, m, n, n, 1.0, A, lda, b.Q, n, 0.0, b.C64, m, false, s));
        }
        MPJ_TRY(copy_pad_f64(b.Q, n, n, n, b.V64, N, N, N, true, s));                      // V = Q
        tm.mark(3);
        int fl = 0;
        MPJ_TRY(read_flag(b.sc.flag, &fl, s));
        if (fl) { if (st) st->status = MPJ_RANK_DEFICIENT; return MPJ_RANK_DEFICIENT; }
    } else {
        MPJ_TRY(copy_pad_f64(A, lda, m, n, b.C64, m, m, N, false, s));
        MPJ_TRY(set_identity_f64(b.V64, N, N, N, s));
        tm.mark(1); tm.mark(2); tm.mark(3);
    }
    if (!knobs().simt_sweeps && onesided_tc64_supported(m, N, B)) {                        // steps 4-10
        MPJ_TRY(onesided_sweeps_tc64(b.C64, b.V64, m, N, n, tol, op.ju_ratio, op.max_sweeps, op.max_inner, b.eng,
                                     s, &r2));
    } else {
        MPJ_TRY(onesided_sweeps<double>(b.C64, m, b.V64, m, N, n, B, tol, op.ju_ratio, op.max_sweeps,
                                        op.max_inner, b.eng, s, &r2));
    }
    MPJ_TRY(colnorms_f64(b.C64, m, m, n, b.nrm, s));                                       // steps 11-13
    MPJ_TRY(rank_sort(b.nrm, 1, n, true, b.sc.perm, s));
    MPJ_TRY(svd_post(b.C64, m, b.V64, N, b.nrm, b.sc.perm, m, n, Sigma, U, ldu, V, ldv, b.sc.flag, s));
    tm.mark(4);
    int fl = 0;
    MPJ_TRY(read_flag(b.sc.flag, &fl, s));
    prof_flush();
    const double Np = 0.5 * (double)n * (double)(n - 1);
    int status = fl ? MPJ_RANK_DEFICIENT : r2.status;
    if (st) {
        st->sweeps = r2.sweeps;
        st->sweeps_stage1 = r1.sweeps;
        st->rotations = Np > 0 ? r2.rotations / Np : 0.0;
        st->rotations_stage1 = Np > 0 ? r1.rotations / Np : 0.0;
        st->ms_stage[0] = tm.ms(0, 1);
        st->ms_stage[1] = tm.ms(1, 2);
        st->ms_stage[2] = tm.ms(2, 3);
        st->ms_stage[3] = tm.ms(3, 4);
        st->status = status;
    }
    return status;
}

}  // namespace

// ==================================================================== C ABI
extern "C" {

int mpj_syevj_mp(const double* A, int n, int lda, double* Lambda, double* V, int ldv, double tol,
                 const mpj_options* opts, mpj_stats* stats, void* work, size_t work_bytes,
                 void* stream) {
    return syevj_impl(true, A, n, lda, Lambda, V, ldv, tol, opts, stats, work, work_bytes, stream);
}

int mpj_syevj_plain(const double* A, int n, int lda, double* Lambda, double* V, int ldv, double tol,
                    const mpj_options* opts, mpj_stats* stats, void* work, size_t work_bytes,
                    void* stream) {
    return syevj_impl(false, A, n, lda, Lambda, V, ldv, tol, opts, stats, work, work_bytes, stream);
}

size_t mpj_syevj_workspace_bytes(int n) {
    if (n < 1) return 0;
    return max2(evd_bytes(n, true, nullptr), evd_bytes(n, false, nullptr));
}

int mpj_gesvj_mp(const double* A, int m, int n, int lda, double* Sigma, double* U, int ldu,
                 double* V, int ldv, double tol, const mpj_options* opts, mpj_stats* stats,
                 void* work, size_t work_bytes, void* stream) {
    return gesvj_impl(true, A, m, n, lda, Sigma, U, ldu, V, ldv, tol, opts, stats, work, work_bytes,
                      stream);
}

int mpj_gesvj_plain(const double* A, int m, int n, int lda, double* Sigma, double* U, int ldu,
                    double* V, int ldv, double tol, const mpj_options* opts, mpj_stats* stats,
                    void* work, size_t work_bytes, void* stream) {
    return gesvj_impl(false, A, m, n, lda, Sigma, U, ldu, V, ldv, tol, opts, stats, work, work_bytes,
                      stream);
}

size_t mpj_gesvj_workspace_bytes(int m, int n) {
    if (n < 1 || m < n) return 0;
    return max2(svd_bytes(m, n, true, nullptr), svd_bytes(m, n, false, nullptr));
}

int mpj_stage1_syevj32(const double* A, int n, int lda, double* Z, int ldz, double* D,
                       const mpj_options* opts, mpj_stats* st, void* work, size_t work_bytes,
                       void* stream) {
    KnobScope knob_scope(opts);
    if (st) memset(st, 0, sizeof(*st));
    if (!A || !Z || !D || n < 1 || lda < n || ldz < n) { set_error_msg("invalid argument"); return MPJ_BAD_ARG; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Opts op = read_opts(opts);
    const int B = choose_block(n, opts);
    const int N = padded(n, B);
    Workspace ws;
    size_t need = evd_bytes(n, true, opts);
    MPJ_TRY(ws.acquire(work, work_bytes, need, s));
    Arena a;
    a.base = static_cast<char*>(ws.ptr);
    a.size = work ? work_bytes : need;
    EvdBufs b;
    if (evd_layout(a, n, N, B, true, b) != MPJ_SUCCESS) { set_error_msg("workspace layout"); return MPJ_BAD_ARG; }
    double normA;
    MPJ_TRY(frob_norm(A, lda, n, n, b.sc, &normA, s));
    if (!std::isfinite(normA)) return MPJ_NONFINITE_INPUT;
    SweepResult r1;
    MPJ_TRY(stage1_evd(A, lda, n, N, B, normA, op, b, &r1, s));
    MPJ_TRY(copy_f64(b.Q, n, n, n, Z, ldz, s));
    // D in the order of Z: D[i] = d[perm[i]] (FP32 diagonal widened exactly)
    MPJ_TRY(gather_vec(b.sc.d, b.sc.perm, n, D, s));
    MPJ_CUDA_TRY(cudaStreamSynchronize(s));
    if (st) {
        st->sweeps_stage1 = r1.sweeps;
        st->rotations_stage1 = n > 1 ? r1.rotations / (0.5 * n * (n - 1.0)) : 0.0;
        st->norm_A = normA;
        st->block = B;
        st->status = r1.status;
    }
    return r1.status;
}

// Large problems take the block MGS whose panel projections run on the tensor cores.
static bool mgs_use_oz(int m, int n) { return n >= 1024 && oz_enabled() && oz_supported(n, n, m); }

size_t mpj_mgs_workspace_bytes(int m, int n) {
    size_t b = mgs_workspace_bytes(m, n) + 1024;
    if (m >= 1 && n >= 1 && mgs_use_oz(m, n))
        b += oz_operand_bytes(n, m) + mgs_panel_oz_bytes(m, n) + sizeof(double) * 256 * (size_t)n + 1024;
    return b;
}

int mpj_mgs(const double* Z, int m, int n, int ldz, double* Q, int ldq, void* work,
            size_t work_bytes, void* stream) {
    if (!Z || !Q || n < 1 || m < n || ldz < m || ldq < m) { set_error_msg("invalid argument"); return MPJ_BAD_ARG; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace ws;
    size_t need = mpj_mgs_workspace_bytes(m, n);
    MPJ_TRY(ws.acquire(work, work_bytes, need, s));
    Arena a;
    a.base = static_cast<char*>(ws.ptr);
    a.size = work ? work_bytes : need;
    int* flag = a.take<int>(4);
    void* mw = a.take<char>(mgs_workspace_bytes(m, n));
    if (!flag || !mw) { set_error_msg("workspace layout"); return MPJ_BAD_ARG; }
    MPJ_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
    MPJ_TRY(copy_f64(Z, ldz, m, n, Q, ldq, s));
    if (mgs_use_oz(m, n)) {
        void* ozw = a.take<char>(oz_operand_bytes(n, m));
        void* ozs = a.take<char>(mgs_panel_oz_bytes(m, n));
        double* rb = a.take<double>(256 * (size_t)n);
        if (!ozw || !ozs || !rb) { set_error_msg("workspace layout"); return MPJ_BAD_ARG; }
        MPJ_TRY(mgs_blocked_oz(Q, m, n, ldq, mw, flag, ozw, ozs, rb, s));
    } else {
        MPJ_TRY(mgs_inplace(Q, m, n, ldq, mw, flag, s));
    }
    int fl = 0;
    MPJ_TRY(read_flag(flag, &fl, s));
    return fl ? MPJ_RANK_DEFICIENT : MPJ_SUCCESS;
}

size_t mpj_congruence_workspace_bytes(int n) {
    return n < 1 ? 0 : sizeof(double) * (size_t)n * n + 2 * oz_operand_bytes(n, n) + 4096;
}

int mpj_congruence(const double* A, int lda, const double* Q, int ldq, int n, double* T, int ldt,
                   void* work, size_t work_bytes, void* stream) {
    if (!A || !Q || !T || n < 1 || lda < n || ldq < n || ldt < n) { set_error_msg("invalid argument"); return MPJ_BAD_ARG; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace ws;
    size_t need = mpj_congruence_workspace_bytes(n);
    MPJ_TRY(ws.acquire(work, work_bytes, need, s));
    Arena a;
    a.base = static_cast<char*>(ws.ptr);
    a.size = work ? work_bytes : need;
    double* W = a.take<double>((size_t)n * n);
    void* oz1 = a.take<char>(oz_operand_bytes(n, n));
    void* oz2 = a.take<char>(oz_operand_bytes(n, n));
    int* flag = a.take<int>(4);
    if (!W || !oz1 || !oz2 || !flag) { set_error_msg("workspace layout"); return MPJ_BAD_ARG; }
    MPJ_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
    MPJ_TRY(congruence_fp64(A, lda, Q, ldq, n, W, T, ldt, oz1, oz2, flag, s));
    int fl = 0;
    MPJ_TRY(read_flag(flag, &fl, s));
    return MPJ_SUCCESS;
}

size_t mpj_sweeps_workspace_bytes(int n) {
    if (n < 1) return 0;
    int B = choose_block(n, nullptr);
    int N = padded(n, B);
    Arena a;
    a.take<double>((size_t)N * N);
    a.take<double>((size_t)N * N);
    a.take<char>(twosided_workspace_bytes<double>(N, B));
    return a.used + 512;
}

int mpj_sweeps(double* T, int ldt, double* P, int ldp, int n, double tol, double normA,
               const mpj_options* opts, mpj_stats* st, void* work, size_t work_bytes,
               void* stream) {
    KnobScope knob_scope(opts);
    if (st) memset(st, 0, sizeof(*st));
    if (!T || !P || n < 1 || ldt < n || ldp < n || !(tol > 0) || !(normA >= 0)) {
        set_error_msg("invalid argument");
        return MPJ_BAD_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Opts op = read_opts(opts);
    const int B = choose_block(n, opts);
    const int N = padded(n, B);
    Workspace ws;
    Arena sz;
    sz.take<double>((size_t)N * N);
    sz.take<double>((size_t)N * N);
    sz.take<char>(twosided_workspace_bytes<double>(N, B));
    size_t need = sz.used + 512;
    MPJ_TRY(ws.acquire(work, work_bytes, need, s));
    Arena a;
    a.base = static_cast<char*>(ws.ptr);
    a.size = work ? work_bytes : need;
    double* T64 = a.take<double>((size_t)N * N);
    double* V64 = a.take<double>((size_t)N * N);
    void* eng = a.take<char>(twosided_workspace_bytes<double>(N, B));
    if (!T64 || !V64 || !eng) { set_error_msg("workspace layout"); return MPJ_BAD_ARG; }
    MPJ_TRY(copy_pad_f64(T, ldt, n, n, T64, N, N, N, false, s));
    MPJ_TRY(copy_pad_f64(P, ldp, n, n, V64, N, N, N, true, s));
    SweepResult r;
    MPJ_TRY(twosided_sweeps<double>(T64, V64, N, n, B, tol * normA, kU, op.max_sweeps, op.max_inner,
                                    eng, s, &r));
    MPJ_TRY(copy_f64(T64, N, n, n, T, ldt, s));
    MPJ_TRY(copy_f64(V64, N, n, n, P, ldp, s));
    MPJ_CUDA_TRY(cudaStreamSynchronize(s));
    if (st) {
        st->sweeps = r.sweeps;
        st->rotations = n > 1 ? r.rotations / (0.5 * n * (n - 1.0)) : 0.0;
        st->off_T0 = r.off_initial;
        st->off_final = r.off_final;
        st->norm_A = normA;
        st->block = B;
        st->status = r.status;
    }
    return r.status;
}

const char* mpj_status_string(int status) {
    switch (status) {
        case MPJ_SUCCESS: return "success";
        case MPJ_BAD_ARG: return "invalid argument";
        case MPJ_NONFINITE_INPUT: return "input holds NaN or Inf";
        case MPJ_NOT_CONVERGED: return "not converged within max_sweeps";
        case MPJ_RANK_DEFICIENT: return "rank deficient (zero column norm)";
        case MPJ_CUDA_ERROR: return "CUDA error";
        case MPJ_NO_DEVICE: return "no sm_103 device";
        default: return "unknown status";
    }
}

const char* mpj_last_error(void) { return mpj::last_error(); }

const char* mpj_version(void) { return "mpjacobi 0.1 (sm_103a)"; }

}  // extern "C"
