// onesided.cu -- parallel-ordered one-sided block Jacobi (Algorithm 5.1, and
// steps 4-10 of Algorithm 5.2; in single precision also step 1 of Alg. 5.2).
//
// The padded column count N of C (m x N) is split into 2K blocks of b columns;
// each round of the round-robin tournament pairs the blocks disjointly and:
//   k_gram1   G = C[:, IJ]^T C[:, IJ] for every pair, split over row slabs
//             (partial Grams are summed in a fixed order by the solver);
//   k_solve1  one CTA per pair: cyclic Jacobi on the 2b x 2b Gram matrix.  A
//             rotation of Lemma 3.1 on G is exactly the rotation of Lemma 5.1
//             (mu = (c_j^T c_j - c_i^T c_i) / (2 c_i^T c_j)); a pair is rotated
//             only while |g_ij| > tol sqrt(g_ii g_jj).  The rotations are
//             accumulated into W (2b x 2b);
//   k_apply1  C[:, IJ] = C[:, IJ] W and V[:, IJ] = V[:, IJ] W, 64-row slabs.
// The number of applied rotations is read back once per sweep (Sec. 6 stop rule).
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "internal.h"
#include "jacobi_device.cuh"
#include "tile_device.cuh"

namespace mpj {

// Error-free transformations (Knuth's TwoSum, FMA-based TwoProd) for the
// compensated inner products of Ogita, Rump and Oishi (Dot2, SIAM J. Sci.
// Comput. 2005): the result is as accurate as if computed in twice the working
// precision and then rounded.
// Rounded arithmetic that nvcc may not contract into FMAs (the error-free
// transforms below depend on every product and sum being rounded separately).
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }

template <class Real>
__device__ __forceinline__ void dot2_step(Real a, Real b, Real& s, Real& c) {
    Real p = rmul(a, b);
    Real pe = fma(a, b, -p);
    Real t = radd(s, p);
    Real z = rsub(t, s);
    Real e = radd(rsub(s, rsub(t, z)), rsub(p, z));
    s = t;
    c = radd(c, radd(pe, e));
}

// Partial Gram of pair `blockIdx.x` over rows [split*rows_per, ...) of C.  With
// comp != 0 the products are accumulated with Dot2 and the partial is stored
// as an unevaluated sum hi + lo (Ghi, Glo); otherwise lo = 0.
template <class Real, int B>
__global__ void __launch_bounds__(kThreads)
k_gram1(const Real* __restrict__ C, size_t ldc, int m, int N, int round, int rows_per,
        Real* __restrict__ Ghi, Real* __restrict__ Glo, int nsplit, int comp) {
    constexpr int M = 2 * B;
    constexpr int LDS = M + SmemPad<Real>::value;
    constexpr int RC = 32;                     // rows per chunk
    __shared__ __align__(16) Real Xs[RC * LDS];
    const int nblocks = N / B;
    int I, J;
    round_pair(round, blockIdx.x, nblocks, I, J);
    const int split = blockIdx.y;
    const int r0 = split * rows_per;
    const int r1 = min(m, r0 + rows_per);
    constexpr int RM = M / 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    Real acc[RM][RM], cmp[RM][RM];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RM; ++j) { acc[i][j] = Real(0); cmp[i][j] = Real(0); }
    for (int rc = r0; rc < r1; rc += RC) {
        for (int t = threadIdx.x; t < RC * M; t += kThreads) {
            int r = t % RC, c = t / RC;
            int gr = rc + r;
            Real v = Real(0);
            if (gr < r1) v = C[(size_t)gr + (size_t)pair_global(c, I, J, B) * ldc];
            Xs[r * LDS + c] = v;                  // Xs[row][col]
        }
        __syncthreads();
        if (comp) {
            for (int r = 0; r < RC; ++r) {
                Real a[RM], b[RM];
#pragma unroll
                for (int i = 0; i < RM; ++i) a[i] = Xs[r * LDS + ty * RM + i];
#pragma unroll
                for (int j = 0; j < RM; ++j) b[j] = Xs[r * LDS + tx * RM + j];
#pragma unroll
                for (int i = 0; i < RM; ++i)
#pragma unroll
                    for (int j = 0; j < RM; ++j) dot2_step(a[i], b[j], acc[i][j], cmp[i][j]);
            }
        } else {
#pragma unroll 4
            for (int r = 0; r < RC; ++r) {
                Real a[RM], b[RM];
#pragma unroll
                for (int i = 0; i < RM; ++i) a[i] = Xs[r * LDS + ty * RM + i];
#pragma unroll
                for (int j = 0; j < RM; ++j) b[j] = Xs[r * LDS + tx * RM + j];
#pragma unroll
                for (int i = 0; i < RM; ++i)
#pragma unroll
                    for (int j = 0; j < RM; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
        }
        __syncthreads();
    }
    size_t base = ((size_t)blockIdx.x * nsplit + split) * M * M;
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RM; ++j) {
            size_t idx = base + (size_t)(tx * RM + j) * M + ty * RM + i;
            Real h = radd(acc[i][j], cmp[i][j]);
            Ghi[idx] = h;
            Glo[idx] = rsub(cmp[i][j], rsub(h, acc[i][j]));
        }
}

// Threads of a block solve: FP32 solves are chains of short dependent steps
// (more warps hide more of their latency, as in the FP32 two-sided solves);
// FP64 solves are bound by the FP64 pipe.
template <class Real>
constexpr int solve1_threads() { return sizeof(Real) == 4 ? 1024 : kSolveThreads; }

template <class Real, int B>
__global__ void __launch_bounds__(solve1_threads<Real>())
k_solve1(const Real* __restrict__ Ghi, const Real* __restrict__ Glo, int nsplit,
         Real* __restrict__ Fbuf, Real tol_rot,
         Real gate, int max_inner, int cross_round, unsigned long long* __restrict__ rot_counter) {
    constexpr int M = 2 * B;
    constexpr int LD = M + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    Real* S = reinterpret_cast<Real*>(smraw);
    Real* F = S + M * LD;
    Real* G2 = F + M * LD;
    Real* cs = G2 + M * LD;
    int* ip = reinterpret_cast<int*>(cs + InnerLayout<Real, M>::kRealRot);
    int* flag = ip + InnerLayout<Real, M>::kFlagOffset;
    const size_t off = (size_t)blockIdx.x * nsplit * M * M;
    for (int t = threadIdx.x; t < M * M; t += blockDim.x) {
        int r = t % M, c = t / M;
        // compensated sum of the split partials (hi + lo pairs)
        Real sacc = Real(0), cacc = Real(0);
        for (int sp = 0; sp < nsplit; ++sp) {
            size_t idx = off + (size_t)sp * M * M + (size_t)c * M + r;
            Real p = Ghi[idx];
            Real tt = radd(sacc, p), z = rsub(tt, sacc);
            cacc = radd(cacc, radd(radd(rsub(sacc, rsub(tt, z)), rsub(p, z)), Glo[idx]));
            sacc = tt;
        }
        S[c * LD + r] = sacc + cacc;
        F[c * LD + r] = Real(0);
    }
    __syncthreads();
    int applied = inner_jacobi<Real, M>(S, F, cs, ip, tol_rot, Real(0), max_inner, cross_round);
    finish_block<Real, M>(F, G2, Fbuf + (size_t)blockIdx.x * M * M, gate, flag, nullptr);
    if (threadIdx.x == 0 && applied) atomicAdd(rot_counter, (unsigned long long)applied);
}

template <class Real, int B>
__global__ void __launch_bounds__(kThreads)
k_apply1(Real* __restrict__ C, size_t ldc, int m, Real* __restrict__ V, int N,
         const Real* __restrict__ Wbuf, int round, int n_ctiles) {
    constexpr int M = 2 * B;
    constexpr int LDS = M + SmemPad<Real>::value;
    extern __shared__ __align__(16) unsigned char smraw[];
    Real* Xs = reinterpret_cast<Real*>(smraw);
    Real* Wb = Xs + M * LDS;
    const int nblocks = N / B;
    const int K = nblocks / 2;
    int tile = blockIdx.x;
    int Ib, Jb;
    if (tile < n_ctiles) {
        int rb = tile / K, b = tile % K;
        round_pair(round, b, nblocks, Ib, Jb);
        load_w<Real, M, LDS>(Wb, Wbuf, b);
        right_multiply_rows<Real, B>(C, ldc, m, rb * M, Ib, Jb, Xs, Wb);
    } else {
        int t2 = tile - n_ctiles;
        int rb = t2 / K, b = t2 % K;
        round_pair(round, b, nblocks, Ib, Jb);
        load_w<Real, M, LDS>(Wb, Wbuf, b);
        right_multiply_rows<Real, B>(V, (size_t)N, N, rb * M, Ib, Jb, Xs, Wb);
    }
}

static void gram_split(int m, int K, int M, int* nsplit, int* rows_per) {
    int want = (304 + K - 1) / K;                         // ~2 CTAs per SM in total
    int max_split = (m + M - 1) / M;
    int ns = want < 1 ? 1 : (want > max_split ? max_split : want);
    int rp = (m + ns - 1) / ns;
    rp = (rp + 31) / 32 * 32;
    ns = (m + rp - 1) / rp;
    *nsplit = ns < 1 ? 1 : ns;
    *rows_per = rp < 32 ? 32 : rp;
}

template <class Real>
size_t onesided_workspace_bytes(int m, int N, int B) {
    int M = 2 * B, K = N / M, ns, rp;
    gram_split(m, K, M, &ns, &rp);
    Arena a;
    a.take<Real>((size_t)K * M * M);
    a.take<Real>((size_t)K * ns * M * M);
    a.take<Real>((size_t)K * ns * M * M);
    a.take<unsigned long long>(4);
    return a.used + 256;
}

template <class Real, int B>
static int configure_onesided() {
    constexpr int M = 2 * B;
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_solve1<Real, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)InnerLayout<Real, M>::bytes));
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_apply1<Real, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(sizeof(Real) * 2 * M * (M + SmemPad<Real>::value))));
    return MPJ_SUCCESS;
}

template <class Real, int B>
static int launch_round1(Real* C, int ldc, Real* V, int m, int N, Real* Wbuf, Real* Ghi, Real* Glo,
                         int nsplit, int rows_per, int r, Real tol_rot, Real gate, int max_inner,
                         int comp, int cross, unsigned long long* rot, cudaStream_t s) {
    constexpr int M = 2 * B;
    const int K = N / M;
    dim3 g(K, nsplit);
    { MPJ_PROF(sizeof(Real) == 8 ? PC_GRAM1_F64 : PC_GRAM1_F32, s);
    k_gram1<Real, B><<<g, kThreads, 0, s>>>(C, (size_t)ldc, m, N, r, rows_per, Ghi, Glo, nsplit, comp); }
    MPJ_LAUNCH_CHECK("k_gram1");
    { MPJ_PROF(sizeof(Real) == 8 ? PC_SOLVE1_F64 : PC_SOLVE1_F32, s);
    k_solve1<Real, B><<<K, solve1_threads<Real>(), InnerLayout<Real, M>::bytes, s>>>(Ghi, Glo, nsplit, Wbuf, tol_rot,
                                                                      gate, max_inner, cross ? r : -1, rot); }
    MPJ_LAUNCH_CHECK("k_solve1");
    int n_ctiles = ((m + M - 1) / M) * K;
    int n_vtiles = (N / M) * K;
    { MPJ_PROF(sizeof(Real) == 8 ? PC_APPLY1_F64 : PC_APPLY1_F32, s);
    k_apply1<Real, B><<<n_ctiles + n_vtiles, kThreads,
                        sizeof(Real) * 2 * M * (M + SmemPad<Real>::value), s>>>(
        C, (size_t)ldc, m, V, N, Wbuf, r, n_ctiles); }
    MPJ_LAUNCH_CHECK("k_apply1");
    return MPJ_SUCCESS;
}

// Fraction of N below which a sweep's rotation count turns the compensated
// Gram on (0: only once a sweep passes the stopping rule).
constexpr double kCompSwitch = 0.0;
template <class Real>
int onesided_sweeps(Real* C, int ldc, Real* V, int m, int N, int n, int B, double tol_rot,
                    double ju_ratio, int max_sweeps, int max_inner, void* work, cudaStream_t s,
                    SweepResult* res) {
    const int M = 2 * B, K = N / M;
    int nsplit, rows_per;
    gram_split(m, K, M, &nsplit, &rows_per);
    Arena ar;
    ar.base = static_cast<char*>(work);
    ar.size = onesided_workspace_bytes<Real>(m, N, B);
    Real* Wbuf = ar.take<Real>((size_t)K * M * M);
    Real* Ghi = ar.take<Real>((size_t)K * nsplit * M * M);
    Real* Glo = ar.take<Real>((size_t)K * nsplit * M * M);
    unsigned long long* rot = ar.take<unsigned long long>(4);
    if (!Wbuf || !Ghi || !Glo || !rot) { set_error_msg("workspace too small"); return MPJ_BAD_ARG; }
    HostScratch hs;
    MPJ_TRY(hs.init());
    if (B == 16) { MPJ_TRY((configure_onesided<Real, 16>())); }
    else         { MPJ_TRY((configure_onesided<Real, 32>())); }
    const double Npairs = 0.5 * (double)n * (double)(n - 1);
    res->sweeps = 0;
    res->rotations = 0;
    res->status = MPJ_NOT_CONVERGED;
    const int rounds = 2 * K - 1;
    const Real gate = (Real)(sizeof(Real) == 8 ? 1.0 / 67108864.0 : 1.0 / 4096.0);   // 2^-26 / 2^-12
    // FP64 only: the compensated (Dot2) Gram makes the cosines that decide
    // convergence (and the orthogonality of U) accurate to working precision
    // whatever the growth of the partial sums, at about four times the cost of
    // an uncompensated sweep.  By default the sweeps run uncompensated until one
    // passes the stopping rule; then compensated sweeps continue until one
    // passes it again, so the final decision rests on cosines accurate to
    // working precision (comp_switch > 0 turns compensation on earlier, once a
    // sweep applies fewer than comp_switch * N rotations; comp_switch < 0
    // never, the first sweep that passes the rule ends the iteration).
    const bool dbl = sizeof(Real) == 8;
    const double comp_switch = dbl ? kCompSwitch : -1.0;
    int comp = 0;
    // FP32: the cross-pair inner schedule of inner_jacobi once the rounds of a
    // sweep cover the intra-block tournament (N >= b^2); FP64 keeps the full one
    const int cross = !dbl && N >= B * B && !knobs().full_inner;
    while (res->sweeps < max_sweeps) {
        MPJ_CUDA_TRY(cudaMemsetAsync(rot, 0, sizeof(unsigned long long), s));
        for (int r = 0; r < rounds; ++r) {
            if (B == 16) {
                MPJ_TRY((launch_round1<Real, 16>(C, ldc, V, m, N, Wbuf, Ghi, Glo, nsplit, rows_per, r,
                                                 (Real)tol_rot, gate, max_inner, comp, cross, rot, s)));
            } else {
                MPJ_TRY((launch_round1<Real, 32>(C, ldc, V, m, N, Wbuf, Ghi, Glo, nsplit, rows_per, r,
                                                 (Real)tol_rot, gate, max_inner, comp, cross, rot, s)));
            }
        }
        MPJ_CUDA_TRY(cudaMemcpyAsync(hs.u, rot, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        MPJ_CUDA_TRY(cudaStreamSynchronize(s));
        prof_flush();
        res->sweeps += 1;
        res->rotations += (double)hs.u[0];
        if (trace_on())
            fprintf(stderr, "[mpj] onesided<%s> m=%d n=%d sweep %d: %llu rotations (%.4f N) comp=%d\n",
                    dbl ? "f64" : "f32", m, n, res->sweeps, hs.u[0], hs.u[0] / Npairs, comp);
        const double applied = (double)hs.u[0];
        const bool rule = hs.u[0] == 0 || applied < ju_ratio * Npairs;
        if (rule && (comp || comp_switch < 0.0)) { res->status = MPJ_SUCCESS; break; }
        if (!comp && comp_switch >= 0.0 && (rule || applied < comp_switch * Npairs)) comp = 1;
    }
    return MPJ_SUCCESS;
}

// The FP32 block solves of one round (b = 32) on Gram partials formed by the
// caller -- the tensor-core step 1 of Alg. 5.2 (tc_apply.cu): W_b - I to Wbuf.
int configure_solve1_f32() { return configure_onesided<float, 32>(); }
int solve1_f32_round(const float* Ghi, const float* Glo, int nsplit, int K, float* Wbuf, double tol_rot,
                     int max_inner, int cross_round, unsigned long long* rot, cudaStream_t s) {
    {
        MPJ_PROF(PC_SOLVE1_F32, s);
        k_solve1<float, 32><<<K, solve1_threads<float>(), InnerLayout<float, 64>::bytes, s>>>(
            Ghi, Glo, nsplit, Wbuf, (float)tol_rot, 1.0f / 4096.0f, max_inner, cross_round, rot);
    }
    MPJ_LAUNCH_CHECK("k_solve1<float>");
    return MPJ_SUCCESS;
}

template size_t onesided_workspace_bytes<float>(int, int, int);
template size_t onesided_workspace_bytes<double>(int, int, int);
template int onesided_sweeps<float>(float*, int, float*, int, int, int, int, double, double, int,
                                    int, void*, cudaStream_t, SweepResult*);
template int onesided_sweeps<double>(double*, int, double*, int, int, int, int, double, double,
                                     int, int, void*, cudaStream_t, SweepResult*);

}  // namespace mpj
