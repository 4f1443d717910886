// twosided.cu -- parallel-ordered block Jacobi for a symmetric matrix
// (Algorithm 3.2 with a parallel order; step 4 of Algorithm 4.1; and, in single
// precision, the eigensolver of step 1).
//
// The padded order N is split into 2K blocks of b indices.  One sweep is 2K-1
// rounds of the round-robin tournament; in a round the K block pairs (I, J) are
// disjoint, so:
//   k_solve2  one CTA per pair: the 2b x 2b problem T[IJ, IJ] is diagonalised
//             in shared memory by cyclic Jacobi (Lemma 3.1 rotations, Remark 3.7
//             skip rule), the rotations are accumulated into W (2b x 2b) and the
//             rotated diagonal tile is written back;
//   k_apply2  every off-diagonal tile T[IJ_a, IJ_b] (a < b) becomes
//             W_a^T T[IJ_a, IJ_b] W_b (and its transpose is mirrored), and every
//             64-row slab of V becomes V[:, IJ_b] W_b.
// ||off(T)||_F is reduced once per sweep and read back for the while-test.
// k_apply2 is two kernels: k_apply2T (tiles of T) and k_apply2V (slabs of V).
#include <cmath>
#include <cstdio>

#include "internal.h"
#include <cstdlib>
#include "jacobi_device.cuh"
#include "tile_device.cuh"

namespace mpj {

template <class Real, int B>
__global__ void __launch_bounds__(kSolveThreads)
k_solve2(Real* __restrict__ T, int N, Real* __restrict__ Fbuf, float* __restrict__ fmax, int round,
         Real eps, Real tau, Real gate, int max_inner, unsigned long long* __restrict__ rot_counter) {
    constexpr int M = 2 * B;
    constexpr int LD = M + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    Real* S = reinterpret_cast<Real*>(smraw);
    Real* F = S + M * LD;
    Real* G = F + M * LD;
    Real* cs = G + M * LD;
    int* ip = reinterpret_cast<int*>(cs + 4 * (M / 2));
    int* flag = ip + 3 * (M / 2) + 2;
    const int nblocks = N / B;
    int I, J;
    round_pair(round, blockIdx.x, nblocks, I, J);
    for (int t = threadIdx.x; t < M * M; t += blockDim.x) {
        int r = t % M, c = t / M;
        S[c * LD + r] = T[(size_t)pair_global(r, I, J, B) + (size_t)pair_global(c, I, J, B) * N];
        F[c * LD + r] = Real(0);
    }
    __syncthreads();
    int applied = inner_jacobi<Real, M>(S, F, cs, ip, eps, tau, max_inner);
    for (int t = threadIdx.x; t < M * M; t += blockDim.x) {
        int r = t % M, c = t / M;
        T[(size_t)pair_global(r, I, J, B) + (size_t)pair_global(c, I, J, B) * N] = S[c * LD + r];
    }
    finish_block<Real, M>(F, G, Fbuf + (size_t)blockIdx.x * M * M, gate, flag, fmax + blockIdx.x);
    if (threadIdx.x == 0 && applied) atomicAdd(rot_counter, (unsigned long long)applied);
}

// Tile (a, b), a < b, of the current pairing: decode from the linear tile index.
__device__ __forceinline__ void decode_tile(int tile, int K, int& a, int& b) {
    a = 0;
    int rem = tile;
    while (rem >= K - 1 - a) { rem -= K - 1 - a; ++a; }
    b = a + 1 + rem;
}

// Shared memory of the tile kernels: FP path 3 (T) or 2 (V) planes of M*LDS
// Real; double-float path 6 (T) or 4 (V) float planes of M*(M+4).
template <class Real, int B>
struct ApplySmem {
    static constexpr int M = 2 * B;
    static constexpr size_t fp_t = sizeof(Real) * 3 * M * (M + SmemPad<Real>::value);
    static constexpr size_t fp_v = sizeof(Real) * 2 * M * (M + SmemPad<Real>::value);
    static constexpr size_t df_t = sizeof(Real) == 8 ? sizeof(float) * 6 * M * (M + 4) : 0;
    static constexpr size_t df_v = sizeof(Real) == 8 ? sizeof(float) * 4 * M * (M + 4) : 0;
    static constexpr size_t t = fp_t > df_t ? fp_t : df_t;
    static constexpr size_t v = fp_v > df_v ? fp_v : df_v;
};

// Double-float version of the off-diagonal tile update (Real = double only).
template <int B>
__device__ void apply_tile_df(double* T, int N, const double* __restrict__ Fbuf, int a, int b,
                              int Ia, int Ja, int Ib, int Jb, float* smf) {
    constexpr int M = 2 * B;
    constexpr int LDSF = M + 4;
    constexpr int LDS = M + SmemPad<double>::value;
    constexpr int RM = M / 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float* Xh = smf;
    float* Xl = Xh + M * LDSF;
    float* Bh = Xl + M * LDSF;     // F_b, then Z
    float* Bl = Bh + M * LDSF;
    float* Ah = Bl + M * LDSF;     // F_a
    float* Al = Ah + M * LDSF;
    const double* Fb = Fbuf + (size_t)b * M * M;
    const double* Fa = Fbuf + (size_t)a * M * M;
    double z[RM][RM];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RM; ++j)
            z[i][j] = T[(size_t)pair_global(ty * RM + i, Ia, Ja, B) +
                        (size_t)pair_global(tx * RM + j, Ib, Jb, B) * N];
    for (int t = threadIdx.x; t < M * M; t += kThreads) {
        int r = t % M, kc = t / M;
        double v = T[(size_t)pair_global(r, Ia, Ja, B) + (size_t)pair_global(kc, Ib, Jb, B) * N];
        split_df(v, Xh[kc * LDSF + r], Xl[kc * LDSF + r]);
        int k = t / M, c = t % M;
        split_df(Fb[t], Bh[k * LDSF + c], Bl[k * LDSF + c]);
        split_df(Fa[t], Ah[k * LDSF + c], Al[k * LDSF + c]);
    }
    __syncthreads();
    float ah[RM][RM], al[RM][RM];
    tile_mm_df<M, LDSF>(Xh, Xl, Bh, Bl, ah, al);                  // X F_b
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RM; ++j) z[i][j] += (double)ah[i][j] + (double)al[i][j];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RM; ++j) {
            int R = ty * RM + i, C = tx * RM + j;
            split_df(z[i][j], Bh[R * LDSF + C], Bl[R * LDSF + C]);  // Z row-major
        }
    __syncthreads();
    tile_mm_df<M, LDSF>(Ah, Al, Bh, Bl, ah, al);                  // F_a^T Z
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RM; ++j) z[i][j] += (double)ah[i][j] + (double)al[i][j];
    __syncthreads();
    double* Ys = reinterpret_cast<double*>(smf);                  // col-major
    double* Yr = Ys + M * LDS;                                    // row-major
    tile_store_colmajor<double, M, LDS>(Ys, z);
    tile_store_rowmajor<double, M, LDS>(Yr, z);
    __syncthreads();
    for (int t = threadIdx.x; t < M * M; t += kThreads) {
        int r = t % M, c = t / M;
        T[(size_t)pair_global(r, Ia, Ja, B) + (size_t)pair_global(c, Ib, Jb, B) * N] = Ys[c * LDS + r];
        int c2 = t % M, r2 = t / M;
        T[(size_t)pair_global(c2, Ib, Jb, B) + (size_t)pair_global(r2, Ia, Ja, B) * N] = Yr[r2 * LDS + c2];
    }
}

// Off-diagonal tiles in delta form: Z = X + X F_b, Y = Z + F_a^T Z = W_a^T X W_b.
// A tile whose two block rotations have max |F| <= df_gate is computed in
// double-float arithmetic (Real = double), the others in Real.
template <class Real, int B>
__global__ void __launch_bounds__(kThreads)
k_apply2T(Real* __restrict__ T, int N, const Real* __restrict__ Fbuf, const float* __restrict__ fmax,
          int round, float df_gate) {
    constexpr int M = 2 * B;
    constexpr int LDS = M + SmemPad<Real>::value;
    constexpr int RM = M / 16;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nblocks = N / B;
    const int K = nblocks / 2;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int a, b;
    decode_tile(blockIdx.x, K, a, b);
    int Ia, Ja, Ib, Jb;
    round_pair(round, a, nblocks, Ia, Ja);
    round_pair(round, b, nblocks, Ib, Jb);
    const float fa = fmax[a], fb = fmax[b];
    if (fa == 0.f && fb == 0.f) return;              // W_a = W_b = I: the tile is unchanged
    if constexpr (sizeof(Real) == 8) {
        if (fa <= df_gate && fb <= df_gate) {
            apply_tile_df<B>(reinterpret_cast<double*>(T), N, reinterpret_cast<const double*>(Fbuf),
                             a, b, Ia, Ja, Ib, Jb, reinterpret_cast<float*>(smraw));
            return;
        }
    }
    Real* Xs = reinterpret_cast<Real*>(smraw);
    Real* Fb = Xs + M * LDS;     // F_b, then Z
    Real* Fa = Fb + M * LDS;
    gather_tile<Real, B>(Xs, T, N, Ia, Ja, Ib, Jb);
    load_w<Real, M, LDS>(Fb, Fbuf, b);
    load_w<Real, M, LDS>(Fa, Fbuf, a);
    __syncthreads();
    Real acc[M / 16][M / 16];
    tile_mm<Real, M, LDS>(Xs, Fb, acc);              // (X F_b)[r][c]
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RM; ++j) acc[i][j] += Xs[(tx * RM + j) * LDS + ty * RM + i];
    __syncthreads();
    tile_store_rowmajor<Real, M, LDS>(Fb, acc);      // Z row-major over F_b
    __syncthreads();
    tile_mm<Real, M, LDS>(Fa, Fb, acc);              // (F_a^T Z)[r][c]
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RM; ++j) acc[i][j] += Fb[(ty * RM + i) * LDS + tx * RM + j];
    __syncthreads();
    tile_store_colmajor<Real, M, LDS>(Xs, acc);      // Xs[c*LDS + r]
    tile_store_rowmajor<Real, M, LDS>(Fb, acc);      // Fb[r*LDS + c]
    __syncthreads();
    for (int t = threadIdx.x; t < M * M; t += kThreads) {
        int r = t % M, c = t / M;
        T[(size_t)pair_global(r, Ia, Ja, B) + (size_t)pair_global(c, Ib, Jb, B) * N] = Xs[c * LDS + r];
        int c2 = t % M, r2 = t / M;                  // mirrored tile, coalesced in c2
        T[(size_t)pair_global(c2, Ib, Jb, B) + (size_t)pair_global(r2, Ia, Ja, B) * N] =
            Fb[r2 * LDS + c2];
    }
}

// 2b-row slabs of V times the block rotation of their pair: V[:, IJ_b] (I + F_b).
template <class Real, int B>
__global__ void __launch_bounds__(kThreads)
k_apply2V(Real* __restrict__ V, int N, const Real* __restrict__ Fbuf, const float* __restrict__ fmax,
          int round, float df_gate) {
    constexpr int M = 2 * B;
    constexpr int LDS = M + SmemPad<Real>::value;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nblocks = N / B;
    const int K = nblocks / 2;
    int rb = blockIdx.x / K, b = blockIdx.x % K;
    int Ib, Jb;
    round_pair(round, b, nblocks, Ib, Jb);
    const float fb = fmax[b];
    if (fb == 0.f) return;                           // W_b = I: the slab is unchanged
    if constexpr (sizeof(Real) == 8) {
        if (fb <= df_gate) {
            right_multiply_rows_df<B>(reinterpret_cast<double*>(V), (size_t)N, N, rb * M, Ib, Jb,
                                      reinterpret_cast<const double*>(Fbuf) + (size_t)b * M * M,
                                      reinterpret_cast<float*>(smraw));
            return;
        }
    }
    Real* Xs = reinterpret_cast<Real*>(smraw);
    Real* Fb = Xs + M * LDS;
    load_w<Real, M, LDS>(Fb, Fbuf, b);
    right_multiply_rows<Real, B>(V, (size_t)N, N, rb * M, Ib, Jb, Xs, Fb);
}

// MPJ_DF_GATE overrides the double-float gate (a negative value disables the
// double-float path); used to compare both arithmetics on the same inputs.
static float df_gate_override(float dflt) {
    const char* e = std::getenv("MPJ_DF_GATE");
    return e ? (float)atof(e) : dflt;
}

template <class Real>
size_t twosided_workspace_bytes(int N, int B) {
    Arena a;
    int K = N / (2 * B), M = 2 * B;
    a.take<Real>((size_t)K * M * M);
    a.take<float>((size_t)K);
    a.take<double>(1024);
    a.take<double>(4);
    a.take<unsigned long long>(4);
    return a.used + 256;
}

template <class Real, int B>
static int configure_twosided() {
    constexpr int M = 2 * B;
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_solve2<Real, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)InnerLayout<Real, M>::bytes));
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_apply2T<Real, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)ApplySmem<Real, B>::t));
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_apply2V<Real, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)ApplySmem<Real, B>::v));
    return MPJ_SUCCESS;
}

template <class Real, int B>
static int launch_round(Real* T, Real* V, int N, Real* Wbuf, float* fmax, int r, Real eps, Real tau,
                        Real gate, float df_gate, int max_inner, unsigned long long* rot,
                        cudaStream_t s) {
    constexpr int M = 2 * B;
    const int K = N / M;
    const bool dbl = sizeof(Real) == 8;
    { MPJ_PROF(dbl ? PC_SOLVE2_F64 : PC_SOLVE2_F32, s);
      k_solve2<Real, B><<<K, kSolveThreads, InnerLayout<Real, M>::bytes, s>>>(T, N, Wbuf, fmax, r, eps, tau,
                                                                         gate, max_inner, rot); }
    MPJ_LAUNCH_CHECK("k_solve2");
    int n_ttiles = K * (K - 1) / 2;
    if (n_ttiles > 0) {
        MPJ_PROF(dbl ? PC_APPLY2_F64 : PC_APPLY2_F32, s);
        k_apply2T<Real, B><<<n_ttiles, kThreads, ApplySmem<Real, B>::t, s>>>(T, N, Wbuf, fmax, r, df_gate);
        MPJ_LAUNCH_CHECK("k_apply2T");
    }
    {
        MPJ_PROF(dbl ? PC_APPLY2V_F64 : PC_APPLY2V_F32, s);
        k_apply2V<Real, B><<<(N / M) * K, kThreads, ApplySmem<Real, B>::v, s>>>(V, N, Wbuf, fmax, r, df_gate);
        MPJ_LAUNCH_CHECK("k_apply2V");
    }
    return MPJ_SUCCESS;
}

template <class Real>
int twosided_sweeps(Real* T, Real* V, int N, int n, int B, double tol_abs, double eps_skip,
                    int max_sweeps, int max_inner, void* work, cudaStream_t s, SweepResult* res) {
    const int M = 2 * B;
    const int K = N / M;
    Arena ar;
    ar.base = static_cast<char*>(work);
    ar.size = twosided_workspace_bytes<Real>(N, B);
    Real* Wbuf = ar.take<Real>((size_t)K * M * M);
    float* fmax = ar.take<float>((size_t)K);
    double* partial = ar.take<double>(1024);
    double* offv = ar.take<double>(4);
    unsigned long long* rot = ar.take<unsigned long long>(4);
    if (!Wbuf || !fmax || !partial || !offv || !rot) { set_error_msg("workspace too small"); return MPJ_BAD_ARG; }
    HostScratch hs;
    MPJ_TRY(hs.init());
    const bool dbl = sizeof(Real) == 8;
    if (B == 16) { MPJ_TRY((configure_twosided<Real, 16>())); }
    else         { MPJ_TRY((configure_twosided<Real, 32>())); }

    // Scale T by a power of two so that ||T||_F is about 1: exact, and it keeps the
    // float halves of the double-float products far from the FP32 exponent limits.
    int e2 = 0;
    if (dbl) {
        MPJ_TRY(sumsq_f64(reinterpret_cast<const double*>(T), N, N, N, partial, offv, s));
        MPJ_CUDA_TRY(cudaMemcpyAsync(hs.d, offv, sizeof(double), cudaMemcpyDeviceToHost, s));
        MPJ_CUDA_TRY(cudaStreamSynchronize(s));
        double nt = sqrt(hs.d[0]);
        if (nt > 0 && std::isfinite(nt)) e2 = -ilogb(nt);
        if (e2 != 0) MPJ_TRY(scale_pow2_f64(reinterpret_cast<double*>(T), N, N, N, e2, s));
        tol_abs = ldexp(tol_abs, e2);
    }
    MPJ_TRY(offnorm2(T, dbl, N, n, partial, offv, s));
    MPJ_CUDA_TRY(cudaMemcpyAsync(hs.d, offv, sizeof(double), cudaMemcpyDeviceToHost, s));
    MPJ_CUDA_TRY(cudaStreamSynchronize(s));
    double off = sqrt(hs.d[0]);
    res->off_initial = ldexp(off, -e2);
    res->sweeps = 0;
    res->rotations = 0;
    res->status = MPJ_NOT_CONVERGED;
    const int rounds = 2 * K - 1;
    // entries below tau cannot keep ||off(T)||_F above tol_abs once all are below it
    const Real tau = (Real)(tol_abs / (double)N);
    // Newton-Schulz re-orthogonalisation of W = I + F when some |F| >= 2^-6 (FP64)
    // or 2^-12 (FP32): with F accumulated in delta form, smaller blocks stay
    // orthogonal to working precision without it.
    const Real gate = (Real)(dbl ? 1.0 / 64.0 : 1.0 / 4096.0);
    // double-float tile products when both block rotations have max |F| <= 2^-8
    const float df_gate = dbl ? df_gate_override(1.0f / 256.0f) : -1.0f;
    while (res->sweeps < max_sweeps) {
        if (!std::isfinite(off)) { res->status = MPJ_NONFINITE_INPUT; break; }
        if (!(off > tol_abs)) { res->status = MPJ_SUCCESS; break; }
        MPJ_CUDA_TRY(cudaMemsetAsync(rot, 0, sizeof(unsigned long long), s));
        for (int r = 0; r < rounds; ++r) {
            if (B == 16) {
                MPJ_TRY((launch_round<Real, 16>(T, V, N, Wbuf, fmax, r, (Real)eps_skip, tau, gate,
                                                df_gate, max_inner, rot, s)));
            } else {
                MPJ_TRY((launch_round<Real, 32>(T, V, N, Wbuf, fmax, r, (Real)eps_skip, tau, gate,
                                                df_gate, max_inner, rot, s)));
            }
        }
        MPJ_TRY(offnorm2(T, dbl, N, n, partial, offv, s));
        MPJ_CUDA_TRY(cudaMemcpyAsync(hs.d, offv, sizeof(double), cudaMemcpyDeviceToHost, s));
        MPJ_CUDA_TRY(cudaMemcpyAsync(hs.u, rot, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        MPJ_CUDA_TRY(cudaStreamSynchronize(s));
        prof_flush();
        off = sqrt(hs.d[0]);
        res->sweeps += 1;
        res->rotations += (double)hs.u[0];
        if (hs.u[0] == 0) { res->status = MPJ_SUCCESS; break; }
    }
    if (res->status == MPJ_NOT_CONVERGED && std::isfinite(off) && !(off > tol_abs))
        res->status = MPJ_SUCCESS;
    res->off_final = ldexp(off, -e2);
    if (e2 != 0) MPJ_TRY(scale_pow2_f64(reinterpret_cast<double*>(T), N, N, N, -e2, s));
    return MPJ_SUCCESS;
}

template size_t twosided_workspace_bytes<float>(int, int);
template size_t twosided_workspace_bytes<double>(int, int);
template int twosided_sweeps<float>(float*, float*, int, int, int, double, double, int, int, void*,
                                    cudaStream_t, SweepResult*);
template int twosided_sweeps<double>(double*, double*, int, int, int, double, double, int, int,
                                     void*, cudaStream_t, SweepResult*);

}  // namespace mpj
