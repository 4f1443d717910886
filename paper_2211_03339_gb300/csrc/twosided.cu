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
#include <cmath>
#include <cstdio>

#include "internal.h"
#include "jacobi_device.cuh"
#include "tile_device.cuh"

namespace mpj {

template <class Real, int B>
__global__ void __launch_bounds__(kThreads)
k_solve2(Real* __restrict__ T, int N, Real* __restrict__ Fbuf, int round, Real eps, Real tau,
         Real gate, int max_inner, unsigned long long* __restrict__ rot_counter) {
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
    for (int t = threadIdx.x; t < M * M; t += kThreads) {
        int r = t % M, c = t / M;
        S[c * LD + r] = T[(size_t)pair_global(r, I, J, B) + (size_t)pair_global(c, I, J, B) * N];
        F[c * LD + r] = Real(0);
    }
    __syncthreads();
    int applied = inner_jacobi<Real, M>(S, F, cs, ip, eps, tau, max_inner);
    for (int t = threadIdx.x; t < M * M; t += kThreads) {
        int r = t % M, c = t / M;
        T[(size_t)pair_global(r, I, J, B) + (size_t)pair_global(c, I, J, B) * N] = S[c * LD + r];
    }
    finish_block<Real, M>(F, G, Fbuf + (size_t)blockIdx.x * M * M, gate, flag);
    if (threadIdx.x == 0 && applied) atomicAdd(rot_counter, (unsigned long long)applied);
}

// Off-diagonal tiles in delta form: Z = X + X F_b, Y = Z + F_a^T Z = W_a^T X W_b.
template <class Real, int B>
__global__ void __launch_bounds__(kThreads)
k_apply2(Real* __restrict__ T, Real* __restrict__ V, int N, const Real* __restrict__ Fbuf,
         int round, int n_ttiles) {
    constexpr int M = 2 * B;
    constexpr int LDS = M + SmemPad<Real>::value;
    constexpr int RM = M / 16;
    extern __shared__ __align__(16) unsigned char smraw[];
    Real* Xs = reinterpret_cast<Real*>(smraw);
    Real* Fb = Xs + M * LDS;
    Real* Fa = Fb + M * LDS;
    Real* Tm = Fa + M * LDS;
    const int nblocks = N / B;
    const int K = nblocks / 2;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int tile = blockIdx.x;
    if (tile < n_ttiles) {
        // off-diagonal tile (a, b), a < b, of the current pairing
        int a = 0, rem = tile;
        while (rem >= K - 1 - a) { rem -= K - 1 - a; ++a; }
        int b = a + 1 + rem;
        int Ia, Ja, Ib, Jb;
        round_pair(round, a, nblocks, Ia, Ja);
        round_pair(round, b, nblocks, Ib, Jb);
        for (int t = threadIdx.x; t < M * M; t += kThreads) {
            int r = t % M, kc = t / M;
            Xs[kc * LDS + r] =
                T[(size_t)pair_global(r, Ia, Ja, B) + (size_t)pair_global(kc, Ib, Jb, B) * N];
        }
        load_w<Real, M, LDS>(Fb, Fbuf, b);
        load_w<Real, M, LDS>(Fa, Fbuf, a);
        __syncthreads();
        Real acc[M / 16][M / 16];
        tile_mm<Real, M, LDS>(Xs, Fb, acc);              // (X F_b)[r][c]
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < RM; ++j) acc[i][j] += Xs[(tx * RM + j) * LDS + ty * RM + i];
        tile_store_rowmajor<Real, M, LDS>(Tm, acc);      // Z row-major
        __syncthreads();
        tile_mm<Real, M, LDS>(Fa, Tm, acc);              // (F_a^T Z)[r][c]
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < RM; ++j) acc[i][j] += Tm[(ty * RM + i) * LDS + tx * RM + j];
        __syncthreads();
        tile_store_colmajor<Real, M, LDS>(Xs, acc);      // Xs[c*LDS + r]
        tile_store_rowmajor<Real, M, LDS>(Tm, acc);      // Tm[r*LDS + c]
        __syncthreads();
        for (int t = threadIdx.x; t < M * M; t += kThreads) {
            int r = t % M, c = t / M;
            T[(size_t)pair_global(r, Ia, Ja, B) + (size_t)pair_global(c, Ib, Jb, B) * N] =
                Xs[c * LDS + r];
            int c2 = t % M, r2 = t / M;                  // mirrored tile, coalesced in c2
            T[(size_t)pair_global(c2, Ib, Jb, B) + (size_t)pair_global(r2, Ia, Ja, B) * N] =
                Tm[r2 * LDS + c2];
        }
    } else {
        int t2 = tile - n_ttiles;
        int rb = t2 / K, b = t2 % K;
        int Ib, Jb;
        round_pair(round, b, nblocks, Ib, Jb);
        load_w<Real, M, LDS>(Fb, Fbuf, b);
        right_multiply_rows<Real, B>(V, (size_t)N, N, rb * M, Ib, Jb, Xs, Fb);
    }
}

template <class Real>
size_t twosided_workspace_bytes(int N, int B) {
    Arena a;
    int K = N / (2 * B), M = 2 * B;
    a.take<Real>((size_t)K * M * M);
    a.take<double>(1024);
    a.take<double>(4);
    a.take<unsigned long long>(4);
    return a.used + 256;
}

template <class Real, int B>
static int configure_twosided() {
    constexpr int M = 2 * B;
    const size_t sm_solve = InnerLayout<Real, M>::bytes;
    const size_t sm_apply = sizeof(Real) * 4 * M * (M + SmemPad<Real>::value);
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_solve2<Real, B>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_solve));
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_apply2<Real, B>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_apply));
    return MPJ_SUCCESS;
}

template <class Real, int B>
static int launch_round(Real* T, Real* V, int N, Real* Wbuf, int r, Real eps, Real tau, Real gate,
                        int max_inner, unsigned long long* rot, cudaStream_t s) {
    constexpr int M = 2 * B;
    const int K = N / M;
    const size_t sm_solve = InnerLayout<Real, M>::bytes;
    const size_t sm_apply = sizeof(Real) * 4 * M * (M + SmemPad<Real>::value);
    { MPJ_PROF(sizeof(Real) == 8 ? PC_SOLVE2_F64 : PC_SOLVE2_F32, s);
    k_solve2<Real, B><<<K, kThreads, sm_solve, s>>>(T, N, Wbuf, r, eps, tau, gate, max_inner, rot); }
    MPJ_LAUNCH_CHECK("k_solve2");
    int n_ttiles = K * (K - 1) / 2;
    int n_vtiles = (N / M) * K;
    if (n_ttiles + n_vtiles > 0) {
        { MPJ_PROF(sizeof(Real) == 8 ? PC_APPLY2_F64 : PC_APPLY2_F32, s);
    k_apply2<Real, B><<<n_ttiles + n_vtiles, kThreads, sm_apply, s>>>(T, V, N, Wbuf, r, n_ttiles); }
        MPJ_LAUNCH_CHECK("k_apply2");
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
    double* partial = ar.take<double>(1024);
    double* offv = ar.take<double>(4);
    unsigned long long* rot = ar.take<unsigned long long>(4);
    if (!Wbuf || !partial || !offv || !rot) { set_error_msg("workspace too small"); return MPJ_BAD_ARG; }
    HostScratch hs;
    MPJ_TRY(hs.init());
    const bool dbl = sizeof(Real) == 8;
    if (B == 16) { MPJ_TRY((configure_twosided<Real, 16>())); }
    else         { MPJ_TRY((configure_twosided<Real, 32>())); }

    MPJ_TRY(offnorm2(T, dbl, N, n, partial, offv, s));
    MPJ_CUDA_TRY(cudaMemcpyAsync(hs.d, offv, sizeof(double), cudaMemcpyDeviceToHost, s));
    MPJ_CUDA_TRY(cudaStreamSynchronize(s));
    double off = sqrt(hs.d[0]);
    res->off_initial = off;
    res->sweeps = 0;
    res->rotations = 0;
    res->status = MPJ_NOT_CONVERGED;
    const int rounds = 2 * K - 1;
    // entries below tau cannot keep ||off(T)||_F above tol_abs once all are below it
    const Real tau = (Real)(tol_abs / (double)N);
    const Real gate = (Real)(dbl ? 1.0 / 67108864.0 : 1.0 / 4096.0);   // 2^-26 / 2^-12
    while (res->sweeps < max_sweeps) {
        if (!std::isfinite(off)) { res->status = MPJ_NONFINITE_INPUT; break; }
        if (!(off > tol_abs)) { res->status = MPJ_SUCCESS; break; }
        MPJ_CUDA_TRY(cudaMemsetAsync(rot, 0, sizeof(unsigned long long), s));
        for (int r = 0; r < rounds; ++r) {
            if (B == 16) {
                MPJ_TRY((launch_round<Real, 16>(T, V, N, Wbuf, r, (Real)eps_skip, tau, gate, max_inner,
                                                rot, s)));
            } else {
                MPJ_TRY((launch_round<Real, 32>(T, V, N, Wbuf, r, (Real)eps_skip, tau, gate, max_inner,
                                                rot, s)));
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
    res->off_final = off;
    return MPJ_SUCCESS;
}

template size_t twosided_workspace_bytes<float>(int, int);
template size_t twosided_workspace_bytes<double>(int, int);
template int twosided_sweeps<float>(float*, float*, int, int, int, double, double, int, int, void*,
                                    cudaStream_t, SweepResult*);
template int twosided_sweeps<double>(double*, double*, int, int, int, double, double, int, int,
                                     void*, cudaStream_t, SweepResult*);

}  // namespace mpj
