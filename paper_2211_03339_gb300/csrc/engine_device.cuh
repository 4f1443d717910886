// engine_device.cuh -- one round of the parallel-ordered block Jacobi as device
// functions, shared by the grid-wide engine (twosided.cu: one CTA per pair or
// per tile) and the batched solver (batched.cu: one CTA per matrix).
//
//   pair_solve     the 2b x 2b problem T[IJ, IJ] of block pair `pair` in round
//                  `round`: cyclic Jacobi in shared memory (Lemma 3.1, Remark 3.7),
//                  F = W - I accumulated, written back with max|F|.
//   apply_tile     off-diagonal tile T[IJ_a, IJ_b] <- W_a^T T[IJ_a, IJ_b] W_b (and its
//                  mirror), FP path or double-float path.
//   apply_slab     2b-row slab of V <- V[:, IJ_b] W_b.
#pragma once

#include "jacobi_device.cuh"
#include "tile_device.cuh"

namespace mpj {

// Tile (a, b), a < b, of the current pairing: decode from the linear tile index.
__device__ __forceinline__ void decode_tile(int tile, int K, int& a, int& b) {
    a = 0;
    int rem = tile;
    while (rem >= K - 1 - a) { rem -= K - 1 - a; ++a; }
    b = a + 1 + rem;
}

// Shared memory of the tile updates: FP path 3 (T) or 2 (V) planes of M*LDS
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

// Block-pair solve.  smem: InnerLayout<Real, 2B>::bytes.  Returns the number of
// rotations applied (all threads).  Fout: M*M row-major F of this pair.  With
// WriteBack the rotated 2b x 2b block is stored back to T; without it T is left
// as it was and the rotated block goes to Sout (M*M row-major) instead (the
// tensor-core engine applies W to the whole of T and then puts the solver's
// block, with its exact zeros, in place of the recomputed diagonal block).
template <class Real, int B, bool WriteBack = true>
__device__ int pair_solve(Real* __restrict__ T, int N, int round, int pair, Real eps, Real tau,
                          Real gate, int max_inner, Real* __restrict__ Fout, float* fmax_out,
                          unsigned char* smraw, Real* __restrict__ Sout = nullptr,
                          int cross_round = -1) {
    constexpr int M = 2 * B;
    constexpr int LD = M + 1;
    Real* S = reinterpret_cast<Real*>(smraw);
    Real* F = S + M * LD;
    Real* G = F + M * LD;
    Real* cs = G + M * LD;
    int* ip = reinterpret_cast<int*>(cs + InnerLayout<Real, M>::kRealRot);
    int* flag = ip + InnerLayout<Real, M>::kFlagOffset;
    const int nblocks = N / B;
    int I, J;
    round_pair(round, pair, nblocks, I, J);
    for (int t = threadIdx.x; t < M * M; t += blockDim.x) {
        int r = t % M, c = t / M;
        S[c * LD + r] = T[(size_t)pair_global(r, I, J, B) + (size_t)pair_global(c, I, J, B) * N];
        F[c * LD + r] = Real(0);
    }
    __syncthreads();
    int applied = inner_jacobi<Real, M>(S, F, cs, ip, eps, tau, max_inner, cross_round);
    if (WriteBack) {
        for (int t = threadIdx.x; t < M * M; t += blockDim.x) {
            int r = t % M, c = t / M;
            T[(size_t)pair_global(r, I, J, B) + (size_t)pair_global(c, I, J, B) * N] = S[c * LD + r];
        }
    } else if (Sout) {
        for (int t = threadIdx.x; t < M * M; t += blockDim.x) {
            int c = t % M, r = t / M;
            Sout[t] = S[c * LD + r];                 // row-major: Sout[r*M + c]
        }
    }
    finish_block<Real, M>(F, G, Fout, gate, flag, fmax_out);
    __syncthreads();
    return applied;
}

// Double-float version of the off-diagonal tile update (Real = double only):
// Y = X + D1 + D2 with D1 = X F_b and D2 = F_a^T (X + D1), both products in
// double-float on the FP32 pipe.  X + D1 enters the second product as a
// double-float sum (48 bits of X suffice there: it is multiplied by |F_a| <=
// 2^-8), and D1 + D2 is added to the exact FP64 X once, so the FP64 pipe only
// splits X and forms the final sum.  F comes from the precomputed float planes
// when Fsplit is given (the grid engine), else it is split here (batched).
template <int B>
__device__ void apply_tile_df(double* T, int N, const double* __restrict__ Fbuf, int a, int b,
                              int Ia, int Ja, int Ib, int Jb, float* smf,
                              const float* __restrict__ Fsplit = nullptr) {
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
    const float* Sb = Fsplit ? Fsplit + (size_t)b * 2 * M * M : nullptr;
    const float* Sa = Fsplit ? Fsplit + (size_t)a * 2 * M * M : nullptr;
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
        if (Fsplit) {
            Bh[k * LDSF + c] = Sb[t]; Bl[k * LDSF + c] = Sb[M * M + t];
            Ah[k * LDSF + c] = Sa[t]; Al[k * LDSF + c] = Sa[M * M + t];
        } else {
            split_df(Fb[t], Bh[k * LDSF + c], Bl[k * LDSF + c]);
            split_df(Fa[t], Ah[k * LDSF + c], Al[k * LDSF + c]);
        }
    }
    __syncthreads();
    float d1h[RM][RM], d1l[RM][RM];
    tile_mm_df<M, LDSF>(Xh, Xl, Bh, Bl, d1h, d1l);                // D1 = X F_b
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RM; ++j) {
            const int R = ty * RM + i, C = tx * RM + j;
            float h, l;                                           // Z = X + D1 (double-float)
            add_df(Xh[C * LDSF + R], Xl[C * LDSF + R], d1h[i][j], d1l[i][j], h, l);
            Bh[R * LDSF + C] = h;                                 // Z row-major
            Bl[R * LDSF + C] = l;
            Xh[C * LDSF + R] = d1h[i][j];                         // park D1 over X (this
            Xl[C * LDSF + R] = d1l[i][j];                         // thread's own entries)
        }
    __syncthreads();
    float d2h[RM][RM], d2l[RM][RM];
    tile_mm_df<M, LDSF>(Ah, Al, Bh, Bl, d2h, d2l);                // D2 = F_a^T Z
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RM; ++j) {
            const int R = ty * RM + i, C = tx * RM + j;
            float h, l;
            add_df(Xh[C * LDSF + R], Xl[C * LDSF + R], d2h[i][j], d2l[i][j], h, l);
            z[i][j] += (double)h + (double)l;                      // Y = X + (D1 + D2)
        }
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
    __syncthreads();
}

// Off-diagonal tile (a, b), a < b, in delta form: Z = X + X F_b, Y = Z + F_a^T Z
// = W_a^T X W_b, written with its mirror.  Skipped when both rotations are the
// identity; double-float products when both have max |F| <= df_gate (Real =
// double).  smem: ApplySmem<Real, B>::t.  Ends with a barrier.
template <class Real, int B>
__device__ void apply_tile(Real* __restrict__ T, int N, const Real* __restrict__ Fbuf,
                           const float* __restrict__ fmax, int round, int a, int b, float df_gate,
                           unsigned char* smraw, const float* __restrict__ Fsplit = nullptr) {
    constexpr int M = 2 * B;
    constexpr int LDS = M + SmemPad<Real>::value;
    constexpr int RM = M / 16;
    const int nblocks = N / B;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const float fa = fmax[a], fb = fmax[b];
    if (fa == 0.f && fb == 0.f) return;              // W_a = W_b = I: the tile is unchanged
    int Ia, Ja, Ib, Jb;
    round_pair(round, a, nblocks, Ia, Ja);
    round_pair(round, b, nblocks, Ib, Jb);
    if constexpr (sizeof(Real) == 8) {
        if (fa <= df_gate && fb <= df_gate) {
            apply_tile_df<B>(reinterpret_cast<double*>(T), N, reinterpret_cast<const double*>(Fbuf),
                             a, b, Ia, Ja, Ib, Jb, reinterpret_cast<float*>(smraw), Fsplit);
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
    __syncthreads();
}

// 2b-row slab rb of V (N x N) times the block rotation of pair b.  smem:
// ApplySmem<Real, B>::v.  Ends with a barrier.
template <class Real, int B>
__device__ void apply_slab(Real* __restrict__ V, int N, const Real* __restrict__ Fbuf,
                           const float* __restrict__ fmax, int round, int rb, int b, float df_gate,
                           unsigned char* smraw, const float* __restrict__ Fsplit = nullptr) {
    constexpr int M = 2 * B;
    constexpr int LDS = M + SmemPad<Real>::value;
    const int nblocks = N / B;
    const float fb = fmax[b];
    if (fb == 0.f) return;                           // W_b = I: the slab is unchanged
    int Ib, Jb;
    round_pair(round, b, nblocks, Ib, Jb);
    if constexpr (sizeof(Real) == 8) {
        if (fb <= df_gate) {
            right_multiply_rows_df<B>(reinterpret_cast<double*>(V), (size_t)N, N, rb * M, Ib, Jb,
                                      reinterpret_cast<const double*>(Fbuf) + (size_t)b * M * M,
                                      reinterpret_cast<float*>(smraw),
                                      Fsplit ? Fsplit + (size_t)b * 2 * M * M : nullptr);
            __syncthreads();
            return;
        }
    }
    Real* Xs = reinterpret_cast<Real*>(smraw);
    Real* Fs = Xs + M * LDS;
    load_w<Real, M, LDS>(Fs, Fbuf, b);
    right_multiply_rows<Real, B>(V, (size_t)N, N, rb * M, Ib, Jb, Xs, Fs);
    __syncthreads();
}

}  // namespace mpj
