// tile_device.cuh -- shared-memory tile products used to apply the block
// rotations W (2b x 2b) of one parallel round to the rows and columns of a
// matrix.  256 threads; thread (ty, tx) on a 16 x 16 grid owns an RM x RM
// patch of the M x M result (RM = M/16).
#pragma once

#include "jacobi_device.cuh"

namespace mpj {

template <class Real> struct SmemPad { static constexpr int value = 4; };
template <> struct SmemPad<double> { static constexpr int value = 2; };

// acc[i][j] = sum_k A[k*LDS + ty*RM + i] * B[k*LDS + tx*RM + j]
template <class Real, int M, int LDS>
__device__ __forceinline__ void tile_mm(const Real* __restrict__ A, const Real* __restrict__ B,
                                        Real (&acc)[M / 16][M / 16]) {
    constexpr int RM = M / 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RM; ++j) acc[i][j] = Real(0);
#pragma unroll 4
    for (int k = 0; k < M; ++k) {
        Real a[RM], b[RM];
#pragma unroll
        for (int i = 0; i < RM; ++i) a[i] = A[k * LDS + ty * RM + i];
#pragma unroll
        for (int j = 0; j < RM; ++j) b[j] = B[k * LDS + tx * RM + j];
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < RM; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
}

// Store acc (rows ty*RM+i, cols tx*RM+j) row-major: D[r*LDS + c].
template <class Real, int M, int LDS>
__device__ __forceinline__ void tile_store_rowmajor(Real* D, const Real (&acc)[M / 16][M / 16]) {
    constexpr int RM = M / 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RM; ++j) D[(ty * RM + i) * LDS + tx * RM + j] = acc[i][j];
}

// Store acc column-major: D[c*LDS + r].
template <class Real, int M, int LDS>
__device__ __forceinline__ void tile_store_colmajor(Real* D, const Real (&acc)[M / 16][M / 16]) {
    constexpr int RM = M / 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RM; ++j) D[(tx * RM + j) * LDS + ty * RM + i] = acc[i][j];
}

// Load the block rotation W of pair `pair` (stored row-major M x M in Wbuf)
// into Ws[k*LDS + c] = W[k][c].
template <class Real, int M, int LDS>
__device__ __forceinline__ void load_w(Real* Ws, const Real* __restrict__ Wbuf, int pair) {
    const Real* src = Wbuf + (size_t)pair * M * M;
    for (int t = threadIdx.x; t < M * M; t += kThreads) {
        int k = t / M, c = t % M;
        Ws[k * LDS + c] = src[t];
    }
}

// Rows [row0, row0+M) of X (ld ldx, valid rows < nrows) restricted to the
// columns of block pair (Ib, Jb) are multiplied on the right by W_b = I + F_b,
// in place, in delta form: X <- X + X F_b (the rounding of the update is then
// relative to |X F_b|, plus one rounding of the sum).
// Xs: M*LDS scratch; Fs must already hold F_b (row-major) and be synced.
template <class Real, int B>
__device__ void right_multiply_rows(Real* X, size_t ldx, int nrows, int row0, int Ib, int Jb,
                                    Real* Xs, const Real* Fs) {
    constexpr int M = 2 * B;
    constexpr int LDS = M + SmemPad<Real>::value;
    constexpr int RM = M / 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int t = threadIdx.x; t < M * M; t += kThreads) {
        int r = t % M, kc = t / M;
        int gr = row0 + r;
        Real v = Real(0);
        if (gr < nrows) v = X[(size_t)gr + (size_t)pair_global(kc, Ib, Jb, B) * ldx];
        Xs[kc * LDS + r] = v;                     // Xs[k][r] = X[r][k]
    }
    __syncthreads();
    Real acc[M / 16][M / 16];
    tile_mm<Real, M, LDS>(Xs, Fs, acc);           // (X F)[r][c]
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RM; ++j) acc[i][j] += Xs[(tx * RM + j) * LDS + ty * RM + i];
    __syncthreads();
    tile_store_colmajor<Real, M, LDS>(Xs, acc);   // Xs[c*LDS + r] = Y[r][c]
    __syncthreads();
    for (int t = threadIdx.x; t < M * M; t += kThreads) {
        int r = t % M, c = t / M;
        int gr = row0 + r;
        if (gr < nrows) X[(size_t)gr + (size_t)pair_global(c, Ib, Jb, B) * ldx] = Xs[c * LDS + r];
    }
}

}  // namespace mpj
