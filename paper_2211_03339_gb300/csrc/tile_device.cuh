// tile_device.cuh -- shared-memory tile products used to apply the block
// rotations W (2b x 2b) of one parallel round to the rows and columns of a
// matrix.  256 threads; thread (ty, tx) on a 16 x 16 grid owns an RM x RM
// patch of the M x M result (RM = M/16).
#pragma once

#include <type_traits>

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

// ---------------------------------------------------------------- double-float products
// When the block rotations of a round are small (|F| <= 2^-8, the preconditioned
// sweeps), the FP64 tile products X F are formed on the FP32 pipe (about 70 times
// the FP64 rate on GB300) in double-float arithmetic: X and F are split into
// float pairs (hi + lo, 48 significant bits), every product hi*hi is made exact
// with an FMA (TwoProd), the cross terms hi*lo + lo*hi are added to the error
// term, and the sum is accumulated with Knuth's TwoSum into a float pair.  The
// relative error of X F is then ~2^-45, i.e. an absolute error below 2^-53 |X|
// when |F| <= 2^-8, at the level of the FP64 rounding of the final sum X + X F.
// The _rn intrinsics keep nvcc from contracting the transforms into FMAs.

__device__ __forceinline__ void split_df(double v, float& h, float& l) {
    h = __double2float_rn(v);
    l = __double2float_rn(v - (double)h);
}

// (h, l) = (ah, al) + (bh, bl) in double-float arithmetic (TwoSum of the high
// parts, low parts added to the error, renormalised).
__device__ __forceinline__ void add_df(float ah, float al, float bh, float bl, float& h, float& l) {
    const float s = __fadd_rn(ah, bh);
    const float bb = __fsub_rn(s, ah);
    const float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
    const float t = __fadd_rn(e, __fadd_rn(al, bl));
    h = __fadd_rn(s, t);
    l = __fsub_rn(t, __fsub_rn(h, s));
}

// Float planes of the block rotations F (row-major M x M per pair, hi plane then
// lo plane), written once per round by the block solves so that the tile
// kernels read them instead of splitting F in every tile.
__device__ __forceinline__ void store_f_split(const double* F, int LD, int M, float* out) {
    for (int t = threadIdx.x; t < M * M; t += blockDim.x) {
        const int k = t / M, c = t % M;
        float h, l;
        split_df(F[c * LD + k], h, l);
        out[t] = h;
        out[M * M + t] = l;
    }
}

// ah/al[i][j] = double-float sum_k A[k][ty*RM+i] * B[k][tx*RM+j] with the float
// planes (Ah, Al), (Bh, Bl) laid out like tile_mm's operands (ld LDSF).
template <int M, int LDSF>
__device__ __forceinline__ void tile_mm_df(const float* __restrict__ Ah, const float* __restrict__ Al,
                                           const float* __restrict__ Bh, const float* __restrict__ Bl,
                                           float (&ah)[M / 16][M / 16], float (&al)[M / 16][M / 16]) {
    constexpr int RM = M / 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RM; ++j) { ah[i][j] = 0.f; al[i][j] = 0.f; }
#pragma unroll 2
    for (int k = 0; k < M; ++k) {
        float a0[RM], a1[RM], b0[RM], b1[RM];
#pragma unroll
        for (int i = 0; i < RM; ++i) { a0[i] = Ah[k * LDSF + ty * RM + i]; a1[i] = Al[k * LDSF + ty * RM + i]; }
#pragma unroll
        for (int j = 0; j < RM; ++j) { b0[j] = Bh[k * LDSF + tx * RM + j]; b1[j] = Bl[k * LDSF + tx * RM + j]; }
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < RM; ++j) {
                float p = __fmul_rn(a0[i], b0[j]);
                float e = __fmaf_rn(a0[i], b0[j], -p);          // TwoProd: a0 b0 = p + e exactly
                e = __fmaf_rn(a0[i], b1[j], e);
                e = __fmaf_rn(a1[i], b0[j], e);
                float sh = __fadd_rn(ah[i][j], p);              // TwoSum(ah, p)
                float bb = __fsub_rn(sh, ah[i][j]);
                float er = __fadd_rn(__fsub_rn(ah[i][j], __fsub_rn(sh, bb)), __fsub_rn(p, bb));
                ah[i][j] = sh;
                al[i][j] = __fadd_rn(al[i][j], __fadd_rn(er, e));
            }
    }
}

// Split the FP64 matrix D (ld LDSD, D[k*LDSD + c]) into float planes H, L (ld LDSF).
template <int M, int LDSD, int LDSF>
__device__ __forceinline__ void split_tile(const double* D, float* H, float* L) {
    for (int t = threadIdx.x; t < M * M; t += kThreads) {
        int k = t / M, c = t % M;
        float h, l;
        split_df(D[k * LDSD + c], h, l);
        H[k * LDSF + c] = h;
        L[k * LDSF + c] = l;
    }
}

// Rows [row0, row0+M) of X restricted to the columns of pair (Ib, Jb) times
// W_b = I + F_b in delta form, with the product X F_b in double-float
// arithmetic (see tile_mm_df).  The FP64 sum X + X F_b is formed with the exact
// X, which each thread reads into registers.  smem: 4 float planes of M*LDSF.
template <int B>
__device__ void right_multiply_rows_df(double* X, size_t ldx, int nrows, int row0, int Ib, int Jb,
                                       const double* __restrict__ Fsrc, float* smf,
                                       const float* __restrict__ Fsplit = nullptr) {
    constexpr int M = 2 * B;
    constexpr int LDSF = M + 4;
    constexpr int LDS = M + SmemPad<double>::value;
    constexpr int RM = M / 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float* Xh = smf;
    float* Xl = Xh + M * LDSF;
    float* Fh = Xl + M * LDSF;
    float* Fl = Fh + M * LDSF;
    double xr[RM][RM];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RM; ++j) {
            int gr = row0 + ty * RM + i;
            xr[i][j] = gr < nrows ? X[(size_t)gr + (size_t)pair_global(tx * RM + j, Ib, Jb, B) * ldx] : 0.0;
        }
    for (int t = threadIdx.x; t < M * M; t += kThreads) {
        int r = t % M, kc = t / M;
        int gr = row0 + r;
        double v = gr < nrows ? X[(size_t)gr + (size_t)pair_global(kc, Ib, Jb, B) * ldx] : 0.0;
        split_df(v, Xh[kc * LDSF + r], Xl[kc * LDSF + r]);
        int k = t / M, c = t % M;
        if (Fsplit) {                                              // precomputed planes
            Fh[k * LDSF + c] = Fsplit[t];
            Fl[k * LDSF + c] = Fsplit[M * M + t];
        } else {
            split_df(Fsrc[t], Fh[k * LDSF + c], Fl[k * LDSF + c]); // Fsrc row-major
        }
    }
    __syncthreads();
    float ah[RM][RM], al[RM][RM];
    tile_mm_df<M, LDSF>(Xh, Xl, Fh, Fl, ah, al);
    double y[RM][RM];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RM; ++j) y[i][j] = xr[i][j] + ((double)ah[i][j] + (double)al[i][j]);
    __syncthreads();
    double* Ys = reinterpret_cast<double*>(smf);
    tile_store_colmajor<double, M, LDS>(Ys, y);
    __syncthreads();
    for (int t = threadIdx.x; t < M * M; t += kThreads) {
        int r = t % M, c = t / M;
        int gr = row0 + r;
        if (gr < nrows) X[(size_t)gr + (size_t)pair_global(c, Ib, Jb, B) * ldx] = Ys[c * LDS + r];
    }
}

// Gather the tile T[IJ_a, IJ_b] (rows from pair a, columns from pair b) into
// Xs[k*LDS + r] with 16-byte loads: each half column is b contiguous entries.
template <class Real, int B>
__device__ __forceinline__ void gather_tile(Real* Xs, const Real* __restrict__ T, int N, int Ia, int Ja,
                                            int Ib, int Jb) {
    constexpr int M = 2 * B;
    constexpr int LDS = M + SmemPad<Real>::value;
    constexpr int VEC = 16 / sizeof(Real);
    using V4 = typename std::conditional<sizeof(Real) == 8, double2, float4>::type;
    for (int t = threadIdx.x; t < M * M / VEC; t += kThreads) {
        int rv = t % (M / VEC), kc = t / (M / VEC);
        int r = rv * VEC;
        V4 v = *reinterpret_cast<const V4*>(
            T + (size_t)pair_global(r, Ia, Ja, B) + (size_t)pair_global(kc, Ib, Jb, B) * N);
        *reinterpret_cast<V4*>(Xs + kc * LDS + r) = v;
    }
}

}  // namespace mpj

