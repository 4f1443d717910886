// gemm64.cu -- FP64 GEMM for the congruence T = Q^T (A Q) (step 3 of Alg. 4.1),
// C = A Q (step 3 of Alg. 5.2) and the panel projections of the blocked MGS.
//
// 64 x 64 output tile per CTA, 16-deep K slices staged through shared memory,
// 256 threads with a 4 x 4 register patch each (DFMA).  On GB300 the FP64 pipe
// (about 1 TFLOP/s) is the bound of this kernel by a wide margin: at 64 x 64 x 16
// per slice a CTA moves 16 KB for 65,536 FMAs.
#include "internal.h"
#include "jacobi_device.cuh"

namespace mpj {

constexpr int GT = 64;   // tile edge
constexpr int GK = 16;   // K slice

template <bool TA, bool TB>
__global__ void __launch_bounds__(kThreads)
k_dgemm(int M, int N, int K, double alpha, const double* __restrict__ A, int lda,
        const double* __restrict__ B, int ldb, double beta, double* __restrict__ C, int ldc,
        int upper_mirror, long long sA, long long sB, long long sC) {
    const int bm = blockIdx.x, bn = blockIdx.y;
    A += (size_t)blockIdx.z * sA;                     // batch (grid.z) strides
    B += (size_t)blockIdx.z * sB;
    C += (size_t)blockIdx.z * sC;
    if (upper_mirror && bm > bn) return;
    __shared__ __align__(16) double As[GK][GT + 2];   // As[k][m] = op(A)[m][k]
    __shared__ __align__(16) double Bs[GK][GT + 2];   // Bs[k][n] = op(B)[k][n]
    const int m0 = bm * GT, n0 = bn * GT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < K; k0 += GK) {
        for (int t = threadIdx.x; t < GT * GK; t += kThreads) {
            int mm, kk;
            if (!TA) { mm = t % GT; kk = t / GT; } else { kk = t % GK; mm = t / GK; }
            int gm = m0 + mm, gk = k0 + kk;
            double v = 0.0;
            if (gm < M && gk < K) v = TA ? A[(size_t)gk + (size_t)gm * lda] : A[(size_t)gm + (size_t)gk * lda];
            As[kk][mm] = v;
        }
        for (int t = threadIdx.x; t < GT * GK; t += kThreads) {
            int nn, kk;
            if (!TB) { kk = t % GK; nn = t / GK; } else { nn = t % GT; kk = t / GT; }
            int gn = n0 + nn, gk = k0 + kk;
            double v = 0.0;
            if (gn < N && gk < K) v = TB ? B[(size_t)gn + (size_t)gk * ldb] : B[(size_t)gk + (size_t)gn * ldb];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    // epilogue straight from registers: each thread writes 4 contiguous rows of 4 columns
#pragma unroll
    for (int j = 0; j < 4; ++j) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
            if (gm >= M || gn >= N) continue;
            if (upper_mirror && gm > gn) continue;
            double v = alpha * acc[i][j];
            size_t idx = (size_t)gm + (size_t)gn * ldc;
            if (beta != 0.0) v += beta * C[idx];
            C[idx] = v;
            if (upper_mirror && gm != gn) C[(size_t)gn + (size_t)gm * ldc] = v;
        }
    }
}

int dgemm_batched(bool transA, bool transB, int M, int N, int K, double alpha, const double* A,
                  int lda, long long sA, const double* B, int ldb, long long sB, double beta,
                  double* C, int ldc, long long sC, int batch, bool upper_mirror, cudaStream_t s) {
    if (M <= 0 || N <= 0 || batch <= 0) return MPJ_SUCCESS;
    dim3 grid((M + GT - 1) / GT, (N + GT - 1) / GT, batch);
    int um = upper_mirror ? 1 : 0;
    MPJ_PROF(PC_DGEMM, s);
    if (!transA && !transB)
        k_dgemm<false, false><<<grid, kThreads, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, um, sA, sB, sC);
    else if (transA && !transB)
        k_dgemm<true, false><<<grid, kThreads, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, um, sA, sB, sC);
    else if (!transA && transB)
        k_dgemm<false, true><<<grid, kThreads, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, um, sA, sB, sC);
    else
        k_dgemm<true, true><<<grid, kThreads, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, um, sA, sB, sC);
    MPJ_LAUNCH_CHECK("k_dgemm");
    return MPJ_SUCCESS;
}

int dgemm(bool transA, bool transB, int M, int N, int K, double alpha, const double* A, int lda,
          const double* B, int ldb, double beta, double* C, int ldc, bool upper_mirror,
          cudaStream_t s) {
    return dgemm_batched(transA, transB, M, N, K, alpha, A, lda, 0, B, ldb, 0, beta, C, ldc, 0, 1,
                         upper_mirror, s);
}

}  // namespace mpj
