// backward.cu -- reverse-mode derivative of the symmetric eigendecomposition
// A = V diag(lambda) V^T (the differentiation pattern of the batched solver):
//
//   A_bar = V ( diag(lambda_bar) + sym(F o (V^T V_bar)) ) V^T,
//   F_ij = 1 / (lambda_j - lambda_i) for i != j (0 on the diagonal),
//   sym(X) = (X + X^T) / 2,
//
// for a batch of equal-size matrices.  Three batched FP64 GEMMs (V^T V_bar,
// V M, (V M) V^T with the upper triangle mirrored, so A_bar is exactly
// symmetric) and one fused elementwise kernel for M.  The paper has no
// counterpart: this serves training pipelines that differentiate through the
// solver.
#include <cmath>

#include "internal.h"
#include "jacobi_device.cuh"

namespace mpj {

// M = diag(lambda_bar) + sym(F o G), G = V^T V_bar (column-major n x n per matrix):
// M_ij = (G_ij - G_ji) / (2 (lambda_j - lambda_i)) for i != j; 0 for a zero gap.
__global__ void k_backward_mid(const double* __restrict__ G, const double* __restrict__ lam,
                               const double* __restrict__ glam, int n, int batch,
                               double* __restrict__ Mo) {
    const size_t nn = (size_t)n * n;
    const size_t total = nn * batch;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        size_t b = t / nn, e = t % nn;
        int i = (int)(e % n), j = (int)(e / n);
        const double* Gb = G + b * nn;
        double v;
        if (i == j) {
            v = glam ? glam[b * n + i] : 0.0;
        } else {
            double d = lam[b * n + j] - lam[b * n + i];
            v = d != 0.0 ? (Gb[(size_t)i + (size_t)j * n] - Gb[(size_t)j + (size_t)i * n]) / (2.0 * d) : 0.0;
        }
        Mo[t] = v;
    }
}

}  // namespace mpj

extern "C" {

size_t mpj_syev_backward_workspace_bytes(int n, int batch) {
    if (n < 1 || batch < 1) return 0;
    return sizeof(double) * 2 * (size_t)n * n * batch + 512;
}

int mpj_syev_backward_batched(const double* Lambda, const double* V, const double* gLambda,
                              const double* gV, int n, int batch, double* gA, void* work,
                              size_t work_bytes, void* stream) {
    using namespace mpj;
    if (!Lambda || !V || !gA || n < 1 || batch < 1) { set_error_msg("invalid argument"); return MPJ_BAD_ARG; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Workspace ws;
    size_t need = mpj_syev_backward_workspace_bytes(n, batch);
    MPJ_TRY(ws.acquire(work, work_bytes, need, s));
    const long long nn = (long long)n * n;
    double* G = static_cast<double*>(ws.ptr);        // V^T V_bar, then V M
    double* Mm = G + nn * batch;                     // M
    if (gV) {
        MPJ_TRY(dgemm_batched(true, false, n, n, n, 1.0, V, n, nn, gV, n, nn, 0.0, G, n, nn, batch,
                              false, s));
    } else {
        MPJ_CUDA_TRY(cudaMemsetAsync(G, 0, sizeof(double) * nn * batch, s));
    }
    {
        MPJ_PROF(PC_AUX, s);
        size_t total = (size_t)nn * batch;
        int grid = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
        k_backward_mid<<<grid, 256, 0, s>>>(G, Lambda, gLambda, n, batch, Mm);
    }
    MPJ_LAUNCH_CHECK("k_backward_mid");
    MPJ_TRY(dgemm_batched(false, false, n, n, n, 1.0, V, n, nn, Mm, n, nn, 0.0, G, n, nn, batch,
                          false, s));                                        // P = V M
    MPJ_TRY(dgemm_batched(false, true, n, n, n, 1.0, G, n, nn, V, n, nn, 0.0, gA, n, nn, batch,
                          true, s));                                         // A_bar = P V^T
    return MPJ_SUCCESS;
}

}  // extern "C"
