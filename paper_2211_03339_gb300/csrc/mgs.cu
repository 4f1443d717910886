// mgs.cu -- blocked modified Gram-Schmidt (Lemma 2.1; step 2 of Alg. 4.1/5.2).
//
// The columns are processed in panels of 32.  A panel is orthogonalised by
// classic column-by-column MGS:
//     r_jj = ||w_j||,  q_j = w_j / r_jj,  w_k = w_k - (q_j^T w_k) q_j  (k > j in panel)
// by ONE thread-block cluster (16 CTAs where the device runs clusters that
// large, else 8) that splits the m rows between its CTAs; each CTA keeps its
// rows of the panel in shared memory (k_mgs_panel_smem; k_mgs_panel reads them
// from global memory when they do not fit).  For each column the CTAs form
// partial inner products w_j^T w_k over their rows, exchange them through
// distributed shared memory (one cluster barrier per column, double-buffered),
// sum them in a fixed order, and update their rows.  The trailing columns then
// receive the panel's projections, W = W - Q_p (Q_p^T W), as two FP64 GEMMs
// (block MGS); for n >= 1024 the columns are first grouped in 256-column panels
// whose projections run on the tensor cores (mgs_blocked_oz).
#include <cooperative_groups.h>
#include <cmath>
#include <cstdlib>
#include <mutex>

#include "internal.h"
#include "jacobi_device.cuh"

namespace cg = cooperative_groups;

namespace mpj {

constexpr int PB = 32;        // panel width
constexpr int CL = 8;         // CTAs per cluster (portable size)

__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(kThreads)
k_mgs_panel(double* __restrict__ Q, int m, int ldq, int j0, int pb, int* __restrict__ flag) {
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    __shared__ double part[2][PB];      // this CTA's partial inner products
    __shared__ double red[PB];          // warp partials folded per column
    const int rows_per = (m + CL - 1) / CL;
    const int r0 = rank * rows_per;
    const int r1 = min(m, r0 + rows_per);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NW = kThreads / 32;
    double* P = Q + (size_t)j0 * ldq;
    for (int jj = 0; jj < pb; ++jj) {
        const int buf = jj & 1;
        const double* wj = P + (size_t)jj * ldq;
        // partial g_k = sum_rows w_j * w_k for k = jj..pb-1: warp w takes k = jj+w, jj+w+NW, ...
        for (int k = jj + warp; k < pb; k += NW) {
            const double* wk = P + (size_t)k * ldq;
            double sacc = 0.0;
            for (int r = r0 + lane; r < r1; r += 32) sacc = fma(wj[r], wk[r], sacc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
            if (lane == 0) part[buf][k] = sacc;
        }
        cluster.sync();                 // partials of this column visible cluster-wide
        if (threadIdx.x < PB) {
            int k = threadIdx.x;
            double g = 0.0;
            if (k >= jj && k < pb) {
                for (int c = 0; c < CL; ++c) {
                    double* remote = cluster.map_shared_rank(&part[buf][0], c);
                    g += remote[k];
                }
            }
            red[k] = g;
        }
        __syncthreads();
        const double rjj = sqrt(red[jj]);
        if (rjj == 0.0 || !(rjj == rjj)) {
            if (threadIdx.x == 0 && rank == 0) atomicOr(flag, 1);
        }
        const double inv = (rjj > 0.0) ? 1.0 / rjj : 0.0;
        // q_j = w_j / r_jj ; w_k -= (g_k / r_jj) q_j for k > jj
        for (int r = r0 + threadIdx.x; r < r1; r += kThreads) {
            double q = P[(size_t)jj * ldq + r] * inv;
            P[(size_t)jj * ldq + r] = q;
            for (int k = jj + 1; k < pb; ++k) {
                double rk = red[k] * inv;
                P[(size_t)k * ldq + r] = fma(-rk, q, P[(size_t)k * ldq + r]);
            }
        }
        __syncthreads();                // own rows updated before the next column's dots
    }
    cluster.sync();                     // no CTA leaves while others may read its part[]
}

// Shared-memory resident panel MGS: the same column MGS, by a cluster of 8 or
// 16 CTAs, each holding its `rows_per` rows of the 32-column panel in shared
// memory (column-major, ld rows_per; rows past m are zero) from the first
// column to the last, so every column costs only shared-memory traffic, one
// cluster barrier and the FP64 arithmetic of its dots and updates.  After the
// cluster-wide sums, warp 0 forms r_jj, 1/r_jj and the update coefficients
// -r_jk/r_jj once for the CTA.
__global__ void __launch_bounds__(kThreads)
k_mgs_panel_smem(double* __restrict__ Q, int m, int ldq, int j0, int pb, int rows_per,
                 int* __restrict__ flag) {
    extern __shared__ __align__(16) double Ps[];
    __shared__ double part[2][PB];
    __shared__ double coef[PB];
    __shared__ double sinv;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int ncl = (int)cluster.num_blocks();
    const int r0 = rank * rows_per;
    const int nr = max(0, min(m, r0 + rows_per) - r0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NW = kThreads / 32;
    double* P = Q + (size_t)j0 * ldq + r0;
    for (int t = threadIdx.x; t < pb * rows_per; t += kThreads) {
        const int k = t / rows_per, rr = t - k * rows_per;
        Ps[t] = rr < nr ? P[(size_t)k * ldq + rr] : 0.0;
    }
    __syncthreads();
    for (int jj = 0; jj < pb; ++jj) {
        const int buf = jj & 1;
        const double* wj = Ps + (size_t)jj * rows_per;
        for (int k = jj + warp; k < pb; k += NW) {
            const double* wk = Ps + (size_t)k * rows_per;
            double sacc = 0.0;
            for (int rr = lane; rr < rows_per; rr += 32) sacc = fma(wj[rr], wk[rr], sacc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
            if (lane == 0) part[buf][k] = sacc;
        }
        cluster.sync();                 // partials of this column visible cluster-wide
        if (warp == 0) {
            const int k = lane;
            double g = 0.0;
            if (k >= jj && k < pb)
                for (int c = 0; c < ncl; ++c) g += cluster.map_shared_rank(&part[buf][0], c)[k];
            const double gjj = __shfl_sync(0xffffffffu, g, jj);
            const double rjj = sqrt(gjj);
            if ((rjj == 0.0 || !(rjj == rjj)) && lane == 0 && rank == 0) atomicOr(flag, 1);
            const double inv = rjj > 0.0 ? 1.0 / rjj : 0.0;
            coef[k] = -(g * inv);
            if (lane == 0) sinv = inv;
        }
        __syncthreads();
        const double inv = sinv;
        // q_j = w_j / r_jj ; w_k -= (r_jk / r_jj) q_j for k > jj
        for (int rr = threadIdx.x; rr < rows_per; rr += kThreads) {
            const double q = Ps[(size_t)jj * rows_per + rr] * inv;
            Ps[(size_t)jj * rows_per + rr] = q;
            for (int k = jj + 1; k < pb; ++k)
                Ps[(size_t)k * rows_per + rr] = fma(coef[k], q, Ps[(size_t)k * rows_per + rr]);
        }
        __syncthreads();                // own rows updated before the next column's dots
    }
    for (int t = threadIdx.x; t < pb * rows_per; t += kThreads) {
        const int k = t / rows_per, rr = t - k * rows_per;
        if (rr < nr) P[(size_t)k * ldq + rr] = Ps[t];
    }
    cluster.sync();                     // no CTA leaves while others may read its part[]
}

constexpr size_t kPanelSmemMax = 200 * 1024;

// Cluster size for k_mgs_panel_smem on the current device: 16 CTAs when the
// device can run such a cluster with `smem` bytes each (non-portable size), else 8;
// 0 when neither fits.  Cached per device and shared-memory size class.
static int panel_cluster_size(size_t smem) {
    constexpr int kDev = 64;
    static std::mutex mu;
    static int cache[kDev][2] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDev) return 0;
    const int cls = smem > 100 * 1024 ? 1 : 0;      // sizes are probed at the class maximum
    std::lock_guard<std::mutex> lk(mu);
    if (cache[dev][cls]) return cache[dev][cls] > 0 ? cache[dev][cls] : 0;
    const size_t probe = cls ? kPanelSmemMax : 100 * 1024;
    int best = -1;
    if (cudaFuncSetAttribute(k_mgs_panel_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPanelSmemMax) ==
            cudaSuccess &&
        cudaFuncSetAttribute(k_mgs_panel_smem, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        for (int cl : {16, 8}) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = cl; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(cl); cfg.blockDim = dim3(kThreads); cfg.dynamicSmemBytes = probe;
            cfg.attrs = at; cfg.numAttrs = 1;
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, k_mgs_panel_smem, &cfg) == cudaSuccess && nclusters > 0) {
                best = cl;
                break;
            }
        }
    }
    cudaGetLastError();                 // a refused probe leaves no sticky error
    cache[dev][cls] = best;
    return best > 0 ? best : 0;
}

// One 32-column panel: the shared-memory kernel when the panel's rows fit the
// cluster's shared memory, else the global-memory kernel.
static int mgs_panel(double* Q, int m, int ldq, int j0, int pb, int* d_flag, cudaStream_t s) {
    const bool smem_off = knobs().mgs_global;
    int cl = 0;
    int rows_per = 0;
    size_t smem = 0;
    if (!smem_off) {
        for (int c : {16, 8}) {
            rows_per = (m + c - 1) / c;
            smem = sizeof(double) * (size_t)rows_per * PB;
            if (smem <= kPanelSmemMax && panel_cluster_size(smem) >= c) { cl = c; break; }
        }
    }
    if (cl) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cl; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(cl); cfg.blockDim = dim3(kThreads); cfg.dynamicSmemBytes = smem;
        cfg.stream = s; cfg.attrs = at; cfg.numAttrs = 1;
        MPJ_PROF(PC_MGS_PANEL, s);
        MPJ_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_mgs_panel_smem, Q, m, ldq, j0, pb, rows_per, d_flag));
        return MPJ_SUCCESS;
    }
    { MPJ_PROF(PC_MGS_PANEL, s);
      k_mgs_panel<<<CL, kThreads, 0, s>>>(Q, m, ldq, j0, pb, d_flag); }
    MPJ_LAUNCH_CHECK("k_mgs_panel");
    return MPJ_SUCCESS;
}

// Panel projections R = Q_p^T W (pb x rest, K = m rows): the contraction is
// long and the output small, so the rows are split across CTAs (grid.y) and
// the partial products are summed in a fixed order by k_proj_reduce.
constexpr int KSPLIT_ROWS = 256;

__global__ void __launch_bounds__(kThreads)
k_proj_partial(const double* __restrict__ Qp, const double* __restrict__ Wr, int ldq, int m,
               int pb, int rest, double* __restrict__ Rpart) {
    __shared__ __align__(16) double Qs[16][PB + 1];     // Qs[row][j]
    __shared__ __align__(16) double Ws[16][64 + 2];     // Ws[row][c]
    const int c0 = blockIdx.x * 64;
    const int r0 = blockIdx.y * KSPLIT_ROWS;
    const int r1 = min(m, r0 + KSPLIT_ROWS);
    // thread -> 2 rows (j) x 4 cols of the 32 x 64 partial
    const int tj = threadIdx.x >> 4, tc = threadIdx.x & 15;
    double acc[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    for (int rc = r0; rc < r1; rc += 16) {
        for (int t = threadIdx.x; t < 16 * PB; t += kThreads) {
            int rr = t % 16, j = t / 16;
            int gr = rc + rr;
            Qs[rr][j] = (gr < r1 && j < pb) ? Qp[(size_t)gr + (size_t)j * ldq] : 0.0;
        }
        for (int t = threadIdx.x; t < 16 * 64; t += kThreads) {
            int rr = t % 16, c = t / 16;
            int gr = rc + rr, gc = c0 + c;
            Ws[rr][c] = (gr < r1 && gc < rest) ? Wr[(size_t)gr + (size_t)gc * ldq] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < 16; ++rr) {
            double a0 = Qs[rr][tj * 2], a1 = Qs[rr][tj * 2 + 1];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                double b = Ws[rr][tc * 4 + k];
                acc[0][k] = fma(a0, b, acc[0][k]);
                acc[1][k] = fma(a1, b, acc[1][k]);
            }
        }
        __syncthreads();
    }
    double* Rp = Rpart + (size_t)blockIdx.y * PB * rest;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int j = tj * 2 + i, c = c0 + tc * 4 + k;
            if (j < pb && c < rest) Rp[(size_t)c * PB + j] = acc[i][k];
        }
}

__global__ void k_proj_reduce(const double* __restrict__ Rpart, int nsplit, int pb, int rest,
                              double* __restrict__ R) {
    size_t total = (size_t)PB * rest;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        int j = (int)(t % PB);
        double v = 0.0;
        if (j < pb)
            for (int sp = 0; sp < nsplit; ++sp) v += Rpart[(size_t)sp * PB * rest + t];
        R[t] = v;
    }
}

static int ksplit_for(int m) { return (m + KSPLIT_ROWS - 1) / KSPLIT_ROWS; }

size_t mgs_workspace_bytes(int m, int n) {
    size_t nn = (size_t)(n > 0 ? n : 1);
    return sizeof(double) * (size_t)PB * nn * (1 + (size_t)ksplit_for(m > 0 ? m : 1)) + 1024;
}

// In place: Q (m x n, ld ldq) <- orthonormal factor of the QR factorisation.
int mgs_inplace(double* Q, int m, int n, int ldq, void* work, int* d_flag, cudaStream_t s) {
    double* R = static_cast<double*>(work);      // PB x (n - j0 - pb) panel projections
    double* Rpart = R + (size_t)PB * n;          // ksplit partials of R
    const int ksplit = ksplit_for(m);
    for (int j0 = 0; j0 < n; j0 += PB) {
        int pb = (n - j0) < PB ? (n - j0) : PB;
        MPJ_TRY(mgs_panel(Q, m, ldq, j0, pb, d_flag, s));
        int rest = n - j0 - pb;
        if (rest > 0) {
            const double* Qp = Q + (size_t)j0 * ldq;
            double* Wr = Q + (size_t)(j0 + pb) * ldq;
            // R = Q_p^T W   (pb x rest), split over row slabs
            dim3 g((rest + 63) / 64, ksplit);
            { MPJ_PROF(PC_MGS_PROJ, s);
    k_proj_partial<<<g, kThreads, 0, s>>>(Qp, Wr, ldq, m, pb, rest, Rpart); }
            MPJ_LAUNCH_CHECK("k_proj_partial");
            size_t tot = (size_t)PB * rest;
            int rg = (int)((tot + kThreads - 1) / kThreads);
            { MPJ_PROF(PC_MGS_PROJ, s);
    k_proj_reduce<<<rg, kThreads, 0, s>>>(Rpart, ksplit, pb, rest, R); }
            MPJ_LAUNCH_CHECK("k_proj_reduce");
            // W = W - Q_p R
            MPJ_TRY(dgemm(false, false, m, rest, pb, -1.0, Qp, ldq, R, PB, 1.0, Wr, ldq, false, s));
        }
    }
    return MPJ_SUCCESS;
}

// Block MGS with 256-column panels: each panel is orthogonalised by the 32-column
// blocked MGS above, then the trailing columns W lose their projection on it,
// W <- W - Q_p (Q_p^T W) -- the projection (K = m) and the update (K = 256) on
// the tensor cores by exact splitting.  Panels are processed in order, each
// against the already updated W (modified Gram-Schmidt at the panel level).
// ozW: oz_operand_bytes(n, m) (columns of W); ozS: mgs_panel_oz_bytes(m, n);
// Rbuf: 256 x n doubles.
size_t mgs_panel_oz_bytes(int m, int n) {
    return oz_operand_bytes(256, m) + oz_operand_bytes(m, 256) + oz_operand_bytes(n, 256) + 1024;
}

int mgs_blocked_oz(double* Q, int m, int n, int ldq, void* work, int* d_flag, void* ozW, void* ozS,
                   double* Rbuf, cudaStream_t s) {
    constexpr int BP = 256;
    char* base = static_cast<char*>(ozS);
    OzOperand opT, opR, oR, oW;
    const size_t a1 = (oz_operand_bytes(256, m) + 255) & ~size_t(255);
    const size_t a2 = (oz_operand_bytes(m, 256) + 255) & ~size_t(255);
    MPJ_TRY(oz_operand(base, 256, m, &opT));
    MPJ_TRY(oz_operand(base + a1, m, 256, &opR));
    MPJ_TRY(oz_operand(base + a1 + a2, n, 256, &oR));
    MPJ_TRY(oz_operand(ozW, n, m, &oW));
    for (int j0 = 0; j0 < n; j0 += BP) {
        const int nb = n - j0 < BP ? n - j0 : BP;
        double* Qp = Q + (size_t)j0 * ldq;
        MPJ_TRY(mgs_inplace(Qp, m, nb, ldq, work, d_flag, s));
        const int rest = n - j0 - nb;
        if (rest <= 0) break;
        double* W = Q + (size_t)(j0 + nb) * ldq;
        opT.rows = nb; opT.K = m;
        oW.rows = rest; oW.K = m;
        MPJ_TRY(oz_slice(Qp, ldq, 1, nb, m, &opT, s));          // rows of Q_p^T (columns of Q_p)
        MPJ_TRY(oz_slice(W, ldq, 1, rest, m, &oW, s));          // columns of W
        MPJ_TRY(oz_gemm(opT, oW, 1.0, 0.0, Rbuf, nb, false, d_flag, s));   // R = Q_p^T W
        opR.rows = m; opR.K = nb;
        oR.rows = rest; oR.K = nb;
        MPJ_TRY(oz_slice(Qp, 1, ldq, m, nb, &opR, s));          // rows of Q_p
        MPJ_TRY(oz_slice(Rbuf, nb, 1, rest, nb, &oR, s));       // columns of R
        MPJ_TRY(oz_gemm(opR, oR, -1.0, 1.0, W, ldq, false, d_flag, s));    // W -= Q_p R
    }
    return MPJ_SUCCESS;
}

// ---------------------------------------------------------------- no-allocation variant
// mpj_mgs_noalloc runs the same blocked MGS as mpj_mgs but takes its scratch
// (the panel projections R and their split partials, plus the rank flag) from
// a fixed array compiled into the library instead of allocating it.  The array
// lives in device global memory on every GPU where the library's module is
// loaded, from the first call there until the process exits.  In host code
// g_mgs_noalloc_scratch is only a host-side stand-in for the device array, so
// its device address is looked up with cudaGetSymbolAddress and passed to the
// kernels.  The address belongs to the CUDA context that is current, not to
// the device ordinal, so it is looked up again on every call (a cheap query
// once the module is loaded; it allocates nothing): a cached address would be
// stale after cudaDeviceReset or under another context on the same device.
static __device__ __align__(256) double g_mgs_noalloc_scratch[MPJ_MGS_NOALLOC_MAX_SCRATCH_DOUBLES + 32];

namespace {
// Device address of the scratch array in the current context.
int noalloc_scratch(double** out) {
    void* p = nullptr;
    MPJ_CUDA_TRY(cudaGetSymbolAddress(&p, g_mgs_noalloc_scratch));
    *out = static_cast<double*>(p);
    return MPJ_SUCCESS;
}
}  // namespace

size_t mgs_noalloc_scratch_doubles(int m, int n) {
    return (size_t)PB * (size_t)n * (1 + (size_t)ksplit_for(m));
}

}  // namespace mpj

extern "C" int mpj_mgs_noalloc(const double* Z, int m, int n, int ldz, double* Q, int ldq,
                               void* stream) {
    using namespace mpj;
    if (!Z || !Q || n < 1 || m < n || ldz < m || ldq < m) { set_error_msg("invalid argument"); return MPJ_BAD_ARG; }
    if (mgs_noalloc_scratch_doubles(m, n) > (size_t)MPJ_MGS_NOALLOC_MAX_SCRATCH_DOUBLES) {
        set_error_msg("mpj_mgs_noalloc: 32*n*(1+ceil(m/256)) doubles of scratch exceed "
                      "MPJ_MGS_NOALLOC_MAX_SCRATCH_DOUBLES; use mpj_mgs with a workspace");
        return MPJ_BAD_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* scratch = nullptr;
    MPJ_TRY(noalloc_scratch(&scratch));
    int* flag = reinterpret_cast<int*>(scratch + MPJ_MGS_NOALLOC_MAX_SCRATCH_DOUBLES);
    // the array keeps the previous call's contents: the rank flag must start at zero
    MPJ_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
    MPJ_TRY(copy_f64(Z, ldz, m, n, Q, ldq, s));
    MPJ_TRY(mgs_inplace(Q, m, n, ldq, scratch, flag, s));
    int fl = 0;
    MPJ_CUDA_TRY(cudaMemcpyAsync(&fl, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    MPJ_CUDA_TRY(cudaStreamSynchronize(s));
    return fl ? MPJ_RANK_DEFICIENT : MPJ_SUCCESS;
}

