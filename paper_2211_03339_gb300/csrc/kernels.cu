// kernels.cu -- data movement, reductions and post-processing kernels of the
// pipeline (padding, norms, ||off(T)||_F, ordering of the results), plus the
// host-side workspace and error plumbing.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "internal.h"
#include "jacobi_device.cuh"

namespace mpj {

// ------------------------------------------------------------------ errors
static thread_local char g_err[512] = "";

void set_error(const char* where, cudaError_t e) {
    snprintf(g_err, sizeof(g_err), "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
}
void set_error_msg(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }
const char* last_error() { return g_err; }

// ------------------------------------------------------------------ workspace
int Workspace::acquire(void* caller, size_t caller_bytes, size_t need, cudaStream_t s) {
    stream = s;
    if (caller != nullptr) {
        if (caller_bytes < need) { set_error_msg("caller workspace smaller than required"); return MPJ_BAD_ARG; }
        ptr = caller;
        owned = false;
        return MPJ_SUCCESS;
    }
    cudaError_t e = cudaMallocAsync(&ptr, need, s);
    if (e != cudaSuccess) { set_error("cudaMallocAsync(workspace)", e); ptr = nullptr; return MPJ_CUDA_ERROR; }
    owned = true;
    return MPJ_SUCCESS;
}

Workspace::~Workspace() {
    if (owned && ptr) cudaFreeAsync(ptr, stream);
}

int SideStream::init(cudaStream_t s) {
    caller = s;
    int lo = 0, hi = 0;                                   // numerically lower = higher priority
    MPJ_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    MPJ_CUDA_TRY(cudaStreamCreateWithPriority(&main, cudaStreamNonBlocking, hi));
    MPJ_CUDA_TRY(cudaStreamCreateWithPriority(&sv, cudaStreamNonBlocking, lo));
    for (int i = 0; i < 2; ++i) {
        MPJ_CUDA_TRY(cudaEventCreateWithFlags(&solved[i], cudaEventDisableTiming));
        MPJ_CUDA_TRY(cudaEventCreateWithFlags(&vdone[i], cudaEventDisableTiming));
    }
    MPJ_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    MPJ_CUDA_TRY(cudaEventCreateWithFlags(&fin, cudaEventDisableTiming));
    MPJ_CUDA_TRY(cudaEventRecord(start, caller));         // the sweeps follow the caller's work
    MPJ_CUDA_TRY(cudaStreamWaitEvent(main, start, 0));
    MPJ_CUDA_TRY(cudaStreamWaitEvent(sv, start, 0));
    return MPJ_SUCCESS;
}

int SideStream::begin_round() {
    const int set = g & 1;
    if (pending[set] && cudaStreamWaitEvent(main, vdone[set], 0) != cudaSuccess) {
        set_error("cudaStreamWaitEvent", cudaGetLastError());
        return -1;
    }
    return set;
}

int SideStream::after_solve() {
    const int set = g & 1;
    MPJ_CUDA_TRY(cudaEventRecord(solved[set], main));
    MPJ_CUDA_TRY(cudaStreamWaitEvent(sv, solved[set], 0));
    return MPJ_SUCCESS;
}

int SideStream::after_v() {
    const int set = g & 1;
    MPJ_CUDA_TRY(cudaEventRecord(vdone[set], sv));
    pending[set] = true;
    return MPJ_SUCCESS;
}

SideStream::~SideStream() {
    if (caller != main || caller != sv) {
        for (int i = 0; i < 2; ++i)
            if (pending[i]) cudaStreamWaitEvent(caller, vdone[i], 0);
        if (main && fin && cudaEventRecord(fin, main) == cudaSuccess) cudaStreamWaitEvent(caller, fin, 0);
    }
    for (int i = 0; i < 2; ++i) {
        if (solved[i]) cudaEventDestroy(solved[i]);
        if (vdone[i]) cudaEventDestroy(vdone[i]);
    }
    if (start) cudaEventDestroy(start);
    if (fin) cudaEventDestroy(fin);
    if (main) cudaStreamDestroy(main);
    if (sv) cudaStreamDestroy(sv);
}

int HostScratch::init() {
    // one pinned block per thread, kept for the life of the process
    static thread_local char* blk = nullptr;
    if (!blk) {
        cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&blk), 64);
        if (e != cudaSuccess) { blk = nullptr; set_error("cudaMallocHost", e); return MPJ_CUDA_ERROR; }
    }
    d = reinterpret_cast<double*>(blk);
    u = reinterpret_cast<unsigned long long*>(blk + 32);
    return MPJ_SUCCESS;
}
HostScratch::~HostScratch() {}

int choose_block(int n, const mpj_options* o) {
    if (o && (o->block == 16 || o->block == 32)) return o->block;
    return n <= 256 ? 16 : 32;
}

// ------------------------------------------------------------------ per-call switches
namespace {
thread_local Knobs g_knobs;
}

const Knobs& knobs() { return g_knobs; }

KnobScope::KnobScope(const mpj_options* o) : saved(g_knobs) {
    Knobs k;
    if (o) {
        k.simt_stage1 = (o->flags & MPJ_OPT_SIMT_STAGE1) != 0;
        k.simt_sweeps = (o->flags & MPJ_OPT_SIMT_SWEEPS) != 0;
        k.fp64_products = (o->flags & MPJ_OPT_FP64_PRODUCTS) != 0;
        k.full_inner = (o->flags & MPJ_OPT_FULL_INNER) != 0;
        k.mgs_global = (o->flags & MPJ_OPT_MGS_GLOBAL) != 0;
        k.trace = (o->flags & MPJ_OPT_TRACE) != 0;
        k.fp64_solves = (o->flags & MPJ_OPT_FP64_SOLVES) != 0;
        if (o->stage1_tf32_terms == 1 || o->stage1_tf32_terms == 3) k.stage1_terms = o->stage1_tf32_terms;
    }
    g_knobs = k;
}

KnobScope::~KnobScope() { g_knobs = saved; }

// ------------------------------------------------------------------ copies
template <class Out>
__global__ void k_copy_pad(const double* __restrict__ A, int lda, int rows, int cols,
                           Out* __restrict__ T, int ldt, int Rpad, int Cpad, int identity_pad) {
    size_t total = (size_t)Rpad * Cpad;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(t % Rpad), c = (int)(t / Rpad);
        Out v;
        if (r < rows && c < cols) v = (Out)A[(size_t)r + (size_t)c * lda];
        else v = (identity_pad && r == c) ? Out(1) : Out(0);
        T[(size_t)r + (size_t)c * ldt] = v;
    }
}

static int grid_for(size_t total) {
    size_t g = (total + kThreads - 1) / kThreads;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

int copy_pad_f64(const double* A, int lda, int rows, int cols, double* T, int ldt, int Rpad,
                 int Cpad, bool identity_pad, cudaStream_t s) {
    { MPJ_PROF(PC_AUX, s);
    k_copy_pad<double><<<grid_for((size_t)Rpad * Cpad), kThreads, 0, s>>>(A, lda, rows, cols, T, ldt,
                                                                         Rpad, Cpad, identity_pad);
    }
    MPJ_LAUNCH_CHECK("k_copy_pad<double>");
    return MPJ_SUCCESS;
}
int copy_pad_f32(const double* A, int lda, int rows, int cols, float* T, int ldt, int Rpad,
                 int Cpad, bool identity_pad, cudaStream_t s) {
    { MPJ_PROF(PC_AUX, s);
    k_copy_pad<float><<<grid_for((size_t)Rpad * Cpad), kThreads, 0, s>>>(A, lda, rows, cols, T, ldt,
                                                                        Rpad, Cpad, identity_pad);
    }
    MPJ_LAUNCH_CHECK("k_copy_pad<float>");
    return MPJ_SUCCESS;
}

__global__ void k_scale_pow2(double* A, int ld, int rows, int cols, int e) {
    size_t total = (size_t)rows * cols;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(t % rows), c = (int)(t / rows);
        double* p = A + (size_t)r + (size_t)c * ld;
        *p = scalbn(*p, e);
    }
}
int scale_pow2_f64(double* A, int ld, int rows, int cols, int e, cudaStream_t s) {
    MPJ_PROF(PC_AUX, s);
    k_scale_pow2<<<grid_for((size_t)rows * cols), kThreads, 0, s>>>(A, ld, rows, cols, e);
    MPJ_LAUNCH_CHECK("k_scale_pow2");
    return MPJ_SUCCESS;
}

template <class Out>
__global__ void k_identity(Out* V, int ld, int rows, int cols) {
    size_t total = (size_t)rows * cols;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(t % rows), c = (int)(t / rows);
        V[(size_t)r + (size_t)c * ld] = (r == c) ? Out(1) : Out(0);
    }
}
int set_identity_f64(double* V, int ld, int rows, int cols, cudaStream_t s) {
    { MPJ_PROF(PC_AUX, s);
    k_identity<double><<<grid_for((size_t)rows * cols), kThreads, 0, s>>>(V, ld, rows, cols);
    }
    MPJ_LAUNCH_CHECK("k_identity<double>");
    return MPJ_SUCCESS;
}
int set_identity_f32(float* V, int ld, int rows, int cols, cudaStream_t s) {
    { MPJ_PROF(PC_AUX, s);
    k_identity<float><<<grid_for((size_t)rows * cols), kThreads, 0, s>>>(V, ld, rows, cols);
    }
    MPJ_LAUNCH_CHECK("k_identity<float>");
    return MPJ_SUCCESS;
}

__global__ void k_copy(const double* __restrict__ src, int lds, int rows, int cols,
                       double* __restrict__ dst, int ldd) {
    size_t total = (size_t)rows * cols;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(t % rows), c = (int)(t / rows);
        dst[(size_t)r + (size_t)c * ldd] = src[(size_t)r + (size_t)c * lds];
    }
}
int copy_f64(const double* src, int lds, int rows, int cols, double* dst, int ldd, cudaStream_t s) {
    { MPJ_PROF(PC_AUX, s);
    k_copy<<<grid_for((size_t)rows * cols), kThreads, 0, s>>>(src, lds, rows, cols, dst, ldd);
    }
    MPJ_LAUNCH_CHECK("k_copy");
    return MPJ_SUCCESS;
}

// ------------------------------------------------------------------ reductions
// Two-pass deterministic sum of squares: up to 1024 block partials, then one block.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;
}

template <class In, bool OFF>
__global__ void k_sumsq_partial(const In* __restrict__ A, int ld, int rows, int cols,
                                double* __restrict__ partial) {
    __shared__ double sh[32];
    double acc = 0.0;
    size_t total = (size_t)rows * cols;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(t % rows), c = (int)(t / rows);
        if (OFF && r == c) continue;
        double v = (double)A[(size_t)r + (size_t)c * ld];
        acc = fma(v, v, acc);
    }
    double b = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = b;
}

__global__ void k_sum_final(const double* __restrict__ partial, int np, double* __restrict__ out) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partial[i];
    double b = block_sum(acc, sh);
    if (threadIdx.x == 0) out[0] = b;
}

static int nblocks_reduce(size_t total) {
    size_t g = (total + kThreads - 1) / kThreads;
    if (g > 1024) g = 1024;
    if (g < 1) g = 1;
    return (int)g;
}

int sumsq_f64(const double* A, int lda, int rows, int cols, double* partial, double* out,
              cudaStream_t s) {
    int g = nblocks_reduce((size_t)rows * cols);
    { MPJ_PROF(PC_AUX, s);
    k_sumsq_partial<double, false><<<g, kThreads, 0, s>>>(A, lda, rows, cols, partial);
    }
    MPJ_LAUNCH_CHECK("k_sumsq_partial");
    { MPJ_PROF(PC_AUX, s);
    k_sum_final<<<1, kThreads, 0, s>>>(partial, g, out);
    }
    MPJ_LAUNCH_CHECK("k_sum_final");
    return MPJ_SUCCESS;
}

// out = sum_{i != j < n} T_ij^2 (the square of ||off(T)||_F)
int offnorm2(const void* T, bool is_double, int ld, int n, double* partial, double* out,
             cudaStream_t s) {
    int g = nblocks_reduce((size_t)n * n);
    if (is_double)
        { MPJ_PROF(PC_AUX, s);
        k_sumsq_partial<double, true><<<g, kThreads, 0, s>>>(static_cast<const double*>(T), ld, n, n, partial);
        }
    else
        { MPJ_PROF(PC_AUX, s);
        k_sumsq_partial<float, true><<<g, kThreads, 0, s>>>(static_cast<const float*>(T), ld, n, n, partial);
        }
    MPJ_LAUNCH_CHECK("k_sumsq_partial(off)");
    { MPJ_PROF(PC_AUX, s);
    k_sum_final<<<1, kThreads, 0, s>>>(partial, g, out);
    }
    MPJ_LAUNCH_CHECK("k_sum_final");
    return MPJ_SUCCESS;
}

// ------------------------------------------------------------------ ordering
// rank_i = #{j : key_j < key_i or (key_j == key_i and j < i)} (ascending), NaN
// treated as +inf, so the ranks always form a permutation; perm[rank_i] = i.
__global__ void k_rank(const double* __restrict__ keys, int stride, int n, int descending,
                       int* __restrict__ perm) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double ki = keys[(size_t)i * stride];
    if (ki != ki) ki = INFINITY;
    if (descending) ki = -ki;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
        double kj = keys[(size_t)j * stride];
        if (kj != kj) kj = INFINITY;
        if (descending) kj = -kj;
        rank += (kj < ki) || (kj == ki && j < i);
    }
    perm[rank] = i;
}

int rank_sort(const double* keys, int stride, int n, bool descending, int* perm, cudaStream_t s) {
    { MPJ_PROF(PC_AUX, s);
    k_rank<<<(n + 127) / 128, 128, 0, s>>>(keys, stride, n, descending ? 1 : 0, perm);
    }
    MPJ_LAUNCH_CHECK("k_rank");
    return MPJ_SUCCESS;
}

template <class In>
__global__ void k_diag(const In* __restrict__ T, int ld, int n, double* __restrict__ d) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = (double)T[(size_t)i * ld + i];
}
int diag_to_f64(const void* T, bool is_double, int ld, int n, double* d, cudaStream_t s) {
    MPJ_PROF(PC_AUX, s);
    if (is_double) k_diag<double><<<(n + 255) / 256, 256, 0, s>>>(static_cast<const double*>(T), ld, n, d);
    else           k_diag<float><<<(n + 255) / 256, 256, 0, s>>>(static_cast<const float*>(T), ld, n, d);
    MPJ_LAUNCH_CHECK("k_diag");
    return MPJ_SUCCESS;
}

__device__ __forceinline__ int clamp_idx(int p, int n) { return p < 0 ? 0 : (p >= n ? n - 1 : p); }

__global__ void k_gather_vec(const double* __restrict__ in, const int* __restrict__ perm, int n,
                             double* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[clamp_idx(perm[i], n)];
}
int gather_vec(const double* in, const int* perm, int n, double* out, cudaStream_t s) {
    { MPJ_PROF(PC_AUX, s);
    k_gather_vec<<<(n + 255) / 256, 256, 0, s>>>(in, perm, n, out);
    }
    MPJ_LAUNCH_CHECK("k_gather_vec");
    return MPJ_SUCCESS;
}

__global__ void k_gather_eig(const double* __restrict__ T, int ldt, const double* __restrict__ Vw,
                             int ldvw, const int* __restrict__ perm, int n,
                             double* __restrict__ Lambda, double* __restrict__ V, int ldv) {
    size_t total = (size_t)n * n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(t % n), c = (int)(t / n);
        int p = clamp_idx(perm[c], n);
        V[(size_t)r + (size_t)c * ldv] = Vw[(size_t)r + (size_t)p * ldvw];
        if (r == 0) Lambda[c] = T[(size_t)p * ldt + p];
    }
}
int gather_eig(const double* T, int ldt, const double* Vw, int ldvw, const int* perm, int n,
               double* Lambda, double* V, int ldv, cudaStream_t s) {
    { MPJ_PROF(PC_AUX, s);
    k_gather_eig<<<grid_for((size_t)n * n), kThreads, 0, s>>>(T, ldt, Vw, ldvw, perm, n, Lambda, V, ldv);
    }
    MPJ_LAUNCH_CHECK("k_gather_eig");
    return MPJ_SUCCESS;
}

__global__ void k_gather_z32(const float* __restrict__ V32, int ld32, const int* __restrict__ perm,
                             int n, double* __restrict__ Z, int ldz) {
    size_t total = (size_t)n * n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        int r = (int)(t % n), c = (int)(t / n);
        int p = clamp_idx(perm[c], n);
        Z[(size_t)r + (size_t)c * ldz] = (double)V32[(size_t)r + (size_t)p * ld32];
    }
}
int gather_z32(const float* V32, int ld32, const int* perm, int n, double* Z, int ldz,
               cudaStream_t s) {
    { MPJ_PROF(PC_AUX, s);
    k_gather_z32<<<grid_for((size_t)n * n), kThreads, 0, s>>>(V32, ld32, perm, n, Z, ldz);
    }
    MPJ_LAUNCH_CHECK("k_gather_z32");
    return MPJ_SUCCESS;
}

// one block per column
template <class In, bool SQRT>
__global__ void k_colnorm(const In* __restrict__ C, int ldc, int m, double* __restrict__ out) {
    __shared__ double sh[32];
    const In* col = C + (size_t)blockIdx.x * ldc;
    double acc = 0.0;
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        double v = (double)col[r];
        acc = fma(v, v, acc);
    }
    double b = block_sum(acc, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = SQRT ? sqrt(b) : b;
}
int colnorms_f64(const double* C, int ldc, int m, int n, double* nrm, cudaStream_t s) {
    { MPJ_PROF(PC_AUX, s);
    k_colnorm<double, true><<<n, kThreads, 0, s>>>(C, ldc, m, nrm);
    }
    MPJ_LAUNCH_CHECK("k_colnorm<double>");
    return MPJ_SUCCESS;
}
int colnorms2_f32(const float* C, int ldc, int m, int n, double* nrm2, cudaStream_t s) {
    { MPJ_PROF(PC_AUX, s);
    k_colnorm<float, false><<<n, kThreads, 0, s>>>(C, ldc, m, nrm2);
    }
    MPJ_LAUNCH_CHECK("k_colnorm<float>");
    return MPJ_SUCCESS;
}

// Alg. 5.2 steps 11-13: sigma_j = ||c_perm(j)||, u_j = c_perm(j) / sigma_j, v_j = v_perm(j)
__global__ void k_svd_post(const double* __restrict__ C, int ldc, const double* __restrict__ Vw,
                           int ldvw, const double* __restrict__ nrm, const int* __restrict__ perm,
                           int m, int n, double* __restrict__ Sigma, double* __restrict__ U, int ldu,
                           double* __restrict__ V, int ldv, int* __restrict__ flag) {
    int j = blockIdx.x;
    int p = clamp_idx(perm[j], n);
    double sg = nrm[p];
    double inv = sg > 0.0 ? 1.0 / sg : 0.0;
    if (threadIdx.x == 0) {
        Sigma[j] = sg;
        if (!(sg > 0.0)) atomicOr(flag, 1);
    }
    for (int r = threadIdx.x; r < m; r += blockDim.x) U[(size_t)r + (size_t)j * ldu] = C[(size_t)r + (size_t)p * ldc] * inv;
    for (int r = threadIdx.x; r < n; r += blockDim.x) V[(size_t)r + (size_t)j * ldv] = Vw[(size_t)r + (size_t)p * ldvw];
}
int svd_post(const double* C, int ldc, const double* Vw, int ldvw, const double* nrm,
             const int* perm, int m, int n, double* Sigma, double* U, int ldu, double* V,
             int ldv, int* d_flag, cudaStream_t s) {
    { MPJ_PROF(PC_AUX, s);
    k_svd_post<<<n, kThreads, 0, s>>>(C, ldc, Vw, ldvw, nrm, perm, m, n, Sigma, U, ldu, V, ldv, d_flag);
    }
    MPJ_LAUNCH_CHECK("k_svd_post");
    return MPJ_SUCCESS;
}

}  // namespace mpj
