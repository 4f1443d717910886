// batched.cu -- many independent small eigendecompositions in one persistent
// launch (Algorithm 4.1 or Algorithm 3.2 per matrix, n <= 256).
//
// One CTA solves one matrix at a time and takes the next one from an atomic
// work counter (jobs ordered by decreasing n^3, so the long solves start
// first).  Every step runs inside the CTA with the same device functions as
// the single-matrix engine (engine_device.cuh): block size b chosen by n, a
// matrix with n <= 2b is one block pair and is diagonalised by the inner solve
// alone; larger ones run the round-robin block sweeps over a per-CTA slot of
// global scratch.  A plan (sizes, job order, scratch) is built once on the host;
// a run is one memset and one kernel on the caller's stream, with no host
// synchronisation, so it can be captured in a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "engine_device.cuh"
#include "internal.h"

namespace mpj {

constexpr int kNmax = 256;          // largest order of the batched solver
constexpr int kBatchThreads = kThreads;

struct BatchJob {
    long long a_off;                // offset of A_i, V_i (n_i^2 each, column-major, ld n_i)
    long long l_off;                // offset of Lambda_i
    int n;
    int idx;                        // index in the caller's order
};

// ------------------------------------------------------------------ CTA helpers
// Block-wide sum (all threads get the result).  sh: 32 doubles.
__device__ double cta_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    int nw = blockDim.x >> 5;
    for (int w = 0; w < nw; ++w) r += sh[w];          // fixed order: identical in all threads
    __syncthreads();
    return r;
}

// sum_{i != j < n} T_ij^2 and, with diag, sum over all entries
template <class Real>
__device__ double cta_sumsq(const Real* T, int ld, int n, bool off_only, double* sh) {
    double acc = 0.0;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        int r = t % n, c = t / n;
        if (off_only && r == c) continue;
        double v = (double)T[(size_t)r + (size_t)c * ld];
        acc = fma(v, v, acc);
    }
    return cta_sum(acc, sh);
}

// C (m x nc, ldc) = op(A) B with op(A) = A (m x k) or A^T (A k x m); when
// upper_mirror, only entries with row <= col are computed and mirrored.
// FP64, 64 x 64 output tiles, 16-deep slices through smem (2 x 16 x 66 doubles).
__device__ void cta_dgemm(bool transA, int m, int nc, int k, const double* A, int lda,
                          const double* Bm, int ldb, double* C, int ldc, bool upper_mirror,
                          double* sm) {
    double (*As)[66] = reinterpret_cast<double (*)[66]>(sm);
    double (*Bs)[66] = reinterpret_cast<double (*)[66]>(sm + 16 * 66);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int m0 = 0; m0 < m; m0 += 64) {
        for (int n0 = 0; n0 < nc; n0 += 64) {
            if (upper_mirror && m0 > n0) continue;
            double acc[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
            for (int k0 = 0; k0 < k; k0 += 16) {
                for (int t = threadIdx.x; t < 64 * 16; t += blockDim.x) {
                    int mm, kk;
                    if (!transA) { mm = t % 64; kk = t / 64; } else { kk = t % 16; mm = t / 16; }
                    int gm = m0 + mm, gk = k0 + kk;
                    double v = 0.0;
                    if (gm < m && gk < k) v = transA ? A[(size_t)gk + (size_t)gm * lda] : A[(size_t)gm + (size_t)gk * lda];
                    As[kk][mm] = v;
                    int kb = t % 16, nn = t / 16;
                    int gn = n0 + nn, gkb = k0 + kb;
                    Bs[kb][nn] = (gn < nc && gkb < k) ? Bm[(size_t)gkb + (size_t)gn * ldb] : 0.0;
                }
                __syncthreads();
#pragma unroll
                for (int kk = 0; kk < 16; ++kk) {
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
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
                    if (gm >= m || gn >= nc) continue;
                    if (upper_mirror && gm > gn) continue;
                    C[(size_t)gm + (size_t)gn * ldc] = acc[i][j];
                    if (upper_mirror && gm != gn) C[(size_t)gn + (size_t)gm * ldc] = acc[i][j];
                }
            __syncthreads();
        }
    }
}

// Modified Gram-Schmidt (Lemma 2.1) in place on the n x n matrix Q (ld ldq):
// for j: g_k = w_j^T w_k (k >= j), w_k -= (g_k / g_j) w_j (k > j), w_j /= sqrt(g_j).
// g: n doubles of smem.  Returns 1 if some r_jj == 0 (all threads).
__device__ int cta_mgs(double* Q, int ldq, int n, double* g) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    int bad = 0;
    for (int j = 0; j < n; ++j) {
        const double* wj = Q + (size_t)j * ldq;
        for (int k = j + warp; k < n; k += nw) {
            const double* wk = Q + (size_t)k * ldq;
            double s = 0.0;
            for (int r = lane; r < n; r += 32) s = fma(wj[r], wk[r], s);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) g[k] = s;
        }
        __syncthreads();
        const double gj = g[j];
        if (!(gj > 0.0)) bad = 1;
        const double inv2 = gj > 0.0 ? 1.0 / gj : 0.0;
        const int cols = n - j - 1;
        for (int t = threadIdx.x; t < n * cols; t += blockDim.x) {
            int r = t % n, k = j + 1 + t / n;
            Q[(size_t)r + (size_t)k * ldq] = fma(-(g[k] * inv2), wj[r], Q[(size_t)r + (size_t)k * ldq]);
        }
        __syncthreads();
        const double inv = gj > 0.0 ? 1.0 / sqrt(gj) : 0.0;
        for (int r = threadIdx.x; r < n; r += blockDim.x) Q[(size_t)r + (size_t)j * ldq] *= inv;
        __syncthreads();
    }
    return bad;
}

// perm[k] = index of the k-th smallest diagonal entry of T (ties by index).
template <class Real>
__device__ void cta_rank_diag(const Real* T, int ld, int n, int* perm) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double di = (double)T[(size_t)i * ld + i];
        if (di != di) di = INFINITY;
        int rank = 0;
        for (int j = 0; j < n; ++j) {
            double dj = (double)T[(size_t)j * ld + j];
            if (dj != dj) dj = INFINITY;
            rank += (dj < di) || (dj == di && j < i);
        }
        perm[rank] = i;
    }
    __syncthreads();
}

// Parallel-ordered block Jacobi sweeps of one matrix by one CTA (the same
// rounds as twosided_sweeps, executed pair after pair and tile after tile).
// T, V: N x N (ld N) in the CTA's scratch slot; Fs: K M^2 Real; fmax: K floats.
// A matrix that is a single block pair (K == 1) is diagonalised by the inner
// solve alone (inner sweeps until no rotation).  Returns the status; *sweeps
// receives the number of (outer) sweeps.
template <class Real, int B>
__device__ int cta_block_jacobi(Real* T, Real* V, int N, int n, double tol_abs, Real eps,
                                int max_sweeps, int max_inner, Real* Fs, float* fmax,
                                unsigned char* sm, double* red, int* sweeps) {
    constexpr int M = 2 * B;
    const int K = N / M;
    const int rounds = 2 * K - 1;
    const int inner = (K == 1) ? 4 * max_sweeps : max_inner;
    const Real tau = (Real)(tol_abs / (double)N);
    const Real gate = (Real)(sizeof(Real) == 8 ? 1.0 / 64.0 : 1.0 / 4096.0);
    const float df_gate = sizeof(Real) == 8 ? 1.0f / 256.0f : -1.0f;
    int status = MPJ_NOT_CONVERGED;
    int sw = 0;
    double off = sqrt(cta_sumsq(T, N, n, true, red));
    while (sw < max_sweeps) {
        if (!(off > tol_abs)) { status = MPJ_SUCCESS; break; }
        int rot = 0;
        for (int r = 0; r < rounds; ++r) {
            for (int a = 0; a < K; ++a)
                rot += pair_solve<Real, B>(T, N, r, a, eps, tau, gate, inner, Fs + (size_t)a * M * M,
                                           fmax + a, sm);
            for (int t = 0; t < K * (K - 1) / 2; ++t) {
                int a, b;
                decode_tile(t, K, a, b);
                apply_tile<Real, B>(T, N, Fs, fmax, r, a, b, df_gate, sm);
            }
            for (int rb = 0; rb < N / M; ++rb)
                for (int b = 0; b < K; ++b) apply_slab<Real, B>(V, N, Fs, fmax, r, rb, b, df_gate, sm);
        }
        ++sw;
        off = sqrt(cta_sumsq(T, N, n, true, red));
        if (rot == 0) { status = MPJ_SUCCESS; break; }
    }
    if (status == MPJ_NOT_CONVERGED && !(off > tol_abs)) status = MPJ_SUCCESS;
    *sweeps = sw;
    return status;
}

// Scratch slot of one CTA (Nmax = 256): T, V, Q, W (FP64), T32, V32 (FP32),
// block rotations (K M^2 doubles, also used as floats) and max|F| per pair.
struct Slot {
    double *T, *V, *Q, *W, *F;
    float *T32, *V32, *fmax;
    __device__ Slot(char* base) {
        const size_t NN = (size_t)kNmax * kNmax;
        T = reinterpret_cast<double*>(base);
        V = T + NN;
        Q = V + NN;
        W = Q + NN;
        F = W + NN;                                   // 4 x 64 x 64 doubles
        T32 = reinterpret_cast<float*>(F + 4 * 64 * 64);
        V32 = T32 + NN;
        fmax = V32 + NN;                              // 64 floats
    }
    static constexpr size_t bytes =
        sizeof(double) * ((size_t)4 * kNmax * kNmax + 4 * 64 * 64) +
        sizeof(float) * ((size_t)2 * kNmax * kNmax + 64);
};

// Entries of the padded working copies: A (n x n, ld n) into X (N x N, ld N),
// zero outside, identity on the padded diagonal when id_pad.
template <class Out>
__device__ void cta_pad(const double* A, int lda, int rows, int cols, Out* X, int N, bool id_pad) {
    for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
        int r = t % N, c = t / N;
        Out v;
        if (r < rows && c < cols) v = (Out)A[(size_t)r + (size_t)c * lda];
        else v = (id_pad && r == c) ? Out(1) : Out(0);
        X[(size_t)r + (size_t)c * N] = v;
    }
    __syncthreads();
}

template <class Real>
__device__ void cta_identity(Real* X, int N) {
    for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
        int r = t % N, c = t / N;
        X[(size_t)r + (size_t)c * N] = (r == c) ? Real(1) : Real(0);
    }
    __syncthreads();
}

template <class Real>
__device__ void cta_scale(Real* X, int N, int e) {
    if (e == 0) return;
    for (int t = threadIdx.x; t < N * N; t += blockDim.x) X[t] = scalbn(X[t], e);
    __syncthreads();
}

struct BatchArgs {
    const BatchJob* jobs;
    int count;
    unsigned int* counter;
    const double* A;
    double* Lambda;
    double* V;
    int* status;
    int* sweeps;
    char* slots;
    size_t slot_bytes;
    int method;                 // 0 plain (Alg. 3.2), 1 preconditioned (Alg. 4.1)
    double tol;                 // relative; <= 0: n * 2^-53 per matrix
    double tol1;                // step-1 relative tolerance
    int max_sweeps, max_sweeps1, max_inner, block_large;
};

constexpr double kUb = 1.1102230246251565e-16;    // 2^-53
constexpr double kUpsb = 5.9604644775390625e-08;  // 2^-24

// One matrix of the batch with block size B (N = n rounded up to 2B).
template <int B>
__device__ void solve_job(const BatchArgs& a, const BatchJob& job, Slot& sl, unsigned char* sm,
                          double* red, int* perm, double* g) {
    const int n = job.n;
    int N = (n + 2 * B - 1) / (2 * B) * (2 * B);
    const double* A = a.A + job.a_off;
    const double normA = sqrt(cta_sumsq(A, n, n, false, red));
    double tol_abs = (a.tol > 0 ? a.tol : n * kUb) * normA;
    int status = MPJ_SUCCESS, sw1 = 0, sw = 0;
    if (a.method == 1) {
        // step 1: FP32 block Jacobi of fl32(A); Z = eigenvectors by ascending eigenvalue
        cta_pad<float>(A, n, n, n, sl.T32, N, false);
        cta_identity<float>(sl.V32, N);
        cta_block_jacobi<float, B>(sl.T32, sl.V32, N, n, a.tol1 * normA, (float)kUpsb, a.max_sweeps1,
                                   a.max_inner, reinterpret_cast<float*>(sl.F), sl.fmax, sm, red, &sw1);
        cta_rank_diag<float>(sl.T32, N, n, perm);
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            int r = t % n, k = t / n;
            sl.Q[(size_t)r + (size_t)k * N] = (double)sl.V32[(size_t)r + (size_t)perm[k] * N];
        }
        __syncthreads();
        // step 2: Q = MGS(Z)
        if (cta_mgs(sl.Q, N, n, g)) status = MPJ_RANK_DEFICIENT;
        // step 3: T = Q^T (A Q), P = Q
        cta_dgemm(false, n, n, n, A, n, sl.Q, N, sl.W, N, false, reinterpret_cast<double*>(sm));
        cta_pad<double>(nullptr, 0, 0, 0, sl.T, N, false);
        cta_dgemm(true, n, n, n, sl.Q, N, sl.W, N, sl.T, N, true, reinterpret_cast<double*>(sm));
        __syncthreads();
        cta_pad<double>(sl.Q, N, n, n, sl.V, N, true);
    } else {
        cta_pad<double>(A, n, n, n, sl.T, N, false);
        cta_identity<double>(sl.V, N);
    }
    // step 4 (or Alg. 3.2): FP64 sweeps on T scaled by a power of two to ||T||_F ~ 1
    double nt = sqrt(cta_sumsq(sl.T, N, n, false, red));
    int e2 = (nt > 0 && isfinite(nt)) ? -ilogb(nt) : 0;
    cta_scale<double>(sl.T, N, e2);
    int st = cta_block_jacobi<double, B>(sl.T, sl.V, N, n, ldexp(tol_abs, e2), kUb, a.max_sweeps,
                                         a.max_inner, sl.F, sl.fmax, sm, red, &sw);
    cta_scale<double>(sl.T, N, -e2);
    if (status == MPJ_SUCCESS) status = st;
    cta_rank_diag<double>(sl.T, N, n, perm);
    double* L = a.Lambda + job.l_off;
    double* Vo = a.V + job.a_off;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        int r = t % n, k = t / n;
        int p = perm[k];
        Vo[(size_t)r + (size_t)k * n] = sl.V[(size_t)r + (size_t)p * N];
        if (r == 0) L[k] = sl.T[(size_t)p * N + p];
    }
    if (threadIdx.x == 0) {
        if (a.status) a.status[job.idx] = status;
        if (a.sweeps) a.sweeps[job.idx] = sw + 1000 * sw1;
    }
    __syncthreads();
}

// Dynamic shared memory of the batched kernel: the largest need of its steps.
constexpr size_t cmax(size_t x, size_t y) { return x > y ? x : y; }
constexpr size_t kBatchSmem =
    cmax(cmax(cmax(InnerLayout<double, 64>::bytes, ApplySmem<double, 32>::t),
              cmax(ApplySmem<double, 32>::v, InnerLayout<float, 64>::bytes)),
         cmax(ApplySmem<float, 32>::t, sizeof(double) * 2 * 16 * 66));

__global__ void __launch_bounds__(kBatchThreads, 2) k_batched(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ double red[32];
    __shared__ int perm[kNmax];
    __shared__ double g[kNmax];
    __shared__ int job_sh;
    Slot sl(a.slots + (size_t)blockIdx.x * a.slot_bytes);
    for (;;) {
        if (threadIdx.x == 0) job_sh = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int j = job_sh;
        __syncthreads();
        if (j >= a.count) break;
        const BatchJob job = a.jobs[j];
        if (job.n <= 16)      solve_job<8>(a, job, sl, sm, red, perm, g);
        else if (job.n <= 32) solve_job<16>(a, job, sl, sm, red, perm, g);
        else if (job.n <= 64 || a.block_large == 32) solve_job<32>(a, job, sl, sm, red, perm, g);
        else                  solve_job<16>(a, job, sl, sm, red, perm, g);
    }
}

}  // namespace mpj

// ==================================================================== plan + C ABI
struct mpj_batch_plan_s {
    int count = 0;
    int method = 1;
    int ctas = 0;
    int device = 0;
    mpj::BatchJob* d_jobs = nullptr;
    unsigned int* d_counter = nullptr;
    char* d_slots = nullptr;
    size_t slot_bytes = 0;
    mpj_batch_tuning tuning = {};
    long long total_a = 0, total_l = 0;
};

namespace {
void plan_free(mpj_batch_plan_s* p) {
    if (!p) return;
    if (p->d_jobs) cudaFree(p->d_jobs);
    if (p->d_counter) cudaFree(p->d_counter);
    if (p->d_slots) cudaFree(p->d_slots);
    delete p;
}
}  // namespace

extern "C" {

int mpj_batch_plan_create(const int* ns, int count, int method, const mpj_batch_tuning* tuning,
                          mpj_batch_plan** out) {
    using namespace mpj;
    if (!out || !ns || count < 1 || (method != 0 && method != 1)) { set_error_msg("invalid argument"); return MPJ_BAD_ARG; }
    *out = nullptr;
    for (int i = 0; i < count; ++i)
        if (ns[i] < 1 || ns[i] > kNmax) { set_error_msg("batched sizes must satisfy 1 <= n <= 256"); return MPJ_BAD_ARG; }
    auto* p = new mpj_batch_plan_s();
    p->count = count;
    p->method = method;
    mpj_batch_tuning t = {2, 1, 32, 0, 0};
    if (tuning) {
        if (tuning->ctas_per_sm == 1 || tuning->ctas_per_sm == 2) t.ctas_per_sm = tuning->ctas_per_sm;
        if (tuning->max_inner >= 1 && tuning->max_inner <= 8) t.max_inner = tuning->max_inner;
        if (tuning->block_large == 16 || tuning->block_large == 32) t.block_large = tuning->block_large;
        t.max_sweeps = tuning->max_sweeps;
        t.max_sweeps_stage1 = tuning->max_sweeps_stage1;
    }
    p->tuning = t;
    // caller-order offsets, then jobs by decreasing n (longest solves first)
    std::vector<BatchJob> jobs(count);
    long long ao = 0, lo = 0;
    for (int i = 0; i < count; ++i) {
        jobs[i] = BatchJob{ao, lo, ns[i], i};
        ao += (long long)ns[i] * ns[i];
        lo += ns[i];
    }
    p->total_a = ao;
    p->total_l = lo;
    std::stable_sort(jobs.begin(), jobs.end(), [](const BatchJob& x, const BatchJob& y) { return x.n > y.n; });
    cudaError_t e = cudaGetDevice(&p->device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem);
    p->ctas = std::min(count, sms * t.ctas_per_sm);
    p->slot_bytes = (Slot::bytes + 255) & ~size_t(255);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_jobs, sizeof(BatchJob) * count);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_counter, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_slots, p->slot_bytes * (size_t)p->ctas);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_jobs, jobs.data(), sizeof(BatchJob) * count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { set_error("mpj_batch_plan_create", e); plan_free(p); return MPJ_CUDA_ERROR; }
    *out = p;
    return MPJ_SUCCESS;
}

void mpj_batch_plan_destroy(mpj_batch_plan* plan) { plan_free(plan); }

int mpj_batch_plan_info(const mpj_batch_plan* p, long long* a_elems, long long* lambda_elems,
                        int* ctas, size_t* scratch_bytes) {
    if (!p) return MPJ_BAD_ARG;
    if (a_elems) *a_elems = p->total_a;
    if (lambda_elems) *lambda_elems = p->total_l;
    if (ctas) *ctas = p->ctas;
    if (scratch_bytes) *scratch_bytes = p->slot_bytes * (size_t)p->ctas;
    return MPJ_SUCCESS;
}

int mpj_syevj_batched(mpj_batch_plan* p, const double* A, double* Lambda, double* V, double tol,
                      int* status, int* sweeps, void* stream) {
    using namespace mpj;
    if (!p || !A || !Lambda || !V || !(tol == tol)) { set_error_msg("invalid argument"); return MPJ_BAD_ARG; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    BatchArgs a;
    a.jobs = p->d_jobs;
    a.count = p->count;
    a.counter = p->d_counter;
    a.A = A;
    a.Lambda = Lambda;
    a.V = V;
    a.status = status;
    a.sweeps = sweeps;
    a.slots = p->d_slots;
    a.slot_bytes = p->slot_bytes;
    a.method = p->method;
    a.tol = tol;
    a.tol1 = 5.9604644775390625e-08;
    a.max_sweeps = p->tuning.max_sweeps > 0 ? p->tuning.max_sweeps : 40;
    a.max_sweeps1 = p->tuning.max_sweeps_stage1 > 0 ? p->tuning.max_sweeps_stage1 : 40;
    a.max_inner = p->tuning.max_inner;
    a.block_large = p->tuning.block_large;
    MPJ_CUDA_TRY(cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned int), s));
    {
        MPJ_PROF(PC_BATCHED, s);
        k_batched<<<p->ctas, kBatchThreads, kBatchSmem, s>>>(a);
    }
    MPJ_LAUNCH_CHECK("k_batched");
    return MPJ_SUCCESS;
}

}  // extern "C"
