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
// k_apply2 is two kernels: k_apply2T (tiles of T) and k_apply2V (slabs of V);
// k_apply2V runs on a low-priority second stream, overlapping the next round's
// block solves (the rotations of two rounds are double buffered).  FP64 sweeps
// of a nearly diagonal T switch from b = 32 to b = 16 from the third sweep on.
#include <cmath>
#include <cstdio>

#include "internal.h"
#include <cstdlib>
#include "engine_device.cuh"

namespace mpj {

template <class Real, int B>
__global__ void __launch_bounds__(kSolveThreads)
k_solve2(Real* __restrict__ T, int N, Real* __restrict__ Fbuf, float* __restrict__ fmax, int round,
         Real eps, Real tau, Real gate, int max_inner, int cross, unsigned long long* __restrict__ rot_counter,
         float* __restrict__ Fsplit) {
    constexpr int M = 2 * B;
    extern __shared__ __align__(16) unsigned char smraw[];
    int applied = pair_solve<Real, B>(T, N, round, blockIdx.x, eps, tau, gate, max_inner,
                                      Fbuf + (size_t)blockIdx.x * M * M, fmax + blockIdx.x, smraw, nullptr,
                                      cross ? round : -1);
    if (threadIdx.x == 0 && applied) atomicAdd(rot_counter, (unsigned long long)applied);
    if constexpr (sizeof(Real) == 8) {
        // float planes of F for the double-float tile products (F is still in shared memory)
        if (Fsplit)
            store_f_split(reinterpret_cast<const double*>(smraw) + M * (M + 1), M + 1, M,
                          Fsplit + (size_t)blockIdx.x * 2 * M * M);
    }
}

template <class Real, int B>
__global__ void __launch_bounds__(kThreads)
k_apply2T(Real* __restrict__ T, int N, const Real* __restrict__ Fbuf, const float* __restrict__ fmax,
          int round, float df_gate, const float* __restrict__ Fsplit) {
    extern __shared__ __align__(16) unsigned char smraw[];
    int a, b;
    decode_tile(blockIdx.x, N / (2 * B), a, b);
    apply_tile<Real, B>(T, N, Fbuf, fmax, round, a, b, df_gate, smraw, Fsplit);
}

template <class Real, int B>
__global__ void __launch_bounds__(kThreads)
k_apply2V(Real* __restrict__ V, int N, const Real* __restrict__ Fbuf, const float* __restrict__ fmax,
          int round, float df_gate, const float* __restrict__ Fsplit) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int K = N / (2 * B);
    apply_slab<Real, B>(V, N, Fbuf, fmax, round, blockIdx.x / K, blockIdx.x % K, df_gate, smraw, Fsplit);
}

// Inner-sweep schedule of the block solves: the cross-pair schedule (inner_jacobi
// with cross_round) for the FP32 sweeps of step 1, where it halves the steps of a
// block solve at the same outer sweep count, and for the tensor-core FP64 sweeps,
// whose tile products do not depend on the size of the block rotations (measured
// at n = 4096: uniform 547 -> 513 ms, clustered 1660 -> 1340 ms, equal or fewer
// sweeps; MPJ_OPT_FULL_INNER restores the full tournament there).  The SIMT FP64
// engine keeps the full tournament: the cross schedule leaves larger block
// rotations on clustered spectra, so fewer of its tiles qualify for the
// double-float products.  The callers use it only when an outer sweep has at
// least b - 1 rounds (N >= b^2), so that the intra steps of the rounds of one
// sweep cover every pair inside a block.
int cross_schedule(bool fp64, bool tc64) {
    if (!fp64) return 1;
    return tc64 && !knobs().full_inner ? 1 : 0;
}

// First FP64 sweep run with b = 16 on a nearly diagonal T in the SIMT engine (2:
// the third sweep).
constexpr int kLateB16Sweep = 2;
// Double-float tile products when both block rotations have max |F| <= 2^-8.
constexpr float kDfGate = 1.0f / 256.0f;

template <class Real>
size_t twosided_workspace_bytes(int N, int B) {
    Arena a;
    int K = N / (2 * B), M = 2 * B;
    const int Kf = K > N / 32 ? K : N / 32;             // max|F| for b = 16 as well (late FP64 sweeps)
    for (int set = 0; set < 2; ++set) {                 // block rotations of two consecutive rounds
        a.take<Real>((size_t)K * M * M);
        a.take<float>((size_t)Kf);
        if (sizeof(Real) == 8) a.take<float>((size_t)K * 2 * M * M);   // F split planes
    }
    a.take<double>(1024);
    a.take<double>(4);
    a.take<unsigned long long>(4);
    size_t bytes = a.used + 256;
    if (sizeof(Real) == 8 && tc64_supported(N, B)) {
        const size_t t = tc64_workspace_bytes(N);
        bytes = t > bytes ? t : bytes;
    }
    return bytes;
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
                        float* Fsplit, cudaStream_t s, SideStream& side) {
    cudaStream_t sv = side.sv;
    constexpr int M = 2 * B;
    const int K = N / M;
    const bool dbl = sizeof(Real) == 8;
    { MPJ_PROF(dbl ? PC_SOLVE2_F64 : PC_SOLVE2_F32, s);
      k_solve2<Real, B><<<K, kSolveThreads, InnerLayout<Real, M>::bytes, s>>>(T, N, Wbuf, fmax, r, eps, tau,
                                                                         gate, max_inner, N >= B * B ? cross_schedule(dbl, false) : 0, rot,
                                                                         Fsplit); }
    MPJ_LAUNCH_CHECK("k_solve2");
    // the V update waits only for the block solve, so it overlaps the tile update as
    // well (measured: waiting for the tile update costs 5 ms at n = 4096)
    const bool v_late = false;
    if (!v_late) MPJ_TRY(side.after_solve());
    int n_ttiles = K * (K - 1) / 2;
    if (n_ttiles > 0) {
        MPJ_PROF(dbl ? PC_APPLY2_F64 : PC_APPLY2_F32, s);
        k_apply2T<Real, B><<<n_ttiles, kThreads, ApplySmem<Real, B>::t, s>>>(T, N, Wbuf, fmax, r, df_gate, Fsplit);
        MPJ_LAUNCH_CHECK("k_apply2T");
    }
    if (v_late) MPJ_TRY(side.after_solve());
    {
        MPJ_PROF(dbl ? PC_APPLY2V_F64 : PC_APPLY2V_F32, sv);
        k_apply2V<Real, B><<<(N / M) * K, kThreads, ApplySmem<Real, B>::v, sv>>>(V, N, Wbuf, fmax, r, df_gate, Fsplit);
        MPJ_LAUNCH_CHECK("k_apply2V");
    }
    MPJ_TRY(side.after_v());
    return MPJ_SUCCESS;
}

template <class Real>
int twosided_sweeps(Real* T, Real* V, int N, int n, int B, double tol_abs, double eps_skip,
                    int max_sweeps, int max_inner, void* work, cudaStream_t s, SweepResult* res) {
    if constexpr (sizeof(Real) == 8) {
        // b = 32: the block rotations are applied on the tensor cores (tc64_apply.cu)
        if (!knobs().simt_sweeps && tc64_supported(N, B))
            return twosided_sweeps_tc64(T, V, N, n, tol_abs, eps_skip, max_sweeps, max_inner,
                                        cross_schedule(true, true), work, s, res);
    }
    const int M = 2 * B;
    const int K = N / M;
    const int Kf = K > N / 32 ? K : N / 32;
    Arena ar;
    ar.base = static_cast<char*>(work);
    ar.size = twosided_workspace_bytes<Real>(N, B);
    Real* Wbuf[2];
    float* fmax[2];
    float* Fsplit[2] = {nullptr, nullptr};
    for (int set = 0; set < 2; ++set) {
        Wbuf[set] = ar.take<Real>((size_t)K * M * M);
        fmax[set] = ar.take<float>((size_t)Kf);
        if (sizeof(Real) == 8) Fsplit[set] = ar.take<float>((size_t)K * 2 * M * M);
    }
    double* partial = ar.take<double>(1024);
    double* offv = ar.take<double>(4);
    unsigned long long* rot = ar.take<unsigned long long>(4);
    if (!Wbuf[0] || !Wbuf[1] || !fmax[0] || !fmax[1] || !partial || !offv || !rot ||
        (sizeof(Real) == 8 && (!Fsplit[0] || !Fsplit[1]))) {
        set_error_msg("workspace too small");
        return MPJ_BAD_ARG;
    }
    HostScratch hs;
    MPJ_TRY(hs.init());
    // V is updated on a second stream: the V slabs of round r need only that round's
    // block rotations, so they overlap the next block solves (which occupy K SMs).
    // The rotations of two consecutive rounds are double buffered; the solve of
    // round g + 2 waits until the V update of round g has read its buffers.  The
    // rest runs on the side object's high-priority stream.
    SideStream side;
    MPJ_TRY(side.init(s));
    s = side.main;
    const bool dbl = sizeof(Real) == 8;
    // On a nearly diagonal T (the preconditioned step 4), FP64 sweeps from the third on
    // use b = 16 when they started with b = 32: a spectrum that still needs them
    // (clusters, tiny eigenvalues) gains from twice as many, four times cheaper block
    // solves, while one that converges in two sweeps never switches (measured at
    // n = 4096: geometric 1644 -> 1529 ms, clustered 2803 -> 2739 ms; the plain
    // algorithm on a dense T took one sweep more with the switch, so it keeps b).
    // The b = 32 buffers hold the b = 16 ones (K M^2 = N M shrinks with M).
    int switch_sweep = (sizeof(Real) == 8 && B == 32) ? kLateB16Sweep : -1;
    MPJ_TRY((configure_twosided<Real, 16>()));
    if (B == 32) MPJ_TRY((configure_twosided<Real, 32>()));

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
    if (!(off <= 1.0 / 1024.0)) switch_sweep = -1;      // ||T||_F is about 1 here
    res->sweeps = 0;
    res->rotations = 0;
    res->status = MPJ_NOT_CONVERGED;
    // entries below tau cannot keep ||off(T)||_F above tol_abs once all are below it
    const Real tau = (Real)(tol_abs / (double)N);
    // Newton-Schulz re-orthogonalisation of W = I + F when some |F| >= 2^-6 (FP64)
    // or 2^-12 (FP32): with F accumulated in delta form, smaller blocks stay
    // orthogonal to working precision without it.
    const Real gate = (Real)(dbl ? 1.0 / 64.0 : 1.0 / 4096.0);
    // double-float tile products when both block rotations have max |F| <= 2^-8
    const float df_gate = dbl ? kDfGate : -1.0f;
    while (res->sweeps < max_sweeps) {
        if (!std::isfinite(off)) { res->status = MPJ_NONFINITE_INPUT; break; }
        if (!(off > tol_abs)) { res->status = MPJ_SUCCESS; break; }
        MPJ_CUDA_TRY(cudaMemsetAsync(rot, 0, sizeof(unsigned long long), s));
        const int Bs = (switch_sweep >= 0 && res->sweeps >= switch_sweep) ? 16 : B;
        const int rounds = N / Bs - 1;
        for (int r = 0; r < rounds; ++r) {
            const int set = side.begin_round();
            if (set < 0) return MPJ_CUDA_ERROR;
            if (Bs == 16) {
                MPJ_TRY((launch_round<Real, 16>(T, V, N, Wbuf[set], fmax[set], r, (Real)eps_skip, tau, gate,
                                                df_gate, max_inner, rot, Fsplit[set], s, side)));
            } else {
                MPJ_TRY((launch_round<Real, 32>(T, V, N, Wbuf[set], fmax[set], r, (Real)eps_skip, tau, gate,
                                                df_gate, max_inner, rot, Fsplit[set], s, side)));
            }
            side.end_round();
        }
        MPJ_TRY(offnorm2(T, dbl, N, n, partial, offv, s));
        MPJ_CUDA_TRY(cudaMemcpyAsync(hs.d, offv, sizeof(double), cudaMemcpyDeviceToHost, s));
        MPJ_CUDA_TRY(cudaMemcpyAsync(hs.u, rot, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        MPJ_CUDA_TRY(cudaStreamSynchronize(s));
        prof_flush();
        off = sqrt(hs.d[0]);
        res->sweeps += 1;
        res->rotations += (double)hs.u[0];
        if (trace_on())
            fprintf(stderr, "[mpj] twosided<%s> n=%d sweep %d: %llu rotations, off %.3e\n",
                    dbl ? "f64" : "f32", n, res->sweeps, hs.u[0], ldexp(off, -e2));
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
