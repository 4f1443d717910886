// tc64_apply.cu -- the FP64 sweeps of Algorithm 3.2 and of step 4 of
// Algorithm 4.1 with the block rotations applied on the 5th-generation tensor
// cores (tcgen05, kind::f16 with bf16 operands) by exact splitting.
//
// A round of the parallel order replaces T by W^T T W and V by V W, where W is
// block diagonal over the disjoint block pairs of the round (W_b = I + F_b,
// 2b x 2b, from the block-pair solves).  As in the FP32 stage (tc_apply.cu)
// both are right multiplications of 128-row slabs by W_b, in delta form:
//
//   pass 1   P = T W      read T through its transpose (T is symmetric), write
//                         P through its transpose (memory holds P^T);
//   pass 2   T' = P^T W   read P^T = memory of pass 1 column-major, write T'
//                         column-major; rows in IJ_b take the solver's rotated
//                         block (exact zeros at the rotated entries);
//   V pass   V' = V W     column-major in place (side stream).
//
// Each tile Y = X + X F_b (X: 128 rows x 64 columns of FP64) is formed from
// exact integer slices (the Ozaki scheme, Ozaki, Ogita, Oishi, Rump, Numer.
// Algorithms 59, 2012) cut from the FP64 bit patterns with integer operations:
// with E_r the largest biased exponent of row r of X (of column c of F),
//
//   M = sign(x) trunc(|x| 2^(1078 - E_r)),  |M| < 2^56,  M = sum_s a_s 2^(49 - 7 s),
//   |a_0| <= 128, a_s in [-64, 63] (s = 1..7, balanced digits),
//
// so x = 2^(E_r - 1029) sum_s a_s 2^(-7 s) up to 2^(E_r - 1078) (every entry
// within 2^3 of the row maximum is cut exactly).  Digits are exact in bf16 and
// their products exact in FP32; the 36 slice products with s + t <= 7 are
// accumulated per level d = s + t in eight FP32 TMEM accumulators (128 x 64
// each, the whole TMEM of the SM), exact since |T_d| < 2^22 for K = 64.  The
// epilogue turns the eight levels into one 64-bit integer
// S = sum_d T_d 2^(42 - 7 d) (the last level truncated by 2^-7) with integer
// operations and forms y = x + 2^(E_r + E_c - 2100) S with one FP64 FMA.  The
// dropped levels d >= 8 and the truncations are below 2^-54 K max|X_r:|
// max|F_:c|, the order of an FP64 dot product's rounding error.
//
// The block solves (FP64, Lemma 3.1, Remark 3.7) are the ones of the SIMT
// engine without writing the rotated block back; they also cut F_b into its
// digit planes, already in the swizzled shared-memory layout of the MMA's B
// operand, so that a pass CTA loads them with one bulk copy.
#include <cmath>
#include <cstdio>

#include "internal.h"
#include "engine_device.cuh"
#include "tc64_device.cuh"

namespace mpj {

namespace {

// ---------------------------------------------------------------- block solve
// The 2b x 2b block-pair solve of the SIMT engine (no write-back: the rotated
// block goes to Sbuf for pass 2), then F_b = W_b - I cut into its 8 digit planes
// (B operand: row c = column c of F over k) and 64 column exponent classes.
__global__ void __launch_bounds__(kSolveThreads)
k_solve2_tc64(double* __restrict__ T, int N, double* __restrict__ Fbuf, double* __restrict__ Sbuf,
              unsigned char* __restrict__ Fpl, float* __restrict__ fmax, int round, double eps, double tau,
              double gate, int max_inner, int cross, unsigned long long* __restrict__ rot_counter) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int b = blockIdx.x;
    int applied = pair_solve<double, kB, false>(T, N, round, b, eps, tau, gate, max_inner,
                                                Fbuf + (size_t)b * kM * kM, fmax + b, smraw,
                                                Sbuf + (size_t)b * kM * kM, cross ? round : -1);
    if (threadIdx.x == 0 && applied) atomicAdd(rot_counter, (unsigned long long)applied);
    // F is still in shared memory after S: F[c * (M + 1) + k] = F(k, c)
    const double* Fs = reinterpret_cast<const double*>(smraw) + kM * (kM + 1);
    unsigned char* dst = Fpl + (size_t)b * kFplBytes;
    const int t = threadIdx.x;                       // 512 threads: (column c, chunk j)
    const int c = t >> 3, j = t & 7;
    double x[8];
    int cls = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        x[e] = Fs[c * (kM + 1) + 8 * j + e];
        cls = max(cls, exp_class(x[e]));
    }
    // the 8 threads of column c are consecutive lanes of one warp
    cls = max(cls, __shfl_xor_sync(0xffffffffu, cls, 1));
    cls = max(cls, __shfl_xor_sync(0xffffffffu, cls, 2));
    cls = max(cls, __shfl_xor_sync(0xffffffffu, cls, 4));
    if (j == 0) reinterpret_cast<int*>(dst + kS * kBPlane)[c] = cls;
    uint64_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = scaled_signed(x[e], cls);
#pragma unroll
    for (int p = 0; p < kS; ++p)
        *reinterpret_cast<uint4*>(dst + p * kBPlane + sw_chunk(c, j)) =
            make_uint4(digit_pair(v[0], v[1], p), digit_pair(v[2], v[3], p), digit_pair(v[4], v[5], p),
                       digit_pair(v[6], v[7], p));
}

}  // namespace


size_t tc64_workspace_bytes(int N) {
    Arena a;
    const size_t K = (size_t)(N / kM);
    for (int set = 0; set < 2; ++set) {
        a.take<double>(K * kM * kM);          // F
        a.take<double>(K * kM * kM);          // rotated diagonal blocks
        a.take<unsigned char>(K * kFplBytes); // digit planes of F
        a.take<float>(K);                     // max |F|
    }
    a.take<double>((size_t)N * N);            // P of pass 1
    a.take<double>(1024);
    a.take<double>(4);
    a.take<unsigned long long>(4);
    return a.used + 256;
}

bool tc64_supported(int N, int B) { return B == kB && N % kM == 0 && N >= kM; }

int twosided_sweeps_tc64(double* T, double* V, int N, int n, double tol_abs, double eps_skip, int max_sweeps,
                         int max_inner, int cross, void* work, cudaStream_t s, SweepResult* res) {
    if (!tc64_supported(N, kB)) { set_error_msg("tensor-core FP64 engine: N must be a multiple of 64"); return MPJ_BAD_ARG; }
    const int K = N / kM;
    Arena ar;
    ar.base = static_cast<char*>(work);
    ar.size = tc64_workspace_bytes(N);
    double *Fbuf[2], *Sbuf[2];
    unsigned char* Fpl[2];
    float* fmax[2];
    for (int set = 0; set < 2; ++set) {
        Fbuf[set] = ar.take<double>((size_t)K * kM * kM);
        Sbuf[set] = ar.take<double>((size_t)K * kM * kM);
        Fpl[set] = ar.take<unsigned char>((size_t)K * kFplBytes);
        fmax[set] = ar.take<float>((size_t)K);
    }
    double* P = ar.take<double>((size_t)N * N);
    double* partial = ar.take<double>(1024);
    double* offv = ar.take<double>(4);
    unsigned long long* rot = ar.take<unsigned long long>(4);     // [0] rotations, [1] error flag
    if (!Fbuf[1] || !Sbuf[1] || !Fpl[1] || !fmax[1] || !P || !partial || !offv || !rot) {
        set_error_msg("workspace too small");
        return MPJ_BAD_ARG;
    }
    HostScratch hs;
    MPJ_TRY(hs.init());
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_solve2_tc64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)InnerLayout<double, kM>::bytes));
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_pass_tc64<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPassSmem));
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_pass_tc64<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPassSmem));
    Tc64Maps m1, m2, mv;
    MPJ_TRY(encode_tile_map(&m1.in, T, N, true));      // pass 1: T^T (= T) in, P^T out
    MPJ_TRY(encode_tile_map(&m1.out, P, N, true));
    MPJ_TRY(encode_tile_map(&m2.in, P, N, false));     // pass 2: P^T in, T' out
    MPJ_TRY(encode_tile_map(&m2.out, T, N, false));
    MPJ_TRY(encode_tile_map(&mv.in, V, N, false));     // V pass, in place
    mv.out = mv.in;
    SideStream side;
    MPJ_TRY(side.init(s));
    s = side.main;
    MPJ_CUDA_TRY(cudaMemsetAsync(rot, 0, 2 * sizeof(unsigned long long), s));
    MPJ_TRY(offnorm2(T, true, N, n, partial, offv, s));
    MPJ_CUDA_TRY(cudaMemcpyAsync(hs.d, offv, sizeof(double), cudaMemcpyDeviceToHost, s));
    MPJ_CUDA_TRY(cudaStreamSynchronize(s));
    double off = sqrt(hs.d[0]);
    res->off_initial = off;
    res->sweeps = 0;
    res->rotations = 0;
    res->status = MPJ_NOT_CONVERGED;
    const int rounds = 2 * K - 1;
    const int n_slabs = (N + kSlab - 1) / kSlab;     // a ragged last slab: TMA fills and clips rows >= N
    const int items = n_slabs * K;
    const int nsm = sm_count();
    const int gridT = items < nsm ? items : nsm;
    const int perT = (items + gridT - 1) / gridT;
    const int perV = 8;                               // short CTAs: SM slots free up for the next solve
    const int gridV = (items + perV - 1) / perV;
    const double tau = tol_abs / (double)N;
    const double gate = 1.0 / 64.0;                  // Newton-Schulz when some |F| >= 2^-6
    const int xs = N >= kB * kB ? cross : 0;
    while (res->sweeps < max_sweeps) {
        if (!std::isfinite(off)) { res->status = MPJ_NONFINITE_INPUT; break; }
        if (!(off > tol_abs)) { res->status = MPJ_SUCCESS; break; }
        MPJ_CUDA_TRY(cudaMemsetAsync(rot, 0, sizeof(unsigned long long), s));
        for (int r = 0; r < rounds; ++r) {
            const int set = side.begin_round();
            if (set < 0) return MPJ_CUDA_ERROR;
            {
                MPJ_PROF(PC_SOLVE2_F64, s);
                k_solve2_tc64<<<K, kSolveThreads, InnerLayout<double, kM>::bytes, s>>>(
                    T, N, Fbuf[set], Sbuf[set], Fpl[set], fmax[set], r, eps_skip, tau, gate, max_inner, xs, rot);
            }
            MPJ_LAUNCH_CHECK("k_solve2_tc64");
            {
                MPJ_PROF(PC_TCP1_F64, s);
                k_pass_tc64<true, false><<<gridT, kThr, kPassSmem, s>>>(m1, N, n_slabs, items, perT, Fpl[set], fmax[set],
                                                                  nullptr, r, 0, rot + 1, nullptr);
            }
            MPJ_LAUNCH_CHECK("k_pass_tc64 pass 1");
            {
                MPJ_PROF(PC_TCP2_F64, s);
                k_pass_tc64<false, false><<<gridT, kThr, kPassSmem, s>>>(m2, N, n_slabs, items, perT, Fpl[set], fmax[set],
                                                                   Sbuf[set], r, 0, rot + 1, nullptr);
            }
            MPJ_LAUNCH_CHECK("k_pass_tc64 pass 2");
            MPJ_TRY(side.after_solve());                 // V joins after pass 2 (overlaps the next solve)
            {
                MPJ_PROF(PC_TCV_F64, side.sv);
                k_pass_tc64<false, false><<<gridV, kThr, kPassSmem, side.sv>>>(mv, N, n_slabs, items, perV, Fpl[set],
                                                                         fmax[set], nullptr, r, 1, rot + 1, nullptr);
            }
            MPJ_LAUNCH_CHECK("k_pass_tc64 V");
            MPJ_TRY(side.after_v());
            side.end_round();
        }
        MPJ_TRY(offnorm2(T, true, N, n, partial, offv, s));
        MPJ_CUDA_TRY(cudaMemcpyAsync(hs.d, offv, sizeof(double), cudaMemcpyDeviceToHost, s));
        MPJ_CUDA_TRY(cudaMemcpyAsync(hs.u, rot, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        MPJ_CUDA_TRY(cudaStreamSynchronize(s));
        prof_flush();
        if (hs.u[1]) { set_error_msg("tensor-core FP64 pass: TMA or MMA wait timed out"); return MPJ_CUDA_ERROR; }
        off = sqrt(hs.d[0]);
        res->sweeps += 1;
        res->rotations += (double)hs.u[0];
        if (trace_on())
            fprintf(stderr, "[mpj] twosided<tc64> n=%d sweep %d: %llu rotations, off %.3e\n", n, res->sweeps,
                    hs.u[0], off);
        if (hs.u[0] == 0) { res->status = MPJ_SUCCESS; break; }
    }
    if (res->status == MPJ_NOT_CONVERGED && std::isfinite(off) && !(off > tol_abs)) res->status = MPJ_SUCCESS;
    res->off_final = off;
    return MPJ_SUCCESS;
}

}  // namespace mpj
