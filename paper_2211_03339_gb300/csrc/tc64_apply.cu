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
//   M = trunc(|x| 2^(1078 - E_r)) < 2^56,   M = sum_s a_s 2^(49 - 7 s),
//   a_0 in [0, 128], a_s in [-64, 63] (s = 1..7, balanced digits),
//
// so x = +-2^(E_r - 1029) sum_s a_s 2^(-7 s) up to 2^(E_r - 1078) (every entry
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

#include <cuda.h>

#include "internal.h"
#include "engine_device.cuh"
#include "tc_device.cuh"

namespace mpj {

namespace {

constexpr int kB = 32;                       // block size b
constexpr int kM = 2 * kB;                   // pair width = K = N of the MMA
constexpr int kSlab = 128;                   // tile rows = M of the MMA
constexpr int kThr = 256;                    // pass kernel threads
constexpr int kS = 8;                        // digits (slices) per operand
constexpr int kXBytes = kSlab * kM * 8;      // FP64 tile, 64 KB
constexpr int kAPlane = kSlab * 128;         // A digit plane: 128 rows x 64 bf16
constexpr int kBPlane = kM * 128;            // B digit plane: 64 rows x 64 bf16
constexpr int kAGroup = 4;                   // A planes resident at a time
constexpr int kFplBytes = kS * kBPlane + 256;   // per pair: 8 planes + 64 exponents
constexpr int kOffA = kXBytes;
constexpr int kOffB = kOffA + kAGroup * kAPlane;
constexpr int kOffE = kOffB + kS * kBPlane;
constexpr size_t kPassSmem = (size_t)kOffE + 256 + 1024;
constexpr int kWait = 1 << 22;               // mbarrier polls before a CTA gives up
// 64 at each of the seven lower 7-bit digit positions: adding it to M makes the
// truncated base-128 digits of M + kBias minus 64 the balanced digits of M.
constexpr uint64_t kBias =
    64ull * ((1ull << 42) + (1ull << 35) + (1ull << 28) + (1ull << 21) + (1ull << 14) + (1ull << 7) + 1ull);

// ---------------------------------------------------------------- slicing
// Exponent class of x for a row maximum: 0 for x == 0, else max(E, 1) with E the
// biased exponent (subnormals count as 1).  Integer operations only.
__device__ __forceinline__ int exp_class(double x) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const int E = (hi >> 20) & 0x7FF;
    const int nz = ((hi & 0xFFFFFu) | lo) != 0u;
    return E ? E : nz;
}

// M + kBias for M = trunc(|x| 2^(1078 - Er)) (Er >= exp_class(x)), and the sign.
__device__ __forceinline__ uint64_t scaled_mag(double x, int Er, uint32_t& neg) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    neg = (uint32_t)(b >> 63);
    const int E = (int)((b >> 52) & 0x7FF);
    uint64_t mant = b & 0xFFFFFFFFFFFFFull;
    if (E) mant |= 1ull << 52;
    const int sh = (E ? E : 1) - Er + 3;          // <= 3
    const uint64_t M = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> -sh) : 0ull);
    return M + kBias;
}

// Digits S0 .. S0+NP-1 of 8 consecutive elements as NP 16-byte chunks of bf16
// (element e in halfword e).  A digit r becomes a float through the magic
// constant 2^23 (exact), its bias is subtracted, and the bf16 is the float's
// upper half (exact: at most 8 significant bits); sg holds the sign bits of the
// element pairs.
template <int S0, int NP>
__device__ __forceinline__ void digits8(const uint64_t (&Mb)[8], const uint32_t (&sg)[4], uint4 (&out)[NP]) {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int s = S0 + p;
        const int shift = 49 - 7 * s;
        const float K = s == 0 ? 8388608.0f : 8388672.0f;      // 2^23 + bias
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t r0 = (uint32_t)(Mb[2 * q] >> shift), r1 = (uint32_t)(Mb[2 * q + 1] >> shift);
            if (s > 0) { r0 &= 127u; r1 &= 127u; }
            const float v0 = __fsub_rn(__uint_as_float(0x4B000000u | r0), K);
            const float v1 = __fsub_rn(__uint_as_float(0x4B000000u | r1), K);
            w[q] = __byte_perm(__float_as_uint(v0), __float_as_uint(v1), 0x7632) ^ sg[q];
        }
        out[p] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

__device__ __forceinline__ void prep8(const double (&x)[8], int Er, uint64_t (&Mb)[8], uint32_t (&sg)[4]) {
    uint32_t ng[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) Mb[e] = scaled_mag(x[e], Er, ng[e]);
#pragma unroll
    for (int q = 0; q < 4; ++q) sg[q] = (ng[2 * q] << 15) | (ng[2 * q + 1] << 31);
}

// Byte offset of 16-byte chunk j (elements 8j..8j+7 along K) of row r in a
// K-major operand of 128-byte rows with the 128-byte swizzle.
__device__ __forceinline__ int sw_chunk(int r, int j) {
    return (r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4);
}

// The eight levels T_d (exact integers in FP32, |T_d| < 2^22) as one 64-bit
// integer sum_d T_d 2^(42 - 7 d) (T_7 truncated by 2^-7): each float becomes
// its integer through the magic constant 1.5 * 2^23.
__device__ __forceinline__ long long combine8(const float (&a)[8]) {
    int t[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) t[d] = __float_as_int(__fadd_rn(a[d], 12582912.0f)) - 0x4B400000;
    return ((long long)t[0] << 42) + ((long long)t[1] << 35) + ((long long)t[2] << 28) +
           ((long long)t[3] << 21) + ((long long)t[4] << 14) + ((long long)t[5] << 7) + (long long)t[6] +
           (long long)(t[7] >> 7);
}

// y = x + 2^(Er + Ec - 2100) S.
__device__ __forceinline__ double apply_level_sum(double x, long long S, int Er, int Ec) {
    if (S == 0) return x;
    const int be = Er + Ec - 1077;                   // biased exponent of the scale
    const double v = __ll2double_rn(S);
    if (be >= 1) return fma(v, __longlong_as_double((long long)be << 52), x);
    return x + scalbn(v, be - 1023);                 // tiny operands: not on the fast path
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            tc::smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(tc::smem_u32(mbar))
        : "memory");
}

// Byte offset of X(m, c) in the FP64 tile.  Column layout (Lc): two TMA boxes
// of 128 rows x 32 columns, column c at c * 1024.  Row layout (Lr): four boxes
// of 16 columns x 128 rows with the 128-byte swizzle (box q = c / 16).
template <bool kLr>
__device__ __forceinline__ int xoff(int m, int c) {
    if constexpr (kLr) {
        const int q = c >> 4, cc = c & 15;
        return q * 16384 + m * 128 + ((((cc >> 1) ^ (m & 7)) << 4) | ((cc & 1) << 3));
    } else {
        return (c * kSlab + m) * 8;
    }
}

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
    uint64_t Mb[8];
    uint32_t sg[4];
    prep8(x, cls, Mb, sg);
    uint4 d[kS];
    digits8<0, kS>(Mb, sg, d);
#pragma unroll
    for (int p = 0; p < kS; ++p) *reinterpret_cast<uint4*>(dst + p * kBPlane + sw_chunk(c, j)) = d[p];
}

// ---------------------------------------------------------------- pass kernel
struct Tc64Maps {
    CUtensorMap in, out;
};

template <bool kLr>
__device__ __forceinline__ void tile_io(const CUtensorMap* map, bool load, unsigned char* Xs, int row0, int I,
                                        int J, uint64_t* bar) {
    if constexpr (kLr) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int col = (q < 2 ? I : J) * kB + (q & 1) * 16;
            if (load) tc::tma_load_2d(Xs + q * 16384, map, col, row0, bar);
            else tc::tma_store_2d(map, col, row0, Xs + q * 16384);
        }
    } else {
        if (load) {
            tc::tma_load_2d(Xs, map, row0, I * kB, bar);
            tc::tma_load_2d(Xs + 32768, map, row0, J * kB, bar);
        } else {
            tc::tma_store_2d(map, row0, I * kB, Xs);
            tc::tma_store_2d(map, row0, J * kB, Xs + 32768);
        }
    }
}

// One CTA per SM (the eight accumulators take the whole TMEM).  Items are
// (slab s, pair b), b-major; CTA k takes items [k per_cta, (k+1) per_cta), so
// that the digit planes of F_b are reloaded only when the pair changes.  With
// skip_identity, items whose W_b is the identity are skipped (in place V);
// otherwise they are copied.  With Sbuf, rows in IJ_b take the solver's block.
template <bool kLr>
__global__ void __launch_bounds__(kThr, 1)
k_pass_tc64(const __grid_constant__ Tc64Maps maps, int N, int n_slabs, int total, int per_cta,
            const unsigned char* __restrict__ Fpl, const float* __restrict__ fmax,
            const double* __restrict__ Sbuf, int round, int skip_identity, unsigned long long* __restrict__ err) {
    extern __shared__ unsigned char smraw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) &
                                                         ~uintptr_t(1023));
    unsigned char* Xs = sm;
    unsigned char* Ap = sm + kOffA;
    unsigned char* Bp = sm + kOffB;
    const int* exc = reinterpret_cast<const int*>(sm + kOffE);
    __shared__ __align__(8) uint64_t bar_ld, bar_mma;
    __shared__ uint32_t tmem_slot;
    __shared__ int exr[kSlab];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nblocks = N / kB;
    if (tid == 0) {
        tc::mbar_init(&bar_ld, 1);
        tc::mbar_init(&bar_mma, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const int it0 = blockIdx.x * per_cta;
    const int it1 = min(total, it0 + per_cta);
    int cur = -1;                                   // pair whose F planes are in Bp
    uint32_t pl = 0, pm = 0;                        // mbarrier phases
    bool failed = false;
    // slicing items of this thread: row ms = tid % 128, chunks js = tid / 128 + 2 i
    const int ms = tid & (kSlab - 1), jh = tid >> 7;
    for (int it = it0; it < it1 && !failed; ++it) {
        const int b = it / n_slabs, s = it % n_slabs;
        const bool ident = fmax[b] == 0.f;
        if (ident && skip_identity) continue;
        int I, J;
        round_pair(round, b, nblocks, I, J);
        const int row0 = s * kSlab;
        const bool loadF = !ident && b != cur;
        if (tid < kSlab) exr[tid] = 0;
        if (tid == 0) {
            tc::mbar_expect_tx(&bar_ld, kXBytes + (loadF ? kFplBytes : 0));
            if (loadF) bulk_load(Bp, Fpl + (size_t)b * kFplBytes, kFplBytes, &bar_ld);
            tile_io<kLr>(&maps.in, true, Xs, row0, I, J, &bar_ld);
        }
        if (loadF) cur = b;
        bool ok = tc::mbar_wait(&bar_ld, pl, kWait);
        pl ^= 1;
        if (__syncthreads_or(!ok)) { failed = true; break; }
        if (!ident) {
            double xv[4][8];
            int emax = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    xv[i][e] = *reinterpret_cast<const double*>(Xs + xoff<kLr>(ms, 8 * (jh + 2 * i) + e));
                    emax = max(emax, exp_class(xv[i][e]));
                }
            atomicMax(&exr[ms], emax);
            __syncthreads();
            const int Er = exr[ms];
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                if (g == 1) {                       // the A planes are free once group 0's MMAs are done
                    ok = tc::mbar_wait(&bar_mma, pm, kWait);
                    pm ^= 1;
                    tc::fence_after_sync();
                    if (__syncthreads_or(!ok)) { failed = true; break; }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    uint64_t Mb[8];
                    uint32_t sg[4];
                    prep8(xv[i], Er, Mb, sg);
                    uint4 d[kAGroup];
                    if (g == 0) digits8<0, kAGroup>(Mb, sg, d);
                    else digits8<kAGroup, kAGroup>(Mb, sg, d);
                    const int off = sw_chunk(ms, jh + 2 * i);
#pragma unroll
                    for (int p = 0; p < kAGroup; ++p) *reinterpret_cast<uint4*>(Ap + p * kAPlane + off) = d[p];
                }
                tc::fence_proxy_async();
                tc::fence_before_sync();
                __syncthreads();
                tc::fence_after_sync();
                if (tid == 0) {
                    constexpr uint32_t idesc = tc::instr_desc(tc::kFmtBF16, kSlab, kM);
                    const uint32_t a0 = tc::smem_u32(Ap), b0 = tc::smem_u32(Bp);
#pragma unroll
                    for (int sl = 0; sl < kAGroup; ++sl) {
                        const int sa = g * kAGroup + sl;
#pragma unroll
                        for (int t = 0; t + sa < kS; ++t)
#pragma unroll
                            for (int ks = 0; ks < kM / 16; ++ks)
                                tc::mma_f16(tmem + (uint32_t)((sa + t) * kM),
                                            tc::smem_desc_sw128(a0 + sl * kAPlane + ks * 32),
                                            tc::smem_desc_sw128(b0 + t * kBPlane + ks * 32), idesc,
                                            (sa == 0 && ks == 0) ? 0u : 1u);
                    }
                    tc::commit(&bar_mma);
                }
            }
            if (failed) break;
            ok = tc::mbar_wait(&bar_mma, pm, kWait);
            pm ^= 1;
            tc::fence_after_sync();
            if (__syncthreads_or(!ok)) { failed = true; break; }
        }
        // epilogue: thread (warp w, lane) = tile row m = 32 (w % 4) + lane (its TMEM
        // lane), columns 32 (w / 4) .. +31
        {
            const int m = 32 * (warp & 3) + lane;
            const int cb = 32 * (warp >> 2);
            const int row = row0 + m;
            const int Er = exr[m];
            const double* Srow = nullptr;
            if (Sbuf) {
                const int blk = row / kB;
                if (blk == I) Srow = Sbuf + (size_t)b * kM * kM + (size_t)(row % kB) * kM;
                else if (blk == J) Srow = Sbuf + (size_t)b * kM * kM + (size_t)(kB + row % kB) * kM;
            }
            const uint32_t lanebase = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll 1
            for (int c0 = cb; c0 < cb + 32; c0 += 8) {
                float a[kS][8];
                if (!ident) {
#pragma unroll
                    for (int d = 0; d < kS; ++d) tmem_ld8(lanebase + (uint32_t)(d * kM + c0), a[d]);
                    tc::tmem_wait_ld();
                }
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int c = c0 + e;
                    double* px = reinterpret_cast<double*>(Xs + xoff<kLr>(m, c));
                    double y = *px;
                    if (!ident) {
                        float lv[kS];
#pragma unroll
                        for (int d = 0; d < kS; ++d) lv[d] = a[d][e];
                        y = apply_level_sum(y, combine8(lv), Er, exc[c]);
                    }
                    if (Srow) y = Srow[c];
                    *px = y;
                }
            }
        }
        tc::fence_proxy_async();                     // the tile's generic writes -> TMA store
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            tile_io<kLr>(&maps.out, false, Xs, row0, I, J, nullptr);
            tc::bulk_commit();
            tc::bulk_wait_read();                    // Xs is reloaded by the next item
        }
    }
    if (failed && tid == 0) atomicExch(err, 1ull);
    if (tid == 0) tc::bulk_wait_all();
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// N x N column-major FP64 matrix viewed in the boxes of the column (Lc) or row
// (Lr) tile layout.
int encode_tile_map(CUtensorMap* m, const double* base, int N, bool lr) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) { set_error_msg("cuTensorMapEncodeTiled is not available"); return MPJ_CUDA_ERROR; }
    cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)N};
    cuuint64_t strides[1] = {(cuuint64_t)N * sizeof(double)};
    cuuint32_t box[2] = {lr ? 16u : (cuuint32_t)kSlab, lr ? (cuuint32_t)kSlab : 32u};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(base), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, lr ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_error_msg("cuTensorMapEncodeTiled failed (FP64 tile map)"); return MPJ_CUDA_ERROR; }
    return MPJ_SUCCESS;
}

int sm_count() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        v = 148;
    return v;
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
                                      (int)solve_smem(InnerLayout<double, kM>::bytes)));
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_pass_tc64<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPassSmem));
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_pass_tc64<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPassSmem));
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
                k_solve2_tc64<<<K, kSolveThreads, solve_smem(InnerLayout<double, kM>::bytes), s>>>(
                    T, N, Fbuf[set], Sbuf[set], Fpl[set], fmax[set], r, eps_skip, tau, gate, max_inner, xs, rot);
            }
            MPJ_LAUNCH_CHECK("k_solve2_tc64");
            {
                MPJ_PROF(PC_TCP1_F64, s);
                k_pass_tc64<true><<<gridT, kThr, kPassSmem, s>>>(m1, N, n_slabs, items, perT, Fpl[set], fmax[set],
                                                                  nullptr, r, 0, rot + 1);
            }
            MPJ_LAUNCH_CHECK("k_pass_tc64 pass 1");
            {
                MPJ_PROF(PC_TCP2_F64, s);
                k_pass_tc64<false><<<gridT, kThr, kPassSmem, s>>>(m2, N, n_slabs, items, perT, Fpl[set], fmax[set],
                                                                   Sbuf[set], r, 0, rot + 1);
            }
            MPJ_LAUNCH_CHECK("k_pass_tc64 pass 2");
            MPJ_TRY(side.after_solve());                 // V joins after pass 2 (overlaps the next solve)
            {
                MPJ_PROF(PC_TCV_F64, side.sv);
                k_pass_tc64<false><<<gridV, kThr, kPassSmem, side.sv>>>(mv, N, n_slabs, items, perV, Fpl[set],
                                                                         fmax[set], nullptr, r, 1, rot + 1);
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
