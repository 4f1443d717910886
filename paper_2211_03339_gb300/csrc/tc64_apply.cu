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

#include <cuda.h>

#include "internal.h"
#include "engine_device.cuh"
#include "tc_device.cuh"
#include "slice_device.cuh"

namespace mpj {

using namespace slice;

namespace {

constexpr int kB = 32;                       // block size b
constexpr int kM = 2 * kB;                   // pair width = K = N of the MMA
constexpr int kSlab = 128;                   // tile rows = M of the MMA
constexpr int kThr = 576;                    // pass kernel: 18 warps (see k_pass_tc64)
constexpr int kSlicers = 256, kEpi = 256;    // threads of the slicer and epilogue roles
constexpr int kS = 8;                        // digits (slices) per operand
constexpr int kXBytes = kSlab * kM * 8;      // FP64 tile, 64 KB
constexpr int kAPlane = kSlab * 128;         // A digit plane: 128 rows x 64 bf16
constexpr int kBPlane = kM * 128;            // B digit plane: 64 rows x 64 bf16
constexpr int kFplBytes = kS * kBPlane + 256;   // per pair: 8 planes + 64 exponents
constexpr int kOffX = 0;                     // two X stages
constexpr int kOffA = 2 * kXBytes;           // two A plane slots
constexpr int kOffB = kOffA + 2 * kAPlane;   // the 8 B planes and column exponents
constexpr int kOffE = kOffB + kS * kBPlane;   // column exponents, one copy per X stage
constexpr size_t kPassSmem = (size_t)kOffE + 2 * 256 + 1024;
// Byte offset of 16-byte chunk j (elements 8j..8j+7 along K) of row r in a
// K-major operand of 128-byte rows with the 128-byte swizzle.
__device__ __forceinline__ int sw_chunk(int r, int j) {
    return (r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4);
}

// The eight levels T_d (exact integers in FP32, |T_d| < 2^22) as one 64-bit
// integer sum_d T_d 2^(42 - 7 d) (T_7 truncated by 2^-7).  A float v with
// |v| < 2^22 added to 1.5 * 2^23 has the bit pattern 0x4B400000 + v, so the
// lower levels are summed as bit patterns with 32 x 32 -> 64-bit multiply-adds
// and the constant part is removed once; the two upper levels go into the
// upper word.
__device__ __forceinline__ long long combine8(const float (&a)[8]) {
    constexpr unsigned long long kMagic = 0x4B400000ull;
    uint32_t u[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) u[d] = __float_as_uint(__fadd_rn(a[d], 12582912.0f));
    // levels 2..6 as bit patterns: sum u_d 2^(42 - 7 d) < 2^60; level 7 truncated
    unsigned long long lo = (unsigned long long)(u[7] >> 7);
    lo += (unsigned long long)u[6];
    lo += (unsigned long long)u[5] << 7;
    lo += (unsigned long long)u[4] << 14;
    lo += (unsigned long long)u[3] << 21;
    lo += (unsigned long long)u[2] << 28;
    constexpr unsigned long long kLoConst = (kMagic >> 7) + kMagic + (kMagic << 7) + (kMagic << 14) +
                                            (kMagic << 21) + (kMagic << 28);
    const long long t0 = (long long)u[0] - (long long)kMagic, t1 = (long long)u[1] - (long long)kMagic;
    return (long long)(lo - kLoConst) + (t0 << 42) + (t1 << 35);
}

// y = x + 2^(Er + Ec - 2100) S: the integer rounded to FP64 once, then one FMA
// with the exact power of two.  (An all-integer conversion that leaves a single
// FP64 addition measured slower: the FP64 unit is not the tile's limit.)
__device__ __forceinline__ double apply_level_sum(double x, long long S, int Er, int Ec) {
    if (S == 0) return x;
    const int be = Er + Ec - 1077;                   // biased exponent of the scale
    const double v = __ll2double_rn(S);
    if (be >= 1) return fma(v, __longlong_as_double((long long)be << 52), x);
    return x + scalbn(v, be - 1023);                 // tiny operands: not on the fast path
}

__device__ __forceinline__ void tmem_ld2(uint32_t taddr, float& v0, float& v1) {
    uint32_t r0, r1;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(taddr));
    v0 = __uint_as_float(r0);
    v1 = __uint_as_float(r1);
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
    uint64_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = scaled_signed(x[e], cls);
#pragma unroll
    for (int p = 0; p < kS; ++p)
        *reinterpret_cast<uint4*>(dst + p * kBPlane + sw_chunk(c, j)) =
            make_uint4(digit_pair(v[0], v[1], p), digit_pair(v[2], v[3], p), digit_pair(v[4], v[5], p),
                       digit_pair(v[6], v[7], p));
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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

// Named barrier over `count` threads that also ORs a predicate across them, so
// that every thread of a role takes the same decision.
__device__ __forceinline__ bool bar_or(int id, int count, bool p) {
    uint32_t r;
    asm volatile(
        "{\n.reg .pred pi, po;\nsetp.ne.u32 pi, %1, 0;\nbar.red.or.pred po, %2, %3, pi;\nselp.u32 %0, 1, 0, po;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)p), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

// Wait for phase `parity` of an mbarrier: try_wait polls, each of which may
// suspend the thread for a short, system-defined time.
__device__ __forceinline__ bool mbar_poll(uint64_t* bar, uint32_t parity, int polls) {
    uint32_t done = 0;
    for (int it = 0; it < polls && !done; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(tc::smem_u32(bar)), "r"(parity)
            : "memory");
    }
    return done != 0;
}

// Bounded wait (a few million polls, seconds at most) that gives up early once
// another role has recorded a failure.
__device__ __forceinline__ bool wait_or_fail(uint64_t* bar, uint32_t parity, volatile int* failed) {
    for (int r = 0; r < 256; ++r) {
        if (mbar_poll(bar, parity, 16384)) return true;
        if (*failed) return false;
    }
    *failed = 1;
    return false;
}

__device__ __forceinline__ bool item_taken(int it, int n_slabs, int skip_identity, const float* __restrict__ fmax,
                                           int& b, int& s) {
    b = it / n_slabs;
    s = it - b * n_slabs;
    return !(skip_identity && fmax[b] == 0.f);
}

// Warp-specialised, software-pipelined pass (one CTA per SM; the eight level
// accumulators take the whole TMEM):
//   warp 0     producer: TMA loads of the FP64 tiles into a 2-stage ring, and
//              the digit planes of F_b (one bulk copy) when the pair changes;
//   warp 1     MMA issuer (one thread): for each digit plane s of the tile the
//              products (s, t), t <= 7 - s, into the level accumulators s + t, as
//              MMAs with N = 64 g over groups of g <= 4 consecutive B planes (12
//              MMAs per K step of 16; a single thread issuing 36 MMAs of N = 64
//              per K step was the tile's bottleneck);
//   warps 2-9  slicers: per tile row, the row exponent class, then the 8 digit
//              planes one by one into a 2-slot ring;
//   warps 10-17 epilogue: the levels of its 32 columns folded into 64-bit
//              integers (TMEM is then released to the next tile's MMAs), then
//              y = x + 2^e S in place in the tile's stage and one TMA store.
// Items are (slab s, pair b), b-major; CTA k takes items [k per_cta, (k+1)
// per_cta).  With skip_identity, items whose W_b is the identity are skipped
// (in place V); otherwise they are copied.  With Sbuf, rows in IJ_b take the
// solver's rotated block.  Every wait is bounded: a timeout sets *err and the
// roles leave their loops.
template <bool kLr>
__global__ void __launch_bounds__(kThr, 1)
k_pass_tc64(const __grid_constant__ Tc64Maps maps, int N, int n_slabs, int total, int per_cta,
            const unsigned char* __restrict__ Fpl, const float* __restrict__ fmax,
            const double* __restrict__ Sbuf, int round, int skip_identity, unsigned long long* __restrict__ err) {
    extern __shared__ unsigned char smraw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) &
                                                         ~uintptr_t(1023));
    unsigned char* Xst = sm + kOffX;
    unsigned char* Ap = sm + kOffA;
    unsigned char* Bp = sm + kOffB;
    unsigned char* Ec = sm + kOffE;                 // stage st: 64 ints at Ec + 256 st
    __shared__ __align__(8) uint64_t xfull[2], xempty[2], afull[2], aempty[2], rowx[2], accfull, accempty;
    __shared__ uint32_t tmem_slot;
    __shared__ int exr[2][kSlab];
    __shared__ volatile int failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nblocks = N / kB;
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&xfull[i], 1);
            tc::mbar_init(&xempty[i], 1);
            tc::mbar_init(&afull[i], kSlicers);
            tc::mbar_init(&aempty[i], 1);
            tc::mbar_init(&rowx[i], kSlicers);
        }
        tc::mbar_init(&accfull, 1);
        tc::mbar_init(&accempty, kEpi);
        tc::fence_mbar_init();
        failed = 0;
    }
    if (warp == 1) tc::tmem_alloc(&tmem_slot, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const int it0 = blockIdx.x * per_cta;
    const int it1 = min(total, it0 + per_cta);

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int k = 0, cur = -1;
            for (int it = it0; it < it1; ++it) {
                int b, s;
                if (!item_taken(it, n_slabs, skip_identity, fmax, b, s)) continue;
                const int st = k & 1;
                if (k >= 2 && !wait_or_fail(&xempty[st], ((k >> 1) - 1) & 1, &failed)) break;
                const bool needF = b != cur;
                // the B planes are overwritten only once the previous tile's MMAs are done
                if (needF && k >= 1 && !wait_or_fail(&accfull, (k - 1) & 1, &failed)) break;
                int I, J;
                round_pair(round, b, nblocks, I, J);
                // the exponents go with every tile (the epilogue of the previous tile of
                // this stage has released them); the planes only when the pair changes
                const unsigned char* src = Fpl + (size_t)b * kFplBytes;
                tc::mbar_expect_tx(&xfull[st], kXBytes + 256 + (needF ? kS * kBPlane : 0));
                bulk_load(Ec + 256 * st, src + kS * kBPlane, 256, &xfull[st]);
                if (needF) {
                    bulk_load(Bp, src, kS * kBPlane, &xfull[st]);
                    cur = b;
                }
                tile_io<kLr>(&maps.in, true, Xst + st * kXBytes, s * kSlab, I, J, &xfull[st]);
                ++k;
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            // descriptors of the slot and plane bases; a K step or another plane only
            // moves the start-address field (address / 16, no carry: smem < 256 KB)
            const uint64_t adesc0 = tc::smem_desc_sw128(tc::smem_u32(Ap));
            const uint64_t bdesc0 = tc::smem_desc_sw128(tc::smem_u32(Bp));
            int k = 0;
            uint32_t q = 0;
            bool ok = true;
            for (int it = it0; it < it1 && ok; ++it) {
                int b, s;
                if (!item_taken(it, n_slabs, skip_identity, fmax, b, s)) continue;
                if (k >= 1 && !wait_or_fail(&accempty, (k - 1) & 1, &failed)) break;
                tc::fence_after_sync();
                for (int sa = 0; sa < kS; ++sa, ++q) {
                    const int slot = q & 1;
                    if (!wait_or_fail(&afull[slot], (q >> 1) & 1, &failed)) { ok = false; break; }
                    tc::fence_after_sync();
                    const uint64_t ad = adesc0 + (uint64_t)(slot * (kAPlane >> 4));
                    // The 8 B planes lie one after another (64 rows each, 1024-byte row
                    // groups throughout), i.e. they form one K-major operand of 512 rows,
                    // and level s + t sits at TMEM column 64 (s + t): the products of this
                    // A plane with B planes t0 .. t0 + g - 1 are ONE MMA with N = 64 g and
                    // D at column 64 (s + t0).  Groups of at most 4 planes (N <= 256).
                    for (int t0 = 0; t0 + sa < kS; t0 += 4) {
                        const int g = min(4, kS - sa - t0);
                        const uint32_t idesc = tc::instr_desc(tc::kFmtBF16, kSlab, kM * g);
                        const uint64_t bd = bdesc0 + (uint64_t)(t0 * (kBPlane >> 4));
                        const uint32_t dcol = tmem + (uint32_t)((sa + t0) * kM);
#pragma unroll
                        for (int ks = 0; ks < kM / 16; ++ks)
                            tc::mma_f16(dcol, ad + (uint64_t)(ks * 2), bd + (uint64_t)(ks * 2), idesc,
                                        (sa == 0 && ks == 0) ? 0u : 1u);
                    }
                    tc::commit(&aempty[slot]);
                }
                if (!ok) break;
                tc::commit(&accfull);
                ++k;
            }
        }
    } else if (warp < 10) {
        // ------------------------------------------------------------ slicers
        // lane pair (2r, 2r+1) of warp w holds row m = 16 (w - 2) + r, halves h = 0, 1
        const int m = 16 * (warp - 2) + (lane >> 1), h = lane & 1;
        int k = 0;
        uint32_t q = 0;
        bool bad = false;
        for (int it = it0; it < it1; ++it) {
            int b, s;
            if (!item_taken(it, n_slabs, skip_identity, fmax, b, s)) continue;
            const int st = k & 1;
            const bool ok = !bad && wait_or_fail(&xfull[st], (k >> 1) & 1, &failed);
            if (bar_or(1, kSlicers, !ok)) break;
            const unsigned char* X = Xst + st * kXBytes;
            int cls = 0;
#pragma unroll 8
            for (int c = 0; c < 32; ++c)
                cls = max(cls, exp_class(*reinterpret_cast<const double*>(X + xoff<kLr>(m, 32 * h + c))));
            cls = max(cls, __shfl_xor_sync(0xffffffffu, cls, 1));
            if (h == 0) exr[st][m] = cls;
            mbar_arrive(&rowx[st]);
            uint64_t Mb[32];
#pragma unroll
            for (int c = 0; c < 32; ++c)
                Mb[c] = scaled_signed(*reinterpret_cast<const double*>(X + xoff<kLr>(m, 32 * h + c)), cls);
#pragma unroll
            for (int sp = 0; sp < kS; ++sp, ++q) {
                const int slot = q & 1;
                if (!bad && q >= 2 && !wait_or_fail(&aempty[slot], ((q >> 1) - 1) & 1, &failed)) bad = true;
                if (!bad) {
                    unsigned char* A = Ap + slot * kAPlane;
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        *reinterpret_cast<uint4*>(A + sw_chunk(m, 4 * h + i)) = make_uint4(
                            digit_pair(Mb[8 * i], Mb[8 * i + 1], sp), digit_pair(Mb[8 * i + 2], Mb[8 * i + 3], sp),
                            digit_pair(Mb[8 * i + 4], Mb[8 * i + 5], sp), digit_pair(Mb[8 * i + 6], Mb[8 * i + 7], sp));
                    tc::fence_proxy_async();
                }
                mbar_arrive(&afull[slot]);
            }
            ++k;
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int quarter = warp & 3;
        const int m = 32 * quarter + lane;
        const int cb = 32 * ((warp - 10) >> 2);
        const uint32_t lanebase = tmem + ((uint32_t)(32 * quarter) << 16);
        int k = 0;
        for (int it = it0; it < it1; ++it) {
            int b, s;
            if (!item_taken(it, n_slabs, skip_identity, fmax, b, s)) continue;
            const int st = k & 1;
            bool ok = wait_or_fail(&accfull, k & 1, &failed);
            ok = ok && wait_or_fail(&rowx[st], (k >> 1) & 1, &failed);
            ok = ok && wait_or_fail(&xfull[st], (k >> 1) & 1, &failed);
            tc::fence_after_sync();
            if (bar_or(2, kEpi, !ok)) break;
            int I, J;
            round_pair(round, b, nblocks, I, J);
            const int row0 = s * kSlab;
            const int Er = exr[st][m];
            long long S[32];
#pragma unroll
            for (int c = 0; c < 32; c += 2) {
                float l0[kS], l1[kS];
#pragma unroll
                for (int d = 0; d < kS; ++d) tmem_ld2(lanebase + (uint32_t)(d * kM + cb + c), l0[d], l1[d]);
                tc::tmem_wait_ld();
                S[c] = combine8(l0);
                S[c + 1] = combine8(l1);
            }
            tc::fence_before_sync();
            mbar_arrive(&accempty);                  // TMEM is free for the next tile's MMAs
            const int row = row0 + m;
            const double* Srow = nullptr;
            if (Sbuf) {
                const int blk = row / kB;
                if (blk == I) Srow = Sbuf + (size_t)b * kM * kM + (size_t)(row % kB) * kM;
                else if (blk == J) Srow = Sbuf + (size_t)b * kM * kM + (size_t)(kB + row % kB) * kM;
            }
            unsigned char* X = Xst + st * kXBytes;
            const int* exc = reinterpret_cast<const int*>(Ec + 256 * st);
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                double* px = reinterpret_cast<double*>(X + xoff<kLr>(m, cb + c));
                double y = apply_level_sum(*px, S[c], Er, exc[cb + c]);
                if (Srow) y = Srow[cb + c];
                *px = y;
            }
            tc::fence_proxy_async();                 // the tile's generic writes -> TMA store
            bar_or(2, kEpi, false);
            if (tid == 10 * 32) {
                tile_io<kLr>(&maps.out, false, X, row0, I, J, nullptr);
                tc::bulk_commit();
                tc::bulk_wait_read();
                mbar_arrive(&xempty[st]);
            }
            ++k;
        }
        if (tid == 10 * 32) tc::bulk_wait_all();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (failed && tid == 0) atomicExch(err, 1ull);
    if (warp == 1) tc::tmem_dealloc(tmem, 512);
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
                                      (int)InnerLayout<double, kM>::bytes));
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
                k_solve2_tc64<<<K, kSolveThreads, InnerLayout<double, kM>::bytes, s>>>(
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
