// tc64_device.cuh -- the tensor-core FP64 tile pass shared by the two-sided
// sweeps (tc64_apply.cu) and the one-sided sweeps (tc64_onesided.cu): a 128-row
// slab X of the 64 columns of one block pair is replaced by Y = X + X F_b
// (W_b = I + F_b, 2b x 2b) with the product X F_b formed on the 5th-generation
// tensor cores (tcgen05, kind::f16, bf16 operands) from exact integer digits
// (the Ozaki scheme: Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012; the
// digit arithmetic is in slice_device.cuh).
//
// Two ways to scale the digits of X:
//   row scaling     (kColX = false) E_r = the largest exponent class of row r of
//                   X: y = x + 2^(E_r + E_c - 2100) S, E_c the class of column c
//                   of F (the rows of a symmetric T, the rows of V);
//   column scaling  (kColX = true)  E_k = the class of column k of the whole
//                   matrix (the largest over its rows), so that a column keeps
//                   its own relative accuracy next to much larger columns (the
//                   columns of C in one-sided Jacobi).  Then
//                   sum_k x_rk F_kc = 2^(E* - 1078) sum_k M_rk G_kc with
//                   G = diag(2^(E_k - E*)) F, E* = max_k E_k; the pair record
//                   carries the digits of G, its column classes folded with E*,
//                   and the E_k.
// Either way the eight level sums T_d = sum_{s+t=d} A_s B_t (exact integers in
// FP32, |T_d| < 2^22 for K = 64) become one 64-bit integer
// S = sum_d T_d 2^(42 - 7 d) (T_7 truncated by 2^-7) and y = x + 2^e S takes one
// FP64 FMA.  The dropped levels d >= 8 and the truncations are below
// 2^-54 K max|X_r:| max|F_:c| (row scaling), or 2^-54 K max_k 2^E_k |F_kc| per
// entry (column scaling): the order of an FP64 dot product's rounding error.
#pragma once

#include <cmath>
#include <cstdint>

#include <cuda.h>

#include "internal.h"
#include "jacobi_device.cuh"
#include "tc_device.cuh"
#include "slice_device.cuh"

namespace mpj {
namespace {

using namespace slice;

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
constexpr int kFplColBytes = kFplBytes + 256;   // column scaling: + the 64 E_k of X
constexpr int kOffX = 0;                     // two X stages
constexpr int kOffA = 2 * kXBytes;           // two A plane slots
constexpr int kOffB = kOffA + 2 * kAPlane;   // the 8 B planes
constexpr int kOffE = kOffB + kS * kBPlane;  // column exponents, one copy per X stage; then the E_k
constexpr size_t kPassSmem = (size_t)kOffE + 3 * 256 + 1024;

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

using tc::bulk_load;

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

using tc::mbar_arrive;

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
//   warps 2-9  slicers: per tile row, the row exponent class (row scaling), then
//              the 8 digit planes one by one into a 2-slot ring;
//   warps 10-17 epilogue: the levels of its 32 columns folded into 64-bit
//              integers (TMEM is then released to the next tile's MMAs), then
//              y = x + 2^e S in place in the tile's stage and one TMA store.
// Items are (slab s, pair b), b-major; CTA k takes items [k per_cta, (k+1)
// per_cta).  With skip_identity, items whose W_b is the identity are skipped
// (in place passes); otherwise they are copied.  With Sbuf, rows in IJ_b take
// the solver's rotated block.  With ncls_out (column scaling), the epilogue
// folds the exponent classes of its outputs into ncls_out[column] (atomicMax):
// the column classes of the next round.  Every wait is bounded: a timeout sets
// *err and the roles leave their loops.
template <bool kLr, bool kColX>
__global__ void __launch_bounds__(kThr, 1)
k_pass_tc64(const __grid_constant__ Tc64Maps maps, int N, int n_slabs, int total, int per_cta,
            const unsigned char* __restrict__ Fpl, const float* __restrict__ fmax,
            const double* __restrict__ Sbuf, int round, int skip_identity, unsigned long long* __restrict__ err,
            int* __restrict__ ncls_out) {
    static_assert(!(kLr && kColX), "column scaling reads the column layout");
    constexpr int kRec = kColX ? kFplColBytes : kFplBytes;
    extern __shared__ unsigned char smraw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) &
                                                         ~uintptr_t(1023));
    unsigned char* Xst = sm + kOffX;
    unsigned char* Ap = sm + kOffA;
    unsigned char* Bp = sm + kOffB;
    unsigned char* Ec = sm + kOffE;                 // stage st: 64 ints at Ec + 256 st
    const int* xcls = reinterpret_cast<const int*>(Ec + 512);   // column scaling: E_k of the pair
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
                // the B planes (and the E_k) are overwritten only once the previous
                // tile's MMAs are done, i.e. once its slicers are done too
                if (needF && k >= 1 && !wait_or_fail(&accfull, (k - 1) & 1, &failed)) break;
                int I, J;
                round_pair(round, b, nblocks, I, J);
                // the exponents go with every tile (the epilogue of the previous tile of
                // this stage has released them); the planes only when the pair changes
                const unsigned char* src = Fpl + (size_t)b * kRec;
                tc::mbar_expect_tx(&xfull[st],
                                   kXBytes + 256 + (needF ? kS * kBPlane + (kColX ? 256 : 0) : 0));
                bulk_load(Ec + 256 * st, src + kS * kBPlane, 256, &xfull[st]);
                if (needF) {
                    bulk_load(Bp, src, kS * kBPlane, &xfull[st]);
                    if constexpr (kColX) bulk_load(Ec + 512, src + kFplBytes, 256, &xfull[st]);
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
            uint64_t Mb[32];
            if constexpr (kColX) {
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    Mb[c] = scaled_signed(*reinterpret_cast<const double*>(X + xoff<kLr>(m, 32 * h + c)),
                                          xcls[32 * h + c]);
                mbar_arrive(&rowx[st]);
            } else {
                int cls = 0;
#pragma unroll 8
                for (int c = 0; c < 32; ++c)
                    cls = max(cls, exp_class(*reinterpret_cast<const double*>(X + xoff<kLr>(m, 32 * h + c))));
                cls = max(cls, __shfl_xor_sync(0xffffffffu, cls, 1));
                if (h == 0) exr[st][m] = cls;
                mbar_arrive(&rowx[st]);
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    Mb[c] = scaled_signed(*reinterpret_cast<const double*>(X + xoff<kLr>(m, 32 * h + c)), cls);
            }
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
            // column scaling: E* is folded into the record's column exponents
            const int Er = kColX ? 1023 : exr[st][m];
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
            int mycls = 0;                           // column scaling: class of column cb + lane
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                double* px = reinterpret_cast<double*>(X + xoff<kLr>(m, cb + c));
                double y = apply_level_sum(*px, S[c], Er, exc[cb + c]);
                if (Srow) y = Srow[cb + c];
                *px = y;
                if constexpr (kColX) {
                    const int cmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)exp_class(y));
                    if (lane == c) mycls = cmax;
                }
            }
            if constexpr (kColX) {
                if (mycls > 0) atomicMax(ncls_out + (cb + lane < kB ? I * kB + cb + lane : J * kB + cb + lane - kB),
                                         mycls);
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

inline EncodeTiledFn encode_fn() {
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

// rows x cols column-major FP64 matrix (leading dimension rows) viewed in boxes
// of box_rows x box_cols, optionally with the 128-byte swizzle (box_rows * 8
// must then be at most 128).  Rows outside the matrix are zero-filled on loads
// and clipped on stores.
inline int encode_fp64_map(CUtensorMap* m, const double* base, int rows, int cols, int box_rows, int box_cols,
                           bool swizzle) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) { set_error_msg("cuTensorMapEncodeTiled is not available"); return MPJ_CUDA_ERROR; }
    cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
    cuuint64_t strides[1] = {(cuuint64_t)rows * sizeof(double)};
    cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(base), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_error_msg("cuTensorMapEncodeTiled failed (FP64 tile map)"); return MPJ_CUDA_ERROR; }
    return MPJ_SUCCESS;
}

// N x N column-major FP64 matrix viewed in the boxes of the column (Lc) or row
// (Lr) tile layout.
inline int encode_tile_map(CUtensorMap* m, const double* base, int N, bool lr) {
    return lr ? encode_fp64_map(m, base, N, N, 16, kSlab, true) : encode_fp64_map(m, base, N, N, kSlab, 32, false);
}

inline int sm_count() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        v = 148;
    return v;
}

}  // namespace
}  // namespace mpj
