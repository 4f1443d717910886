// tc64_onesided.cu -- the FP64 one-sided block Jacobi sweeps (Algorithm 5.1;
// steps 4-10 of Algorithm 5.2) with the block Gram matrices and the block
// rotations on the 5th-generation tensor cores by exact splitting.
//
// For every block pair (I, J) of a round of the parallel order:
//   k_gram_tc64    G = C_IJ^T C_IJ (2b x 2b, K = m), split over row ranges;
//   k_solve1_tc64  cyclic Jacobi on G with the rotations of Lemma 5.1 (a pair
//                  is rotated while |g_ij| > tol sqrt(g_ii g_jj)), W = I + F,
//                  and F cut into the digit records of the two passes;
//   C pass         C_IJ <- C_IJ W (k_pass_tc64, column scaling), in place;
//   V pass         V_IJ <- V_IJ W (k_pass_tc64, row scaling), in place, on a
//                  side stream.
//
// Exact digits (slice_device.cuh) with one scale per column of C: E_j is the
// largest exponent class over column j (the C pass's epilogue folds the
// classes of its outputs into the next round's E_j), x = 2^(E_j - 1078) M,
// M = sum_s a_s 2^(49 - 7 s).  With A_s the digit planes of C_IJ^T (64 pair
// columns x 64 rows of C per chunk) the Gram levels are
//
//   T_d = sum_{s + t = d} A_s A_t^T,   d = 0 .. 7,
//   G_ij = 2^(E_i + E_j - 2107) (hi 2^28 + lo),
//   hi = sum_{d<4} T_d 2^(7 (3 - d)),   lo = sum_{d>=4} T_d 2^(7 (7 - d)).
//
// Per row of C a level grows by at most 2^14 + 6 2^12 = 10 2^12, so over the
// 256 rows between two drains |T_d| < 10 2^20 < 2^24 (exact in the FP32 TMEM
// accumulators and in their conversion to int32), and over at most 8192 rows
// per CTA the int32 totals stay below 2^29 and hi, lo below 2^50 (exact in
// FP64).  A CTA writes the integers hi and lo of its row range; the solve adds
// them over the row ranges exactly (64-bit integers) and rounds
// 2^(E_i + E_j - 2107) (hi 2^28 + lo) to FP64 once.  The dropped levels
// d >= 8 and the truncated digits put an error of at most about
// 2^-54 (||c_i||_1 max|c_j| + ||c_j||_1 max|c_i|) on g_ij, independent of the
// other columns' scales: the cosines that decide the rotations are accurate to
// about 2^-54 sqrt(m) at worst.
#include <cmath>
#include <cstdio>

#include <cooperative_groups.h>

#include "internal.h"
#include "tc64_device.cuh"

namespace cg = cooperative_groups;

namespace mpj {

namespace {

constexpr int kGRows = 64;                   // rows of C per chunk (K of the Gram MMAs)
constexpr int kGBox = 16 * 32 * 8;           // TMA box: 16 rows x 32 columns with the 128-byte swizzle
constexpr int kGXBytes = 8 * kGBox;          // one chunk: 64 rows x 64 columns, 32 KB
constexpr int kGPlane = kM * 128;            // digit plane: 64 pair columns x 64 rows of bf16
constexpr int kGSlot = kS * kGPlane;         // the 8 planes of a chunk, 64 KB
constexpr int kGDrain = 4;                   // chunks between drains (256 rows)
constexpr int kGMaxRows = 8192;              // rows per CTA (bounds of the integer totals)
constexpr int kGThr = 448;                   // warp 0 TMA, 1 MMA, 2-9 slicers, 10-13 drain
constexpr int kGDrainThr = 128;
constexpr int kGramCtas = 152;               // target CTA count of a Gram launch (one per SM)
constexpr size_t kGramSmem = 2 * (size_t)kGXBytes + 2 * (size_t)kGSlot + 1024;
constexpr int kNoMixed = 1 << 20;            // k_solve1_tc64: S stays FP64

__device__ __forceinline__ void tmem_ld16u(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_st16u(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
__device__ __forceinline__ void tmem_ld8u(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(taddr));
}

// x * 2^e, exact for results in the normal range.
__device__ __forceinline__ double times_pow2(double x, int e) {
    if (e >= -1022 && e <= 1023) return x * __longlong_as_double((long long)(e + 1023) << 52);
    return ldexp(x, e);
}

// ---------------------------------------------------------------- Gram kernel
// One CTA per (pair b, row range split); a pair's 64 columns over its rows:
//   warp 0     producer: per chunk of 64 rows, eight TMA boxes (16 rows x 32
//              columns, 128-byte swizzle) into a 2-stage ring;
//   warp 1     MMA issuer: for each digit plane s the products (s, t),
//              t <= 7 - s, as MMAs with M = 64 (the pair's columns), N = 64 g
//              over groups of g <= 4 consecutive planes and K = 64 rows, into
//              level s + t at TMEM column 64 (s + t);
//   warps 2-9  slicers: thread (column c, 8-row chunk j) cuts 8 entries into
//              the 8 planes (K-major, 128-byte swizzle);
//   warps 10-13 drain: every 4 chunks the FP32 levels (TMEM lanes 0-15 of each
//              lane quarter: the M = 64 accumulator) are converted to int32 and
//              added to totals kept in the lanes 16-31 that the M = 64 MMAs do
//              not use; at the end the totals become the integers hi and lo
//              of G_ij = 2^(E_i + E_j - 2107) (hi 2^28 + lo) for this row range.
// Every wait is bounded; a timeout sets *err and the roles leave their loops.
__global__ void __launch_bounds__(kGThr, 1)
k_gram_tc64(const __grid_constant__ CUtensorMap map, int m, int N, int round, int rows_per,
            const int* __restrict__ ncls, long long* __restrict__ Ghi, long long* __restrict__ Glo,
            unsigned long long* __restrict__ err) {
    extern __shared__ unsigned char smraw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) &
                                                         ~uintptr_t(1023));
    unsigned char* Xst = sm;                          // 2 chunk stages
    unsigned char* Pst = sm + 2 * kGXBytes;           // 2 plane slots
    __shared__ __align__(8) uint64_t xfull[2], xempty[2], pfull[2], pempty[2], accfull, accempty;
    __shared__ uint32_t tmem_slot;
    __shared__ int cls_s[kM];
    __shared__ volatile int failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.x, split = blockIdx.y, nsplit = gridDim.y;
    int I, J;
    round_pair(round, b, N / kB, I, J);
    const int r0 = split * rows_per;
    const int r1 = min(m, r0 + rows_per);
    const int nq = (r1 - r0 + kGRows - 1) / kGRows;
    if (tid < kM) cls_s[tid] = ncls[pair_global(tid, I, J, kB)];
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&xfull[i], 1);
            tc::mbar_init(&xempty[i], kSlicers);
            tc::mbar_init(&pfull[i], kSlicers);
            tc::mbar_init(&pempty[i], 1);
        }
        tc::mbar_init(&accfull, 1);
        tc::mbar_init(&accempty, kGDrainThr);
        tc::fence_mbar_init();
        failed = 0;
    }
    if (warp == 1) tc::tmem_alloc(&tmem_slot, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            for (int q = 0; q < nq; ++q) {
                const int st = q & 1;
                if (q >= 2 && !wait_or_fail(&xempty[st], ((q >> 1) - 1) & 1, &failed)) break;
                tc::mbar_expect_tx(&xfull[st], kGXBytes);
                const int row = r0 + q * kGRows;
                unsigned char* X = Xst + st * kGXBytes;
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int rq = 0; rq < 4; ++rq)
                        tc::tma_load_2d(X + (h * 4 + rq) * kGBox, &map, row + 16 * rq, (h ? J : I) * kB, &xfull[st]);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint64_t pdesc0 = tc::smem_desc_sw128(tc::smem_u32(Pst));
            for (int q = 0; q < nq; ++q) {
                const int slot = q & 1;
                const bool first = (q % kGDrain) == 0;
                if (first && q > 0 && !wait_or_fail(&accempty, ((q / kGDrain) - 1) & 1, &failed)) break;
                if (!wait_or_fail(&pfull[slot], (q >> 1) & 1, &failed)) break;
                tc::fence_after_sync();
                const uint64_t base = pdesc0 + (uint64_t)(slot * (kGSlot >> 4));
                for (int sa = 0; sa < kS; ++sa) {
                    const uint64_t ad = base + (uint64_t)(sa * (kGPlane >> 4));
                    for (int t0 = 0; t0 + sa < kS; t0 += 4) {
                        const int g = min(4, kS - sa - t0);
                        const uint32_t idesc = tc::instr_desc(tc::kFmtBF16, kM, kM * g);
                        const uint64_t bd = base + (uint64_t)(t0 * (kGPlane >> 4));
                        const uint32_t dcol = tmem + (uint32_t)((sa + t0) * kM);
#pragma unroll
                        for (int ks = 0; ks < kGRows / 16; ++ks)
                            tc::mma_f16(dcol, ad + (uint64_t)(ks * 2), bd + (uint64_t)(ks * 2), idesc,
                                        (first && sa == 0 && ks == 0) ? 0u : 1u);
                    }
                }
                tc::commit(&pempty[slot]);
                if (q % kGDrain == kGDrain - 1 || q == nq - 1) tc::commit(&accfull);
            }
        }
    } else if (warp < 10) {
        // ------------------------------------------------------------ slicers
        // item = (column c, chunk j of 8 rows); 8 consecutive lanes take 8
        // consecutive columns, so their 16-byte loads (swizzled by column) and
        // their plane stores (swizzled by row c) fall in distinct bank groups
        const int ts = tid - 64;
        for (int q = 0; q < nq; ++q) {
            const int st = q & 1;
            bool ok = wait_or_fail(&xfull[st], (q >> 1) & 1, &failed);
            ok = ok && (q < 2 || wait_or_fail(&pempty[st], ((q >> 1) - 1) & 1, &failed));
            if (bar_or(1, kSlicers, !ok)) break;
            const unsigned char* X = Xst + st * kGXBytes;
            unsigned char* P = Pst + st * kGSlot;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int item = ts + kSlicers * i;
                const int c = item & 63, j = item >> 6;
                const int cl = c & 31;
                const unsigned char* colp = X + ((c >> 5) * 4 + (j >> 1)) * kGBox + cl * 128;
                const int cls = cls_s[c];
                uint64_t v[8];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const double2 d2 =
                        *reinterpret_cast<const double2*>(colp + ((((j & 1) * 4 + e) ^ (cl & 7)) << 4));
                    v[2 * e] = scaled_signed(d2.x, cls);
                    v[2 * e + 1] = scaled_signed(d2.y, cls);
                }
#pragma unroll
                for (int p = 0; p < kS; ++p)
                    *reinterpret_cast<uint4*>(P + p * kGPlane + sw_chunk(c, j)) =
                        make_uint4(digit_pair(v[0], v[1], p), digit_pair(v[2], v[3], p), digit_pair(v[4], v[5], p),
                                   digit_pair(v[6], v[7], p));
            }
            tc::fence_proxy_async();
            mbar_arrive(&xempty[st]);
            mbar_arrive(&pfull[st]);
        }
    } else {
        // ------------------------------------------------------------ drain
        const int quarter = warp & 3;
        const uint32_t lanebase = tmem + ((uint32_t)(32 * quarter) << 16);
        const int ng = (nq + kGDrain - 1) / kGDrain;
        bool ok = true;
        for (int g = 0; g < ng; ++g) {
            const bool got = wait_or_fail(&accfull, g & 1, &failed);
            tc::fence_after_sync();
            if (bar_or(2, kGDrainThr, !got)) { ok = false; break; }
            for (int d = 0; d < kS; ++d) {
#pragma unroll
                for (int cg = 0; cg < kM / 16; ++cg) {
                    const uint32_t ta = lanebase + (uint32_t)(d * kM + 16 * cg);
                    uint32_t v[16];
                    tmem_ld16u(ta, v);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        // lane 16 + r receives the level of row r from lane r
                        const uint32_t a = __shfl_up_sync(0xffffffffu, v[jj], 16);
                        if (lane >= 16) {
                            const int iv = __float2int_rn(__uint_as_float(a));
                            v[jj] = (uint32_t)(g == 0 ? iv : (int)v[jj] + iv);
                        }
                    }
                    tmem_st16u(ta, v);
                }
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc::fence_before_sync();
            mbar_arrive(&accempty);
        }
        if (ok && nq > 0) {
            const int i = 16 * quarter + (lane & 15);      // row i of G (pair column i)
            const size_t gbase = ((size_t)b * nsplit + split) * kM * kM;
            for (int c8 = 0; c8 < kM / 8; ++c8) {
                uint32_t T[kS][8];
#pragma unroll
                for (int d = 0; d < kS; ++d) tmem_ld8u(lanebase + (uint32_t)(d * kM + 8 * c8), T[d]);
                tc::tmem_wait_ld();
                if (lane >= 16) {
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) {
                        const int j = 8 * c8 + jj;
                        long long hi = 0, lo = 0;
#pragma unroll
                        for (int d = 0; d < 4; ++d) {
                            hi = hi * 128 + (long long)(int)T[d][jj];
                            lo = lo * 128 + (long long)(int)T[d + 4][jj];
                        }
                        Ghi[gbase + (size_t)j * kM + i] = hi;
                        Glo[gbase + (size_t)j * kM + i] = lo;
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (failed && tid == 0) atomicExch(err, 1ull);
    if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

// Largest exponent class of each column of the m x N matrix C (one warp per column).
__global__ void k_colcls(const double* __restrict__ C, int m, int N, int* __restrict__ ncls) {
    const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (col >= N) return;
    unsigned c = 0;
    for (int r = lane; r < m; r += 32) c = max(c, (unsigned)exp_class(C[(size_t)col * m + r]));
    c = __reduce_max_sync(0xffffffffu, c);
    if (lane == 0) ncls[col] = (int)c;
}

// ---------------------------------------------------------------- block solve
// Digit record of one pair from the thread's 8 entries x[e] = F(8 j + e, c)
// (threads 8c .. 8c + 7 hold column c): the column class (folded with `fold`),
// and the 8 digit planes in the swizzled layout of the passes' B operand.
__device__ __forceinline__ void slice_record(const double (&x)[8], int c, int j, int fold, unsigned char* dst) {
    int cls = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) cls = max(cls, exp_class(x[e]));
    cls = max(cls, __shfl_xor_sync(0xffffffffu, cls, 1));
    cls = max(cls, __shfl_xor_sync(0xffffffffu, cls, 2));
    cls = max(cls, __shfl_xor_sync(0xffffffffu, cls, 4));
    if (j == 0) reinterpret_cast<int*>(dst + kS * kBPlane)[c] = cls + fold;
    uint64_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = scaled_signed(x[e], cls);
#pragma unroll
    for (int p = 0; p < kS; ++p)
        *reinterpret_cast<uint4*>(dst + p * kBPlane + sw_chunk(c, j)) =
            make_uint4(digit_pair(v[0], v[1], p), digit_pair(v[2], v[3], p), digit_pair(v[4], v[5], p),
                       digit_pair(v[6], v[7], p));
}

// The 2b x 2b solve of pair b: the integer Gram totals of the row ranges summed
// exactly and rounded to FP64 once, cyclic Jacobi (Lemma 5.1 rotations, relative threshold tol_rot; with
// cross_round >= 0 the cross-pair inner schedule of inner_jacobi; with mixed,
// the FP32 off-diagonal of inner_jacobi_mixed where the diagonal range allows),
// W = I + F (re-orthogonalised when some |F| >= gate), then the two digit
// records: Fv = digits of F for the V pass (row scaling) and Fc = digits of
// G = diag(2^(E_k - E*)) F with E* folded into its column classes, plus the E_k,
// for the C pass (column scaling).  Columns of an identity W keep their class
// for the next round; the others get theirs from the C pass.  Launched as
// clusters of R CTAs per pair: each CTA repeats the cheap part (Gram sum, S
// updates, rotations; bit-identical in every CTA) and accumulates M/R rows of F
// in FP64, the part that bounds the solve; the leader gathers F through
// distributed shared memory and finishes alone.
__global__ void __launch_bounds__(kSolveThreads, 1)
k_solve1_tc64(const long long* __restrict__ Ghi, const long long* __restrict__ Glo, int nsplit, int N, int round,
              double* __restrict__ Fbuf, float* __restrict__ fmax, unsigned char* __restrict__ Fv,
              unsigned char* __restrict__ Fc, const int* __restrict__ ncls_cur, int* __restrict__ ncls_nxt,
              double tol_rot, double gate, int max_inner, int cross_round, int mixed,
              unsigned long long* __restrict__ rot_counter) {
    static_assert(kM * kM % kSolveThreads == 0, "entries per thread");
    constexpr int LD = kM + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    double* S = reinterpret_cast<double*>(smraw);
    double* F = S + kM * LD;
    double* G2 = F + kM * LD;
    double* cs = G2 + kM * LD;
    int* ip = reinterpret_cast<int*>(cs + InnerLayout<double, kM>::kRealRot);
    int* flag = ip + InnerLayout<double, kM>::kFlagOffset;
    __shared__ int xc[kM];
    __shared__ int ecmax_s, mixed_s;
    // R CTAs per pair (a cluster) form the same rotations; CTA `rank` accumulates
    // rows [rank M/R, (rank+1) M/R) of F, which are gathered in the leader
    cg::cluster_group cl = cg::this_cluster();
    const int R = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int nrows = kM / R, row0 = rank * nrows;
    const int b = blockIdx.x / R, t = threadIdx.x;
    int I, J;
    round_pair(round, b, N / kB, I, J);
    if (t < kM) xc[t] = ncls_cur[pair_global(t, I, J, kB)];
    const size_t off = (size_t)b * nsplit * kM * kM;
    __syncthreads();                                     // xc
    {
        // the row ranges' totals, exact: below 2^57 for m < 2^20 (16 loads in flight per thread)
        constexpr int kPer = kM * kM / kSolveThreads;
        long long hi[kPer], lo[kPer];
#pragma unroll
        for (int i = 0; i < kPer; ++i) { hi[i] = 0; lo[i] = 0; }
        for (int sp = 0; sp < nsplit; ++sp) {
            const size_t base = off + (size_t)sp * kM * kM;
#pragma unroll
            for (int i = 0; i < kPer; ++i) {
                hi[i] += __ldg(Ghi + base + t + kSolveThreads * i);
                lo[i] += __ldg(Glo + base + t + kSolveThreads * i);
            }
        }
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int q = t + kSolveThreads * i, r = q % kM, c = q / kM;
            const double v = fma(__ll2double_rn(hi[i]), 268435456.0, __ll2double_rn(lo[i]));
            S[c * LD + r] = times_pow2(v, xc[r] + xc[c] - 2107);
            F[c * LD + r] = 0.0;
        }
    }
    __syncthreads();
    // Mixed-precision solve (FP32 off-diagonal, inner_jacobi_mixed) when the
    // diagonal spans at most 2^76: scaled by 2^-e (2^e <= d_max < 2^(e+1)), every
    // entry above the threshold, |s_pq| > 2^-50 sqrt(s_pp s_qq) >= 2^-50 d_min,
    // is then a normal FP32 number.
    if (t < 32) {
        const double a0 = S[t * LD + t], a1 = S[(t + 32) * LD + t + 32];
        double mx = a0 > a1 ? a0 : a1;
        double mn = a0 > 0.0 ? a0 : INFINITY;
        if (a1 > 0.0 && a1 < mn) mn = a1;
        for (int o = 16; o > 0; o >>= 1) {
            const double ox = __shfl_xor_sync(0xffffffffu, mx, o), on = __shfl_xor_sync(0xffffffffu, mn, o);
            mx = ox > mx ? ox : mx;
            mn = on < mn ? on : mn;
        }
        if (t == 0) {
            const int e = mx > 0.0 ? ilogb(mx) : 0;
            mixed_s = mixed && mx > 0.0 && mn >= 0x1p-76 * mx && e >= -1000 && e <= 1000 ? e : kNoMixed;
        }
    }
    __syncthreads();
    int applied;
    if (mixed_s != kNoMixed) {
        const double sc = __longlong_as_double((long long)(1023 - mixed_s) << 52);
        double v[kM * kM / kSolveThreads];
#pragma unroll
        for (int i = 0; i < kM * kM / kSolveThreads; ++i) {
            const int q = t + kSolveThreads * i;
            v[i] = S[(q / kM) * LD + q % kM] * sc;
        }
        __syncthreads();
        const MixedBufs<kM> mb(reinterpret_cast<unsigned char*>(S));
        static_assert(MixedBufs<kM>::bytes <= sizeof(double) * kM * LD, "mixed buffers fit in S");
#pragma unroll
        for (int i = 0; i < kM * kM / kSolveThreads; ++i) {
            const int q = t + kSolveThreads * i, r = q % kM, c = q / kM;
            mb.E[c * LD + r] = (float)v[i];
            if (r == c) { mb.dg[r] = v[i]; mb.dgf[r] = (float)v[i]; }
        }
        __syncthreads();
        applied = inner_jacobi_mixed<kM>(mb, F, ip + 6 * (kM / 2), (float)tol_rot, max_inner, cross_round, row0,
                                         nrows);
    } else {
        applied = inner_jacobi<double, kM>(S, F, cs, ip, tol_rot, 0.0, max_inner, cross_round, row0, nrows);
    }
    if (R > 1) {
        cl.sync();                                       // every CTA past its zeroing of F
        if (rank != 0) {
            double* F0 = cl.map_shared_rank(F, 0);
            for (int q = t; q < kM * nrows; q += blockDim.x) {
                const int c = q / nrows, k = row0 + q % nrows;
                F0[c * LD + k] = F[c * LD + k];
            }
        }
        cl.sync();                                       // the leader holds all of F
        if (rank != 0) return;
    }
    finish_block<double, kM>(F, G2, Fbuf + (size_t)b * kM * kM, gate, flag, fmax + b);
    __syncthreads();
    const bool ident = __uint_as_float(reinterpret_cast<const unsigned*>(flag)[1]) == 0.f;
    if (t < kM) ncls_nxt[pair_global(t, I, J, kB)] = ident ? xc[t] : 0;
    if (t == 0) {
        int e = 0;
        for (int k = 0; k < kM; ++k) e = max(e, xc[k]);
        ecmax_s = e;
    }
    __syncthreads();
    // F(k, c) = F[c * LD + k]; thread t holds column c = t / 8, rows 8 j .. 8 j + 7
    const int c = t >> 3, j = t & 7;
    double x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) x[e] = F[c * LD + 8 * j + e];
    slice_record(x, c, j, 0, Fv + (size_t)b * kFplBytes);
    const int es = ecmax_s;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int d = xc[8 * j + e] - es;                 // <= 0
        x[e] = d >= -1022 ? x[e] * __longlong_as_double((long long)(d + 1023) << 52) : 0.0;
    }
    unsigned char* rc = Fc + (size_t)b * kFplColBytes;
    slice_record(x, c, j, es - 1023, rc);
    if (t < kM) reinterpret_cast<int*>(rc + kFplBytes)[t] = xc[t];
    if (t == 0 && applied) atomicAdd(rot_counter, (unsigned long long)applied);
}

void gram_split_tc(int m, int K, int* nsplit, int* rows_per) {
    const int want = kGramCtas / K > 1 ? kGramCtas / K : 1;
    const int chunks = (m + kGRows - 1) / kGRows;
    int per = (chunks + want - 1) / want;
    if (per > kGMaxRows / kGRows) per = kGMaxRows / kGRows;
    if (per < 1) per = 1;
    *rows_per = per * kGRows;
    *nsplit = (m + *rows_per - 1) / *rows_per;
}

}  // namespace

bool onesided_tc64_supported(int m, int N, int B) {
    return B == kB && N % kM == 0 && N >= kM && m >= kSlab && m % 2 == 0 && m < (1 << 20);
}

size_t onesided_tc64_workspace_bytes(int m, int N) {
    const size_t K = (size_t)(N / kM);
    int nsplit = 1, rows_per = kGRows;
    if (K > 0) gram_split_tc(m, (int)K, &nsplit, &rows_per);
    Arena a;
    for (int set = 0; set < 2; ++set) {
        a.take<double>(K * kM * kM);                // F
        a.take<float>(K);                           // max |F|
        a.take<unsigned char>(K * kFplBytes);       // V pass records
        a.take<unsigned char>(K * kFplColBytes);    // C pass records
    }
    a.take<long long>(K * nsplit * kM * kM);        // Gram totals per row range: hi
    a.take<long long>(K * nsplit * kM * kM);        //                            lo
    a.take<int>(2 * (size_t)N);                     // column classes, two rounds
    a.take<unsigned long long>(4);
    return a.used + 256;
}

int onesided_sweeps_tc64(double* C, double* V, int m, int N, int n, double tol_rot, double ju_ratio,
                         int max_sweeps, int max_inner, void* work, cudaStream_t s, SweepResult* res) {
    if (!onesided_tc64_supported(m, N, kB)) {
        set_error_msg("tensor-core one-sided engine: needs b = 32, N a multiple of 64, m even, 128 <= m < 2^20");
        return MPJ_BAD_ARG;
    }
    const int K = N / kM;
    int nsplit, rows_per;
    gram_split_tc(m, K, &nsplit, &rows_per);
    Arena ar;
    ar.base = static_cast<char*>(work);
    ar.size = onesided_tc64_workspace_bytes(m, N);
    double* Fbuf[2];
    float* fmax[2];
    unsigned char *Fv[2], *Fc[2];
    for (int set = 0; set < 2; ++set) {
        Fbuf[set] = ar.take<double>((size_t)K * kM * kM);
        fmax[set] = ar.take<float>((size_t)K);
        Fv[set] = ar.take<unsigned char>((size_t)K * kFplBytes);
        Fc[set] = ar.take<unsigned char>((size_t)K * kFplColBytes);
    }
    long long* Ghi = ar.take<long long>((size_t)K * nsplit * kM * kM);
    long long* Glo = ar.take<long long>((size_t)K * nsplit * kM * kM);
    int* ncls = ar.take<int>(2 * (size_t)N);
    unsigned long long* rot = ar.take<unsigned long long>(4);     // [0] rotations, [1] error flag
    if (!Fc[1] || !Ghi || !Glo || !ncls || !rot) {
        set_error_msg("workspace too small");
        return MPJ_BAD_ARG;
    }
    HostScratch hs;
    MPJ_TRY(hs.init());
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_gram_tc64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGramSmem));
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_solve1_tc64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)InnerLayout<double, kM>::bytes));
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_pass_tc64<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kPassSmem));
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_pass_tc64<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kPassSmem));
    CUtensorMap mg;
    Tc64Maps mc, mv;
    MPJ_TRY(encode_fp64_map(&mg, C, m, N, 16, 32, true));          // Gram: 16 x 32 boxes, swizzled
    MPJ_TRY(encode_fp64_map(&mc.in, C, m, N, kSlab, 32, false));   // C pass, in place
    mc.out = mc.in;
    MPJ_TRY(encode_tile_map(&mv.in, V, N, false));                 // V pass, in place
    mv.out = mv.in;
    SideStream side;
    MPJ_TRY(side.init(s));
    s = side.main;
    MPJ_CUDA_TRY(cudaMemsetAsync(rot, 0, 2 * sizeof(unsigned long long), s));
    k_colcls<<<(N + 7) / 8, 256, 0, s>>>(C, m, N, ncls);
    MPJ_LAUNCH_CHECK("k_colcls");
    res->sweeps = 0;
    res->rotations = 0;
    res->status = MPJ_NOT_CONVERGED;
    const int rounds = 2 * K - 1;
    const int nsm = sm_count();
    const int slabsC = (m + kSlab - 1) / kSlab, itemsC = slabsC * K;
    const int gridC = itemsC < nsm ? itemsC : nsm;
    const int perC = (itemsC + gridC - 1) / gridC;
    const int slabsV = (N + kSlab - 1) / kSlab, itemsV = slabsV * K;
    const int perV = 8;
    const int gridV = (itemsV + perV - 1) / perV;
    // Newton-Schulz re-orthogonalisation of W = I + F only when some |F| >= 2^-6:
    // F is accumulated with rounding relative to |F|, so below that W is
    // orthogonal to a few ulps (each NS step costs two 64^3 FP64 products, more
    // than the whole inner sweep)
    const double gate = 1.0 / 64.0;
    const double Npairs = 0.5 * (double)n * (double)(n - 1);
    // cross-pair inner schedule once the rounds of a sweep cover the intra-block tournament
    const bool cross = N >= kB * kB && !knobs().full_inner;
    const int mixed = knobs().fp64_solves ? 0 : 1;
    // CTAs per pair of a solve (cluster size): the largest of 8, 4, 2, 1 that keeps
    // the launch within one CTA per SM
    int R = 8;
    while (R > 1 && K * R > nsm) R >>= 1;
    long long g = 0;                                     // rounds so far: parity of the class buffers
    while (res->sweeps < max_sweeps) {
        MPJ_CUDA_TRY(cudaMemsetAsync(rot, 0, sizeof(unsigned long long), s));
        for (int r = 0; r < rounds; ++r, ++g) {
            const int set = side.begin_round();
            if (set < 0) return MPJ_CUDA_ERROR;
            int* nc = ncls + (g & 1) * N;
            int* nn = ncls + ((g + 1) & 1) * N;
            {
                MPJ_PROF(PC_GRAM_TC64, s);
                k_gram_tc64<<<dim3(K, nsplit), kGThr, kGramSmem, s>>>(mg, m, N, r, rows_per, nc, Ghi, Glo, rot + 1);
            }
            MPJ_LAUNCH_CHECK("k_gram_tc64");
            {
                MPJ_PROF(PC_SOLVE1_F64, s);
                cudaLaunchConfig_t cfg = {};
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = (unsigned)R;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.gridDim = dim3((unsigned)(K * R));
                cfg.blockDim = dim3(kSolveThreads);
                cfg.dynamicSmemBytes = InnerLayout<double, kM>::bytes;
                cfg.stream = s;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                MPJ_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_solve1_tc64, (const long long*)Ghi, (const long long*)Glo,
                                                nsplit, N, r, Fbuf[set], fmax[set], Fv[set], Fc[set],
                                                (const int*)nc, nn, tol_rot, gate, max_inner, cross ? r : -1, mixed,
                                                rot));
            }
            MPJ_LAUNCH_CHECK("k_solve1_tc64");
            MPJ_TRY(side.after_solve());
            {
                MPJ_PROF(PC_TCV1_F64, side.sv);
                k_pass_tc64<false, false><<<gridV, kThr, kPassSmem, side.sv>>>(
                    mv, N, slabsV, itemsV, perV, Fv[set], fmax[set], nullptr, r, 1, rot + 1, nullptr);
            }
            MPJ_LAUNCH_CHECK("k_pass_tc64 V (one-sided)");
            MPJ_TRY(side.after_v());
            {
                MPJ_PROF(PC_TCC_F64, s);
                k_pass_tc64<false, true><<<gridC, kThr, kPassSmem, s>>>(mc, N, slabsC, itemsC, perC, Fc[set],
                                                                        fmax[set], nullptr, r, 1, rot + 1, nn);
            }
            MPJ_LAUNCH_CHECK("k_pass_tc64 C");
            side.end_round();
        }
        MPJ_CUDA_TRY(cudaMemcpyAsync(hs.u, rot, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        MPJ_CUDA_TRY(cudaStreamSynchronize(s));
        prof_flush();
        if (hs.u[1]) { set_error_msg("tensor-core one-sided sweep: TMA or MMA wait timed out"); return MPJ_CUDA_ERROR; }
        res->sweeps += 1;
        res->rotations += (double)hs.u[0];
        if (trace_on())
            fprintf(stderr, "[mpj] onesided<tc64> m=%d n=%d sweep %d: %llu rotations (%.4f N)\n", m, n, res->sweeps,
                    hs.u[0], hs.u[0] / Npairs);
        const double applied = (double)hs.u[0];
        if (hs.u[0] == 0 || applied < ju_ratio * Npairs) { res->status = MPJ_SUCCESS; break; }
    }
    return MPJ_SUCCESS;
}

}  // namespace mpj
