// ozaki.cu -- FP64 matrix products on the bf16 tensor cores (tcgen05 kind::f16)
// by exact splitting (the Ozaki scheme: Ozaki, Ogita, Oishi, Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 59, 2012).
//
// Each row i of op(A) is scaled by 2^(7 - e_i) (e_i the binary exponent of the
// row's largest |entry|, so the scaled row lies in (-128, 128)) and cut into
// S = 8 balanced integer slices of 7 bits from the FP64 bit patterns with
// integer operations (slice_device.cuh): a = sum_s a_s 2^(-7 s), |a_0| <= 128,
// a_s in [-64, 63].  Eight slices reach down to 2^-49 of the scaled row, i.e.
// 2^-56 of 2^e_i: every entry within 2^3 of the row maximum is cut exactly.
// Columns of op(B) likewise.  Integers of magnitude <= 128 are exact in bf16,
// their products exact in FP32, and
//
//   C_ij = 2^(e_i + f_j - 14) sum_d 2^(-7 d) T_d(i, j),
//   T_d  = sum_{s + t = d} sum_k a_s(i, k) b_t(k, j),     d = 0 .. 7,
//
// where the pairs with s + t >= 8 are dropped (each such product term is below
// 2^-55 of 2^(e_i + f_j)).  Each T_d is a sum of integers: per K element the
// pairs of one d add up to at most 2 * 2^13 + 6 * 2^12 = 2^15, so over a K block
// of 128 a partial sum stays below 2^22 and the FP32 tensor-core accumulation
// is exact; after every K block the eight FP32 accumulators are converted to
// int32 and added to eight int32 totals kept in TMEM (exact while K < 65536).
// FP64 arithmetic is used only once per output element, to combine the totals
// (Horner in 2^-7, exact up to the final rounding).  The result carries the
// dropped-pair error (at most about K 2^-55 max|A_i:| max|B_:j|), the order of
// the rounding error of an FP64 dot product; products of exactly sliced
// operands (e.g. permutations) come out exact.
//
// Kernel: one CTA per 128 x 32 tile of C; warp 4 streams the 8 + 8 slice planes
// of each K step of 32 with TMA (3-D boxes, 64-byte swizzle) into a 2-stage
// ring, warp 5 issues the slice products of a K step into eight 32-column TMEM
// accumulators (one MMA per A plane, its N spanning the B planes of all its
// levels), warps 0-3 drain each K block into the int32 totals and finally
// write C.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cuda.h>
#include <cuda_bf16.h>

#include "internal.h"
#include "tc_device.cuh"
#include "slice_device.cuh"

namespace mpj {

namespace {

constexpr int kS = 8;                // slices per operand
constexpr int kTM = 128, kTN = 32;   // tile of C
constexpr int kKS = 32;              // K per pipeline stage (64-byte rows of bf16)
constexpr int kKB = 4;               // stages per drained K block (K = 128)
constexpr int kStages = 2;
constexpr int kAPlane = kTM * kKS * 2;                    // bytes of one A slice plane per stage
constexpr int kBPlane = kTN * kKS * 2;
constexpr uint32_t kStageBytes = kS * (kAPlane + kBPlane); // 81920
constexpr size_t kGemmSmem = (size_t)kStages * kStageBytes + 1024;
constexpr int kAccCols = kS * kTN;   // FP32 accumulators, then the int32 totals
constexpr int kWait = 1 << 22;

struct OzMaps {
    CUtensorMap a, b;                // planes: {K, rows, 8}, box {32, kTM or kTN, 8}
};

// --------------------------------------------------------------- slicing
// The row exponent e_i is kept in frexp form (max |row| in [2^(e_i - 1), 2^e_i)):
// e_i = E_r - 1022 for the row's exponent class E_r.

// 8 consecutive entries of one row, sliced against class Er, as one 16-byte
// chunk per plane at P + p pstride.
__device__ __forceinline__ void slice8_store(const double (&x)[8], int Er, __nv_bfloat16* P, size_t pstride) {
    uint64_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = slice::scaled_signed(x[e], Er);
#pragma unroll
    for (int p = 0; p < kS; ++p)
        *reinterpret_cast<uint4*>(P + p * pstride) =
            make_uint4(slice::digit_pair(v[0], v[1], p), slice::digit_pair(v[2], v[3], p),
                       slice::digit_pair(v[4], v[5], p), slice::digit_pair(v[6], v[7], p));
}

// Rows contiguous: row r is X[r * rs + k], k < K.  One CTA (128 threads) per row;
// each thread slices 8 consecutive entries at a time.
__global__ void __launch_bounds__(128)
k_oz_slice_rows(const double* __restrict__ X, long long rs, int rows, int K, int Kp,
                __nv_bfloat16* __restrict__ P, long long pstride, int* __restrict__ ex) {
    __shared__ int red[4];
    const int r = blockIdx.x;
    const double* x = X + (size_t)r * rs;
    int cls = 0;
    for (int k = threadIdx.x; k < K; k += 128) cls = max(cls, slice::exp_class(x[k]));
    for (int o = 16; o > 0; o >>= 1) cls = max(cls, __shfl_xor_sync(0xffffffffu, cls, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cls;
    __syncthreads();
    cls = max(max(red[0], red[1]), max(red[2], red[3]));
    if (threadIdx.x == 0) ex[r] = cls - 1022;
    for (int k0 = 8 * threadIdx.x; k0 < Kp; k0 += 8 * 128) {
        double xv[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) xv[e] = k0 + e < K ? x[k0 + e] : 0.0;
        slice8_store(xv, cls, P + (size_t)r * Kp + k0, (size_t)pstride);
    }
}

// Rows of a column-major matrix (row r is X[r + k * ks]), in two passes: the row
// exponents (one thread per row; the reads of a warp are coalesced for each k),
// then 32-row x 64-column tiles transposed through shared memory so that the
// slice planes are written along k.
__global__ void __launch_bounds__(128)
k_oz_rowexp_strided(const double* __restrict__ X, long long ks, int rows, int K, int* __restrict__ ex) {
    const int r = blockIdx.x * 128 + threadIdx.x;
    if (r >= rows) return;
    int cls = 0;
    for (int k = 0; k < K; ++k) cls = max(cls, slice::exp_class(X[(size_t)r + (size_t)k * ks]));
    ex[r] = cls - 1022;
}

__global__ void __launch_bounds__(256)
k_oz_slice_tiled(const double* __restrict__ X, long long ks, int rows, int K, int Kp,
                 __nv_bfloat16* __restrict__ P, long long pstride, const int* __restrict__ ex) {
    __shared__ double tile[64][33];                          // [k][row]
    const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 64;
    const int tid = threadIdx.x;
    for (int i = tid; i < 32 * 64; i += 256) {
        const int rr = i % 32, kk = i / 32;
        const int r = r0 + rr, k = k0 + kk;
        tile[kk][rr] = (r < rows && k < K) ? X[(size_t)r + (size_t)k * ks] : 0.0;
    }
    __syncthreads();
    const int rr = tid / 8, kg = (tid % 8) * 8;              // 8 consecutive k per thread
    const int r = r0 + rr;
    const int kb = k0 + kg;
    if (r >= rows || kb + 8 > Kp) return;
    double xv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) xv[j] = tile[kg + j][rr];
    slice8_store(xv, ex[r] + 1022, P + (size_t)r * Kp + kb, (size_t)pstride);
}

// --------------------------------------------------------------- product
__device__ __forceinline__ void named_bar_drain() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t* r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
        "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
        "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
    d |= static_cast<uint64_t>(1) << 16;
    d |= static_cast<uint64_t>(512 >> 4) << 32;       // 8 rows x 64 bytes
    d |= static_cast<uint64_t>(1) << 46;
    d |= static_cast<uint64_t>(4) << 61;              // 64-byte swizzle
    return d;
}

// C = alpha * op(A) op(B) + beta * C for one 128 x 32 tile per CTA (192 threads).
__global__ void __launch_bounds__(192, 1)
k_oz_gemm(const __grid_constant__ OzMaps maps, const int* __restrict__ exA, const int* __restrict__ exB,
          double* __restrict__ C, int ldc, int M, int N, int K, double alpha, double beta, int nM, int nN,
          int upper_only, int* __restrict__ err) {
    extern __shared__ unsigned char smraw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) &
                                                         ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], accfull, accempty;
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // tile order: groups of 8 row tiles sweep all column tiles (operand reuse in L2)
    const int id = blockIdx.x;
    const int group = id / (8 * nN), m0 = group * 8;
    const int gsz = nM - m0 < 8 ? nM - m0 : 8;
    const int local = id % (8 * nN);
    const int mt = m0 + local % gsz, nt = local / gsz;
    // a tile strictly below the diagonal is not needed when the caller mirrors the upper triangle
    if (upper_only && nt * kTN + kTN - 1 < mt * kTM) return;
    const int nk = (K + kKS - 1) / kKS;
    const int nkb = (nk + kKB - 1) / kKB;
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) { tc::mbar_init(&full[i], 1); tc::mbar_init(&empty[i], 1); }
        tc::mbar_init(&accfull, 1);
        tc::mbar_init(&accempty, 1);
        tc::fence_mbar_init();
        failed = 0;
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;

    if (warp == 4) {
        if (lane == 0) {                                   // TMA producer
            for (int g = 0; g < nk; ++g) {
                const int slot = g % kStages;
                if (g >= kStages && !tc::mbar_wait(&empty[slot], ((g / kStages) - 1) & 1, kWait)) {
                    atomicExch(&failed, 1);
                    break;
                }
                unsigned char* st = sm + (size_t)slot * kStageBytes;
                tc::mbar_expect_tx(&full[slot], kStageBytes);
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
                        tc::smem_u32(st)),
                    "l"(&maps.a), "r"(g * kKS), "r"(mt * kTM), "r"(0), "r"(tc::smem_u32(&full[slot]))
                    : "memory");
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
                        tc::smem_u32(st + kS * kAPlane)),
                    "l"(&maps.b), "r"(g * kKS), "r"(nt * kTN), "r"(0), "r"(tc::smem_u32(&full[slot]))
                    : "memory");
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {                                   // MMA issuer
            bool ok = true;
            for (int kb = 0; kb < nkb && ok; ++kb) {
                if (kb > 0) {
                    ok = tc::mbar_wait(&accempty, (kb - 1) & 1, kWait);
                    tc::fence_after_sync();
                    if (!ok) break;
                }
                for (int st = 0; st < kKB; ++st) {
                    const int g = kb * kKB + st;
                    if (g >= nk) break;
                    const int slot = g % kStages;
                    if (!tc::mbar_wait(&full[slot], (g / kStages) & 1, kWait)) { ok = false; break; }
                    tc::fence_after_sync();
                    const uint32_t a0 = tc::smem_u32(sm + (size_t)slot * kStageBytes);
                    const uint32_t b0 = a0 + kS * kAPlane;
                    // The 8 B planes of the stage lie one after another (32 rows each,
                    // 512-byte row groups throughout): one K-major operand of 256 rows.
                    // Level s + t sits at TMEM column 32 (s + t), so the products of A
                    // plane s with B planes 0 .. 7 - s are one MMA with N = 32 (8 - s)
                    // and D at column 32 s (8 MMAs per K step of 16 instead of 36).
#pragma unroll
                    for (int ks = 0; ks < kKS / 16; ++ks) {
#pragma unroll
                        for (int s = 0; s < kS; ++s) {
                            const uint32_t acc = (st == 0 && ks == 0 && s == 0) ? 0u : 1u;
                            tc::mma_f16(tmem + s * kTN, desc_sw64(a0 + s * kAPlane + ks * 32),
                                        desc_sw64(b0 + ks * 32), tc::instr_desc(tc::kFmtBF16, kTM, kTN * (kS - s)),
                                        acc);
                        }
                    }
                    tc::commit(&empty[slot]);                // the stage is free once these complete
                }
                if (ok) tc::commit(&accfull);
            }
            if (!ok) atomicExch(&failed, 1);
        }
    } else {                                               // warps 0-3: drain and epilogue
        const uint32_t lanebase = tmem + ((uint32_t)(warp * 32) << 16);
        bool ok = true;
        for (int kb = 0; kb < nkb; ++kb) {
            ok = tc::mbar_wait(&accfull, kb & 1, kWait) && ok;
            tc::fence_after_sync();
            if (ok) {
                for (int d = 0; d < kS; ++d) {
                    uint32_t f[32], t[32];
                    tmem_ld32(lanebase + d * kTN, f);
                    if (kb > 0) tmem_ld32(lanebase + kAccCols + d * kTN, t);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        // |f| < 2^22: f + 1.5 2^23 has the bit pattern 0x4B400000 + f
                        const int v = (int)__float_as_uint(__fadd_rn(__uint_as_float(f[j]), 12582912.0f)) - 0x4B400000;
                        t[j] = kb > 0 ? (uint32_t)((int)t[j] + v) : (uint32_t)v;
                    }
                    tmem_st32(lanebase + kAccCols + d * kTN, t);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            }
            tc::fence_before_sync();
            named_bar_drain();
            if (tid == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&accempty)) : "memory");
        }
        // epilogue: C_ij = alpha 2^(e_i + f_j - 14) sum_d 2^(-7 d) T_d + beta C_ij.  The
        // levels are summed exactly as two integers, S_hi = sum_{d<4} T_d 2^(7 (3 - d))
        // and S_lo = sum_{d>=4} T_d 2^(7 (7 - d)) (|T_d| < 2^30: both below 2^52, exact
        // in FP64), so that sum_d 2^(-7 d) T_d = 2^-49 (S_hi 2^28 + S_lo) takes two
        // conversions and one FMA per element.
        const int row = mt * kTM + warp * 32 + lane;
        if (ok && nkb > 0) {
            const int ea = row < M ? exA[row] : 0;
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                long long hi[16], lo[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) { hi[j] = 0; lo[j] = 0; }
#pragma unroll
                for (int d = 0; d < kS; ++d) {
                    float tf[16];
                    tc::tmem_ld16(lanebase + kAccCols + d * kTN + 16 * h, tf);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const long long tv = (long long)__float_as_int(tf[j]);
                        if (d < 4) hi[j] = (hi[j] << 7) + tv;
                        else lo[j] = (lo[j] << 7) + tv;
                    }
                }
                if (row < M) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = nt * kTN + 16 * h + j;
                        if (col < N) {
                            const double sum = fma(__ll2double_rn(hi[j]), 268435456.0, __ll2double_rn(lo[j]));
                            const int e = ea + exB[col] - 63;
                            const double v = alpha * (e >= -1022 && e <= 1023
                                                          ? sum * __longlong_as_double((long long)(e + 1023) << 52)
                                                          : ldexp(sum, e));
                            double* cp = C + (size_t)row + (size_t)col * ldc;
                            *cp = beta != 0.0 ? fma(beta, *cp, v) : v;
                        }
                    }
                }
            }
        }
        if (!ok && tid == 0) atomicExch(&failed, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && failed) atomicOr(err, 2);               // bit 2: a tensor-core wait timed out
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// Mirror the upper triangle of the n x n matrix C onto the lower one.
__global__ void k_mirror_upper(double* __restrict__ C, int ldc, int n) {
    __shared__ double tile[32][33];
    const int bi = blockIdx.y, bj = blockIdx.x;            // tile row, tile column
    if (bi < bj) return;                                   // lower-triangle tiles (bi >= bj) only
    const int tx = threadIdx.x, ty = threadIdx.y;          // 32 x 8
    for (int r = ty; r < 32; r += 8) {                     // read the upper tile (bj, bi):
        const int i = bj * 32 + tx, j = bi * 32 + r;       // tile[r][tx] = C(bj*32 + tx, bi*32 + r)
        tile[r][tx] = (i < n && j < n) ? C[(size_t)i + (size_t)j * ldc] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {                     // C(bi*32 + tx, bj*32 + r) = C(bj*32 + r, bi*32 + tx)
        const int i = bi * 32 + tx, j = bj * 32 + r;
        if (i < n && j < n && i > j) C[(size_t)i + (size_t)j * ldc] = tile[tx][r];
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn oz_encode_fn() {
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

int encode_planes(CUtensorMap* m, const __nv_bfloat16* P, int K, int Kp, int rows, int box_rows) {
    EncodeTiledFn enc = oz_encode_fn();
    if (!enc) { set_error_msg("cuTensorMapEncodeTiled is not available"); return MPJ_CUDA_ERROR; }
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)kS};
    cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * 2 * (cuuint64_t)rows};
    cuuint32_t box[3] = {(cuuint32_t)kKS, (cuuint32_t)box_rows, (cuuint32_t)kS};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(P), dims, strides, box,
                     es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_error_msg("cuTensorMapEncodeTiled failed (slice planes)"); return MPJ_CUDA_ERROR; }
    return MPJ_SUCCESS;
}

size_t planes_bytes(int rows, int K) { return (size_t)kS * rows * (size_t)round_up(K, 8) * 2; }

}  // namespace

size_t oz_operand_bytes(int rows, int K) { return planes_bytes(rows, K) + sizeof(int) * (size_t)rows + 1024; }

int oz_operand(void* base, int rows, int K, OzOperand* op) {
    if (!base) return MPJ_BAD_ARG;
    char* p = static_cast<char*>(base);
    op->planes = reinterpret_cast<__nv_bfloat16*>(p);
    op->ex = reinterpret_cast<int*>(p + ((planes_bytes(rows, K) + 255) & ~size_t(255)));
    op->rows = rows;
    op->K = K;
    return MPJ_SUCCESS;
}

bool oz_supported(int M, int N, int K) { return M >= 1 && N >= 1 && K >= 1 && K <= 32768; }

int oz_slice(const double* X, long long row_stride, long long k_stride, int rows, int K, OzOperand* op,
             cudaStream_t s) {
    const int Kp = round_up(K, 8);
    const long long pstride = (long long)rows * Kp;
    op->rows = rows;
    op->K = K;
    {
        MPJ_PROF(PC_OZ_SLICE, s);
        if (k_stride == 1) {
            k_oz_slice_rows<<<rows, 128, 0, s>>>(X, row_stride, rows, K, Kp, op->planes, pstride, op->ex);
        } else {
            k_oz_rowexp_strided<<<(rows + 127) / 128, 128, 0, s>>>(X, k_stride, rows, K, op->ex);
            dim3 g((rows + 31) / 32, (Kp + 63) / 64);
            k_oz_slice_tiled<<<g, 256, 0, s>>>(X, k_stride, rows, K, Kp, op->planes, pstride, op->ex);
        }
    }
    MPJ_LAUNCH_CHECK("k_oz_slice");
    return MPJ_SUCCESS;
}

int oz_gemm(const OzOperand& A, const OzOperand& B, double alpha, double beta, double* C, int ldc,
            bool upper_mirror, int* d_flag, cudaStream_t s) {
    const int M = A.rows, N = B.rows, K = A.K;
    if (B.K != K || !oz_supported(M, N, K)) { set_error_msg("oz_gemm: bad shapes"); return MPJ_BAD_ARG; }
    OzMaps maps;
    MPJ_TRY(encode_planes(&maps.a, A.planes, K, round_up(K, 8), M, kTM));
    MPJ_TRY(encode_planes(&maps.b, B.planes, K, round_up(K, 8), N, kTN));
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem));
    const int upper_only = upper_mirror && M == N ? 1 : 0;
    const int nM = (M + kTM - 1) / kTM, nN = (N + kTN - 1) / kTN;
    {
        MPJ_PROF(PC_OZ_GEMM, s);
        k_oz_gemm<<<nM * nN, 192, kGemmSmem, s>>>(maps, A.ex, B.ex, C, ldc, M, N, K, alpha, beta, nM, nN, upper_only,
                                                       d_flag);
    }
    MPJ_LAUNCH_CHECK("k_oz_gemm");
    if (upper_mirror && M == N) {
        MPJ_PROF(PC_AUX, s);
        dim3 g((N + 31) / 32, (N + 31) / 32);
        k_mirror_upper<<<g, dim3(32, 8), 0, s>>>(C, ldc, N);
    }
    MPJ_LAUNCH_CHECK("k_mirror_upper");
    return MPJ_SUCCESS;
}

}  // namespace mpj
