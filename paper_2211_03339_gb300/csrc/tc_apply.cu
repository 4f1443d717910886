// tc_apply.cu -- the FP32 block Jacobi of step 1 of Algorithm 4.1 with the
// rotation application on the 5th-generation tensor cores (tcgen05, kind::tf32).
//
// A round of the parallel order replaces T by W^T T W and V by V W, where W is
// block diagonal over the disjoint block pairs (I, J) of the round (one 2b x 2b
// orthogonal block W_b = I + F_b per pair, from the block-pair solves).  Both
// are written as right multiplications of 128-row slabs by W_b:
//
//   pass 1   P = T W          P[rows, IJ_b] = T[rows, IJ_b] + T[rows, IJ_b] F_b
//   pass 2   T' = P^T W       (= W^T T W, as T is symmetric), and V' = V W
//
// Every tile is one 128 x 64 x 64 product on the tensor cores in delta form
// (X + X F), with X and F split into TF32 pairs (hi + lo) and the three
// products hi*hi + hi*lo + lo*hi accumulated in FP32 in TMEM, which carries
// about 21 bits of each product -- the accuracy of the FP32 SIMT products it
// replaces.  The operand X must be K-major (the 64 columns of the pair
// contiguous for each row): T is read through its transpose (T and P are
// column-major, so T^T[rows, IJ_b] is contiguous along IJ_b), and V is kept
// row-major (Vt = V^T column-major).  Pass 1 and pass 2 write column-major
// (each warp stores 32 consecutive rows of one column); V is written row-major
// through a shared-memory staging tile.
//
// Traffic per round: T and P are read and written once each, V read and written
// once: 6 N^2 floats.  The block-pair solves are the FP32 k_solve2 kernels of
// the SIMT engine, without writing the rotated block back (pass 1 and 2 rotate
// the diagonal blocks too).
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include <cuda.h>

#include "internal.h"
#include "engine_device.cuh"
#include "tc_device.cuh"

namespace mpj {

namespace {

constexpr int kSlab = 128;          // rows of one tile = M of the MMA
constexpr int kTcThreads = 128;     // warp w owns TMEM lanes 32w .. 32w+31 (rows)
constexpr int kTcWait = 1 << 22;    // mbarrier polls before a tile gives up
constexpr int kB = 32;              // block size b; pair width 2b = 64 = K = N of the MMA
constexpr int kM = 2 * kB;
// Threads of the FP32 block solves: an inner step is a chain of short
// dependent phases, and more warps hide more of their latency (measured at
// n = 4096: 256 threads 122 ms, 512 threads 78 ms, 1024 threads 74 ms of solves).
constexpr int kSolve32Threads = 1024;


__global__ void __launch_bounds__(kSolve32Threads)
k_solve2_nb(float* __restrict__ T, int N, float* __restrict__ Fbuf, float* __restrict__ Sbuf,
            float* __restrict__ Fimg, float* __restrict__ fmax, int round, float eps, float tau,
            float gate, int max_inner, int cross, unsigned long long* __restrict__ rot_counter) {
    extern __shared__ __align__(16) unsigned char smraw[];
    int applied = pair_solve<float, kB, false>(T, N, round, blockIdx.x, eps, tau, gate, max_inner,
                                               Fbuf + (size_t)blockIdx.x * kM * kM,
                                               fmax + blockIdx.x, smraw,
                                               Sbuf + (size_t)blockIdx.x * kM * kM, cross ? round : -1);
    if (threadIdx.x == 0 && applied) atomicAdd(rot_counter, (unsigned long long)applied);
    // TF32 hi / lo image of F_b^T (row n, column k holds F_b[k][n]) for the pass
    // kernel's B operand; the block's F is still in shared memory (after S).
    const float* Fs = reinterpret_cast<const float*>(smraw) + kM * (kM + 1);
    float* img = Fimg + (size_t)blockIdx.x * 2 * kM * kM;
    for (int t = threadIdx.x; t < kM * kM; t += blockDim.x) {
        const int n = t / kM, k = t % kM;
        float h, l;
        tc::split_tf32(Fs[n * (kM + 1) + k], h, l);
        img[t] = h;
        img[kM * kM + t] = l;
    }
}

// Per-CTA shared memory of the pass kernel (offsets in floats from a 1024-byte
// aligned base): the load slot -- the two 32-column chunks of the X tile (128
// rows x 128 bytes, 128-byte swizzle, as the TMA writes them; split in place
// into the TF32 hi part) and the TF32 hi/lo image of F_b^T for the two K halves
// (64 rows x 128 bytes each) -- then the TF32 lo part of X.  96 KB: two CTAs
// share an SM, so one's loads overlap the other's MMAs and stores.
constexpr int kChunk = kSlab * 32;                   // floats of one X chunk (16 KB)
constexpr int kFChunk = kM * 32;                     // floats of one F chunk (8 KB)
constexpr int kSlotFloats = 2 * kChunk + 4 * kFChunk;
constexpr int kXlOff = kSlotFloats;
constexpr size_t kPassSmem = sizeof(float) * (size_t)(kXlOff + 2 * kChunk) + 1024;
constexpr uint32_t kSlotBytes = sizeof(float) * kSlotFloats;   // TMA bytes per item

struct PassMaps {
    CUtensorMap in_t;       // X source of the T tiles (T in pass 1, P in pass 2)
    CUtensorMap v;          // Vt (row-major V), loads and stores
    CUtensorMap f;          // F image: (pairs x 128) rows of 64 floats
};

// The item sequence of a CTA: it, it + gridDim.x, ...; V tiles whose W_b is the
// identity are skipped (they are unchanged).
__device__ __forceinline__ int next_item(int it, int total, int items_T, int n_slabs,
                                         const float* __restrict__ fmax) {
    while (it < total && it >= items_T && fmax[(it - items_T) / n_slabs] == 0.f) it += gridDim.x;
    return it;
}

__device__ __forceinline__ void issue_item(const PassMaps& maps, int it, int items_T, int n_slabs,
                                           int round, int nblocks, float* slot, uint64_t* full) {
    const bool vt = it >= items_T;
    const int item = vt ? it - items_T : it;
    const int s = item % n_slabs, b = item / n_slabs;
    int I, J;
    round_pair(round, b, nblocks, I, J);
    const CUtensorMap* mx = vt ? &maps.v : &maps.in_t;
    tc::mbar_expect_tx(full, kSlotBytes);
    tc::tma_load_2d(slot, mx, I * kB, s * kSlab, full);
    tc::tma_load_2d(slot + kChunk, mx, J * kB, s * kSlab, full);
    float* F = slot + 2 * kChunk;
    tc::tma_load_2d(F, &maps.f, 0, b * 2 * kM, full);                      // hi, k < 32
    tc::tma_load_2d(F + kFChunk, &maps.f, 32, b * 2 * kM, full);           // hi, k >= 32
    tc::tma_load_2d(F + 2 * kFChunk, &maps.f, 0, b * 2 * kM + kM, full);   // lo, k < 32
    tc::tma_load_2d(F + 3 * kFChunk, &maps.f, 32, b * 2 * kM + kM, full);  // lo, k >= 32
}

// Persistent pass kernel (two CTAs per SM).  Items [0, items_T): Tout[rows, IJ_b]
// = X + X F_b with X[m][k] = In[col(k) + (row0 + m) N] (In^T, K-major), written
// column-major; with Sbuf the rows in IJ_b take the solver's rotated block
// instead.  Items [items_T, total): the rows slab of the row-major V times W_b,
// stored back with TMA.
__global__ void __launch_bounds__(kTcThreads, 2)
k_pass_tc(const __grid_constant__ PassMaps maps, float* __restrict__ Tout, int N, int n_slabs,
          int items_T, int total, const float* __restrict__ Sbuf, const float* __restrict__ fmax,
          int round, int terms, unsigned long long* __restrict__ err) {
    extern __shared__ unsigned char smraw[];
    float* sl = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full;
    __shared__ __align__(8) uint64_t mma_done;
    __shared__ uint32_t tmem_slot;
    float* Xh = sl;                                  // split in place
    float* Xl = sl + kXlOff;
    const float* F = sl + 2 * kChunk;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nblocks = N / kB;
    if (tid == 0) {
        tc::mbar_init(&full, 1);
        tc::mbar_init(&mma_done, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot, kM);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const int it0 = next_item(blockIdx.x, total, items_T, n_slabs, fmax);
    if (tid == 0 && it0 < total) issue_item(maps, it0, items_T, n_slabs, round, nblocks, sl, &full);
    bool ok = true;
    int k = 0;
    for (int it = it0; it < total; ++k) {
        const bool vt = it >= items_T;
        const int item = vt ? it - items_T : it;
        const int s = item % n_slabs, b = item / n_slabs;
        int I, J;
        round_pair(round, b, nblocks, I, J);
        const int row0 = s * kSlab;
        ok = tc::mbar_wait(&full, k & 1, kTcWait) && ok;         // waited even after an error
        // split X in place: hi over the loaded tile, lo to Xl (same swizzled offsets)
#pragma unroll 4
        for (int i = tid; i < 2 * kChunk / 4; i += kTcThreads) {
            const float4 x = reinterpret_cast<const float4*>(Xh)[i];
            float4 h, l;
            tc::split_tf32(x.x, h.x, l.x);
            tc::split_tf32(x.y, h.y, l.y);
            tc::split_tf32(x.z, h.z, l.z);
            tc::split_tf32(x.w, h.w, l.w);
            reinterpret_cast<float4*>(Xh)[i] = h;
            reinterpret_cast<float4*>(Xl)[i] = l;
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0 && ok) {
            constexpr uint32_t idesc = tc::instr_desc(tc::kFmtTF32, kSlab, kM);
#pragma unroll
            for (int ks = 0; ks < kM / 8; ++ks) {          // K = 8 per MMA, 32 bytes along the row
                const int ch = ks >> 2;
                const uint32_t off = (ks & 3) * 32;
                const uint32_t xh = tc::smem_u32(Xh + ch * kChunk) + off;
                const uint32_t xl = tc::smem_u32(Xl + ch * kChunk) + off;
                const uint32_t fh = tc::smem_u32(F + ch * kFChunk) + off;
                const uint32_t fl = tc::smem_u32(F + (2 + ch) * kFChunk) + off;
                if (terms == 3) {            // the two cross terms of the three-term split
                    tc::mma_tf32(tmem, tc::smem_desc_sw128(xl), tc::smem_desc_sw128(fh), idesc, ks > 0);
                    tc::mma_tf32(tmem, tc::smem_desc_sw128(xh), tc::smem_desc_sw128(fl), idesc, 1);
                }
                tc::mma_tf32(tmem, tc::smem_desc_sw128(xh), tc::smem_desc_sw128(fh), idesc,
                             terms == 3 || ks > 0);
            }
            tc::commit(&mma_done);
        }
        ok = tc::mbar_wait(&mma_done, k & 1, kTcWait) && ok;
        tc::fence_after_sync();
        const int m = warp * 32 + lane;
        const int row = row0 + m;
        float o[kM];
        if (ok) {
#pragma unroll
            for (int c0 = 0; c0 < kM; c0 += 16)
                tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, o + c0);
            tc::tmem_wait_ld();
#pragma unroll
            for (int ch = 0; ch < 2; ++ch)
#pragma unroll
                for (int j = 0; j < 8; ++j) {               // delta form: + X (= hi + lo exactly)
                    const int off = ch * kChunk + tc::sw128_off(m, j);
                    const float4 h = *reinterpret_cast<const float4*>(Xh + off);
                    const float4 l = *reinterpret_cast<const float4*>(Xl + off);
                    float* oo = o + ch * 32 + j * 4;
                    oo[0] += h.x + l.x; oo[1] += h.y + l.y; oo[2] += h.z + l.z; oo[3] += h.w + l.w;
                }
        }
        if (!vt) {
            if (ok && row < N) {
                if (Sbuf && (row / kB == I || row / kB == J)) {
                    const float* Sr = Sbuf + (size_t)b * kM * kM +
                                      (size_t)(row / kB == I ? row % kB : kB + row % kB) * kM;
#pragma unroll
                    for (int c = 0; c < kM; ++c) o[c] = __ldg(Sr + c);
                }
#pragma unroll
                for (int c = 0; c < kM; ++c) Tout[(size_t)row + (size_t)pair_global(c, I, J, kB) * N] = o[c];
            }
        } else {
            __syncthreads();                         // every thread has read its X row
            if (ok) {
                // stage over the X tile and store with TMA
#pragma unroll
                for (int ch = 0; ch < 2; ++ch)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float* oo = o + ch * 32 + j * 4;
                        *reinterpret_cast<float4*>(Xh + ch * kChunk + tc::sw128_off(m, j)) =
                            make_float4(oo[0], oo[1], oo[2], oo[3]);
                    }
                tc::fence_proxy_async();
            }
        }
        tc::fence_before_sync();
        __syncthreads();                             // TMEM, X and the staging tile are settled
        const int itn = next_item(it + gridDim.x, total, items_T, n_slabs, fmax);
        if (tid == 0) {
            if (vt && ok) {
                tc::tma_store_2d(&maps.v, I * kB, row0, Xh);
                tc::tma_store_2d(&maps.v, J * kB, row0, Xh + kChunk);
                tc::bulk_commit();
                tc::bulk_wait_read();                // the slot is reloaded next
            }
            if (itn < total) issue_item(maps, itn, items_T, n_slabs, round, nblocks, sl, &full);
        }
        it = itn;
    }
    if (!ok && tid == 0) atomicExch(err, 1ull);
    if (tid == 0) tc::bulk_wait_all();
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kM);
}

// ---------------------------------------------------------------- one-sided FP32
// Step 1 of Algorithm 5.2 on the tensor cores: C (m x N) and V (N x N) are kept
// row-major, so that the block rotations C_IJ <- C_IJ W_b and V_IJ <- V_IJ W_b
// are the V-type items of k_pass_tc (a row slab times W_b, stored back by TMA).
// The block Grams G_b = C_IJ^T C_IJ contract over the rows of C: k_gram_tc32
// loads chunks of 32 rows of the pair's 64 columns by TMA, transposes them in
// shared memory into the TF32 hi / lo planes of C_IJ^T (64 rows, K-major,
// 128-byte swizzle), and accumulates hi hi^T + hi lo^T (one MMA with N = 128
// over the hi and lo planes) and lo hi^T (N = 64) in FP32 in TMEM: about FP32
// accuracy, like the SIMT FP32 Gram it replaces.  M = 64 (the pair's columns):
// row i of the accumulator sits in TMEM lane 32 (i / 16) + i % 16.
constexpr int kG32Thr = 128;
constexpr int kG32Stage = 2 * 32 * 32;               // floats: two TMA boxes of 32 rows x 32 columns
constexpr int kG32Plane = kM * 32;                   // floats: 64 pair columns x 32 rows of C
constexpr int kG32Slot = 2 * kG32Plane;              // hi and lo planes, one after the other
constexpr size_t kGram32Smem = sizeof(float) * (size_t)(2 * kG32Stage + 2 * kG32Slot) + 1024;
constexpr int kGram32Ctas = 304;                     // target CTAs of a Gram launch (two per SM)

// One CTA per (pair b, row range); the partial Gram of its rows to
// Ghi[(b nsplit + split) M^2 + c M + r] (Glo = 0), the layout the FP32 block
// solves sum.  Bounded waits; a timeout sets *err.
__global__ void __launch_bounds__(kG32Thr, 2)
k_gram_tc32(const __grid_constant__ CUtensorMap map, int m, int N, int round, int rows_per,
            float* __restrict__ Ghi, float* __restrict__ Glo, unsigned long long* __restrict__ err) {
    extern __shared__ unsigned char smraw[];
    float* sm = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    float* Xs = sm;                                  // two load stages
    float* Ps = sm + 2 * kG32Stage;                  // two plane slots
    __shared__ __align__(8) uint64_t xfull[2], mdone[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.x, split = blockIdx.y, nsplit = gridDim.y;
    int I, J;
    round_pair(round, b, N / kB, I, J);
    const int r0 = split * rows_per;
    const int r1 = min(m, r0 + rows_per);
    const int nq = (r1 - r0 + 31) / 32;
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) { tc::mbar_init(&xfull[i], 1); tc::mbar_init(&mdone[i], 1); }
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot, 256);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    auto load = [&](int q) {
        const int st = q & 1;
        tc::mbar_expect_tx(&xfull[st], sizeof(float) * kG32Stage);
        tc::tma_load_2d(Xs + st * kG32Stage, &map, I * kB, r0 + 32 * q, &xfull[st]);
        tc::tma_load_2d(Xs + st * kG32Stage + 1024, &map, J * kB, r0 + 32 * q, &xfull[st]);
    };
    if (tid == 0)
        for (int q = 0; q < nq && q < 2; ++q) load(q);
    bool ok = true;
    constexpr uint32_t idesc1 = tc::instr_desc(tc::kFmtTF32, kM, 2 * kM);
    constexpr uint32_t idesc2 = tc::instr_desc(tc::kFmtTF32, kM, kM);
    for (int q = 0; q < nq; ++q) {
        const int st = q & 1;
        ok = tc::mbar_wait(&xfull[st], (q >> 1) & 1, kTcWait) && ok;
        if (q >= 2) ok = tc::mbar_wait(&mdone[st], ((q >> 1) - 1) & 1, kTcWait) && ok;
        {
            // thread (4-row group rb, 4-column group cb): a 4 x 4 block transposed
            // through registers, split into TF32 hi and lo
            const float* X = Xs + st * kG32Stage;
            float* H = Ps + st * kG32Slot;
            float* L = H + kG32Plane;
            const int rb = tid >> 4, cb = tid & 15;
            const float* Xb = X + (cb >> 3) * 1024;
            const int cc = cb & 7;
            float v[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = 4 * rb + i;
                const float4 x = *reinterpret_cast<const float4*>(Xb + r * 32 + ((cc ^ (r & 7)) << 2));
                v[i][0] = x.x; v[i][1] = x.y; v[i][2] = x.z; v[i][3] = x.w;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = 4 * cb + j;
                float4 h, l;
                tc::split_tf32(v[0][j], h.x, l.x);
                tc::split_tf32(v[1][j], h.y, l.y);
                tc::split_tf32(v[2][j], h.z, l.z);
                tc::split_tf32(v[3][j], h.w, l.w);
                const int off = tc::sw128_off(c, rb);
                *reinterpret_cast<float4*>(H + off) = h;
                *reinterpret_cast<float4*>(L + off) = l;
            }
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();                             // stage st read, planes of slot st written
        tc::fence_after_sync();
        if (tid == 0) {
            if (q + 2 < nq) load(q + 2);
            if (ok) {
                const uint32_t h0 = tc::smem_u32(Ps + st * kG32Slot);
                const uint32_t l0 = h0 + sizeof(float) * kG32Plane;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {     // K = 8 per MMA: 32 bytes along the 128-byte row
                    const uint32_t acc = (q > 0 || ks > 0) ? 1u : 0u;
                    // [hi hi^T | hi lo^T]: the hi and lo planes form one 128-row operand
                    tc::mma_tf32(tmem, tc::smem_desc_sw128(h0 + ks * 32), tc::smem_desc_sw128(h0 + ks * 32),
                                 idesc1, acc);
                    tc::mma_tf32(tmem + 2 * kM, tc::smem_desc_sw128(l0 + ks * 32),
                                 tc::smem_desc_sw128(h0 + ks * 32), idesc2, acc);
                }
            }
            tc::commit(&mdone[st]);
        }
    }
    if (nq > 0) ok = tc::mbar_wait(&mdone[(nq - 1) & 1], ((nq - 1) >> 1) & 1, kTcWait) && ok;
    tc::fence_after_sync();
    if (ok && nq > 0) {
        const uint32_t lanebase = tmem + ((uint32_t)(32 * warp) << 16);
        const int i = 16 * warp + (lane & 15);       // row i of G (lanes 16-31 unused)
        const size_t base = ((size_t)b * nsplit + split) * kM * kM;
#pragma unroll 1
        for (int c0 = 0; c0 < kM; c0 += 16) {
            float a[16], x[16], y[16];
            tc::tmem_ld16(lanebase + (uint32_t)c0, a);
            tc::tmem_ld16(lanebase + (uint32_t)(kM + c0), x);
            tc::tmem_ld16(lanebase + (uint32_t)(2 * kM + c0), y);
            tc::tmem_wait_ld();
            if (lane < 16) {
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    Ghi[base + (size_t)(c0 + jj) * kM + i] = a[jj] + (x[jj] + y[jj]);
                    Glo[base + (size_t)(c0 + jj) * kM + i] = 0.f;
                }
            }
        }
    }
    if (!ok && tid == 0) atomicExch(err, 1ull);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// TF32 hi / lo image of F_b^T (row n, column k: F_b[k][n]) from the block solve's
// row-major F_b, for the B operand of k_pass_tc, and max |F_b|.
__global__ void __launch_bounds__(256)
k_fimg32(const float* __restrict__ Wbuf, float* __restrict__ Fimg, float* __restrict__ fmax) {
    __shared__ float red[8];
    const int b = blockIdx.x;
    const float* F = Wbuf + (size_t)b * kM * kM;
    float* img = Fimg + (size_t)b * 2 * kM * kM;
    float mx = 0.f;
    for (int t = threadIdx.x; t < kM * kM; t += blockDim.x) {
        const int n = t / kM, k = t % kM;
        const float v = F[k * kM + n];
        float h, l;
        tc::split_tf32(v, h, l);
        img[t] = h;
        img[kM * kM + t] = l;
        mx = fmaxf(mx, fabsf(v));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float r = 0.f;
        for (int w = 0; w < 8; ++w) r = fmaxf(r, red[w]);
        fmax[b] = r;
    }
}

// C[r N + c] = fl32(A[r + c lda]) for c < n, 0 for n <= c < N (row-major, padded).
__global__ void k_copy_rowmajor_f32(const double* __restrict__ A, int lda, int m, int n, float* __restrict__ C,
                                    int N) {
    __shared__ float tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int r = r0 + threadIdx.x, c = c0 + k;
        tile[k][threadIdx.x] = (r < m && c < n) ? (float)A[(size_t)r + (size_t)c * lda] : 0.f;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < m && c < N) C[(size_t)r * N + c] = tile[threadIdx.x][k];
    }
}

// out[c] += sum over this block's rows of C[r N + c]^2 (row-major C; out zeroed first).
__global__ void k_colnorms2_rowmajor(const float* __restrict__ C, int m, int N, int n, int rows_per,
                                     double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int r0 = blockIdx.y * rows_per, r1 = min(m, r0 + rows_per);
    double acc = 0.0;
    for (int r = r0; r < r1; ++r) {
        const double v = (double)C[(size_t)r * N + c];
        acc = fma(v, v, acc);
    }
    atomicAdd(out + c, acc);
}

__global__ void k_gather_z32_rowmajor(const float* __restrict__ Vt, int ld, const int* __restrict__ perm,
                                      int n, double* __restrict__ Z, int ldz) {
    // Z[:, c] = V[:, perm[c]] with V row-major (V[r][p] = Vt[p + r ld]); one row of
    // V per block iteration, so the reads of a row are served from one cache line set.
    for (int r = blockIdx.x; r < n; r += gridDim.x) {
        const float* row = Vt + (size_t)r * ld;
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            int p = perm[c];
            p = p < 0 ? 0 : (p >= n ? n - 1 : p);
            Z[(size_t)r + (size_t)c * ldz] = (double)row[p];
        }
    }
}

}  // namespace

size_t tc32_workspace_bytes(int N) {
    const size_t K = (size_t)(N / kM);
    // two sets of (W, S, F image (2 planes), max|F|), plus the sweep scratch
    return 2 * (sizeof(float) * K * kM * kM * 4 + sizeof(float) * K + 1024) + sizeof(double) * 1100 + 4096;
}

namespace {

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

// Row-major 2-D FP32 array (outer x inner, rows of `inner` floats) viewed in
// boxes of box_outer rows x 32 floats, 128-byte swizzle.
int encode_rows(CUtensorMap* m, const float* base, uint64_t inner, uint64_t outer, uint32_t box_outer) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) { set_error_msg("cuTensorMapEncodeTiled is not available"); return MPJ_CUDA_ERROR; }
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * sizeof(float)};
    cuuint32_t box[2] = {32, box_outer};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_error_msg("cuTensorMapEncodeTiled failed"); return MPJ_CUDA_ERROR; }
    return MPJ_SUCCESS;
}

int sm_count() {
    static int n = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            v = 148;
        return v;
    }();
    return n;
}

}  // namespace

int gather_z32_rowmajor(const float* Vt, int ld, const int* perm, int n, double* Z, int ldz,
                        cudaStream_t s) {
    {
        MPJ_PROF(PC_AUX, s);
        k_gather_z32_rowmajor<<<n < 152 * 8 ? n : 152 * 8, 256, 0, s>>>(Vt, ld, perm, n, Z, ldz);
    }
    MPJ_LAUNCH_CHECK("k_gather_z32_rowmajor");
    return MPJ_SUCCESS;
}

int twosided_sweeps_tc32(float* T, float* Vt, float* P, int N, int n, double tol_abs,
                         double eps_skip, int max_sweeps, int max_inner, void* work, cudaStream_t s,
                         SweepResult* res) {
    if (N % kM != 0) { set_error_msg("tensor-core engine: N must be a multiple of 64"); return MPJ_BAD_ARG; }
    const int K = N / kM;
    Arena ar;
    ar.base = static_cast<char*>(work);
    ar.size = tc32_workspace_bytes(N);
    // Two sets of block-rotation buffers: the V pass of round g runs on a side
    // stream (after the solve of round g), overlapping the next block solves.
    float *Wbuf[2], *Sbuf[2], *Fimg[2], *fmax[2];
    for (int set = 0; set < 2; ++set) {
        Wbuf[set] = ar.take<float>((size_t)K * kM * kM);
        Sbuf[set] = ar.take<float>((size_t)K * kM * kM);
        Fimg[set] = ar.take<float>((size_t)K * 2 * kM * kM);
        fmax[set] = ar.take<float>((size_t)K);
    }
    double* partial = ar.take<double>(1024);
    double* offv = ar.take<double>(4);
    unsigned long long* rot = ar.take<unsigned long long>(4);     // [0] rotations, [1] error flag
    if (!Wbuf[1] || !Sbuf[1] || !Fimg[1] || !fmax[1] || !partial || !offv || !rot) {
        set_error_msg("workspace too small");
        return MPJ_BAD_ARG;
    }
    HostScratch hs;
    MPJ_TRY(hs.init());
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_solve2_nb, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)InnerLayout<float, kM>::bytes));
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_pass_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPassSmem));
    PassMaps maps1[2], maps2[2];                         // per buffer set: pass 1, pass 2 and V
    for (int set = 0; set < 2; ++set) {
        MPJ_TRY(encode_rows(&maps1[set].in_t, T, N, N, kSlab));
        MPJ_TRY(encode_rows(&maps1[set].v, Vt, N, N, kSlab));
        MPJ_TRY(encode_rows(&maps1[set].f, Fimg[set], kM, (uint64_t)K * 2 * kM, kM));
        maps2[set] = maps1[set];
        MPJ_TRY(encode_rows(&maps2[set].in_t, P, N, N, kSlab));
    }
    SideStream side;
    MPJ_TRY(side.init(s));
    s = side.main;                                       // high priority: the critical path
    MPJ_CUDA_TRY(cudaMemsetAsync(rot, 0, 2 * sizeof(unsigned long long), s));
    MPJ_TRY(offnorm2(T, false, N, n, partial, offv, s));
    MPJ_CUDA_TRY(cudaMemcpyAsync(hs.d, offv, sizeof(double), cudaMemcpyDeviceToHost, s));
    MPJ_CUDA_TRY(cudaStreamSynchronize(s));
    double off = sqrt(hs.d[0]);
    res->off_initial = off;
    res->sweeps = 0;
    res->rotations = 0;
    res->status = MPJ_NOT_CONVERGED;
    const int rounds = 2 * K - 1;
    const int n_slabs = (N + kSlab - 1) / kSlab;
    const int items = n_slabs * K;
    const int grid1 = items < 2 * sm_count() ? items : 2 * sm_count();
    const int gridv = N >= 8192 ? items : grid1;
    const float tau = (float)(tol_abs / (double)N);
    const float gate = 1.0f / 4096.0f;                   // Newton-Schulz when some |F| >= 2^-12
    // TF32 products per tile: 3 (about FP32 accuracy) or 1 (hi*hi only, about
    // 2^-11: a lower-precision step 1, mpj_options.stage1_tf32_terms)
    const int terms = knobs().stage1_terms;
    const int cross = N >= kB * kB ? cross_schedule(false, false) : 0;     // see cross_schedule
    // the V pass joins after pass 2, so that it overlaps only the next round's
    // block solves (measured at n = 4096: stage 1 238 -> 223 ms)
    const bool v_late = true;
    while (res->sweeps < max_sweeps) {
        if (!std::isfinite(off)) { res->status = MPJ_NONFINITE_INPUT; break; }
        if (!(off > tol_abs)) { res->status = MPJ_SUCCESS; break; }
        MPJ_CUDA_TRY(cudaMemsetAsync(rot, 0, sizeof(unsigned long long), s));
        for (int r = 0; r < rounds; ++r) {
            const int set = side.begin_round();
            if (set < 0) return MPJ_CUDA_ERROR;
            {
                MPJ_PROF(PC_SOLVE2_F32, s);
                k_solve2_nb<<<K, kSolve32Threads, InnerLayout<float, kM>::bytes, s>>>(
                    T, N, Wbuf[set], Sbuf[set], Fimg[set], fmax[set], r, (float)eps_skip, tau, gate, max_inner,
                    cross, rot);
            }
            MPJ_LAUNCH_CHECK("k_solve2_nb");
            if (!v_late) MPJ_TRY(side.after_solve());
            {
                MPJ_PROF(PC_TC1_F32, s);
                k_pass_tc<<<grid1, kTcThreads, kPassSmem, s>>>(maps1[set], P, N, n_slabs, items, items, nullptr,
                                                               fmax[set], r, terms, rot + 1);
            }
            MPJ_LAUNCH_CHECK("k_pass_tc pass 1");
            {
                MPJ_PROF(PC_TC2_F32, s);
                k_pass_tc<<<grid1, kTcThreads, kPassSmem, s>>>(maps2[set], T, N, n_slabs, items, items, Sbuf[set],
                                                               fmax[set], r, terms, rot + 1);
            }
            MPJ_LAUNCH_CHECK("k_pass_tc pass 2");
            if (v_late) MPJ_TRY(side.after_solve());
            {
                // Persistent (two CTAs per SM) while a CTA has few tiles; one tile per CTA
                // for N >= 8192, where the SM slots then free up tile by tile for the next
                // block solve on the high-priority stream (measured: 273 vs 284 ms of
                // step 1 at n = 4096, 1443 vs 1352 ms at n = 8192).
                MPJ_PROF(PC_TCV_F32, side.sv);
                k_pass_tc<<<gridv, kTcThreads, kPassSmem, side.sv>>>(maps2[set], T, N, n_slabs, 0, items, nullptr,
                                                                     fmax[set], r, terms, rot + 1);
            }
            MPJ_LAUNCH_CHECK("k_pass_tc V");
            MPJ_TRY(side.after_v());
            side.end_round();
        }
        MPJ_TRY(offnorm2(T, false, N, n, partial, offv, s));
        MPJ_CUDA_TRY(cudaMemcpyAsync(hs.d, offv, sizeof(double), cudaMemcpyDeviceToHost, s));
        MPJ_CUDA_TRY(cudaMemcpyAsync(hs.u, rot, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        MPJ_CUDA_TRY(cudaStreamSynchronize(s));
        prof_flush();
        if (hs.u[1]) { set_error_msg("tensor-core tile: MMA completion wait timed out"); return MPJ_CUDA_ERROR; }
        off = sqrt(hs.d[0]);
        res->sweeps += 1;
        res->rotations += (double)hs.u[0];
        if (trace_on())
            fprintf(stderr, "[mpj] twosided<tc32> n=%d sweep %d: %llu rotations, off %.3e\n", n,
                    res->sweeps, hs.u[0], off);
        if (hs.u[0] == 0) { res->status = MPJ_SUCCESS; break; }
    }
    if (res->status == MPJ_NOT_CONVERGED && std::isfinite(off) && !(off > tol_abs))
        res->status = MPJ_SUCCESS;
    res->off_final = off;
    return MPJ_SUCCESS;
}

// ---------------------------------------------------------------- one-sided FP32 engine
namespace {
void gram32_split(int m, int K, int* nsplit, int* rows_per) {
    const int want = kGram32Ctas / K > 1 ? kGram32Ctas / K : 1;
    const int chunks = (m + 31) / 32;
    int per = (chunks + want - 1) / want;
    if (per < 1) per = 1;
    *rows_per = per * 32;
    *nsplit = (m + *rows_per - 1) / *rows_per;
}
}  // namespace

bool onesided_tc32_supported(int m, int N, int B) { return B == kB && N % kM == 0 && N >= kM && m >= kSlab; }

size_t onesided_tc32_workspace_bytes(int m, int N) {
    const size_t K = (size_t)(N / kM);
    int nsplit = 1, rows_per = 32;
    if (K > 0) gram32_split(m, (int)K, &nsplit, &rows_per);
    Arena a;
    for (int set = 0; set < 2; ++set) {
        a.take<float>(K * kM * kM);               // W_b - I
        a.take<float>(K * 2 * kM * kM);           // TF32 image of F_b^T
        a.take<float>(K);                         // max |F_b|
    }
    a.take<float>(K * nsplit * kM * kM);          // Gram partials (hi)
    a.take<float>(K * nsplit * kM * kM);          //               (lo, zero)
    a.take<unsigned long long>(4);
    return a.used + 256;
}

int onesided_sweeps_tc32(float* C, float* V, int m, int N, int n, double tol_rot, double ju_ratio,
                         int max_sweeps, int max_inner, void* work, cudaStream_t s, SweepResult* res) {
    if (!onesided_tc32_supported(m, N, kB)) {
        set_error_msg("tensor-core FP32 one-sided engine: needs b = 32, N a multiple of 64, m >= 128");
        return MPJ_BAD_ARG;
    }
    const int K = N / kM;
    int nsplit, rows_per;
    gram32_split(m, K, &nsplit, &rows_per);
    Arena ar;
    ar.base = static_cast<char*>(work);
    ar.size = onesided_tc32_workspace_bytes(m, N);
    float *Wbuf[2], *Fimg[2], *fmax[2];
    for (int set = 0; set < 2; ++set) {
        Wbuf[set] = ar.take<float>((size_t)K * kM * kM);
        Fimg[set] = ar.take<float>((size_t)K * 2 * kM * kM);
        fmax[set] = ar.take<float>((size_t)K);
    }
    float* Ghi = ar.take<float>((size_t)K * nsplit * kM * kM);
    float* Glo = ar.take<float>((size_t)K * nsplit * kM * kM);
    unsigned long long* rot = ar.take<unsigned long long>(4);     // [0] rotations, [1] error flag
    if (!fmax[1] || !Ghi || !Glo || !rot) { set_error_msg("workspace too small"); return MPJ_BAD_ARG; }
    HostScratch hs;
    MPJ_TRY(hs.init());
    MPJ_TRY(configure_solve1_f32());
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_gram_tc32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGram32Smem));
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_pass_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPassSmem));
    CUtensorMap mg;
    MPJ_TRY(encode_rows(&mg, C, N, m, 32));              // Gram: 32 rows x 32 columns per box
    PassMaps mc[2], mv[2];                               // rotations: row slabs of C and of V
    for (int set = 0; set < 2; ++set) {
        MPJ_TRY(encode_rows(&mc[set].v, C, N, m, kSlab));
        mc[set].in_t = mc[set].v;
        MPJ_TRY(encode_rows(&mc[set].f, Fimg[set], kM, (uint64_t)K * 2 * kM, kM));
        MPJ_TRY(encode_rows(&mv[set].v, V, N, N, kSlab));
        mv[set].in_t = mv[set].v;
        mv[set].f = mc[set].f;
    }
    SideStream side;
    MPJ_TRY(side.init(s));
    s = side.main;
    MPJ_CUDA_TRY(cudaMemsetAsync(rot, 0, 2 * sizeof(unsigned long long), s));
    res->sweeps = 0;
    res->rotations = 0;
    res->status = MPJ_NOT_CONVERGED;
    const int rounds = 2 * K - 1;
    const int slabsC = (m + kSlab - 1) / kSlab, itemsC = slabsC * K;
    const int slabsV = (N + kSlab - 1) / kSlab, itemsV = slabsV * K;
    const int gridC = itemsC < 2 * sm_count() ? itemsC : 2 * sm_count();
    const int gridV = itemsV < 2 * sm_count() ? itemsV : 2 * sm_count();
    const double Npairs = 0.5 * (double)n * (double)(n - 1);
    const bool cross = N >= kB * kB && !knobs().full_inner;
    while (res->sweeps < max_sweeps) {
        MPJ_CUDA_TRY(cudaMemsetAsync(rot, 0, sizeof(unsigned long long), s));
        for (int r = 0; r < rounds; ++r) {
            const int set = side.begin_round();
            if (set < 0) return MPJ_CUDA_ERROR;
            {
                MPJ_PROF(PC_GRAM1_F32, s);
                k_gram_tc32<<<dim3(K, nsplit), kG32Thr, kGram32Smem, s>>>(mg, m, N, r, rows_per, Ghi, Glo, rot + 1);
            }
            MPJ_LAUNCH_CHECK("k_gram_tc32");
            MPJ_TRY(solve1_f32_round(Ghi, Glo, nsplit, K, Wbuf[set], tol_rot, max_inner, cross ? r : -1, rot, s));
            {
                MPJ_PROF(PC_AUX, s);
                k_fimg32<<<K, 256, 0, s>>>(Wbuf[set], Fimg[set], fmax[set]);
            }
            MPJ_LAUNCH_CHECK("k_fimg32");
            MPJ_TRY(side.after_solve());
            {
                MPJ_PROF(PC_APPLY1_F32, side.sv);
                k_pass_tc<<<gridV, kTcThreads, kPassSmem, side.sv>>>(mv[set], nullptr, N, slabsV, 0, itemsV, nullptr,
                                                                     fmax[set], r, 3, rot + 1);
            }
            MPJ_LAUNCH_CHECK("k_pass_tc V (one-sided)");
            MPJ_TRY(side.after_v());
            {
                MPJ_PROF(PC_APPLY1_F32, s);
                k_pass_tc<<<gridC, kTcThreads, kPassSmem, s>>>(mc[set], nullptr, N, slabsC, 0, itemsC, nullptr,
                                                               fmax[set], r, 3, rot + 1);
            }
            MPJ_LAUNCH_CHECK("k_pass_tc C (one-sided)");
            side.end_round();
        }
        MPJ_CUDA_TRY(cudaMemcpyAsync(hs.u, rot, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        MPJ_CUDA_TRY(cudaStreamSynchronize(s));
        prof_flush();
        if (hs.u[1]) { set_error_msg("tensor-core FP32 one-sided sweep: a wait timed out"); return MPJ_CUDA_ERROR; }
        res->sweeps += 1;
        res->rotations += (double)hs.u[0];
        if (trace_on())
            fprintf(stderr, "[mpj] onesided<tc32> m=%d n=%d sweep %d: %llu rotations (%.4f N)\n", m, n, res->sweeps,
                    hs.u[0], hs.u[0] / Npairs);
        const double applied = (double)hs.u[0];
        if (hs.u[0] == 0 || applied < ju_ratio * Npairs) { res->status = MPJ_SUCCESS; break; }
    }
    return MPJ_SUCCESS;
}

int copy_rowmajor_f32(const double* A, int lda, int m, int n, float* C, int N, cudaStream_t s) {
    {
        MPJ_PROF(PC_AUX, s);
        k_copy_rowmajor_f32<<<dim3((N + 31) / 32, (m + 31) / 32), dim3(32, 8), 0, s>>>(A, lda, m, n, C, N);
    }
    MPJ_LAUNCH_CHECK("k_copy_rowmajor_f32");
    return MPJ_SUCCESS;
}

int colnorms2_rowmajor_f32(const float* C, int m, int N, int n, double* nrm2, cudaStream_t s) {
    MPJ_CUDA_TRY(cudaMemsetAsync(nrm2, 0, sizeof(double) * (size_t)n, s));
    const int splits = (m + 255) / 256;
    {
        MPJ_PROF(PC_AUX, s);
        k_colnorms2_rowmajor<<<dim3((n + 255) / 256, splits), 256, 0, s>>>(C, m, N, n, 256, nrm2);
    }
    MPJ_LAUNCH_CHECK("k_colnorms2_rowmajor");
    return MPJ_SUCCESS;
}

}  // namespace mpj
