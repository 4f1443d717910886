// tc_apply.cu -- the FP32 block Jacobi of step 1 of Algorithm 4.1 with the
// rotation application on the 5th-generation tensor cores (tcgen05, kind::tf32).
//
// A round of the parallel order replaces T by W^T T W and V by V W, where W is
// block diagonal over the disjoint block pairs (I, J) of the round (one 2b x 2b
// orthogonal block W_b = I + F_b per pair, from the block-pair solves):
//
//   tile pass   T'[IJ_a, IJ_b] = W_a^T T[IJ_a, IJ_b] W_b for every a < b, written
//               with its mirror (the diagonal blocks are the solver's)
//   slab pass   V'[rows, IJ_b] = V[rows, IJ_b] W_b for 128-row slabs of V
//
// Every product runs on the tensor cores in delta form (X + X F), with X and F
// split into TF32 pairs (hi + lo) and the three products hi*hi + hi*lo + lo*hi
// accumulated in FP32 in TMEM, which carries about 21 bits of each product --
// the accuracy of the FP32 SIMT products it replaces.  Operands are K-major:
// T tiles are read through the transposed view that T's symmetry allows, V is
// kept row-major (Vt = V^T column-major), and the rotations are stored as TF32
// images of F_b^T.
//
// Traffic per round: the off-diagonal tiles of T read once and written twice
// (3 N (N - 2b) floats), V read and written once (2 N^2 floats).  The block-pair
// solves are the FP32 pair solves of the SIMT engine.
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


// The TF32 image of a block rotation F_b, the B operand of the slab pass and of
// product 1 of the tile pass and the A operand of product 2: row n holds
// F_b[:, n] (K-major), split into hi and lo planes, each plane two chunks of 64
// rows x 32 floats (k < 32, k >= 32) in the 128-byte swizzled order that a
// 1024-byte aligned shared-memory copy of it needs.  One pair's image is 32 KB,
// contiguous, so that one bulk copy loads it.
constexpr int kFChunk = kM * 32;                     // floats of one image chunk (8 KB)
constexpr int kFImage = 4 * kFChunk;                 // floats of one pair's image
constexpr uint32_t kFImageBytes = sizeof(float) * kFImage;

__device__ __forceinline__ int fimg_off(int n, int k) {
    return (k >> 5) * kFChunk + tc::sw128_off(n, (k & 31) >> 2) + (k & 3);
}

// Image of one F (element F[k][n] = at(k, n)) into img, by the whole block.
template <class At>
__device__ __forceinline__ void write_fimage(float* __restrict__ img, At at) {
    for (int t = threadIdx.x; t < kM * kM; t += blockDim.x) {
        const int n = t / kM, k = t % kM;
        float h, l;
        tc::split_tf32(at(k, n), h, l);
        img[fimg_off(n, k)] = h;
        img[2 * kFChunk + fimg_off(n, k)] = l;
    }
}

// Block-pair solves of one round.  The rotated block goes back to T: the tile
// pass updates the off-diagonal tiles only.
__global__ void __launch_bounds__(kSolve32Threads)
k_solve2_nb(float* __restrict__ T, int N, float* __restrict__ Fbuf, float* __restrict__ Fimg,
            float* __restrict__ fmax, int round, float eps, float tau, float gate, int max_inner, int cross,
            unsigned long long* __restrict__ rot_counter) {
    extern __shared__ __align__(16) unsigned char smraw[];
    int applied = pair_solve<float, kB, true>(T, N, round, blockIdx.x, eps, tau, gate, max_inner,
                                              Fbuf + (size_t)blockIdx.x * kM * kM, fmax + blockIdx.x, smraw,
                                              nullptr, cross ? round : -1);
    if (threadIdx.x == 0 && applied) atomicAdd(rot_counter, (unsigned long long)applied);
    // the block's F is still in shared memory (after S), column-major with ld 2b + 1
    const float* Fs = reinterpret_cast<const float*>(smraw) + kM * (kM + 1);
    write_fimage(Fimg + (size_t)blockIdx.x * kFImage, [&](int k, int n) { return Fs[n * (kM + 1) + k]; });
}

// ---------------------------------------------------------------- slab pass
// X <- X + X F_b for the 128-row slabs of a row-major X (V, or C of the SVD)
// and every pair b: X[rows, IJ_b] is two TMA boxes of 128 rows x 32 floats
// (K-major), F_b's image one bulk copy.  One 128 x 64 x 64 product per item in
// delta form with the three-term TF32 split, stored back in place by TMA.
// Items whose W_b is the identity are skipped.
//
// Shared memory: three regions of 32 KB from a 1024-byte aligned base.  Q holds
// the TF32 lo part of the slab and then the staging of the result; the other
// two take turns as the slab (split in place to hi) and the F image: once item
// k's product has completed, its F region receives slab k + 1, and once the
// slab has been drained, its region receives F for item k + 1.  The three terms
// are issued by three warps into three 64-column accumulators (one thread
// issues tcgen05.mma at about 80 cycles an instruction); lane 0 of warp 3
// issues the copies.  Two CTAs share an SM.
constexpr int kChunk = kSlab * 32;                   // floats of one slab chunk (16 KB)
constexpr int kRegion = 2 * kChunk;                  // floats of one region (32 KB)
constexpr size_t kPassSmem = sizeof(float) * (size_t)(3 * kRegion) + 1024;
constexpr uint32_t kXBytes = sizeof(float) * kRegion;
constexpr int kPassTmemCols = 256;                   // three 64-column accumulators

struct PassMaps {
    CUtensorMap x;          // row-major X (rows of N floats), boxes of 128 rows x 32 floats
};

__device__ __forceinline__ int next_item(int it, int total, int n_slabs, const float* __restrict__ fmax) {
    while (it < total && fmax[it / n_slabs] == 0.f) it += gridDim.x;
    return it;
}

__device__ __forceinline__ void issue_slab(const PassMaps& maps, int it, int n_slabs, int round, int nblocks,
                                           float* dst, uint64_t* bar) {
    const int s = it % n_slabs, b = it / n_slabs;
    int I, J;
    round_pair(round, b, nblocks, I, J);
    tc::mbar_expect_tx(bar, kXBytes);
    tc::tma_load_2d(dst, &maps.x, I * kB, s * kSlab, bar);
    tc::tma_load_2d(dst + kChunk, &maps.x, J * kB, s * kSlab, bar);
}

__global__ void __launch_bounds__(kTcThreads, 2)
k_pass_tc(const __grid_constant__ PassMaps maps, const float* __restrict__ Fimg, int N, int n_slabs, int total,
          const float* __restrict__ fmax, int round, int terms, unsigned long long* __restrict__ err) {
    extern __shared__ unsigned char smraw[];
    float* base = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    float* Q = base + 2 * kRegion;
    __shared__ __align__(8) uint64_t fullX, fullF, qfree, mma_done;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nblocks = N / kB;
    const int nterm = terms == 3 ? 3 : 1;
    const bool mma_lane = lane == 0 && warp < nterm;
    const bool copy_lane = tid == 96;
    if (tid == 0) {
        tc::mbar_init(&fullX, 1);
        tc::mbar_init(&fullF, 1);
        tc::mbar_init(&qfree, 1);
        tc::mbar_init(&mma_done, nterm);
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot, kPassTmemCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const int m = warp * 32 + lane;                      // slab row = accumulator row
    const uint32_t lanebase = tmem + ((uint32_t)(warp * 32) << 16);
    const int it0 = next_item(blockIdx.x, total, n_slabs, fmax);
    if (copy_lane) {
        tc::mbar_arrive(&qfree);                         // Q starts free (phase 0)
        if (it0 < total) {
            issue_slab(maps, it0, n_slabs, round, nblocks, base, &fullX);
            tc::mbar_expect_tx(&fullF, kFImageBytes);
            tc::bulk_load(base + kRegion, Fimg + (size_t)(it0 / n_slabs) * kFImage, kFImageBytes, &fullF);
        }
    }
    bool ok = true;
    constexpr uint32_t idesc = tc::instr_desc(tc::kFmtTF32, kSlab, kM);
    int k = 0;
    for (int it = it0; it < total; ++k) {
        float* X = base + (k & 1) * kRegion;            // the slab's region
        float* F = base + ((k + 1) & 1) * kRegion;      // the F image's region
        const int s = it % n_slabs, b = it / n_slabs;
        int I, J;
        round_pair(round, b, nblocks, I, J);
        const int row0 = s * kSlab;
        const int itn = next_item(it + gridDim.x, total, n_slabs, fmax);
        ok = tc::mbar_wait(&fullX, k & 1, kTcWait) && ok;          // waited even after an error
        ok = tc::mbar_wait(&qfree, k & 1, kTcWait) && ok;
        // split the slab in place: hi over it, lo to Q (same swizzled offsets)
#pragma unroll 4
        for (int i = tid; i < kRegion / 4; i += kTcThreads) {
            const float4 x = reinterpret_cast<const float4*>(X)[i];
            float4 h, l;
            tc::split_tf32(x.x, h.x, l.x);
            tc::split_tf32(x.y, h.y, l.y);
            tc::split_tf32(x.z, h.z, l.z);
            tc::split_tf32(x.w, h.w, l.w);
            reinterpret_cast<float4*>(X)[i] = h;
            reinterpret_cast<float4*>(Q)[i] = l;
        }
        ok = tc::mbar_wait(&fullF, k & 1, kTcWait) && ok;
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (mma_lane && ok) {            // term of this warp: 0 hi hi, 1 lo hi, 2 hi lo
            const float* A = warp == 1 ? Q : X;
            const float* B = F + (warp == 2 ? 2 * kFChunk : 0);
            const uint32_t d = tmem + (uint32_t)(64 * warp);
#pragma unroll
            for (int ks = 0; ks < kM / 8; ++ks) {      // K = 8 per MMA, 32 bytes along the row
                const int ch = ks >> 2;
                const uint32_t off = (ks & 3) * 32;
                tc::mma_tf32(d, tc::smem_desc_sw128(tc::smem_u32(A + ch * kChunk) + off),
                             tc::smem_desc_sw128(tc::smem_u32(B + ch * kFChunk) + off), idesc, ks > 0);
            }
            tc::commit(&mma_done);
        }
        ok = tc::mbar_wait(&mma_done, k & 1, kTcWait) && ok;
        tc::fence_after_sync();
        if (copy_lane && itn < total) issue_slab(maps, itn, n_slabs, round, nblocks, F, &fullX);   // F is dead
        float o[kM];
#pragma unroll
        for (int c0 = 0; c0 < kM; c0 += 16) {
            float w[16];
            tc::tmem_ld16(lanebase + (uint32_t)c0, o + c0);
            if (nterm == 3) {
                tc::tmem_ld16(lanebase + 64 + (uint32_t)c0, w);
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) o[c0 + j] += w[j];
                tc::tmem_ld16(lanebase + 128 + (uint32_t)c0, w);
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) o[c0 + j] += w[j];
            }
        }
        tc::tmem_wait_ld();
#pragma unroll
        for (int ch = 0; ch < 2; ++ch)
#pragma unroll
            for (int j = 0; j < 8; ++j) {                   // delta form: + X (= hi + lo exactly)
                const int off = ch * kChunk + tc::sw128_off(m, j);
                const float4 h = *reinterpret_cast<const float4*>(X + off);
                const float4 l = *reinterpret_cast<const float4*>(Q + off);
                float* oo = o + ch * 32 + j * 4;
                oo[0] += h.x + l.x; oo[1] += h.y + l.y; oo[2] += h.z + l.z; oo[3] += h.w + l.w;
            }
        tc::fence_before_sync();
        __syncthreads();                                 // the slab, Q and TMEM are read
        if (copy_lane && itn < total) {                  // the slab region takes the next F
            tc::mbar_expect_tx(&fullF, kFImageBytes);
            tc::bulk_load(X, Fimg + (size_t)(itn / n_slabs) * kFImage, kFImageBytes, &fullF);
        }
        if (ok) {                                        // staging in Q, the slab's layout
#pragma unroll
            for (int ch = 0; ch < 2; ++ch)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float* oo = o + ch * 32 + j * 4;
                    *reinterpret_cast<float4*>(Q + ch * kChunk + tc::sw128_off(m, j)) =
                        make_float4(oo[0], oo[1], oo[2], oo[3]);
                }
            tc::fence_proxy_async();
        }
        __syncthreads();                                 // the staging is written
        if (copy_lane) {
            if (ok) {
                tc::tma_store_2d(&maps.x, I * kB, row0, Q);
                tc::tma_store_2d(&maps.x, J * kB, row0, Q + kChunk);
                tc::bulk_commit();
                tc::bulk_wait_read();
            }
            tc::mbar_arrive(&qfree);                     // Q may take the next lo part
        }
        it = itn;
    }
    if (copy_lane) tc::bulk_wait_all();
    if (!ok) atomicExch(err, 1ull);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kPassTmemCols);
}

// ---------------------------------------------------------------- one-pass tile update
// T' = W^T T W in one pass over the off-diagonal pair tiles: for a < b,
//
//   X = T_ab + T_ab F_b            (product 1: M = 64 rows m of IJ_a, N = K = 64)
//   Y = X + F_a^T X                (product 2: M = 64 rows j of IJ_a, K over m)
//
// and Y is stored at T[IJ_a, IJ_b] and, transposed, at T[IJ_b, IJ_a] (T' is
// symmetric by construction).  T is read once through the K-major view of the
// T[IJ_b, IJ_a] sub-blocks (T symmetric) and written in place: the two regions
// of tile (a, b) belong to no other tile.  The diagonal blocks are the block
// solver's (written back by it).  Both products are three-term TF32 with FP32
// accumulation in TMEM, as in the slab pass.
//
// Shared memory, 8 KB chunks of 64 rows x 128 bytes (128-byte swizzle):
//   R0  chunks 0-1   T tile (K-major, chunk = k half), split in place to TF32 hi
//   R1  chunks 2-3   TF32 lo of the T tile
//   R2  chunks 4-7   F_b image; after product 1 X^T hi / lo (rows n, chunk = m
//                    half), the B operand of product 2
//   R3  chunks 8-11  F_a image, the A operand of product 2 (row j holds F_a[:, j]);
//                    after product 2 the staging of Y (rows m, chunk = n half)
//   then max |F| of every pair (K floats).
// A thread holds half a row of Y: T[IJ_a, IJ_b] = Y is written from registers
// (a warp's 16 rows are 64-byte column segments), T[IJ_b, IJ_a] = Y^T through the
// staging and TMA.
// A single thread issues tcgen05.mma at about one instruction per 80 cycles,
// slower than the tensor core runs these 64 x 64 x 8 products, so the three
// terms of a product are issued by three warps (lane 0 of warps 0, 1, 2) into
// three accumulators of 64 TMEM columns, which the drains add.  Lane 0 of warp 3
// issues the copies while the products run: the store of the previous tile's
// staging and this tile's F_a during product 1, the next T tile (R0, R1 dead)
// during product 2, the next F_b once product 2 has completed.
// The M = 64 accumulator holds row i in TMEM lane 32 (i / 16) + i % 16; each warp
// drains its 16 rows, lanes 16-31 taking the upper 32 columns through a shuffle.
constexpr int kTileChunks = 12;
constexpr uint32_t kTileTBytes = sizeof(float) * 2 * kFChunk;       // the T tile
size_t tile_smem_bytes(int K) { return sizeof(float) * ((size_t)kTileChunks * kFChunk + (size_t)K) + 1024; }

struct TileMaps {
    CUtensorMap t;          // T, boxes of 32 x 32
};

__device__ __forceinline__ int next_tile(int t, int ntiles, int K, const float* fm, int& a, int& b) {
    for (; t < ntiles; t += gridDim.x) {
        decode_tile(t, K, a, b);
        if (fm[a] != 0.f || fm[b] != 0.f) break;         // W_a = W_b = I: unchanged
    }
    return t;
}

__device__ __forceinline__ void issue_tile_t(const TileMaps& maps, int Ia, int Ja, int Ib, int Jb, float* R0,
                                             uint64_t* bar) {
    tc::mbar_expect_tx(bar, kTileTBytes);
#pragma unroll
    for (int c = 0; c < 2; ++c)                          // k half: columns I_b, J_b of the tile
#pragma unroll
        for (int r = 0; r < 2; ++r)                      // m half: rows I_a, J_a of the tile
            tc::tma_load_2d(R0 + c * kFChunk + r * 32 * 32, &maps.t, (c ? Jb : Ib) * kB, (r ? Ja : Ia) * kB, bar);
}

__device__ __forceinline__ void issue_fimage(const float* __restrict__ Fimg, int p, float* dst, uint64_t* bar) {
    tc::mbar_expect_tx(bar, kFImageBytes);
    tc::bulk_load(dst, Fimg + (size_t)p * kFImage, kFImageBytes, bar);
}

constexpr int kTileTmemCols = 256;                   // three 64-column accumulators

// 32 columns [32 h, 32 h + 32) of row 16 (warp) + lane % 16 of the sum of the
// nacc accumulators (64 columns apart) for h = lane / 16: lanes 16-31 receive
// the upper half of lane - 16's row.
__device__ __forceinline__ void drain_half(uint32_t lanebase, int h, int nacc, float* d) {
    float v[32], w[32];
    tc::tmem_ld16(lanebase + 32, v);
    tc::tmem_ld16(lanebase + 48, v + 16);
    if (nacc == 3) {
        tc::tmem_ld16(lanebase + 64 + 32, w);
        tc::tmem_ld16(lanebase + 64 + 48, w + 16);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] += w[j];
        tc::tmem_ld16(lanebase + 128 + 32, w);
        tc::tmem_ld16(lanebase + 128 + 48, w + 16);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] += w[j];
    } else {
        tc::tmem_wait_ld();
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) d[j] = __shfl_up_sync(0xffffffffu, v[j], 16);
    tc::tmem_ld16(lanebase, v);
    tc::tmem_ld16(lanebase + 16, v + 16);
    if (nacc == 3) {
        tc::tmem_ld16(lanebase + 64, w);
        tc::tmem_ld16(lanebase + 64 + 16, w + 16);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] += w[j];
        tc::tmem_ld16(lanebase + 128, w);
        tc::tmem_ld16(lanebase + 128 + 16, w + 16);
        tc::tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] += w[j];
    } else {
        tc::tmem_wait_ld();
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) d[j] = h ? d[j] : v[j];
}

// The term of a three-term product issued by this warp (0: hi hi, 1: lo hi,
// 2: hi lo; A and B each a hi chunk pair followed by a lo chunk pair) into its
// own accumulator, then a commit to done.
__device__ __forceinline__ void issue_term(uint32_t tmem, int warp, const float* A, const float* B,
                                          uint32_t idesc, uint64_t* done) {
    const float* Ap = A + (warp == 1 ? 2 * kFChunk : 0);
    const float* Bp = B + (warp == 2 ? 2 * kFChunk : 0);
    const uint32_t d = tmem + (uint32_t)(64 * warp);
#pragma unroll
    for (int ks = 0; ks < kM / 8; ++ks) {
        const int ch = ks >> 2;
        const uint32_t off = (ks & 3) * 32;
        tc::mma_tf32(d, tc::smem_desc_sw128(tc::smem_u32(Ap + ch * kFChunk) + off),
                     tc::smem_desc_sw128(tc::smem_u32(Bp + ch * kFChunk) + off), idesc, ks > 0);
    }
    tc::commit(done);
}

// Element (row n, column m) of a transposed plane (chunks by m half, rows n):
// lanes 16-31 visit their rows in the order j ^ 4, which puts their 16-byte
// units in the other half of the 128-byte row and keeps the stores conflict-free.
__device__ __forceinline__ int tposed_off(int n, int m) {
    return (m >> 5) * kFChunk + tc::sw128_off(n, (m & 31) >> 2) + (m & 3);
}

// T[IJ_b, IJ_a] = Y^T from the staging in R3 (boxes of 32 rows m x 32 floats n).
__device__ __forceinline__ void store_staging(const TileMaps& maps, const float* R3, int Ia, int Ja, int Ib,
                                              int Jb) {
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int r = 0; r < 2; ++r)
            tc::tma_store_2d(&maps.t, (c ? Jb : Ib) * kB, (r ? Ja : Ia) * kB, R3 + c * kFChunk + r * 1024);
    tc::bulk_commit();
}

__global__ void __launch_bounds__(kTcThreads, 2)
k_tile_tc(const __grid_constant__ TileMaps maps, float* __restrict__ T, const float* __restrict__ Fimg, int N,
          int ntiles, const float* __restrict__ fmax, int round, int terms, unsigned long long* __restrict__ err,
          unsigned long long* __restrict__ tiles_done) {
    extern __shared__ unsigned char smraw[];
    float* R0 = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    float* R1 = R0 + 2 * kFChunk;
    float* R2 = R0 + 4 * kFChunk;
    float* R3 = R0 + 8 * kFChunk;
    float* fm = R0 + kTileChunks * kFChunk;
    __shared__ __align__(8) uint64_t fullT, fullFb, fullFa, mma_done;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nblocks = N / kB, K = N / kM;
    const int nterm = terms == 3 ? 3 : 1;                // issuing warps = accumulators
    if (tid == 0) {
        tc::mbar_init(&fullT, 1);
        tc::mbar_init(&fullFb, 1);
        tc::mbar_init(&fullFa, 1);
        tc::mbar_init(&mma_done, nterm);
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot, kTileTmemCols);
    for (int i = tid; i < K; i += kTcThreads) fm[i] = fmax[i];
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t lanebase = tmem + ((uint32_t)(32 * warp) << 16);
    const int h = lane >> 4;                             // column half of this lane
    const int m = 16 * warp + (lane & 15);               // tile row (accumulator row)
    const bool mma_lane = lane == 0 && warp < nterm;    // issues one term of each product
    const bool copy_lane = tid == 96;                    // issues the asynchronous copies
    int a, b;
    int t = next_tile(blockIdx.x, ntiles, K, fm, a, b);
    if (copy_lane && t < ntiles) {
        int Ia, Ja, Ib, Jb;
        round_pair(round, a, nblocks, Ia, Ja);
        round_pair(round, b, nblocks, Ib, Jb);
        issue_tile_t(maps, Ia, Ja, Ib, Jb, R0, &fullT);
        issue_fimage(Fimg, b, R2, &fullFb);
        issue_fimage(Fimg, a, R3, &fullFa);
    }
    bool ok = true;
    unsigned long long done = 0;
    int pIa = 0, pJa = 0, pIb = 0, pJb = 0;              // the tile whose staging is pending (copy lane)
    bool pending = false;
    constexpr uint32_t idesc = tc::instr_desc(tc::kFmtTF32, kM, kM);
    for (int k = 0; t < ntiles; ++k) {
        int Ia, Ja, Ib, Jb;
        round_pair(round, a, nblocks, Ia, Ja);
        round_pair(round, b, nblocks, Ib, Jb);
        int an = 0, bn = 0;
        const int tn = next_tile(t + gridDim.x, ntiles, K, fm, an, bn);
        ok = tc::mbar_wait(&fullT, k & 1, kTcWait) && ok;
        // split the T tile: hi in place, lo to R1 (same swizzled offsets)
#pragma unroll
        for (int i = tid; i < 2 * kFChunk / 4; i += kTcThreads) {
            const float4 x = reinterpret_cast<const float4*>(R0)[i];
            float4 hh, ll;
            tc::split_tf32(x.x, hh.x, ll.x);
            tc::split_tf32(x.y, hh.y, ll.y);
            tc::split_tf32(x.z, hh.z, ll.z);
            tc::split_tf32(x.w, hh.w, ll.w);
            reinterpret_cast<float4*>(R0)[i] = hh;
            reinterpret_cast<float4*>(R1)[i] = ll;
        }
        ok = tc::mbar_wait(&fullFb, k & 1, kTcWait) && ok;
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();                                 // also: the previous staging is written
        tc::fence_after_sync();
        if (mma_lane && ok) issue_term(tmem, warp, R0, R2, idesc, &mma_done);   // product 1: D = T_ab F_b
        if (copy_lane && pending) {                      // the previous tile's Y^T, then this F_a
            store_staging(maps, R3, pIa, pJa, pIb, pJb);
            tc::bulk_wait_read();
            pending = false;
            issue_fimage(Fimg, a, R3, &fullFa);
        }
        ok = tc::mbar_wait(&mma_done, 0, kTcWait) && ok;
        tc::fence_after_sync();
        // X = T_ab + D (delta form; hi + lo = T exactly), kept in registers, and
        // its TF32 split written transposed over F_b
        float x[32];
        drain_half(lanebase, h, nterm, x);
#pragma unroll
        for (int j4 = 0; j4 < 8; ++j4) {
            const int off = h * kFChunk + tc::sw128_off(m, j4);
            const float4 th = *reinterpret_cast<const float4*>(R0 + off);
            const float4 tl = *reinterpret_cast<const float4*>(R1 + off);
            x[4 * j4 + 0] += th.x + tl.x;
            x[4 * j4 + 1] += th.y + tl.y;
            x[4 * j4 + 2] += th.z + tl.z;
            x[4 * j4 + 3] += th.w + tl.w;
        }
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
            const float v = h ? x[jj ^ 4] : x[jj];
            const int n = 32 * h + (jj ^ (4 * h));
            float vh, vl;
            tc::split_tf32(v, vh, vl);
            R2[tposed_off(n, m)] = vh;
            R2[2 * kFChunk + tposed_off(n, m)] = vl;
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (mma_lane) {                                  // product 2: D = F_a^T X
            ok = tc::mbar_wait(&fullFa, k & 1, kTcWait) && ok;
            if (ok) issue_term(tmem, warp, R3, R2, idesc, &mma_done);
        }
        if (copy_lane && tn < ntiles) {                  // R0 and R1 are dead: the next T tile
            int Ian, Jan, Ibn, Jbn;
            round_pair(round, an, nblocks, Ian, Jan);
            round_pair(round, bn, nblocks, Ibn, Jbn);
            issue_tile_t(maps, Ian, Jan, Ibn, Jbn, R0, &fullT);
        }
        ok = tc::mbar_wait(&mma_done, 1, kTcWait) && ok;
        tc::fence_after_sync();
        if (copy_lane && tn < ntiles) issue_fimage(Fimg, bn, R2, &fullFb);     // X^T is dead
        float d[32];
        drain_half(lanebase, h, nterm, d);
        tc::fence_before_sync();                         // TMEM is read (product 1 follows a barrier)
        if (ok) {
#pragma unroll
            for (int j = 0; j < 32; ++j) x[j] += d[j];   // Y row m, columns [32 h, 32 h + 32)
            // T[IJ_a, IJ_b] = Y: row gm of columns gn0 .. gn0 + 31 (16 lanes: 64 bytes per column)
            const int gm = m < kB ? Ia * kB + m : Ja * kB + m - kB;
            const int gn0 = (h ? Jb : Ib) * kB;
            float* col = T + (size_t)gn0 * N + gm;
#pragma unroll
            for (int j = 0; j < 32; ++j) col[(size_t)j * N] = x[j];
            // staging of Y over F_a (dead since product 2): rows m, chunk = n half
#pragma unroll
            for (int j4 = 0; j4 < 8; ++j4)
                *reinterpret_cast<float4*>(R3 + h * kFChunk + tc::sw128_off(m, j4)) =
                    make_float4(x[4 * j4], x[4 * j4 + 1], x[4 * j4 + 2], x[4 * j4 + 3]);
            tc::fence_proxy_async();
        }
        if (copy_lane && ok) {
            ++done;
            pending = true;
            pIa = Ia; pJa = Ja; pIb = Ib; pJb = Jb;
        }
        t = tn;
        a = an;
        b = bn;
    }
    __syncthreads();                                     // the last staging is written
    if (copy_lane) {
        if (pending) store_staging(maps, R3, pIa, pJa, pIb, pJb);
        tc::bulk_wait_all();
        if (done) atomicAdd(tiles_done, done);
    }
    if (!ok) atomicExch(err, 1ull);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTileTmemCols);
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

// TF32 image of F_b (the slab pass's B operand) from the block solve's
// row-major F_b, and max |F_b|.
__global__ void __launch_bounds__(256)
k_fimg32(const float* __restrict__ Wbuf, float* __restrict__ Fimg, float* __restrict__ fmax) {
    __shared__ float red[8];
    const int b = blockIdx.x;
    const float* F = Wbuf + (size_t)b * kM * kM;
    write_fimage(Fimg + (size_t)b * kFImage, [&](int k, int n) { return F[k * kM + n]; });
    float mx = 0.f;
    for (int t = threadIdx.x; t < kM * kM; t += blockDim.x) mx = fmaxf(mx, fabsf(F[t]));
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
    // two sets of (W, F image (2 planes), max|F|), plus the sweep scratch
    return 2 * (sizeof(float) * K * kM * kM * 3 + sizeof(float) * K + 1024) + sizeof(double) * 1100 + 4096;
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

int twosided_sweeps_tc32(float* T, float* Vt, int N, int n, double tol_abs, double eps_skip, int max_sweeps,
                         int max_inner, void* work, cudaStream_t s, SweepResult* res) {
    if (N % kM != 0) { set_error_msg("tensor-core engine: N must be a multiple of 64"); return MPJ_BAD_ARG; }
    const int K = N / kM;
    Arena ar;
    ar.base = static_cast<char*>(work);
    ar.size = tc32_workspace_bytes(N);
    // Two sets of block-rotation buffers: the V pass of round g runs on a side
    // stream (after the tile pass of round g), overlapping the next block solves.
    float *Wbuf[2], *Fimg[2], *fmax[2];
    for (int set = 0; set < 2; ++set) {
        Wbuf[set] = ar.take<float>((size_t)K * kM * kM);
        Fimg[set] = ar.take<float>((size_t)K * kFImage);
        fmax[set] = ar.take<float>((size_t)K);
    }
    double* partial = ar.take<double>(1024);
    double* offv = ar.take<double>(4);
    // [0] rotations, [1] error flag, [2] tiles updated by the tile pass
    unsigned long long* rot = ar.take<unsigned long long>(4);
    if (!Wbuf[1] || !Fimg[1] || !fmax[1] || !partial || !offv || !rot) {
        set_error_msg("workspace too small");
        return MPJ_BAD_ARG;
    }
    HostScratch hs;
    MPJ_TRY(hs.init());
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_solve2_nb, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)InnerLayout<float, kM>::bytes));
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_pass_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPassSmem));
    const size_t tile_smem = tile_smem_bytes(K);
    MPJ_CUDA_TRY(cudaFuncSetAttribute(k_tile_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem));
    TileMaps tmaps;                                      // the tile pass: T in boxes of 32 x 32
    PassMaps vmaps;                                      // the V pass: slabs of V
    MPJ_TRY(encode_rows(&tmaps.t, T, N, N, kB));
    MPJ_TRY(encode_rows(&vmaps.x, Vt, N, N, kSlab));
    SideStream side;
    MPJ_TRY(side.init(s));
    s = side.main;                                       // high priority: the critical path
    MPJ_CUDA_TRY(cudaMemsetAsync(rot, 0, 3 * sizeof(unsigned long long), s));
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
    const int ntiles = K * (K - 1) / 2;
    const int gridt = ntiles < 2 * sm_count() ? (ntiles > 0 ? ntiles : 1) : 2 * sm_count();
    const int gridv = N >= 8192 ? items : (items < 2 * sm_count() ? items : 2 * sm_count());
    const float tau = (float)(tol_abs / (double)N);
    const float gate = 1.0f / 4096.0f;                   // Newton-Schulz when some |F| >= 2^-12
    // TF32 products per tile: 3 (about FP32 accuracy) or 1 (hi*hi only, about
    // 2^-11: a lower-precision step 1, mpj_options.stage1_tf32_terms)
    const int terms = knobs().stage1_terms;
    const int cross = N >= kB * kB ? cross_schedule(false, false) : 0;     // see cross_schedule
    while (res->sweeps < max_sweeps) {
        if (!std::isfinite(off)) { res->status = MPJ_NONFINITE_INPUT; break; }
        if (!(off > tol_abs)) { res->status = MPJ_SUCCESS; break; }
        MPJ_CUDA_TRY(cudaMemsetAsync(rot, 0, sizeof(unsigned long long), s));
        MPJ_CUDA_TRY(cudaMemsetAsync(rot + 2, 0, sizeof(unsigned long long), s));
        for (int r = 0; r < rounds; ++r) {
            const int set = side.begin_round();
            if (set < 0) return MPJ_CUDA_ERROR;
            {
                MPJ_PROF(PC_SOLVE2_F32, s);
                k_solve2_nb<<<K, kSolve32Threads, InnerLayout<float, kM>::bytes, s>>>(
                    T, N, Wbuf[set], Fimg[set], fmax[set], r, (float)eps_skip, tau, gate, max_inner, cross, rot);
            }
            MPJ_LAUNCH_CHECK("k_solve2_nb");
            if (ntiles > 0) {
                MPJ_PROF(PC_TILE_F32, s);
                k_tile_tc<<<gridt, kTcThreads, tile_smem, s>>>(tmaps, T, Fimg[set], N, ntiles, fmax[set], r, terms,
                                                               rot + 1, rot + 2);
            }
            MPJ_LAUNCH_CHECK("k_tile_tc");
            // the V pass joins after the tile pass, so that it overlaps only the
            // next round's block solves
            MPJ_TRY(side.after_solve());
            {
                // Persistent (two CTAs per SM) while a CTA has few tiles; one tile per CTA
                // for N >= 8192, where the SM slots then free up tile by tile for the next
                // block solve on the high-priority stream.
                MPJ_PROF(PC_TCV_F32, side.sv);
                k_pass_tc<<<gridv, kTcThreads, kPassSmem, side.sv>>>(vmaps, Fimg[set], N, n_slabs, items, fmax[set],
                                                                     r, terms, rot + 1);
            }
            MPJ_LAUNCH_CHECK("k_pass_tc V");
            MPJ_TRY(side.after_v());
            side.end_round();
        }
        MPJ_TRY(offnorm2(T, false, N, n, partial, offv, s));
        MPJ_CUDA_TRY(cudaMemcpyAsync(hs.d, offv, sizeof(double), cudaMemcpyDeviceToHost, s));
        MPJ_CUDA_TRY(cudaMemcpyAsync(hs.u, rot, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        MPJ_CUDA_TRY(cudaStreamSynchronize(s));
        prof_flush();
        if (hs.u[1]) { set_error_msg("tensor-core tile: MMA completion wait timed out"); return MPJ_CUDA_ERROR; }
        // algorithmic bytes of the tile pass: each updated tile is read once and
        // written twice (64 x 64 FP32 each)
        prof_add_units(PC_TILE_F32, (double)hs.u[2] * 3.0 * sizeof(float) * kM * kM);
        off = sqrt(hs.d[0]);
        res->sweeps += 1;
        res->rotations += (double)hs.u[0];
        if (trace_on())
            fprintf(stderr, "[mpj] twosided<tc32> n=%d sweep %d: %llu rotations, %llu tiles, off %.3e\n", n,
                    res->sweeps, hs.u[0], hs.u[2], off);
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
        Fimg[set] = ar.take<float>((size_t)K * kFImage);
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
    PassMaps mc, mv;                                     // rotations: row slabs of C and of V
    MPJ_TRY(encode_rows(&mc.x, C, N, m, kSlab));
    MPJ_TRY(encode_rows(&mv.x, V, N, N, kSlab));
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
                k_pass_tc<<<gridV, kTcThreads, kPassSmem, side.sv>>>(mv, Fimg[set], N, slabsV, itemsV, fmax[set], r,
                                                                     3, rot + 1);
            }
            MPJ_LAUNCH_CHECK("k_pass_tc V (one-sided)");
            MPJ_TRY(side.after_v());
            {
                MPJ_PROF(PC_APPLY1_F32, s);
                k_pass_tc<<<gridC, kTcThreads, kPassSmem, s>>>(mc, Fimg[set], N, slabsC, itemsC, fmax[set], r, 3,
                                                               rot + 1);
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
