// jacobi_device.cuh -- device building blocks of the block Jacobi engines.
//
//   rr_index        parallel (round-robin tournament) ordering: in round r the
//                   2K blocks are paired so that every pair meets once in 2K-1
//                   rounds; pairs of one round are disjoint (the GPU analogue of
//                   the "merry-go-round" order of Sec. 6).
//   rotation_cs     Lemma 3.1 (and, on a Gram matrix, Lemma 5.1); in FP64 with
//                   reciprocals and inverse square roots (rotation_cs_fast).
//   inner_jacobi    cyclic Jacobi on one 2b x 2b block-pair problem held in
//                   shared memory, parallel order inside the block, with the
//                   rotations accumulated into the orthogonal 2b x 2b block W.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace mpj {

constexpr int kThreads = 256;       // tile kernels: a 16 x 16 thread grid
constexpr int kSolveThreads = 512;  // block-pair solves: more threads per inner round

// Player at position `pos` (0 <= pos < P, P even) in round r of the circle method:
// position 0 holds player 0, the others rotate through players 1..P-1.
__device__ __forceinline__ int rr_index(int r, int pos, int P) {
    return pos == 0 ? 0 : 1 + (pos - 1 + r) % (P - 1);
}

template <class Real> __device__ __forceinline__ Real rabs(Real x) { return x < Real(0) ? -x : x; }

// Lemma 3.1: (c, s) with mu = (a_qq - a_pp)/(2 a_pq), t = sign(mu)/(|mu| + sqrt(1+mu^2)),
// c = 1/sqrt(1+t^2), s = t c (IEEE arithmetic; the FP32 solves use it as it stands).
template <class Real>
__device__ __forceinline__ void rotation_cs(Real app, Real aqq, Real apq, Real& c, Real& s, Real& t) {
    Real mu = (aqq - app) / (Real(2) * apq);
    Real am = mu < Real(0) ? -mu : mu;
    t = Real(1) / (am + sqrt(Real(1) + mu * mu));
    if (mu < Real(0)) t = -t;
    c = Real(1) / sqrt(Real(1) + t * t);
    s = t * c;
}

// Lemma 3.1 in FP64 with reciprocals and reciprocal square roots in place of
// the divisions and square roots (a few ulps in t, c, s; the serial chain of a
// step's rotations is a fraction as long, and on this GPU the block solves wait
// on that chain).  For |mu| > 2^26, t = 1/(2 mu) to working precision.  Also
// returns c - 1 = -s^2 / (1 + c) without cancellation.
__device__ __forceinline__ void rotation_cs_fast(double app, double aqq, double apq, double& c, double& s,
                                                 double& cm, double& t) {
    const double mu = (aqq - app) * (0.5 * __drcp_rn(apq));
    const double am = mu < 0.0 ? -mu : mu;
    if (am > 67108864.0) {
        t = 0.5 * __drcp_rn(mu);
    } else {
        const double h = fma(mu, mu, 1.0);
        t = __drcp_rn(am + h * rsqrt(h));
        if (mu < 0.0) t = -t;
    }
    c = rsqrt(fma(t, t, 1.0));
    s = t * c;
    cm = -(s * s) * __drcp_rn(1.0 + c);
}

// The rotation of a mixed-precision one-sided solve (Lemma 5.1 on a Gram
// matrix, FP64 diagonal, FP32 entry), in two parts.
//   rotation_angle_mixed  FP32 (its error only perturbs the rotation's effect,
//                         a convergence matter): t = tan(theta) from
//                         mu = (a_qq - a_pp) / (2 a_pq), the difference taken in
//                         FP64, and the half-angle tangent
//                         tau = t / (1 + sqrt(1 + t^2)), |tau| <= tan(pi/8);
//   rotation_from_tau     FP64, with r = 1 / (1 + tau^2) (an FP32 seed and two
//                         Newton steps): c = (1 - tau^2) r, s = 2 tau r,
//                         c - 1 = -2 tau^2 r, a rotation orthogonal to working
//                         precision whose c - 1 has no cancellation.
__device__ __forceinline__ void rotation_angle_mixed(double app, double aqq, float apq, float& tf, float& tauf) {
    const float mu = (float)(aqq - app) / (2.0f * apq);
    const float am = fabsf(mu);
    if (am > 1.0e9f) tf = 0.5f / mu;
    else tf = copysignf(1.0f / (am + sqrtf(fmaf(mu, mu, 1.0f))), mu);
    tauf = tf / (1.0f + sqrtf(fmaf(tf, tf, 1.0f)));
}
__device__ __forceinline__ void rotation_from_tau(float tauf, double& c, double& s, double& cm) {
    const float seed = 1.0f / fmaf(tauf, tauf, 1.0f);
    const double tau = (double)tauf;
    const double t2 = tau * tau;                     // exact: tau has 24 bits
    const double x = 1.0 + t2;
    double r = (double)seed;
    r = fma(r, fma(-x, r, 1.0), r);
    r = fma(r, fma(-x, r, 1.0), r);
    c = (1.0 - t2) * r;
    s = (2.0 * tau) * r;
    cm = (-2.0 * t2) * r;
}

// Shared-memory footprint of a block-pair solve for M = 2b: S, F and a third
// M x (M+1) buffer (the Gram/correction matrix of the re-orthogonalisation),
// two buffers of c, s, c-1, t of the M/2 rotations of a step, two buffers of
// pair indices and skip flags, a counter and two flags.  Carving: the Real
// arrays start at `cs` (8 (M/2) values); the int arrays at ip = cs + 8 (M/2)
// (6 (M/2) indices, then the counter at ip + 6 (M/2) and the caller's flags
// at ip + 6 (M/2) + 2).
template <class Real, int M>
struct InnerLayout {
    static constexpr int LD = M + 1;
    static constexpr int kRealRot = 8 * (M / 2);
    static constexpr int kFlagOffset = 6 * (M / 2) + 2;
    static constexpr size_t bytes =
        sizeof(Real) * (3 * M * LD + kRealRot) + sizeof(int) * (6 * (M / 2) + 8);
};

// Rotations of step r of an inner sweep (warp 0): pair (p, q) of lane `tid`, its
// (c, s, c - 1, t) or the identity when skipped, into one buffer of the step
// arrays.  Returns the number of rotations of the step (all lanes of warp 0).
template <class Real, int M>
__device__ __forceinline__ int step_rotations(const Real* S, Real* cs, int* ip, int r, int cross_round, Real eps,
                                              Real tau) {
    constexpr int LD = M + 1;
    constexpr int P = M / 2;
    const int tid = threadIdx.x;
    int mine = 0;
    if (tid < P) {
        int p, q;
        if (cross_round < 0) {
            p = rr_index(r, tid, M);
            q = rr_index(r, M - 1 - tid, M);
        } else if (r < P) {
            p = tid;
            q = P + (tid + r) % P;
        } else {
            const int qr = cross_round % (P - 1), h = tid / (P / 2), i = tid % (P / 2);
            p = h * P + rr_index(qr, i, P);
            q = h * P + rr_index(qr, P - 1 - i, P);
        }
        if (p > q) { int t = p; p = q; q = t; }
        Real apq = S[q * LD + p], app = S[p * LD + p], aqq = S[q * LD + q];
        Real c = Real(1), s = Real(0), t = Real(0), cm = Real(0);
        int skip = 1;
        Real aa = rabs(apq);
        if (apq != Real(0) && aa > tau && !(aa <= eps * sqrt(rabs(app * aqq)))) {
            if constexpr (sizeof(Real) == 8) {
                rotation_cs_fast(app, aqq, apq, c, s, cm, t);
            } else {
                rotation_cs(app, aqq, apq, c, s, t);
                cm = -(s * s) / (Real(1) + c);
            }
            skip = 0;
        }
        cs[tid] = c; cs[P + tid] = s; cs[2 * P + tid] = cm; cs[3 * P + tid] = t;
        ip[tid] = p; ip[P + tid] = q; ip[2 * P + tid] = skip;
        mine = !skip;
    }
    return __popc(__ballot_sync(0xffffffffu, mine));
}

// Work items of the two-sided S update, u in [0, P(P+1)/2): the P diagonal 2x2
// blocks first (u < P, a = b = u), then the strictly upper blocks (a < b) row by
// row.  Enumerating only a <= b keeps whole warps on the same branch, so the
// FP64 pipe is not spent on masked-off lanes.  Packed as a | b << 8, -1 past
// the end.  Each thread keeps its (at most three) items for the whole solve.
template <int P>
__device__ __forceinline__ int upper_item(int u) {
    if (u >= P * (P + 1) / 2) return -1;
    if (u < P) return u | (u << 8);
    int v = u - P, a = 0;
    while (v >= P - 1 - a) { v -= P - 1 - a; ++a; }
    return a | ((a + 1 + v) << 8);
}

// Two-sided update of S by the rotations of one step buffer: the 2x2 blocks
// (a, b), a <= b, of this thread's items, mirrored below the diagonal.
template <class Real, int M>
__device__ __forceinline__ void step_update_s(Real* S, const Real* cs, const int* ip, const int (&items)[3]) {
    constexpr int LD = M + 1;
    constexpr int P = M / 2;
    const Real* sn = cs + P;
    const Real* tt = cs + 3 * P;
    const int* iq = ip + P;
    const int* sk = ip + 2 * P;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (items[k] < 0) continue;
        const int a = items[k] & 255, b = items[k] >> 8;
        int pa = ip[a], qa = iq[a];
        Real ca = cs[a], sa = sn[a];
        if (a == b) {
            // b_pp = c^2 a_pp - 2 s c a_pq + s^2 a_qq and b_qq = s^2 a_pp + 2 s c a_pq
            // + c^2 a_qq reduce, for the (c, s) of Lemma 3.1, to a_pp - t a_pq and
            // a_qq + t a_pq: one rounding of a small correction instead of three
            // rounded products of the full diagonal entries.
            Real apq = S[qa * LD + pa], ta = tt[a];
            S[pa * LD + pa] = S[pa * LD + pa] - ta * apq;
            S[qa * LD + qa] = S[qa * LD + qa] + ta * apq;
            S[qa * LD + pa] = Real(0);
            S[pa * LD + qa] = Real(0);
        } else {
            if (sk[a] && sk[b]) continue;     // both rotations are the identity
            int pb = ip[b], qb = iq[b];
            Real cb = cs[b], sb = sn[b];
            Real x00 = S[pb * LD + pa], x01 = S[qb * LD + pa];
            Real x10 = S[pb * LD + qa], x11 = S[qb * LD + qa];
            // rows: J_a^T X
            Real y00 = ca * x00 - sa * x10, y01 = ca * x01 - sa * x11;
            Real y10 = sa * x00 + ca * x10, y11 = sa * x01 + ca * x11;
            // columns: (J_a^T X) J_b
            Real z00 = cb * y00 - sb * y01, z01 = sb * y00 + cb * y01;
            Real z10 = cb * y10 - sb * y11, z11 = sb * y10 + cb * y11;
            S[pb * LD + pa] = z00; S[qb * LD + pa] = z01;
            S[pb * LD + qa] = z10; S[qb * LD + qa] = z11;
            S[pa * LD + pb] = z00; S[pa * LD + qb] = z01;
            S[qa * LD + pb] = z10; S[qa * LD + qb] = z11;
        }
    }
}

// F <- F J + (J - I) for the rotations of one step buffer (columns p, q of every
// rotation), by the threads t0, t0 + nt, ... (t0 = this thread's index among them).
// FP64: items [0, P (M - 2)) are the rows other than p and q of each rotation
// (plain rotations of two entries); the last 2P items are rows p and q, which
// also get the entries of J - I (c - 1 and +-s).  Keeping those few rows apart
// spares the other lanes predicated FP64 corrections, which occupy the FP64
// pipe like executed ones.  FP32 keeps one item per (row, rotation).
template <class Real, int M>
__device__ __forceinline__ void step_update_f(Real* F, const Real* cs, const int* ip, int t0, int nt) {
    constexpr int LD = M + 1;
    constexpr int P = M / 2;
    constexpr int R = M - 2;
    const Real* sn = cs + P;
    const Real* cm = cs + 2 * P;
    const int* iq = ip + P;
    const int* sk = ip + 2 * P;
    if constexpr (sizeof(Real) != 8) {
        // One warp per rotation (t0 and nt are whole warps): its parameters are
        // loaded once, and the lanes take the rows.
        const int lane = t0 & 31;
        for (int a = t0 >> 5; a < P; a += nt >> 5) {
            if (sk[a]) continue;
            const int pa = ip[a], qa = iq[a];
            const Real c = cs[a], s = sn[a], cma = cm[a];
#pragma unroll
            for (int row = lane; row < M; row += 32) {
                const Real fp = F[pa * LD + row], fq = F[qa * LD + row];
                Real np = c * fp - s * fq, nq = s * fp + c * fq;
                if (row == pa) { np += cma; nq += s; }
                else if (row == qa) { np -= s; nq += cma; }
                F[pa * LD + row] = np;
                F[qa * LD + row] = nq;
            }
        }
        return;
    }
    for (int t = t0; t < M * P; t += nt) {
        int a, row;
        const bool regular = t < P * R;
        if (regular) {
            a = t / R;
            row = t - a * R;
        } else {
            a = (t - P * R) >> 1;
            row = 0;
        }
        if (sk[a]) continue;
        const int pa = ip[a], qa = iq[a];                  // pa < qa
        if (regular) {
            row += row >= pa;
            row += row >= qa;
        } else {
            row = (t & 1) ? qa : pa;
        }
        const Real c = cs[a], s = sn[a];
        const Real fp = F[pa * LD + row], fq = F[qa * LD + row];
        Real np = c * fp - s * fq, nq = s * fp + c * fq;
        if (!regular) {
            const bool atq = (t & 1) != 0;
            np += atq ? -s : cm[a];
            nq += atq ? cm[a] : s;
        }
        F[pa * LD + row] = np;
        F[qa * LD + row] = nq;
    }
}

// step_update_f restricted to rows [row0, row0 + nrows) of F (items (row, rotation)),
// for solves whose F rows are spread over the CTAs of a cluster.
template <class Real, int M>
__device__ __forceinline__ void step_update_f_rows(Real* F, const Real* cs, const int* ip, int t0, int nt, int row0,
                                                   int nrows) {
    constexpr int LD = M + 1;
    constexpr int P = M / 2;
    const Real* sn = cs + P;
    const Real* cm = cs + 2 * P;
    const int* iq = ip + P;
    const int* sk = ip + 2 * P;
    for (int t = t0; t < nrows * P; t += nt) {
        const int a = t / nrows, row = row0 + (t - a * nrows);
        if (sk[a]) continue;
        const int pa = ip[a], qa = iq[a];
        const Real c = cs[a], s = sn[a];
        const Real fp = F[pa * LD + row], fq = F[qa * LD + row];
        Real np = c * fp - s * fq, nq = s * fp + c * fq;
        if (row == pa) { np += cm[a]; nq += s; }
        else if (row == qa) { np -= s; nq += cm[a]; }
        F[pa * LD + row] = np;
        F[qa * LD + row] = nq;
    }
}

// Cyclic Jacobi on the symmetric M x M matrix S (shared, column-major, ld M+1).
// The accumulated rotation W = J_1 J_2 ... is kept as F = W - I (F must hold
// the start, e.g. 0): F <- F J + (J - I), so that the rounding errors of F are
// relative to |F| and W = I + F stays orthogonal to working precision when
// the rotations are small (the nearly diagonal T of step 4 of Alg. 4.1).
// One inner sweep = M-1 parallel rounds of M/2 disjoint rotations.  A pair is
// skipped (its entry set to zero, not counted) when |s_pq| <= eps sqrt(|s_pp s_qq|)
// (Remark 3.7) or |s_pq| <= tau (entries that cannot matter for the stopping
// test).  Stops after an inner sweep with no rotation or after max_inner
// sweeps.  Returns the number of rotations applied (all threads).  With
// nrows < M only rows [row0, row0 + nrows) of F are accumulated.
// Must be called by all threads of the block (any multiple of 32, at least 256,
// so that three S-update items per thread cover the P(P+1)/2 <= 528 blocks).
// With cross_round >= 0 an inner sweep is the M/2 steps that rotate every pair
// (i, j) with i in the first block and j in the second once, followed by one
// step over pairs inside each block (round cross_round mod (M/2 - 1) of the
// tournament over that block), so that over the rounds of an outer sweep every
// intra-block pair is still visited.
// Software pipeline: the rotations of a step depend only on S after the
// previous step, not on F, so warp 0 forms those of step r + 1 (the serial
// chain of divisions and square roots) while the other warps accumulate
// step r into F; the step arrays are double buffered.
template <class Real, int M>
__device__ int inner_jacobi(Real* S, Real* F, Real* cs, int* ip, Real eps, Real tau, int max_inner,
                            int cross_round = -1, int row0 = 0, int nrows = M) {
    constexpr int P = M / 2;
    static_assert(P <= 32, "pair count must fit one warp");
    volatile int* cnt = ip + 6 * P;  // [0] applied in this sweep
    const int tid = threadIdx.x;
    const int nsteps = cross_round >= 0 ? P + 1 : M - 1;
    int items[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) items[k] = upper_item<P>(tid + k * (int)blockDim.x);
    int total = 0;
    for (int sweep = 0; sweep < max_inner; ++sweep) {
        int applied = 0;
        if (tid < 32) applied += step_rotations<Real, M>(S, cs, ip, 0, cross_round, eps, tau);
        __syncthreads();
        for (int r = 0; r < nsteps; ++r) {
            const int cur = r & 1;
            Real* csc = cs + cur * 4 * P;
            int* ipc = ip + cur * 3 * P;
            step_update_s<Real, M>(S, csc, ipc, items);
            __syncthreads();
            const bool more = r + 1 < nsteps;
            if (more && tid < 32)
                applied += step_rotations<Real, M>(S, cs + (cur ^ 1) * 4 * P, ip + (cur ^ 1) * 3 * P, r + 1,
                                                   cross_round, eps, tau);
            else if (nrows != M)
                step_update_f_rows<Real, M>(F, csc, ipc, more ? tid - 32 : tid, more ? blockDim.x - 32 : blockDim.x,
                                            row0, nrows);
            else if (more) {
                if (sizeof(Real) == 4 && (blockDim.x & 127) == 0) {
                    // FP32: the F work goes to the warps of the other three
                    // sub-partitions (warp w runs on sub-partition w mod 4), so that
                    // warp 0's chain of rotations has its sub-partition to itself
                    const int w = tid >> 5;
                    if (w & 3)
                        step_update_f<Real, M>(F, csc, ipc, ((w >> 2) * 3 + (w & 3) - 1) * 32 + (tid & 31),
                                               (int)(blockDim.x >> 7) * 96);
                } else {
                    step_update_f<Real, M>(F, csc, ipc, tid - 32, blockDim.x - 32);
                }
            } else
                step_update_f<Real, M>(F, csc, ipc, tid, blockDim.x);
            __syncthreads();
        }
        if (tid == 0) cnt[0] = applied;
        __syncthreads();
        int c = cnt[0];
        __syncthreads();
        total += c;
        if (c == 0) break;
    }
    return total;
}

// ---------------------------------------------------------------- mixed precision
// inner_jacobi for a problem whose S only steers the rotations (the Gram matrix
// of a one-sided solve: C and V change through W alone).  S is held as an FP64
// diagonal dg (with an FP32 copy dgf for the threshold test) and an FP32
// off-diagonal E (both scaled by the same power of two, ld M+1, diagonal
// entries of E unused); the Rutishauser update moves the diagonal in FP64
// (d_p - t e_pq, d_q + t e_pq) and E is rotated in FP32, so the rounding of E
// is relative to the off-diagonal entries themselves.  The angles are formed in
// FP32 (rotation_angle_mixed), and F = W - I is accumulated in FP64 with the
// FP64 rotations of the same half-angle tangents (rotation_from_tau), so W
// stays orthogonal to working precision; FP32 rounding in E and in the angles
// only perturbs their effect (a convergence matter).
//
// Three-stage software pipeline over the steps k of an inner sweep, two
// barriers per step:
//   A_k  all warps: S update with the FP32 rotations of step k;
//   B_k  warp 0: the FP32 rotations of step k+1 from S;
//        warp 1: the FP64 (c, s, c - 1) of step k;
//        other warps: F <- F J + (J - I) with the FP64 rotations of step k-1.
// So the FP64 work never sits on the chain of dependent steps through S.
template <int M>
struct MixedBufs {
    static constexpr int P = M / 2, LD = M + 1;
    static constexpr size_t kOffDg = ((size_t)M * LD * 4 + 7) / 8 * 8;
    static constexpr size_t kOffDgf = kOffDg + 8 * M;
    static constexpr size_t kOffRf = kOffDgf + 4 * M;                 // 2 sets of (c, s, t, tau), FP32
    static constexpr size_t kOffRd = (kOffRf + 2 * 4 * P * 4 + 7) / 8 * 8;   // 2 sets of (c, s, c - 1), FP64
    static constexpr size_t kOffIp = kOffRd + 2 * 3 * P * 8;          // 3 sets of (p, q, skip)
    static constexpr size_t bytes = kOffIp + 3 * 3 * P * 4;
    float* E;
    double* dg;
    float* dgf;
    float* rf;
    double* rd;
    int* ip;
    __device__ explicit MixedBufs(unsigned char* base)
        : E(reinterpret_cast<float*>(base)), dg(reinterpret_cast<double*>(base + kOffDg)),
          dgf(reinterpret_cast<float*>(base + kOffDgf)), rf(reinterpret_cast<float*>(base + kOffRf)),
          rd(reinterpret_cast<double*>(base + kOffRd)), ip(reinterpret_cast<int*>(base + kOffIp)) {}
};

// FP32 rotations of step r (warp 0; lane a < P takes pair a) into one rf set
// (c, s, t, tau) and one ip set (p, q, skip).  Returns the number of
// rotations of the step (all lanes of warp 0).
template <int M>
__device__ __forceinline__ int step_angles_mixed(const MixedBufs<M>& b, float* rf, int* ipw, int r, int cross_round,
                                                 float eps) {
    constexpr int LD = M + 1;
    constexpr int P = M / 2;
    const int lane = threadIdx.x & 31;
    int mine = 0;
    if (lane < P) {
        int p, q;
        if (cross_round < 0) {
            p = rr_index(r, lane, M);
            q = rr_index(r, M - 1 - lane, M);
        } else if (r < P) {
            p = lane;
            q = P + (lane + r) % P;
        } else {
            const int qr = cross_round % (P - 1), h = lane / (P / 2), i = lane % (P / 2);
            p = h * P + rr_index(qr, i, P);
            q = h * P + rr_index(qr, P - 1 - i, P);
        }
        if (p > q) { int t = p; p = q; q = t; }
        const float ef = b.E[q * LD + p];
        float c = 1.f, s = 0.f, t = 0.f, tau = 0.f;
        int skip = 1;
        // |s_pq| > eps sqrt(s_pp s_qq) in FP32 on the FP32 copies of the diagonal
        // (scaled to at most 2 and at least 2^-76: the products stay normal)
        if (ef != 0.f && fabsf(ef) > eps * (sqrtf(fabsf(b.dgf[p])) * sqrtf(fabsf(b.dgf[q])))) {
            rotation_angle_mixed(b.dg[p], b.dg[q], ef, t, tau);
            const float r1 = 1.0f / fmaf(tau, tau, 1.0f);
            c = fmaf(-tau, tau, 1.0f) * r1;
            s = (2.0f * tau) * r1;
            skip = 0;
        }
        rf[lane] = c; rf[P + lane] = s; rf[2 * P + lane] = t; rf[3 * P + lane] = tau;
        ipw[lane] = p; ipw[P + lane] = q; ipw[2 * P + lane] = skip;
        mine = !skip;
    }
    return __popc(__ballot_sync(0xffffffffu, mine));
}

// S update of one step: the FP64 diagonal (Rutishauser, with the step's t) and
// the FP32 2 x 2 blocks of E, as step_update_s.
template <int M>
__device__ __forceinline__ void step_update_s_mixed(const MixedBufs<M>& b, const float* rf, const int* ipr,
                                                    const int (&items)[3]) {
    constexpr int LD = M + 1;
    constexpr int P = M / 2;
    float* E = b.E;
    const int* iq = ipr + P;
    const int* sk = ipr + 2 * P;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (items[k] < 0) continue;
        const int a = items[k] & 255, bb = items[k] >> 8;
        const int pa = ipr[a], qa = iq[a];
        if (a == bb) {
            // a skipped pair (t = 0) keeps its diagonal and loses its entry, as in inner_jacobi
            const double apq = (double)E[qa * LD + pa], ta = (double)rf[2 * P + a];
            const double dp = fma(-ta, apq, b.dg[pa]), dq = fma(ta, apq, b.dg[qa]);
            b.dg[pa] = dp;
            b.dg[qa] = dq;
            b.dgf[pa] = (float)dp;
            b.dgf[qa] = (float)dq;
            E[qa * LD + pa] = 0.f;
            E[pa * LD + qa] = 0.f;
        } else {
            if (sk[a] && sk[bb]) continue;
            const int pb = ipr[bb], qb = iq[bb];
            const float ca = rf[a], sa = rf[P + a], cb = rf[bb], sb = rf[P + bb];
            const float x00 = E[pb * LD + pa], x01 = E[qb * LD + pa];
            const float x10 = E[pb * LD + qa], x11 = E[qb * LD + qa];
            const float y00 = ca * x00 - sa * x10, y01 = ca * x01 - sa * x11;
            const float y10 = sa * x00 + ca * x10, y11 = sa * x01 + ca * x11;
            const float z00 = cb * y00 - sb * y01, z01 = sb * y00 + cb * y01;
            const float z10 = cb * y10 - sb * y11, z11 = sb * y10 + cb * y11;
            E[pb * LD + pa] = z00; E[qb * LD + pa] = z01;
            E[pb * LD + qa] = z10; E[qb * LD + qa] = z11;
            E[pa * LD + pb] = z00; E[pa * LD + qb] = z01;
            E[qa * LD + pb] = z10; E[qa * LD + qb] = z11;
        }
    }
}

// F update of one step with its FP64 rotations (rd set) on rows
// [row0, row0 + nrows), by threads t0, t0 + nt, ...
template <int M>
__device__ __forceinline__ void step_f_mixed(double* F, const double* rdr, const int* ipr, int t0, int nt, int row0,
                                             int nrows) {
    if (nrows != M) step_update_f_rows<double, M>(F, rdr, ipr, t0, nt, row0, nrows);
    else step_update_f<double, M>(F, rdr, ipr, t0, nt);
}

// Same schedule, counting and stopping rule as inner_jacobi (tau = 0); the
// caller has filled b.E, b.dg and b.dgf.  With nrows < M only rows
// [row0, row0 + nrows) of F are accumulated (the other CTAs of a cluster, which
// form the same rotations, hold the rest).  cnt: one int of shared scratch.
template <int M>
__device__ int inner_jacobi_mixed(const MixedBufs<M>& b, double* F, volatile int* cnt, float eps, int max_inner,
                                  int cross_round = -1, int row0 = 0, int nrows = M) {
    constexpr int P = M / 2;
    static_assert(P <= 32, "pair count must fit one warp");
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nt = (int)blockDim.x;
    const int nsteps = cross_round >= 0 ? P + 1 : M - 1;
    int items[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) items[k] = upper_item<P>(tid + k * nt);
    int total = 0;
    for (int sweep = 0; sweep < max_inner; ++sweep) {
        int applied = 0;
        if (warp == 0) applied += step_angles_mixed<M>(b, b.rf, b.ip, 0, cross_round, eps);
        __syncthreads();
        for (int k = 0; k < nsteps; ++k) {
            const float* rfk = b.rf + (k & 1) * 4 * P;
            const int* ipk = b.ip + (k % 3) * 3 * P;
            step_update_s_mixed<M>(b, rfk, ipk, items);
            __syncthreads();
            if (warp == 0) {
                if (k + 1 < nsteps)
                    applied += step_angles_mixed<M>(b, b.rf + ((k + 1) & 1) * 4 * P, b.ip + ((k + 1) % 3) * 3 * P,
                                                    k + 1, cross_round, eps);
            } else if (warp == 1) {
                const int a = tid & 31;
                if (a < P) {
                    double c = 1.0, s = 0.0, cm = 0.0;
                    if (!ipk[2 * P + a]) rotation_from_tau(rfk[3 * P + a], c, s, cm);
                    double* rdk = b.rd + (k & 1) * 3 * P;
                    rdk[a] = c; rdk[P + a] = s; rdk[2 * P + a] = cm;
                }
            } else if (k >= 1) {
                step_f_mixed<M>(F, b.rd + ((k - 1) & 1) * 3 * P, b.ip + ((k - 1) % 3) * 3 * P, tid - 64, nt - 64,
                                row0, nrows);
            }
            __syncthreads();
        }
        step_f_mixed<M>(F, b.rd + ((nsteps - 1) & 1) * 3 * P, b.ip + ((nsteps - 1) % 3) * 3 * P, tid, nt, row0,
                        nrows);
        if (tid == 0) cnt[0] = applied;
        __syncthreads();
        const int c = cnt[0];
        __syncthreads();
        total += c;
        if (c == 0) break;
    }
    return total;
}

// One Newton-Schulz step towards the orthogonal polar factor of W = I + F:
// G = W^T W - I = F + F^T + F^T F,  W <- W (I - G/2), i.e.
// F <- F - G/2 - F G/2.  G is the scratch buffer (ld M+1).  Used when the
// block rotation is far from the identity, where the M-1 rounds of rotations
// leave W non-orthogonal by a few hundred ulps.
template <class Real, int M>
__device__ void reorthogonalise(Real* F, Real* G) {
    constexpr int LD = M + 1;
    constexpr int RM = M / 16;
    const bool active = threadIdx.x < 256;             // a 16 x 16 grid of RM x RM patches
    const int tx = threadIdx.x & 15, ty = (threadIdx.x >> 4) & 15;
    Real acc[RM][RM];
    if (active) {
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < RM; ++j) acc[i][j] = Real(0);
        for (int k = 0; k < M; ++k) {
            Real a[RM], b[RM];
#pragma unroll
            for (int i = 0; i < RM; ++i) a[i] = F[(ty * RM + i) * LD + k];   // F[k][R]
#pragma unroll
            for (int j = 0; j < RM; ++j) b[j] = F[(tx * RM + j) * LD + k];   // F[k][C]
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < RM; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < RM; ++j) {
                int R = ty * RM + i, C = tx * RM + j;
                G[C * LD + R] = (F[C * LD + R] + F[R * LD + C]) + acc[i][j];
            }
    }
    __syncthreads();
    // acc = (F G)[R][C]
    if (active) {
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < RM; ++j) acc[i][j] = Real(0);
        for (int k = 0; k < M; ++k) {
            Real a[RM], b[RM];
#pragma unroll
            for (int i = 0; i < RM; ++i) a[i] = F[k * LD + ty * RM + i];     // F[R][k]
#pragma unroll
            for (int j = 0; j < RM; ++j) b[j] = G[(tx * RM + j) * LD + k];   // G[k][C]
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < RM; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < RM; ++j) {
                int R = ty * RM + i, C = tx * RM + j;
                F[C * LD + R] = F[C * LD + R] - Real(0.5) * (G[C * LD + R] + acc[i][j]);
            }
    }
    __syncthreads();
}

// Block solve epilogue shared by the two engines: optionally re-orthogonalise
// W = I + F (when max |F| >= gate), then store F row-major to Fout and, when
// fmax_out is given, max |F| (as a float) to *fmax_out -- the apply kernels use
// it to pick the arithmetic of the tile products.
template <class Real, int M>
__device__ void finish_block(Real* F, Real* G, Real* Fout, Real gate, int* flag, float* fmax_out) {
    constexpr int LD = M + 1;
    if (threadIdx.x == 0) { flag[0] = 0; flag[1] = 0; }
    __syncthreads();
    for (int t = threadIdx.x; t < M * M; t += blockDim.x) {
        int r = t % M, c = t / M;
        if (rabs(F[c * LD + r]) >= gate) flag[0] = 1;
    }
    __syncthreads();
    if (flag[0]) reorthogonalise<Real, M>(F, G);
    float mx = 0.f;
    for (int t = threadIdx.x; t < M * M; t += blockDim.x) {
        int k = t / M, c = t % M;
        Real v = F[c * LD + k];
        Fout[t] = v;                             // row-major: Fout[k*M + c] = F[k][c]
        float a = (float)rabs(v);
        mx = a > mx ? a : mx;
    }
    if (fmax_out) {
        // non-negative floats order like their bit patterns
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned int*>(flag + 1), __float_as_uint(mx));
        __syncthreads();
        if (threadIdx.x == 0) *fmax_out = __uint_as_float(reinterpret_cast<unsigned int*>(flag)[1]);
    }
}

// Local index l in [0, 2b) of the block pair (I, J) -> global row/column index.
__device__ __forceinline__ int pair_global(int l, int I, int J, int b) {
    return l < b ? I * b + l : J * b + (l - b);
}

// Block pair handled by CTA `pair` in round `round` (2K = number of blocks).
__device__ __forceinline__ void round_pair(int round, int pair, int nblocks, int& I, int& J) {
    I = rr_index(round, pair, nblocks);
    J = rr_index(round, nblocks - 1 - pair, nblocks);
    if (I > J) { int t = I; I = J; J = t; }
}

}  // namespace mpj
