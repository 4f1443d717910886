/*
 * oracle.c -- plain, slow, obviously-correct CPU reference for the mixed
 * precision preconditioned Jacobi method (Zhang & Bai, arXiv 2211.03339).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant with
 * the CUDA library.
 *
 * Conventions
 *   - every matrix is column-major with leading dimension = number of rows;
 *   - scalar, single-threaded loops in the order the paper states them;
 *   - compiled with -ffp-contract=off so that no FMA is formed and results
 *     are identical on x86-64 and AArch64;
 *   - "u"  = 2^-53 (double precision, the paper's omega),
 *     "ups" = 2^-24 (single precision, the paper's upsilon), Sec. 6.
 *
 * Functions and the passages they follow
 *   orc_rotation        Lemma 3.1 (cosine-sine pair that zeroes a_ij)
 *   orc_rotation_f      Lemma 3.1 evaluated in single precision
 *   orc_offnorm         ||off(A)||_F, notation of Sec. 1
 *   orc_syev_cyclic     Algorithm 3.2, row-cyclic order, skip rule of Remark 3.7
 *   orc_syev_cyclic_f   the same algorithm in single precision (step 1 of Alg. 4.1)
 *   orc_mgs             modified Gram-Schmidt QR (Lemma 2.1, textbook MGS)
 *   orc_congruence      T = Q^T A Q (step 3 of Algorithm 4.1)
 *   orc_syevj_plain     Algorithm 3.2 from T = A, P = I
 *   orc_syevj_mp        Algorithm 4.1 (steps 1-4)
 *   orc_gesvj_cyclic    Algorithm 5.1 (one-sided, Lemma 5.1 rotations)
 *   orc_gesvj_plain     Algorithm 5.1 followed by the post-processing of Alg. 5.2
 *   orc_gesvj_mp        Algorithm 5.2 (steps 1-3 + sweeps + post-processing)
 *
 * Readings where the paper is silent (also listed in the design notes):
 *   - the rotated entry t_pq is stored as exactly zero after a rotation;
 *   - a pair is skipped (t_pq := 0, not counted in JU) when
 *       |t_pq| <= eps_skip * sqrt(|t_pp t_qq|)    (Remark 3.7, eps_skip = u);
 *   - the while-test of Alg. 3.2/4.1 is made at the start of a sweep; a
 *     sweep that applies no rotation also ends the iteration;
 *   - one-sided Jacobi: a pair is skipped when |c_i^T c_j| <= tol_rot *
 *     ||c_i|| ||c_j||; the iteration stops when a sweep applies fewer than
 *     ju_ratio * N rotations (Sec. 6 uses ju_ratio = 2e-4) or none;
 *   - eigenvalues are returned in ascending order with the columns of the
 *     eigenvector matrix permuted to match; singular values descending.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_U   1.1102230246251565e-16   /* 2^-53 */
#define ORC_UPS 5.9604644775390625e-08   /* 2^-24 */

typedef struct {
    int    sweeps;          /* SP: sweeps executed                          */
    long   rotations;       /* rotations applied (not skipped)              */
    double off_initial;     /* ||off(T)||_F before the first sweep          */
    double off_final;       /* ||off(T)||_F after the last sweep            */
    int    sweeps_stage1;   /* Alg. 4.1/5.2: sweeps of the low-precision step */
    long   rotations_stage1;
} orc_stats;

static void stats_clear(orc_stats* st) { if (st) memset(st, 0, sizeof(*st)); }

/* ------------------------------------------------------------------ */
/* Lemma 3.1: for the 2x2 symmetric block [[a_ii, a_ij], [a_ij, a_jj]] */
/* return (c, s) with c = (1+t^2)^(-1/2), s = t c and                   */
/* mu = (a_jj - a_ii) / (2 a_ij), t = 1/(mu + sqrt(1+mu^2)) for mu >= 0,*/
/* t = 1/(mu - sqrt(1+mu^2)) otherwise; (1, 0) when a_ij = 0.           */
/* ------------------------------------------------------------------ */
void orc_rotation(double aii, double ajj, double aij, double* c, double* s)
{
    if (aij == 0.0) { *c = 1.0; *s = 0.0; return; }
    double mu = (ajj - aii) / (2.0 * aij);
    double t;
    if (mu >= 0.0) t = 1.0 / (mu + sqrt(1.0 + mu * mu));
    else           t = 1.0 / (mu - sqrt(1.0 + mu * mu));
    *c = 1.0 / sqrt(1.0 + t * t);
    *s = t * (*c);
}

void orc_rotation_f(float aii, float ajj, float aij, float* c, float* s)
{
    if (aij == 0.0f) { *c = 1.0f; *s = 0.0f; return; }
    float mu = (ajj - aii) / (2.0f * aij);
    float t;
    if (mu >= 0.0f) t = 1.0f / (mu + sqrtf(1.0f + mu * mu));
    else            t = 1.0f / (mu - sqrtf(1.0f + mu * mu));
    *c = 1.0f / sqrtf(1.0f + t * t);
    *s = t * (*c);
}

/* ||off(A)||_F = sqrt(sum_{i != j} a_ij^2) */
double orc_offnorm(const double* A, int n)
{
    double s = 0.0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
            if (i != j) s += A[(size_t)j * n + i] * A[(size_t)j * n + i];
    return sqrt(s);
}

static double offnorm_f(const float* A, int n)
{
    double s = 0.0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
            if (i != j) s += (double)A[(size_t)j * n + i] * (double)A[(size_t)j * n + i];
    return sqrt(s);
}

double orc_fnorm(const double* A, int m, int n)
{
    double s = 0.0;
    for (size_t k = 0; k < (size_t)m * n; ++k) s += A[k] * A[k];
    return sqrt(s);
}

/* ------------------------------------------------------------------ */
/* One Jacobi step in the (p,q) plane, B = J^T A J with J = J(p,q;c,s)  */
/* of eq. (3.1): J_pp = J_qq = c, J_pq = s, J_qp = -s.  The entries      */
/* follow the proofs of Lemmas 3.4/3.5:                                  */
/*   b_pp = c^2 a_pp - 2 s c a_pq + s^2 a_qq                             */
/*   b_qq = s^2 a_pp + 2 s c a_pq + c^2 a_qq                             */
/*   b_pj = c a_pj - s a_qj,  b_qj = s a_pj + c a_qj   (j != p, q)       */
/*   b_pq = b_qp = 0                                                     */
/* and P = P J updates columns p and q of P the same way.               */
/* ------------------------------------------------------------------ */
static void rotate_two_sided(double* T, double* P, int n, int p, int q, double c, double s)
{
    double app = T[(size_t)p * n + p], aqq = T[(size_t)q * n + q], apq = T[(size_t)q * n + p];
    for (int j = 0; j < n; ++j) {
        if (j == p || j == q) continue;
        double apj = T[(size_t)j * n + p], aqj = T[(size_t)j * n + q];
        double bpj = c * apj - s * aqj;
        double bqj = s * apj + c * aqj;
        T[(size_t)j * n + p] = bpj; T[(size_t)p * n + j] = bpj;   /* row p and column p */
        T[(size_t)j * n + q] = bqj; T[(size_t)q * n + j] = bqj;   /* row q and column q */
    }
    T[(size_t)p * n + p] = c * c * app - 2.0 * s * c * apq + s * s * aqq;
    T[(size_t)q * n + q] = s * s * app + 2.0 * s * c * apq + c * c * aqq;
    T[(size_t)q * n + p] = 0.0;
    T[(size_t)p * n + q] = 0.0;
    if (P) {
        for (int i = 0; i < n; ++i) {
            double xp = P[(size_t)p * n + i], xq = P[(size_t)q * n + i];
            P[(size_t)p * n + i] = c * xp - s * xq;
            P[(size_t)q * n + i] = s * xp + c * xq;
        }
    }
}

static void rotate_two_sided_f(float* T, float* P, int n, int p, int q, float c, float s)
{
    float app = T[(size_t)p * n + p], aqq = T[(size_t)q * n + q], apq = T[(size_t)q * n + p];
    for (int j = 0; j < n; ++j) {
        if (j == p || j == q) continue;
        float apj = T[(size_t)j * n + p], aqj = T[(size_t)j * n + q];
        float bpj = c * apj - s * aqj;
        float bqj = s * apj + c * aqj;
        T[(size_t)j * n + p] = bpj; T[(size_t)p * n + j] = bpj;
        T[(size_t)j * n + q] = bqj; T[(size_t)q * n + j] = bqj;
    }
    T[(size_t)p * n + p] = c * c * app - 2.0f * s * c * apq + s * s * aqq;
    T[(size_t)q * n + q] = s * s * app + 2.0f * s * c * apq + c * c * aqq;
    T[(size_t)q * n + p] = 0.0f;
    T[(size_t)p * n + q] = 0.0f;
    if (P) {
        for (int i = 0; i < n; ++i) {
            float xp = P[(size_t)p * n + i], xq = P[(size_t)q * n + i];
            P[(size_t)p * n + i] = c * xp - s * xq;
            P[(size_t)q * n + i] = s * xp + c * xq;
        }
    }
}

/* Apply a single rotation (p,q) -- exposed so that tests can check the   */
/* invariants of Lemma 3.1 on one step.                                   */
void orc_jacobi_step(double* T, double* P, int n, int p, int q)
{
    double c, s;
    orc_rotation(T[(size_t)p * n + p], T[(size_t)q * n + q], T[(size_t)q * n + p], &c, &s);
    rotate_two_sided(T, P, n, p, q, c, s);
}

/* ------------------------------------------------------------------ */
/* Algorithm 3.2 in the row-cyclic order, in place on T (n x n) and P.  */
/* The while-test ||off(T)||_F > tol * normA is made before each sweep. */
/* off_hist (optional, length max_sweeps+1) receives ||off(T)||_F        */
/* before each sweep and after the last one.                            */
/* Returns 0 when converged, 3 when max_sweeps was reached first.       */
/* ------------------------------------------------------------------ */
int orc_syev_cyclic(double* T, double* P, int n, double tol, double normA,
                    double eps_skip, int max_sweeps, orc_stats* st, double* off_hist)
{
    int sweeps = 0; long rot = 0; int status = 3;
    double off = orc_offnorm(T, n);
    if (st) st->off_initial = off;
    if (off_hist) off_hist[0] = off;
    while (sweeps < max_sweeps) {
        if (!(off > tol * normA)) { status = 0; break; }
        long rot_sweep = 0;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = T[(size_t)q * n + p];
                double app = T[(size_t)p * n + p], aqq = T[(size_t)q * n + q];
                if (apq == 0.0) continue;
                if (fabs(apq) <= eps_skip * sqrt(fabs(app * aqq))) {     /* Remark 3.7 */
                    T[(size_t)q * n + p] = 0.0; T[(size_t)p * n + q] = 0.0;
                    continue;
                }
                double c, s;
                orc_rotation(app, aqq, apq, &c, &s);
                rotate_two_sided(T, P, n, p, q, c, s);
                ++rot_sweep;
            }
        }
        ++sweeps; rot += rot_sweep;
        off = orc_offnorm(T, n);
        if (off_hist) off_hist[sweeps] = off;
        if (rot_sweep == 0) { status = 0; break; }
    }
    if (status == 3 && !(off > tol * normA)) status = 0;
    if (st) { st->sweeps = sweeps; st->rotations = rot; st->off_final = off; }
    return status;
}

/* Step 1 of Algorithm 4.1 in precision upsilon: the same cyclic Jacobi  */
/* carried out entirely in single precision.                            */
int orc_syev_cyclic_f(float* T, float* P, int n, double tol, double normA,
                      float eps_skip, int max_sweeps, orc_stats* st)
{
    int sweeps = 0; long rot = 0; int status = 3;
    double off = offnorm_f(T, n);
    while (sweeps < max_sweeps) {
        if (!(off > tol * normA)) { status = 0; break; }
        long rot_sweep = 0;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                float apq = T[(size_t)q * n + p];
                float app = T[(size_t)p * n + p], aqq = T[(size_t)q * n + q];
                if (apq == 0.0f) continue;
                if (fabsf(apq) <= eps_skip * sqrtf(fabsf(app * aqq))) {
                    T[(size_t)q * n + p] = 0.0f; T[(size_t)p * n + q] = 0.0f;
                    continue;
                }
                float c, s;
                orc_rotation_f(app, aqq, apq, &c, &s);
                rotate_two_sided_f(T, P, n, p, q, c, s);
                ++rot_sweep;
            }
        }
        ++sweeps; rot += rot_sweep;
        off = offnorm_f(T, n);
        if (rot_sweep == 0) { status = 0; break; }
    }
    if (status == 3 && !(off > tol * normA)) status = 0;
    if (st) { st->sweeps = sweeps; st->rotations = rot; st->off_final = off; }
    return status;
}

/* ------------------------------------------------------------------ */
/* Modified Gram-Schmidt, Z (m x n, rank n) = Q R with r_jj > 0.        */
/*   for j = 1..n: r_jj = ||z_j||, q_j = z_j / r_jj,                     */
/*                 for k > j: r_jk = q_j^T z_k, z_k = z_k - r_jk q_j     */
/* R (n x n, may be NULL) receives the upper triangle.                  */
/* Returns 4 if some r_jj == 0 (rank deficient), else 0.                */
/* ------------------------------------------------------------------ */
int orc_mgs(const double* Z, int m, int n, double* Q, double* R)
{
    memcpy(Q, Z, sizeof(double) * (size_t)m * n);
    if (R) memset(R, 0, sizeof(double) * (size_t)n * n);
    for (int j = 0; j < n; ++j) {
        double* qj = Q + (size_t)j * m;
        double nrm = 0.0;
        for (int i = 0; i < m; ++i) nrm += qj[i] * qj[i];
        nrm = sqrt(nrm);
        if (nrm == 0.0) return 4;
        for (int i = 0; i < m; ++i) qj[i] = qj[i] / nrm;
        if (R) R[(size_t)j * n + j] = nrm;
        for (int k = j + 1; k < n; ++k) {
            double* zk = Q + (size_t)k * m;
            double r = 0.0;
            for (int i = 0; i < m; ++i) r += qj[i] * zk[i];
            for (int i = 0; i < m; ++i) zk[i] = zk[i] - r * qj[i];
            if (R) R[(size_t)k * n + j] = r;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Step 3 of Algorithm 4.1: T = Q^T A Q in double precision.             */
/* W = A Q, then t_ij = q_i^T w_j for i <= j; t_ji := t_ij (the computed */
/* product is made exactly symmetric from its upper triangle).          */
/* ------------------------------------------------------------------ */
void orc_congruence(const double* A, const double* Q, int n, double* T)
{
    double* W = (double*)malloc(sizeof(double) * (size_t)n * n);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += A[(size_t)k * n + i] * Q[(size_t)j * n + k];
            W[(size_t)j * n + i] = s;
        }
    for (int j = 0; j < n; ++j)
        for (int i = 0; i <= j; ++i) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += Q[(size_t)i * n + k] * W[(size_t)j * n + k];
            T[(size_t)j * n + i] = s;
            T[(size_t)i * n + j] = s;
        }
    free(W);
}

/* ascending sort of diag(T) into Lambda, columns of V permuted to match */
static void sort_eig(const double* T, const double* P, int n, double* Lambda, double* V)
{
    int* idx = (int*)malloc(sizeof(int) * (size_t)n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    /* insertion sort: plain and stable */
    for (int i = 1; i < n; ++i) {
        int k = idx[i]; double key = T[(size_t)k * n + k]; int j = i - 1;
        while (j >= 0 && T[(size_t)idx[j] * n + idx[j]] > key) { idx[j + 1] = idx[j]; --j; }
        idx[j + 1] = k;
    }
    for (int i = 0; i < n; ++i) {
        Lambda[i] = T[(size_t)idx[i] * n + idx[i]];
        if (V) memcpy(V + (size_t)i * n, P + (size_t)idx[i] * n, sizeof(double) * (size_t)n);
    }
    free(idx);
}

/* Algorithm 3.2 from T = A, P = I. */
int orc_syevj_plain(const double* A, int n, double* Lambda, double* V, double tol,
                    int max_sweeps, orc_stats* st)
{
    stats_clear(st);
    double* T = (double*)malloc(sizeof(double) * (size_t)n * n);
    double* P = (double*)calloc((size_t)n * n, sizeof(double));
    memcpy(T, A, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i) P[(size_t)i * n + i] = 1.0;
    double normA = orc_fnorm(A, n, n);
    int status = orc_syev_cyclic(T, P, n, tol, normA, ORC_U, max_sweeps, st, NULL);
    sort_eig(T, P, n, Lambda, V);
    free(T); free(P);
    return status;
}

/* Step 1 of Alg. 4.1: A32 = fl32(A), cyclic Jacobi in single precision,  */
/* Z sorted by ascending eigenvalue and widened exactly to double.        */
int orc_stage1_syev_f(const double* A, int n, double tol1, int max_sweeps,
                      double* Z, double* D, orc_stats* st)
{
    float* T = (float*)malloc(sizeof(float) * (size_t)n * n);
    float* P = (float*)calloc((size_t)n * n, sizeof(float));
    for (size_t k = 0; k < (size_t)n * n; ++k) T[k] = (float)A[k];
    for (int i = 0; i < n; ++i) P[(size_t)i * n + i] = 1.0f;
    double norm32 = 0.0;                 /* ||A32||_F */
    for (size_t k = 0; k < (size_t)n * n; ++k) norm32 += (double)T[k] * (double)T[k];
    norm32 = sqrt(norm32);
    orc_stats s1; stats_clear(&s1);
    int status = orc_syev_cyclic_f(T, P, n, tol1, norm32, (float)ORC_UPS, max_sweeps, &s1);
    /* widen and sort */
    double* Td = (double*)malloc(sizeof(double) * (size_t)n * n);
    double* Pd = (double*)malloc(sizeof(double) * (size_t)n * n);
    for (size_t k = 0; k < (size_t)n * n; ++k) { Td[k] = (double)T[k]; Pd[k] = (double)P[k]; }
    sort_eig(Td, Pd, n, D, Z);
    if (st) { st->sweeps_stage1 = s1.sweeps; st->rotations_stage1 = s1.rotations; }
    free(T); free(P); free(Td); free(Pd);
    return status;
}

/* Algorithm 4.1.  Optional outputs T0 (n x n) and Q (n x n) expose the   */
/* intermediate results of steps 2-3 for stage-wise checks.              */
int orc_syevj_mp(const double* A, int n, double* Lambda, double* V, double tol,
                 double tol1, int max_sweeps, orc_stats* st, double* Q_out, double* T0_out)
{
    stats_clear(st);
    size_t nn = (size_t)n * n;
    double* Z = (double*)malloc(sizeof(double) * nn);
    double* D = (double*)malloc(sizeof(double) * (size_t)n);
    double* Q = (double*)malloc(sizeof(double) * nn);
    double* T = (double*)malloc(sizeof(double) * nn);
    orc_stats s1; stats_clear(&s1);
    orc_stage1_syev_f(A, n, tol1, 4 * max_sweeps, Z, D, &s1);                /* step 1 */
    int status = orc_mgs(Z, n, n, Q, NULL);                                  /* step 2 */
    if (status == 0) {
        orc_congruence(A, Q, n, T);                                          /* step 3 */
        if (Q_out) memcpy(Q_out, Q, sizeof(double) * nn);
        if (T0_out) memcpy(T0_out, T, sizeof(double) * nn);
        double normA = orc_fnorm(A, n, n);
        status = orc_syev_cyclic(T, Q, n, tol, normA, ORC_U, max_sweeps, st, NULL);  /* step 4, P = Q */
        sort_eig(T, Q, n, Lambda, V);
    }
    if (st) { st->sweeps_stage1 = s1.sweeps_stage1; st->rotations_stage1 = s1.rotations_stage1; }
    free(Z); free(D); free(Q); free(T);
    return status;
}

/* ------------------------------------------------------------------ */
/* Algorithm 5.1: one-sided cyclic Jacobi on C (m x n), V (n x n).       */
/* Lemma 5.1: alpha = c_i^T c_i, beta = c_j^T c_j, gamma = c_i^T c_j,    */
/* mu = (beta - alpha)/(2 gamma), t as in Lemma 3.1, C = C J, V = V J.    */
/* While-test ||off(C^T C)||_F > eps * ||C^T C||_F at the start of each  */
/* sweep; a pair is skipped when |gamma| <= tol_rot sqrt(alpha beta); a  */
/* sweep that applies fewer than ju_ratio*N rotations (or none) ends it. */
/* ------------------------------------------------------------------ */
static void gram_norms(const double* C, int m, int n, double* off, double* full)
{
    double so = 0.0, sf = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double g = 0.0;
            for (int k = 0; k < m; ++k) g += C[(size_t)i * m + k] * C[(size_t)j * m + k];
            sf += g * g;
            if (i != j) so += g * g;
        }
    *off = sqrt(so); *full = sqrt(sf);
}

int orc_gesvj_cyclic(double* C, double* V, int m, int n, double eps, double tol_rot,
                     double ju_ratio, int max_sweeps, orc_stats* st)
{
    int sweeps = 0; long rot = 0; int status = 3;
    double off, full;
    gram_norms(C, m, n, &off, &full);
    if (st) st->off_initial = off;
    double N = 0.5 * (double)n * (double)(n - 1);
    while (sweeps < max_sweeps) {
        if (!(off > eps * full)) { status = 0; break; }
        long rot_sweep = 0;
        for (int i = 0; i < n - 1; ++i) {
            for (int j = i + 1; j < n; ++j) {
                double* ci = C + (size_t)i * m;
                double* cj = C + (size_t)j * m;
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int k = 0; k < m; ++k) {
                    alpha += ci[k] * ci[k];
                    beta  += cj[k] * cj[k];
                    gamma += ci[k] * cj[k];
                }
                if (gamma == 0.0) continue;
                if (fabs(gamma) <= tol_rot * sqrt(alpha) * sqrt(beta)) continue;
                double mu = (beta - alpha) / (2.0 * gamma);
                double t;
                if (mu >= 0.0) t = 1.0 / (mu + sqrt(1.0 + mu * mu));
                else           t = 1.0 / (mu - sqrt(1.0 + mu * mu));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < m; ++k) {
                    double x = ci[k], y = cj[k];
                    ci[k] = c * x - s * y;
                    cj[k] = s * x + c * y;
                }
                if (V) {
                    double* vi = V + (size_t)i * n;
                    double* vj = V + (size_t)j * n;
                    for (int k = 0; k < n; ++k) {
                        double x = vi[k], y = vj[k];
                        vi[k] = c * x - s * y;
                        vj[k] = s * x + c * y;
                    }
                }
                ++rot_sweep;
            }
        }
        ++sweeps; rot += rot_sweep;
        gram_norms(C, m, n, &off, &full);
        if (rot_sweep == 0 || (double)rot_sweep < ju_ratio * N) { status = 0; break; }
    }
    if (status == 3 && !(off > eps * full)) status = 0;
    if (st) { st->sweeps = sweeps; st->rotations = rot; st->off_final = off; }
    return status;
}

/* Steps 11-13 of Alg. 5.2: order columns by decreasing ||c_j||, then     */
/* sigma_j = ||c_j|| and u_j = c_j / sigma_j.  Returns 4 on a zero column. */
static int svd_post(const double* C, const double* Vw, int m, int n,
                    double* Sigma, double* U, double* V)
{
    double* nrm = (double*)malloc(sizeof(double) * (size_t)n);
    int* idx = (int*)malloc(sizeof(int) * (size_t)n);
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int k = 0; k < m; ++k) s += C[(size_t)j * m + k] * C[(size_t)j * m + k];
        nrm[j] = sqrt(s); idx[j] = j;
    }
    for (int i = 1; i < n; ++i) {
        int k = idx[i]; double key = nrm[k]; int j = i - 1;
        while (j >= 0 && nrm[idx[j]] < key) { idx[j + 1] = idx[j]; --j; }
        idx[j + 1] = k;
    }
    int status = 0;
    for (int j = 0; j < n; ++j) {
        int src = idx[j];
        double sg = nrm[src];
        Sigma[j] = sg;
        if (sg == 0.0) status = 4;
        if (U) for (int k = 0; k < m; ++k) U[(size_t)j * m + k] = (sg == 0.0) ? 0.0 : C[(size_t)src * m + k] / sg;
        if (V) memcpy(V + (size_t)j * n, Vw + (size_t)src * n, sizeof(double) * (size_t)n);
    }
    free(nrm); free(idx);
    return status;
}

/* Algorithm 5.1 from C = A, V = I, with the post-processing of Alg. 5.2. */
int orc_gesvj_plain(const double* A, int m, int n, double* Sigma, double* U, double* V,
                    double eps, double tol_rot, double ju_ratio, int max_sweeps, orc_stats* st)
{
    stats_clear(st);
    double* C = (double*)malloc(sizeof(double) * (size_t)m * n);
    double* Vw = (double*)calloc((size_t)n * n, sizeof(double));
    memcpy(C, A, sizeof(double) * (size_t)m * n);
    for (int i = 0; i < n; ++i) Vw[(size_t)i * n + i] = 1.0;
    int status = orc_gesvj_cyclic(C, Vw, m, n, eps, tol_rot, ju_ratio, max_sweeps, st);
    int ps = svd_post(C, Vw, m, n, Sigma, U, V);
    if (status == 0) status = ps;
    free(C); free(Vw);
    return status;
}

/* Step 1 of Alg. 5.2 in precision upsilon: one-sided Jacobi of fl32(A) in */
/* single precision; Z = accumulated right rotations, columns ordered by   */
/* decreasing column norm, widened exactly to double.                      */
int orc_stage1_gesvj_f(const double* A, int m, int n, float tol_rot, double ju_ratio,
                       int max_sweeps, double* Z, orc_stats* st)
{
    float* C = (float*)malloc(sizeof(float) * (size_t)m * n);
    float* P = (float*)calloc((size_t)n * n, sizeof(float));
    for (size_t k = 0; k < (size_t)m * n; ++k) C[k] = (float)A[k];
    for (int i = 0; i < n; ++i) P[(size_t)i * n + i] = 1.0f;
    double N = 0.5 * (double)n * (double)(n - 1);
    int sweeps = 0; long rot = 0;
    while (sweeps < max_sweeps) {
        long rot_sweep = 0;
        for (int i = 0; i < n - 1; ++i) {
            for (int j = i + 1; j < n; ++j) {
                float* ci = C + (size_t)i * m;
                float* cj = C + (size_t)j * m;
                float alpha = 0.0f, beta = 0.0f, gamma = 0.0f;
                for (int k = 0; k < m; ++k) {
                    alpha += ci[k] * ci[k];
                    beta  += cj[k] * cj[k];
                    gamma += ci[k] * cj[k];
                }
                if (gamma == 0.0f) continue;
                if (fabsf(gamma) <= tol_rot * sqrtf(alpha) * sqrtf(beta)) continue;
                float mu = (beta - alpha) / (2.0f * gamma);
                float t;
                if (mu >= 0.0f) t = 1.0f / (mu + sqrtf(1.0f + mu * mu));
                else            t = 1.0f / (mu - sqrtf(1.0f + mu * mu));
                float c = 1.0f / sqrtf(1.0f + t * t), s = t * c;
                for (int k = 0; k < m; ++k) {
                    float x = ci[k], y = cj[k];
                    ci[k] = c * x - s * y;
                    cj[k] = s * x + c * y;
                }
                float* vi = P + (size_t)i * n;
                float* vj = P + (size_t)j * n;
                for (int k = 0; k < n; ++k) {
                    float x = vi[k], y = vj[k];
                    vi[k] = c * x - s * y;
                    vj[k] = s * x + c * y;
                }
                ++rot_sweep;
            }
        }
        ++sweeps; rot += rot_sweep;
        if (rot_sweep == 0 || (double)rot_sweep < ju_ratio * N) break;
    }
    /* order by decreasing column norm of C (largest singular value first) */
    double* nrm = (double*)malloc(sizeof(double) * (size_t)n);
    int* idx = (int*)malloc(sizeof(int) * (size_t)n);
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int k = 0; k < m; ++k) s += (double)C[(size_t)j * m + k] * (double)C[(size_t)j * m + k];
        nrm[j] = s; idx[j] = j;
    }
    for (int i = 1; i < n; ++i) {
        int k = idx[i]; double key = nrm[k]; int j = i - 1;
        while (j >= 0 && nrm[idx[j]] < key) { idx[j + 1] = idx[j]; --j; }
        idx[j + 1] = k;
    }
    for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) Z[(size_t)j * n + k] = (double)P[(size_t)idx[j] * n + k];
    if (st) { st->sweeps_stage1 = sweeps; st->rotations_stage1 = rot; }
    free(C); free(P); free(nrm); free(idx);
    return 0;
}

/* Algorithm 5.2. */
int orc_gesvj_mp(const double* A, int m, int n, double* Sigma, double* U, double* V,
                 double eps, double tol_rot, double ju_ratio, int max_sweeps, orc_stats* st)
{
    stats_clear(st);
    size_t nn = (size_t)n * n;
    double* Z = (double*)malloc(sizeof(double) * nn);
    double* Q = (double*)malloc(sizeof(double) * nn);
    double* C = (double*)malloc(sizeof(double) * (size_t)m * n);
    orc_stats s1; stats_clear(&s1);
    orc_stage1_gesvj_f(A, m, n, (float)(sqrt((double)m) * ORC_UPS), ju_ratio, 4 * max_sweeps, Z, &s1); /* step 1 */
    int status = orc_mgs(Z, n, n, Q, NULL);                                        /* step 2 */
    if (status == 0) {
        for (int j = 0; j < n; ++j)                                                /* step 3: C = A Q */
            for (int i = 0; i < m; ++i) {
                double s = 0.0;
                for (int k = 0; k < n; ++k) s += A[(size_t)k * m + i] * Q[(size_t)j * n + k];
                C[(size_t)j * m + i] = s;
            }
        status = orc_gesvj_cyclic(C, Q, m, n, eps, tol_rot, ju_ratio, max_sweeps, st); /* steps 4-10, V = Q */
        int ps = svd_post(C, Q, m, n, Sigma, U, V);                                /* steps 11-13 */
        if (status == 0) status = ps;
    }
    if (st) { st->sweeps_stage1 = s1.sweeps_stage1; st->rotations_stage1 = s1.rotations_stage1; }
    free(Z); free(Q); free(C);
    return status;
}
