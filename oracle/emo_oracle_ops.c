/*
 * FP64 CPU oracle, second part: the generation around the selection and the
 * TensorMOEA/D environmental selection (arXiv 2503.20286).
 *
 * TEST INFRASTRUCTURE ONLY, like emo_oracle.c (which provides the Philox
 * generator used here). Shares nothing with the CUDA path.
 *
 *   - Simulated binary crossover and polynomial mutation: Appendix S.I
 *     (original operators, and their tensorized forms over the population).
 *   - Random mating selection: Appendix S.I "Mating Selection" (uniform
 *     random choice of parents).
 *   - TensorMOEA/D environmental selection: Algorithm S.8 (the dense
 *     n x n index tensor I_new and the per-subproblem argmin, in the
 *     paper's order), with the PBI aggregation of Section IV-B.
 *   - IGD: mean over the reference front of the distance to the nearest
 *     population point (the quality measure of the experiments, Section V).
 *
 * Readings of silent or ambiguous points:
 *   - PM: the tensorized step printed in Appendix S.I drops the "- 1" of the
 *     original operator; the original (with "- 1") is used, so that mu = 0.5
 *     leaves x unchanged and mu = 0 moves it to the lower bound.
 *   - SBX children are clipped to [L, U] before PM (PM needs
 *     (X_c - L) / (U - L) in [0, 1]); the mutated values are clipped again.
 *   - Per-element mutation with probability p_m (1/D in the paper's runs):
 *     an element mutates when its Bernoulli draw hits; p_m = 1 is the
 *     printed tensor form. Crossover of a pair happens with probability p_c
 *     (1.0 in the paper's runs); the printed tensor form is p_c = 1.
 *   - PBI: d2 = ||(f - z) - d1 w / ||w|| ||, the distance from f - z to
 *     the line along w when (f - z) . w >= 0 (always so in the method:
 *     f >= z_min and w >= 0); the printed (f - z) - d1 w is the same when
 *     ||w|| = 1. d1 keeps the printed absolute value.
 *   - H(0) = 1 (Section III): an offspring replaces a neighbour when its
 *     aggregated value is lower or equal, as in Algorithm S.7.
 *   - argmin over the n positions of a subproblem's column takes the first
 *     minimum; positions that were not replaced hold the current solution.
 *   - z_min = per-objective minimum of z and the offspring objectives F_2.
 *   - All decisions are taken in FP64 from the FP32 inputs, k ascending, no
 *     fused multiply-add (compile with -ffp-contract=off).
 *
 * Random numbers of the generation (mating, SBX, PM) come from
 * Philox-4x32-10 keyed by the seed, counter (row, 0x80000000 | tag << 24 |
 * slot, generation): tag 1 parents (slot 0/1; x1 of slot 0 decides
 * crossover), tag 2 SBX spread (slot = variable), tag 3 mutation (slot =
 * variable; x0 decides, x1 is mu), tag 5 MOEA/D neighbour picks. A 32-bit
 * word x maps to the uniform x * 2^-32 and to the index (x * n) >> 32.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]);

#define OPS_OK 0
#define OPS_EINVAL 1
#define OPS_ENONFINITE 2
#define OPS_ENOMEM 7

static void gen_random(uint64_t seed, uint64_t gen, int64_t row, int tag, int64_t slot, uint32_t out[4])
{
    uint32_t ctr[4], key[2];
    ctr[0] = (uint32_t)row;
    ctr[1] = 0x80000000u | ((uint32_t)tag << 24) | ((uint32_t)slot & 0x00FFFFFFu);
    ctr[2] = (uint32_t)(gen & 0xFFFFFFFFu);
    ctr[3] = (uint32_t)(gen >> 32);
    key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    key[1] = (uint32_t)(seed >> 32);
    oracle_philox4x32_10(ctr, key, out);
}

static double unit_of(uint32_t x) { return (double)x * (1.0 / 4294967296.0); }

static int64_t index_of(uint32_t x, int64_t n) { return (int64_t)(((uint64_t)x * (uint64_t)n) >> 32); }

/* Bernoulli(p) from one 32-bit word: hit when x < p * 2^32 */
static int hit(uint32_t x, double p)
{
    if (p >= 1.0) return 1;
    if (!(p > 0.0)) return 0;
    return (double)x < p * 4294967296.0;
}

static double clip(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ---------------------------------------------------------------------- */
/* SBX on one variable (Appendix S.I): spread factor beta from mu and     */
/* eta_c, children 0.5[(1 + beta) x1 + (1 - beta) x2] and the mirror.     */
/* ---------------------------------------------------------------------- */
void oracle_sbx_pair(double x1, double x2, double mu, double eta_c, double* c1, double* c2)
{
    double beta;
    if (mu <= 0.5) beta = pow(2.0 * mu, 1.0 / (eta_c + 1.0));
    else beta = pow(1.0 / (2.0 - 2.0 * mu), 1.0 / (eta_c + 1.0));
    *c1 = 0.5 * ((1.0 + beta) * x1 + (1.0 - beta) * x2);
    *c2 = 0.5 * ((1.0 - beta) * x1 + (1.0 + beta) * x2);
}

/* ---------------------------------------------------------------------- */
/* Polynomial mutation of one variable (Appendix S.I, original form):     */
/* eta = eta_m + 1, delta1 = (x - l) / (u - l), delta2 = (u - x) / (u - l).*/
/* ---------------------------------------------------------------------- */
double oracle_pm_value(double x, double lo, double hi, double mu, double eta_m)
{
    const double eta = eta_m + 1.0;
    const double width = hi - lo;
    double step;
    if (mu <= 0.5) {
        const double delta1 = (x - lo) / width;
        step = pow(2.0 * mu + (1.0 - 2.0 * mu) * pow(1.0 - delta1, eta), 1.0 / eta) - 1.0;
    } else {
        const double delta2 = (hi - x) / width;
        step = 1.0 - pow(2.0 - 2.0 * mu + (2.0 * mu - 1.0) * pow(1.0 - delta2, eta), 1.0 / eta);
    }
    return x + step * width;
}

/* ---------------------------------------------------------------------- */
/* One generation's offspring for NSGA-III: random mating, SBX of each    */
/* pair, clipping, polynomial mutation, clipping, rounding to FP32.       */
/* Pair p (0 <= p < ceil(n_off / 2)) writes its first child to row p and   */
/* its second to row ceil(n_off / 2) + p when that row exists (the        */
/* tensorized SBX stacks the two children blocks). parents_out (nullable) */
/* receives the two parent indices of every pair.                         */
/* ---------------------------------------------------------------------- */
int oracle_variation(const float* X, int64_t n, int64_t d, const float* lo, const float* hi, int64_t n_off,
                     uint64_t seed, uint64_t gen, double eta_c, double eta_m, double p_c, double p_m, float* Xoff,
                     int32_t* parents_out)
{
    if (!X || !lo || !hi || !Xoff || n < 1 || d < 1 || d > 0x00FFFFFF || n_off < 1 || n > INT32_MAX ||
        n_off > INT32_MAX || !(eta_c >= 0.0) || !(eta_m >= 0.0))
        return OPS_EINVAL;
    for (int64_t k = 0; k < d; ++k)
        if (!isfinite(lo[k]) || !isfinite(hi[k]) || !(hi[k] > lo[k])) return OPS_EINVAL;
    for (int64_t i = 0; i < n * d; ++i)
        if (!isfinite(X[i])) return OPS_ENONFINITE;
    const int64_t pairs = (n_off + 1) / 2;
    for (int64_t p = 0; p < pairs; ++p) {
        uint32_t r0[4], r1[4];
        gen_random(seed, gen, p, 1, 0, r0);
        gen_random(seed, gen, p, 1, 1, r1);
        const int64_t a = index_of(r0[0], n), b = index_of(r1[0], n);
        const int cross = hit(r0[1], p_c);
        if (parents_out) { parents_out[2 * p] = (int32_t)a; parents_out[2 * p + 1] = (int32_t)b; }
        for (int child = 0; child < 2; ++child) {
            const int64_t row = child == 0 ? p : pairs + p;
            if (row >= n_off) continue;
            for (int64_t k = 0; k < d; ++k) {
                const double x1 = (double)X[a * d + k], x2 = (double)X[b * d + k];
                double c1 = x1, c2 = x2;
                if (cross) {
                    uint32_t rs[4];
                    gen_random(seed, gen, p, 2, k, rs);
                    oracle_sbx_pair(x1, x2, unit_of(rs[0]), eta_c, &c1, &c2);
                }
                double v = clip(child == 0 ? c1 : c2, (double)lo[k], (double)hi[k]);
                uint32_t rm[4];
                gen_random(seed, gen, row, 3, k, rm);
                if (hit(rm[0], p_m))
                    v = clip(oracle_pm_value(v, (double)lo[k], (double)hi[k], unit_of(rm[1]), eta_m), (double)lo[k],
                             (double)hi[k]);
                Xoff[row * d + k] = (float)v;
            }
        }
    }
    return OPS_OK;
}

/* ---------------------------------------------------------------------- */
/* PBI aggregation (Section IV-B): d1 = |(f - z) . w| / ||w||,            */
/* d2 = || (f - z) - d1 w / ||w|| ||, g = d1 + theta d2.                  */
/* ---------------------------------------------------------------------- */
double oracle_pbi(const float* f, const float* w, const float* z, int m, double theta)
{
    double ww = 0.0, fw = 0.0;
    for (int k = 0; k < m; ++k) ww = ww + (double)w[k] * (double)w[k];
    const double nw = sqrt(ww);
    for (int k = 0; k < m; ++k) fw = fw + ((double)f[k] - (double)z[k]) * (double)w[k];
    const double d1 = fabs(fw) / nw;
    double dd = 0.0;
    for (int k = 0; k < m; ++k) {
        const double r = ((double)f[k] - (double)z[k]) - d1 * ((double)w[k] / nw);
        dd = dd + r * r;
    }
    return d1 + theta * sqrt(dd);
}

/* ---------------------------------------------------------------------- */
/* TensorMOEA/D environmental selection, Algorithm S.8.                    */
/*   z_min <- min(z, rows of F2)                                           */
/*   I_new[i][.] = identity with -1 at every neighbour j of offspring i   */
/*                 whose PBI value does not exceed the neighbour's own     */
/*   column j: f_i = F2[i] where I_new[i][j] = -1, else F1[j];             */
/*             winner = first argmin_i PBI(f_i | w_j, z_min)               */
/*   X_next[j], F_next[j] from the winner; z <- z_min.                     */
/* winner_out[j] = the offspring index taken, or -1 when F1[j] stays.      */
/* I_new is materialised (n x n), as in the paper, so n is kept small.     */
/* ---------------------------------------------------------------------- */
int oracle_moead_select(const float* X, const float* F1, const float* O, const float* F2, int64_t n, int64_t d,
                        int m, float* z, const float* W, const int32_t* Inb, int32_t T, double theta, float* Xnext,
                        float* Fnext, int32_t* winner_out)
{
    if (!X || !F1 || !O || !F2 || !z || !W || !Inb || !Xnext || !Fnext || n < 1 || n > (1 << 15) || d < 1 ||
        m < 2 || m > 16 || T < 1 || T > n || !(theta >= 0.0))
        return OPS_EINVAL;
    for (int64_t i = 0; i < n * T; ++i)
        if (Inb[i] < 0 || Inb[i] >= n) return OPS_EINVAL;
    for (int64_t i = 0; i < n * m; ++i)
        if (!isfinite(F1[i]) || !isfinite(F2[i]) || !isfinite(W[i])) return OPS_ENONFINITE;
    for (int k = 0; k < m; ++k)
        if (!isfinite(z[k])) return OPS_ENONFINITE;
    for (int64_t j = 0; j < n; ++j) {
        double ww = 0.0;
        for (int k = 0; k < m; ++k) ww = ww + (double)W[j * m + k] * (double)W[j * m + k];
        if (!(ww > 0.0)) return OPS_ENONFINITE;
    }
    float zmin[16];
    for (int k = 0; k < m; ++k) {
        float v = z[k];
        for (int64_t i = 0; i < n; ++i) if (F2[i * m + k] < v) v = F2[i * m + k];
        zmin[k] = v;
    }
    int32_t* Inew = (int32_t*)malloc((size_t)n * (size_t)n * sizeof(int32_t));
    uint8_t* M = (uint8_t*)malloc((size_t)n);
    if (!Inew || !M) { free(Inew); free(M); return OPS_ENOMEM; }
    /* comparison and population update: one row of I_new per offspring */
    for (int64_t i = 0; i < n; ++i) {
        memset(M, 0, (size_t)n);
        for (int32_t t = 0; t < T; ++t) {
            const int64_t j = Inb[i * T + t];
            const double g_old = oracle_pbi(F1 + j * m, W + j * m, zmin, m, theta);
            const double g_new = oracle_pbi(F2 + i * m, W + j * m, zmin, m, theta);
            M[j] = (g_old - g_new) >= 0.0;     /* H(g_old - g_new), H(0) = 1 */
        }
        for (int64_t j = 0; j < n; ++j) Inew[i * n + j] = M[j] ? -1 : (int32_t)j;
    }
    /* elite selection: one argmin per column of I_new */
    for (int64_t j = 0; j < n; ++j) {
        int64_t best = 0;
        double best_g = INFINITY;
        for (int64_t i = 0; i < n; ++i) {
            const float* f = Inew[i * n + j] == -1 ? F2 + i * m : F1 + j * m;
            const double g = oracle_pbi(f, W + j * m, zmin, m, theta);
            if (g < best_g) { best_g = g; best = i; }
        }
        const int from_offspring = Inew[best * n + j] == -1;
        const float* xs = from_offspring ? O + best * d : X + j * d;
        const float* fs = from_offspring ? F2 + best * m : F1 + j * m;
        memcpy(Xnext + j * d, xs, (size_t)d * sizeof(float));
        memcpy(Fnext + j * m, fs, (size_t)m * sizeof(float));
        if (winner_out) winner_out[j] = from_offspring ? (int32_t)best : -1;
    }
    for (int k = 0; k < m; ++k) z[k] = zmin[k];
    free(Inew);
    free(M);
    return OPS_OK;
}

/* ---------------------------------------------------------------------- */
/* MOEA/D reproduction (Algorithm S.7, "Randomly select two indices p, q  */
/* from B(i)", done for all i at once as in TensorMOEA/D): the first SBX  */
/* child of (x_p, x_q), clipped, then polynomial mutation, clipped.       */
/* ---------------------------------------------------------------------- */
int oracle_moead_offspring(const float* X, int64_t n, int64_t d, const float* lo, const float* hi,
                           const int32_t* Inb, int32_t T, uint64_t seed, uint64_t gen, double eta_c, double eta_m,
                           double p_m, float* O, int32_t* parents_out)
{
    if (!X || !lo || !hi || !Inb || !O || n < 1 || n > INT32_MAX || d < 1 || d > 0x00FFFFFF || T < 1 ||
        !(eta_c >= 0.0) || !(eta_m >= 0.0))
        return OPS_EINVAL;
    for (int64_t i = 0; i < n * T; ++i)
        if (Inb[i] < 0 || Inb[i] >= n) return OPS_EINVAL;
    for (int64_t k = 0; k < d; ++k)
        if (!isfinite(lo[k]) || !isfinite(hi[k]) || !(hi[k] > lo[k])) return OPS_EINVAL;
    for (int64_t i = 0; i < n * d; ++i)
        if (!isfinite(X[i])) return OPS_ENONFINITE;
    for (int64_t i = 0; i < n; ++i) {
        uint32_t r0[4], r1[4];
        gen_random(seed, gen, i, 5, 0, r0);
        gen_random(seed, gen, i, 5, 1, r1);
        const int64_t a = Inb[i * T + index_of(r0[0], T)], b = Inb[i * T + index_of(r1[0], T)];
        if (parents_out) { parents_out[2 * i] = (int32_t)a; parents_out[2 * i + 1] = (int32_t)b; }
        for (int64_t k = 0; k < d; ++k) {
            uint32_t rs[4], rm[4];
            double c1, c2;
            gen_random(seed, gen, i, 2, k, rs);
            oracle_sbx_pair((double)X[a * d + k], (double)X[b * d + k], unit_of(rs[0]), eta_c, &c1, &c2);
            double v = clip(c1, (double)lo[k], (double)hi[k]);
            gen_random(seed, gen, i, 3, k, rm);
            if (hit(rm[0], p_m))
                v = clip(oracle_pm_value(v, (double)lo[k], (double)hi[k], unit_of(rm[1]), eta_m), (double)lo[k],
                         (double)hi[k]);
            O[i * d + k] = (float)v;
        }
    }
    return OPS_OK;
}

/* ---------------------------------------------------------------------- */
/* IGD: (1 / |Ref|) sum_r min_i ||Ref_r - F_i||, FP64, k ascending.        */
/* ---------------------------------------------------------------------- */
double oracle_igd(const float* F, int64_t n, int m, const float* Ref, int64_t nref)
{
    if (!F || !Ref || n < 1 || nref < 1 || m < 1) return NAN;
    double* nearest = (double*)malloc((size_t)nref * sizeof(double));
    if (!nearest) return NAN;
    /* the nearest distance of each reference point (independent; the
       all-core build runs them in parallel), then the sum in index order */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t r = 0; r < nref; ++r) {
        double best = INFINITY;
        for (int64_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int k = 0; k < m; ++k) {
                const double e = (double)Ref[r * m + k] - (double)F[i * m + k];
                s = s + e * e;
            }
            if (s < best) best = s;
        }
        nearest[r] = sqrt(best);
    }
    double total = 0.0;
    for (int64_t r = 0; r < nref; ++r) total = total + nearest[r];
    free(nearest);
    return total / (double)nref;
}
