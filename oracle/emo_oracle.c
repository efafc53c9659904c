/*
 * FP64 CPU oracle for NSGA-III environmental selection (arXiv 2503.20286).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Every routine is a plain, slow, literal statement of the paper's steps:
 *   - Pareto dominance: Section III-C, Listing 1 (all <= and some <).
 *   - Nondominated sorting: Deb's fast sort, Algorithm S.2; the tensorized
 *     front peeling of Algorithm S.3 as a second, independent formulation.
 *   - Environmental selection: Algorithm S.1 (fill fronts, normalise S_t,
 *     associate, niche counts, niche-preserving fill of the last front).
 *   - Normalisation: Algorithm S.5 (ideal point, ASF extreme points,
 *     hyperplane intercepts, nadir fallback when rank(E) < m).
 *   - Association: perpendicular distance to each reference line,
 *     Section IV-A "Association" equation.
 *
 * Readings of silent or ambiguous points (the paper does not fix them):
 *   - c is the number of dominators of each point (column sum of D); the
 *     row sum printed in Section IV-A / Algorithm S.3 would not reproduce
 *     Algorithm S.2.
 *   - l = rank of the N-th best point (0-based ranks, sort(r)[N-1]).
 *   - normalisation runs over S_t = P_{t+1} U F_l (Algorithm S.1), i.e. the
 *     NaN mask of Algorithm S.4 hides r > l only; niche counts count r < l.
 *   - ASF weights: w_jj = 1, w_jk = 1e-6 (k != j).
 *   - Intercepts: Gaussian elimination with partial pivoting on [E | 1],
 *     singular when |pivot| <= 1e-12 * max|E|; fallback to the nadir
 *     a_k = max_{i in S}(F_ik - z_k) when singular, non-finite or <= 1e-10;
 *     after the fallback any a_k <= 1e-10 becomes 1.
 *   - Perpendicular distance in the cancellation-free form
 *     d^2 = sum_k (f_k - t r_k)^2, t = (f.r)/(r.r), equal in exact arithmetic
 *     to ||f|| sqrt(1 - cos^2).
 *   - argmin ties go to the lowest index everywhere.
 *   - Niching is Algorithm S.1 with the ties among least-crowded reference
 *     points broken by a counter-based random stream (Philox-4x32-10 keyed
 *     by the seed, counter (j, 2c + tag, generation)); all references at the
 *     current minimum niche count are served in one level.
 *   - Survivors are returned as ascending indices (Section IV-A, i_next).
 *   - One-shot niching (the tensorized niche selection of Algorithm S.4 and
 *     Update-Rank, Algorithm S.6), selected by mode 1: every reference with
 *     niche count 0 and at least one last-front candidate takes its nearest
 *     candidate (d, then index); with n_dif = K - (number taken), the first
 *     n_dif of the remaining last-front points are added (n_dif > 0) or the
 *     first -n_dif of the taken points are dropped (n_dif < 0). "First" is in
 *     the order of the shuffled input in the paper; here it is the order of
 *     Philox keys (x0 of counter (i, 0xFFFFFFF0 + tag, generation), tag 1 to
 *     add, 2 to drop; ties by index).
 *
 * Compile with -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_NOT_RANKED INT32_MAX

/* The same source builds a single-threaded library and, with -fopenmp, an
   all-core one. Only two loops run in parallel, each over independent
   points with no shared writes: the pairwise dominance relation (one row i
   per iteration) and the association (one point per iteration). Every
   value is computed by the same operations in the same order either way,
   so both builds return identical results. Sets the thread count when
   n > 0 and returns the count in use (1 without OpenMP). */
int oracle_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random     */
/* numbers: as easy as 1, 2, 3"): ten rounds of two 32x32->64 multiplies,   */
/* an S-box of xors with the round key, and a Weyl-sequence key schedule.   */
/* ---------------------------------------------------------------------- */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)mul0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)mul1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += weyl0; k1 += weyl1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* First output word of the niching stream for reference j, level c, tag. */
static uint32_t niche_random(uint64_t seed, uint64_t gen, int64_t j, int64_t c, int tag)
{
    uint32_t ctr[4], key[2], out[4];
    ctr[0] = (uint32_t)j;
    ctr[1] = (uint32_t)(2 * c + tag);
    ctr[2] = (uint32_t)(gen & 0xFFFFFFFFu);
    ctr[3] = (uint32_t)(gen >> 32);
    key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    key[1] = (uint32_t)(seed >> 32);
    oracle_philox4x32_10(ctr, key, out);
    return out[0];
}

/* First output word of the one-shot stream for point i (Algorithm S.6's
   fill / drop order; tag 1 = add, 2 = drop). */
static uint32_t oneshot_random(uint64_t seed, uint64_t gen, int64_t i, int tag)
{
    uint32_t ctr[4], key[2], out[4];
    ctr[0] = (uint32_t)i;
    ctr[1] = 0xFFFFFFF0u + (uint32_t)tag;
    ctr[2] = (uint32_t)(gen & 0xFFFFFFFFu);
    ctr[3] = (uint32_t)(gen >> 32);
    key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    key[1] = (uint32_t)(seed >> 32);
    oracle_philox4x32_10(ctr, key, out);
    return out[0];
}

/* ---------------------------------------------------------------------- */
/* Pareto dominance, Listing 1: a dominates b iff every a_k <= b_k and at  */
/* least one a_k < b_k (minimisation).                                     */
/* ---------------------------------------------------------------------- */
int oracle_dominates(const double* a, const double* b, int m)
{
    int all_le = 1, any_lt = 0;
    for (int k = 0; k < m; ++k) {
        if (!(a[k] <= b[k])) all_le = 0;
        if (a[k] < b[k]) any_lt = 1;
    }
    return all_le && any_lt;
}

static int dominates_rows(const float* F, int m, int64_t i, int64_t j)
{
    double a[64], b[64];
    for (int k = 0; k < m; ++k) {
        a[k] = (double)F[i * m + k];
        b[k] = (double)F[j * m + k];
    }
    return oracle_dominates(a, b, m);
}

/* Bit-packed dominance matrix: row i, word w, bit b <=> D[i][32w + b]. */
void oracle_dominance_bits(const float* F, int64_t n, int m, uint32_t* D, int64_t ld)
{
    memset(D, 0, (size_t)n * (size_t)ld * sizeof(uint32_t));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            if (i != j && dominates_rows(F, m, i, j))
                D[i * ld + (j >> 5)] |= 1u << (j & 31);
}

/* Dominators count of each point: c_j = sum_i D_ij. */
void oracle_domination_counts(const float* F, int64_t n, int m, int32_t* c)
{
    for (int64_t j = 0; j < n; ++j) {
        int32_t s = 0;
        for (int64_t i = 0; i < n; ++i)
            if (i != j && dominates_rows(F, m, i, j)) ++s;
        c[j] = s;
    }
}

/* ---------------------------------------------------------------------- */
/* Deb's fast nondominated sort, Algorithm S.2. S_i (points dominated by   */
/* i) is kept as a bitset row; n_i counts the dominators of i. Ranks are   */
/* 0-based front indices. Returns the number of fronts, or -1 on OOM.      */
/* ---------------------------------------------------------------------- */
int64_t oracle_nd_sort_deb(const float* F, int64_t n, int m, int32_t* rank)
{
    int64_t words = (n + 63) / 64;
    uint64_t* S = (uint64_t*)calloc((size_t)(n * words), sizeof(uint64_t));
    int64_t* cnt = (int64_t*)calloc((size_t)n, sizeof(int64_t));
    int64_t* cur = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    int64_t* nxt = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    if (!S || !cnt || !cur || !nxt) { free(S); free(cnt); free(cur); free(nxt); return -1; }

    /* Row i compares point i with every other point j; both relations
       follow from the per-objective < and > flags (same definition as
       Listing 1): i dominates j puts j into S_i, j dominates i counts one
       dominator of i. Each iteration writes only row i of S and n_i. */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < n; ++i) {
        int64_t ni = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            int lt = 0, gt = 0;
            for (int k = 0; k < m; ++k) {
                double a = (double)F[i * m + k], b = (double)F[j * m + k];
                if (a < b) lt = 1;
                else if (a > b) gt = 1;
            }
            if (lt && !gt) S[i * words + (j >> 6)] |= 1ull << (j & 63);   /* i dominates j */
            else if (gt && !lt) ni += 1;                                  /* j dominates i */
        }
        cnt[i] = ni;
    }
    int64_t ncur = 0;
    for (int64_t i = 0; i < n; ++i) {
        rank[i] = ORACLE_NOT_RANKED;
        if (cnt[i] == 0) { cur[ncur++] = i; rank[i] = 0; }
    }
    int64_t k = 0;
    while (ncur > 0) {
        int64_t nn = 0;
        for (int64_t a = 0; a < ncur; ++a) {
            int64_t i = cur[a];
            for (int64_t w = 0; w < words; ++w) {
                uint64_t bits = S[i * words + w];
                while (bits) {
                    int b = __builtin_ctzll(bits);
                    bits &= bits - 1;
                    int64_t j = w * 64 + b;
                    if (--cnt[j] == 0) { nxt[nn++] = j; rank[j] = (int32_t)(k + 1); }
                }
            }
        }
        int64_t* t = cur; cur = nxt; nxt = t;
        ncur = nn;
        ++k;
    }
    free(S); free(cnt); free(cur); free(nxt);
    return k;
}

/* ---------------------------------------------------------------------- */
/* Tensorized front peeling, Algorithm S.3, with c = column sums of D:     */
/* p = 1[c = 0]; loop { r[p] = k; d_j = sum_i p_i D_ij; c -= d + p; k++ }. */
/* ---------------------------------------------------------------------- */
int64_t oracle_nd_sort_peel(const float* F, int64_t n, int m, int32_t* rank)
{
    int64_t words = (n + 31) / 32;
    uint32_t* D = (uint32_t*)malloc((size_t)(n * words) * sizeof(uint32_t));
    int64_t* c = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    int64_t* d = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    uint8_t* p = (uint8_t*)malloc((size_t)n);
    if (!D || !c || !d || !p) { free(D); free(c); free(d); free(p); return -1; }
    oracle_dominance_bits(F, n, m, D, words);
    for (int64_t j = 0; j < n; ++j) {
        int64_t s = 0;
        for (int64_t i = 0; i < n; ++i) s += (D[i * words + (j >> 5)] >> (j & 31)) & 1u;
        c[j] = s;
        rank[j] = ORACLE_NOT_RANKED;
    }
    int64_t any = 0;
    for (int64_t j = 0; j < n; ++j) { p[j] = (c[j] == 0); any |= p[j]; }
    int64_t k = 0;
    while (any) {
        for (int64_t j = 0; j < n; ++j) if (p[j]) rank[j] = (int32_t)k;
        for (int64_t j = 0; j < n; ++j) {
            int64_t s = 0;
            for (int64_t i = 0; i < n; ++i)
                if (p[i]) s += (D[i * words + (j >> 5)] >> (j & 31)) & 1u;
            d[j] = s;
        }
        /* c <- c - d - p: points of the current front drop to -1 and never
           re-enter; others reach 0 once all their dominators are ranked. */
        for (int64_t j = 0; j < n; ++j) c[j] = c[j] - d[j] - p[j];
        ++k;
        any = 0;
        for (int64_t j = 0; j < n; ++j) { p[j] = (c[j] == 0); any |= p[j]; }
    }
    free(D); free(c); free(d); free(p);
    return k;
}

/* ---------------------------------------------------------------------- */
/* Environmental selection, Algorithm S.1 with Algorithm S.5.              */
/* ---------------------------------------------------------------------- */
typedef struct {
    int32_t* rank;     /* [n2] 0-based front index (all fronts)            */
    double* z;         /* [m] ideal point over S                           */
    int32_t* extreme;  /* [m] ASF extreme point indices                    */
    double* a;         /* [m] intercepts (after fallback)                  */
    double* fnorm;     /* [n2*m] normalised objectives, NaN outside S      */
    int32_t* pi;       /* [n2] associated reference, -1 outside S          */
    double* dist;      /* [n2] perpendicular distance, NaN outside S       */
    int32_t* rho;      /* [n_r] niche counts of P = {r < l}                */
    uint8_t* picked;   /* [n2] 1 when chosen by niching                    */
    int32_t last_rank, n_before, n_last, fallback, n_levels, near_ties;
} oracle_trace;

enum { ORACLE_OK = 0, ORACLE_EINVAL = 1, ORACLE_ENONFINITE = 2, ORACLE_ENOMEM = 3 };

static int cmp_u64(const void* x, const void* y)
{
    uint64_t a = *(const uint64_t*)x, b = *(const uint64_t*)y;
    return (a > b) - (a < b);
}

static int cmp_i32(const void* x, const void* y)
{
    int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
    return (a > b) - (a < b);
}

/* Gaussian elimination with partial pivoting on [E | 1]; b = E^{-1} 1.
   Returns 1 when singular (|pivot| <= 1e-12 max|E|). */
static int solve_hyperplane(int m, const double* E_in, double* b)
{
    double A[16][16], rhs[16];
    double maxabs = 0.0;
    for (int r = 0; r < m; ++r) {
        rhs[r] = 1.0;
        for (int c = 0; c < m; ++c) {
            A[r][c] = E_in[r * m + c];
            double v = fabs(A[r][c]);
            if (v > maxabs) maxabs = v;
        }
    }
    for (int col = 0; col < m; ++col) {
        int piv = col;
        for (int r = col + 1; r < m; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (!(fabs(A[piv][col]) > 1e-12 * maxabs)) return 1;
        if (piv != col) {
            for (int c = 0; c < m; ++c) { double t = A[col][c]; A[col][c] = A[piv][c]; A[piv][c] = t; }
            double t = rhs[col]; rhs[col] = rhs[piv]; rhs[piv] = t;
        }
        for (int r = col + 1; r < m; ++r) {
            double f = A[r][col] / A[col][col];
            for (int c = col; c < m; ++c) A[r][c] = A[r][c] - f * A[col][c];
            rhs[r] = rhs[r] - f * rhs[col];
        }
    }
    for (int col = m - 1; col >= 0; --col) {
        double s = rhs[col];
        for (int c = col + 1; c < m; ++c) s = s - A[col][c] * b[c];
        b[col] = s / A[col][col];
    }
    return 0;
}

/* mode 0: niching of Algorithm S.1 (level form); mode 1: one-shot niche
   selection of Algorithm S.4 with Update-Rank (Algorithm S.6). */
int oracle_nsga3_select_mode(const float* F, int64_t n2, int m, const float* R, int32_t n_r,
                             int64_t n_keep, uint64_t seed, uint64_t gen, int mode,
                             int32_t* survivors, oracle_trace* tr)
{
    if (mode != 0 && mode != 1) return ORACLE_EINVAL;
    if (!F || !R || !survivors || m < 2 || m > 16 || n_r < 1 || n2 < 1 || n_keep < 1 || n_keep > n2)
        return ORACLE_EINVAL;
    for (int64_t i = 0; i < n2 * m; ++i) if (!isfinite(F[i])) return ORACLE_ENONFINITE;
    for (int64_t i = 0; i < (int64_t)n_r * m; ++i) if (!isfinite(R[i])) return ORACLE_ENONFINITE;

    int status = ORACLE_ENOMEM;
    int32_t* rank = (int32_t*)malloc((size_t)n2 * sizeof(int32_t));
    int32_t* sorted = (int32_t*)malloc((size_t)n2 * sizeof(int32_t));
    uint8_t* inS = (uint8_t*)calloc((size_t)n2, 1);
    double* fn = (double*)malloc((size_t)(n2 * m) * sizeof(double));
    int32_t* pi = (int32_t*)malloc((size_t)n2 * sizeof(int32_t));
    double* dist = (double*)malloc((size_t)n2 * sizeof(double));
    int64_t* rho = (int64_t*)calloc((size_t)n_r, sizeof(int64_t));
    int64_t* cnt = (int64_t*)calloc((size_t)n_r, sizeof(int64_t));
    int64_t* off = (int64_t*)calloc((size_t)n_r + 1, sizeof(int64_t));
    int64_t* lst = NULL;
    uint8_t* picked = (uint8_t*)calloc((size_t)n2, 1);
    uint8_t* alive = (uint8_t*)calloc((size_t)n_r, 1);
    int64_t* E = (int64_t*)malloc((size_t)n_r * sizeof(int64_t));
    uint64_t* keyed = (uint64_t*)malloc((size_t)n_r * sizeof(uint64_t));
    if (!keyed || !rank || !sorted || !inS || !fn || !pi || !dist || !rho || !cnt || !off || !picked || !alive || !E)
        goto done;
    for (int32_t j = 0; j < n_r; ++j) {
        double rr = 0.0;
        for (int k = 0; k < m; ++k) rr = rr + (double)R[(int64_t)j * m + k] * (double)R[(int64_t)j * m + k];
        if (!(rr > 0.0)) { status = ORACLE_EINVAL; goto done; }
    }

    /* 1-2. Nondominated sorting (Algorithm S.2). */
    if (oracle_nd_sort_deb(F, n2, m, rank) < 0) goto done;

    /* 3. l = rank of the n-th best point; P = {r < l}, L = {r = l}. */
    memcpy(sorted, rank, (size_t)n2 * sizeof(int32_t));
    qsort(sorted, (size_t)n2, sizeof(int32_t), cmp_i32);
    int32_t l = sorted[n_keep - 1];
    int64_t nP = 0, nL = 0;
    for (int64_t i = 0; i < n2; ++i) {
        if (rank[i] < l) ++nP;
        else if (rank[i] == l) ++nL;
        inS[i] = rank[i] <= l;
    }
    int64_t K = n_keep - nP;

    /* 4. Ideal point over S_t (Algorithm S.5, first line). */
    double z[16];
    for (int k = 0; k < m; ++k) {
        double mn = INFINITY;
        for (int64_t i = 0; i < n2; ++i)
            if (inS[i] && (double)F[i * m + k] < mn) mn = (double)F[i * m + k];
        z[k] = mn;
    }

    /* 5. Extreme points: e_j = argmin_i max_k (F_ik - z_k) / w_jk. */
    int32_t ext[16];
    for (int j = 0; j < m; ++j) {
        double best = INFINITY;
        int64_t bi = -1;
        for (int64_t i = 0; i < n2; ++i) {
            if (!inS[i]) continue;
            double asf = -INFINITY;
            for (int k = 0; k < m; ++k) {
                double w = (k == j) ? 1.0 : 1e-6;
                double t = ((double)F[i * m + k] - z[k]) / w;
                if (t > asf) asf = t;
            }
            if (asf < best) { best = asf; bi = i; }
        }
        ext[j] = (int32_t)bi;
    }

    /* 6. Hyperplane intercepts, with the nadir fallback. */
    double Em[256], bvec[16], a[16];
    for (int j = 0; j < m; ++j)
        for (int k = 0; k < m; ++k)
            Em[j * m + k] = (double)F[(int64_t)ext[j] * m + k] - z[k];
    int fallback = solve_hyperplane(m, Em, bvec);
    if (!fallback) {
        for (int k = 0; k < m; ++k) {
            a[k] = 1.0 / bvec[k];
            if (!isfinite(a[k]) || a[k] <= 1e-10) fallback = 1;
        }
    }
    if (fallback) {
        for (int k = 0; k < m; ++k) {
            double mx = -INFINITY;
            for (int64_t i = 0; i < n2; ++i)
                if (inS[i] && (double)F[i * m + k] - z[k] > mx) mx = (double)F[i * m + k] - z[k];
            a[k] = mx;
        }
        for (int k = 0; k < m; ++k) if (a[k] <= 1e-10) a[k] = 1.0;
    }

    /* 7-8. Normalise S and associate each point with the nearest line
       (points are independent: each iteration writes only its own row). */
    int32_t near_ties = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : near_ties)
#endif
    for (int64_t i = 0; i < n2; ++i) {
        pi[i] = -1;
        dist[i] = NAN;
        for (int k = 0; k < m; ++k) fn[i * m + k] = NAN;
        if (!inS[i]) continue;
        for (int k = 0; k < m; ++k) fn[i * m + k] = ((double)F[i * m + k] - z[k]) / a[k];
        double b1 = INFINITY, b2 = INFINITY;
        int32_t j1 = -1;
        for (int32_t j = 0; j < n_r; ++j) {
            const float* r = R + (int64_t)j * m;
            double rr = 0.0, fr = 0.0;
            for (int k = 0; k < m; ++k) rr = rr + (double)r[k] * (double)r[k];
            for (int k = 0; k < m; ++k) fr = fr + fn[i * m + k] * (double)r[k];
            double t = fr / rr;
            double d2 = 0.0;
            for (int k = 0; k < m; ++k) {
                double e = fn[i * m + k] - t * (double)r[k];
                d2 = d2 + e * e;
            }
            if (d2 < b1) { b2 = b1; b1 = d2; j1 = j; }
            else if (d2 < b2) b2 = d2;
        }
        pi[i] = j1;
        dist[i] = sqrt(b1);
        if (n_r > 1) {
            double s1 = sqrt(b1), s2 = sqrt(b2);
            if (s2 - s1 < 1e-6 * s2 || s2 == 0.0) ++near_ties;
        }
    }

    /* 9. Niche counts of P and candidate lists C_j of the last front. */
    for (int64_t i = 0; i < n2; ++i) {
        if (rank[i] < l) rho[pi[i]] += 1;
        else if (rank[i] == l) cnt[pi[i]] += 1;
    }
    for (int32_t j = 0; j < n_r; ++j) off[j + 1] = off[j] + cnt[j];
    lst = (int64_t*)malloc((size_t)(nL > 0 ? nL : 1) * sizeof(int64_t));
    if (!lst) goto done;
    memset(cnt, 0, (size_t)n_r * sizeof(int64_t));
    for (int64_t i = 0; i < n2; ++i)          /* ascending i: lists sorted */
        if (rank[i] == l) { int32_t j = pi[i]; lst[off[j] + cnt[j]] = i; cnt[j] += 1; }
    if (tr && tr->rho) for (int32_t j = 0; j < n_r; ++j) tr->rho[j] = (int32_t)rho[j];

    /* 10. Niching: serve every least-crowded live reference once per level. */
    for (int32_t j = 0; j < n_r; ++j) alive[j] = cnt[j] > 0;
    int64_t remaining = mode == 0 ? K : 0;
    int32_t levels = 0;
    if (mode == 1) {
        /* 10'. One-shot niche selection (Algorithm S.4): each reference with
           rho_j = 0 and rho_{l,j} > 0 takes the last-front point of smallest
           distance d associated with it (D' argmin; ties: lowest index). */
        int64_t n_sel = 0;
        for (int32_t j = 0; j < n_r; ++j) {
            if (rho[j] != 0 || cnt[j] == 0) continue;
            const int64_t* Cj = lst + off[j];
            int64_t best = Cj[0];
            for (int64_t q = 1; q < cnt[j]; ++q)
                if (dist[Cj[q]] < dist[best] || (dist[Cj[q]] == dist[best] && Cj[q] < best)) best = Cj[q];
            picked[best] = 1;
            ++n_sel;
        }
        /* Update-Rank (Algorithm S.6): n_dif = n - n_s, n_s = |P| + n_sel. */
        int64_t n_dif = K - n_sel;
        int64_t nk = 0;
        uint64_t* ord = (uint64_t*)malloc((size_t)(nL > 0 ? nL : 1) * sizeof(uint64_t));
        if (!ord) goto done;
        if (n_dif > 0) {            /* add the first n_dif remaining last-front points */
            for (int64_t i = 0; i < n2; ++i)
                if (rank[i] == l && !picked[i])
                    ord[nk++] = ((uint64_t)oneshot_random(seed, gen, i, 1) << 32) | (uint64_t)i;
            qsort(ord, (size_t)nk, sizeof(uint64_t), cmp_u64);
            for (int64_t e = 0; e < n_dif; ++e) picked[ord[e] & 0xFFFFFFFFu] = 1;
        } else if (n_dif < 0) {     /* drop the first -n_dif taken points */
            for (int64_t i = 0; i < n2; ++i)
                if (picked[i]) ord[nk++] = ((uint64_t)oneshot_random(seed, gen, i, 2) << 32) | (uint64_t)i;
            qsort(ord, (size_t)nk, sizeof(uint64_t), cmp_u64);
            for (int64_t e = 0; e < -n_dif; ++e) picked[ord[e] & 0xFFFFFFFFu] = 0;
        }
        free(ord);
        levels = 1;
    }
    while (remaining > 0) {
        int64_t c = INT64_MAX;
        for (int32_t j = 0; j < n_r; ++j) if (alive[j] && rho[j] < c) c = rho[j];
        int64_t nE = 0;
        for (int32_t j = 0; j < n_r; ++j) if (alive[j] && rho[j] == c) E[nE++] = j;
        if (nE > remaining) {
            /* keep the `remaining` references with the smallest (x0, j) */
            for (int64_t e = 0; e < nE; ++e)
                keyed[e] = ((uint64_t)niche_random(seed, gen, E[e], c, 0) << 32) | (uint64_t)E[e];
            qsort(keyed, (size_t)nE, sizeof(uint64_t), cmp_u64);
            for (int64_t e = 0; e < remaining; ++e) E[e] = (int64_t)(keyed[e] & 0xFFFFFFFFu);
            nE = remaining;
        }
        for (int64_t e = 0; e < nE; ++e) {
            int64_t j = E[e];
            int64_t len = cnt[j];
            int64_t* Cj = lst + off[j];
            int64_t pos;
            if (c == 0) {                       /* nearest member (S.1) */
                pos = 0;
                for (int64_t q = 1; q < len; ++q) {
                    double dq = dist[Cj[q]], dp = dist[Cj[pos]];
                    if (dq < dp || (dq == dp && Cj[q] < Cj[pos])) pos = q;
                }
            } else {                            /* random member (S.1) */
                uint32_t u = niche_random(seed, gen, j, c, 1);
                pos = (int64_t)(((uint64_t)u * (uint64_t)len) >> 32);
            }
            picked[Cj[pos]] = 1;
            for (int64_t q = pos; q + 1 < len; ++q) Cj[q] = Cj[q + 1];
            cnt[j] = len - 1;
            rho[j] += 1;
            alive[j] = cnt[j] > 0;
        }
        remaining -= nE;
        ++levels;
    }

    /* 11. Survivors: ascending indices of P U picked. */
    int64_t ns = 0;
    for (int64_t i = 0; i < n2; ++i)
        if (rank[i] < l || picked[i]) survivors[ns++] = (int32_t)i;

    if (tr) {
        if (tr->rank) memcpy(tr->rank, rank, (size_t)n2 * sizeof(int32_t));
        if (tr->z) for (int k = 0; k < m; ++k) tr->z[k] = z[k];
        if (tr->extreme) for (int k = 0; k < m; ++k) tr->extreme[k] = ext[k];
        if (tr->a) for (int k = 0; k < m; ++k) tr->a[k] = a[k];
        if (tr->fnorm) memcpy(tr->fnorm, fn, (size_t)(n2 * m) * sizeof(double));
        if (tr->pi) memcpy(tr->pi, pi, (size_t)n2 * sizeof(int32_t));
        if (tr->dist) memcpy(tr->dist, dist, (size_t)n2 * sizeof(double));
        if (tr->picked) memcpy(tr->picked, picked, (size_t)n2);
        tr->last_rank = l;
        tr->n_before = (int32_t)nP;
        tr->n_last = (int32_t)nL;
        tr->fallback = fallback;
        tr->n_levels = levels;
        tr->near_ties = near_ties;
    }
    status = (ns == n_keep) ? ORACLE_OK : ORACLE_EINVAL;

done:
    free(rank); free(sorted); free(inS); free(fn); free(pi); free(dist); free(rho);
    free(cnt); free(off); free(lst); free(picked); free(alive); free(E); free(keyed);
    return status;
}

int oracle_nsga3_select(const float* F, int64_t n2, int m, const float* R, int32_t n_r,
                        int64_t n_keep, uint64_t seed, uint64_t gen,
                        int32_t* survivors, oracle_trace* tr)
{
    return oracle_nsga3_select_mode(F, n2, m, R, n_r, n_keep, seed, gen, 0, survivors, tr);
}

/* ---------------------------------------------------------------------- */
/* TensorHypE environmental selection (Algorithm S.10) with the Monte      */
/* Carlo hypervolume estimation of Algorithm S.11.                          */
/*   - r, l: Algorithm S.2 ranks, l = rank of the n-th best point;          */
/*     the mask H(l - r) keeps S = {r <= l}, k = |S| - n points to drop.     */
/*   - lambda_1 = 1, lambda_i = (k - (i - 1)) / (n1 - (i - 1)) (i >= 2),     */
/*     alpha_c = (lambda_1 ... lambda_c) / c, n1 = 2N (all points); the     */
/*     product reaches 0 at c = k + 1, so alpha_c = 0 beyond k.             */
/*   - samples S_i = f_l + U_i (v_ref - f_l) with f_l = min_i F_i, in float */
/*     (one subtraction, one multiply, one add, no fused multiply-add);     */
/*     U (uniform [0,1) numbers) is an input.                               */
/*   - t_pds(p, i) = 1 iff F_p <= S_i in every objective; c_i = sum_p.      */
/*   - v_hv(p) = (sum of alpha_{c_i} over the samples i that p dominates,   */
/*     i ascending) * vol / s; vol = prod_j (v_ref_j - f_l_j) in double.     */
/*     Only the points of front l are ordered by it, so it is reported for  */
/*     them and 0 elsewhere; with k = 0 nothing is dropped and it is 0.     */
/*   - I = lexsort(r, -d)[:n]: every point with r < l, then the points of   */
/*     front l by d descending (ties: lower index); output ascending.       */
/* ---------------------------------------------------------------------- */
int oracle_hype_select(const float* F, int64_t n2, int m, const float* vref, const float* U, int32_t s,
                       int64_t n_keep, int32_t* survivors, double* vhv_out, int32_t* last_rank_out)
{
    if (!F || !vref || !U || !survivors || m < 2 || m > 16 || n2 < 1 || s < 1 || n_keep < 1 || n_keep > n2)
        return ORACLE_EINVAL;
    for (int64_t i = 0; i < n2 * m; ++i) if (!isfinite(F[i])) return ORACLE_ENONFINITE;
    int status = ORACLE_ENOMEM;
    int32_t* rank = (int32_t*)malloc((size_t)n2 * sizeof(int32_t));
    int32_t* sorted = (int32_t*)malloc((size_t)n2 * sizeof(int32_t));
    double* alpha = (double*)malloc((size_t)(n2 + 1) * sizeof(double));
    float* S = (float*)malloc((size_t)s * (size_t)m * sizeof(float));
    int64_t* c = (int64_t*)calloc((size_t)s, sizeof(int64_t));
    double* vhv = (double*)malloc((size_t)n2 * sizeof(double));
    int64_t* order = (int64_t*)malloc((size_t)n2 * sizeof(int64_t));
    if (!rank || !sorted || !alpha || !S || !c || !vhv || !order) goto done_h;

    if (oracle_nd_sort_deb(F, n2, m, rank) < 0) goto done_h;
    memcpy(sorted, rank, (size_t)n2 * sizeof(int32_t));
    qsort(sorted, (size_t)n2, sizeof(int32_t), cmp_i32);
    int32_t l = sorted[n_keep - 1];
    int64_t nS = 0, nP = 0;
    for (int64_t i = 0; i < n2; ++i) { nS += rank[i] <= l; nP += rank[i] < l; }
    int64_t k = nS - n_keep;

    /* alpha_c, c = 1 .. n1 (alpha[0] unused) */
    {
        double prod = 1.0;                         /* lambda_1 = 1 */
        alpha[0] = 0.0;
        for (int64_t cc = 1; cc <= n2; ++cc) {
            if (cc >= 2) prod = prod * ((double)(k - (cc - 1)) / (double)(n2 - (cc - 1)));
            alpha[cc] = prod / (double)cc;
        }
    }
    /* samples in [f_l, v_ref] */
    float fl[16];
    for (int j = 0; j < m; ++j) {
        float mn = INFINITY;
        for (int64_t i = 0; i < n2; ++i) if (F[i * m + j] < mn) mn = F[i * m + j];
        fl[j] = mn;
    }
    for (int32_t i = 0; i < s; ++i)
        for (int j = 0; j < m; ++j) {
            volatile float width = vref[j] - fl[j];
            volatile float step = U[(int64_t)i * m + j] * width;
            S[(int64_t)i * m + j] = fl[j] + step;
        }
    /* c_i: points weakly dominating sample i */
    for (int32_t i = 0; i < s; ++i)
        for (int64_t p = 0; p < n2; ++p) {
            int dom = 1;
            for (int j = 0; j < m; ++j) if (!(F[p * m + j] <= S[(int64_t)i * m + j])) { dom = 0; break; }
            c[i] += dom;
        }
    double vol = 1.0;
    for (int j = 0; j < m; ++j) vol = vol * ((double)vref[j] - (double)fl[j]);
    /* v_hv(p): the weights of the samples p dominates, in sample order */
    for (int64_t p = 0; p < n2; ++p) {
        double v = 0.0;
        if (rank[p] != l || k == 0) { vhv[p] = 0.0; continue; }
        for (int32_t i = 0; i < s; ++i) {
            int dom = 1;
            for (int j = 0; j < m; ++j) if (!(F[p * m + j] <= S[(int64_t)i * m + j])) { dom = 0; break; }
            if (dom) v = v + alpha[c[i]];
        }
        vhv[p] = v * vol / (double)s;
    }
    /* I = lexsort(r, -d)[:n]: P, then front l by (d descending, index) */
    int64_t nl = 0;
    for (int64_t i = 0; i < n2; ++i) if (rank[i] == l) order[nl++] = i;
    for (int64_t a = 1; a < nl; ++a) {           /* insertion sort, stable */
        int64_t x = order[a], b = a;
        while (b > 0) {
            int64_t y = order[b - 1];
            if (vhv[x] > vhv[y] || (vhv[x] == vhv[y] && x < y)) { order[b] = y; --b; } else break;
        }
        order[b] = x;
    }
    {
        uint8_t* keep = (uint8_t*)calloc((size_t)n2, 1);
        if (!keep) goto done_h;
        for (int64_t i = 0; i < n2; ++i) keep[i] = rank[i] < l;
        for (int64_t e = 0; e < n_keep - nP; ++e) keep[order[e]] = 1;
        int64_t ns = 0;
        for (int64_t i = 0; i < n2; ++i) if (keep[i]) survivors[ns++] = (int32_t)i;
        free(keep);
        status = ns == n_keep ? ORACLE_OK : ORACLE_EINVAL;
    }
    if (vhv_out) memcpy(vhv_out, vhv, (size_t)n2 * sizeof(double));
    if (last_rank_out) *last_rank_out = l;

done_h:
    free(rank); free(sorted); free(alpha); free(S); free(c); free(vhv); free(order);
    return status;
}
