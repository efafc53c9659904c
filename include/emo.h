/*
 * emo.h -- C ABI of the GB300 (sm_103a) NSGA-III environmental-selection
 * library (arXiv 2503.20286, "Bridging Evolutionary Multiobjective
 * Optimization and GPU Acceleration via Tensorization").
 *
 * Conventions shared by every entry point:
 *  - Every array argument is a DEVICE pointer owned by the caller. The
 *    library never allocates device memory; the multi-stage calls take a
 *    caller-allocated workspace whose size the *_workspace_size queries give.
 *    Workspaces must be 256-byte aligned (cudaMalloc / torch allocations are).
 *  - Objectives are row-major float32: F[i * m + k], i < n2, k < m.
 *    Reference directions are row-major float32: R[j * m + k], j < n_r.
 *    Objectives are minimised.
 *  - Calls are asynchronous and ordered on `stream` (a cudaStream_t; NULL
 *    is the legacy default stream). Argument errors are returned
 *    immediately and nothing is launched. Errors found on the device
 *    (non-finite objectives, a bounded wait that ran out) are written to
 *    `info->status` when `info` is given, and always to the workspace
 *    status word read by emo_workspace_status().
 *  - Several calls may run concurrently on different streams as long as each
 *    has its own workspace and outputs.
 *  - The library sets up each device once per process (launch attributes,
 *    occupancy, the address of the built-in scratch of
 *    emo_nsga3_select_noalloc). After cudaDeviceReset on a device, do not
 *    call the library on that device again in the same process.
 */
#ifndef EMO_H
#define EMO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* emo_stream_t; /* a cudaStream_t */

typedef enum {
    EMO_OK = 0,
    EMO_ERR_INVALID_ARG = 1,     /* bad size, null pointer, misaligned buffer */
    EMO_ERR_NONFINITE = 2,       /* NaN/Inf in F or R, or a zero reference    */
    EMO_ERR_WORKSPACE = 3,       /* workspace smaller than required           */
    EMO_ERR_CUDA = 4,            /* a CUDA runtime call failed                */
    EMO_ERR_TIMEOUT = 5,         /* a bounded device wait ran out             */
    EMO_ERR_NOT_IMPLEMENTED = 6
} emo_status;

/* Upper limits accepted by every entry point. */
#define EMO_MAX_OBJECTIVES 16
#define EMO_MAX_BATCH 128
#define EMO_NOT_RANKED 2147483647 /* rank of points beyond the last needed front */

/* Per-call facts written on the device (all fields int32). */
typedef struct {
    int32_t status;        /* emo_status detected on the device            */
    int32_t last_rank;     /* l: rank of the n_keep-th best point           */
    int32_t n_before;      /* |P| = #{rank < l}                             */
    int32_t n_last;        /* |L| = #{rank == l}                            */
    int32_t fallback_used; /* 1: nadir point replaced the intercepts        */
    int32_t n_recheck;     /* points associated by an all-reference FP64 scan */
    int32_t n_fronts;      /* fronts peeled (l + 1 for selection)           */
    int32_t n_levels;      /* niching levels run (0: all of front l kept)   */
} emo_select_info;

/* Optional intermediate outputs of emo_nsga3_select_debug (device pointers,
 * each nullable). Index order is the caller's point order. */
typedef struct {
    int32_t* rank;    /* [n2] front index, EMO_NOT_RANKED beyond l          */
    float* z;         /* [m] ideal point over S = {rank <= l}               */
    int32_t* extreme; /* [m] index of the ASF extreme point of each axis    */
    double* a;        /* [m] hyperplane intercepts (after any fallback)     */
    float* fnorm;     /* [n2*m] normalised objectives, NaN outside S        */
    int32_t* pi;      /* [n2] associated reference, -1 outside S            */
    double* dist;     /* [n2] perpendicular distance, NaN outside S         */
    int32_t* rho;     /* [n_r] niche counts of P = {rank < l}               */
    uint8_t* picked;  /* [n2] 1 when chosen by niching                      */
} emo_select_debug;

/* One population of a batched call. */
typedef struct {
    const float* F;        /* [n2*m] objectives                              */
    const float* R;        /* [n_r*m] reference directions                   */
    int32_t* survivors;    /* [n_keep] output, ascending point indices       */
    emo_select_info* info; /* nullable                                       */
    int64_t n2;
    int64_t n_keep;
    int32_t m;
    int32_t n_r;
    uint64_t seed;
    uint64_t generation;
    int32_t niche_mode;    /* EMO_NICHE_EXACT (0) or EMO_NICHE_ONESHOT; zero-initialise */
    int32_t reserved;      /* 0 */
} emo_problem;

typedef enum {
    EMO_OP_DOMINANCE = 0,
    EMO_OP_ND_RANK = 1,
    EMO_OP_NSGA3_SELECT = 2,
    EMO_OP_HYPE_SELECT = 3,
    EMO_OP_MOEAD_SELECT = 4, /* emo_workspace_size(EMO_OP_MOEAD_SELECT, n, m, T) */
    EMO_OP_IGD = 5,          /* emo_workspace_size(EMO_OP_IGD, n_ref, m, 0) */
    EMO_OP_SELECT_RANKED = 6, /* emo_nsga3_select_ranked (no dominance matrix) */
    EMO_OP_DOMINANCE_WS = 7   /* emo_dominance_ws (0 for m > 5: no workspace needed) */
} emo_op;

/* Front shapes of the stand-in objective functions (emo_standin_objectives). */
#define EMO_SHAPE_LINEAR 0
#define EMO_SHAPE_SPHERE 1

/* Bytes of workspace needed by `op` for a population of n2 points with m
 * objectives and n_r reference directions (n_r ignored for ranking). Returns
 * 0 when the sizes are out of range. EMO_OP_DOMINANCE needs none. */
size_t emo_workspace_size(int op, int64_t n2, int32_t m, int32_t n_r);

/*
 * Pareto-dominance matrix (Section III-C, Listing 1; Section IV-A "D_ij =
 * F_i dominates F_j"; Algorithm S.3 first line) and the number of dominators
 * of each point (Algorithm S.3 second line, read as the column sum).
 *   F         [n2*m] objectives, 1 <= n2 <= 2^21, 2 <= m <= 16.
 *   D         [n2*ld_words] uint32 output. Row i, word w, bit b is 1 iff
 *             F_i dominates F_{32w+b} (all <= and some <). Bits of columns
 *             >= n2 are zero. ld_words >= ceil(n2/32).
 *   dom_count [n2] int32 output, nullable: dom_count[j] = sum_i D[i][j].
 * Comparisons are exact in float32; -0 equals +0.
 */
emo_status emo_dominance(const float* F, int64_t n2, int32_t m, uint32_t* D, int64_t ld_words,
                         int32_t* dom_count, emo_stream_t stream);

/*
 * The same matrix and counts as emo_dominance, computed through sorted
 * per-objective prefix sets of 1024-column blocks of the caller's order
 * instead of pair-by-pair compares: q is dominated by p iff it lies in every
 * objective's prefix {q : f_k(q) >= f_k(p)} and is not identical to p
 * (identical points are the runs of a lexicographic sort). For m <= 5; for
 * larger m it runs the direct kernel of emo_dominance (ws unused). ws:
 * emo_workspace_size(EMO_OP_DOMINANCE_WS, n2, m, 0) bytes, 256-byte aligned
 * (about 0.2 x n2 x m KB: the prefix sets). Non-finite objectives give
 * EMO_ERR_NONFINITE in the workspace status word (the matrix is then
 * undefined).
 */
emo_status emo_dominance_ws(const float* F, int64_t n2, int32_t m, uint32_t* D, int64_t ld_words, int32_t* dom_count,
                            void* ws, size_t ws_bytes, emo_stream_t stream);

/*
 * emo_dominance restricted to the columns [col_lo, col_hi) (col_lo a multiple
 * of 1024, col_hi <= n2): row i (all n2 rows), word w, bit b of D is 1 iff
 * F_i dominates F_{col_lo + 32w + b}; ld_words >= ceil((col_hi - col_lo) / 32);
 * dom_count[j - col_lo] (nullable) = the dominators of column j. One rank's
 * share of the matrix when the columns of one population are split over
 * several GPUs (each GPU holds D[:, its columns]).
 */
emo_status emo_dominance_cols(const float* F, int64_t n2, int32_t m, int64_t col_lo, int64_t col_hi, uint32_t* D,
                              int64_t ld_words, int32_t* dom_count, emo_stream_t stream);

/*
 * One peeling step (Algorithm S.3, "c -= d") on a rank's columns: with D as
 * written by emo_dominance_cols (ncols columns, leading dimension ld_words),
 * counts[j] -= the number of the n_rows rows listed in `rows` (device int32,
 * row indices of the current front) whose bit j is set, and next_front[j]
 * (device uint8) = 1 when counts[j] reached zero in this step, else 0. The
 * rows of one front never dominate each other, so a column of the current
 * front is never flagged again.
 */
emo_status emo_front_counts(const uint32_t* D, int64_t ld_words, int64_t ncols, const int32_t* rows, int64_t n_rows,
                            int32_t* counts, uint8_t* next_front, emo_stream_t stream);

/*
 * Nondominated sorting (Section IV-A "Nondominated Sorting", Algorithm S.3,
 * equal to Deb's sort of Algorithm S.2).
 *   n_keep    0 ranks every point; otherwise peeling stops at the first
 *             front l whose cumulative size reaches n_keep, and points of
 *             later fronts get EMO_NOT_RANKED.
 *   rank      [n2] int32 output, 0-based front index.
 *   last_rank device int32*, nullable: l (rank of the n_keep-th best point;
 *             the last front when n_keep == 0).
 *   ws        workspace of emo_workspace_size(EMO_OP_ND_RANK, n2, m, 0) bytes.
 */
emo_status emo_nd_rank(const float* F, int64_t n2, int32_t m, int64_t n_keep, int32_t* rank,
                       int32_t* last_rank, void* ws, size_t ws_bytes, emo_stream_t stream);

/*
 * NSGA-III environmental selection (Algorithm S.1; tensorized form in
 * Section IV-A and Algorithm S.4): nondominated sorting, normalisation by
 * the ideal point, ASF extreme points and hyperplane intercepts with the
 * nadir fallback (Algorithm S.5; FP64), association to the reference lines
 * by perpendicular distance, niche counts, and niching of the last front.
 *   R          [n_r*m] reference directions: finite, non-negative, non-zero
 *              rows (Das-Dennis points of the unit simplex are). A negative
 *              component gives EMO_ERR_INVALID_ARG on the device.
 *   n_keep     N, 1 <= N <= n2.
 *   seed, generation  key and counter of the Philox-4x32-10 stream that
 *              breaks niching ties (same inputs give the same survivors).
 *   survivors  [n_keep] int32 output: indices of the survivors, ascending.
 *   info       device emo_select_info*, nullable.
 *   ws         workspace of emo_workspace_size(EMO_OP_NSGA3_SELECT, ...)
 *              bytes; about n2^2/16 bytes for the dominance tiles plus
 *              O(n2 + n_r) for the rest.
 */
emo_status emo_nsga3_select(const float* F, int64_t n2, int32_t m, const float* R, int32_t n_r,
                            int64_t n_keep, uint64_t seed, uint64_t generation, int32_t* survivors,
                            emo_select_info* info, void* ws, size_t ws_bytes, emo_stream_t stream);

/* Niche selection of the last front. */
#define EMO_NICHE_EXACT 0   /* Algorithm S.1: least-crowded references served level by level */
#define EMO_NICHE_ONESHOT 1 /* the tensorized one-shot niche selection of Algorithm S.4 followed
                               by Update-Rank (Algorithm S.6): every reference with niche count 0
                               and last-front candidates takes its nearest candidate; then the
                               remaining slots are filled from the other last-front points, or
                               the surplus is dropped from the taken ones, in the order of Philox
                               keys (counter (i, 0xFFFFFFF0 + tag, generation); tag 1 fills, tag 2
                               drops) where the paper relies on a shuffled input. */

/*
 * emo_nsga3_select with the niche selection chosen by `niche_mode`
 * (EMO_NICHE_EXACT or EMO_NICHE_ONESHOT; anything else gives
 * EMO_ERR_INVALID_ARG) and the optional intermediates of `dbg` (a host
 * pointer to a struct of device pointers, nullable). Steps a0-a8 are shared
 * by both modes; other arguments as for emo_nsga3_select.
 */
emo_status emo_nsga3_select_ex(const float* F, int64_t n2, int32_t m, const float* R, int32_t n_r,
                               int64_t n_keep, uint64_t seed, uint64_t generation, int32_t niche_mode,
                               int32_t* survivors, emo_select_info* info, const emo_select_debug* dbg,
                               void* ws, size_t ws_bytes, emo_stream_t stream);

/*
 * emo_nsga3_select for a population whose nondominated ranks are already
 * known (computed, for instance, by several GPUs that split the columns of
 * its dominance matrix): rank is device int32 [n2] in caller order, 0-based
 * fronts for at least the first n_keep points of the order by rank, and
 * EMO_NOT_RANKED (or any rank) beyond. l, |P| and |L| follow from the ranks;
 * normalisation, association, niching and survivors are those of
 * emo_nsga3_select. No dominance matrix is built: ws of
 * emo_workspace_size(EMO_OP_SELECT_RANKED, n2, m, n_r) bytes. Fewer than
 * n_keep ranked points gives EMO_ERR_INVALID_ARG on the device.
 */
emo_status emo_nsga3_select_ranked(const float* F, int64_t n2, int32_t m, const float* R, int32_t n_r,
                                   int64_t n_keep, uint64_t seed, uint64_t generation, const int32_t* rank,
                                   int32_t* survivors, emo_select_info* info, void* ws, size_t ws_bytes,
                                   emo_stream_t stream);

/*
 * The two halves of emo_nsga3_select_ranked for a population split over
 * several GPUs, each GPU owning the points [col_lo, col_hi) of the caller
 * order (Section IV-A "Association" and "Niche Count Calculation": the
 * association is independent per point, the niche counts are sums over the
 * points of P = {rank < l}, so the GPUs associate their own points and add
 * up their counts).
 *
 * emo_nsga3_associate_range: the normalisation over all of S = {rank <= l}
 * (every GPU computes the same ideal point, extreme points and intercepts
 * from the whole F, as emo_nsga3_select does), then the association of the
 * points of S in [col_lo, col_hi) only. Arguments F .. rank as for
 * emo_nsga3_select_ranked (no seed: nothing random happens here). Outputs
 * (device): pi int32 [col_hi - col_lo], the associated reference of point
 * col_lo + i, -1 outside S; dist double [col_hi - col_lo], its FP64
 * perpendicular distance, NaN outside S; rho int32 [n_r], the niche counts of
 * the range's points of P. pi and dist may be null when col_lo == col_hi.
 * The values are those emo_nsga3_select computes for these points. info
 * (nullable, device): last_rank, n_before, n_last, fallback_used and n_fronts
 * of the whole population, n_recheck over the range, n_levels 0. ws of
 * emo_workspace_size(EMO_OP_SELECT_RANKED, n2, m, n_r) bytes.
 *
 * emo_nsga3_niche_given: the niche selection and the survivors (Algorithm
 * S.1 from its niche counts; the selection of emo_nsga3_select with
 * niche_mode) from the association gathered from the GPUs: rank as above;
 * rho int32 [n_r], the niche counts of all of P (the sum of every GPU's rho);
 * last int32 [n_last], the members of front l in ascending caller order (the
 * concatenation of the GPUs' members when they own increasing ranges),
 * last_pi int32 [n_last] and last_dist double [n_last], their references
 * and distances. survivors int32 [n_keep] and info as for
 * emo_nsga3_select_ex; the survivors are those of emo_nsga3_select_ranked on
 * the same ranks. Checked on the device (EMO_ERR_INVALID_ARG): n_last = |L|,
 * last strictly ascending with every member of rank l, references in
 * [0, n_r), distances finite and non-negative, counts non-negative and
 * adding up to |P|. ws of emo_workspace_size(EMO_OP_SELECT_RANKED, n2, 2,
 * n_r) bytes (no objectives are read).
 */
emo_status emo_nsga3_associate_range(const float* F, int64_t n2, int32_t m, const float* R, int32_t n_r,
                                     int64_t n_keep, const int32_t* rank, int64_t col_lo, int64_t col_hi,
                                     int32_t* pi, double* dist, int32_t* rho, emo_select_info* info, void* ws,
                                     size_t ws_bytes, emo_stream_t stream);
emo_status emo_nsga3_niche_given(int64_t n2, int32_t n_r, int64_t n_keep, uint64_t seed, uint64_t generation,
                                 int32_t niche_mode, const int32_t* rank, const int32_t* rho, const int32_t* last,
                                 const int32_t* last_pi, const double* last_dist, int64_t n_last,
                                 int32_t* survivors, emo_select_info* info, void* ws, size_t ws_bytes,
                                 emo_stream_t stream);

/* As emo_nsga3_select, also writing the intermediates named in `dbg` (a
 * host pointer to a struct of device pointers, nullable). */
emo_status emo_nsga3_select_debug(const float* F, int64_t n2, int32_t m, const float* R,
                                  int32_t n_r, int64_t n_keep, uint64_t seed, uint64_t generation,
                                  int32_t* survivors, emo_select_info* info,
                                  const emo_select_debug* dbg, void* ws, size_t ws_bytes,
                                  emo_stream_t stream);

/*
 * Many independent populations (uneven n2, m, n_r) in one sequence of
 * launches: each stage is one persistent launch that serves every
 * population, so the whole batch can be captured in one CUDA graph.
 * Batching is not in the paper; its vmap over populations (Section III-C)
 * is the analogue. `descs` is a HOST array of `batch` descriptors
 * (1 <= batch <= EMO_MAX_BATCH) whose pointers are device pointers; it is
 * read during the call only.
 */
size_t emo_batch_workspace_size(const emo_problem* descs, int32_t batch);
emo_status emo_nsga3_select_batch(const emo_problem* descs, int32_t batch, void* ws,
                                  size_t ws_bytes, emo_stream_t stream);

/*
 * TensorHypE environmental selection (Algorithm S.10) with the Monte Carlo
 * hypervolume estimation of Algorithm S.11: ranks and l as for
 * emo_nsga3_select; k = |{rank <= l}| - n_keep; samples S_i = f_l + U_i
 * (v_ref - f_l) (float, f_l = the column minima of F); c_i = the points
 * weakly dominating S_i; a point's contribution = vol / s times the sum of
 * alpha_{c_i} over the samples it dominates, in sample order, with
 * alpha_c = (lambda_1 ... lambda_c) / c, lambda_1 = 1,
 * lambda_i = (k - i + 1) / (n2 - i + 1) (zero beyond c = k); survivors =
 * every point with rank < l plus the points of front l with the largest
 * contributions (ties: lower index), ascending.
 *   F          [n2*m] objectives (device), as for emo_nsga3_select.
 *   v_ref      [m] reference point (device), finite.
 *   U          [n_samples*m] uniform numbers in [0, 1) (device), the caller's
 *              random draws of the samples.
 *   n_samples  s >= 1.
 *   survivors  [n_keep] int32 output, ascending.
 *   info       device emo_select_info*, nullable (n_levels = 0).
 *   hv         [n2] double output (device, nullable): the contribution of
 *              each point of front l, 0 elsewhere.
 *   ws         workspace of emo_workspace_size(EMO_OP_HYPE_SELECT, n2, m,
 *              n_samples) bytes.
 */
emo_status emo_hype_select(const float* F, int64_t n2, int32_t m, const float* v_ref, const float* U,
                           int32_t n_samples, int64_t n_keep, int32_t* survivors, emo_select_info* info,
                           double* hv, void* ws, size_t ws_bytes, emo_stream_t stream);

/*
 * TensorMOEA/D environmental selection (Algorithm S.8, PBI aggregation of
 * Section IV-B): n subproblems, each with a current solution and one
 * offspring per subproblem.
 *   X, O       device float [n][d]: current solutions and offspring
 *   F1, F2     device float [n][m]: their objectives (finite)
 *   z          device float [m], in/out: the ideal point; on return
 *              z_min = per-objective minimum of z and F2 (a zero is +0)
 *   W          device float [n][m]: weight vectors (finite, non-zero)
 *   I_nb       device int32 [n][T]: neighbour subproblems of each offspring
 *              (0 <= I_nb < n; a neighbour listed twice counts once)
 *   theta      PBI penalty (>= 0, finite; 5 is customary)
 *   X_next, F_next  device outputs [n][d], [n][m]; X_next may be X and
 *              F_next may be F1 (in place); neither may overlap O or F2
 *   winner     device int32 [n] or NULL: the offspring each subproblem took,
 *              -1 when it kept its solution
 *   status_out device int32 or NULL: EMO_OK, EMO_ERR_INVALID_ARG (an
 *              I_nb entry out of range) or EMO_ERR_NONFINITE (non-finite
 *              F1, F2, W or z, or a zero weight vector); outputs are
 *              undefined when it is not EMO_OK. Also folded into the sticky
 *              status of emo_get_last_device_status.
 *   ws         workspace of emo_workspace_size(EMO_OP_MOEAD_SELECT, n, m, T)
 *              bytes, 256-byte aligned.
 * Semantics: offspring i marks neighbour j when PBI(F2_i | W_j, z_min) <=
 * PBI(F1_j | W_j, z_min); subproblem j then takes the first minimum, over
 * positions i = 0 .. n-1, of PBI(f_i | W_j, z_min) where f_i = F2_i if i
 * marked j and F1_j otherwise. PBI: d1 = |(f - z).w| / ||w||,
 * d2 = ||(f - z) - d1 w / ||w|| ||, g = d1 + theta d2, in FP64 from the
 * float inputs (k ascending, no contraction). Asynchronous on `stream`;
 * argument errors are returned at once. 1 <= n <= 2^21, 2 <= m <= 16,
 * 1 <= T <= min(n, 4096).
 */
emo_status emo_moead_select(const float* X, const float* F1, const float* O, const float* F2, int64_t n, int64_t d,
                            int32_t m, float* z, const float* W, const int32_t* I_nb, int32_t T, double theta,
                            float* X_next, float* F_next, int32_t* winner, int32_t* status_out, void* ws,
                            size_t ws_bytes, emo_stream_t stream);

/*
 * Offspring of one generation (Appendix S.I): pair p (0 <= p < ceil(n_off/2))
 * draws two parents uniformly from the n rows of X, crosses every variable
 * by SBX with probability p_c per pair (distribution index eta_c), clips to
 * [lo, hi], mutates each variable with probability p_m by polynomial
 * mutation (original form, eta_m), clips again and writes its children to
 * rows p and ceil(n_off/2) + p of X_off (the second when it exists).
 * Randomness: Philox-4x32-10 keyed by `seed`, counter (row, 0x80000000 |
 * tag << 24 | slot, generation lo, hi); tag 1 parents (slot 0 / 1, word 1
 * of slot 0 decides crossover), tag 2 SBX spread (slot = variable), tag 3
 * mutation (slot = variable; word 0 decides, word 1 is mu); a word x is the
 * uniform x 2^-32 and the index (x n) >> 32. FP64 arithmetic, rounded to
 * float once. X, X_off device float; lo, hi device float [d] (each
 * lo < hi; a variable with hi <= lo is not mutated, so it never turns into
 * NaN), or both NULL for [0, 1]; parents device int32
 * [ceil(n_off/2)][2] or NULL. d < 2^24.
 */
emo_status emo_variation(const float* X, int64_t n, int64_t d, const float* lo, const float* hi, int64_t n_off,
                         uint64_t seed, uint64_t generation, double eta_c, double eta_m, double p_c, double p_m,
                         float* X_off, int32_t* parents, emo_stream_t stream);

/*
 * Stand-in objectives with the front shapes of DTLZ1 / DTLZ2 (the DTLZ
 * definitions themselves are not part of this library): for decision
 * vectors x in [0,1]^d (d >= m), g = sum_{i >= m-1} (x_i - 0.5)^2;
 * EMO_SHAPE_LINEAR: f = 0.5 (1 + 100 g) s with s the stick-breaking simplex
 * point of x_0 .. x_{m-2} (sum f = 0.5 when g = 0); EMO_SHAPE_SPHERE:
 * f = (1 + g) u with u the unit vector of angles x_i pi / 2 (||f|| = 1 when
 * g = 0). FP64, rounded to float once. X device float [n][d], F device
 * float [n][m].
 */
emo_status emo_standin_objectives(const float* X, int64_t n, int64_t d, int32_t m, int32_t shape, float* F,
                                  emo_stream_t stream);

/*
 * Inverted generational distance: the mean over the n_ref points of `Ref`
 * of the distance to the nearest of the n points of F (squared distances in
 * float, square roots and the sum in double, summed in index order). F, Ref
 * device float [.][m]; igd_out device double; ws of
 * emo_workspace_size(EMO_OP_IGD, n_ref, m, 0) bytes (8-byte aligned).
 */
emo_status emo_igd(const float* F, int64_t n, int32_t m, const float* Ref, int64_t n_ref, double* igd_out, void* ws,
                   size_t ws_bytes, emo_stream_t stream);

/*
 * One NSGA-III generation in place on the device, in stream order (and so
 * capturable in a CUDA graph): N offspring of (X, F) by emo_variation
 * (bounds [0, 1]), their stand-in objectives (`shape`), the merged
 * population of 2N points, emo_nsga3_select_ex (keep N, `niche_mode`,
 * `seed`, `generation`), and the survivors' rows gathered back into X
 * [N][d] and F [N][m]. ws of emo_generation_workspace_size(N, d, m, n_r)
 * bytes, 256-byte aligned; info as for emo_nsga3_select. m <= d <= 2^20.
 */
size_t emo_generation_workspace_size(int64_t n, int64_t d, int32_t m, int32_t n_r);
emo_status emo_nsga3_generation(float* X, float* F, int64_t n, int64_t d, int32_t m, const float* R, int32_t n_r,
                                int32_t shape, uint64_t seed, uint64_t generation, double eta_c, double eta_m,
                                double p_c, double p_m, int32_t niche_mode, emo_select_info* info, void* ws,
                                size_t ws_bytes, emo_stream_t stream);

/*
 * emo_nsga3_select without a caller workspace, for callers that cannot
 * allocate device memory (a plug-in whose host owns every allocation, a loop
 * that must not enter an allocator, a fixed memory budget). The paper has no
 * counterpart; this is a deployment convenience. The selection runs in an
 * 9 MiB scratch array built into the library (held on every GPU that loads
 * it until the process exits); populations with n2 <= 7168 and n_r <= 7168
 * (any m <= 16) always fit on devices with up to 304 SMs, and n2 <= 8192
 * with n_r <= 8192 (m <= 8) on devices with up to 152 SMs (the workspace
 * grows with the CTAs of a cooperative launch, up to 2 per SM); what does
 * not fit returns EMO_ERR_WORKSPACE. The call
 * makes no device allocation. Its first call on a device looks up the
 * scratch address (cudaGetSymbolAddress) and should come before any stream
 * capture. Calls share the scratch: every call initialises what it reads,
 * but calls that overlap on the GPU race and must be ordered by the caller.
 * Other arguments as for emo_nsga3_select.
 */
emo_status emo_nsga3_select_noalloc(const float* F, int64_t n2, int32_t m, const float* R, int32_t n_r,
                                    int64_t n_keep, uint64_t seed, uint64_t generation, int32_t* survivors,
                                    emo_select_info* info, emo_stream_t stream);

/* Synchronises `stream` and reads the device status word of a workspace
 * last used on it (EMO_OK when every problem finished cleanly). */
emo_status emo_workspace_status(const void* ws, emo_stream_t stream, int32_t* status_out);

/* The first status a device-side check reported on the current device
 * (EMO_ERR_NONFINITE, EMO_ERR_INVALID_ARG, EMO_ERR_TIMEOUT from any call,
 * 0 when none) since the last read; waits for `stream`'s prior work and
 * clears the word, like cudaGetLastError. */
emo_status emo_get_last_device_status(emo_stream_t stream, int32_t* status_out);

/* Offline tuning of the launch shapes for populations of m objectives and
 * about n2 points (same floor(log2 n2)) on the current device's
 * architecture, by a coordinate search timed with the stage events on a
 * synthetic population (a sphere-shaped front and n2/2 directions on the
 * simplex), each candidate the best of three selections, in this order:
 *   1. dominance work-item size (row blocks per item: 64 .. 1024) by the
 *      dominance kernel's time;
 *   2. the schedule of the peeling by its time: one grid barrier per front,
 *      or the wavefront (a block's task for front k starts as soon as every
 *      lower column block has finished front k - 1; no grid barrier); then
 *      how many CTAs serve it (every CTA, half, a quarter, ... down to a
 *      single CTA);
 *   3. the CTAs of the other cooperative stages (sort, statistics, CSR,
 *      niching, survivors; at most as many as step 2) by their summed time;
 *   4. the association kernel's blocks per SM (2, 4, 8, 16, 32).
 * It allocates device memory and synchronises, so it belongs outside timed
 * regions and graph captures. With a non-null `cache_path`, results found in
 * that text file (lines "arch m bucket assoc_bps dom_chunk cap_wide
 * cap_narrow peel_wave", arch = 10 * major + minor compute capability,
 * bucket = floor(log2 n2), a cap of 0 = every CTA; lines of the first four
 * or seven fields also load) are loaded and reused, and a new
 * result is appended. Later calls of the same process use the tuned shapes,
 * and the first selection of a process loads the file named by the
 * environment variable EMO_AUTOTUNE_CACHE, if set. Untuned sizes use 8
 * association blocks per SM, the largest dominance items that give every SM
 * at least two, and no caps. Survivors do not depend on the shapes.
 * EMO_ERR_INVALID_ARG for n2 < 64 or sizes out of range. */
emo_status emo_autotune(int32_t m, int64_t n2, const char* cache_path);

/* The launch shapes a selection of n2 points with m objectives would use on
 * the current device now (tuned or default), into shape_out[5]: [0]
 * association blocks per SM, [1] dominance row blocks per work item, [2]
 * CTAs of the peeling group, [3] CTAs of the other cooperative groups (a
 * batch can give a population fewer), [4] the peeling schedule (1
 * wavefront, 0 a grid barrier per front). */
emo_status emo_launch_shape(int32_t m, int64_t n2, int32_t* shape_out);

/* Forgets every tuned shape of this process (later calls use the defaults
 * until emo_autotune runs or EMO_AUTOTUNE_CACHE is loaded again). */
void emo_autotune_reset(void);

/* Bounded-wait budget (in SM clock cycles) for the device-side barriers of
 * later calls in this process; 0 restores the default (about 2 s). */
void emo_set_spin_budget(int64_t cycles);

/* Static description of a status code. */
const char* emo_status_string(int status);

/* Library version, e.g. 100 for 0.1.0. */
int32_t emo_version(void);

/* Human-readable report of the current device as the library sees it (SM
 * count, cooperative-launch support, registers, shared memory and resident
 * CTAs of the cooperative kernels) into buf (NUL-terminated, truncated to
 * len). Returns the full report length, -1 on bad arguments. */
int32_t emo_device_report(char* buf, int32_t len);

/* Opt-in stage timing for profiling. While enabled, every multi-stage call
 * records CUDA events on its stream between its stages (prep, sort,
 * colprep, dominance, peel, stats, assoc, rescan, csr, niche, finish). After a call,
 * emo_stage_times synchronises on the last event and writes up to max_n
 * stage durations (ms, host array) and static stage names (host array of
 * const char*, nullable). Returns the number of stages, 0 when nothing was
 * recorded on this host thread, -1 on a CUDA error. */
void emo_set_stage_timing(int32_t enable);
int32_t emo_stage_times(float* ms_out, const char** names_out, int32_t max_n);

#ifdef __cplusplus
}
#endif

#endif /* EMO_H */
