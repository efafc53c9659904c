// Internal definitions of the sm_103a NSGA-III selection library.
//
// Data layout in HBM, per population ("problem"):
//   * points are first put in lexicographic order of their objective vectors
//     (stable LSD radix sort).  In that order p < q implies that q cannot
//     dominate p, so the dominance matrix is strictly upper triangular;
//   * the triangle is stored as 4 KB tiles of 32 rows x 1024 columns
//     (32 rows x 32 uint32 words).  Row block rb = rows [32 rb, 32 rb + 32),
//     column block cb = columns [1024 cb, 1024 cb + 1024); tile (rb, cb)
//     exists for cb >= rb / 32.  Tiles of a row block are contiguous; inside
//     a tile, word w of row r (columns 32 w .. 32 w + 31 of the block, bit b
//     = column 32 w + b) sits at position r * 32 + w;
//   * the objective keys used by the dominance kernel are the objectives
//     2..m of each point in sorted order, array-of-structs with stride m-1,
//     padded to a multiple of 1024 points with -inf;
//   * everything downstream of the peeling works in the caller's order.
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/emo.h"

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace emo {

constexpr int kMaxM = EMO_MAX_OBJECTIVES;
constexpr int kMaxBatch = EMO_MAX_BATCH;
constexpr int kTileRows = 32;         // rows per row block
constexpr int kTileWords = 32;        // words per tile row
constexpr int kColBlock = 1024;       // columns per column block
constexpr int kDomRowChunk = 1024;    // row blocks per dominance work item (largest; emo_dominance)
constexpr int kDomChunkMin = 64;      // smallest row-block chunk of a selection's dominance items
constexpr int kCoopThreads = 512;     // threads of the cooperative kernels
constexpr int kNicheBins = 4096;      // niching select: bins of the top 12 bits of a priority
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int64_t kMaxN2 = int64_t(1) << 21;
constexpr int32_t kNotRanked = EMO_NOT_RANKED;

enum Mode : int32_t { MODE_RANK = 1, MODE_SELECT = 2, MODE_HYPE = 3, MODE_DOM = 4 };

// What the host knows about one problem.
struct ProbIn {
    const float* F;
    const float* R;
    int32_t* survivors;
    emo_select_info* info;
    int64_t n2;
    int64_t n_keep;     // 0 = rank everything (MODE_RANK only)
    int32_t m;
    int32_t n_r;
    uint64_t seed;
    uint64_t gen;
    int32_t mode;
    int32_t niche;           // EMO_NICHE_EXACT or EMO_NICHE_ONESHOT (MODE_SELECT)
    const float* U;          // MODE_HYPE: [n_r * m] uniform numbers of the samples (n_r = samples; R = v_ref)
    double* hv_out;          // MODE_HYPE: [n2] contributions of front l (nullable)
    int32_t* rank_out;       // MODE_RANK
    int32_t* last_rank_out;  // nullable
    emo_select_debug dbg;
    uint64_t ws_off;         // byte offset of this problem's region
    // launch shapes (tuned per device, objective count and size; survivors
    // never depend on them)
    int32_t dom_chunk;       // row blocks per dominance work item: 64 .. 1024, a power of two
    int32_t cap_wide;        // most CTAs of the peeling (and TensorHypE) group; 0 = no cap
    int32_t cap_narrow;      // most CTAs of the sort / statistics / CSR / niching / survivor groups; 0 = no cap
    int32_t ranked;          // MODE_SELECT from the given ranks rank_in (no dominance matrix, no peeling)
    const int32_t* rank_in;  // [n2] caller-order ranks (EMO_NOT_RANKED beyond the last needed front)
    uint32_t* dom_out;       // MODE_DOM: [n2][dom_ld] caller-order dominance matrix
    int32_t* dom_count;      // MODE_DOM: [n2] dominator counts (nullable)
    int64_t dom_ld;          // MODE_DOM: words per row
};

// Per-problem scalars; zeroed by the prep kernel.
struct Scal {
    int32_t status;
    int32_t l;
    int32_t nP, nL, nS;
    int32_t ranked;          // points ranked so far
    int32_t nfronts;
    int32_t fallback;
    int32_t nflag;           // points needing the all-reference FP64 scan
    int32_t levels;
    int32_t front_total[2];  // members of the current / next front
    int32_t idx_buf;         // idx half holding the sorted order
    int32_t lbuf;            // llist half holding the sorted candidate lists
    int32_t rbuf;            // rord half holding the angle order
    uint32_t zkey[kMaxM];
    uint32_t kor[kMaxM];     // OR of the order-preserving keys of each objective over all points
    uint32_t kinv[kMaxM];    // OR of their complements (a bit varies iff set in both)
    uint32_t asf32[kMaxM];
    unsigned long long asf64[kMaxM];
    int32_t ext[kMaxM];
    unsigned long long nadir[kMaxM];
    float z[kMaxM];
    float inv_a32[kMaxM];
    double a[kMaxM];
    unsigned int bar_count;
    unsigned int bar_gen;
    int32_t ncol;            // niching: keys collected from the selected histogram bin
    int32_t nsel;            // one-shot niching: references that took their nearest candidate
    int32_t longrun;         // sort: a run of equal f_1 longer than the in-place fix-up handles
    int32_t lfinal1;         // wavefront peeling: l + 1 once known, 0 before
    unsigned long long rho_sum;  // niching from a given association: sum of the given niche counts
};

// Device-side descriptor with every workspace pointer of one problem.
struct ProbDev {
    ProbIn in;
    int32_t nrb, ncb;        // row blocks (32 rows), column blocks (1024 columns)
    int64_t n2p;             // n2 padded to ncb * 1024
    int64_t ntiles;
    Scal* sc;
    uint32_t* D;             // dominance tiles
    int32_t* idx;            // [2][n2p] sorted position -> caller index (ping-pong)
    float* keys;             // [n2p][m-1] objectives 2..m in sorted order
    int32_t* runstart;       // [n2p] first sorted position of the run of equal points
    int32_t* minrs;          // [ncb] min runstart of non-leading run members
    int32_t* cnt;            // [n2p] dominator counts (sorted order)
    int32_t* rank_s;         // [n2p] ranks (sorted order)
    int32_t* rank_o;         // [n2]  ranks (caller order)
    int32_t* front;          // [3][n2p] front members grouped by column block (3 buffers); the
                             // wavefront peeling keeps each block's members in front order in the first
    int32_t* front_n;        // [3][ncb] members per column block
    int32_t* wdone;          // [ncb] wavefront: fronts whose counts block cb has applied (INT32_MAX: exhausted)
    int32_t* wmaxf;          // [ncb] wavefront: last front with offsets of an exhausted block
    int32_t* wcnt;           // [n2 + 2] wavefront: members of front k
    uint16_t* wofs;          // [ncb][n2 + 2] wavefront: start of front k in block cb's member list
    int32_t* slist;          // [n2] caller indices of S = {rank <= l}
    int32_t* pi;             // [n2] associated reference
    double* d64;             // [n2] perpendicular distance (FP64)
    float* rhat;             // [n_r][m] unit reference directions (FP32)
    int32_t* rord;           // [2][n_r] references sorted by polar angle from axis 1 (ping-pong)
    float* rphi;             // [n_r] sorted polar angles (from axis 1)
    float* rphi2;            // [n_r] angles from axis 2, in the same order
    float* rsort;            // [n_r][m] unit directions in polar-angle order
    int32_t* flagged;        // [n2] points for the exhaustive FP64 scan
    float* flagged_bound;    // [n2] angular half-width of that scan (inf = all references)
    int32_t* rho;            // [n_r] niche counts of P (evolving during niching)
    int32_t* lcnt;           // [n_r] last-front members per reference (evolving)
    int32_t* loff;           // [n_r + 1] CSR offsets of the candidate lists
    int32_t* llist;          // [2][n2] last-front members (CSR order after sorting)
    int32_t* fen;            // [n2] Fenwick trees over each candidate list
    unsigned long long* ekeys;  // [max(n_r, n2)] niching keys collected from one histogram bin
    int32_t* nhist;          // niching: [kNicheBins] key histogram | [G] packed per-CTA (min, count)
    int32_t* elist;          // [n_r] references served in a level
    int32_t* flag;           // [n2] survivor flags / scan scratch
    int32_t* hist;           // [G][256] radix histograms, reused by the scans
    unsigned char* colpre;   // [ncb][K] column-block prefix sets (colprep_obj_bytes each; K = m - 1 key
                             // objectives, or all m of the caller-order columns in MODE_DOM)
    float* ckeys;            // MODE_DOM: [n2p][m] objectives in caller order (padding -inf)
    int32_t* spos;           // MODE_DOM: [2][n2] run of identical points of each caller index: first
                             // sorted position (-1 when alone), one past the last
};

// A population split over several GPUs (one problem per call, ranks given):
// the association of one GPU's points, or the niching from the association
// gathered from all of them.
enum SplitKind : int32_t { SPLIT_NONE = 0, SPLIT_ASSOC = 1, SPLIT_NICHE = 2 };
struct SplitArgs {
    int32_t kind;
    int32_t pad_;
    int64_t col_lo, col_hi;  // SPLIT_ASSOC: the caller indices associated
    int32_t* pi_out;         // SPLIT_ASSOC: [col_hi - col_lo] reference, -1 outside S
    double* d_out;           // SPLIT_ASSOC: [col_hi - col_lo] FP64 distance, NaN outside S
    int32_t* rho;            // SPLIT_ASSOC: output [n_r] niche counts of P in the range;
                             // SPLIT_NICHE: input [n_r] niche counts of all of P
    const int32_t* last;     // SPLIT_NICHE: [n_last] front l, ascending caller indices
    const int32_t* last_pi;  // SPLIT_NICHE: [n_last] their references
    const double* last_d;    // SPLIT_NICHE: [n_last] their FP64 distances
    int64_t n_last;
};

struct Plan {
    int32_t nprob;
    int32_t G;               // CTAs of every cooperative launch
    long long spin_budget;   // cycles a bounded wait may spin
    int32_t grp_first[kMaxBatch + 1];     // cooperative CTA groups of the peeling and TensorHypE kernels
    int32_t grpn_first[kMaxBatch + 1];    // groups of the other cooperative kernels (at most as large)
    long long dom_item_start[kMaxBatch + 1];
    long long dom_items;
    unsigned long long dom_ctr[kMaxM + 1];  // dynamic work counters per objective count
    unsigned long long asc_next[kMaxM + 1];  // tile counters of the all-reference association, per m
    int32_t status;                       // OR of problem statuses
    int32_t pad_;
    SplitArgs split;                      // problem 0 of a one-problem call
    ProbDev p[kMaxBatch];
};

struct SetupArgs {
    int32_t nprob;
    int32_t G;
    long long spin_budget;
    ProbIn in[kMaxBatch];
};

__host__ __device__ __forceinline__ int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
__host__ __device__ __forceinline__ int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Number of stored tiles before row block rb (tiles of row block b are the
// column blocks cb in [b / 32, ncb)).
__host__ __device__ __forceinline__ int64_t tiles_before(int64_t rb, int64_t ncb)
{
    int64_t s = rb / 32, t = rb % 32;
    return rb * ncb - 32 * (s * (s - 1) / 2) - t * s;
}
__host__ __device__ __forceinline__ int64_t tile_index(int64_t rb, int64_t cb, int64_t ncb)
{
    return tiles_before(rb, ncb) + (cb - rb / 32);
}

// Column-block prefix sets of the dominance kernel. Each 1024-column block
// is split into two halves of 512 columns. For each key objective k
// (objectives 2..m) the block stores:
//   fv   -- the block's 1024 values of f_k sorted descending (entry i at
//           slot i ^ ((i / 32) % 32), which spreads a binary search's
//           candidates over the shared-memory banks);
//   cum0 -- cum0[j] = how many of the first j entries of fv lie in half 0
//           (so a count j of values >= x splits into cum0[j] and j - cum0[j]);
//   pb   -- for each half, the bitsets of its first c * cps columns in the
//           order of f_k descending, c = 0..512/cps. Row c holds 32 words,
//           words 0-15 from half 0 and 16-31 from half 1, so the word w of a
//           tile row always comes from half w / 16;
//   ord  -- (cps > 1 only) each half's local column indices in that order.
//   per objective: float fv[1024] | uint16 cum0[1025] (+pad) | uint32 pb[512/cps + 1][32] | uint16 ord[2][512]
constexpr int kPrefCumOff = kColBlock * 4;
constexpr int kPrefPbOff = kPrefCumOff + 2176;  // 1025 uint16 rounded up to 128 bytes
__host__ __device__ constexpr int colprep_log_cps(int K)
{
    return K <= 3 ? 0 : (K <= 5 ? 1 : (K <= 6 ? 2 : (K <= 9 ? 3 : 4)));
}
__host__ __device__ constexpr int64_t colprep_ord_off(int K)
{
    return kPrefPbOff + (((kColBlock / 2) >> colprep_log_cps(K)) + 1) * 32 * 4;
}
// Objectives with at most two prefix-set keys also carry a bucket index of
// the block's descending values (header: lowest finite value, bucket scale;
// then per bucket the first and one-past-last positions of the values in
// it), which turns the search for a row's count into one lookup and a search
// among the few values of one bucket.
constexpr int kPrefBuckets = 4096;
__host__ __device__ constexpr bool colprep_has_buckets(int K) { return K <= 2; }
__host__ __device__ constexpr int64_t colprep_bkt_off(int K)
{
    return colprep_ord_off(K) + (colprep_log_cps(K) > 0 ? kColBlock * 2 : 0);
}
__host__ __device__ constexpr int64_t colprep_obj_bytes(int K)
{
    return colprep_bkt_off(K) + (colprep_has_buckets(K) ? 128 + kPrefBuckets * 4 : 0);
}

// Byte layout of one problem region; fills `d` when base != 0. Returns the
// region size. The same function sizes the workspace on the host and carves
// it on the device.
__host__ __device__ inline int64_t layout_problem(const ProbIn& in, int G, char* base, ProbDev* d)
{
    const int64_t n2 = in.n2, m = in.m, nr = (in.mode == MODE_SELECT || in.mode == MODE_HYPE) ? in.n_r : 1;
    const int64_t nrb = cdiv(n2, 32), ncb = cdiv(n2, kColBlock), n2p = ncb * kColBlock;
    const int64_t ntiles = tiles_before(nrb, ncb);
    int64_t off = 0;
    auto take = [&](int64_t bytes) { int64_t o = off; off = align_up(off + bytes, 256); return o; };
    int64_t o_sc = take(sizeof(Scal));
    int64_t o_idx = take(2 * n2p * 4);
    int64_t o_keys = take(n2p * (m - 1) * 4);
    int64_t o_runstart = take(n2p * 4);
    int64_t o_minrs = take(ncb * 4);
    int64_t o_cnt = take(n2p * 4);
    int64_t o_rank_s = take(n2p * 4);
    int64_t o_rank_o = take(n2 * 4);
    int64_t o_front = take(3 * n2p * 4);
    int64_t o_front_n = take(3 * ncb * 4);
    int64_t o_wdone = take(2 * ncb * 4);
    int64_t o_wcnt = take((n2 + 2) * 4);
    int64_t o_wofs = (in.ranked || in.mode == MODE_DOM) ? 0 : take(ncb * (n2 + 2) * 2);
    int64_t o_slist = take(n2 * 4);
    int64_t o_hist = take(int64_t(G) * kRadix * 4);
    int64_t o_flag = take((n2p + 1) * 4);
    int64_t o_pi = 0, o_d64 = 0, o_rhat = 0, o_flagged = 0, o_rho = 0, o_lcnt = 0, o_loff = 0,
            o_llist = 0, o_fen = 0, o_ekeys = 0, o_elist = 0, o_rord = 0, o_rphi = 0, o_rsort = 0, o_fbound = 0,
            o_nhist = 0, o_rphi2 = 0;
    if (in.mode == MODE_SELECT) {
        o_pi = take(n2 * 4);
        o_d64 = take(n2 * 8);
        o_rhat = take(nr * m * 4);
        o_flagged = take(n2 * 4);
        o_rho = take(nr * 4);
        o_lcnt = take(nr * 4);
        o_loff = take((nr + 1) * 4);
        o_llist = take(2 * n2 * 4);
        o_fen = take(n2 * 4);
        o_ekeys = take((nr > n2 ? nr : n2) * 8);
        o_elist = take(nr * 4);
        o_rord = take(2 * nr * 4);
        o_rphi = take(nr * 4);
        o_rphi2 = take(nr * 4);
        o_rsort = take(nr * m * 4);
        o_fbound = take(n2 * 4);
        o_nhist = take(kNicheBins * 4 + int64_t(G) * 8);
    } else if (in.mode == MODE_HYPE) {
        // d64: contributions; rhat: samples; rho: their dominator counts;
        // llist: the last front and its sorted copy; ekeys: the weights alpha_c
        o_d64 = take(n2 * 8);
        o_rhat = take(nr * m * 4);
        o_rho = take(nr * 4);
        o_llist = take(2 * n2 * 4);
        o_ekeys = take((n2 + 1) * 8);
    }
    // the prefix sets, the dominance tiles and the wavefront offsets are not
    // needed when the ranks are given
    const int64_t kobj = in.mode == MODE_DOM ? m : m - 1;  // objectives with prefix sets
    int64_t o_colpre = in.ranked ? 0 : take(ncb * kobj * colprep_obj_bytes((int)kobj));
    int64_t o_D = (in.ranked || in.mode == MODE_DOM) ? 0 : take(ntiles * 4096);
    int64_t o_ckeys = in.mode == MODE_DOM ? take(n2p * m * 4) : 0;
    int64_t o_spos = in.mode == MODE_DOM ? take(2 * n2 * 4) : 0;
    if (base && d) {
        d->in = in;
        d->nrb = (int32_t)nrb;
        d->ncb = (int32_t)ncb;
        d->n2p = n2p;
        d->ntiles = ntiles;
        d->sc = (Scal*)(base + o_sc);
        d->idx = (int32_t*)(base + o_idx);
        d->keys = (float*)(base + o_keys);
        d->runstart = (int32_t*)(base + o_runstart);
        d->minrs = (int32_t*)(base + o_minrs);
        d->cnt = (int32_t*)(base + o_cnt);
        d->rank_s = (int32_t*)(base + o_rank_s);
        d->rank_o = (int32_t*)(base + o_rank_o);
        d->front = (int32_t*)(base + o_front);
        d->front_n = (int32_t*)(base + o_front_n);
        d->wdone = (int32_t*)(base + o_wdone);
        d->wmaxf = d->wdone + ncb;
        d->wcnt = (int32_t*)(base + o_wcnt);
        d->wofs = (in.ranked || in.mode == MODE_DOM) ? nullptr : (uint16_t*)(base + o_wofs);
        d->slist = (int32_t*)(base + o_slist);
        d->hist = (int32_t*)(base + o_hist);
        d->flag = (int32_t*)(base + o_flag);
        d->pi = in.mode == MODE_SELECT ? (int32_t*)(base + o_pi) : nullptr;
        d->d64 = (in.mode == MODE_SELECT || in.mode == MODE_HYPE) ? (double*)(base + o_d64) : nullptr;
        d->rhat = (in.mode == MODE_SELECT || in.mode == MODE_HYPE) ? (float*)(base + o_rhat) : nullptr;
        d->flagged = in.mode == MODE_SELECT ? (int32_t*)(base + o_flagged) : nullptr;
        d->rho = (in.mode == MODE_SELECT || in.mode == MODE_HYPE) ? (int32_t*)(base + o_rho) : nullptr;
        d->lcnt = in.mode == MODE_SELECT ? (int32_t*)(base + o_lcnt) : nullptr;
        d->loff = in.mode == MODE_SELECT ? (int32_t*)(base + o_loff) : nullptr;
        d->llist = (in.mode == MODE_SELECT || in.mode == MODE_HYPE) ? (int32_t*)(base + o_llist) : nullptr;
        d->fen = in.mode == MODE_SELECT ? (int32_t*)(base + o_fen) : nullptr;
        d->ekeys = (in.mode == MODE_SELECT || in.mode == MODE_HYPE) ? (unsigned long long*)(base + o_ekeys) : nullptr;
        d->elist = in.mode == MODE_SELECT ? (int32_t*)(base + o_elist) : nullptr;
        d->nhist = in.mode == MODE_SELECT ? (int32_t*)(base + o_nhist) : nullptr;
        d->rord = in.mode == MODE_SELECT ? (int32_t*)(base + o_rord) : nullptr;
        d->rphi = in.mode == MODE_SELECT ? (float*)(base + o_rphi) : nullptr;
        d->rphi2 = in.mode == MODE_SELECT ? (float*)(base + o_rphi2) : nullptr;
        d->rsort = in.mode == MODE_SELECT ? (float*)(base + o_rsort) : nullptr;
        d->flagged_bound = in.mode == MODE_SELECT ? (float*)(base + o_fbound) : nullptr;
        d->colpre = in.ranked ? nullptr : (unsigned char*)(base + o_colpre);
        d->D = (in.ranked || in.mode == MODE_DOM) ? nullptr : (uint32_t*)(base + o_D);
        d->ckeys = in.mode == MODE_DOM ? (float*)(base + o_ckeys) : nullptr;
        d->spos = in.mode == MODE_DOM ? (int32_t*)(base + o_spos) : nullptr;
    }
    return off;
}

// Dominance work items of one problem: column block cb covers row blocks
// [0, min(nrb, 32 (cb + 1))), split into chunks of `chunk` row blocks (a
// power of two from kDomChunkMin to kDomRowChunk).
__host__ __device__ __forceinline__ int64_t dom_items_of_cb(int64_t cb, int64_t nrb, int64_t chunk)
{
    int64_t rbs = nrb < 32 * (cb + 1) ? nrb : 32 * (cb + 1);
    return cdiv(rbs, chunk);
}
// Items of column blocks 0 .. c-1 in closed form: with B = chunk / 32
// column blocks' worth of row blocks per item, block cb < nrb / 32 has
// cb / B + 1 items (its 32 (cb + 1) row blocks in chunks of `chunk`),
// every later block has cdiv(nrb, chunk).
static_assert(kDomChunkMin % 64 == 0 && kDomRowChunk % 64 == 0, "dom_items_prefix assumes an even B");
__host__ __device__ __forceinline__ int64_t dom_items_prefix(int64_t c, int64_t nrb, int64_t chunk)
{
    const int64_t B = chunk / 32;
    const int64_t A = nrb / 32, a = c < A ? c : A, q = a / B, r = a % B;
    return (q + 1) * (B / 2 * q + r) + (c > A ? (c - A) * cdiv(nrb, chunk) : 0);
}
__host__ __device__ inline int64_t dom_items_of(int64_t n2, int64_t chunk)
{
    return dom_items_prefix(cdiv(n2, kColBlock), cdiv(n2, 32), chunk);
}
__host__ __device__ inline bool dom_chunk_ok(int64_t chunk)
{
    return chunk >= kDomChunkMin && chunk <= kDomRowChunk && (chunk & (chunk - 1)) == 0;
}


}  // namespace emo

#ifdef __CUDACC__
namespace emo {

// ------------------------------------------------------------------ basics
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// Order-preserving map float -> uint32 with -0 == +0 (finite inputs).
__device__ __forceinline__ uint32_t float_key(float f)
{
    uint32_t u = __float_as_uint(f + 0.0f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k)
{
    uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
    return __uint_as_float(u);
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v)
{
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *(volatile const int*)p; }

__device__ __forceinline__ void set_status(Scal* sc, int code) { atomicCAS(&sc->status, 0, code); }

// Group of CTAs serving one problem inside a cooperative launch.
struct Group {
    int prob;
    int rank;    // CTA rank inside the group
    int size;    // CTAs in the group
};
// The group of this CTA in the wide (peeling, TensorHypE) or the narrow
// (every other cooperative kernel) assignment; prob = -1 for a CTA that
// serves no problem (groups are capped by the problems' launch shapes), which
// returns at once.
__device__ __forceinline__ Group group_of(const Plan* plan, bool wide)
{
    const int32_t* first = wide ? plan->grp_first : plan->grpn_first;
    Group g;
    int b = blockIdx.x, p = 0;
    while (p + 1 < plan->nprob && first[p + 1] <= b) ++p;
    g.prob = b < first[plan->nprob] ? p : -1;
    g.rank = b - first[p];
    g.size = first[p + 1] - first[p];
    return g;
}

// Barrier over the CTAs of one group with a bounded spin. Returns false (in
// every thread of the CTA) when the problem has failed or the wait ran out.
__device__ inline bool group_sync(Scal* sc, int nblocks, long long budget)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (nblocks > 1) {
            unsigned g = ld_acquire(&sc->bar_gen);
            unsigned arrived = atom_add_acq_rel(&sc->bar_count, 1u);
            if (arrived == (unsigned)nblocks - 1) {
                atomicExch(&sc->bar_count, 0u);
                __threadfence();
                st_release(&sc->bar_gen, g + 1);
            } else {
                long long t0 = clock64();
                while (ld_acquire(&sc->bar_gen) == g) {
                    if (clock64() - t0 > budget) {
                        set_status(sc, EMO_ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
        } else {
            __threadfence();
        }
        if (ld_volatile(&sc->status) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ------------------------------------------------------------ Philox-4x32-10
// Salmon et al., SC'11: ten rounds of two 32x32->64 multiplies with a Weyl
// key schedule. Written from the published definition.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        uint4 n;
        n.x = hi1 ^ c.y ^ k.x;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k.y;
        n.w = lo0;
        c = n;
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}
// Polar angle of a direction from objective axis 1, atan2(|v_2..m|, v_1):
// well conditioned everywhere (unlike acos of a cosine near 0).
__device__ __forceinline__ float polar_angle(const float* v, int m)
{
    float s = 0.0f;
    for (int k = 1; k < m; ++k) s = fmaf(v[k], v[k], s);
    return atan2f(sqrtf(s), v[0]);
}
// Angle from axis 2, by the same formula (the second pivot of the association
// index).
__device__ __forceinline__ float polar_angle2(const float* v, int m)
{
    float s = v[0] * v[0];
    for (int k = 2; k < m; ++k) s = fmaf(v[k], v[k], s);
    return atan2f(sqrtf(s), v[1]);
}

// Niching stream: key = seed, counter = (j, 2 c + tag, generation).
__device__ __forceinline__ uint32_t niche_random(uint64_t seed, uint64_t gen, uint32_t j, uint32_t c, uint32_t tag)
{
    uint4 ctr = make_uint4(j, 2u * c + tag, (uint32_t)gen, (uint32_t)(gen >> 32));
    uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    return philox4x32_10(ctr, key).x;
}

// ------------------------------------------------------------ block scans
template <int NT>
__device__ __forceinline__ int block_exclusive_scan(int v, int* s_warp, int& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < NT / 32 ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    int prefix = (warp > 0 ? s_warp[warp - 1] : 0) + x - v;
    total = s_warp[NT / 32 - 1];
    __syncthreads();
    return prefix;
}

template <int NT>
__device__ __forceinline__ int block_reduce_min(int v, int* s_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int w = lane < NT / 32 ? s_warp[lane] : INT32_MAX;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w = min(w, __shfl_xor_sync(0xffffffffu, w, o));
        if (lane == 0) s_warp[32] = w;
    }
    __syncthreads();
    int r = s_warp[32];
    __syncthreads();
    return r;
}

template <int NT>
__device__ __forceinline__ int block_reduce_sum(int v, int* s_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int w = lane < NT / 32 ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (lane == 0) s_warp[32] = w;
    }
    __syncthreads();
    int r = s_warp[32];
    __syncthreads();
    return r;
}

// ------------------------------------------- group-wide stable compaction
// Writes the positions i in [0, n) with pred(i) true, in ascending order, to
// out[0..count). Every CTA of the group calls it; returns count. Uses
// d.hist[0..G) as scratch; needs group_sync in between (two barriers).
template <typename Pred, typename Emit>
__device__ inline int group_compact(const ProbDev& d, const Group& g, long long budget, int64_t n, Pred pred,
                                    Emit emit, bool& ok)
{
    __shared__ int s_warp[33];
    const int64_t chunk = cdiv(n, g.size);
    const int64_t lo = min(n, chunk * g.rank), hi = min(n, lo + chunk);
    int local = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) local += pred(i) ? 1 : 0;
    local = block_reduce_sum<kCoopThreads>(local, s_warp);
    if (threadIdx.x == 0) d.hist[g.rank] = local;
    ok = group_sync(d.sc, g.size, budget);
    if (!ok) return 0;
    int base = 0, total = 0;
    for (int c = threadIdx.x; c < g.size; c += blockDim.x) {
        int v = ld_volatile(&d.hist[c]);
        if (c < g.rank) base += v;
        total += v;
    }
    base = block_reduce_sum<kCoopThreads>(base, s_warp);
    total = block_reduce_sum<kCoopThreads>(total, s_warp);
    for (int64_t i0 = lo; i0 < hi; i0 += blockDim.x) {
        int64_t i = i0 + threadIdx.x;
        int f = (i < hi && pred(i)) ? 1 : 0;
        int tot;
        int pos = block_exclusive_scan<kCoopThreads>(f, s_warp, tot);
        if (f) emit(base + pos, i);
        base += tot;
    }
    ok = group_sync(d.sc, g.size, budget);
    return total;
}

}  // namespace emo
#endif
