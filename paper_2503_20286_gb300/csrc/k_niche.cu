// Niche counts, candidate lists of the last front, niching and the survivor
// list (Algorithm S.1 lines "Compute the niche counts" to the end; Section
// IV-A "Niche Count Calculation", "Niche Selection" and i_next).
//
// Niching follows Algorithm S.1 level by level: at niche count c = the
// minimum over live references (references with candidates left in the last
// front), every live reference with count c receives one member -- the
// nearest one when c = 0, a uniformly drawn one otherwise -- unless fewer
// picks remain than such references, in which case the references with the
// smallest Philox priorities (x0, j) are served. Random members are drawn
// from the ascending candidate list with a Fenwick tree per list, so a draw
// costs O(log |C_j|).
#include "emo_kernels.cuh"
#include "emo_launch.cuh"
#include "group_radix.cuh"

namespace emo {

// ------------------------------------------------------------ k_csr
__global__ void __launch_bounds__(kCoopThreads, 1) k_csr(Plan* plan)
{
    const Group g = group_of(plan, false);
    if (g.prob < 0) return;  // a CTA beyond every problem's group
    const ProbDev& d = plan->p[g.prob];
    const ProbIn& in = d.in;
    const long long budget = plan->spin_budget;
    if (in.mode != MODE_SELECT || ld_volatile(&d.sc->status) != 0) return;
    Scal* sc = d.sc;
    const int l = ld_volatile(&sc->l);
    const int nS = ld_volatile(&sc->nS);
    const int nr = in.n_r;
    const int64_t n2 = in.n2;
    const int64_t t0 = (int64_t)g.rank * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)g.size * blockDim.x;

    // niche counts of P = {rank < l} (given, summed over the GPUs, for the
    // niching of a split population: they must add up to |P|)
    if (plan->split.kind == SPLIT_NICHE) {
        if (__ldcg(&sc->rho_sum) != (unsigned long long)__ldcg(&sc->nP)) {  // both from earlier launches
            if (g.rank == 0 && threadIdx.x == 0) set_status(sc, EMO_ERR_INVALID_ARG);
            return;
        }
    } else {
        for (int64_t i = t0; i < nS; i += stride) {
            const int v = d.slist[i];
            if (d.rank_o[v] < l) atomicAdd(&d.rho[d.pi[v]], 1);
        }
    }
    // the last front in ascending index order
    bool ok = true;
    int32_t* L0 = d.llist;
    const int nL = group_compact(
        d, g, budget, n2, [&](int64_t i) { return __ldcg(&d.rank_o[i]) == l; },
        [&](int pos, int64_t i) { L0[pos] = (int32_t)i; }, ok);
    if (!ok) return;
    if (in.dbg.rho)
        for (int64_t j = t0; j < nr; j += stride) in.dbg.rho[j] = __ldcg(&d.rho[j]);

    // stable sort of the last front by associated reference
    int bits = 1;
    while ((1ll << bits) < (long long)nr) ++bits;
    int buf = 0;
    __shared__ RadixSmem rsm;
    const int gs = (int)max((int64_t)1, min((int64_t)g.size, cdiv(nL, 4096)));
    for (int shift = 0; shift < bits; shift += kRadixBits) {
        const int32_t* src = d.llist + (int64_t)buf * n2;
        int32_t* dst = d.llist + (int64_t)(buf ^ 1) * n2;
        bool skipped = false;
        auto key = [&](int32_t v) { return (uint32_t)__ldcg(&d.pi[v]); };
        if (!radix_pass(d, g, gs, budget, nL, src, dst, shift, key, skipped, rsm)) return;
        if (!skipped) buf ^= 1;
    }
    const int32_t* L = d.llist + (int64_t)buf * n2;
    if (g.rank == 0 && threadIdx.x == 0) sc->lbuf = buf;

    // CSR offsets: loff[q] = first position of the sorted list whose point is
    // associated with a reference >= q (one binary search per reference)
    for (int64_t q = t0; q <= nr; q += stride) {
        int lo = 0, hi = nL;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (__ldcg(&d.pi[__ldcg(&L[mid])]) < q) lo = mid + 1;
            else hi = mid;
        }
        d.loff[q] = lo;
    }
    if (!group_sync(sc, g.size, budget)) return;
    for (int64_t t = t0; t < nL; t += stride) {
        const int j = __ldcg(&d.pi[__ldcg(&L[t])]);
        const int x = (int)(t - __ldcg(&d.loff[j])) + 1;
        d.fen[t] = x & -x;  // Fenwick tree of an all-present list
    }
    for (int64_t j = t0; j < nr; j += stride) d.lcnt[j] = __ldcg(&d.loff[j + 1]) - __ldcg(&d.loff[j]);
}

// ------------------------------------------------------------ Fenwick helpers
// fen[x - 1] holds the number of present slots in (x - lowbit(x), x].
__device__ __forceinline__ int fen_select(const int32_t* fen, int n, int rank)
{
    int step = 1;
    while (step * 2 <= n) step *= 2;
    int pos = 0;
    for (; step > 0; step >>= 1) {
        if (pos + step <= n && fen[pos + step - 1] <= rank) {
            pos += step;
            rank -= fen[pos - 1];
        }
    }
    return pos;  // 0-based slot of the (rank)-th present element
}
__device__ __forceinline__ void fen_remove(int32_t* fen, int n, int slot)
{
    for (int x = slot + 1; x <= n; x += x & -x) fen[x - 1] -= 1;
}

// ------------------------------------------------------------ threshold select
// The key of rank k (0-based) among the distinct 64-bit keys that the CTAs of
// a group emit, computed by every CTA of the group: a histogram of the top 12
// bits, the bin holding rank k, the keys of that bin collected in d.ekeys, and
// the rank inside the bin (ranked in shared memory, or by a byte-wise radix
// select when the bin is large). The caller clears `hist` and sc->ncol and
// passes a group barrier before the call. for_keys(f) calls f(key) for each
// key of the calling thread's share.
constexpr int kNicheSmallSel = 2048;  // collected keys ranked in shared memory

struct NicheSmem {
    int warp[33];
    unsigned long long keys[kNicheSmallSel];
    int hist[kRadix];
    unsigned long long prefix, thresh;
    int k, bin, kbin;
};

template <class ForKeys>
__device__ bool group_kth_key(const ProbDev& d, const Group& g, long long budget, int k, ForKeys for_keys,
                              NicheSmem& sm, unsigned long long& thresh)
{
    Scal* sc = d.sc;
    int32_t* hist = d.nhist;
    const int tid = threadIdx.x;
    for_keys([&](unsigned long long key) { atomicAdd(&hist[key >> 52], 1); });
    if (!group_sync(sc, g.size, budget)) return false;

    {  // the bin of the key of rank k (each thread scans 8 bins)
        constexpr int PER = kNicheBins / kCoopThreads;
        int h[PER], v = 0;
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            h[e] = __ldcg(&hist[tid * PER + e]);
            v += h[e];
        }
        int tot;
        int pre = block_exclusive_scan<kCoopThreads>(v, sm.warp, tot);
        if (pre <= k && k < pre + v) {
#pragma unroll
            for (int e = 0; e < PER; ++e) {
                if (k < pre + h[e]) {
                    sm.bin = tid * PER + e;
                    sm.kbin = k - pre;
                    break;
                }
                pre += h[e];
            }
        }
        __syncthreads();
    }
    const int bin = sm.bin, kbin = sm.kbin;
    for_keys([&](unsigned long long key) {
        if ((int)(key >> 52) == bin) d.ekeys[atomicAdd(&sc->ncol, 1)] = key;
    });
    if (!group_sync(sc, g.size, budget)) return false;

    const int nc = ld_volatile(&sc->ncol);  // the rank-kbin key among the collected ones
    if (nc <= kNicheSmallSel) {
        for (int i = tid; i < nc; i += blockDim.x) sm.keys[i] = __ldcg(&d.ekeys[i]);
        __syncthreads();
        for (int i = tid; i < nc; i += blockDim.x) {
            const unsigned long long key = sm.keys[i];
            int r = 0;
            for (int q = 0; q < nc; ++q) r += sm.keys[q] < key ? 1 : 0;
            if (r == kbin) sm.thresh = key;
        }
        __syncthreads();
    } else {  // many keys in one bin: byte-wise radix select
        if (tid == 0) {
            sm.prefix = 0ull;
            sm.k = kbin;
        }
        unsigned long long mask = 0ull;
        for (int shift = 56; shift >= 0; shift -= 8) {
            for (int i = tid; i < kRadix; i += blockDim.x) sm.hist[i] = 0;
            __syncthreads();
            const unsigned long long prefix = sm.prefix;
            for (int e = tid; e < nc; e += blockDim.x) {
                const unsigned long long key = __ldcg(&d.ekeys[e]);
                if ((key & mask) == prefix) atomicAdd(&sm.hist[(key >> shift) & 0xFF], 1);
            }
            __syncthreads();
            if (tid == 0) {
                int acc = 0, dg = 0;
                for (; dg < kRadix; ++dg) {
                    if (acc + sm.hist[dg] > sm.k) break;
                    acc += sm.hist[dg];
                }
                sm.k -= acc;
                sm.prefix = prefix | ((unsigned long long)dg << shift);
            }
            mask |= 0xFFull << shift;
            __syncthreads();
        }
        if (tid == 0) sm.thresh = sm.prefix;
        __syncthreads();
    }
    thresh = sm.thresh;
    __syncthreads();
    return true;
}

// Nearest member of reference j's candidate list (d, then index).
__device__ __forceinline__ int niche_nearest(const ProbDev& d, const int32_t* L, int off, int full)
{
    int pos = 0;
    double bd = d.d64[L[off]];
    int bi = L[off];
    for (int t = 1; t < full; ++t) {
        const int v = L[off + t];
        const double dv = d.d64[v];
        if (dv < bd || (dv == bd && v < bi)) {
            bd = dv;
            bi = v;
            pos = t;
        }
    }
    return pos;
}

// ------------------------------------------------------------ k_niche
// One cooperative launch; the references of a problem are spread over its CTA
// group, and a reference's list, Fenwick tree and counts are touched by one
// thread only. Per level:
//   (A) every CTA: the minimum niche count over its live references and how
//       many hold it; the histogram of the threshold select is cleared;
//   (B) every CTA: the group's minimum c and its count from the partials; if
//       the level cannot be served in full, the priority (x0, j) of rank
//       remaining - 1 among the level's references (group_kth_key);
//   (C) every CTA: the picks of its references.
// Every phase ends with a bounded group barrier.
__device__ __forceinline__ unsigned long long niche_key(uint64_t seed, uint64_t gen, int64_t j, int c)
{
    return ((unsigned long long)niche_random(seed, gen, (uint32_t)j, (uint32_t)c, 0u) << 32) | (unsigned)j;
}

constexpr int kNicheDirectLevels = 3;  // levels served one at a time before the bulk form

// Pick of reference j at level c (the level form's step): its nearest
// candidate at level 0 (the list is untouched then), else the candidate of
// rank (u |C_j|) >> 32 among the remaining ones (Fenwick tree over the list).
__device__ __forceinline__ void niche_pick(const ProbDev& d, const int32_t* L, uint64_t seed, uint64_t gen, int64_t j,
                                           int c, int len)
{
    const int off = d.loff[j], full = d.loff[j + 1] - off;
    int pos;
    if (c == 0) {
        pos = niche_nearest(d, L, off, full);
    } else {
        const uint32_t u = niche_random(seed, gen, (uint32_t)j, (uint32_t)c, 1u);
        const int rank = (int)(((unsigned long long)u * (unsigned long long)len) >> 32);
        pos = fen_select(d.fen + off, full, rank);
    }
    d.flag[L[off + pos]] = 1;
    fen_remove(d.fen + off, full, pos);
}

// The picks of one reference by a whole warp (lists of at most
// kWarpPickMax members): the list's remaining members as bit masks in
// registers (lane i holds list positions [32 R i, 32 R (i + 1)), R words),
// rebuilt from the survivor flags; each pick finds the member of rank
// (u len) >> 32 among the remaining ones by a warp scan of the lanes' counts
// and a bit select inside the lane that holds it. The same member as
// niche_pick (nearest at level 0, else the same rank among the remaining
// members in list order) and the same draws, without the Fenwick tree's
// dependent loads. Returns false on an inconsistent count.
constexpr int kWarpPickWords = 4;
constexpr int kWarpPickMax = 32 * 32 * kWarpPickWords;

__device__ __forceinline__ int select_bit(uint32_t w, int k)  // position of the k-th set bit
{
    int bit = 0;
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) {
        const int c = __popc(w & ((1u << sh) - 1u));
        if (k >= c) {
            k -= c;
            w >>= sh;
            bit += sh;
        }
    }
    return bit;
}

__device__ bool warp_picks(const ProbDev& d, const int32_t* L, uint64_t seed, uint64_t gen, int64_t j, int r, int n,
                           int take, int lane)
{
    constexpr int R = kWarpPickWords;
    const int off = d.loff[j], full = d.loff[j + 1] - off;
    uint32_t mask[R];
#pragma unroll
    for (int q = 0; q < R; ++q) mask[q] = 0u;
    for (int base = 0; base < full; base += 32) {  // coalesced: word base / 32 of the list
        const int pos = base + lane;
        const bool live = pos < full && __ldcg(&d.flag[L[off + pos]]) == 0;
        const uint32_t bal = __ballot_sync(0xffffffffu, live);
        const int word = base >> 5, owner = word / R, wq = word - owner * R;
#pragma unroll
        for (int q = 0; q < R; ++q)
            if (lane == owner && q == wq) mask[q] = bal;
    }
    for (int t = 0; t < take; ++t) {
        const int c = r + t, len = n - t;
        int pos;
        if (c == 0) {  // nearest member (distance, then caller index); the list is whole at level 0
            double bd = INFINITY;
            int bi = INT32_MAX, bp = -1;
            for (int q = lane; q < full; q += 32) {
                const int v = L[off + q];
                const double dv = d.d64[v];
                if (dv < bd || (dv == bd && v < bi)) { bd = dv; bi = v; bp = q; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double od = __shfl_xor_sync(0xffffffffu, bd, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                const int op = __shfl_xor_sync(0xffffffffu, bp, o);
                if (od < bd || (od == bd && oi < bi)) { bd = od; bi = oi; bp = op; }
            }
            pos = bp;
        } else {
            const uint32_t u = niche_random(seed, gen, (uint32_t)j, (uint32_t)c, 1u);
            const int rank = (int)(((unsigned long long)u * (unsigned long long)len) >> 32);
            int cnt = 0;
#pragma unroll
            for (int q = 0; q < R; ++q) cnt += __popc(mask[q]);
            int inc = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            const unsigned hit = __ballot_sync(0xffffffffu, inc > rank);
            if (!hit) return false;  // fewer remaining members than len
            const int owner = __ffs(hit) - 1;
            int k = rank - (inc - cnt);  // rank inside the owner lane (valid there)
            int p = 0;
            if (lane == owner) {
                int wq = 0;
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int cq = __popc(mask[q]);
                    if (wq == q && k >= cq) { k -= cq; ++wq; }
                }
                uint32_t w = 0u;
#pragma unroll
                for (int q = 0; q < R; ++q)
                    if (q == wq) w = mask[q];
                p = (owner * R + wq) * 32 + select_bit(w, k);
            }
            pos = __shfl_sync(0xffffffffu, p, owner);
        }
        if (pos < 0 || pos >= full) return false;
        const int word = pos >> 5, owner = word / R, wq = word - owner * R;
#pragma unroll
        for (int q = 0; q < R; ++q)
            if (lane == owner && q == wq) mask[q] &= ~(1u << (pos & 31));
        if (lane == 0) d.flag[L[off + pos]] = 1;
    }
    return true;
}

// The remaining picks in bulk (water-filling). From the current niche counts
// rho_j and live list lengths n_j, the level form serves reference j at the
// levels c = rho_j .. rho_j + n_j - 1 (one member per level while its list
// lasts). With ne(c) = #{j : rho_j <= c < rho_j + n_j} references at level c
// and P(c) = sum_{c' < c} ne(c') picks before it, the level form stops at the
// smallest c* with P(c*) + ne(c*) >= remaining and there serves only the
// remaining - P(c*) references of smallest priority. Each reference then
// makes its picks itself, in level order, with the level form's draws, so the
// picks are the same. The levels are histogrammed over a window of at most
// kNicheBins values from c_lo (references whose interval starts beyond it
// add nothing inside it); when c* lies beyond the window, every level of the
// window is served in full, `remaining` drops by their picks and `handled`
// is false (the caller goes on from the next level); otherwise remaining
// becomes 0 and `handled` true.
__device__ bool niche_bulk(const ProbDev& d, const Group& g, long long budget, int& remaining, NicheSmem& sm,
                           const int32_t* L, int& levels, bool& handled)
{
    Scal* sc = d.sc;
    const ProbIn& in = d.in;
    const int tid = threadIdx.x;
    const int nr = in.n_r;
    const uint64_t seed = in.seed, gen = in.gen;
    const int64_t t0 = (int64_t)g.rank * blockDim.x + tid;
    const int64_t stride = (int64_t)g.size * blockDim.x;
    int32_t* hist = d.nhist;
    unsigned long long* part = reinterpret_cast<unsigned long long*>(d.nhist + kNicheBins);
    __shared__ int s_cstar, s_pstar, s_nestar, s_lev, s_pwin;
    handled = false;

    // (1) the span of levels [c_lo, c_end) of the live references
    int cmin = INT32_MAX, cend = 0;
    for (int64_t j = t0; j < nr; j += stride) {
        const int n = __ldcg(&d.lcnt[j]);
        if (n > 0) {
            const int r = __ldcg(&d.rho[j]);
            cmin = min(cmin, r);
            cend = max(cend, r + n);
        }
    }
    const int bmin = block_reduce_min<kCoopThreads>(cmin, sm.warp);
    const int bend = -block_reduce_min<kCoopThreads>(-cend, sm.warp);
    if (tid == 0) part[g.rank] = ((unsigned long long)(unsigned)bmin << 32) | (unsigned)bend;
    for (int64_t b = t0; b < kNicheBins; b += stride) hist[b] = 0;
    if (!group_sync(sc, g.size, budget)) return false;
    int lm = INT32_MAX, le = 0;
    for (int r = tid; r < g.size; r += blockDim.x) {
        const unsigned long long v = __ldcg(&part[r]);
        lm = min(lm, (int)(v >> 32));
        le = max(le, (int)(v & 0xFFFFFFFFull));
    }
    const int c_lo = block_reduce_min<kCoopThreads>(lm, sm.warp);
    const int c_end = -block_reduce_min<kCoopThreads>(-le, sm.warp);
    if (c_lo == INT32_MAX) {  // no live reference although picks remain
        if (g.rank == 0 && tid == 0) set_status(sc, EMO_ERR_INVALID_ARG);
        return false;
    }
    const bool windowed = c_end - c_lo > kNicheBins;
    const int R = windowed ? kNicheBins : c_end - c_lo;

    // (2) ne(c) as a difference array over the window
    for (int64_t j = t0; j < nr; j += stride) {
        const int n = __ldcg(&d.lcnt[j]);
        if (n > 0) {
            const int r = __ldcg(&d.rho[j]) - c_lo;
            if (r < R) atomicAdd(&hist[r], 1);
            if (r + n < R) atomicAdd(&hist[r + n], -1);
        }
    }
    if (!group_sync(sc, g.size, budget)) return false;

    // (3) every CTA: ne(c), P(c), c*, and the levels served up to c*
    {
        constexpr int PER = kNicheBins / kCoopThreads;
        int dv[PER], run = 0;
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const int c = tid * PER + e;
            dv[e] = c < R ? __ldcg(&hist[c]) : 0;
            run += dv[e];
        }
        int tot;
        int pre = block_exclusive_scan<kCoopThreads>(run, sm.warp, tot);  // ne at this thread's first level
        int ne[PER], nsum = 0;
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            pre += dv[e];
            ne[e] = pre;
            nsum += pre;
        }
        int ppre = block_exclusive_scan<kCoopThreads>(nsum, sm.warp, tot);  // P at this thread's first level
        if (tid == 0) {
            s_cstar = INT32_MAX;
            s_pwin = tot;  // picks of every level of the window
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const int c = tid * PER + e;
            if (c < R && ne[e] > 0 && ppre + ne[e] >= remaining) atomicMin(&s_cstar, c);
            ppre += ne[e];
        }
        __syncthreads();
        const int cs = s_cstar;
        int lev = 0;
        ppre -= nsum;
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const int c = tid * PER + e;
            if (c == cs) {
                s_pstar = ppre;
                s_nestar = ne[e];
            }
            if (c <= cs && c < R && ne[e] > 0) ++lev;
            ppre += ne[e];
        }
        lev = block_reduce_sum<kCoopThreads>(lev, sm.warp);
        if (tid == 0) s_lev = lev;
        __syncthreads();
    }
    const int cstar = s_cstar;
    const bool found = cstar != INT32_MAX;
    if (!found && !windowed) {  // fewer live candidates than picks: inconsistent lists
        if (g.rank == 0 && tid == 0) set_status(sc, EMO_ERR_INVALID_ARG);
        return false;
    }
    // not found: every level below c_lo + R in full, none at c_star itself
    const int c_star = found ? c_lo + cstar : c_lo + R;
    const int rem = found ? remaining - s_pstar : 0, ne_star = found ? s_nestar : 0;
    const bool all = ne_star <= rem;
    unsigned long long thresh = ~0ull;
    if (!all) {  // the rem references of smallest priority among those at level c*
        if (!group_sync(sc, g.size, budget)) return false;  // every CTA is done with the histogram
        for (int64_t b = t0; b < kNicheBins; b += stride) hist[b] = 0;
        if (g.rank == 0 && tid == 0) sc->ncol = 0;
        if (!group_sync(sc, g.size, budget)) return false;
        auto level_keys = [&](auto&& f) {
            for (int64_t j = t0; j < nr; j += stride) {
                const int n = __ldcg(&d.lcnt[j]), r = __ldcg(&d.rho[j]);
                if (n > 0 && r <= c_star && c_star < r + n) f(niche_key(seed, gen, j, c_star));
            }
        };
        if (!group_kth_key(d, g, budget, rem - 1, level_keys, sm, thresh)) return false;
    }

    // (4) the picks of every reference, in level order; references dealt
    // round-robin over the CTAs (each walk is sequential: spread over SMs):
    // lists of at most kWarpPickMax members one warp each, longer lists one
    // thread each (Fenwick tree)
    auto take_of = [&](int64_t j, int n, int r) {
        int take = r < c_star ? min(c_star, r + n) - r : 0;
        if (found && r <= c_star && c_star < r + n && (all || niche_key(seed, gen, j, c_star) <= thresh)) ++take;
        return take;
    };
    {
        const int lane = tid & 31, nw = blockDim.x >> 5;
        for (int64_t jj = tid >> 5;; jj += nw) {
            const int64_t j = jj * g.size + g.rank;
            if (j >= nr) break;
            const int n = d.lcnt[j];
            if (n <= 0 || d.loff[j + 1] - d.loff[j] > kWarpPickMax) continue;
            const int r = d.rho[j];
            const int take = take_of(j, n, r);
            if (take > 0 && !warp_picks(d, L, seed, gen, j, r, n, take, lane)) {
                if (lane == 0) set_status(sc, EMO_ERR_INVALID_ARG);
                continue;
            }
            __syncwarp();
            if (lane == 0) {
                d.lcnt[j] = n - take;
                d.rho[j] = r + take;
            }
        }
    }
    for (int64_t jj = tid;; jj += blockDim.x) {
        const int64_t j = jj * g.size + g.rank;
        if (j >= nr) break;
        const int n = d.lcnt[j];
        if (n <= 0 || d.loff[j + 1] - d.loff[j] <= kWarpPickMax) continue;
        const int r = d.rho[j];
        const int take = take_of(j, n, r);
        for (int t = 0; t < take; ++t) niche_pick(d, L, seed, gen, j, r + t, n - t);
        d.lcnt[j] = n - take;
        d.rho[j] = r + take;
    }
    if (!group_sync(sc, g.size, budget)) return false;
    levels += s_lev;
    handled = found;
    remaining = found ? 0 : remaining - s_pwin;
    return true;
}

__global__ void __launch_bounds__(kCoopThreads, 1) k_niche(Plan* plan)
{
    __shared__ NicheSmem sm;
    const Group g = group_of(plan, false);
    if (g.prob < 0) return;  // a CTA beyond every problem's group
    const ProbDev& d = plan->p[g.prob];
    const ProbIn& in = d.in;
    const long long budget = plan->spin_budget;
    if (in.mode != MODE_SELECT || in.niche != EMO_NICHE_EXACT || ld_volatile(&d.sc->status) != 0) return;
    Scal* sc = d.sc;
    const int tid = threadIdx.x;
    const int nr = in.n_r;
    const int nP = ld_volatile(&sc->nP), nL = ld_volatile(&sc->nL);
    const int K = (int)(in.n_keep - nP);
    const int32_t* L = d.llist + (int64_t)ld_volatile(&sc->lbuf) * in.n2;
    const uint64_t seed = in.seed, gen = in.gen;
    const int64_t t0 = (int64_t)g.rank * blockDim.x + tid;
    const int64_t stride = (int64_t)g.size * blockDim.x;
    int32_t* hist = d.nhist;
    unsigned long long* part = reinterpret_cast<unsigned long long*>(d.nhist + kNicheBins);

    if (K == nL) {  // the whole last front survives
        for (int64_t t = t0; t < nL; t += stride) d.flag[L[t]] = 1;
        if (g.rank == 0 && tid == 0) sc->levels = 0;
        return;
    }
    int remaining = K, levels = 0;
    while (remaining > 0) {
        // (A) this CTA's minimum niche count over live references, and its count
        int cmin = INT32_MAX, cnt = 0;
        for (int64_t j = t0; j < nr; j += stride) {
            if (__ldcg(&d.lcnt[j]) > 0) {
                const int r = __ldcg(&d.rho[j]);
                if (r < cmin) {
                    cmin = r;
                    cnt = 1;
                } else if (r == cmin) {
                    ++cnt;
                }
            }
        }
        const int bmin = block_reduce_min<kCoopThreads>(cmin, sm.warp);
        const int bcnt = block_reduce_sum<kCoopThreads>(cmin == bmin ? cnt : 0, sm.warp);
        if (tid == 0) part[g.rank] = ((unsigned long long)(unsigned)bmin << 32) | (unsigned)bcnt;
        for (int64_t b = t0; b < kNicheBins; b += stride) hist[b] = 0;
        if (g.rank == 0 && tid == 0) sc->ncol = 0;
        if (!group_sync(sc, g.size, budget)) return;

        // (B) the level: minimum c over the group and the number of references holding it
        int lm = INT32_MAX;
        for (int r = tid; r < g.size; r += blockDim.x) lm = min(lm, (int)(__ldcg(&part[r]) >> 32));
        const int c = block_reduce_min<kCoopThreads>(lm, sm.warp);
        if (c == INT32_MAX) {  // no live reference although picks remain
            if (g.rank == 0 && tid == 0) set_status(sc, EMO_ERR_INVALID_ARG);
            return;
        }
        int lc = 0;
        for (int r = tid; r < g.size; r += blockDim.x) {
            const unsigned long long v = __ldcg(&part[r]);
            if ((int)(v >> 32) == c) lc += (int)(v & 0xFFFFFFFFull);
        }
        const int ne = block_reduce_sum<kCoopThreads>(lc, sm.warp);
        const bool all = ne <= remaining;
        unsigned long long thresh = ~0ull;
        if (!all) {  // keep the `remaining` references with the smallest priorities
            auto level_keys = [&](auto&& f) {
                for (int64_t j = t0; j < nr; j += stride)
                    if (__ldcg(&d.lcnt[j]) > 0 && __ldcg(&d.rho[j]) == c) f(niche_key(seed, gen, j, c));
            };
            if (!group_kth_key(d, g, budget, remaining - 1, level_keys, sm, thresh)) return;
        }

        // (C) picks: every level reference (all) or those with priority <= thresh;
        // references dealt round-robin over the CTAs
        for (int64_t jj = tid;; jj += blockDim.x) {
            const int64_t j = jj * g.size + g.rank;
            if (j >= nr) break;
            const int len = d.lcnt[j];
            if (len <= 0 || d.rho[j] != c) continue;
            if (!all && niche_key(seed, gen, j, c) > thresh) continue;
            const int off = d.loff[j], full = d.loff[j + 1] - off;
            int pos;
            if (c == 0) {  // nearest member; the list is untouched at level 0
                pos = niche_nearest(d, L, off, full);
            } else {
                const uint32_t u = niche_random(seed, gen, (uint32_t)j, (uint32_t)c, 1u);
                const int rank = (int)(((unsigned long long)u * (unsigned long long)len) >> 32);
                pos = fen_select(d.fen + off, full, rank);
            }
            d.flag[L[off + pos]] = 1;
            fen_remove(d.fen + off, full, pos);
            d.lcnt[j] = len - 1;
            d.rho[j] = c + 1;
        }
        if (!group_sync(sc, g.size, budget)) return;
        remaining -= all ? ne : remaining;
        ++levels;
        if (remaining > 0 && levels >= kNicheDirectLevels) {  // the rest in bulk when the span allows
            bool handled = false;
            if (!niche_bulk(d, g, budget, remaining, sm, L, levels, handled)) return;
        }
    }
    if (g.rank == 0 && tid == 0) sc->levels = levels;
}

// ------------------------------------------------------------ k_niche_oneshot
// The tensorized one-shot niche selection (Algorithm S.4) with Update-Rank
// (Algorithm S.6), as one cooperative launch over the problem's CTA group:
//   (A) every reference with niche count 0 and at least one last-front
//       candidate takes its nearest candidate (d, then index); the taken
//       points are counted (n_sel); the select histogram is cleared;
//   (B) n_dif = K - n_sel. n_dif > 0: the n_dif remaining last-front points
//       with the smallest add keys are added; n_dif < 0: the -n_dif taken
//       points with the smallest drop keys are dropped. The keys, Philox x0 of
//       counter (i, 0xFFFFFFF0 + tag, generation) with the index below, stand
//       for the paper's shuffled input order.
__device__ __forceinline__ unsigned long long oneshot_key(uint64_t seed, uint64_t gen, int64_t i, uint32_t tag)
{
    const uint4 ctr = make_uint4((uint32_t)i, 0xFFFFFFF0u + tag, (uint32_t)gen, (uint32_t)(gen >> 32));
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    return ((unsigned long long)philox4x32_10(ctr, key).x << 32) | (unsigned)i;
}

__global__ void __launch_bounds__(kCoopThreads, 1) k_niche_oneshot(Plan* plan)
{
    __shared__ NicheSmem sm;
    const Group g = group_of(plan, false);
    if (g.prob < 0) return;  // a CTA beyond every problem's group
    const ProbDev& d = plan->p[g.prob];
    const ProbIn& in = d.in;
    const long long budget = plan->spin_budget;
    if (in.mode != MODE_SELECT || in.niche != EMO_NICHE_ONESHOT || ld_volatile(&d.sc->status) != 0) return;
    Scal* sc = d.sc;
    const int tid = threadIdx.x;
    const int nr = in.n_r;
    const int nP = ld_volatile(&sc->nP), nL = ld_volatile(&sc->nL);
    const int K = (int)(in.n_keep - nP);
    const int32_t* L = d.llist + (int64_t)ld_volatile(&sc->lbuf) * in.n2;
    const uint64_t seed = in.seed, gen = in.gen;
    const int64_t t0 = (int64_t)g.rank * blockDim.x + tid;
    const int64_t stride = (int64_t)g.size * blockDim.x;

    // (A) nearest candidate of every empty niche
    int taken = 0;
    for (int64_t j = t0; j < nr; j += stride) {
        const int len = d.lcnt[j];
        if (len <= 0 || d.rho[j] != 0) continue;
        const int off = d.loff[j];
        d.flag[L[off + niche_nearest(d, L, off, len)]] = 1;
        ++taken;
    }
    taken = block_reduce_sum<kCoopThreads>(taken, sm.warp);
    if (tid == 0 && taken) atomicAdd(&sc->nsel, taken);
    for (int64_t b = t0; b < kNicheBins; b += stride) d.nhist[b] = 0;
    if (g.rank == 0 && tid == 0) {
        sc->ncol = 0;
        sc->levels = 1;
    }
    if (!group_sync(sc, g.size, budget)) return;

    // (B) Update-Rank: add or drop in Philox order
    const int n_dif = K - ld_volatile(&sc->nsel);
    if (n_dif == 0) return;
    const uint32_t tag = n_dif > 0 ? 1u : 2u;
    const int want = n_dif > 0 ? 0 : 1;  // add from the untaken points, drop from the taken ones
    auto keys = [&](auto&& f) {
        for (int64_t t = t0; t < nL; t += stride) {
            const int i = __ldcg(&L[t]);
            if (__ldcg(&d.flag[i]) == want) f(oneshot_key(seed, gen, i, tag));
        }
    };
    unsigned long long thresh;
    if (!group_kth_key(d, g, budget, (n_dif > 0 ? n_dif : -n_dif) - 1, keys, sm, thresh)) return;
    for (int64_t t = t0; t < nL; t += stride) {
        const int i = __ldcg(&L[t]);
        if (__ldcg(&d.flag[i]) == want && oneshot_key(seed, gen, i, tag) <= thresh) d.flag[i] = 1 - want;
    }
}

// ------------------------------------------------------------ k_finish
__device__ int32_t g_sticky_status;  // first failure since the last read (per device)

cudaError_t sticky_status(cudaStream_t s, int32_t* out, bool clear)
{
    cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_sticky_status, sizeof(int32_t), 0, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && clear) {
        static const int32_t zero = 0;
        e = cudaMemcpyToSymbolAsync(g_sticky_status, &zero, sizeof(int32_t), 0, cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

__global__ void k_sticky_merge(const int32_t* status)
{
    const int32_t st = *status;
    if (st != 0) atomicCAS(&g_sticky_status, 0, st);
}

cudaError_t sticky_merge(const int32_t* status, cudaStream_t s)
{
    k_sticky_merge<<<1, 1, 0, s>>>(status);
    return cudaGetLastError();
}

// Survivors (ascending indices of P and the picked members), the info block
// and the optional intermediates.
__global__ void __launch_bounds__(kCoopThreads, 1) k_finish(Plan* plan)
{
    const Group g = group_of(plan, false);
    if (g.prob < 0) return;  // a CTA beyond every problem's group
    const ProbDev& d = plan->p[g.prob];
    const ProbIn& in = d.in;
    Scal* sc = d.sc;
    const long long budget = plan->spin_budget;
    const int tid = threadIdx.x;
    const int m = in.m;
    const int64_t n2 = in.n2;
    const int64_t t0 = (int64_t)g.rank * blockDim.x + tid;
    const int64_t stride = (int64_t)g.size * blockDim.x;
    bool ok = ld_volatile(&sc->status) == 0;
    int ns = 0;
    // (the association of a split population has no survivors: its outputs
    // were written by k_assoc_out)
    if (ok && (in.mode == MODE_SELECT || in.mode == MODE_HYPE) && plan->split.kind != SPLIT_ASSOC) {
        const int l = sc->l;
        ns = group_compact(
            d, g, budget, n2, [&](int64_t i) { return __ldcg(&d.rank_o[i]) < l || __ldcg(&d.flag[i]) != 0; },
            [&](int pos, int64_t i) {
                if (pos < in.n_keep) in.survivors[pos] = (int32_t)i;
            },
            ok);
        if (ok && g.rank == 0 && tid == 0 && ns != in.n_keep) set_status(sc, EMO_ERR_INVALID_ARG);
        // intermediates
        const emo_select_debug& dbg = in.dbg;
        for (int64_t i = t0; i < n2; i += stride) {
            const int r = __ldcg(&d.rank_o[i]);
            const bool inS = r <= l;
            if (dbg.rank) dbg.rank[i] = r;
            if (dbg.pi) dbg.pi[i] = inS ? __ldcg(&d.pi[i]) : -1;
            if (dbg.dist) dbg.dist[i] = inS ? __ldcg(&d.d64[i]) : (double)NAN;
            if (dbg.picked) dbg.picked[i] = (uint8_t)(__ldcg(&d.flag[i]) != 0 && r == l);
            if (dbg.fnorm)
                for (int k = 0; k < m; ++k)
                    dbg.fnorm[i * m + k] = inS ? (in.F[i * m + k] - sc->z[k]) * sc->inv_a32[k] : NAN;
        }
        if (g.rank == 0 && tid < m) {
            if (dbg.z) dbg.z[tid] = sc->z[tid];
            if (dbg.a) dbg.a[tid] = sc->a[tid];
            if (dbg.extreme) dbg.extreme[tid] = sc->ext[tid];
        }
    }
    if (g.rank == 0 && tid == 0) {
        const int st = ld_volatile(&sc->status);
        if (st) {
            atomicCAS(&plan->status, 0, st);
            atomicCAS(&g_sticky_status, 0, st);
        }
        if (in.info) {
            emo_select_info info;
            info.status = st;
            info.last_rank = sc->l;
            info.n_before = sc->nP;
            info.n_last = sc->nL;
            info.fallback_used = sc->fallback;
            info.n_recheck = sc->nflag;
            info.n_fronts = sc->nfronts;
            info.n_levels = sc->levels;
            *in.info = info;
        }
    }
}

}  // namespace emo
