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
#include "group_radix.cuh"

namespace emo {

// ------------------------------------------------------------ k_csr
__global__ void __launch_bounds__(kCoopThreads, 1) k_csr(Plan* plan)
{
    const Group g = group_of(plan);
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

    // niche counts of P = {rank < l}
    for (int64_t i = t0; i < nS; i += stride) {
        const int v = d.slist[i];
        if (d.rank_o[v] < l) atomicAdd(&d.rho[d.pi[v]], 1);
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

    // CSR offsets from the run boundaries of the sorted list
    for (int64_t t = t0; t < nL; t += stride) {
        const int j = __ldcg(&d.pi[__ldcg(&L[t])]);
        const int jp = t > 0 ? __ldcg(&d.pi[__ldcg(&L[t - 1])]) : -1;
        for (int q = jp + 1; q <= j; ++q) d.loff[q] = (int32_t)t;
        if (t == nL - 1)
            for (int q = j + 1; q <= nr; ++q) d.loff[q] = nL;
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

// ------------------------------------------------------------ k_niche
// One cooperative launch; the references of a problem are spread over its CTA
// group, and a reference's list, Fenwick tree and counts are touched by one
// thread only. Per level:
//   (A) every CTA: the minimum niche count over its live references and how
//       many hold it; the histogram of (C) is cleared;
//   (B) every CTA: the group's minimum c and its count from the partials; if
//       the level cannot be served in full, the histogram of the top 12 bits
//       of the level's priorities (x0, j);
//   (C) every CTA: the bin holding the `remaining`-th smallest priority; the
//       keys of that bin are collected;
//   (D) every CTA: the threshold (that priority, selected from the collected
//       keys) and the picks of its references.
// Every phase ends with a bounded group barrier; levels served in full skip
// (B)'s histogram and (C).
constexpr int kNicheSmallSel = 2048;  // collected keys ranked in shared memory

__device__ __forceinline__ unsigned long long niche_key(uint64_t seed, uint64_t gen, int64_t j, int c)
{
    return ((unsigned long long)niche_random(seed, gen, (uint32_t)j, (uint32_t)c, 0u) << 32) | (unsigned)j;
}

__global__ void __launch_bounds__(kCoopThreads, 1) k_niche(Plan* plan)
{
    __shared__ int s_warp[33];
    __shared__ unsigned long long s_keys[kNicheSmallSel];
    __shared__ int s_hist[kRadix];
    __shared__ unsigned long long s_prefix, s_thresh;
    __shared__ int s_k, s_bin, s_kbin;
    const Group g = group_of(plan);
    const ProbDev& d = plan->p[g.prob];
    const ProbIn& in = d.in;
    const long long budget = plan->spin_budget;
    if (in.mode != MODE_SELECT || ld_volatile(&d.sc->status) != 0) return;
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
        const int bmin = block_reduce_min<kCoopThreads>(cmin, s_warp);
        const int bcnt = block_reduce_sum<kCoopThreads>(cmin == bmin ? cnt : 0, s_warp);
        if (tid == 0) part[g.rank] = ((unsigned long long)(unsigned)bmin << 32) | (unsigned)bcnt;
        for (int64_t b = t0; b < kNicheBins; b += stride) hist[b] = 0;
        if (g.rank == 0 && tid == 0) sc->ncol = 0;
        if (!group_sync(sc, g.size, budget)) return;

        // (B) the level: minimum c over the group and the number of references holding it
        int lm = INT32_MAX;
        for (int r = tid; r < g.size; r += blockDim.x) lm = min(lm, (int)(__ldcg(&part[r]) >> 32));
        const int c = block_reduce_min<kCoopThreads>(lm, s_warp);
        if (c == INT32_MAX) {  // no live reference although picks remain
            if (g.rank == 0 && tid == 0) set_status(sc, EMO_ERR_INVALID_ARG);
            return;
        }
        int lc = 0;
        for (int r = tid; r < g.size; r += blockDim.x) {
            const unsigned long long v = __ldcg(&part[r]);
            if ((int)(v >> 32) == c) lc += (int)(v & 0xFFFFFFFFull);
        }
        const int ne = block_reduce_sum<kCoopThreads>(lc, s_warp);
        const bool all = ne <= remaining;
        unsigned long long thresh = ~0ull;
        if (!all) {
            // priorities of the level's references; keep the `remaining` smallest
            for (int64_t j = t0; j < nr; j += stride)
                if (__ldcg(&d.lcnt[j]) > 0 && __ldcg(&d.rho[j]) == c)
                    atomicAdd(&hist[niche_key(seed, gen, j, c) >> 52], 1);
            if (!group_sync(sc, g.size, budget)) return;

            // (C) the bin of the priority of rank remaining - 1 (each thread scans 8 bins)
            {
                constexpr int PER = kNicheBins / kCoopThreads;
                int h[PER], v = 0;
#pragma unroll
                for (int e = 0; e < PER; ++e) {
                    h[e] = __ldcg(&hist[tid * PER + e]);
                    v += h[e];
                }
                int tot;
                int pre = block_exclusive_scan<kCoopThreads>(v, s_warp, tot);
                const int k = remaining - 1;
                if (pre <= k && k < pre + v) {
#pragma unroll
                    for (int e = 0; e < PER; ++e) {
                        if (k < pre + h[e]) {
                            s_bin = tid * PER + e;
                            s_kbin = k - pre;
                            break;
                        }
                        pre += h[e];
                    }
                }
                __syncthreads();
            }
            const int bin = s_bin, kbin = s_kbin;
            for (int64_t j = t0; j < nr; j += stride)
                if (__ldcg(&d.lcnt[j]) > 0 && __ldcg(&d.rho[j]) == c) {
                    const unsigned long long key = niche_key(seed, gen, j, c);
                    if ((int)(key >> 52) == bin) d.ekeys[atomicAdd(&sc->ncol, 1)] = key;
                }
            if (!group_sync(sc, g.size, budget)) return;

            // (D) the kbin-th smallest collected key (keys are distinct: j is in the low bits)
            const int nc = ld_volatile(&sc->ncol);
            if (nc <= kNicheSmallSel) {
                for (int i = tid; i < nc; i += blockDim.x) s_keys[i] = __ldcg(&d.ekeys[i]);
                __syncthreads();
                for (int i = tid; i < nc; i += blockDim.x) {
                    const unsigned long long key = s_keys[i];
                    int r = 0;
                    for (int q = 0; q < nc; ++q) r += s_keys[q] < key ? 1 : 0;
                    if (r == kbin) s_thresh = key;
                }
                __syncthreads();
            } else {  // many keys in one bin: byte-wise radix select
                if (tid == 0) {
                    s_prefix = 0ull;
                    s_k = kbin;
                }
                unsigned long long mask = 0ull;
                for (int shift = 56; shift >= 0; shift -= 8) {
                    for (int i = tid; i < kRadix; i += blockDim.x) s_hist[i] = 0;
                    __syncthreads();
                    const unsigned long long prefix = s_prefix;
                    for (int e = tid; e < nc; e += blockDim.x) {
                        const unsigned long long key = __ldcg(&d.ekeys[e]);
                        if ((key & mask) == prefix) atomicAdd(&s_hist[(key >> shift) & 0xFF], 1);
                    }
                    __syncthreads();
                    if (tid == 0) {
                        int acc = 0, dg = 0;
                        for (; dg < kRadix; ++dg) {
                            if (acc + s_hist[dg] > s_k) break;
                            acc += s_hist[dg];
                        }
                        s_k -= acc;
                        s_prefix = prefix | ((unsigned long long)dg << shift);
                    }
                    mask |= 0xFFull << shift;
                    __syncthreads();
                }
                if (tid == 0) s_thresh = s_prefix;
                __syncthreads();
            }
            thresh = s_thresh;
        }

        // picks: every level reference (all) or those with priority <= thresh
        for (int64_t j = t0; j < nr; j += stride) {
            const int len = d.lcnt[j];
            if (len <= 0 || d.rho[j] != c) continue;
            if (!all && niche_key(seed, gen, j, c) > thresh) continue;
            const int off = d.loff[j], full = d.loff[j + 1] - off;
            int pos;
            if (c == 0) {
                // nearest member; the list is untouched at level 0
                pos = 0;
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
    }
    if (g.rank == 0 && tid == 0) sc->levels = levels;
}

// ------------------------------------------------------------ k_finish
// Survivors (ascending indices of P and the picked members), the info block
// and the optional intermediates.
__global__ void __launch_bounds__(kCoopThreads, 1) k_finish(Plan* plan)
{
    const Group g = group_of(plan);
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
    if (ok && in.mode == MODE_SELECT) {
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
        if (st) atomicCAS(&plan->status, 0, st);
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
