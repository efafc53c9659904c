// Front peeling (Section IV-A "Nondominated Sorting", Algorithm S.3):
//   p = 1[c = 0];  loop { r[p] = k;  d_j = sum_i p_i D_ij;  c -= d + p;  k++ }
// with c the number of dominators of each point (column sums of D).
//
// One cooperative launch per call. Per front, the CTAs of a problem's group
// take whole column blocks (1024 sorted points; their counts live in global
// memory): block cb has about cb + 1 units of work per front, so with more
// than two blocks per CTA of a group of at least 64 CTAs they come from a
// counter, the last block first, and the CTAs finish the front together;
// otherwise each CTA takes the blocks dealt to it in a snake over the CTAs
// (descending). For each
// block the CTA stages the members whose rows reach it in shared memory (a
// prefix of the front's list in block order, so one staging serves the
// smaller blocks the CTA takes next); every warp copies the
// 128-byte row segments of 32 members at a time into its own ring of
// shared-memory stages with cp.async (the next batch in flight while one
// is counted), then adds the words into per-lane Harley-Seal bit-sliced
// counters, giving d_j. Points whose count reaches zero form the next front.
// One bounded group barrier separates fronts. Selection stops once the fronts
// peeled hold n_keep points (that front is l); ranking may continue to the
// end.
#include "emo_kernels.cuh"

namespace emo {

constexpr int kPeelNH = 10;  // counter planes: 4 + 10 bits per column (a chunk holds <= 8192 members)
constexpr int kPeelBits = 4 + kPeelNH;
static_assert(kPeelChunk < (1 << kPeelBits), "column counter overflow");
static_assert(kCoopThreads == 512, "the counter reduction tree assumes 16 warps");

// Exact column counts of the CTA: the 16 warps' bit-sliced counters are added
// in a tree (16 -> 8 -> 4 -> 2 -> 1, ripple-carry over the bit planes, through
// `scratch`), then warp w unpacks bits 2w and 2w + 1 of every word:
// s_cnt[b * 32 + w'] = count of column 32 w' + b. No atomics.
__device__ __forceinline__ void peel_reduce_counts(const VCount<kPeelNH>& vc, uint32_t* scratch, int* s_cnt,
                                                   int warp, int lane)
{
    uint32_t P[kPeelBits];
    P[0] = vc.ones;
    P[1] = vc.twos;
    P[2] = vc.fours;
    P[3] = vc.eights;
#pragma unroll
    for (int i = 0; i < kPeelNH; ++i) P[4 + i] = vc.hi[i];
#pragma unroll 1
    for (int half = 8; half >= 1; half >>= 1) {
        if (warp >= half && warp < 2 * half) {
#pragma unroll
            for (int p = 0; p < kPeelBits; ++p) scratch[((warp - half) * kPeelBits + p) * 32 + lane] = P[p];
        }
        __syncthreads();
        if (warp < half) {
            uint32_t c = 0u;
#pragma unroll
            for (int p = 0; p < kPeelBits; ++p) {
                const uint32_t q = scratch[(warp * kPeelBits + p) * 32 + lane];
                const uint32_t x = P[p] ^ q;
                const uint32_t sum = x ^ c;
                c = (P[p] & q) | (c & x);
                P[p] = sum;
            }
        }
        __syncthreads();
    }
    if (warp == 0) {
#pragma unroll
        for (int p = 0; p < kPeelBits; ++p) scratch[p * 32 + lane] = P[p];
    }
    __syncthreads();
    uint32_t Q[kPeelBits];
#pragma unroll
    for (int p = 0; p < kPeelBits; ++p) Q[p] = scratch[p * 32 + lane];
#pragma unroll
    for (int bb = 0; bb < 2; ++bb) {
        const int b = 2 * warp + bb;
        int c = 0;
#pragma unroll
        for (int p = 0; p < kPeelBits; ++p) c |= (int)((Q[p] >> b) & 1u) << p;
        s_cnt[b * 32 + lane] = c;
    }
    __syncthreads();
}

// Column block dealt to CTA `rank` of a group of G in round r (snake order
// over the blocks from the last to the first); -1 past the end.
__device__ __forceinline__ int peel_block(int r, int rank, int G, int ncb)
{
    const int o = r * G + ((r & 1) ? G - 1 - rank : rank);
    return o < ncb ? ncb - 1 - o : -1;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Front lists hold each member p as (tile base of its row block) * 32 + row,
// with tile (rb, cb) = base + cb: the row segment of p in block cb is
// D[((base + cb) * 32 + p % 32) * 32 ...].
__device__ __forceinline__ int32_t peel_encode(int64_t p, int ncb)
{
    const int64_t rb = p >> 5;
    const uint32_t base = (uint32_t)(tiles_before(rb, ncb) - rb / 32);
    return (int32_t)(base * 32u + (uint32_t)(p & 31));
}

__global__ void __launch_bounds__(kCoopThreads, 1) k_peel(Plan* plan)
{
    constexpr int NW = kCoopThreads / 32;
    __shared__ int s_cnt[kColBlock];
    __shared__ int s_newn, s_base;
    __shared__ int s_warp[33];
    // [ring] per-warp copy stages | [ncb + 1] member prefix per block | [kPeelChunk] staged members
    extern __shared__ __align__(128) int s_dyn[];

    const Group g = group_of(plan, true);
    if (g.prob < 0) return;  // a CTA beyond every problem's group
    const ProbDev& d = plan->p[g.prob];
    const ProbIn& in = d.in;
    const long long budget = plan->spin_budget;
    if (ld_volatile(&d.sc->status) != 0) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n2 = in.n2, n2p = d.n2p;
    const int ncb = d.ncb;
    // workspace pointers in registers: the copy asm clobbers memory, which
    // would otherwise reload them from the plan before every copy
    const uint32_t* const Dm = d.D;
    int32_t* const cntp = d.cnt;
    int32_t* const rank_s = d.rank_s;
    uint32_t* ring = reinterpret_cast<uint32_t*>(s_dyn) + warp * (kPeelStages * 32 * 32);
    int* s_pref = s_dyn + kPeelRingBytes / 4;
    int* s_mem = s_pref + ncb + 1;
    const int64_t target = in.n_keep > 0 ? in.n_keep : n2;

    // ---- front 0: points without dominators
    for (int r = 0;; ++r) {
        const int cb = peel_block(r, g.rank, g.size, ncb);
        if (cb < 0) break;
        if (tid == 0) s_newn = 0;
        __syncthreads();
        for (int q = tid; q < kColBlock; q += blockDim.x) {
            const int64_t s = (int64_t)cb * kColBlock + q;
            if (s < n2 && __ldcg(&cntp[s]) == 0) {
                const int slot = atomicAdd(&s_newn, 1);
                d.front[(int64_t)cb * kColBlock + slot] = peel_encode(s, ncb);
                rank_s[s] = 0;
            }
        }
        __syncthreads();
        if (tid == 0) {
            d.front_n[cb] = s_newn;
            atomicAdd(&d.sc->ranked, s_newn);
        }
    }
    if (!group_sync(d.sc, g.size, budget)) return;

    int64_t prev_total = 0, total = ld_volatile(&d.sc->ranked);
    int k = 0;
    __shared__ int s_item;
    // (a counter round trip per block pays only across many CTAs)
    const bool dynamic = g.size >= 64 && ncb > 2 * g.size;
    while (total < target) {
        if (total == prev_total || k >= n2) {  // empty front before the target: inconsistent counts
            if (tid == 0) set_status(d.sc, EMO_ERR_INVALID_ARG);
            return;
        }
        const int cur = k & 1, nxt = cur ^ 1;
        const int32_t* fr = d.front + (int64_t)cur * n2p;
        const int32_t* frn = d.front_n + (int64_t)cur * ncb;
        int32_t* fw = d.front + (int64_t)nxt * n2p;
        int32_t* fwn = d.front_n + (int64_t)nxt * ncb;
        // the next front's block counter (every CTA left this one's loop
        // before the last barrier)
        if (g.rank == 0 && tid == 0) d.wcnt[nxt] = 0;

        // prefix of the member counts of every column block
        {
            int run = 0;
            for (int base = 0; base < ncb; base += blockDim.x) {
                const int c = base + tid;
                const int v = c < ncb ? __ldcg(&frn[c]) : 0;
                int tot;
                const int pre = block_exclusive_scan<kCoopThreads>(v, s_warp, tot);
                if (c < ncb) s_pref[c] = run + pre;
                run += tot;
                __syncthreads();
            }
            if (tid == 0) s_pref[ncb] = run;
            __syncthreads();
        }

        // With more than two column blocks per CTA over a group of at least
        // 64 CTAs, blocks are taken from a counter, the last (heaviest)
        // first, so that the CTAs finish the front together; otherwise each
        // CTA takes its blocks of the snake
        // (no counter round trip per block). Either way a CTA visits its
        // blocks in descending order: the members reaching block cb are the
        // first s_pref[cb + 1] of the list in block order, so a chunk staged
        // for one block serves every smaller block the CTA takes after it.
        int staged_m0 = -1, staged_mc = 0;
        for (int round = 0;; ++round) {
            int cb;
            if (dynamic) {
                if (tid == 0) s_item = atomicAdd(&d.wcnt[cur], 1);
                __syncthreads();
                const int item = s_item;
                __syncthreads();  // every thread has read s_item
                if (item >= ncb) break;
                cb = ncb - 1 - item;
            } else {
                cb = peel_block(round, g.rank, g.size, ncb);
                if (cb < 0) break;
            }
            const int nreach = s_pref[cb + 1];  // members whose rows reach cb
            if (nreach == 0) {
                if (tid == 0) fwn[cb] = 0;
                continue;
            }
            for (int m0 = 0; m0 < nreach; m0 += kPeelChunk) {
                const int nmem = min(kPeelChunk, nreach - m0);
                if (staged_m0 != m0 || staged_mc < nmem) {
                    // stage the (encoded) members m0 .. m0 + nmem in block order:
                    // warp w copies the lists of blocks w, w + NW, ... with async
                    // 4-byte copies
                    __syncthreads();
                    for (int c = warp; c <= cb; c += NW) {
                        const int b0 = s_pref[c], lo = max(b0, m0), hi = min(s_pref[c + 1], m0 + nmem);
                        for (int o = lo + lane; o < hi; o += 32)
                            cp_async4(smem_u32(s_mem + (o - m0)), fr + (int64_t)c * kColBlock + (o - b0));
                    }
                    cp_async_commit();
                    cp_async_wait<0>();
                    __syncthreads();
                    staged_m0 = m0;
                    staged_mc = nmem;
                }
                // new members of one block may arrive over several member chunks:
                // append after those found in the earlier chunks of this front
                if (tid == 0) s_base = s_newn = m0 == 0 ? 0 : fwn[cb];
                // the block's counts, loaded now and used after the stream
                int cpre[kColBlock / kCoopThreads];
#pragma unroll
                for (int u = 0; u < kColBlock / kCoopThreads; ++u) {
                    const int64_t sq = (int64_t)cb * kColBlock + tid + u * kCoopThreads;
                    cpre[u] = sq < n2 ? __ldcg(&cntp[sq]) : 0;
                }
                __syncthreads();
                VCount<kPeelNH> vc;
                // copies of the warp's batches b = warp, warp + NW, ... (32 members each):
                // lane copies 16 bytes (words 4 q .. 4 q + 3) of row j = 4 it + lane / 8
                const int nb = (nmem + 31) >> 5;
                auto issue = [&](int b, int stage) {
                    uint32_t* dst = ring + stage * (32 * 32);
                    const int q = lane & 7;
#pragma unroll
                    for (int it = 0; it < 8; ++it) {
                        const int j = it * 4 + (lane >> 3), i = b * 32 + j;
                        if (b < nb && i < nmem) {
                            const uint32_t e = (uint32_t)s_mem[i];
                            const int64_t t = (int64_t)(e >> 5) + cb;
                            cp_async16(smem_u32(dst + j * 32 + q * 4), Dm + (t << 10) + ((e & 31u) << 5) + q * 4);
                        }
                    }
                    cp_async_commit();
                };
                int b = warp, st = 0;
#pragma unroll
                for (int q = 0; q + 1 < kPeelStages; ++q) issue(b + q * NW, q);
                for (; b < nb; b += NW) {
                    issue(b + (kPeelStages - 1) * NW, (st + kPeelStages - 1) % kPeelStages);
                    cp_async_wait<kPeelStages - 1>();
                    __syncwarp();
                    const uint32_t* src = ring + st * (32 * 32);
                    const int nrow = min(32, nmem - b * 32);
                    uint32_t x[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) x[j] = j < nrow ? src[j * 32 + lane] : 0u;
                    vc.add16(x);
                    if (nrow > 16) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) x[j] = j + 16 < nrow ? src[(j + 16) * 32 + lane] : 0u;
                        vc.add16(x);
                    }
                    __syncwarp();  // the stage is refilled kPeelStages - 1 iterations later
                    st = (st + 1) % kPeelStages;
                }
                cp_async_wait<0>();  // no copy outlives the block (the tail batches were empty)
                __syncthreads();     // every warp is done with its ring before the tree reuses it
                peel_reduce_counts(vc, reinterpret_cast<uint32_t*>(s_dyn), s_cnt, warp, lane);
#pragma unroll
                for (int u = 0; u < kColBlock / kCoopThreads; ++u) {
                    const int q = tid + u * kCoopThreads;
                    const int dq = s_cnt[(q & 31) * 32 + (q >> 5)];
                    const int64_t s = (int64_t)cb * kColBlock + q;
                    if (dq && s < n2) {
                        const int c = cpre[u] - dq;
                        cntp[s] = c;
                        if (c == 0) {
                            const int slot = atomicAdd(&s_newn, 1);
                            fw[(int64_t)cb * kColBlock + slot] = peel_encode(s, ncb);
                            rank_s[s] = k + 1;
                        }
                    }
                }
                __syncthreads();
                if (tid == 0) {
                    fwn[cb] = s_newn;
                    atomicAdd(&d.sc->ranked, s_newn - s_base);
                }
            }
        }
        if (!group_sync(d.sc, g.size, budget)) return;
        prev_total = total;
        total = ld_volatile(&d.sc->ranked);
        ++k;
    }

    // ---- results: l, |P|, |L|; ranks in caller order; the list of S
    const int l = k;
    if (g.rank == 0 && tid == 0) {
        d.sc->l = l;
        d.sc->nP = (int32_t)prev_total;
        d.sc->nL = (int32_t)(total - prev_total);
        d.sc->nfronts = l + 1;
        if (in.last_rank_out) *in.last_rank_out = l;
    }
    const int32_t* idx = d.idx + (int64_t)ld_volatile(&d.sc->idx_buf) * n2p;
    const int64_t stride = (int64_t)g.size * blockDim.x;
    for (int64_t s0 = (int64_t)g.rank * blockDim.x; s0 < n2; s0 += stride) {
        const int64_t s = s0 + tid;
        int r = kNotRanked;
        int32_t v = 0;
        if (s < n2) {
            r = __ldcg(&rank_s[s]);
            v = __ldcg(&idx[s]);
            d.rank_o[v] = r;
            if (in.mode == MODE_RANK && in.rank_out) in.rank_out[v] = r;
        }
        const bool inS = s < n2 && r <= l;
        const unsigned mask = __ballot_sync(0xffffffffu, inS);
        int base = 0;
        if (lane == 0 && mask) base = atomicAdd(&d.sc->nS, __popc(mask));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (inS) d.slist[base + __popc(mask & lanemask_lt())] = v;
    }
}

}  // namespace emo

namespace emo {

// ---------------------------------------------------------------- wavefront
// The same front peeling (Algorithm S.3) without a grid barrier per front.
// In lexicographic order a row of column block cb' can only reach column
// blocks cb >= cb', so the counts of block cb after front k depend on the
// members of front k in blocks 0..cb alone. A task (cb, k) -- subtract from
// block cb's counts the rows of front k's members in blocks 0..cb, and take
// the points whose count reaches zero as front k + 1 of block cb -- may
// therefore run as soon as every block cb' <= cb has finished its task k - 1
// (front k of cb' is then final). Per block: wdone = tasks finished
// (INT32_MAX once every point of the block is ranked), its members in front
// order in the block's slice of `front`, and wofs = where each front starts
// in that list. A task's dependency test reads the counters of the blocks
// below it in one parallel pass. Each CTA owns its blocks (dealt in
// the same snake as the barrier schedule) and runs whichever owned task is
// ready, earliest front first (lowest block on ties); a low block runs ahead
// only while the others wait, and high (heavy) blocks never wait at a
// barrier for the slowest CTA. The CTA of rank 0 follows the
// fronts in order: once front k is final everywhere (every wdone >= k) it adds
// |front k|; the first front whose running total reaches n_keep is l, and
// tasks of fronts >= l are skipped. Ranks a low block assigned beyond l are
// reported as unranked. Every wait is bounded by the spin budget.
// Every thread: true when each block c <= cb has finished its task k - 1
// (wdone[c] >= k); one parallel pass over the counters, then a fence, so the
// lists and offsets written before those counters were released are seen.
__device__ __forceinline__ bool wave_ready(const ProbDev& d, int cb, int k)
{
    int ok = 1;
    for (int c = threadIdx.x; c <= cb; c += blockDim.x) ok &= ld_volatile(&d.wdone[c]) >= k;
    ok = __syncthreads_and(ok);
    if (ok) __threadfence();
    return ok != 0;
}
__device__ __forceinline__ void st_rel(int* p, int v) { st_release(reinterpret_cast<unsigned*>(p), (unsigned)v); }

__global__ void __launch_bounds__(kCoopThreads, 1) k_peel_wave(Plan* plan)
{
    constexpr int NW = kCoopThreads / 32;
    constexpr int kInf = INT32_MAX;
    __shared__ int s_cnt[kColBlock];
    __shared__ int s_newn;
    __shared__ int s_warp[33];
    __shared__ int s_nown, s_lf, s_st;
    __shared__ long long s_cum;
    __shared__ int s_leadk;
    // [ring] per-warp copy stages | [ncb + 1] member prefix | [kPeelChunk] staged members |
    // [ncb] owned blocks | [ncb] next front of each owned block (kInf: finished)
    extern __shared__ __align__(128) int s_dyn[];

    const Group g = group_of(plan, true);
    if (g.prob < 0) return;  // a CTA beyond every problem's group
    const ProbDev& d = plan->p[g.prob];
    const ProbIn& in = d.in;
    const long long budget = plan->spin_budget;
    if (ld_volatile(&d.sc->status) != 0) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n2 = in.n2;
    const int ncb = d.ncb;
    const uint32_t* const Dm = d.D;
    int32_t* const cntp = d.cnt;
    int32_t* const rank_s = d.rank_s;
    int32_t* const mlist = d.front;
    const int64_t wstride = n2 + 2;  // wofs row length
    uint32_t* ring = reinterpret_cast<uint32_t*>(s_dyn) + warp * (kPeelStages * 32 * 32);
    int* s_pref = s_dyn + kPeelRingBytes / 4;
    int* s_mem = s_pref + ncb + 1;
    int* s_own = s_mem + kPeelChunk;
    int* s_k = s_own + ncb;
    const int64_t target = in.n_keep > 0 ? in.n_keep : n2;

    // ---- owned blocks (ascending) and front 0: points without dominators
    if (tid == 0) {
        int n = 0;
        for (int r = 0;; ++r) {
            const int cb = peel_block(r, g.rank, g.size, ncb);
            if (cb < 0) break;
            s_own[n++] = cb;
        }
        for (int i = 0; i < n / 2; ++i) {  // dealt descending: reverse
            const int t = s_own[i];
            s_own[i] = s_own[n - 1 - i];
            s_own[n - 1 - i] = t;
        }
        s_nown = n;
        s_cum = 0;
        s_leadk = 0;
    }
    __syncthreads();
    const int nown = s_nown;
    for (int i = 0; i < nown; ++i) {
        const int cb = s_own[i];
        const int nvalid = (int)min((int64_t)kColBlock, n2 - (int64_t)cb * kColBlock);
        if (tid == 0) s_newn = 0;
        __syncthreads();
        for (int q = tid; q < nvalid; q += blockDim.x) {
            const int64_t s = (int64_t)cb * kColBlock + q;
            if (__ldcg(&cntp[s]) == 0) {
                const int slot = atomicAdd(&s_newn, 1);
                mlist[(int64_t)cb * kColBlock + slot] = peel_encode(s, ncb);
                rank_s[s] = 0;
            }
        }
        __syncthreads();
        if (tid == 0) {
            uint16_t* of = d.wofs + (int64_t)cb * wstride;
            of[0] = 0;
            of[1] = (uint16_t)s_newn;
            atomicAdd(&d.wcnt[0], s_newn);
            const bool exhausted = s_newn == nvalid;
            d.wmaxf[cb] = 0;
            d.wdone[cb] = exhausted ? kInf : 0;
            s_k[i] = exhausted ? kInf : 0;
        }
    }
    if (!group_sync(d.sc, g.size, budget)) return;

    long long idle_since = clock64();
    for (;;) {
        // ---- the leader follows the fronts in order and fixes l
        if (g.rank == 0) {
            for (;;) {
                if (tid == 0) {
                    s_lf = ld_volatile(&d.sc->lfinal1);
                    s_st = ld_volatile(&d.sc->status);
                }
                __syncthreads();
                const int k = s_leadk;
                if (s_lf || s_st || k >= n2 || !wave_ready(d, ncb - 1, k)) break;
                if (tid == 0) {
                    const int fk = __ldcg(&d.wcnt[k]);
                    const long long cum = s_cum + fk;
                    if (fk == 0) {  // an empty front before n_keep points: inconsistent counts
                        set_status(d.sc, EMO_ERR_INVALID_ARG);
                    } else if (cum >= target) {
                        d.sc->nP = (int32_t)s_cum;
                        d.sc->nL = fk;
                        __threadfence();
                        st_rel(&d.sc->lfinal1, k + 1);
                    } else {
                        s_cum = cum;
                        s_leadk = k + 1;
                    }
                }
                __syncthreads();
            }
        }
        if (tid == 0) {
            s_lf = ld_volatile(&d.sc->lfinal1);
            s_st = ld_volatile(&d.sc->status);
        }
        __syncthreads();
        if (s_st != 0) return;
        const int lf = s_lf;
        // ---- the ready task of the earliest front among the owned blocks
        // (lowest block on ties): fronts proceed in order wherever they can,
        // and a low block runs ahead only while the others must wait
        int gi = -1, bestk = kInf;
        bool left = false;
        for (int i = 0; i < nown; ++i) {
            const int k = s_k[i];
            if (k == kInf || (lf && k >= lf - 1)) continue;  // finished, or a front >= l (not needed)
            if (k >= n2) {  // more fronts than points: inconsistent counts
                if (tid == 0) set_status(d.sc, EMO_ERR_INVALID_ARG);
                return;
            }
            left = true;
            if (k < bestk && wave_ready(d, s_own[i], k)) {
                gi = i;
                bestk = k;
            }
        }
        if (gi < 0) {
            if (!left && (g.rank != 0 || lf)) break;  // nothing left here (the leader waits for l)
            if (clock64() - idle_since > budget) {
                if (tid == 0) set_status(d.sc, EMO_ERR_TIMEOUT);
                return;
            }
            __nanosleep(128);
            continue;
        }
        idle_since = clock64();
        const int cb = s_own[gi], k = s_k[gi];
        const int nvalid = (int)min((int64_t)kColBlock, n2 - (int64_t)cb * kColBlock);

        // ---- members of front k in blocks 0..cb: prefix of their counts
        {
            int run = 0;
            for (int base = 0; base <= cb; base += blockDim.x) {
                const int c = base + tid;
                int v = 0;
                if (c <= cb) {
                    const int dn = ld_volatile(&d.wdone[c]);  // >= k (the task is ready; fenced)
                    const uint16_t* of = d.wofs + (int64_t)c * wstride;
                    if (dn != kInf || k <= __ldcg(&d.wmaxf[c])) v = (int)__ldcg(&of[k + 1]) - (int)__ldcg(&of[k]);
                }
                int tot;
                const int pre = block_exclusive_scan<kCoopThreads>(v, s_warp, tot);
                if (c <= cb) s_pref[c] = run + pre;
                run += tot;
                __syncthreads();
            }
            if (tid == 0) s_pref[cb + 1] = run;
            __syncthreads();
        }
        const int nall = s_pref[cb + 1];
        const int list0 = (int)__ldcg(&d.wofs[(int64_t)cb * wstride + k + 1]);  // block cb's front k + 1 begins
        if (tid == 0) s_newn = 0;
        int cpre[kColBlock / kCoopThreads];
#pragma unroll
        for (int u = 0; u < kColBlock / kCoopThreads; ++u) {
            const int64_t sq = (int64_t)cb * kColBlock + tid + u * kCoopThreads;
            cpre[u] = sq < n2 ? __ldcg(&cntp[sq]) : 0;
        }
        for (int m0 = 0; m0 < nall; m0 += kPeelChunk) {
            const int mc = min(kPeelChunk, nall - m0);
            __syncthreads();
            // stage the members m0 .. m0 + mc (block order, read from L2): warp
            // w copies the ranges of blocks w, w + NW, ...
            for (int c = warp; c <= cb; c += NW) {
                const int b0 = s_pref[c], lo = max(b0, m0), hi = min(s_pref[c + 1], m0 + mc);
                if (lo >= hi) continue;
                const int start = (int)__ldcg(&d.wofs[(int64_t)c * wstride + k]);
                for (int o = lo + lane; o < hi; o += 32)
                    s_mem[o - m0] = __ldcg(mlist + (int64_t)c * kColBlock + start + (o - b0));
            }
            __syncthreads();
            VCount<kPeelNH> vc;
            const int nmem = mc;
            const int nb = (nmem + 31) >> 5;
            auto issue = [&](int b, int stage) {
                uint32_t* dst = ring + stage * (32 * 32);
                const int q = lane & 7;
#pragma unroll
                for (int it = 0; it < 8; ++it) {
                    const int j = it * 4 + (lane >> 3), i = b * 32 + j;
                    if (b < nb && i < nmem) {
                        const uint32_t e = (uint32_t)s_mem[i];
                        const int64_t t = (int64_t)(e >> 5) + cb;
                        cp_async16(smem_u32(dst + j * 32 + q * 4), Dm + (t << 10) + ((e & 31u) << 5) + q * 4);
                    }
                }
                cp_async_commit();
            };
            int b = warp, st = 0;
#pragma unroll
            for (int q = 0; q + 1 < kPeelStages; ++q) issue(b + q * NW, q);
            for (; b < nb; b += NW) {
                issue(b + (kPeelStages - 1) * NW, (st + kPeelStages - 1) % kPeelStages);
                cp_async_wait<kPeelStages - 1>();
                __syncwarp();
                const uint32_t* src = ring + st * (32 * 32);
                const int nrow = min(32, nmem - b * 32);
                uint32_t x[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) x[j] = j < nrow ? src[j * 32 + lane] : 0u;
                vc.add16(x);
                if (nrow > 16) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) x[j] = j + 16 < nrow ? src[(j + 16) * 32 + lane] : 0u;
                    vc.add16(x);
                }
                __syncwarp();
                st = (st + 1) % kPeelStages;
            }
            cp_async_wait<0>();
            __syncthreads();
            peel_reduce_counts(vc, reinterpret_cast<uint32_t*>(s_dyn), s_cnt, warp, lane);
#pragma unroll
            for (int u = 0; u < kColBlock / kCoopThreads; ++u) {
                const int q = tid + u * kCoopThreads;
                const int dq = s_cnt[(q & 31) * 32 + (q >> 5)];
                const int64_t s = (int64_t)cb * kColBlock + q;
                if (dq && q < nvalid) {
                    cpre[u] -= dq;
                    cntp[s] = cpre[u];
                    if (cpre[u] == 0) {
                        const int slot = atomicAdd(&s_newn, 1);
                        mlist[(int64_t)cb * kColBlock + list0 + slot] = peel_encode(s, ncb);
                        rank_s[s] = k + 1;
                    }
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            const int nn = s_newn, total = list0 + nn;
            d.wofs[(int64_t)cb * wstride + k + 2] = (uint16_t)total;
            if (nn) atomicAdd(&d.wcnt[k + 1], nn);
            const bool exhausted = total == nvalid;
            if (exhausted) d.wmaxf[cb] = k + 1;
            __threadfence();
            st_rel(&d.wdone[cb], exhausted ? kInf : k + 1);
            s_k[gi] = exhausted ? kInf : k + 1;
        }
        __syncthreads();
    }
    if (!group_sync(d.sc, g.size, budget)) return;

    // ---- results: l, |P|, |L| (set by the leader); ranks in caller order
    // (beyond l: not ranked); the list of S
    const int l = ld_volatile(&d.sc->lfinal1) - 1;
    if (g.rank == 0 && tid == 0) {
        d.sc->l = l;
        d.sc->nfronts = l + 1;
        if (in.last_rank_out) *in.last_rank_out = l;
    }
    const int32_t* idx = d.idx + (int64_t)ld_volatile(&d.sc->idx_buf) * d.n2p;
    const int64_t stride = (int64_t)g.size * blockDim.x;
    for (int64_t s0 = (int64_t)g.rank * blockDim.x; s0 < n2; s0 += stride) {
        const int64_t s = s0 + tid;
        int r = kNotRanked;
        int32_t v = 0;
        if (s < n2) {
            r = __ldcg(&rank_s[s]);
            if (r > l) r = kNotRanked;
            v = __ldcg(&idx[s]);
            d.rank_o[v] = r;
            if (in.mode == MODE_RANK && in.rank_out) in.rank_out[v] = r;
        }
        const bool inS = s < n2 && r <= l;
        const unsigned mask = __ballot_sync(0xffffffffu, inS);
        int base = 0;
        if (lane == 0 && mask) base = atomicAdd(&d.sc->nS, __popc(mask));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (inS) d.slist[base + __popc(mask & lanemask_lt())] = v;
    }
}

}  // namespace emo
