// Front peeling (Section IV-A "Nondominated Sorting", Algorithm S.3):
//   p = 1[c = 0];  loop { r[p] = k;  d_j = sum_i p_i D_ij;  c -= d + p;  k++ }
// with c the number of dominators of each point (column sums of D).
//
// One cooperative launch per call. Each CTA of a problem's group owns whole
// column blocks (1024 sorted points) and their counts. Per front, the CTA
// stages the members whose rows reach its blocks in shared memory, then for
// every member reads the 128-byte segment of row p that falls in a block it
// owns (one coalesced 4-byte load per lane; the next 16 members' loads are
// in flight while the current 16 are counted) and adds the words into
// per-lane Harley-Seal bit-sliced counters, giving d_j. Points whose count
// reaches zero form the next front. One bounded group barrier separates
// fronts. Selection stops once the fronts peeled hold n_keep points (that
// front is l); ranking may continue to the end.
#include "emo_kernels.cuh"

namespace emo {

constexpr int kPeelNH = 18;  // counter planes: 4 + 18 bits per column and warp

__global__ void __launch_bounds__(kCoopThreads, 1) k_peel(Plan* plan)
{
    constexpr int NW = kCoopThreads / 32;
    __shared__ int s_cnt[kColBlock];
    __shared__ int s_newn;
    __shared__ int s_warp[33];
    extern __shared__ int s_dyn[];  // [ncb + 1] member prefix per block, [kPeelChunk] staged members
    int* s_pref = s_dyn;

    const Group g = group_of(plan);
    const ProbDev& d = plan->p[g.prob];
    const ProbIn& in = d.in;
    const long long budget = plan->spin_budget;
    if (ld_volatile(&d.sc->status) != 0) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n2 = in.n2, n2p = d.n2p;
    const int ncb = d.ncb;
    int* s_mem = s_dyn + ncb + 1;
    const int64_t target = in.n_keep > 0 ? in.n_keep : n2;

    // ---- front 0: points without dominators
    for (int cb = g.rank; cb < ncb; cb += g.size) {
        if (tid == 0) s_newn = 0;
        __syncthreads();
        for (int q = tid; q < kColBlock; q += blockDim.x) {
            const int64_t s = (int64_t)cb * kColBlock + q;
            if (s < n2 && __ldcg(&d.cnt[s]) == 0) {
                const int slot = atomicAdd(&s_newn, 1);
                d.front[(int64_t)cb * kColBlock + slot] = (int32_t)s;
                d.rank_s[s] = 0;
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

        // prefix of the member counts of every column block up to the last owned one
        const int last_cb = g.rank < ncb ? g.rank + ((ncb - 1 - g.rank) / g.size) * g.size : -1;
        if (last_cb >= 0) {
            int run = 0;
            for (int base = 0; base <= last_cb; base += blockDim.x) {
                const int c = base + tid;
                const int v = c <= last_cb ? __ldcg(&frn[c]) : 0;
                int tot;
                const int pre = block_exclusive_scan<kCoopThreads>(v, s_warp, tot);
                if (c <= last_cb) s_pref[c] = run + pre;
                run += tot;
                __syncthreads();
            }
            if (tid == 0) s_pref[last_cb + 1] = run;
            __syncthreads();
        }
        const int nall = last_cb >= 0 ? s_pref[last_cb + 1] : 0;  // members reaching the last owned block

        for (int m0 = 0; m0 < nall; m0 += kPeelChunk) {
            const int mc = min(kPeelChunk, nall - m0);
            __syncthreads();
            for (int i = tid; i < mc; i += blockDim.x) {  // stage members m0 .. m0 + mc in block order
                const int o = m0 + i;
                int lo = 0, hi = last_cb;  // block with s_pref[blk] <= o < s_pref[blk + 1]
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_pref[mid] <= o) lo = mid;
                    else hi = mid - 1;
                }
                // stage (tile base of the member's row block, row): tile (rb, cb) is base + cb
                const int p = __ldcg(&fr[(int64_t)lo * kColBlock + (o - s_pref[lo])]);
                const int rb = p >> 5;
                const uint32_t base = (uint32_t)(tiles_before(rb, ncb) - rb / 32);
                s_mem[i] = (int)(base * 32u + (uint32_t)(p & 31));
            }
            __syncthreads();
            for (int cb = g.rank; cb < ncb; cb += g.size) {
                const int nmem = min(mc, s_pref[cb + 1] - m0);  // staged members reaching cb
                if (nmem <= 0) continue;
                for (int q = tid; q < kColBlock; q += blockDim.x) s_cnt[q] = 0;
                if (tid == 0) s_newn = 0;
                __syncthreads();
                VCount<kPeelNH> vc;
                auto load16 = [&](int b0, uint32_t (&x)[16]) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int i = b0 + j;
                        x[j] = 0u;
                        if (i < nmem) {
                            const uint32_t e = (uint32_t)s_mem[i];
                            const uint32_t r = e & 31u;
                            const int64_t t = (int64_t)(e >> 5) + cb;
                            x[j] = __ldcs(&d.D[(t << 10) + (r << 5) + lane]);
                        }
                    }
                };
                uint32_t xa[16], xb[16];
                int b0 = warp * 16;
                if (b0 < nmem) load16(b0, xa);
                while (b0 < nmem) {
                    const int b1 = b0 + NW * 16;
                    if (b1 < nmem) load16(b1, xb);  // next batch in flight while this one is counted
                    vc.add16(xa);
                    b0 = b1;
                    if (b0 >= nmem) break;
                    const int b2 = b0 + NW * 16;
                    if (b2 < nmem) load16(b2, xa);
                    vc.add16(xb);
                    b0 = b2;
                }
                const int top = vc.top_plane();
                if (top >= 0) {
                    for (int b = 0; b < 32; ++b) {
                        const int c = vc.count_upto(b, top);
                        if (c) atomicAdd(&s_cnt[b * 32 + lane], c);
                    }
                }
                __syncthreads();
                for (int q = tid; q < kColBlock; q += blockDim.x) {
                    const int dq = s_cnt[(q & 31) * 32 + (q >> 5)];
                    const int64_t s = (int64_t)cb * kColBlock + q;
                    if (dq && s < n2) {
                        const int c = d.cnt[s] - dq;
                        d.cnt[s] = c;
                        if (c == 0) {
                            const int slot = atomicAdd(&s_newn, 1);
                            fw[(int64_t)cb * kColBlock + slot] = (int32_t)s;
                            d.rank_s[s] = k + 1;
                        }
                    }
                }
                __syncthreads();
                if (tid == 0) {
                    // counts of one block may arrive over several member chunks
                    const int before = m0 == 0 ? 0 : fwn[cb];
                    fwn[cb] = before + s_newn;
                    atomicAdd(&d.sc->ranked, s_newn);
                }
            }
        }
        // blocks that received no member in this front still need their count of new members
        if (tid == 0)
            for (int cb = g.rank; cb < ncb; cb += g.size)
                if (nall == 0 || s_pref[cb + 1] == 0) fwn[cb] = 0;
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
            r = __ldcg(&d.rank_s[s]);
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
