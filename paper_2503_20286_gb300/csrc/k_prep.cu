// Set-up, input validation and the lexicographic ordering of the points.
//
// The points are put in lexicographic order of (f_1, ..., f_m) by a stable
// LSD radix sort (8-bit digits of an order-preserving uint32 key, objective
// m first, objective 1 last). In that order a point can only be dominated by
// points before it (Section IV-A: p dominates q implies f(p) <= f(q)
// componentwise, hence f(p) <=_lex f(q)), which is what lets the dominance
// kernel compute and store only the upper triangle of D. Runs of identical
// objective vectors (which never dominate each other) are recorded so the
// dominance kernel can clear them.
#include "emo_kernels.cuh"
#include "group_radix.cuh"

namespace emo {

// One thread per problem: carve the workspace, zero the scalars; thread 0
// then splits the cooperative grid into CTA groups and counts work items.
__global__ void k_setup(SetupArgs a, SplitArgs sp, Plan* plan, char* ws)
{
    const int t = threadIdx.x;
    if (t < a.nprob) {
        ProbDev d;
        layout_problem(a.in[t], a.G, ws + a.in[t].ws_off, &d);
        plan->p[t] = d;
        char* sc = (char*)d.sc;
        for (size_t i = 0; i < sizeof(Scal); ++i) sc[i] = 0;
    }
    __syncthreads();
    if (t == 0) {
        plan->nprob = a.nprob;
        plan->G = a.G;
        plan->spin_budget = a.spin_budget;
        plan->split = sp;
        for (int i = 0; i <= kMaxM; ++i) plan->dom_ctr[i] = 0;
        for (int i = 0; i <= kMaxM; ++i) plan->asc_next[i] = 0;
        plan->status = 0;
        // Wide CTA groups (peeling, TensorHypE) proportional to n2^2 (the
        // dominance and peeling work), at least one CTA each and at most the
        // problem's cap_wide; narrow groups (the other cooperative kernels)
        // the first min(wide, cap_narrow) CTAs' worth. CTAs beyond the
        // groups serve no problem.
        double tot = 0.0;
        for (int p = 0; p < a.nprob; ++p) tot += (double)a.in[p].n2 * (double)a.in[p].n2;
        int extra = a.G - a.nprob, given = 0;
        int cnt[kMaxBatch];
        auto cap_of = [&](int p, int32_t c) { return c > 0 ? c : a.G; };
        for (int p = 0; p < a.nprob; ++p) {
            double w = (double)a.in[p].n2 * (double)a.in[p].n2 / tot;
            cnt[p] = min(cap_of(p, a.in[p].cap_wide), 1 + (int)(w * extra));
            given += cnt[p];
        }
        for (bool grew = true; given < a.G && grew;) {
            grew = false;
            for (int p = 0; p < a.nprob && given < a.G; ++p)
                if (cnt[p] < cap_of(p, a.in[p].cap_wide)) { cnt[p]++; given++; grew = true; }
        }
        int acc = 0, accn = 0;
        for (int p = 0; p < a.nprob; ++p) {
            plan->grp_first[p] = acc;
            acc += cnt[p];
            plan->grpn_first[p] = accn;
            accn += min(cnt[p], cap_of(p, a.in[p].cap_narrow));
        }
        plan->grp_first[a.nprob] = acc;
        plan->grpn_first[a.nprob] = accn;
        long long di = 0;
        for (int p = 0; p < a.nprob; ++p) {
            plan->dom_item_start[p] = di;
            di += dom_items_of(a.in[p].n2, a.in[p].dom_chunk);
        }
        plan->dom_item_start[a.nprob] = di;
        plan->dom_items = di;
    }
}

// Validation and initialisation, grid (x, problem).
__global__ void k_prep(Plan* plan)
{
    const ProbDev& d = plan->p[blockIdx.y];
    const ProbIn& in = d.in;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n2 = in.n2, m = in.m;
    bool bad = false;
    if (in.F) {  // null only for the niching from a given association
        // finiteness, and which bits of each objective's sort key vary (a
        // radix pass over a byte that no point changes is skipped)
        uint32_t kor[kMaxM], kinv[kMaxM];
#pragma unroll
        for (int k = 0; k < kMaxM; ++k) kor[k] = kinv[k] = 0u;
        for (int64_t i = tid; i < n2; i += stride) {
#pragma unroll
            for (int k = 0; k < kMaxM; ++k) {
                if (k >= m) break;
                const float f = in.F[i * m + k];
                if (!isfinite(f)) bad = true;
                const uint32_t key = float_key(f);
                kor[k] |= key;
                kinv[k] |= ~key;
            }
        }
#pragma unroll
        for (int k = 0; k < kMaxM; ++k) {
            if (k >= m) break;
            uint32_t a = kor[k], b = kinv[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a |= __shfl_xor_sync(0xffffffffu, a, o);
                b |= __shfl_xor_sync(0xffffffffu, b, o);
            }
            if ((threadIdx.x & 31) == 0) {
                if (a) atomicOr(&d.sc->kor[k], a);
                if (b) atomicOr(&d.sc->kinv[k], b);
            }
        }
    }
    for (int64_t s = tid; s < d.n2p; s += stride) {
        d.idx[s] = (int32_t)s;
        d.cnt[s] = 0;
        d.rank_s[s] = kNotRanked;
        d.flag[s] = 0;
    }
    for (int64_t i = tid; i < n2; i += stride) d.rank_o[i] = kNotRanked;
    for (int64_t c = tid; c < 3 * (int64_t)d.ncb; c += stride) d.front_n[c] = 0;
    for (int64_t c = tid; c < n2 + 2; c += stride) d.wcnt[c] = 0;  // front sizes of the wavefront peeling
    for (int64_t c = tid; c < d.ncb; c += stride) d.minrs[c] = INT32_MAX;
    if (in.mode == MODE_SELECT && !in.R) {
        for (int64_t j = tid; j < in.n_r; j += stride) {
            d.rho[j] = 0;
            d.lcnt[j] = 0;
        }
    } else if (in.mode == MODE_SELECT) {
        for (int64_t j = tid; j < in.n_r; j += stride) {
            double rr = 0.0;
            bool fin = true, neg = false;
            for (int k = 0; k < m; ++k) {
                float r = in.R[j * m + k];
                fin = fin && isfinite(r);
                neg = neg || r < 0.0f;
                rr += (double)r * (double)r;
            }
            if (!fin || !(rr > 0.0)) bad = true;
            if (neg) set_status(d.sc, EMO_ERR_INVALID_ARG);  // directions lie in the non-negative orthant
            double inv = fin && rr > 0.0 ? 1.0 / sqrt(rr) : 0.0;
            for (int k = 0; k < m; ++k) d.rhat[j * m + k] = (float)((double)in.R[j * m + k] * inv);
            d.rho[j] = 0;
            d.lcnt[j] = 0;
            d.rord[j] = (int32_t)j;
        }
    }
    if (bad) set_status(d.sc, EMO_ERR_NONFINITE);
}

// References in order of their polar angle from axis 1 (the index of the
// association scan), their angles from axes 1 and 2 and unit directions in
// that order.
__device__ void sort_references(const ProbDev& d, const Group& g, long long budget, RadixSmem& rsm)
{
    const int nr = d.in.n_r, m = d.in.m;
    const int gr = (int)max((int64_t)1, min((int64_t)g.size, cdiv(nr, 4096)));
    const float* rhat = d.rhat;
    auto rkey = [&](int32_t j) { return float_key(polar_angle(rhat + (int64_t)j * m, m)); };
    int rb = 0;
    for (int shift = 0; shift < 32; shift += kRadixBits) {
        bool skipped = false;
        if (!radix_pass(d, g, gr, budget, nr, d.rord + (int64_t)rb * nr, d.rord + (int64_t)(rb ^ 1) * nr, shift, rkey,
                        skipped, rsm))
            return;
        if (!skipped) rb ^= 1;
    }
    if (g.rank == 0 && threadIdx.x == 0) d.sc->rbuf = rb;
    const int32_t* ro = d.rord + (int64_t)rb * nr;
    for (int64_t s = (int64_t)g.rank * blockDim.x + threadIdx.x; s < nr; s += (int64_t)g.size * blockDim.x) {
        const int64_t j = __ldcg(&ro[s]);
        d.rphi[s] = polar_angle(rhat + j * m, m);
        d.rphi2[s] = polar_angle2(rhat + j * m, m);
        for (int k = 0; k < m; ++k) d.rsort[s * m + k] = rhat[j * m + k];
    }
}

// Lexicographic order, sorted objective keys and runs of equal points.
__global__ void __launch_bounds__(kCoopThreads, 1) k_sort(Plan* plan)
{
    const Group g = group_of(plan, false);
    if (g.prob < 0) return;  // a CTA beyond every problem's group
    const ProbDev& d = plan->p[g.prob];
    const ProbIn& in = d.in;
    const long long budget = plan->spin_budget;
    if (ld_volatile(&d.sc->status) != 0) return;
    const int64_t n2 = in.n2;
    const int m = in.m;
    const int gs = (int)max((int64_t)1, min((int64_t)g.size, cdiv(n2, 4096)));
    const float* F = in.F;
    __shared__ RadixSmem rsm;
    if (in.ranked) {  // selection from given ranks: no dominance matrix, so no point order
        if (in.mode == MODE_SELECT) sort_references(d, g, budget, rsm);
        return;
    }

    // Lexicographic order of (f_1, ..., f_m), ties by index. First a stable
    // radix sort by f_1; then every run of equal f_1 (almost always short for
    // continuous objectives) is put in (f_2, ..., f_m, index) order in place
    // by one thread. If some run is longer than kShortRun, the full stable
    // LSD sort over all objectives runs instead (from the index order).
    int buf = 0;
    const uint32_t* kor = d.sc->kor;  // written by k_prep
    const uint32_t* kinv = d.sc->kinv;
    auto sort_by = [&](int k) -> bool {
        const uint32_t varies = __ldcg(&kor[k]) & __ldcg(&kinv[k]);
        for (int shift = 0; shift < 32; shift += kRadixBits) {
            if (((varies >> shift) & (kRadix - 1)) == 0) continue;  // every point has the same digit
            const int32_t* src = d.idx + (int64_t)buf * d.n2p;
            int32_t* dst = d.idx + (int64_t)(buf ^ 1) * d.n2p;
            bool skipped = false;
            auto key = [&](int32_t v) { return float_key(__ldg(&F[(int64_t)v * m + k])); };
            if (!radix_pass(d, g, gs, budget, n2, src, dst, shift, key, skipped, rsm)) return false;
            if (!skipped) buf ^= 1;
        }
        return true;
    };
    if (!sort_by(0)) return;
    {
        constexpr int kShortRun = 32;
        int32_t* cur = d.idx + (int64_t)buf * d.n2p;
        auto key0 = [&](int64_t s) { return float_key(__ldg(&F[(int64_t)__ldcg(&cur[s]) * m])); };
        // (f_2, ..., f_m, index) order of two points
        auto before = [&](int32_t a, int32_t b) {
            for (int k = 1; k < m; ++k) {
                const uint32_t ka = float_key(__ldg(&F[(int64_t)a * m + k]));
                const uint32_t kb = float_key(__ldg(&F[(int64_t)b * m + k]));
                if (ka != kb) return ka < kb;
            }
            return a < b;
        };
        // a run's f_1 is the same at every one of its positions, so the
        // neighbours' reads below see the same keys while other threads
        // permute their own runs
        const int64_t stride = (int64_t)g.size * blockDim.x;
        for (int64_t s = (int64_t)g.rank * blockDim.x + threadIdx.x; s + 1 < n2; s += stride) {
            const uint32_t k0 = key0(s);
            if ((s > 0 && key0(s - 1) == k0) || key0(s + 1) != k0) continue;  // not the start of a run
            int64_t e = s + 2;
            while (e < n2 && e - s <= kShortRun && key0(e) == k0) ++e;
            if (e - s > kShortRun) {
                d.sc->longrun = 1;
                continue;
            }
            for (int64_t i = s + 1; i < e; ++i) {  // insertion sort, stable (reads bypass L1)
                const int32_t v = __ldcg(&cur[i]);
                int64_t j = i;
                while (j > s) {
                    const int32_t u = __ldcg(&cur[j - 1]);
                    if (!before(v, u)) break;
                    cur[j] = u;
                    --j;
                }
                cur[j] = v;
            }
        }
        if (!group_sync(d.sc, g.size, budget)) return;
        if (ld_volatile(&d.sc->longrun)) {  // full stable LSD sort from the index order
            int32_t* id = d.idx + (int64_t)(buf ^ 1) * d.n2p;
            for (int64_t s = (int64_t)g.rank * blockDim.x + threadIdx.x; s < n2; s += stride) id[s] = (int32_t)s;
            buf ^= 1;
            if (!group_sync(d.sc, g.size, budget)) return;
            for (int k = m - 1; k >= 0; --k)
                if (!sort_by(k)) return;
        }
    }
    if (g.rank == 0 && threadIdx.x == 0) d.sc->idx_buf = buf;
    const int32_t* idx = d.idx + (int64_t)buf * d.n2p;

    // objective keys 2..m in sorted order (padding = -inf), run starts
    const int64_t chunk = cdiv(d.n2p, g.size);
    const int64_t lo = min(d.n2p, chunk * g.rank), hi = min(d.n2p, lo + chunk);
    const int mk = m - 1;
    for (int64_t s = lo + threadIdx.x; s < hi; s += blockDim.x) {
        if (s < n2) {
            const int64_t v = __ldcg(&idx[s]);
            for (int k = 1; k < m; ++k) d.keys[s * mk + k - 1] = F[v * m + k] + 0.0f;
        } else {
            for (int k = 1; k < m; ++k) d.keys[s * mk + k - 1] = -INFINITY;
        }
    }
    auto is_start = [&](int64_t s) -> bool {
        if (s == 0 || s >= n2) return true;
        const int64_t a = __ldcg(&idx[s]), b = __ldcg(&idx[s - 1]);
        for (int k = 0; k < m; ++k)
            if (F[a * m + k] != F[b * m + k]) return true;
        return false;
    };
    // inclusive max-scan of (start ? s : 0) across the group
    __shared__ int s_warp[33];
    int local = -1;
    for (int64_t s = lo + threadIdx.x; s < hi; s += blockDim.x)
        if (is_start(s)) local = max(local, (int)s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local = max(local, __shfl_xor_sync(0xffffffffu, local, o));
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        int mx = -1;
        for (int w = 0; w < kCoopThreads / 32; ++w) mx = max(mx, s_warp[w]);
        d.hist[g.rank] = mx;
    }
    if (!group_sync(d.sc, g.size, budget)) return;
    __shared__ int s_carry;
    if (threadIdx.x == 0) {
        int c = 0;
        for (int r = 0; r < g.rank; ++r) c = max(c, __ldcg(&d.hist[r]));
        s_carry = c;
    }
    __syncthreads();
    int carry = s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = lo; base < hi; base += blockDim.x) {
        const int64_t s = base + threadIdx.x;
        int v = (s < hi && is_start(s)) ? (int)s : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v = max(v, y);
        }
        if (lane == 31) s_warp[warp] = v;
        __syncthreads();
        int pre = carry;
        for (int w = 0; w < warp; ++w) pre = max(pre, s_warp[w]);
        int rs = max(pre, v);
        if (s < hi) {
            d.runstart[s] = rs;
            if (rs < s) atomicMin(&d.minrs[s / kColBlock], rs);
        }
        __syncthreads();
        int tmax = carry;
        for (int w = 0; w < kCoopThreads / 32; ++w) tmax = max(tmax, s_warp[w]);
        carry = tmax;
        __syncthreads();
    }

    // every CTA has read the run-start carries from d.hist before the radix
    // passes of the references reuse it
    if (in.mode != MODE_SELECT) return;
    if (!group_sync(d.sc, g.size, budget)) return;
    sort_references(d, g, budget, rsm);
}

}  // namespace emo
