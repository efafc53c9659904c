// Kernels of the split of one population over several GPUs (column blocks
// of the dominance matrix owned by ranks; Algorithm S.3 with the front
// membership exchanged between ranks after every front):
//   k_front_counts -- the peeling step of one rank: subtract the rows of the
//     current front from the dominator counts of the rank's columns and flag
//     the columns whose count reaches zero (the next front there);
//   k_rank_in -- the selection of a population whose ranks are already
//     known (computed by the ranks together): l, |P|, |L|, the caller-order
//     ranks and the list of S, in place of the sorting-based peeling;
//   k_assoc_out -- the association step of one rank (its points of S
//     associated after the normalisation over all of S): the references and
//     FP64 distances of its points and the niche counts of its points of P,
//     which the ranks add up (an all-reduce of n_r counts);
//   k_given_in -- the niching from the gathered association: the summed
//     niche counts and the references and distances of front l, checked
//     against the ranks, in place of the association.
#include <algorithm>

#include "emo_kernels.cuh"

namespace emo {

constexpr int kFrontThreads = 256;
constexpr int kFrontNH = 17;  // counter planes above four: up to 2^21 - 1 rows

// One thread per 32-column word of the rank's D: the front's rows are added
// into bit-sliced counters (16 rows at a time), then the 32 column counts are
// subtracted from the dominator counts.
__global__ void __launch_bounds__(kFrontThreads) k_front_counts(const uint32_t* __restrict__ D, int64_t ld,
                                                                 int64_t ncols, const int32_t* __restrict__ rows,
                                                                 int64_t n_rows, int32_t* counts, uint8_t* new_front)
{
    const int64_t nwords = cdiv(ncols, 32);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += stride) {
        VCount<kFrontNH> vc;
        for (int64_t r0 = 0; r0 < n_rows; r0 += 16) {
            uint32_t x[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) x[j] = r0 + j < n_rows ? __ldg(&D[(int64_t)__ldg(&rows[r0 + j]) * ld + w]) : 0u;
            vc.add16(x);
        }
        for (int b = 0; b < 32; ++b) {
            const int64_t j = w * 32 + b;
            if (j >= ncols) break;
            const int dq = vc.count(b);
            const int before = counts[j];
            const int after = before - dq;
            if (dq) counts[j] = after;
            new_front[j] = (uint8_t)(dq > 0 && after == 0);
        }
    }
}

// Selection from given ranks (narrow cooperative group): histogram of the
// ranks, l = the rank of the n_keep-th best point, |P| and |L|, then the
// caller-order ranks (beyond l: not ranked) and the list of S.
__global__ void __launch_bounds__(kCoopThreads, 1) k_rank_in(Plan* plan)
{
    __shared__ int s_warp[33];
    __shared__ int s_l, s_np, s_nl;
    const Group g = group_of(plan, false);
    if (g.prob < 0) return;  // a CTA beyond every problem's group
    const ProbDev& d = plan->p[g.prob];
    const ProbIn& in = d.in;
    const long long budget = plan->spin_budget;
    if (!in.ranked || ld_volatile(&d.sc->status) != 0) return;
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t n2 = in.n2;
    const int64_t t0 = (int64_t)g.rank * blockDim.x + tid;
    const int64_t stride = (int64_t)g.size * blockDim.x;
    for (int64_t i = t0; i < n2; i += stride) {
        const int r = in.rank_in[i];
        if (r == kNotRanked) continue;
        if (r < 0 || r >= n2) set_status(d.sc, EMO_ERR_INVALID_ARG);
        else atomicAdd(&d.wcnt[r], 1);
    }
    if (!group_sync(d.sc, g.size, budget)) return;
    if (g.rank == 0) {
        if (tid == 0) s_l = -1;
        int run = 0;
        for (int64_t base = 0; base < n2; base += blockDim.x) {
            const int64_t k = base + tid;
            const int v = k < n2 ? __ldcg(&d.wcnt[k]) : 0;
            int tot;
            const int pre = block_exclusive_scan<kCoopThreads>(v, s_warp, tot);
            if (v > 0 && run + pre < in.n_keep && in.n_keep <= run + pre + v) {
                s_l = (int)k;
                s_np = run + pre;
                s_nl = v;
            }
            run += tot;
            __syncthreads();
            if (s_l >= 0) break;
        }
        if (tid == 0) {
            if (s_l < 0) {
                set_status(d.sc, EMO_ERR_INVALID_ARG);  // fewer than n_keep ranked points
            } else {
                d.sc->l = s_l;
                d.sc->nP = s_np;
                d.sc->nL = s_nl;
                d.sc->nfronts = s_l + 1;
                if (in.last_rank_out) *in.last_rank_out = s_l;
            }
        }
    }
    if (!group_sync(d.sc, g.size, budget)) return;
    const int l = ld_volatile(&d.sc->l);
    for (int64_t s0 = (int64_t)g.rank * blockDim.x; s0 < n2; s0 += stride) {
        const int64_t i = s0 + tid;
        int r = kNotRanked;
        if (i < n2) {
            r = in.rank_in[i];
            if (r > l) r = kNotRanked;
            d.rank_o[i] = r;
        }
        const bool inS = i < n2 && r <= l;
        const unsigned mask = __ballot_sync(0xffffffffu, inS);
        int base = 0;
        if (lane == 0 && mask) base = atomicAdd(&d.sc->nS, __popc(mask));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (inS) d.slist[base + __popc(mask & lanemask_lt())] = (int32_t)i;
    }
}

// Outputs of the association of one rank's points [col_lo, col_hi) (narrow
// cooperative group): reference and distance of each point of S in the
// range, then the niche counts of the range's points of P.
__global__ void __launch_bounds__(kCoopThreads, 1) k_assoc_out(Plan* plan)
{
    const Group g = group_of(plan, false);
    if (g.prob < 0) return;  // a CTA beyond every problem's group
    const SplitArgs& sp = plan->split;
    const ProbDev& d = plan->p[g.prob];
    Scal* sc = d.sc;
    if (sp.kind != SPLIT_ASSOC || ld_volatile(&sc->status) != 0) return;
    const int l = __ldcg(&sc->l);
    const int64_t t0 = (int64_t)g.rank * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)g.size * blockDim.x;
    for (int64_t i = sp.col_lo + t0; i < sp.col_hi; i += stride) {
        const int r = __ldcg(&d.rank_o[i]);
        const bool inS = r <= l;
        const int p = inS ? __ldcg(&d.pi[i]) : -1;
        sp.pi_out[i - sp.col_lo] = p;
        sp.d_out[i - sp.col_lo] = inS ? __ldcg(&d.d64[i]) : (double)NAN;
        if (r < l) atomicAdd(&d.rho[p], 1);
    }
    if (!group_sync(sc, g.size, plan->spin_budget)) return;
    for (int64_t j = t0; j < d.in.n_r; j += stride) sp.rho[j] = __ldcg(&d.rho[j]);
}

// The association gathered from the ranks of a split population (narrow
// cooperative group, after k_rank_in): the niche counts of P, and the
// reference and distance of every member of front l, which must be given in
// ascending caller order, each of rank l, |L| of them (so exactly front l).
__global__ void __launch_bounds__(kCoopThreads, 1) k_given_in(Plan* plan)
{
    const Group g = group_of(plan, false);
    if (g.prob < 0) return;  // a CTA beyond every problem's group
    const SplitArgs& sp = plan->split;
    const ProbDev& d = plan->p[g.prob];
    Scal* sc = d.sc;
    if (sp.kind != SPLIT_NICHE || ld_volatile(&sc->status) != 0) return;
    const int l = __ldcg(&sc->l), nL = __ldcg(&sc->nL);
    const int64_t n2 = d.in.n2;
    const int nr = d.in.n_r;
    const int64_t t0 = (int64_t)g.rank * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)g.size * blockDim.x;
    if (sp.n_last != nL) {
        if (g.rank == 0 && threadIdx.x == 0) set_status(sc, EMO_ERR_INVALID_ARG);
        return;
    }
    for (int64_t t = t0; t < sp.n_last; t += stride) {
        const int32_t v = sp.last[t];
        const int32_t p = sp.last_pi[t];
        const double dd = sp.last_d[t];
        bool good = v >= 0 && v < n2 && (t == 0 || sp.last[t - 1] < v) && p >= 0 && p < nr && isfinite(dd) &&
                    dd >= 0.0;
        if (good) good = __ldcg(&d.rank_o[v]) == l;
        if (!good) {
            set_status(sc, EMO_ERR_INVALID_ARG);
        } else {
            d.pi[v] = p;
            d.d64[v] = dd;
        }
    }
    unsigned long long part = 0;
    for (int64_t j = t0; j < nr; j += stride) {
        const int32_t r = sp.rho[j];
        if (r < 0) {
            set_status(sc, EMO_ERR_INVALID_ARG);
        } else {
            d.rho[j] = r;
            part += (unsigned long long)r;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0 && part) atomicAdd(&sc->rho_sum, part);
}

cudaError_t launch_front_counts(const uint32_t* D, int64_t ld, int64_t ncols, const int32_t* rows, int64_t n_rows,
                                int32_t* counts, uint8_t* new_front, int sms, cudaStream_t s)
{
    const int64_t nwords = cdiv(ncols, 32);
    const int64_t need = cdiv(nwords, kFrontThreads);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * 8));
    k_front_counts<<<grid, kFrontThreads, 0, s>>>(D, ld, ncols, rows, n_rows, counts, new_front);
    return cudaGetLastError();
}

}  // namespace emo
