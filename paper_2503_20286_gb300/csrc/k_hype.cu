// TensorHypE environmental selection (Algorithm S.10) with the Monte Carlo
// hypervolume estimation of Algorithm S.11, after the ranks and l of the
// shared front peeling. Three launches per call:
//   k_hype phase 0 (cooperative):
//   (A) f_l = column minima of F; F and v_ref finite; the points of front l
//       in ascending index order (the list L); sample counts cleared;
//   (B) samples S_i = f_l + U_i (v_ref - f_l) in float (subtract, multiply,
//       add; no fused multiply-add);
//   k_hype_counts:
//   (C) c_i = points weakly dominating S_i, from the column-block prefix sets
//       of the dominance stage (see the kernel);
//   k_hype phase 1 (cooperative):
//       the weights alpha_c for c <= k (one thread, in order: lambda_1 = 1,
//       lambda_c = (k - c + 1) / (n2 - c + 1), alpha_c = (lambda_1 ...
//       lambda_c) / c; alpha_c = 0 beyond k);
//   (D) each point of L (one warp, samples staged in shared memory): its
//       contribution, vol / s times the sum of alpha_{c_i} over the samples
//       it dominates in sample order (double);
//   (E) L sorted stably by (contribution descending) with 64-bit radix passes;
//       its first n_keep - |P| points are flagged as survivors.
#include <cfloat>

#include "emo_kernels.cuh"
#include "group_radix.cuh"

namespace emo {

constexpr int kHypeTile = 6144;  // floats of the shared-memory tile (sample staging)
constexpr long long kHypeCopyWaitCycles = 1ll << 32;

// Slot of entry i of a block's descending values in the prefix-set layout
// (the bank-spreading swizzle of the column-block preparation).
__device__ __forceinline__ int hype_fv_slot(int i) { return i ^ ((i >> 5) & 31); }

// Order-preserving 64-bit key of a double, largest first (0 and -0 equal).
__device__ __forceinline__ unsigned long long hype_desc_key(double v)
{
    if (v == 0.0) v = 0.0;
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned long long ordered = (b >> 63) ? ~b : (b | 0x8000000000000000ull);
    return ~ordered;
}

__device__ __forceinline__ void hype_contributions(const Plan* plan, const Group& g, const ProbDev& d, float* s_pts,
                                                   RadixSmem& rsm);

// phase 0: (A) and (B); phase 1: the weights, (D) and (E).
__global__ void __launch_bounds__(kCoopThreads, 1) k_hype(Plan* plan, int phase)
{
    __shared__ __align__(16) float s_pts[kHypeTile];
    __shared__ RadixSmem rsm;
    __shared__ uint32_t s_key[kMaxM];
    const Group g = group_of(plan, true);
    if (g.prob < 0) return;  // a CTA beyond every problem's group
    const ProbDev& d = plan->p[g.prob];
    const ProbIn& in = d.in;
    const long long budget = plan->spin_budget;
    if (in.mode != MODE_HYPE || ld_volatile(&d.sc->status) != 0) return;
    if (phase == 1) {
        hype_contributions(plan, g, d, s_pts, rsm);
        return;
    }
    Scal* sc = d.sc;
    const int m = in.m, tid = threadIdx.x;
    const int64_t n2 = in.n2;
    const int ns = in.n_r;
    const float* F = in.F;
    const float* vref = in.R;
    const int64_t t0 = (int64_t)g.rank * blockDim.x + tid;
    const int64_t stride = (int64_t)g.size * blockDim.x;
    const int l = ld_volatile(&sc->l);

    // (A) column minima of F (max of the inverted order-preserving keys), checks, L
    if (tid < kMaxM) s_key[tid] = 0u;
    __syncthreads();
    {
        uint32_t best[kMaxM];
        for (int k = 0; k < m; ++k) best[k] = 0u;
        for (int64_t i = t0; i < n2; i += stride)
            for (int k = 0; k < m; ++k) best[k] = max(best[k], ~float_key(F[i * m + k]));
        for (int k = 0; k < m; ++k) atomicMax(&s_key[k], best[k]);
    }
    __syncthreads();
    if (tid < m) atomicMax(&sc->zkey[tid], s_key[tid]);
    if (g.rank == 0 && tid < m && !isfinite(vref[tid])) set_status(sc, EMO_ERR_NONFINITE);
    for (int64_t i = t0; i < (int64_t)ns * m; i += stride)
        if (!isfinite(in.U[i])) set_status(sc, EMO_ERR_NONFINITE);
    for (int64_t i = t0; i < ns; i += stride) d.rho[i] = 0;
    bool ok = true;
    int32_t* L = d.llist;
    group_compact(
        d, g, budget, n2, [&](int64_t i) { return __ldcg(&d.rank_o[i]) == l; },
        [&](int pos, int64_t i) { L[pos] = (int32_t)i; }, ok);  // |L| = sc->nL
    if (!ok) return;

    // (B) samples
    float fl[kMaxM];
    for (int k = 0; k < m; ++k) fl[k] = key_float(~__ldcg(&sc->zkey[k]));
    for (int64_t i = t0; i < (int64_t)ns * m; i += stride) {
        const int k = (int)(i % m);
        const float width = __fsub_rn(vref[k], fl[k]);
        d.rhat[i] = __fadd_rn(fl[k], __fmul_rn(in.U[i], width));
    }
    return;
}

// Phase 1 of k_hype: the weights, (D) and (E).
__device__ __forceinline__ void hype_contributions(const Plan* plan, const Group& g, const ProbDev& d, float* s_pts,
                                                   RadixSmem& rsm)
{
    const ProbIn& in = d.in;
    const long long budget = plan->spin_budget;
    Scal* sc = d.sc;
    const int m = in.m, tid = threadIdx.x;
    const int64_t n2 = in.n2;
    const int ns = in.n_r;
    const float* F = in.F;
    const float* vref = in.R;
    const int64_t t0 = (int64_t)g.rank * blockDim.x + tid;
    const int64_t stride = (int64_t)g.size * blockDim.x;
    const int l = ld_volatile(&sc->l);
    const int64_t nP = ld_volatile(&sc->nP);
    const int64_t nL = ld_volatile(&sc->nL);
    const int64_t want = in.n_keep - nP;  // points of front l that survive
    const int32_t* L = d.llist;           // front l, ascending (phase 0)
    float fl[kMaxM];
    for (int k = 0; k < m; ++k) fl[k] = key_float(~__ldcg(&sc->zkey[k]));
    // the weights alpha_c, c = 1 .. min(k, n2): prod_c = prod_{c-1} *
    // ((k - (c - 1)) / (n2 - (c - 1))) in order from prod_1 = 1, alpha_c =
    // prod_c / c. The ratios and the final divisions are independent (the CTA
    // of rank 0 spreads them over its threads); only the chain of products is
    // sequential (one thread), so every value is rounded as in the plain loop.
    const int64_t kdrop = (nP + nL) - in.n_keep;
    double* alpha = reinterpret_cast<double*>(d.ekeys);
    if (g.rank == 0) {
        const int64_t cmax = min(kdrop, n2);
        for (int64_t c = 2 + tid; c <= cmax; c += blockDim.x)
            alpha[c] = __ddiv_rn((double)(kdrop - (c - 1)), (double)(n2 - (c - 1)));
        __syncthreads();
        if (tid == 0) {
            double prod = 1.0;
            if (cmax >= 1) alpha[1] = 1.0;
            for (int64_t c = 2; c <= cmax; ++c) {
                prod = __dmul_rn(prod, alpha[c]);
                alpha[c] = prod;
            }
        }
        __syncthreads();
        for (int64_t c = 1 + tid; c <= cmax; c += blockDim.x) alpha[c] = __ddiv_rn(alpha[c], (double)c);
    }
    if (!group_sync(sc, g.size, budget)) return;

    // (D) contributions of the points of front l: one warp per point; the
    // samples and their weights alpha_{c_i} (0 beyond c = k, or when no point
    // dominates the sample) pass through shared memory in tiles, each lane
    // tests one sample, and the weights of the dominated samples with a
    // non-zero weight are added in sample order (ballot bits ascending);
    // adding a zero would leave the sum unchanged
    double vol = 1.0;
    for (int k = 0; k < m; ++k) vol = __dmul_rn(vol, __dsub_rn((double)vref[k], (double)fl[k]));
    {
        const int lane = tid & 31, nwb = blockDim.x >> 5;
        const int ts = (kHypeTile * 4) / (4 * m + 8);  // samples per tile (m floats and a double weight each)
        double* s_w = reinterpret_cast<double*>(s_pts);
        float* s_smp = reinterpret_cast<float*>(s_w + ts);
        const int64_t nw_all = (int64_t)g.size * nwb, gw = (int64_t)g.rank * nwb + (tid >> 5);
        for (int64_t b0 = 0; b0 < nL; b0 += nw_all) {  // the same trip count in every CTA
            const int64_t t = b0 + gw;
            const bool has = t < nL;
            const int64_t p = has ? __ldcg(&L[t]) : 0;
            float f[kMaxM];
            for (int k = 0; k < m; ++k) f[k] = has ? F[p * m + k] : 0.0f;
            double v = 0.0;
            for (int i0 = 0; i0 < ns; i0 += ts) {
                const int nt = min(ts, ns - i0);
                __syncthreads();
                for (int e = tid; e < nt * m; e += blockDim.x) s_smp[e] = __ldcg(&d.rhat[(int64_t)i0 * m + e]);
                for (int e = tid; e < nt; e += blockDim.x) {
                    const int c = __ldcg(&d.rho[i0 + e]);
                    s_w[e] = (c >= 1 && c <= kdrop) ? __ldcg(&alpha[c]) : 0.0;
                }
                __syncthreads();
                if (!has) continue;
                for (int j0 = 0; j0 < nt; j0 += 32) {
                    const int j = j0 + lane;
                    bool dom = j < nt && s_w[j < nt ? j : 0] != 0.0;
                    for (int k = 0; k < m; ++k) dom &= f[k] <= s_smp[(j < nt ? j : 0) * m + k];
                    unsigned mask = __ballot_sync(0xffffffffu, dom);
                    while (mask) {
                        const int b = __ffs(mask) - 1;
                        mask &= mask - 1;
                        v = __dadd_rn(v, s_w[j0 + b]);
                    }
                }
            }
            if (has && lane == 0) {
                const double hv = __ddiv_rn(__dmul_rn(v, vol), (double)ns);
                d.d64[p] = hv;
                if (in.hv_out) in.hv_out[p] = hv;
            }
        }
    }
    if (in.hv_out)
        for (int64_t i = t0; i < n2; i += stride)
            if (__ldcg(&d.rank_o[i]) != l) in.hv_out[i] = 0.0;
    if (!group_sync(sc, g.size, budget)) return;

    // (E) L by contribution descending (stable: ties keep the index order)
    if (want >= nL) {
        for (int64_t t = t0; t < nL; t += stride) d.flag[__ldcg(&L[t])] = 1;
        return;
    }
    const int gs = (int)max((int64_t)1, min((int64_t)g.size, cdiv(nL, 4096)));
    int buf = 0;
    for (int shift = 0; shift < 64; shift += kRadixBits) {
        const int32_t* src = d.llist + (int64_t)buf * n2;
        int32_t* dst = d.llist + (int64_t)(buf ^ 1) * n2;
        bool skipped = false;
        auto key = [&](int32_t v) {
            const unsigned long long k64 = hype_desc_key(__ldcg(&d.d64[v]));
            return shift < 32 ? (uint32_t)k64 : (uint32_t)(k64 >> 32);
        };
        if (!radix_pass(d, g, gs, budget, nL, src, dst, shift & 31, key, skipped, rsm)) return;
        if (!skipped) buf ^= 1;
    }
    const int32_t* sorted = d.llist + (int64_t)buf * n2;
    for (int64_t t = t0; t < want; t += stride) d.flag[__ldcg(&sorted[t])] = 1;
}

// (C) The dominator count c_i of every sample, from the column-block prefix
// sets that the dominance stage built (points in lexicographic order). In
// column block cb the points with f_1 <= s_1 are its first t1 positions (f_1
// ascends along the order); for each key objective k >= 2 the points with
// f_k <= s_k are the complement of the block's prefix of f_k-descending
// order that holds the values > s_k (one prefix bitset per half of 512
// columns, plus at most cps - 1 single bits). So
//   c_i = sum over blocks of popc(first-t1 mask AND complemented prefix sets),
// the count of every point with F_p <= S_i in all objectives. Items are
// (column block, range of samples): the CTA copies the block's prefix data
// (all key objectives, contiguous) into shared memory with one bulk copy and
// gathers the block's f_1 values; each warp then takes 32 samples at a time:
// lane = sample for the binary searches (t1 and the packed half counts), then
// lane = word of the block for each of the 32 samples (AND, popcount, warp
// sum), and one atomic add per sample and item.
// The samples [s_lo, s_hi) against the staged column block (see
// k_hype_counts). MM = m at compile time, or kMaxM for any m (the arrays are
// then sized for the largest m and the loops run to the problem's m).
template <int MM>
__device__ __forceinline__ void hype_count_block(const ProbDev& d, const unsigned char* smraw, const float* s_f1,
                                                 int64_t s_lo, int64_t s_hi, int nvalid, int64_t obj_bytes,
                                                 int64_t ord_off, int log_cps)
{
    const int m = MM == kMaxM ? d.in.m : MM, K = m - 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int half = lane >> 4;
    for (int64_t s0 = s_lo + (int64_t)warp * 32; s0 < s_hi; s0 += (int64_t)nw * 32) {
        const int64_t si = s0 + lane;
        const bool live = si < s_hi;
        float sv[MM];
#pragma unroll
        for (int k = 0; k < MM; ++k) sv[k] = (live && k < m) ? __ldcg(&d.rhat[si * m + k]) : -INFINITY;
        // lane = sample: positions with f_1 <= s_1, and per key objective the
        // counts of values > s_k in each half (packed t0 | t1 << 16)
        int t1;
        {
            int pos = 0;
#pragma unroll
            for (int step = kColBlock / 2; step > 0; step >>= 1)
                if (s_f1[pos + step - 1] <= sv[0]) pos += step;
            if (s_f1[pos] <= sv[0]) ++pos;
            t1 = live ? min(pos, nvalid) : 0;
        }
        if (!__any_sync(0xffffffffu, t1 > 0)) continue;
        int packed[MM - 1];
#pragma unroll
        for (int k = 0; k < MM - 1; ++k) {
            packed[k] = 0;
            if (k < K) {
                const unsigned char* ob = smraw + (int64_t)k * obj_bytes;
                const float* fv = reinterpret_cast<const float*>(ob);
                const float x = sv[k + 1];
                int pos = 0;
#pragma unroll
                for (int step = kColBlock / 2; step > 0; step >>= 1)
                    if (fv[hype_fv_slot(pos + step - 1)] > x) pos += step;
                if (fv[hype_fv_slot(pos)] > x) ++pos;
                const int h0 = reinterpret_cast<const uint16_t*>(ob + kPrefCumOff)[pos];
                packed[k] = h0 | ((pos - h0) << 16);
            }
        }
        // lane = word (block columns 32 lane .. 32 lane + 31)
        int acc = 0;
        for (int j = 0; j < 32; ++j) {
            const int tj = __shfl_sync(0xffffffffu, t1, j);
            if (tj == 0) continue;  // uniform over the warp
            uint32_t w = tj >= 32 * (lane + 1) ? 0xffffffffu : (tj <= 32 * lane ? 0u : (1u << (tj - 32 * lane)) - 1u);
#pragma unroll
            for (int k = 0; k < MM - 1; ++k) {  // every lane: the loop holds warp shuffles
                if (k < K) {
                    const int pk = __shfl_sync(0xffffffffu, packed[k], j);
                    const int th = half ? (pk >> 16) : (pk & 0xffff);
                    const unsigned char* ob = smraw + (int64_t)k * obj_bytes;
                    const int c = th >> log_cps;
                    uint32_t pre = reinterpret_cast<const uint32_t*>(ob + kPrefPbOff)[c * 32 + lane];
                    if (log_cps > 0) {
                        const uint16_t* ord = reinterpret_cast<const uint16_t*>(ob + ord_off) + half * (kColBlock / 2);
                        for (int e = c << log_cps; e < th; ++e) {
                            const int col = ord[e];
                            if ((col >> 5) == lane) pre |= 1u << (col & 31);  // col: block-local
                        }
                    }
                    w &= ~pre;
                }
            }
            const int tot = __reduce_add_sync(0xffffffffu, __popc(w));
            if (lane == j) acc = tot;
        }
        if (live && acc) atomicAdd(&d.rho[si], acc);
    }
}

__global__ void __launch_bounds__(kCoopThreads, 1) k_hype_counts(Plan* plan)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ uint64_t s_bar;
    __shared__ int s_skip;
    const int tid = threadIdx.x;
    if (tid == 0) mbar_init(&s_bar, 1);
    __syncthreads();
    uint32_t parity = 0;
    for (int p = 0; p < plan->nprob; ++p) {
        const ProbDev& d = plan->p[p];
        const ProbIn& in = d.in;
        if (in.mode != MODE_HYPE) continue;
        const int m = in.m, K = m - 1, ns = in.n_r, ncb = d.ncb;
        const int64_t n2 = in.n2;
        const int log_cps = colprep_log_cps(K);
        const int64_t obj_bytes = colprep_obj_bytes(K), ord_off = colprep_ord_off(K);
        const uint32_t blk_bytes = (uint32_t)(K * obj_bytes);
        float* s_f1 = reinterpret_cast<float*>(smraw + align_up(blk_bytes, 128));
        const int32_t* idx = d.idx + (int64_t)ld_volatile(&d.sc->idx_buf) * d.n2p;
        const int64_t nsr = max((int64_t)1, min(cdiv(ns, 32), cdiv(2 * (int64_t)gridDim.x, ncb)));
        for (int64_t item = blockIdx.x; item < (int64_t)ncb * nsr; item += gridDim.x) {
            const int cb = (int)(item / nsr);
            const int64_t sr = item % nsr, s_lo = sr * ns / nsr, s_hi = (sr + 1) * ns / nsr;
            const int64_t base = (int64_t)cb * kColBlock;
            const int nvalid = (int)min((int64_t)kColBlock, n2 - base);
            __syncthreads();  // the previous item is done with the staged block
            if (tid == 0) {
                s_skip = ld_volatile(&d.sc->status) != 0;
                if (!s_skip) {
                    fence_proxy_async_smem();
                    bulk_load(smraw, d.colpre + (int64_t)cb * blk_bytes, blk_bytes, &s_bar);
                }
            }
            for (int q = tid; q < kColBlock; q += blockDim.x)
                s_f1[q] = q < nvalid ? in.F[(int64_t)__ldcg(&idx[base + q]) * m] : INFINITY;
            __syncthreads();
            if (s_skip) return;
            if (!mbar_wait(&s_bar, parity, kHypeCopyWaitCycles)) {
                // a local copy always completes; the bound only guards against a
                // lost completion (wait again so that no copy is in flight at exit)
                if (tid == 0) set_status(d.sc, EMO_ERR_TIMEOUT);
                mbar_wait(&s_bar, parity, kHypeCopyWaitCycles);
                return;
            }
            parity ^= 1u;
            switch (m) {  // compile-time objective counts keep the per-sample state in registers
            case 2: hype_count_block<2>(d, smraw, s_f1, s_lo, s_hi, nvalid, obj_bytes, ord_off, log_cps); break;
            case 3: hype_count_block<3>(d, smraw, s_f1, s_lo, s_hi, nvalid, obj_bytes, ord_off, log_cps); break;
            case 4: hype_count_block<4>(d, smraw, s_f1, s_lo, s_hi, nvalid, obj_bytes, ord_off, log_cps); break;
            default: hype_count_block<kMaxM>(d, smraw, s_f1, s_lo, s_hi, nvalid, obj_bytes, ord_off, log_cps);
            }
        }
    }
}

// Bytes of dynamic shared memory k_hype_counts needs for m objectives.
int hype_counts_smem(int m)
{
    const int K = m - 1;
    return (int)(align_up(K * colprep_obj_bytes(K), 128) + kColBlock * 4);
}

}  // namespace emo
