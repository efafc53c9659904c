// TensorHypE environmental selection (Algorithm S.10) with the Monte Carlo
// hypervolume estimation of Algorithm S.11, after the ranks and l of the
// shared front peeling. One cooperative launch per call, phases separated by
// bounded group barriers:
//   (A) f_l = column minima of F; F and v_ref finite; the points of front l
//       in ascending index order (the list L); sample counts cleared;
//   (B) samples S_i = f_l + U_i (v_ref - f_l) in float (subtract, multiply,
//       add; no fused multiply-add);
//   (C) c_i = points weakly dominating S_i: tiles of points in shared memory,
//       one sample per thread; the weights alpha_c for c <= k (one thread, in
//       order: lambda_1 = 1, lambda_c = (k - c + 1) / (n2 - c + 1), alpha_c =
//       (lambda_1 ... lambda_c) / c; alpha_c = 0 beyond k);
//   (D) each point of L (one warp, samples staged in shared memory): its
//       contribution, vol / s times the sum of alpha_{c_i} over the samples
//       it dominates in sample order (double);
//   (E) L sorted stably by (contribution descending) with 64-bit radix passes;
//       its first n_keep - |P| points are flagged as survivors.
#include <cfloat>

#include "emo_kernels.cuh"
#include "group_radix.cuh"

namespace emo {

constexpr int kHypeTile = 6144;  // floats of the point tile in shared memory

// Points of a shared-memory tile that weakly dominate sample smp (compile-time m).
template <int M>
__device__ __forceinline__ int count_dominators(const float* __restrict__ pts, int np, const float* smp)
{
    float sv[M];
#pragma unroll
    for (int k = 0; k < M; ++k) sv[k] = smp[k];
    int cnt = 0;
#pragma unroll 4
    for (int q = 0; q < np; ++q) {
        bool dom = true;
#pragma unroll
        for (int k = 0; k < M; ++k) dom &= pts[q * M + k] <= sv[k];
        cnt += dom ? 1 : 0;
    }
    return cnt;
}
__device__ __forceinline__ int count_dominators_rt(const float* __restrict__ pts, int np, const float* smp, int m)
{
    int cnt = 0;
    for (int q = 0; q < np; ++q) {
        bool dom = true;
        for (int k = 0; k < m; ++k) dom &= pts[q * m + k] <= smp[k];
        cnt += dom ? 1 : 0;
    }
    return cnt;
}

// Order-preserving 64-bit key of a double, largest first (0 and -0 equal).
__device__ __forceinline__ unsigned long long hype_desc_key(double v)
{
    if (v == 0.0) v = 0.0;
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned long long ordered = (b >> 63) ? ~b : (b | 0x8000000000000000ull);
    return ~ordered;
}

__global__ void __launch_bounds__(kCoopThreads, 1) k_hype(Plan* plan)
{
    __shared__ float s_pts[kHypeTile];
    __shared__ RadixSmem rsm;
    __shared__ uint32_t s_key[kMaxM];
    const Group g = group_of(plan, true);
    if (g.prob < 0) return;  // a CTA beyond every problem's group
    const ProbDev& d = plan->p[g.prob];
    const ProbIn& in = d.in;
    const long long budget = plan->spin_budget;
    if (in.mode != MODE_HYPE || ld_volatile(&d.sc->status) != 0) return;
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
    const int64_t want = in.n_keep - nP;  // points of front l that survive

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
    const int nL = group_compact(
        d, g, budget, n2, [&](int64_t i) { return __ldcg(&d.rank_o[i]) == l; },
        [&](int pos, int64_t i) { L[pos] = (int32_t)i; }, ok);
    if (!ok) return;

    // (B) samples
    float fl[kMaxM];
    for (int k = 0; k < m; ++k) fl[k] = key_float(~__ldcg(&sc->zkey[k]));
    for (int64_t i = t0; i < (int64_t)ns * m; i += stride) {
        const int k = (int)(i % m);
        const float width = __fsub_rn(vref[k], fl[k]);
        d.rhat[i] = __fadd_rn(fl[k], __fmul_rn(in.U[i], width));
    }
    if (!group_sync(sc, g.size, budget)) return;

    // (C) dominator count of every sample: items (512 samples, one tile of points)
    const int tp = kHypeTile / m;  // points per tile
    const int64_t nsb = cdiv(ns, (int64_t)blockDim.x), ntile = cdiv(n2, (int64_t)tp);
    for (int64_t item = g.rank; item < nsb * ntile; item += g.size) {
        const int64_t sb = item / ntile, tile = item % ntile;
        const int64_t p0 = tile * tp, np = min((int64_t)tp, n2 - p0);
        __syncthreads();
        for (int64_t e = tid; e < np * m; e += blockDim.x) s_pts[e] = F[p0 * m + e];
        __syncthreads();
        const int64_t si = sb * blockDim.x + tid;
        if (si < ns) {
            float smp[kMaxM];
            for (int k = 0; k < m; ++k) smp[k] = __ldcg(&d.rhat[si * m + k]);
            int cnt;
            switch (m) {
            case 2: cnt = count_dominators<2>(s_pts, (int)np, smp); break;
            case 3: cnt = count_dominators<3>(s_pts, (int)np, smp); break;
            case 4: cnt = count_dominators<4>(s_pts, (int)np, smp); break;
            case 5: cnt = count_dominators<5>(s_pts, (int)np, smp); break;
            case 6: cnt = count_dominators<6>(s_pts, (int)np, smp); break;
            default: cnt = count_dominators_rt(s_pts, (int)np, smp, m);
            }
            if (cnt) atomicAdd(&d.rho[si], cnt);
        }
    }
    // the weights alpha_c, c = 1 .. min(k, n2), in order (one thread)
    const int64_t kdrop = (nP + nL) - in.n_keep;
    double* alpha = reinterpret_cast<double*>(d.ekeys);
    if (g.rank == 0 && tid == 0) {
        double prod = 1.0;
        const int64_t cmax = min(kdrop, n2);
        for (int64_t c = 1; c <= cmax; ++c) {
            if (c >= 2) prod = __dmul_rn(prod, __ddiv_rn((double)(kdrop - (c - 1)), (double)(n2 - (c - 1))));
            alpha[c] = __ddiv_rn(prod, (double)c);
        }
    }
    if (!group_sync(sc, g.size, budget)) return;

    // (D) contributions of the points of front l: one warp per point; the
    // samples and their counts pass through shared memory in tiles, each lane
    // tests one sample, and the weights of the dominated ones are added in
    // sample order (ballot bits ascending)
    double vol = 1.0;
    for (int k = 0; k < m; ++k) vol = __dmul_rn(vol, __dsub_rn((double)vref[k], (double)fl[k]));
    {
        const int lane = tid & 31, nwb = blockDim.x >> 5;
        const int ts = kHypeTile / (m + 1);  // samples per tile (m floats and a count each)
        float* s_smp = s_pts;
        int* s_cnt = reinterpret_cast<int*>(s_pts + ts * m);
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
                for (int e = tid; e < nt; e += blockDim.x) s_cnt[e] = __ldcg(&d.rho[i0 + e]);
                __syncthreads();
                if (!has) continue;
                for (int j0 = 0; j0 < nt; j0 += 32) {
                    const int j = j0 + lane;
                    bool dom = j < nt;
                    for (int k = 0; k < m; ++k) dom &= f[k] <= s_smp[(j < nt ? j : 0) * m + k];
                    unsigned mask = __ballot_sync(0xffffffffu, dom);
                    while (mask) {
                        const int b = __ffs(mask) - 1;
                        mask &= mask - 1;
                        const int c = s_cnt[j0 + b];  // >= 1: p itself
                        if (c <= kdrop) v = __dadd_rn(v, __ldcg(&alpha[c]));
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

}  // namespace emo
