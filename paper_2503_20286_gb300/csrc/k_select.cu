// Normalisation, association, niche counts, niching and survivor extraction
// (Algorithm S.1 with Algorithm S.5; Section IV-A "Normalization",
// "Association", "Niche Count Calculation", "Niche Selection").
//
// Precision: everything that decides an index is taken in the same FP64
// arithmetic, operation order and rounding as the FP64 reference statement
// of the method (no fused multiply-add: explicit __d*_rn intrinsics):
//   * ideal point z = min over S (exact in float);
//   * ASF extreme points: an FP32 pass bounds the minimum, points within the
//     FP32 error band are re-evaluated in FP64;
//   * hyperplane intercepts: Gaussian elimination with partial pivoting in
//     FP64 on one thread (m <= 16), nadir fallback;
//   * association: an FP32 scan over all references keeps the three largest
//     projections f.r/|r|; references whose projection lies within a
//     rigorous error band of the best are re-evaluated with the FP64
//     perpendicular distance d^2 = sum (f_k - t r_k)^2, t = f.r / r.r.
#include "emo_kernels.cuh"
#include "emo_launch.cuh"
#include "group_radix.cuh"

namespace emo {

// ------------------------------------------------------------ FP64 helpers
__device__ __forceinline__ double fnorm64(float F, float z, double a)
{
    return __ddiv_rn(__dsub_rn((double)F, (double)z), a);
}

// Perpendicular distance^2 of normalised point fn[0..m) to the line of r.
__device__ inline double perp_d2(const double* fn, const float* r, int m)
{
    double rr = 0.0, fr = 0.0;
    for (int k = 0; k < m; ++k) rr = __dadd_rn(rr, __dmul_rn((double)r[k], (double)r[k]));
    for (int k = 0; k < m; ++k) fr = __dadd_rn(fr, __dmul_rn(fn[k], (double)r[k]));
    const double t = __ddiv_rn(fr, rr);
    double d2 = 0.0;
    for (int k = 0; k < m; ++k) {
        const double e = __dsub_rn(fn[k], __dmul_rn(t, (double)r[k]));
        d2 = __dadd_rn(d2, __dmul_rn(e, e));
    }
    return d2;
}

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

// ------------------------------------------------------------ k_stats
// Ideal point, ASF extreme points, nadir point, intercepts (Algorithm S.5).
__global__ void __launch_bounds__(kCoopThreads, 1) k_stats(Plan* plan)
{
    const Group g = group_of(plan, false);
    if (g.prob < 0) return;  // a CTA beyond every problem's group
    const ProbDev& d = plan->p[g.prob];
    const ProbIn& in = d.in;
    const long long budget = plan->spin_budget;
    if (in.mode != MODE_SELECT || ld_volatile(&d.sc->status) != 0) return;
    Scal* sc = d.sc;
    const int m = in.m, tid = threadIdx.x, lane = tid & 31;
    const int nS = ld_volatile(&sc->nS);
    const float* F = in.F;
    const int64_t stride = (int64_t)g.size * blockDim.x;
    const int64_t t0 = (int64_t)g.rank * blockDim.x + tid;
    __shared__ uint32_t s_u32[kMaxM];
    __shared__ unsigned long long s_u64[kMaxM];
    __shared__ float s_z[kMaxM];

    // 1. ideal point: keep ~key maxima (Scal is zero-initialised)
    if (tid < kMaxM) s_u32[tid] = 0u;
    __syncthreads();
    {
        uint32_t best[kMaxM];
#pragma unroll
        for (int k = 0; k < kMaxM; ++k) best[k] = 0u;
        for (int64_t i = t0; i < nS; i += stride) {
            const int64_t v = d.slist[i];
#pragma unroll
            for (int k = 0; k < kMaxM; ++k)
                if (k < m) best[k] = max(best[k], ~float_key(F[v * m + k]));
        }
#pragma unroll
        for (int k = 0; k < kMaxM; ++k) {
            if (k >= m) break;
            uint32_t b = best[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
            if (lane == 0 && b) atomicMax(&s_u32[k], b);
        }
    }
    __syncthreads();
    if (tid < m && s_u32[tid]) atomicMax(&sc->zkey[tid], s_u32[tid]);
    if (!group_sync(sc, g.size, budget)) return;
    if (tid < m) s_z[tid] = key_float(~__ldcg(&sc->zkey[tid]));
    if (tid < kMaxM) { s_u32[tid] = 0u; s_u64[tid] = 0ull; }
    __syncthreads();

    // 2. FP32 ASF minima per axis (stored as ~bits maxima) and FP64 nadir
    {
        for (int64_t i = t0; i < nS; i += stride) {
            const int64_t v = d.slist[i];
            float dev[kMaxM];
#pragma unroll
            for (int k = 0; k < kMaxM; ++k) dev[k] = k < m ? F[v * m + k] - s_z[k] : 0.0f;
#pragma unroll
            for (int k = 0; k < kMaxM; ++k) {
                if (k >= m) break;
                const double nd = __dsub_rn((double)F[v * m + k], (double)s_z[k]);
                atomicMax(&s_u64[k], dbits(nd));
            }
            for (int j = 0; j < m; ++j) {
                float asf = 0.0f;
#pragma unroll
                for (int k = 0; k < kMaxM; ++k)
                    if (k < m) asf = fmaxf(asf, k == j ? dev[k] : dev[k] * 1.0e6f);
                atomicMax(&s_u32[j], ~__float_as_uint(asf));
            }
        }
    }
    __syncthreads();
    if (tid < m) {
        atomicMax(&sc->asf32[tid], s_u32[tid]);
        atomicMax(&sc->nadir[tid], s_u64[tid]);
    }
    if (!group_sync(sc, g.size, budget)) return;

    // 3. exact FP64 ASF of the candidates within the FP32 error band
    if (tid < kMaxM) s_u64[tid] = 0ull;
    __syncthreads();
    __shared__ float s_lim[kMaxM];
    if (tid < m) {
        const float mn = __uint_as_float(~__ldcg(&sc->asf32[tid]));
        s_lim[tid] = mn * (1.0f + 0x1p-18f) + 1e-30f;
    }
    __syncthreads();
    auto asf64 = [&](int64_t v, int j) {
        double mx = -INFINITY;
        for (int k = 0; k < m; ++k) {
            const double w = k == j ? 1.0 : 1e-6;
            const double t = __ddiv_rn(__dsub_rn((double)F[v * m + k], (double)s_z[k]), w);
            if (t > mx) mx = t;
        }
        return mx;
    };
    auto asf32 = [&](int64_t v, int j) {
        float asf = 0.0f;
        for (int k = 0; k < m; ++k) {
            const float dv = F[v * m + k] - s_z[k];
            asf = fmaxf(asf, k == j ? dv : dv * 1.0e6f);
        }
        return asf;
    };
    for (int64_t i = t0; i < nS; i += stride) {
        const int64_t v = d.slist[i];
        for (int j = 0; j < m; ++j)
            if (asf32(v, j) <= s_lim[j]) atomicMax(&s_u64[j], ~dbits(asf64(v, j)));
    }
    __syncthreads();
    if (tid < m) atomicMax(&sc->asf64[tid], s_u64[tid]);
    if (!group_sync(sc, g.size, budget)) return;

    // 4. lowest index attaining the FP64 minimum (stored as INT32_MAX - i maxima)
    __shared__ unsigned long long s_best[kMaxM];
    if (tid < m) s_best[tid] = ~__ldcg(&sc->asf64[tid]);
    __syncthreads();
    for (int64_t i = t0; i < nS; i += stride) {
        const int64_t v = d.slist[i];
        for (int j = 0; j < m; ++j)
            if (asf32(v, j) <= s_lim[j] && dbits(asf64(v, j)) == s_best[j])
                atomicMax(&sc->ext[j], INT32_MAX - (int)v);
    }
    if (!group_sync(sc, g.size, budget)) return;

    // 5. intercepts by Gaussian elimination with partial pivoting (FP64)
    if (g.rank == 0 && tid == 0) {
        double A[kMaxM][kMaxM], rhs[kMaxM], b[kMaxM], a[kMaxM];
        int ext[kMaxM];
        double maxabs = 0.0;
        for (int j = 0; j < m; ++j) {
            const int e = ld_volatile(&sc->ext[j]);
            if (e <= 0) {  // no candidate attained the minimum (non-finite values)
                set_status(sc, EMO_ERR_NONFINITE);
                return;
            }
            ext[j] = INT32_MAX - e;
            rhs[j] = 1.0;
            for (int k = 0; k < m; ++k) {
                A[j][k] = __dsub_rn((double)F[(int64_t)ext[j] * m + k], (double)s_z[k]);
                maxabs = fmax(maxabs, fabs(A[j][k]));
            }
        }
        int singular = 0;
        for (int col = 0; col < m && !singular; ++col) {
            int piv = col;
            for (int r = col + 1; r < m; ++r)
                if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
            if (!(fabs(A[piv][col]) > __dmul_rn(1e-12, maxabs))) { singular = 1; break; }
            if (piv != col) {
                for (int c = 0; c < m; ++c) { double t = A[col][c]; A[col][c] = A[piv][c]; A[piv][c] = t; }
                double t = rhs[col]; rhs[col] = rhs[piv]; rhs[piv] = t;
            }
            for (int r = col + 1; r < m; ++r) {
                const double f = __ddiv_rn(A[r][col], A[col][col]);
                for (int c = col; c < m; ++c) A[r][c] = __dsub_rn(A[r][c], __dmul_rn(f, A[col][c]));
                rhs[r] = __dsub_rn(rhs[r], __dmul_rn(f, rhs[col]));
            }
        }
        int fallback = singular;
        if (!singular) {
            for (int col = m - 1; col >= 0; --col) {
                double s = rhs[col];
                for (int c = col + 1; c < m; ++c) s = __dsub_rn(s, __dmul_rn(A[col][c], b[c]));
                b[col] = __ddiv_rn(s, A[col][col]);
            }
            for (int k = 0; k < m; ++k) {
                a[k] = __ddiv_rn(1.0, b[k]);
                if (!isfinite(a[k]) || a[k] <= 1e-10) fallback = 1;
            }
        }
        if (fallback) {
            for (int k = 0; k < m; ++k) {
                a[k] = __longlong_as_double((long long)__ldcg(&sc->nadir[k]));
                if (a[k] <= 1e-10) a[k] = 1.0;
            }
        }
        for (int k = 0; k < m; ++k) {
            sc->a[k] = a[k];
            sc->inv_a32[k] = (float)__ddiv_rn(1.0, a[k]);
            sc->z[k] = s_z[k];
            sc->ext[k] = ext[k];
        }
        sc->fallback = fallback;
        __threadfence();
    }

    // 6. S in the order of the polar angle of its normalised points (16-bit
    // buckets, two radix passes): neighbouring threads of the association
    // then scan neighbouring references. Any order of S gives the same result.
    if (!group_sync(sc, g.size, budget)) return;
    __shared__ RadixSmem rsm;
    float zf[kMaxM], ia[kMaxM];
    for (int k = 0; k < m; ++k) {
        zf[k] = __ldcg(&sc->z[k]);
        ia[k] = __ldcg(&sc->inv_a32[k]);
    }
    auto akey = [&](int32_t v) {
        float f[kMaxM];
        for (int k = 0; k < m; ++k) f[k] = (F[(int64_t)v * m + k] - zf[k]) * ia[k];
        const int b = (int)(polar_angle(f, m) * (65535.0f / 1.5707964f));
        return (uint32_t)(b < 0 ? 0 : (b > 65535 ? 65535 : b));
    };
    int32_t* bufs[2] = {d.slist, d.llist};
    int cur = 0;
    const int gsS = (int)max((int64_t)1, min((int64_t)g.size, cdiv(nS, 4096)));
    for (int shift = 0; shift < 16; shift += kRadixBits) {
        bool skipped = false;
        if (!radix_pass(d, g, gsS, budget, nS, bufs[cur], bufs[cur ^ 1], shift, akey, skipped, rsm)) return;
        if (!skipped) cur ^= 1;
    }
    if (cur == 1) {
        for (int64_t i = t0; i < nS; i += stride) d.slist[i] = __ldcg(&d.llist[i]);
        group_sync(sc, g.size, budget);
    }
}

// ------------------------------------------------------------ association
// FP32 scan: the perpendicular distance is computed in the cancellation-free
// form d^2 = sum_k (f_k - g u_k)^2, g = f.u, u = r/|r| (linear in the angle
// near the optimum, so its error band is narrow). Candidates come from the
// angular index: references sorted by polar angle phi from axis 1; since the
// angle between two directions is at least the difference of their polar
// angles (triangle inequality on the sphere), only references with
// |phi_r - phi_f| <= theta_best + margin can beat the best one found so far.
// The scan walks outward from phi_f and stops on that bound. The same
// inequality for the angle from axis 2 (a second pivot, stored per reference)
// skips the distance of references on the far side of the band's ring.
//
// Error band of the FP32 distance (relative to |f|), two evaluations:
// |delta d| <= (sqrt(m)(m + 10) + (m + 1)/2) u |f| each.
__device__ __forceinline__ float assoc_band(int m)
{
    return (2.0f * sqrtf((float)m) * (float)(m + 10) + (float)(m + 8)) * 1.05f * 0x1p-24f;
}
// Extra angular margin of the index scan: covers the atan2/asin rounding and
// keeps every unscanned reference farther than the band from the best.
__device__ __forceinline__ float assoc_margin(int m) { return 1e-5f + 8.0f * assoc_band(m); }
constexpr float kAssocMaxBound = 0.7853981f;  // beyond pi/4 the scan covers every reference

template <int M>
__device__ __forceinline__ float d2_f32(const float* f, const float* u)
{
    float g = f[0] * u[0];
#pragma unroll
    for (int k = 1; k < M; ++k) g = fmaf(f[k], u[k], g);
    float d2 = 0.0f;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const float e = fmaf(-g, u[k], f[k]);
        d2 = fmaf(e, e, d2);
    }
    return d2;
}

// Exact decision between candidate references (FP64, reference formula).
__device__ inline void decide64(const ProbDev& d, const Scal* sc, int64_t v, int m, const int* cand, int nc,
                                int& best_j, double& best_d2)
{
    double fn[kMaxM];
    for (int k = 0; k < m; ++k) fn[k] = fnorm64(d.in.F[v * m + k], sc->z[k], sc->a[k]);
    best_j = -1;
    best_d2 = INFINITY;
    for (int c = 0; c < nc; ++c) {
        const int j = cand[c];
        const double d2 = perp_d2(fn, d.in.R + (int64_t)j * m, m);
        if (d2 < best_d2 || (d2 == best_d2 && j < best_j)) { best_d2 = d2; best_j = j; }
    }
}

// First sorted position with rphi >= x.
__device__ __forceinline__ int lower_bound_f(const float* a, int n, float x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&a[mid]) < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <int M>
__global__ void __launch_bounds__(256) k_assoc_m(Plan* plan, int pfirst, int plast)
{
    // the points of S of every problem of this m in one sequence (a batch's
    // small problems together fill the grid)
    __shared__ long long s_first[kMaxBatch + 1];
    const int tid = threadIdx.x;
    if (tid == 0) {
        long long acc = 0;
        for (int p = pfirst; p < plast; ++p) {
            s_first[p - pfirst] = acc;
            const ProbDev& d = plan->p[p];
            if (d.in.mode == MODE_SELECT && d.in.m == M && ld_volatile(&d.sc->status) == 0)
                acc += ld_volatile(&d.sc->nS);
        }
        s_first[plast - pfirst] = acc;
    }
    __syncthreads();
    const long long total = s_first[plast - pfirst];
    const float band = assoc_band(M), margin = assoc_margin(M);
    // a population split over GPUs associates only its own points
    const bool ranged = plan->split.kind == SPLIT_ASSOC;
    for (long long gs = (long long)blockIdx.x * 256 + tid; gs < total; gs += (long long)gridDim.x * 256) {
        int plo = 0, phi = plast - pfirst;  // last problem with s_first <= gs
        while (phi - plo > 1) {
            const int mid = (plo + phi) >> 1;
            if (s_first[mid] <= gs) plo = mid;
            else phi = mid;
        }
        while (s_first[plo + 1] <= gs) ++plo;  // skip problems without points
        const ProbDev& d = plan->p[pfirst + plo];
        const Scal* sc = d.sc;
        const int64_t s = gs - s_first[plo];
        const int nr = d.in.n_r;
        const float* __restrict__ rphi = d.rphi;
        const float* __restrict__ rphi2 = d.rphi2;
        const float* __restrict__ rs = d.rsort;
        const int32_t* __restrict__ ro = d.rord + (int64_t)sc->rbuf * nr;
        const int64_t lo = ranged ? plan->split.col_lo : 0, hi = ranged ? plan->split.col_hi : d.in.n2;
        const int64_t v = d.slist[s];
        if (v < lo || v >= hi) continue;
        float f[M];
        float n2 = 0.0f;
#pragma unroll
        for (int k = 0; k < M; ++k) {
            f[k] = (d.in.F[v * M + k] - sc->z[k]) * sc->inv_a32[k];
            n2 = fmaf(f[k], f[k], n2);
        }
        const float nrm = sqrtf(n2);
        if (!(nrm > 0.0f) || !isfinite(nrm)) {  // at the ideal point (or overflow): exhaustive FP64 scan
            const int slot = atomicAdd(&d.sc->nflag, 1);
            d.flagged[slot] = (int32_t)v;
            d.flagged_bound[slot] = INFINITY;
            continue;
        }
        const float phif = polar_angle(f, M);
        const float phi2f = polar_angle2(f, M);
        float c1 = INFINITY, c2 = INFINITY, c3 = INFINITY;  // FP32 d^2, best three
        int s1 = -1, s2 = -1;                                 // sorted positions of the best two
        float bound = INFINITY;                               // angular half-width still to scan
        int L = lower_bound_f(rphi, nr, phif) - 1, Rp = L + 1;
        float dl = L >= 0 ? phif - __ldg(&rphi[L]) : INFINITY;
        float dr = Rp < nr ? __ldg(&rphi[Rp]) - phif : INFINITY;
        while (L >= 0 || Rp < nr) {  // at most n_r steps
            const bool left = L >= 0 && (Rp >= nr || dl <= dr);
            const float dm = left ? dl : dr;
            if (!(dm <= bound)) break;
            int q;  // 0 <= q < n_r
            if (left) {
                q = L--;
                dl = L >= 0 ? phif - __ldg(&rphi[L]) : INFINITY;
            } else {
                q = Rp++;
                dr = Rp < nr ? __ldg(&rphi[Rp]) - phif : INFINITY;
            }
            // second pivot: the angle to the reference is at least the
            // difference of the angles from axis 2 (same margins as axis 1)
            if (M > 2 && !(fabsf(__ldg(&rphi2[q]) - phi2f) <= bound)) continue;
            float u[M];
#pragma unroll
            for (int k = 0; k < M; ++k) u[k] = __ldg(&rs[(int64_t)q * M + k]);
            const float dd = d2_f32<M>(f, u);
            if (dd < c3) {
                if (dd < c2) {
                    c3 = c2;
                    if (dd < c1) { c2 = c1; s2 = s1; c1 = dd; s1 = q; }
                    else { c2 = dd; s2 = q; }
                    // angle of the best so far, bounded from above
                    const float sn = fminf(1.0f, sqrtf(c1) / nrm * 1.00001f + 2.0f * band);
                    const float th = asinf(sn);
                    bound = th + margin > kAssocMaxBound ? INFINITY : th + margin;
                } else {
                    c3 = dd;
                }
            }
        }
        const float d1 = sqrtf(c1), lim = d1 + band * nrm;
        if (sqrtf(c3) <= lim) {  // three or more references inside the band
            const int slot = atomicAdd(&d.sc->nflag, 1);
            d.flagged[slot] = (int32_t)v;
            d.flagged_bound[slot] = bound;
            continue;
        }
        int cand[2];
        int nc = 0;
        cand[nc++] = __ldg(&ro[s1]);
        if (s2 >= 0 && sqrtf(c2) <= lim) cand[nc++] = __ldg(&ro[s2]);
        int bj;
        double bd2;
        decide64(d, sc, v, M, cand, nc, bj, bd2);
        d.pi[v] = bj;
        d.d64[v] = __dsqrt_rn(bd2);
    }
}

// All-reference association for m >= 4, where the polar-angle index prunes
// little: every reference is visited, uniformly across a warp. A CTA takes a
// tile of 64 points of S (two per lane, the same in every warp) and stages
// the unit directions in shared memory, 1024 (m <= 8) or 512 at a time; warp
// w visits the w-th eighth of each staged block for the tile's points,
// keeping the three smallest FP32 distances and the references of the two
// smallest; the eight warps' lists are merged and the decision is the one of
// k_assoc_m (two candidates inside the FP32 band: FP64 decision; three or
// more: the point is re-scanned in FP64 by k_rescan over every reference).
// Which reference of an FP32 tie is kept does not matter: tied candidates
// are inside the band together. Tiles are taken from a counter, problems
// with the most references first. (A per-point angular filter on the
// projection f.u before the distance was measured slower: the 64 points of
// a warp rarely all skip the same reference, and the warp runs the distance
// whenever one of them does not.)
constexpr int kBfWarps = 8;
constexpr int kBfPPL = 2;                    // points per lane
constexpr int kBfTile = 32 * kBfPPL;         // points per CTA tile
constexpr int kBfStageBytes = 32768;         // staged unit directions

struct BfTop {
    float c1, c2, c3;
    int s1, s2;
    __device__ __forceinline__ void init() { c1 = c2 = c3 = INFINITY; s1 = s2 = -1; }
    __device__ __forceinline__ void add(float dd, int j)
    {
        if (dd < c3) {
            if (dd < c2) {
                c3 = c2;
                if (dd < c1) { c2 = c1; s2 = s1; c1 = dd; s1 = j; }
                else { c2 = dd; s2 = j; }
            } else {
                c3 = dd;
            }
        }
    }
};

template <int M>
__global__ void __launch_bounds__(kBfWarps * 32) k_assoc_all(Plan* plan, int pfirst, int plast)
{
    constexpr int MP = (M + 3) / 4 * 4;  // padded to whole float4
    constexpr int kStage = kBfStageBytes / (MP * 4);
    constexpr int kPerWarp = (kStage + kBfWarps - 1) / kBfWarps;
    __shared__ float4 s_u[kStage * MP / 4];
    __shared__ float s_c[3][kBfWarps][kBfTile];
    __shared__ int s_s[2][kBfWarps][kBfTile];
    __shared__ int s_ord[kMaxBatch], s_first[kMaxBatch + 1];
    __shared__ int s_np, s_tile;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {  // problems of this m, most references first; tile prefix
        int np = 0;
        for (int p = pfirst; p < plast; ++p) {
            const ProbDev& d = plan->p[p];
            if (d.in.mode != MODE_SELECT || d.in.m != M || ld_volatile(&d.sc->status) != 0) continue;
            int i = np++;
            while (i > 0 && plan->p[s_ord[i - 1]].in.n_r < d.in.n_r) { s_ord[i] = s_ord[i - 1]; --i; }
            s_ord[i] = p;
        }
        s_first[0] = 0;
        for (int i = 0; i < np; ++i)
            s_first[i + 1] = s_first[i] + (int)cdiv(ld_volatile(&plan->p[s_ord[i]].sc->nS), kBfTile);
        s_np = np;
    }
    __syncthreads();
    const int np = s_np, ntiles = s_first[np];
    for (;;) {
        if (tid == 0) s_tile = (int)atomicAdd(&plan->asc_next[M], 1ull);
        __syncthreads();
        const int t = s_tile;
        __syncthreads();  // every thread has read s_tile
        if (t >= ntiles) break;
        int pi_ = 0;
        while (s_first[pi_ + 1] <= t) ++pi_;
        const ProbDev& d = plan->p[s_ord[pi_]];
        const Scal* sc = d.sc;
        const int nS = ld_volatile(&sc->nS), nr = d.in.n_r;
        const bool ranged = plan->split.kind == SPLIT_ASSOC;
        const int64_t lo = ranged ? plan->split.col_lo : 0, hi = ranged ? plan->split.col_hi : d.in.n2;
        const int64_t s0 = (int64_t)(t - s_first[pi_]) * kBfTile;
        float f[kBfPPL][M];
        float nrm[kBfPPL];
        int64_t v[kBfPPL];
        bool act[kBfPPL];
        BfTop top[kBfPPL];
#pragma unroll
        for (int i = 0; i < kBfPPL; ++i) {
            const int64_t s = s0 + i * 32 + lane;
            v[i] = s < nS ? (int64_t)d.slist[s] : -1;
            act[i] = v[i] >= lo && v[i] < hi;
            float n2 = 0.0f;
#pragma unroll
            for (int k = 0; k < M; ++k) {
                f[i][k] = act[i] ? (d.in.F[v[i] * M + k] - sc->z[k]) * sc->inv_a32[k] : 0.0f;
                n2 = fmaf(f[i][k], f[i][k], n2);
            }
            nrm[i] = sqrtf(n2);
            top[i].init();
        }
        bool scan = false;
#pragma unroll
        for (int i = 0; i < kBfPPL; ++i) scan |= act[i] && nrm[i] > 0.0f && isfinite(nrm[i]);
        if (__syncthreads_or(scan)) {
            for (int r0 = 0; r0 < nr; r0 += kStage) {
                const int cnt = min(kStage, nr - r0);
                __syncthreads();  // the previous block has been scanned
                float* su = (float*)s_u;
                for (int e = tid; e < cnt * MP; e += kBfWarps * 32) {
                    const int q = e / MP, k = e - q * MP;
                    su[e] = k < M ? __ldg(&d.rhat[(int64_t)(r0 + q) * M + k]) : 0.0f;
                }
                __syncthreads();
                const int qa = warp * kPerWarp, qb = min(cnt, qa + kPerWarp);
                for (int q = qa; q < qb; ++q) {
                    float u[MP];
#pragma unroll
                    for (int k4 = 0; k4 < MP / 4; ++k4) {
                        const float4 x = s_u[q * (MP / 4) + k4];
                        u[4 * k4] = x.x;
                        u[4 * k4 + 1] = x.y;
                        u[4 * k4 + 2] = x.z;
                        u[4 * k4 + 3] = x.w;
                    }
#pragma unroll
                    for (int i = 0; i < kBfPPL; ++i) top[i].add(d2_f32<M>(f[i], u), r0 + q);
                }
            }
        }
        // merge the warps' lists; threads 0 .. 63 decide one point each
#pragma unroll
        for (int i = 0; i < kBfPPL; ++i) {
            const int pt = i * 32 + lane;
            s_c[0][warp][pt] = top[i].c1;
            s_c[1][warp][pt] = top[i].c2;
            s_c[2][warp][pt] = top[i].c3;
            s_s[0][warp][pt] = top[i].s1;
            s_s[1][warp][pt] = top[i].s2;
        }
        __syncthreads();
        if (tid < kBfTile) {
            const int64_t s = s0 + tid;  // point tid of the tile (lane tid & 31, slot tid >> 5)
            const int64_t vv = s < nS ? (int64_t)d.slist[s] : -1;
            if (vv >= lo && vv < hi) {
                BfTop b;
                b.init();
                for (int w = 0; w < kBfWarps; ++w) {
                    // the smaller two carry references; a third value only its distance
                    b.add(s_c[0][w][tid], s_s[0][w][tid]);
                    b.add(s_c[1][w][tid], s_s[1][w][tid]);
                    b.add(s_c[2][w][tid], -1);
                }
                float ff[M], n2 = 0.0f;
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    ff[k] = (d.in.F[vv * M + k] - sc->z[k]) * sc->inv_a32[k];
                    n2 = fmaf(ff[k], ff[k], n2);
                }
                const float nm = sqrtf(n2);
                const float band = assoc_band(M);
                if (!(nm > 0.0f) || !isfinite(nm) || sqrtf(b.c3) <= sqrtf(b.c1) + band * nm) {
                    // at the ideal point, or three or more references inside the band
                    const int slot = atomicAdd(&d.sc->nflag, 1);
                    d.flagged[slot] = (int32_t)vv;
                    d.flagged_bound[slot] = INFINITY;
                } else {
                    const float lim = sqrtf(b.c1) + band * nm;
                    int cand[2];
                    int nc = 0;
                    cand[nc++] = b.s1;
                    if (b.s2 >= 0 && sqrtf(b.c2) <= lim) cand[nc++] = b.s2;
                    int bj;
                    double bd2;
                    decide64(d, sc, vv, M, cand, nc, bj, bd2);
                    d.pi[vv] = bj;
                    d.d64[vv] = __dsqrt_rn(bd2);
                }
            }
        }
        __syncthreads();  // s_c / s_s are free again
    }
}

// Points whose FP32 band holds three or more references: one warp per point
// re-evaluates, in FP64, every reference of the scanned angular range whose
// FP32 distance lies within the band of the range minimum.
__global__ void __launch_bounds__(256) k_rescan(Plan* plan)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int p = 0; p < plan->nprob; ++p) {
        const ProbDev& d = plan->p[p];
        Scal* sc = d.sc;
        if (d.in.mode != MODE_SELECT || ld_volatile(&sc->status) != 0) continue;
        const int nflag = ld_volatile(&sc->nflag);
        const int m = d.in.m, nr = d.in.n_r;
        const int32_t* ro = d.rord + (int64_t)sc->rbuf * nr;
        const float band = assoc_band(m);
        for (int64_t w = gw; w < nflag; w += nw) {
            const int64_t v = d.flagged[w];
            const float bound = d.flagged_bound[w];
            float f[kMaxM];
            float n2 = 0.0f;
            for (int k = 0; k < m; ++k) {
                f[k] = (d.in.F[v * m + k] - sc->z[k]) * sc->inv_a32[k];
                n2 = fmaf(f[k], f[k], n2);
            }
            const float nrm = sqrtf(n2);
            // bad: at the ideal point or overflowed, every reference in FP64;
            // otherwise the FP32 band of the range minimum filters the range
            const bool bad = !(nrm > 0.0f) || !isfinite(nrm);
            const bool all = bad || !(bound < INFINITY);
            int lo = 0, hi = nr;
            if (!all) {
                const float phif = polar_angle(f, m);
                lo = lower_bound_f(d.rphi, nr, phif - bound);
                hi = lower_bound_f(d.rphi, nr, nextafterf(phif + bound, INFINITY));
            }
            auto dist32 = [&](int q) {
                const float* u = d.rsort + (int64_t)q * m;
                float g = f[0] * u[0];
                for (int k = 1; k < m; ++k) g = fmaf(f[k], u[k], g);
                float d2 = 0.0f;
                for (int k = 0; k < m; ++k) {
                    const float e = fmaf(-g, u[k], f[k]);
                    d2 = fmaf(e, e, d2);
                }
                return sqrtf(d2);
            };
            float dmin = INFINITY;
            if (!bad)
                for (int q = lo + lane; q < hi; q += 32) dmin = fminf(dmin, dist32(q));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
            const float lim = dmin + band * nrm;
            double fn[kMaxM];
            for (int k = 0; k < m; ++k) fn[k] = fnorm64(d.in.F[v * m + k], sc->z[k], sc->a[k]);
            double bd2 = INFINITY;
            int bj = INT32_MAX;
            for (int q = lo + lane; q < hi; q += 32) {
                if (bad || dist32(q) <= lim) {
                    const int j = __ldg(&ro[q]);
                    const double d2 = perp_d2(fn, d.in.R + (int64_t)j * m, m);
                    if (d2 < bd2 || (d2 == bd2 && j < bj)) { bd2 = d2; bj = j; }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double od = __shfl_xor_sync(0xffffffffu, bd2, o);
                const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
                if (od < bd2 || (od == bd2 && oj < bj)) { bd2 = od; bj = oj; }
            }
            if (lane == 0) {
                if (bj == INT32_MAX) {  // every distance was NaN
                    set_status(sc, EMO_ERR_NONFINITE);
                    bj = 0;
                }
                d.pi[v] = bj;
                d.d64[v] = __dsqrt_rn(bd2);
            }
        }
    }
}

// Host launcher: one instantiation per objective count.
cudaError_t launch_assoc(Plan* plan, int nprob, const int* m_of, int sms, int blocks_per_sm, cudaStream_t s)
{
    for (int p = 0; p < nprob;) {
        int q = p;
        while (q < nprob && m_of[q] == m_of[p]) ++q;
        const unsigned grid = (unsigned)sms * (unsigned)(blocks_per_sm > 0 ? blocks_per_sm : 8);
        // m >= 4: every reference, tiled (tiles from a counter: a few CTAs per SM)
        const unsigned grid_all = (unsigned)sms * 4u;
        switch (m_of[p]) {
#define X(MM) \
    case MM: k_assoc_m<MM><<<grid, 256, 0, s>>>(plan, p, q); break;
#define Y(MM) \
    case MM: k_assoc_all<MM><<<grid_all, kBfWarps * 32, 0, s>>>(plan, p, q); break;
            X(2) X(3) Y(4) Y(5) Y(6) Y(7) Y(8) Y(9) Y(10) Y(11) Y(12) Y(13) Y(14) Y(15) Y(16)
#undef X
#undef Y
        default: return cudaErrorInvalidValue;
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        p = q;
    }
    return cudaSuccess;
}

cudaError_t launch_assoc(Plan* plan, int nprob, const int* m_of, int sms, cudaStream_t s)
{
    return launch_assoc(plan, nprob, m_of, sms, 8, s);  // the default shape: 8 blocks per SM
}

}  // namespace emo
