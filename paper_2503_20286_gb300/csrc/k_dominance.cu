// Pareto-dominance matrix kernels (Section III-C, Listing 1; Section IV-A;
// Algorithm S.3 first two lines).
//
// k_dom_tri  -- selection path. Points are in lexicographic order, so for
//   p < q only "p dominates q" is possible and it holds iff objectives
//   2..m of p are <= those of q and the two points are not identical
//   (objective 1 is ordered by the sort). One warp owns R row blocks, a lane
//   owns one row and keeps its keys in registers; the 1024 column keys of the
//   work item are staged in shared memory by a bulk-async copy and read as
//   broadcasts. Each comparison result is OR-ed into the lane's word, so a
//   lane ends with whole 32-bit words of its row. Finished 4 KB tiles are
//   written from shared memory with bulk-async stores. The dominator count of
//   every column (the column sum c_j of D) is accumulated from the staged
//   tiles with a Harley-Seal bit-sliced vertical counter.
// k_dom_full -- emo_dominance: every ordered pair in the caller's order,
//   "all <= and some <" evaluated directly.
#include "emo_kernels.cuh"

namespace emo {

template <int K>
struct DomShape {
    static constexpr int R = 2;   // row blocks per warp
    static constexpr int NW = 8;  // warps per CTA
    static constexpr int CB = K <= 2 ? 32 : (K <= 4 ? 16 : (K <= 8 ? 8 : 4));  // columns per register batch
};
constexpr int kDomNH = 8;  // high count planes: up to 4095 rows per lane and item
constexpr long long kCopyWaitCycles = 1ll << 32;

template <int K>
struct DomSmem {
    alignas(128) float ck[kColBlock * K];
    alignas(128) int32_t rs[kColBlock];
    alignas(128) uint32_t tiles[DomShape<K>::NW][DomShape<K>::R][kTileRows * kTileWords];
    int32_t cnt[kColBlock];
    uint64_t bar;
    long long item;
    int skip;
};

// Decode a dominance item of one problem: column blocks are served from the
// last (tallest) to the first; each is split into chunks of kDomRowChunk row
// blocks.
__device__ __forceinline__ void dom_decode(long long local, int ncb, int nrb, int& cb, int& chunk)
{
    for (cb = ncb - 1; cb >= 0; --cb) {
        long long n = dom_items_of_cb(cb, nrb);
        if (local < n) break;
        local -= n;
    }
    chunk = (int)local;
}

// Flush a warp's per-lane column counters: lane w holds columns 32 w + b.
template <int NH>
__device__ __forceinline__ void flush_counts(VCount<NH>& vc, int32_t* s_cnt, int lane)
{
    if (__any_sync(0xffffffffu, vc.any())) {
#pragma unroll 4
        for (int b = 0; b < 32; ++b) {
            int c = vc.count(b);
            if (c) atomicAdd(&s_cnt[b * 32 + lane], c);
        }
    }
    vc = VCount<NH>();
}

template <int M>
__global__ void __launch_bounds__(256, 1) k_dom_tri(Plan* plan, long long item_lo, long long item_hi,
                                                    unsigned long long* counter)
{
    constexpr int K = M - 1;
    using S = DomShape<K>;
    constexpr int R = S::R, NW = S::NW, CB = S::CB;
    extern __shared__ __align__(128) unsigned char smraw[];
    DomSmem<K>& sm = *reinterpret_cast<DomSmem<K>*>(smraw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) mbar_init(&sm.bar, 1);
    __syncthreads();
    uint32_t parity = 0;

    while (true) {
        if (tid == 0) {
            sm.item = item_lo + (long long)atomicAdd(counter, 1ull);
        }
        __syncthreads();
        const long long item = sm.item;
        if (item >= item_hi) break;
        int p = 0;
        while (p + 1 < plan->nprob && plan->dom_item_start[p + 1] <= item) ++p;
        const ProbDev& d = plan->p[p];
        int cb, chunk;
        dom_decode(item - plan->dom_item_start[p], d.ncb, d.nrb, cb, chunk);
        if (tid == 0) {
            sm.skip = ld_volatile(&d.sc->status) != 0;
            if (!sm.skip) {
                fence_proxy_async_smem();
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&sm.bar)),
                             "r"((uint32_t)(kColBlock * K * 4 + kColBlock * 4))
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(sm.ck)),
                    "l"(d.keys + (int64_t)cb * kColBlock * K), "r"((uint32_t)(kColBlock * K * 4)),
                    "r"(smem_u32(&sm.bar))
                    : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(sm.rs)),
                    "l"(d.runstart + (int64_t)cb * kColBlock), "r"((uint32_t)(kColBlock * 4)), "r"(smem_u32(&sm.bar))
                    : "memory");
            }
        }
        for (int i = tid; i < kColBlock; i += blockDim.x) sm.cnt[i] = 0;
        __syncthreads();
        if (sm.skip) continue;
        // The copy is a local load that always completes; the bound only
        // guards against a lost completion. On timeout the status is set and
        // the CTA still waits (bounded) so that no copy is in flight at exit.
        if (!mbar_wait(&sm.bar, parity, kCopyWaitCycles)) {
            if (tid == 0) set_status(d.sc, EMO_ERR_TIMEOUT);
            mbar_wait(&sm.bar, parity, kCopyWaitCycles);
            break;
        }
        parity ^= 1u;

        const int64_t n2 = d.in.n2;
        const int rbmax = min(d.nrb, 32 * (cb + 1));
        const int rb_lo = chunk * kDomRowChunk, rb_hi = min(rbmax, rb_lo + kDomRowChunk);
        const int dupcut = d.minrs[cb];
        const int64_t cbase = (int64_t)cb * kColBlock;
        VCount<kDomNH> vc;

        for (int rbg = rb_lo + warp * R; rbg < rb_hi; rbg += NW * R) {
            float rk[R][K];
            int64_t prow[R];
            bool rvalid[R], diag[R];
            bool anydup = false;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int rb = rbg + r;
                rvalid[r] = rb < rb_hi;
                prow[r] = (int64_t)rb * kTileRows + lane;
                const bool live = rvalid[r] && prow[r] < n2;
#pragma unroll
                for (int k = 0; k < K; ++k) rk[r][k] = live ? __ldg(&d.keys[prow[r] * K + k]) : INFINITY;
                diag[r] = rvalid[r] && (int64_t)rb * kTileRows + 31 >= cbase;
                anydup |= rvalid[r] && rb * kTileRows + 31 >= dupcut;
            }
            for (int w = 0; w < kTileWords; ++w) {
                uint32_t wd[R];
#pragma unroll
                for (int r = 0; r < R; ++r) wd[r] = 0u;
#pragma unroll
                for (int cc = 0; cc < 32; cc += CB) {
                    float ck[CB * K];
                    const float4* src = reinterpret_cast<const float4*>(sm.ck + (w * 32 + cc) * K);
#pragma unroll
                    for (int v = 0; v < CB * K / 4; ++v) {
                        float4 t = src[v];
                        ck[4 * v + 0] = t.x;
                        ck[4 * v + 1] = t.y;
                        ck[4 * v + 2] = t.z;
                        ck[4 * v + 3] = t.w;
                    }
#pragma unroll
                    for (int b = 0; b < CB; ++b) {
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            bool le = rk[r][0] <= ck[b * K + 0];
#pragma unroll
                            for (int k = 1; k < K; ++k) le = le & (rk[r][k] <= ck[b * K + k]);
                            if (le) wd[r] |= 1u << (cc + b);
                        }
                    }
                }
                if (anydup) {
                    // identical points (same run) never dominate each other
                    for (int b = 0; b < 32; ++b) {
                        const int rs = sm.rs[w * 32 + b];
#pragma unroll
                        for (int r = 0; r < R; ++r)
                            if ((int64_t)rs <= prow[r]) wd[r] &= ~(1u << b);
                    }
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (diag[r]) {
                        const int64_t off = prow[r] - (cbase + 32 * w);  // keep columns q > p
                        if (off >= 31) wd[r] = 0u;
                        else if (off >= 0) wd[r] &= 0xFFFFFFFFu << (off + 1);
                    }
                    sm.tiles[warp][r][lane * 32 + (w ^ lane)] = wd[r];
                }
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (rvalid[r]) {
                        uint32_t* dst = d.D + tile_index(rbg + r, cb, d.ncb) * (int64_t)(kTileRows * kTileWords);
                        bulk_store(dst, sm.tiles[warp][r], kTileRows * kTileWords * 4);
                    }
                bulk_commit();
            }
            // column counts from the staged tiles: lane = word column
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (!rvalid[r]) continue;
                uint32_t x[32];
#pragma unroll
                for (int row = 0; row < 32; ++row) x[row] = sm.tiles[warp][r][row * 32 + (lane ^ row)];
                vc.add16(x);
                vc.add16(x + 16);
            }
            if (lane == 0) bulk_wait_read_all();
            __syncwarp();
        }
        flush_counts(vc, sm.cnt, lane);
        __syncthreads();
        for (int q = tid; q < kColBlock; q += blockDim.x) {
            const int c = sm.cnt[(q & 31) * 32 + (q >> 5)];
            if (c) atomicAdd(&d.cnt[cbase + q], c);
        }
        __syncthreads();
    }
    if (lane == 0) bulk_wait_all();
}

// Full matrix in caller order: D_ij = all(F_i <= F_j) and any(F_i < F_j).
template <int M>
struct FullSmem {
    alignas(16) float ck[kColBlock * M];
    alignas(16) uint32_t tiles[8][2][kTileRows * kTileWords];
    int32_t cnt[kColBlock];
    long long item;
};

template <int M>
__global__ void __launch_bounds__(256, 1) k_dom_full(const float* __restrict__ F, int64_t n2, uint32_t* D,
                                                     int64_t ld, int32_t* cnt, long long nitems)
{
    constexpr int R = 2, NW = 8;
    extern __shared__ __align__(128) unsigned char smraw[];
    FullSmem<M>& sm = *reinterpret_cast<FullSmem<M>*>(smraw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nrb = (int)cdiv(n2, 32);
    const long long per_cb = cdiv(nrb, kDomRowChunk);
    for (long long item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int cb = (int)(item / per_cb), chunk = (int)(item % per_cb);
        const int64_t cbase = (int64_t)cb * kColBlock;
        for (int i = tid; i < kColBlock * M; i += blockDim.x) {
            const int64_t q = cbase + i / M;
            sm.ck[i] = q < n2 ? F[q * M + i % M] + 0.0f : -INFINITY;
        }
        for (int i = tid; i < kColBlock; i += blockDim.x) sm.cnt[i] = 0;
        __syncthreads();
        const int rb_lo = chunk * kDomRowChunk, rb_hi = min(nrb, rb_lo + kDomRowChunk);
        VCount<kDomNH> vc;
        for (int rbg = rb_lo + warp * R; rbg < rb_hi; rbg += NW * R) {
            float rk[R][M];
            int64_t prow[R];
            bool rvalid[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                rvalid[r] = rbg + r < rb_hi;
                prow[r] = (int64_t)(rbg + r) * kTileRows + lane;
                const bool live = rvalid[r] && prow[r] < n2;
#pragma unroll
                for (int k = 0; k < M; ++k) rk[r][k] = live ? F[prow[r] * M + k] + 0.0f : INFINITY;
            }
            for (int w = 0; w < kTileWords; ++w) {
                uint32_t wd[R];
#pragma unroll
                for (int r = 0; r < R; ++r) wd[r] = 0u;
#pragma unroll 4
                for (int b = 0; b < 32; ++b) {
                    const float* c = sm.ck + (w * 32 + b) * M;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        bool le = true, lt = false;
#pragma unroll
                        for (int k = 0; k < M; ++k) {
                            le = le & (rk[r][k] <= c[k]);
                            lt = lt | (rk[r][k] < c[k]);
                        }
                        if (le & lt) wd[r] |= 1u << b;
                    }
                }
#pragma unroll
                for (int r = 0; r < R; ++r) sm.tiles[warp][r][lane * 32 + (w ^ lane)] = wd[r];
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (!rvalid[r]) continue;
                uint32_t x[32];
#pragma unroll
                for (int row = 0; row < 32; ++row) x[row] = sm.tiles[warp][r][row * 32 + (lane ^ row)];
                vc.add16(x);
                vc.add16(x + 16);
                const int64_t wcol = (int64_t)cb * 32 + lane;
                if (wcol < ld) {
#pragma unroll 4
                    for (int row = 0; row < 32; ++row) {
                        const int64_t pr = (int64_t)(rbg + r) * kTileRows + row;
                        if (pr < n2) D[pr * ld + wcol] = x[row];
                    }
                }
            }
            __syncwarp();
        }
        if (cnt) {
            flush_counts(vc, sm.cnt, lane);
            __syncthreads();
            for (int q = tid; q < kColBlock; q += blockDim.x) {
                const int c = sm.cnt[(q & 31) * 32 + (q >> 5)];
                if (c && cbase + q < n2) atomicAdd(&cnt[cbase + q], c);
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ launchers
template <int M>
static cudaError_t launch_tri_m(Plan* plan, int sms, cudaStream_t s, long long lo, long long hi,
                                unsigned long long* counter)
{
    const size_t smem = sizeof(DomSmem<M - 1>);
    cudaError_t e = cudaFuncSetAttribute(k_dom_tri<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dom_tri<M>, 256, smem);
    if (e != cudaSuccess) return e;
    long long grid = (long long)sms * (occ > 0 ? occ : 1);
    if (grid > hi - lo) grid = hi - lo;
    if (grid < 1) return cudaSuccess;
    k_dom_tri<M><<<(unsigned)grid, 256, smem, s>>>(plan, lo, hi, counter);
    return cudaGetLastError();
}

template <int M>
static cudaError_t launch_full_m(const float* F, int64_t n2, uint32_t* D, int64_t ld, int32_t* cnt, int sms,
                                 cudaStream_t s)
{
    const size_t smem = sizeof(FullSmem<M>);
    cudaError_t e = cudaFuncSetAttribute(k_dom_full<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dom_full<M>, 256, smem);
    if (e != cudaSuccess) return e;
    const long long nitems = cdiv(n2, kColBlock) * cdiv(cdiv(n2, 32), kDomRowChunk);
    long long grid = (long long)sms * (occ > 0 ? occ : 1);
    if (grid > nitems) grid = nitems;
    k_dom_full<M><<<(unsigned)grid, 256, smem, s>>>(F, n2, D, ld, cnt, nitems);
    return cudaGetLastError();
}

#define EMO_FOR_EACH_M(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

// The plan's problems are ordered by m; items of objective count m form one
// contiguous range served by the m-instantiation.
cudaError_t launch_dominance_tri_range(int m, Plan* plan, int sms, cudaStream_t s, long long lo, long long hi,
                                       unsigned long long* counter)
{
    switch (m) {
#define X(MM) \
    case MM: return launch_tri_m<MM>(plan, sms, s, lo, hi, counter);
        EMO_FOR_EACH_M(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_dominance_full_c(const float* F, int64_t n2, int m, uint32_t* D, int64_t ld, int32_t* cnt,
                                    int sms, cudaStream_t s)
{
    switch (m) {
#define X(MM) \
    case MM: return launch_full_m<MM>(F, n2, D, ld, cnt, sms, s);
        EMO_FOR_EACH_M(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace emo
