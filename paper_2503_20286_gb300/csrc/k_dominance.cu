// Pareto-dominance matrix kernels (Section III-C, Listing 1; Section IV-A;
// Algorithm S.3 first two lines).
//
// Selection path (points in lexicographic order, so for p < q only "p
// dominates q" is possible; it holds iff f_k(q) >= f_k(p) for every key
// objective k = 2..m and the points are not identical):
//   k_colprep -- for each 1024-column block, each half of 512 columns and
//     each key objective k, sorts the half's columns by f_k (descending) and
//     stores, every CPS sorted columns, the bitset of the columns seen so far.
//     The set {q in half : f_k(q) >= f_k(p)} is then a prefix of that order:
//     a checkpoint bitset plus at most CPS - 1 extra bits (CPS = 1 for m <= 4,
//     so no extra bits at all).
//   k_dom_pref<M> (m <= 6; k_dom_pref_rt for m >= 7) -- one warp per row
//     block: each lane first counts, for its row and each objective, the
//     columns of both halves that are >= (binary search). Then each half-warp
//     builds one row at a time (lanes 0-15 rows 0-15, lanes 16-31 rows 16-31),
//     a lane owning 64 columns (two words): the words are the AND over the
//     objectives of the prefix bitsets, masked by q > p (diagonal blocks) and
//     by the runs of identical points. One 64-bit store per lane writes two
//     rows' 128-byte segments per warp instruction; the dominator count of
//     every column (column sums of D) is accumulated by Harley-Seal
//     bit-sliced counters per lane.
// emo_dominance (caller order, full matrix): k_dom_full compares every
//   ordered pair directly ("all <= and some <").
#include "emo_kernels.cuh"

namespace emo {

constexpr int kDomNH = 7;  // high count planes: up to 2047 rows per lane and item
static_assert(kDomRowChunk / 16 * 16 < (1 << (4 + kDomNH)), "column counter overflow");
constexpr long long kCopyWaitCycles = 1ll << 32;
constexpr int kHalf = kColBlock / 2;

// Geometry of the per-objective prefix-set blocks (runtime form).
struct PrefGeom {
    int log_cps, cps, obj_bytes, ord_off;
    __device__ __forceinline__ explicit PrefGeom(int K)
        : log_cps(colprep_log_cps(K)), cps(1 << colprep_log_cps(K)), obj_bytes((int)colprep_obj_bytes(K)),
          ord_off((int)colprep_ord_off(K))
    {
    }
};

template <int K>
struct PrefShape {
    static constexpr int LOG_CPS = colprep_log_cps(K);
    static constexpr int CPS = 1 << LOG_CPS;
    static constexpr int OBJ_BYTES = (int)colprep_obj_bytes(K);
    static constexpr int ORD_OFF = (int)colprep_ord_off(K);
};

// Decode a dominance item of one problem: column blocks are served from the
// last (tallest) to the first; each is split into chunks of `rows` row
// blocks (the problem's dom_chunk). Binary search over the closed-form item
// prefix.
__device__ __forceinline__ void dom_decode(long long local, int ncb, int nrb, int rows, int& cb, int& chunk)
{
    const long long u = dom_items_prefix(ncb, nrb, rows) - local;  // in 1 .. total
    int lo = 1, hi = ncb;                                           // smallest c with prefix(c) >= u
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (dom_items_prefix(mid, nrb, rows) >= u) hi = mid;
        else lo = mid + 1;
    }
    cb = lo - 1;
    chunk = (int)(dom_items_prefix(lo, nrb, rows) - u);
}

// Flush a warp's per-lane column counters into s_cnt (column q of the block
// at index (q % 32) * 32 + q / 32, conflict free for the warp): lane l and
// lane l + 16 both count columns 64 (l % 16) .. + 63 over their own rows.
template <int NH>
__device__ __forceinline__ void flush_counts(VCount<NH>& vlo, VCount<NH>& vhi, int32_t* s_cnt, int lane)
{
    const int top = max(vlo.top_plane(), vhi.top_plane());  // planes above are zero in every lane
    if (top >= 0) {
        const int w = 2 * (lane & 15) + (lane >> 4);  // word whose columns this lane flushes
#pragma unroll 2
        for (int b = 0; b < 32; ++b) {
            int c = vlo.count_upto(b, top);
            c += __shfl_down_sync(0xffffffffu, c, 16);
            int e = vhi.count_upto(b, top);
            e += __shfl_up_sync(0xffffffffu, e, 16);
            const int v = lane < 16 ? c : e;
            if (v) atomicAdd(&s_cnt[b * 32 + w], v);
        }
    }
    vlo = VCount<NH>();
    vhi = VCount<NH>();
}

// Bucket of x for a block's header (lowest finite value vmin, scale > 0 or
// 0): non-decreasing in x, the same arithmetic where the index is built and
// where it is searched.
__device__ __forceinline__ int pref_bucket(float x, float vmin, float scale)
{
    const int b = __float2int_rz(__fmul_rn(__fsub_rn(x, vmin), scale));
    return min(max(b, 0), kPrefBuckets - 1);
}

// ------------------------------------------------------------ k_colprep
// Slot of entry i of a block's descending values (bank-spreading swizzle).
__device__ __forceinline__ int fv_slot(int i) { return i ^ ((i >> 5) & 31); }

// Entries of a descending array of 512 floats that are >= x (strict: > x).
template <bool STRICT>
__device__ __forceinline__ int count_before512(const float* v, float x)
{
    int pos = 0;
#pragma unroll
    for (int step = 256; step > 0; step >>= 1) {
        const float y = v[pos + step - 1];
        if (STRICT ? y > x : y >= x) pos += step;
    }
    const float y = v[pos];
    if (STRICT ? y > x : y >= x) ++pos;
    return pos;
}

__global__ void __launch_bounds__(256) k_colprep(Plan* plan, int pfirst, int plast)
{
    __shared__ float s_v[kColBlock];
    __shared__ uint16_t s_i[kColBlock];
    __shared__ uint8_t s_mark[kColBlock];
    __shared__ uint32_t s_part[8][32];
    __shared__ int s_warp[32];
    __shared__ float s_full[kColBlock];  // the full descending order (bucket index)
    __shared__ float s_hdr[2];
    __shared__ int s_bh[kPrefBuckets];  // bucket histogram
    __shared__ long long s_first[kMaxBatch + 1];  // items (column block, objective) before each problem
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // key objectives 2..m of the lexicographic order, or every objective of
    // the caller-order columns (MODE_DOM)
    auto keys_of = [&](const ProbDev& d) { return d.in.mode == MODE_DOM ? d.in.m : d.in.m - 1; };
    if (tid == 0) {
        long long acc = 0;
        for (int p = pfirst; p < plast; ++p) {
            s_first[p - pfirst] = acc;
            const ProbDev& d = plan->p[p];
            if (ld_volatile(&d.sc->status) == 0) acc += (long long)d.ncb * keys_of(d);
        }
        s_first[plast - pfirst] = acc;
    }
    __syncthreads();
    // the items of every problem in one sequence (a batch's small problems
    // together fill the grid)
    const long long total = s_first[plast - pfirst];
    int p = pfirst;
    for (long long it_all = blockIdx.x; it_all < total; it_all += gridDim.x) {
        while (s_first[p + 1 - pfirst] <= it_all) ++p;
        const ProbDev& d = plan->p[p];
        const bool caller = d.in.mode == MODE_DOM;
        const int K = keys_of(d);
        const float* const kv = caller ? d.ckeys : d.keys;
        const PrefGeom G(K);
        const int ncp1 = kHalf >> G.log_cps;  // checkpoints after the first
        const long long it = it_all - s_first[p - pfirst];
        const int cb = (int)(it / K), k = (int)(it % K);
        unsigned char* blk = d.colpre + ((int64_t)cb * K + k) * G.obj_bytes;
        for (int q = tid; q < kColBlock; q += blockDim.x) {
            s_v[q] = kv[((int64_t)cb * kColBlock + q) * K + k];
            s_i[q] = (uint16_t)q;
        }
        __syncthreads();
        // bitonic sort: half ascending, then value descending, then local
        // index ascending (positions 0..511 = half 0, 512..1023 = half 1)
        for (int size = 2; size <= kColBlock; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int t = tid; t < kColBlock / 2; t += blockDim.x) {
                    const int i = 2 * t - (t & (stride - 1)), j = i + stride;
                    const float vi = s_v[i], vj = s_v[j];
                    const int ii = s_i[i], ij = s_i[j];
                    const int hi_ = ii >= kHalf, hj = ij >= kHalf;
                    const bool j_first = hj < hi_ || (hj == hi_ && (vj > vi || (vj == vi && ij < ii)));
                    const bool up = (i & size) == 0;
                    if (up == j_first) {
                        s_v[i] = vj; s_v[j] = vi;
                        s_i[i] = (uint16_t)ij; s_i[j] = (uint16_t)ii;
                    }
                }
                __syncthreads();
            }
        }
        float* fv = reinterpret_cast<float*>(blk);
        uint16_t* cum0 = reinterpret_cast<uint16_t*>(blk + kPrefCumOff);
        uint32_t* pb = reinterpret_cast<uint32_t*>(blk + kPrefPbOff);
        if (G.log_cps > 0) {
            uint16_t* so = reinterpret_cast<uint16_t*>(blk + G.ord_off);
            for (int q = tid; q < kColBlock; q += blockDim.x) so[q] = s_i[q];
        }
        // merge of the halves into the full descending order (ties: half 0
        // first); mark the half-0 positions
        for (int q = tid; q < kColBlock; q += blockDim.x) {
            const float x = s_v[q];
            const int rank = (q & (kHalf - 1)) +
                             (q < kHalf ? count_before512<true>(s_v + kHalf, x) : count_before512<false>(s_v, x));
            fv[fv_slot(rank)] = x;
            s_mark[rank] = q < kHalf;
            if (colprep_has_buckets(K)) s_full[rank] = x;
        }
        if (colprep_has_buckets(K)) {
            // bucket index: header (vmin, scale), then per bucket b the
            // positions [lo, hi) of the values whose bucket is b (the
            // bucket is non-increasing along the descending order)
            __syncthreads();
            float* hdr = reinterpret_cast<float*>(blk + colprep_bkt_off(K));
            uint32_t* tab = reinterpret_cast<uint32_t*>(blk + colprep_bkt_off(K) + 128);
            if (tid == 0) {
                int nf = kColBlock;  // finite entries (padding columns hold -inf)
                while (nf > 1 && !(s_full[nf - 1] > -INFINITY)) --nf;
                const float vmax = s_full[0], vmin = s_full[nf - 1];
                float sc = vmax > vmin ? (float)kPrefBuckets / (vmax - vmin) : 0.0f;
                if (!(sc < 1e30f)) sc = 0.0f;  // overflowed span or tiny span: one bucket
                s_hdr[0] = vmin;
                s_hdr[1] = sc;
                hdr[0] = vmin;
                hdr[1] = sc;
            }
            __syncthreads();
            const float vmin = s_hdr[0], sc = s_hdr[1];
            // histogram of the values' buckets, then per bucket b:
            // lo = #{bucket > b}, hi = #{bucket >= b} (a block scan)
            constexpr int PER = kPrefBuckets / 256;
            for (int b = tid; b < kPrefBuckets; b += blockDim.x) s_bh[b] = 0;
            __syncthreads();
            for (int q = tid; q < kColBlock; q += blockDim.x) atomicAdd(&s_bh[pref_bucket(s_full[q], vmin, sc)], 1);
            __syncthreads();
            int h[PER], sum = 0;
#pragma unroll
            for (int e = 0; e < PER; ++e) {
                h[e] = s_bh[tid * PER + e];
                sum += h[e];
            }
            int tot;
            int below = block_exclusive_scan<256>(sum, s_warp, tot);  // #{bucket < tid * PER}
#pragma unroll
            for (int e = 0; e < PER; ++e) {
                const int hi = kColBlock - below;
                below += h[e];
                tab[tid * PER + e] = (uint32_t)(kColBlock - below) | ((uint32_t)hi << 16);
            }
            __syncthreads();  // s_warp is scanned again below
        }
        // interleaved prefix bitsets: lane w builds word w from the sorted
        // columns of half w / 16; warp v covers checkpoints (v*seg, (v+1)*seg]
        const int hbase = (lane >> 4) * kHalf;
        const int seg = ncp1 / 8;
        uint32_t part = 0u;
        for (int c = warp * seg; c < (warp + 1) * seg; ++c)
            for (int e = 0; e < G.cps; ++e) {
                const int col = s_i[hbase + c * G.cps + e];
                if ((col >> 5) == lane) part |= 1u << (col & 31);
            }
        s_part[warp][lane] = part;
        __syncthreads();
        uint32_t acc = 0u;
        for (int w = 0; w < warp; ++w) acc |= s_part[w][lane];
        if (warp == 0) pb[lane] = 0u;
        for (int c = warp * seg; c < (warp + 1) * seg; ++c) {
            for (int e = 0; e < G.cps; ++e) {
                const int col = s_i[hbase + c * G.cps + e];
                if ((col >> 5) == lane) acc |= 1u << (col & 31);
            }
            pb[(c + 1) * 32 + lane] = acc;
        }
        // cum0[j] = half-0 entries among the first j of the full order
        {
            const int j0 = tid * 4;  // 256 threads x 4 entries
            const int m0 = s_mark[j0], m1 = s_mark[j0 + 1], m2 = s_mark[j0 + 2], m3 = s_mark[j0 + 3];
            int tot;
            const int ex = block_exclusive_scan<256>(m0 + m1 + m2 + m3, s_warp, tot);
            if (tid == 0) cum0[0] = 0;
            cum0[j0 + 1] = (uint16_t)(ex + m0);
            cum0[j0 + 2] = (uint16_t)(ex + m0 + m1);
            cum0[j0 + 3] = (uint16_t)(ex + m0 + m1 + m2);
            cum0[j0 + 4] = (uint16_t)(ex + m0 + m1 + m2 + m3);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ k_dom_pref
// Objectives whose prefix sets have a checkpoint at every count and room in
// shared memory (at most two keys): the rows' checkpoint offsets are staged
// per warp in shared memory instead of being broadcast by shuffles.
template <int K>
constexpr bool kStageOffsets = K <= 2 && PrefShape<K>::LOG_CPS == 0;

template <int K>
struct PrefSmem {
    alignas(128) unsigned char obj[K * PrefShape<K>::OBJ_BYTES];
    alignas(128) int32_t rs[kColBlock];
    int32_t cnt[kColBlock];
    // per warp, objective and half: byte offset t * 128 of each row's checkpoint
    uint32_t off[kStageOffsets<K> ? 16 * K * 64 : 1];
    uint64_t bar;
    long long item;
    int skip;
};

// Packed counts of the block's values >= x in both halves of one objective:
// t0 | t1 << 16 (binary search over the full descending order, then the
// half-0 share of that prefix). Entry i of the order is stored at fv_slot(i):
// the candidates of one search level are i = c * step - 1 for step >= 32, all
// with the same low five bits, and the XOR with i / 32 puts them in distinct
// shared-memory banks.
__device__ __forceinline__ int count_ge_halves(const unsigned char* ob, float x)
{
    const float* fv = reinterpret_cast<const float*>(ob);
    int pos = 0;
#pragma unroll
    for (int step = kColBlock / 2; step > 0; step >>= 1)
        if (fv[fv_slot(pos + step - 1)] >= x) pos += step;
    if (fv[fv_slot(pos)] >= x) ++pos;
    const int t0 = reinterpret_cast<const uint16_t*>(ob + kPrefCumOff)[pos];
    return t0 | ((pos - t0) << 16);
}

// count_ge_halves through the bucket index (objectives with at most two
// keys): every value of a higher bucket is >= x, every value of a lower one
// < x, so the count is the bucket's first position plus the values >= x
// among the bucket's own (a short search, usually over one or none).
template <int K>
__device__ __forceinline__ int count_ge_halves_k(const unsigned char* ob, float x)
{
    if constexpr (!colprep_has_buckets(K)) {
        return count_ge_halves(ob, x);
    } else {
        const float* fv = reinterpret_cast<const float*>(ob);
        const float* hdr = reinterpret_cast<const float*>(ob + colprep_bkt_off(K));
        const uint32_t e =
            reinterpret_cast<const uint32_t*>(ob + colprep_bkt_off(K) + 128)[pref_bucket(x, hdr[0], hdr[1])];
        int lo = (int)(e & 0xffffu), hi = (int)(e >> 16);
        while (lo < hi) {  // first position of the bucket with a value < x
            const int mid = (lo + hi) >> 1;
            if (fv[fv_slot(mid)] >= x) lo = mid + 1;
            else hi = mid;
        }
        const int t0 = reinterpret_cast<const uint16_t*>(ob + kPrefCumOff)[lo];
        return t0 | ((lo - t0) << 16);
    }
}

// Two words (columns 64 l .. 64 l + 63, l = lane % 16) of an objective's
// prefix set for a count t of the lane's half.
template <int LOG_CPS, int ORD_OFF>
__device__ __forceinline__ unsigned long long prefix_word(const unsigned char* ob, int t, int l)
{
    const int c = t >> LOG_CPS;
    unsigned long long w = *reinterpret_cast<const unsigned long long*>(ob + kPrefPbOff + c * 128 + l * 8);
    if (LOG_CPS > 0) {
        constexpr int CPS = 1 << LOG_CPS;
        const int rem = t & (CPS - 1);
        const uint16_t* so = reinterpret_cast<const uint16_t*>(ob + ORD_OFF) + (l >> 3) * kHalf;
#pragma unroll
        for (int e = 0; e < CPS - 1; ++e) {
            const int col = so[min((c << LOG_CPS) + e, kHalf - 1)];
            const bool hit = (e < rem) & ((col >> 6) == l);
            w |= hit ? (1ull << (col & 63)) : 0ull;
        }
    }
    return w;
}

// Keep columns q > p of the lane's 64 (diagonal blocks), drop identical points.
template <bool DIAG, bool DUP>
__device__ __forceinline__ unsigned long long row_masks(unsigned long long word, int64_t prow, int64_t cbase,
                                                        const int32_t* __restrict__ rs, int l)
{
    if (DIAG) {
        const int64_t off = prow - (cbase + 64 * l);
        const int sh = (int)(off < 0 ? 0 : (off > 62 ? 63 : off + 1));  // shift count in [0, 63]
        word &= off >= 63 ? 0ull : (off >= 0 ? ~0ull << sh : ~0ull);
    }
    if (DUP && word) {
#pragma unroll 4
        for (int bb = 0; bb < 64; ++bb) {
            const int b = (bb + l) & 63;
            if ((int64_t)rs[64 * l + b] <= prow) word &= ~(1ull << b);
        }
    }
    return word;
}

// The 32 rows of row block rb in column block cb; t[k] is the packed count
// (half 0 | half 1 << 16) of objective k for the lane's row.
// DIAG: the row block overlaps the column block (keep q > p only).
// DUP: a run of identical points may reach into the column block.
template <int K, bool DIAG, bool DUP>
__device__ __forceinline__ void pref_rows(const unsigned char* __restrict__ obj, const int32_t* __restrict__ rs,
                                          const int (&t)[K], int64_t rowbase, int64_t cbase, uint32_t* tile,
                                          VCount<kDomNH>& vlo, VCount<kDomNH>& vhi, int lane)
{
    using S = PrefShape<K>;
    const int l = lane & 15, h = lane >> 4;
    const unsigned psel = (l >> 3) ? 0x4432u : 0x4410u;  // byte selector of the lane's half count
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(tile + h * 16 * 32) + l;
#pragma unroll 1
    for (int g = 0; g < 2; ++g) {
        uint32_t xl[8], xh[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
            const int j = g * 8 + jj, i = j + 16 * h;
            unsigned long long word = ~0ull;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int tk = (int)__byte_perm((unsigned)__shfl_sync(0xffffffffu, t[k], i), 0u, psel);
                word &= prefix_word<S::LOG_CPS, S::ORD_OFF>(obj + k * S::OBJ_BYTES, tk, l);
            }
            word = row_masks<DIAG, DUP>(word, rowbase + i, cbase, rs, l);
            __stcs(dst + j * 16, word);
            xl[jj] = (uint32_t)word;
            xh[jj] = (uint32_t)(word >> 32);
        }
        vlo.add8_warp(xl);
        vhi.add8_warp(xh);
    }
}

// pref_rows with the rows' checkpoint offsets read from this warp's staged
// offsets `so` ([K][2 halves][32 rows], bytes t * 128 of the half's count):
// one shared load per row and objective replaces a shuffle, a byte permute
// and the offset arithmetic.
template <int K, bool DIAG, bool DUP>
__device__ __forceinline__ void pref_rows_off(const unsigned char* __restrict__ obj,
                                              const int32_t* __restrict__ rs, const uint32_t* so, int64_t rowbase,
                                              int64_t cbase, uint32_t* tile, VCount<kDomNH>& vlo,
                                              VCount<kDomNH>& vhi, int lane)
{
    using S = PrefShape<K>;
    const int l = lane & 15, h = lane >> 4;
    const uint32_t* my = so + (l >> 3) * 32 + 16 * h;  // this lane's half; rows j + 16 h
    const unsigned char* pb = obj + kPrefPbOff + l * 8;
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(tile + h * 16 * 32) + l;
#pragma unroll 1
    for (int g = 0; g < 2; ++g) {
        uint32_t xl[8], xh[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
            const int j = g * 8 + jj;
            unsigned long long word = ~0ull;
#pragma unroll
            for (int k = 0; k < K; ++k)
                word &= *reinterpret_cast<const unsigned long long*>(pb + k * S::OBJ_BYTES + my[k * 64 + j]);
            word = row_masks<DIAG, DUP>(word, rowbase + j + 16 * h, cbase, rs, l);
            __stcs(dst + j * 16, word);
            xl[jj] = (uint32_t)word;
            xh[jj] = (uint32_t)(word >> 32);
        }
        vlo.add8_warp(xl);
        vhi.add8_warp(xh);
    }
}

// Stage the prefix sets of column block cb (and its run starts); returns
// false when the problem is skipped or the copy timed out.
__device__ __forceinline__ bool dom_stage(const ProbDev& d, int cb, int K, int obj_bytes, unsigned char* obj,
                                          int32_t* rs, int32_t* cnt, uint64_t* bar, int* s_skip, uint32_t& parity,
                                          bool& fatal)
{
    const int tid = threadIdx.x;
    const uint32_t ob = (uint32_t)(K * obj_bytes);
    if (tid == 0) {
        *s_skip = ld_volatile(&d.sc->status) != 0 || d.in.m - 1 != K;
        if (!*s_skip) {
            fence_proxy_async_smem();
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                         "r"(ob + (uint32_t)(kColBlock * 4))
                         : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(obj)),
                "l"(d.colpre + (int64_t)cb * ob), "r"(ob), "r"(smem_u32(bar))
                : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(rs)),
                "l"(d.runstart + (int64_t)cb * kColBlock), "r"((uint32_t)(kColBlock * 4)), "r"(smem_u32(bar))
                : "memory");
        }
    }
    for (int i = tid; i < kColBlock; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    if (*s_skip) return false;
    // The copy is a local load that always completes; the bound only guards
    // against a lost completion. On timeout the status is set and the CTA
    // still waits (bounded) so that no copy is in flight at exit.
    if (!mbar_wait(bar, parity, kCopyWaitCycles)) {
        if (tid == 0) set_status(d.sc, EMO_ERR_TIMEOUT);
        mbar_wait(bar, parity, kCopyWaitCycles);
        fatal = true;
        return false;
    }
    parity ^= 1u;
    return true;
}

// Column counts of the item: smem reduction, one global atomic per column.
__device__ __forceinline__ void dom_flush_item(const ProbDev& d, int64_t cbase, VCount<kDomNH>& vlo,
                                               VCount<kDomNH>& vhi, int32_t* cnt, int lane)
{
    flush_counts(vlo, vhi, cnt, lane);
    __syncthreads();
    for (int q = threadIdx.x; q < kColBlock; q += blockDim.x) {
        const int c = cnt[(q & 31) * 32 + (q >> 5)];
        if (c) atomicAdd(&d.cnt[cbase + q], c);
    }
    __syncthreads();
}

template <int M>
__global__ void __launch_bounds__(512, 1) k_dom_pref(Plan* plan, long long item_lo, long long item_hi,
                                                     unsigned long long* counter)
{
    constexpr int K = M - 1, NW = 16;
    using S = PrefShape<K>;
    extern __shared__ __align__(128) unsigned char smraw[];
    PrefSmem<K>& sm = *reinterpret_cast<PrefSmem<K>*>(smraw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) mbar_init(&sm.bar, 1);
    __syncthreads();
    uint32_t parity = 0;

    while (true) {
        if (tid == 0) sm.item = item_lo + (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long item = sm.item;
        if (item >= item_hi) break;
        int p = 0;
        while (p + 1 < plan->nprob && plan->dom_item_start[p + 1] <= item) ++p;
        const ProbDev& d = plan->p[p];
        int cb, chunk;
        const int rows = d.in.dom_chunk;
        dom_decode(item - plan->dom_item_start[p], d.ncb, d.nrb, rows, cb, chunk);
        bool fatal = false;
        if (!dom_stage(d, cb, K, S::OBJ_BYTES, sm.obj, sm.rs, sm.cnt, &sm.bar, &sm.skip, parity, fatal)) {
            if (fatal) break;
            continue;
        }
        const int64_t n2 = d.in.n2;
        const int rbmax = min(d.nrb, 32 * (cb + 1));
        const int rb_lo = chunk * rows, rb_hi = min(rbmax, rb_lo + rows);
        const int dupcut = d.minrs[cb];
        const int64_t cbase = (int64_t)cb * kColBlock;
        // in registers: the tile stores could alias the plan, which would
        // otherwise reload these after every row block
        uint32_t* const Dm = d.D;
        const float* const keys = d.keys;
        const int ncb = d.ncb;
        VCount<kDomNH> vlo, vhi;

        // keys of the lane's row in the warp's next row block (prefetched)
        float key[K];
        {
            const int64_t pl = (int64_t)(rb_lo + warp) * kTileRows + lane;
#pragma unroll
            for (int k = 0; k < K; ++k) key[k] = (rb_lo + warp < rb_hi && pl < n2) ? __ldg(&keys[pl * K + k]) : 0.0f;
        }
        for (int rb = rb_lo + warp; rb < rb_hi; rb += NW) {
            const int64_t pl = (int64_t)rb * kTileRows + lane;
            int t[K];
#pragma unroll
            for (int k = 0; k < K; ++k) t[k] = pl < n2 ? count_ge_halves_k<K>(sm.obj + k * S::OBJ_BYTES, key[k]) : 0;
            {
                const int rbn = rb + NW;
                const int64_t pn = (int64_t)rbn * kTileRows + lane;
#pragma unroll
                for (int k = 0; k < K; ++k) key[k] = (rbn < rb_hi && pn < n2) ? __ldg(&keys[pn * K + k]) : 0.0f;
            }
            const bool diag = (int64_t)rb * kTileRows + 31 >= cbase;
            const bool dup = rb * kTileRows + 31 >= dupcut;
            const int64_t rowbase = (int64_t)rb * kTileRows;
            uint32_t* tile = Dm + tile_index(rb, cb, ncb) * (int64_t)(kTileRows * kTileWords);
            if constexpr (kStageOffsets<K>) {
                uint32_t* so = sm.off + warp * (K * 64);
                __syncwarp();  // the previous row block's offsets have been read
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    so[k * 64 + lane] = (uint32_t)(t[k] & 0xffff) * 128u;
                    so[k * 64 + 32 + lane] = (uint32_t)(t[k] >> 16) * 128u;
                }
                __syncwarp();
                if (dup) pref_rows_off<K, true, true>(sm.obj, sm.rs, so, rowbase, cbase, tile, vlo, vhi, lane);
                else if (diag) pref_rows_off<K, true, false>(sm.obj, sm.rs, so, rowbase, cbase, tile, vlo, vhi, lane);
                else pref_rows_off<K, false, false>(sm.obj, sm.rs, so, rowbase, cbase, tile, vlo, vhi, lane);
            } else {
                if (dup) pref_rows<K, true, true>(sm.obj, sm.rs, t, rowbase, cbase, tile, vlo, vhi, lane);
                else if (diag) pref_rows<K, true, false>(sm.obj, sm.rs, t, rowbase, cbase, tile, vlo, vhi, lane);
                else pref_rows<K, false, false>(sm.obj, sm.rs, t, rowbase, cbase, tile, vlo, vhi, lane);
            }
        }
        dom_flush_item(d, cbase, vlo, vhi, sm.cnt, lane);
    }
}

// ------------------------------------------------------------ k_dom_caller
// The full dominance matrix in the caller's order (emo_dominance_ws) by the
// same prefix sets, built over caller-order column blocks for all K = m
// objectives: the set {q : f_k(q) >= f_k(p) for every k} is the AND of K
// prefix sets, and p dominates q iff q is in that set and is not identical to
// p (all equal: p itself and its exact duplicates, found as the runs of the
// lexicographic sort). Items: (column block, chunk of row blocks) over the
// whole square; a half-warp builds one 1024-column row segment at a time
// (a lane owns 64 columns), written into row p of D; column counts as in
// k_dom_pref. m <= 5 (the blocks' prefix data must fit in shared memory).
// Set-up of the caller-order matrix after the sort: the objectives in the
// caller's order padded with -inf to whole column blocks (the prefix sets of
// every objective are built on them), and each point's run of identical
// points in sorted positions (first, one past the last; first = -1 when the
// point has no duplicate).
__global__ void k_dom_keys(Plan* plan)
{
    const ProbDev& d = plan->p[0];
    if (d.in.mode != MODE_DOM || ld_volatile(&d.sc->status) != 0) return;
    const int m = d.in.m;
    const int64_t n2 = d.in.n2;
    const int32_t* idx = d.idx + (int64_t)ld_volatile(&d.sc->idx_buf) * d.n2p;
    const int32_t* rs = d.runstart;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < d.n2p * m; e += stride)
        d.ckeys[e] = e / m < n2 ? d.in.F[e] + 0.0f : -INFINITY;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n2; s += stride) {
        const int r0 = rs[s];
        int r1 = (int)s + 1;
        while (r1 < n2 && rs[r1] == r0) ++r1;
        const int q = idx[s];
        d.spos[q] = (r1 - r0 > 1) ? r0 : -1;
        d.spos[n2 + q] = r1;
    }
}

template <int K>
struct CallerSmem {
    alignas(128) unsigned char obj[K * PrefShape<K>::OBJ_BYTES];
    int32_t cnt[kColBlock];
    uint64_t bar;
    long long item;
    int skip;
};

template <int K>
__global__ void __launch_bounds__(512, 1) k_dom_caller(Plan* plan, long long nitems, unsigned long long* counter)
{
    constexpr int NW = 16;
    using S = PrefShape<K>;
    extern __shared__ __align__(128) unsigned char smraw[];
    CallerSmem<K>& sm = *reinterpret_cast<CallerSmem<K>*>(smraw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int l = lane & 15, h = lane >> 4;
    const unsigned psel = (l >> 3) ? 0x4432u : 0x4410u;  // byte selector of the lane's half count
    if (tid == 0) mbar_init(&sm.bar, 1);
    __syncthreads();
    uint32_t parity = 0;
    const ProbDev& d = plan->p[0];
    const int64_t n2 = d.in.n2, ld = d.in.dom_ld;
    const int nrb = d.nrb;
    const int rows = d.in.dom_chunk;
    const long long per_cb = cdiv(nrb, rows);
    const bool st64 = (ld % 2 == 0) && ((reinterpret_cast<uintptr_t>(d.in.dom_out) & 7) == 0);
    const int32_t* const idx = d.idx + (int64_t)ld_volatile(&d.sc->idx_buf) * d.n2p;
    const int32_t* const spos = d.spos;
    const float* const ck = d.ckeys;
    uint32_t* const Dout = d.in.dom_out;
    while (true) {
        if (tid == 0) sm.item = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long item = sm.item;
        if (item >= nitems) break;
        const int cb = (int)(item / per_cb), chunk = (int)(item % per_cb);
        if (tid == 0) {
            sm.skip = ld_volatile(&d.sc->status) != 0;
            if (!sm.skip) {
                fence_proxy_async_smem();
                bulk_load(sm.obj, d.colpre + (int64_t)cb * (K * S::OBJ_BYTES), (uint32_t)(K * S::OBJ_BYTES), &sm.bar);
            }
        }
        for (int i = tid; i < kColBlock; i += blockDim.x) sm.cnt[i] = 0;
        __syncthreads();
        if (sm.skip) break;
        if (!mbar_wait(&sm.bar, parity, kCopyWaitCycles)) {
            if (tid == 0) set_status(d.sc, EMO_ERR_TIMEOUT);
            mbar_wait(&sm.bar, parity, kCopyWaitCycles);
            break;
        }
        parity ^= 1u;
        const int64_t cbase = (int64_t)cb * kColBlock;
        const int rb_lo = chunk * rows, rb_hi = min(nrb, rb_lo + rows);
        VCount<kDomNH> vlo, vhi;
        // keys and duplicate run of the lane's row in the warp's next row block (prefetched)
        float key[K];
        int nlo = -1, nhi = 0;
        {
            const int64_t pn = (int64_t)(rb_lo + warp) * kTileRows + lane;
            const bool ok = rb_lo + warp < rb_hi && pn < n2;
#pragma unroll
            for (int k = 0; k < K; ++k) key[k] = ok ? __ldg(&ck[pn * K + k]) : 0.0f;
            if (ok) {
                nlo = __ldg(&spos[pn]);
                nhi = __ldg(&spos[n2 + pn]);
            }
        }
        for (int rb = rb_lo + warp; rb < rb_hi; rb += NW) {
            const int64_t pl = (int64_t)rb * kTileRows + lane;  // the lane's row (search)
            int t[K];
#pragma unroll
            for (int k = 0; k < K; ++k) t[k] = pl < n2 ? count_ge_halves_k<K>(sm.obj + k * S::OBJ_BYTES, key[k]) : 0;
            // duplicates of the lane's row: sorted positions [dup_lo, dup_hi) when it has any
            const int dup_lo = nlo >= 0 ? nlo : 0, dup_hi = nlo >= 0 ? nhi : 0;
            {
                const int rbn = rb + NW;
                const int64_t pn = (int64_t)rbn * kTileRows + lane;
                const bool ok = rbn < rb_hi && pn < n2;
#pragma unroll
                for (int k = 0; k < K; ++k) key[k] = ok ? __ldg(&ck[pn * K + k]) : 0.0f;
                nlo = ok ? __ldg(&spos[pn]) : -1;
                nhi = ok ? __ldg(&spos[n2 + pn]) : 0;
            }
#pragma unroll 1
            for (int g = 0; g < 2; ++g) {
                uint32_t xl[8], xh[8];
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    const int j = g * 8 + jj, i = j + 16 * h;  // row of the block this half-warp builds
                    const int64_t p = (int64_t)rb * kTileRows + i;
                    unsigned long long word = ~0ull;
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const int tk = (int)__byte_perm((unsigned)__shfl_sync(0xffffffffu, t[k], i), 0u, psel);
                        word &= prefix_word<S::LOG_CPS, S::ORD_OFF>(sm.obj + k * S::OBJ_BYTES, tk, l);
                    }
                    // not identical to p: p itself, and its duplicates
                    const int dlo = __shfl_sync(0xffffffffu, dup_lo, i), dhi = __shfl_sync(0xffffffffu, dup_hi, i);
                    if (dhi > dlo) {
                        for (int r = dlo; r < dhi; ++r) {
                            const int64_t off = (int64_t)__ldg(&idx[r]) - cbase - 64 * l;
                            if (off >= 0 && off < 64) word &= ~(1ull << off);
                        }
                    } else {
                        const int64_t off = p - cbase - 64 * l;
                        if (off >= 0 && off < 64) word &= ~(1ull << off);
                    }
                    if (p >= n2) word = 0ull;
                    if (p < n2) {  // words past ld (a short last block) are not stored
                        const int64_t w0 = (int64_t)cb * 32 + 2 * l;
                        uint32_t* dst = Dout + p * ld + w0;
                        if (st64 && w0 + 1 < ld) {
                            __stcs(reinterpret_cast<unsigned long long*>(dst), word);
                        } else {
                            if (w0 < ld) __stcs(dst, (uint32_t)word);
                            if (w0 + 1 < ld) __stcs(dst + 1, (uint32_t)(word >> 32));
                        }
                    }
                    xl[jj] = (uint32_t)word;
                    xh[jj] = (uint32_t)(word >> 32);
                }
                vlo.add8_warp(xl);
                vhi.add8_warp(xh);
            }
        }
        // column counts of the item: shared-memory reduction, one global atomic per column
        flush_counts(vlo, vhi, sm.cnt, lane);
        __syncthreads();
        if (d.in.dom_count)
            for (int q = tid; q < kColBlock; q += blockDim.x) {
                const int c = sm.cnt[(q & 31) * 32 + (q >> 5)];
                if (c && cbase + q < n2) atomicAdd(&d.in.dom_count[cbase + q], c);
            }
        __syncthreads();
    }
}

// Runtime-K variant for m >= 7 (compact code: loops over the key objectives
// are not unrolled; the packed half counts of a row block are staged in
// shared memory).
__global__ void __launch_bounds__(512, 1) k_dom_pref_rt(Plan* plan, long long item_lo, long long item_hi,
                                                        unsigned long long* counter, int K)
{
    constexpr int NW = 16;
    const PrefGeom G(K);
    extern __shared__ __align__(128) unsigned char smraw[];
    const int obj_total = K * G.obj_bytes;
    unsigned char* obj = smraw;
    int32_t* rs = reinterpret_cast<int32_t*>(smraw + ((obj_total + 127) & ~127));
    int32_t* cnt = rs + kColBlock;
    int32_t* st = cnt + kColBlock;  // [NW][K][32] packed half counts of the warp's row block
    uint64_t* bar = reinterpret_cast<uint64_t*>(st + NW * K * 32);
    long long* s_item = reinterpret_cast<long long*>(bar + 1);
    int* s_skip = reinterpret_cast<int*>(s_item + 1);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int32_t* myst = st + warp * K * 32;
    const int l = lane & 15, h = lane >> 4, half = l >> 3, hs = half * 16;
    if (tid == 0) mbar_init(bar, 1);
    __syncthreads();
    uint32_t parity = 0;

    while (true) {
        if (tid == 0) *s_item = item_lo + (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long item = *s_item;
        if (item >= item_hi) break;
        int p = 0;
        while (p + 1 < plan->nprob && plan->dom_item_start[p + 1] <= item) ++p;
        const ProbDev& d = plan->p[p];
        int cb, chunk;
        const int rows = d.in.dom_chunk;
        dom_decode(item - plan->dom_item_start[p], d.ncb, d.nrb, rows, cb, chunk);
        bool fatal = false;
        if (!dom_stage(d, cb, K, G.obj_bytes, obj, rs, cnt, bar, s_skip, parity, fatal)) {
            if (fatal) break;
            continue;
        }
        const int64_t n2 = d.in.n2;
        const int rbmax = min(d.nrb, 32 * (cb + 1));
        const int rb_lo = chunk * rows, rb_hi = min(rbmax, rb_lo + rows);
        const int dupcut = d.minrs[cb];
        const int64_t cbase = (int64_t)cb * kColBlock;
        uint32_t* const Dm = d.D;
        const float* const keys = d.keys;
        const int ncb = d.ncb;
        VCount<kDomNH> vlo, vhi;
        for (int rb = rb_lo + warp; rb < rb_hi; rb += NW) {
            const int64_t pl = (int64_t)rb * kTileRows + lane;
            for (int k = 0; k < K; ++k)
                myst[k * 32 + lane] = pl < n2 ? count_ge_halves(obj + k * G.obj_bytes, __ldg(&keys[pl * K + k])) : 0;
            __syncwarp();
            const bool diag = (int64_t)rb * kTileRows + 31 >= cbase;
            const bool dup = rb * kTileRows + 31 >= dupcut;
            uint32_t* tile = Dm + tile_index(rb, cb, ncb) * (int64_t)(kTileRows * kTileWords);
            unsigned long long* dst = reinterpret_cast<unsigned long long*>(tile + h * 16 * 32) + l;
#pragma unroll 1
            for (int g = 0; g < 2; ++g) {
                uint32_t xl[8], xh[8];
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    const int j = g * 8 + jj, i = j + 16 * h;
                    unsigned long long word = ~0ull;
#pragma unroll 1
                    for (int k = 0; k < K; ++k) {
                        const unsigned char* ob = obj + k * G.obj_bytes;
                        const int t = (myst[k * 32 + i] >> hs) & 0xFFFF;
                        const int c = t >> G.log_cps;
                        unsigned long long wk =
                            *reinterpret_cast<const unsigned long long*>(ob + kPrefPbOff + c * 128 + l * 8);
                        const int rem = t & (G.cps - 1);
                        const uint16_t* so =
                            reinterpret_cast<const uint16_t*>(ob + G.ord_off) + half * kHalf + (c << G.log_cps);
                        for (int e = 0; e < rem; ++e) {
                            const int col = so[e];
                            if ((col >> 6) == l) wk |= 1ull << (col & 63);
                        }
                        word &= wk;
                    }
                    const int64_t prow = (int64_t)rb * kTileRows + i;
                    if (dup) word = row_masks<true, true>(word, prow, cbase, rs, l);
                    else if (diag) word = row_masks<true, false>(word, prow, cbase, rs, l);
                    __stcs(dst + j * 16, word);
                    xl[jj] = (uint32_t)word;
                    xh[jj] = (uint32_t)(word >> 32);
                }
                vlo.add8_warp(xl);
                vhi.add8_warp(xh);
            }
            __syncwarp();
        }
        dom_flush_item(d, cbase, vlo, vhi, cnt, lane);
    }
}

// Full matrix in caller order: D_ij = all(F_i <= F_j) and any(F_i < F_j).
constexpr int kFullNH = 8;  // up to 4095 rows per lane and item
template <int M>
struct FullSmem {
    alignas(16) float ck[kColBlock * M];
    alignas(16) uint32_t tiles[8][2][kTileRows * kTileWords];
    int32_t cnt[kColBlock];
    long long item;
};

// Columns [col_lo, col_hi) (col_lo a multiple of 1024); D word w of a row
// holds columns col_lo + 32 w .. + 31, dom_count[j - col_lo] their sums.
template <int M>
__global__ void __launch_bounds__(256, 1) k_dom_full(const float* __restrict__ F, int64_t n2, int64_t col_lo,
                                                     int64_t col_hi, uint32_t* D, int64_t ld, int32_t* cnt,
                                                     long long nitems)
{
    constexpr int R = 2, NW = 8;
    extern __shared__ __align__(128) unsigned char smraw[];
    FullSmem<M>& sm = *reinterpret_cast<FullSmem<M>*>(smraw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nrb = (int)cdiv(n2, 32);
    const long long per_cb = cdiv(nrb, kDomRowChunk);
    const int cb_lo = (int)(col_lo / kColBlock);
    for (long long item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int cb = cb_lo + (int)(item / per_cb), chunk = (int)(item % per_cb);
        const int64_t cbase = (int64_t)cb * kColBlock;
        for (int i = tid; i < kColBlock * M; i += blockDim.x) {
            const int64_t q = cbase + i / M;
            sm.ck[i] = q < col_hi ? F[q * M + i % M] + 0.0f : -INFINITY;
        }
        for (int i = tid; i < kColBlock; i += blockDim.x) sm.cnt[i] = 0;
        __syncthreads();
        const int rb_lo = chunk * kDomRowChunk, rb_hi = min(nrb, rb_lo + kDomRowChunk);
        VCount<kFullNH> vc;
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
                const int64_t wcol = (int64_t)(cb - cb_lo) * 32 + lane;
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
            if (__any_sync(0xffffffffu, vc.any())) {
#pragma unroll 4
                for (int b = 0; b < 32; ++b) {
                    const int c = vc.count(b);
                    if (c) atomicAdd(&sm.cnt[b * 32 + lane], c);
                }
            }
            __syncthreads();
            for (int q = tid; q < kColBlock; q += blockDim.x) {
                const int c = sm.cnt[(q & 31) * 32 + (q >> 5)];
                if (c && cbase + q < col_hi) atomicAdd(&cnt[cbase + q - col_lo], c);
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
    const size_t smem = sizeof(PrefSmem<M - 1>);
    cudaError_t e = cudaFuncSetAttribute(k_dom_pref<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dom_pref<M>, 512, smem);
    if (e != cudaSuccess) return e;
    long long grid = (long long)sms * (occ > 0 ? occ : 1);
    if (grid > hi - lo) grid = hi - lo;
    if (grid < 1) return cudaSuccess;
    k_dom_pref<M><<<(unsigned)grid, 512, smem, s>>>(plan, lo, hi, counter);
    return cudaGetLastError();
}

static cudaError_t launch_tri_rt(int K, Plan* plan, int sms, cudaStream_t s, long long lo, long long hi,
                                 unsigned long long* counter)
{
    const int obj_total = K * (int)colprep_obj_bytes(K);
    const size_t smem = (size_t)((obj_total + 127) & ~127) + 2 * kColBlock * 4 + 16 * K * 32 * 4 + 64;
    cudaError_t e = cudaFuncSetAttribute(k_dom_pref_rt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dom_pref_rt, 512, smem);
    if (e != cudaSuccess) return e;
    long long grid = (long long)sms * (occ > 0 ? occ : 1);
    if (grid > hi - lo) grid = hi - lo;
    if (grid < 1) return cudaSuccess;
    k_dom_pref_rt<<<(unsigned)grid, 512, smem, s>>>(plan, lo, hi, counter, K);
    return cudaGetLastError();
}

template <int M>
static cudaError_t launch_full_m(const float* F, int64_t n2, int64_t col_lo, int64_t col_hi, uint32_t* D, int64_t ld,
                                 int32_t* cnt, int sms, cudaStream_t s)
{
    const size_t smem = sizeof(FullSmem<M>);
    cudaError_t e = cudaFuncSetAttribute(k_dom_full<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dom_full<M>, 256, smem);
    if (e != cudaSuccess) return e;
    const long long nitems = cdiv(col_hi - col_lo, kColBlock) * cdiv(cdiv(n2, 32), kDomRowChunk);
    long long grid = (long long)sms * (occ > 0 ? occ : 1);
    if (grid > nitems) grid = nitems;
    k_dom_full<M><<<(unsigned)grid, 256, smem, s>>>(F, n2, col_lo, col_hi, D, ld, cnt, nitems);
    return cudaGetLastError();
}

template <int K>
static cudaError_t launch_caller_k(Plan* plan, int sms, cudaStream_t s, long long nitems, unsigned long long* counter)
{
    const size_t smem = sizeof(CallerSmem<K>);
    cudaError_t e = cudaFuncSetAttribute(k_dom_caller<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dom_caller<K>, 512, smem);
    if (e != cudaSuccess) return e;
    long long grid = (long long)sms * (occ > 0 ? occ : 1);
    if (grid > nitems) grid = nitems;
    if (grid < 1) return cudaSuccess;
    k_dom_caller<K><<<(unsigned)grid, 512, smem, s>>>(plan, nitems, counter);
    return cudaGetLastError();
}

cudaError_t launch_dominance_caller(int m, Plan* plan, int sms, cudaStream_t s, long long nitems,
                                    unsigned long long* counter)
{
    k_dom_keys<<<sms * 2, 256, 0, s>>>(plan);
    cudaError_t e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return e0;
    e0 = launch_colprep(plan, sms, s, 1);
    if (e0 != cudaSuccess) return e0;
    switch (m) {
    case 2: return launch_caller_k<2>(plan, sms, s, nitems, counter);
    case 3: return launch_caller_k<3>(plan, sms, s, nitems, counter);
    case 4: return launch_caller_k<4>(plan, sms, s, nitems, counter);
    case 5: return launch_caller_k<5>(plan, sms, s, nitems, counter);
    default: return cudaErrorInvalidValue;
    }
}

#define EMO_FOR_EACH_M(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

// The plan's problems are ordered by m; items of objective count m form one
// contiguous range served by the m-instantiation.
cudaError_t launch_colprep(Plan* plan, int sms, cudaStream_t s, int nprob)
{
    k_colprep<<<sms * 4, 256, 0, s>>>(plan, 0, nprob);
    return cudaGetLastError();
}

cudaError_t launch_dominance_tri_range(int m, Plan* plan, int sms, cudaStream_t s, long long lo, long long hi,
                                       unsigned long long* counter, int pfirst, int plast)
{
    (void)pfirst;
    (void)plast;
    switch (m) {
    case 2: return launch_tri_m<2>(plan, sms, s, lo, hi, counter);
    case 3: return launch_tri_m<3>(plan, sms, s, lo, hi, counter);
    case 4: return launch_tri_m<4>(plan, sms, s, lo, hi, counter);
    case 5: return launch_tri_m<5>(plan, sms, s, lo, hi, counter);
    case 6: return launch_tri_m<6>(plan, sms, s, lo, hi, counter);
    default:
        if (m < 2 || m > kMaxM) return cudaErrorInvalidValue;
        return launch_tri_rt(m - 1, plan, sms, s, lo, hi, counter);
    }
}

cudaError_t launch_dominance_full_c(const float* F, int64_t n2, int64_t col_lo, int64_t col_hi, int m, uint32_t* D,
                                    int64_t ld, int32_t* cnt, int sms, cudaStream_t s)
{
    switch (m) {
#define X(MM) \
    case MM: return launch_full_m<MM>(F, n2, col_lo, col_hi, D, ld, cnt, sms, s);
        EMO_FOR_EACH_M(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace emo
