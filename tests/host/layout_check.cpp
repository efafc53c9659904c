// Host-side check of the dominance-tile layout and the workspace carving
// (compiled by tests/test_layout.py with g++; no GPU involved).
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_2503_20286_gb300/csrc/emo_internal.cuh"

using namespace emo;

static int fail(const char* what, long long a, long long b)
{
    std::printf("FAIL %s: %lld vs %lld\n", what, a, b);
    return 1;
}

int main()
{
    const long long sizes[] = {1, 31, 32, 33, 1023, 1024, 1025, 4096, 5000, 8191, 8192, 8193, 33000, 262145, 400000};
    for (long long n2 : sizes) {
        const long long nrb = cdiv(n2, 32), ncb = cdiv(n2, kColBlock);
        // tiles are enumerated row block by row block, column blocks cb >= rb / 32
        long long idx = 0;
        for (long long rb = 0; rb < nrb; ++rb) {
            if (tiles_before(rb, ncb) != idx) return fail("tiles_before", tiles_before(rb, ncb), idx);
            for (long long cb = rb / 32; cb < ncb; ++cb, ++idx)
                if (tile_index(rb, cb, ncb) != idx) return fail("tile_index", tile_index(rb, cb, ncb), idx);
        }
        if (tiles_before(nrb, ncb) != idx) return fail("ntiles", tiles_before(nrb, ncb), idx);
        // every stored tile holds at least one (p, q) with p < q and the
        // unstored ones hold none
        for (long long rb = 0; rb < nrb; ++rb) {
            long long first_col_block = (rb * 32 + 1) / kColBlock;  // block of column p+1 for the first row
            if (rb / 32 > first_col_block) return fail("unstored tile with pairs", rb, first_col_block);
        }
        // work items cover every (row block, column block) pair of the triangle
        // once, for every item size
        for (long long chunk = kDomChunkMin; chunk <= kDomRowChunk; chunk *= 2) {
            if (!dom_chunk_ok(chunk)) return fail("dom_chunk_ok", chunk, 1);
            std::vector<int> seen(idx, 0);
            long long items = 0;
            for (long long cb = 0; cb < ncb; ++cb) {
                long long n = dom_items_of_cb(cb, nrb, chunk);
                long long rbmax = nrb < 32 * (cb + 1) ? nrb : 32 * (cb + 1);
                for (long long c = 0; c < n; ++c) {
                    for (long long rb = c * chunk; rb < rbmax && rb < (c + 1) * chunk; ++rb)
                        seen[tile_index(rb, cb, ncb)] += 1;
                    ++items;
                }
            }
            if (items != dom_items_of(n2, chunk)) return fail("dom_items_of", items, dom_items_of(n2, chunk));
            // closed-form item prefix against the per-block sum
            long long pre = 0;
            for (long long cb = 0; cb <= ncb; ++cb) {
                if (dom_items_prefix(cb, nrb, chunk) != pre)
                    return fail("dom_items_prefix", dom_items_prefix(cb, nrb, chunk), pre);
                if (cb < ncb) pre += dom_items_of_cb(cb, nrb, chunk);
            }
            for (long long t = 0; t < idx; ++t)
                if (seen[t] != 1) return fail("tile coverage", t, seen[t]);
        }
        if (dom_chunk_ok(32) || dom_chunk_ok(96) || dom_chunk_ok(2048)) return fail("dom_chunk_ok", 0, 0);
        // workspace: regions are 256-byte aligned, disjoint and inside the size
        for (int mode = MODE_RANK; mode <= MODE_SELECT; ++mode) {
            ProbIn in{};
            in.n2 = n2;
            in.m = 3;
            in.n_r = 1000;
            in.mode = mode;
            int64_t bytes = layout_problem(in, 152, nullptr, nullptr);
            std::vector<char> buf(1);
            char* base = (char*)(uintptr_t)4096;  // fake, never dereferenced
            ProbDev d{};
            int64_t b2 = layout_problem(in, 152, base, &d);
            if (b2 != bytes) return fail("layout size", b2, bytes);
            char* end = base + bytes;
            const void* ptrs[] = {d.sc, d.idx, d.keys, d.runstart, d.minrs, d.cnt, d.rank_s, d.rank_o, d.front,
                                  d.front_n, d.slist, d.hist, d.flag, d.D};
            for (const void* p : ptrs) {
                if (((uintptr_t)p % 256) != 0) return fail("alignment", (long long)(uintptr_t)p, 256);
                if ((const char*)p < base || (const char*)p >= end) return fail("bounds", (long long)(uintptr_t)p, 0);
            }
            if ((char*)d.D + d.ntiles * 4096 > end) return fail("D overflow", d.ntiles, bytes);
        }
    }
    // the allocation-free entry point's 9 MiB scratch holds the plan and one
    // selection of 2N = n_r = 7168 at any m for cooperative launches of up
    // to 608 CTAs (304 SMs at the largest occupancy used, 2), and of
    // 2N = n_r = 8192 at m <= 8 for launches of up to 304 CTAs (152 SMs)
    const long long plan_bytes = (long long)((sizeof(Plan) + 255) / 256 * 256);
    for (int m = 2; m <= kMaxM; ++m) {
        for (int big = 0; big < 2; ++big) {
            if (big && m > 8) continue;
            const long long n = big ? 8192 : 7168;
            ProbIn in{};
            in.n2 = n;
            in.m = m;
            in.n_r = (int32_t)n;
            in.mode = MODE_SELECT;
            const long long need = plan_bytes + layout_problem(in, big ? 304 : 608, nullptr, nullptr);
            if (need > (9ll << 20)) return fail("no-alloc scratch", m, need);
        }
    }
    std::printf("layout ok\n");
    return 0;
}
