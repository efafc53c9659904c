// Kernel declarations and small PTX helpers shared by the kernel files.
#pragma once

#include <cuda_runtime.h>

#include "emo_internal.cuh"

namespace emo {

// ------------------------------------------------ async-proxy bulk copies
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Global -> shared bulk copy completing on `bar` (bytes % 16 == 0, both 16-B aligned).
__device__ __forceinline__ void bulk_load(void* sdst, const void* gsrc, uint32_t bytes, uint64_t* bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(sdst)),
        "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Bounded wait for phase `parity` of `bar`; false when the budget ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long budget)
{
    long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > budget) return false;
    }
}
// Shared -> global bulk store (bulk-group completion).
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_u32(ssrc)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// ------------------------------------------- bit-sliced column counting
// Carry-save adder: (hi, lo) = a + b + c per bit position.
__device__ __forceinline__ void csa(uint32_t& hi, uint32_t& lo, uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t u = a ^ b;
    hi = (a & b) | (u & c);
    lo = u ^ c;
}

// Harley-Seal vertical counter: 32 independent per-bit counters held as bit
// planes (ones, twos, fours, eights) plus NH higher planes.
template <int NH>
struct VCount {
    uint32_t ones = 0, twos = 0, fours = 0, eights = 0;
    uint32_t hi[NH];
    __device__ __forceinline__ VCount()
    {
#pragma unroll
        for (int i = 0; i < NH; ++i) hi[i] = 0;
    }
    __device__ __forceinline__ void add16(const uint32_t* x)
    {
        uint32_t twosA, twosB, foursA, foursB, eightsA, eightsB, sixteens;
        csa(twosA, ones, ones, x[0], x[1]);
        csa(twosB, ones, ones, x[2], x[3]);
        csa(foursA, twos, twos, twosA, twosB);
        csa(twosA, ones, ones, x[4], x[5]);
        csa(twosB, ones, ones, x[6], x[7]);
        csa(foursB, twos, twos, twosA, twosB);
        csa(eightsA, fours, fours, foursA, foursB);
        csa(twosA, ones, ones, x[8], x[9]);
        csa(twosB, ones, ones, x[10], x[11]);
        csa(foursA, twos, twos, twosA, twosB);
        csa(twosA, ones, ones, x[12], x[13]);
        csa(twosB, ones, ones, x[14], x[15]);
        csa(foursB, twos, twos, twosA, twosB);
        csa(eightsB, fours, fours, foursA, foursB);
        csa(sixteens, eights, eights, eightsA, eightsB);
        uint32_t c = sixteens;
#pragma unroll
        for (int i = 0; i < NH; ++i) {
            uint32_t t = hi[i] & c;
            hi[i] ^= c;
            c = t;
        }
    }
    // Eight words at once (carry-save tree into the fours plane and below,
    // eights carry rippled into the higher planes).
    __device__ __forceinline__ void add8(const uint32_t* x)
    {
        uint32_t twosA, twosB, foursA, foursB, eightsA;
        csa(twosA, ones, ones, x[0], x[1]);
        csa(twosB, ones, ones, x[2], x[3]);
        csa(foursA, twos, twos, twosA, twosB);
        csa(twosA, ones, ones, x[4], x[5]);
        csa(twosB, ones, ones, x[6], x[7]);
        csa(foursB, twos, twos, twosA, twosB);
        csa(eightsA, fours, fours, foursA, foursB);
        uint32_t c = eightsA, t;
        t = eights & c; eights ^= c; c = t;
#pragma unroll
        for (int i = 0; i < NH; ++i) {
            t = hi[i] & c;
            hi[i] ^= c;
            c = t;
        }
    }
    // add8 for a whole warp (every lane calls it): the carry out of the
    // eights plane is rippled into the higher planes only when some lane has
    // one (sparse inputs rarely carry that far).
    __device__ __forceinline__ void add8_warp(const uint32_t* x)
    {
        uint32_t twosA, twosB, foursA, foursB, eightsA;
        csa(twosA, ones, ones, x[0], x[1]);
        csa(twosB, ones, ones, x[2], x[3]);
        csa(foursA, twos, twos, twosA, twosB);
        csa(twosA, ones, ones, x[4], x[5]);
        csa(twosB, ones, ones, x[6], x[7]);
        csa(foursB, twos, twos, twosA, twosB);
        csa(eightsA, fours, fours, foursA, foursB);
        uint32_t c = eightsA, t;
        t = eights & c; eights ^= c; c = t;
        if (__any_sync(0xffffffffu, c != 0u)) {
#pragma unroll
            for (int i = 0; i < NH; ++i) {
                t = hi[i] & c;
                hi[i] ^= c;
                c = t;
            }
        }
    }
    __device__ __forceinline__ void add1(uint32_t x)
    {
        uint32_t c = x, t;
        t = ones & c; ones ^= c; c = t;
        t = twos & c; twos ^= c; c = t;
        t = fours & c; fours ^= c; c = t;
        t = eights & c; eights ^= c; c = t;
#pragma unroll
        for (int i = 0; i < NH; ++i) {
            t = hi[i] & c;
            hi[i] ^= c;
            c = t;
        }
    }
    __device__ __forceinline__ bool any() const
    {
        uint32_t a = ones | twos | fours | eights;
#pragma unroll
        for (int i = 0; i < NH; ++i) a |= hi[i];
        return a != 0;
    }
    // Highest plane index (0-based, over ones..hi[NH-1]) holding a set bit
    // in any lane of the warp, -1 when all counters are zero.
    __device__ __forceinline__ int top_plane() const
    {
        int t = -1;
        if (ones) t = 0;
        if (twos) t = 1;
        if (fours) t = 2;
        if (eights) t = 3;
#pragma unroll
        for (int i = 0; i < NH; ++i)
            if (hi[i]) t = 4 + i;
        return __reduce_max_sync(0xffffffffu, (unsigned)(t + 1)) - 1;
    }
    // Count of bit b using only planes 0..top.
    __device__ __forceinline__ int count_upto(int b, int top) const
    {
        int c = ((ones >> b) & 1) | (((twos >> b) & 1) << 1) | (((fours >> b) & 1) << 2) | (((eights >> b) & 1) << 3);
#pragma unroll
        for (int i = 0; i < NH; ++i)
            if (4 + i <= top) c |= ((hi[i] >> b) & 1) << (4 + i);
        return c;
    }
    __device__ __forceinline__ int count(int b) const
    {
        int c = ((ones >> b) & 1) | (((twos >> b) & 1) << 1) | (((fours >> b) & 1) << 2) | (((eights >> b) & 1) << 3);
#pragma unroll
        for (int i = 0; i < NH; ++i) c |= ((hi[i] >> b) & 1) << (4 + i);
        return c;
    }
};

// ------------------------------------------------------- kernels
__global__ void k_setup(SetupArgs a, SplitArgs sp, Plan* plan, char* ws);
__global__ void k_prep(Plan* plan);
__global__ void k_sort(Plan* plan);
__global__ void k_peel(Plan* plan);

constexpr int kPeelChunk = 8192;   // front members staged in shared memory at once
constexpr int kPeelStages = 2;     // per-warp ring of 32-row copies (one batch in flight while one is counted)
constexpr int kPeelRingBytes = (kCoopThreads / 32) * kPeelStages * 32 * 128;
// Dynamic shared memory of k_peel for ncb column blocks: the copy ring, the
// member prefix per block and the staged members.
__host__ __device__ constexpr int peel_smem_bytes(int ncb)
{
    return kPeelRingBytes + (ncb + 1 + kPeelChunk) * (int)sizeof(int);
}
__global__ void k_peel_wave(Plan* plan);
__global__ void k_rank_in(Plan* plan);
__global__ void k_assoc_out(Plan* plan);
__global__ void k_given_in(Plan* plan);
cudaError_t launch_front_counts(const uint32_t* D, int64_t ld, int64_t ncols, const int32_t* rows, int64_t n_rows,
                                int32_t* counts, uint8_t* new_front, int sms, cudaStream_t s);
__host__ __device__ constexpr int peel_wave_smem_bytes(int ncb) { return peel_smem_bytes(ncb) + 2 * ncb * (int)sizeof(int); }
__global__ void k_stats(Plan* plan);
__global__ void k_rescan(Plan* plan);
__global__ void k_csr(Plan* plan);
__global__ void k_niche(Plan* plan);
__global__ void k_niche_oneshot(Plan* plan);
__global__ void k_hype(Plan* plan, int phase);
__global__ void k_hype_counts(Plan* plan);
int hype_counts_smem(int m);
__global__ void k_finish(Plan* plan);

// Dominance kernels, one instantiation per objective count (k_dominance.cu).
// The triangle kernel serves items [lo, hi) of the plan through `counter`.
cudaError_t launch_dominance_tri_range(int m, Plan* plan, int sms, cudaStream_t s, long long lo, long long hi,
                                       unsigned long long* counter, int pfirst, int plast);
cudaError_t launch_assoc(Plan* plan, int nprob, const int* m_of, int sms, cudaStream_t s);
cudaError_t launch_colprep(Plan* plan, int sms, cudaStream_t s, int nprob);
// MODE_DOM (one problem, m <= 5): caller-order keys, prefix sets of every
// objective, then the full matrix by prefix sets over `nitems` items.
cudaError_t launch_dominance_caller(int m, Plan* plan, int sms, cudaStream_t s, long long nitems,
                                    unsigned long long* counter);
cudaError_t launch_dominance_full_c(const float* F, int64_t n2, int64_t col_lo, int64_t col_hi, int m, uint32_t* D,
                                    int64_t ld, int32_t* cnt, int sms, cudaStream_t s);

}  // namespace emo
