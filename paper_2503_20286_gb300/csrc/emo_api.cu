// C ABI entry points (include/emo.h): argument checks, workspace layout and
// the launch sequence of each call. All device work is stream ordered; no
// call synchronises except emo_workspace_status.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <cstring>
#include <initializer_list>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "emo_kernels.cuh"
#include "emo_launch.cuh"

using namespace emo;

namespace {

std::atomic<long long> g_spin_budget{0};
constexpr int kPeelDynSmem = peel_smem_bytes((int)(kMaxN2 / kColBlock));
constexpr int kPeelWaveDynSmem = peel_wave_smem_bytes((int)(kMaxN2 / kColBlock));
std::atomic<int> g_timing{0};

// Per-thread stage timing of the last run() (opt-in; events on the launch stream).
constexpr int kMaxStages = 16;
struct StageTimes {
    cudaEvent_t ev[kMaxStages + 1] = {};
    const char* name[kMaxStages] = {};
    int n = 0;
    bool created = false;
    int dev = -1;
};
thread_local StageTimes g_st;

struct StageMarker {
    bool on;
    cudaStream_t s;
    explicit StageMarker(cudaStream_t st) : on(g_timing.load() != 0), s(st)
    {
        if (!on) return;
        int dev = 0;
        cudaGetDevice(&dev);
        if (g_st.created && g_st.dev != dev) {
            for (auto& e : g_st.ev) cudaEventDestroy(e);
            g_st.created = false;
        }
        if (!g_st.created) {
            for (auto& e : g_st.ev) cudaEventCreate(&e);
            g_st.created = true;
            g_st.dev = dev;
        }
        g_st.n = 0;
        cudaEventRecord(g_st.ev[0], s);
    }
    void mark(const char* nm)
    {
        if (!on || g_st.n >= kMaxStages) return;
        g_st.name[g_st.n] = nm;
        cudaEventRecord(g_st.ev[++g_st.n], s);
    }
};

long long spin_budget()
{
    long long b = g_spin_budget.load();
    if (b > 0) return b;
    static long long env = [] {
        const char* e = std::getenv("EMO_SPIN_BUDGET");
        long long v = e ? std::atoll(e) : 0;
        return v > 0 ? v : 4000000000ll;  // ~2 s at 2 GHz
    }();
    return env;
}

struct DevInfo {
    int sms = 0;
    int G = 0;  // CTAs of each cooperative launch
    bool ok = false;
};

DevInfo dev_info()
{
    static std::mutex mu;
    static std::vector<DevInfo> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DevInfo{};
    std::lock_guard<std::mutex> lk(mu);
    if ((int)cache.size() <= dev) cache.resize(dev + 1);
    DevInfo& di = cache[dev];
    if (!di.ok) {
        int sms = 0, coop = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DevInfo{};
        if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
            return DevInfo{};
        if (cudaFuncSetAttribute((const void*)k_peel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPeelDynSmem) !=
                cudaSuccess ||
            cudaFuncSetAttribute((const void*)k_peel_wave, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kPeelWaveDynSmem) != cudaSuccess ||
            cudaFuncSetAttribute((const void*)k_hype_counts, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 hype_counts_smem(4)) != cudaSuccess)
            return DevInfo{};
        int occ = 2;
        // k_peel takes peel_smem_bytes(ncb) of dynamic shared memory, the others none
        const void* kernels[] = {(const void*)k_sort,  (const void*)k_peel,  (const void*)k_peel_wave,
                                 (const void*)k_stats, (const void*)k_csr,   (const void*)k_niche,
                                 (const void*)k_niche_oneshot, (const void*)k_hype, (const void*)k_finish,
                                 (const void*)k_rank_in, (const void*)k_assoc_out, (const void*)k_given_in};
        const int dyn[] = {0, kPeelDynSmem, kPeelWaveDynSmem, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int i = 0; i < (int)(sizeof(dyn) / sizeof(dyn[0])); ++i) {
            int o = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernels[i], kCoopThreads, dyn[i]) != cudaSuccess)
                return DevInfo{};
            occ = std::min(occ, o);
        }
        if (occ < 1) return DevInfo{};
        di.sms = sms;
        di.G = sms * occ;
        di.ok = true;
    }
    return di;
}

constexpr int64_t kPlanBytes = (int64_t)((sizeof(Plan) + 255) / 256 * 256);

bool sizes_ok(int64_t n2, int32_t m) { return n2 >= 1 && n2 <= kMaxN2 && m >= 2 && m <= kMaxM; }

ProbIn make_in(const float* F, const float* R, int64_t n2, int32_t m, int32_t n_r, int64_t n_keep, uint64_t seed,
               uint64_t gen, int32_t* surv, emo_select_info* info, int mode)
{
    ProbIn in;
    std::memset(&in, 0, sizeof(in));
    in.F = F;
    in.R = R;
    in.survivors = surv;
    in.info = info;
    in.n2 = n2;
    in.n_keep = n_keep;
    in.m = m;
    in.n_r = n_r;
    in.seed = seed;
    in.gen = gen;
    in.mode = mode;
    return in;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

cudaError_t coop(const void* fn, int G, size_t smem, cudaStream_t s, Plan* plan)
{
    void* args[] = {&plan};
    return cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kCoopThreads), args, smem, s);
}
cudaError_t coop_phase(const void* fn, int G, size_t smem, cudaStream_t s, Plan* plan, int phase)
{
    void* args[] = {&plan, &phase};
    return cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kCoopThreads), args, smem, s);
}

// Launch shapes, per (compute capability as 10 * major + minor, m,
// floor(log2 n2)); survivors never depend on them. emo_autotune measures
// them; untuned sizes take default_shape().
struct Shape {
    int assoc_bps;   // association kernel: blocks per SM
    int dom_chunk;   // dominance: row blocks per work item (64 .. 1024, a power of two)
    int cap_wide;    // CTAs of the peeling / TensorHypE group of one problem (0 = no cap)
    int cap_narrow;  // CTAs of the other cooperative groups (0 = no cap)
    int peel_wave;   // peeling schedule: 1 wavefront (no grid barrier per front), 0 one grid barrier per front
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, Shape> g_tune;
Shape g_force{0, 0, -1, -1, -1};  // set only while emo_autotune times a candidate (0 / -1 = not forced)
constexpr int kDefaultPeelWave = 0;

int size_bucket(int64_t n2)
{
    int b = 0;
    while ((int64_t(1) << (b + 1)) <= n2) ++b;
    return b;
}

int device_arch(int dev)
{
    int ma = 0, mi = 0;
    cudaDeviceGetAttribute(&ma, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&mi, cudaDevAttrComputeCapabilityMinor, dev);
    return ma * 10 + mi;
}

// Cache file: one line per tuned size, "arch m bucket assoc_bps" optionally
// followed by "dom_chunk cap_wide cap_narrow" and "peel_wave".
void load_tune_cache(const char* path)
{
    FILE* fh = path ? std::fopen(path, "r") : nullptr;
    if (!fh) return;
    char line[256];
    std::lock_guard<std::mutex> lk(g_tune_mu);
    while (std::fgets(line, sizeof(line), fh)) {
        int v[8] = {0, 0, 0, 0, kDomRowChunk, 0, 0, kDefaultPeelWave};
        const int n = std::sscanf(line, "%d %d %d %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6],
                                  &v[7]);
        if ((n != 4 && n != 7 && n != 8) || v[3] < 1 || v[3] > 64 || !dom_chunk_ok(v[4]) || v[5] < 0 || v[6] < 0 ||
            v[7] < 0 || v[7] > 1)
            continue;
        g_tune[std::make_tuple(v[0], v[1], v[2])] = Shape{v[3], v[4], v[5], v[6], v[7]};
    }
    std::fclose(fh);
}

// Without tuning: 8 association blocks per SM, the largest dominance items
// that still give every SM two or more, no group caps.
Shape default_shape(int sms, int64_t n2)
{
    Shape sh{8, kDomRowChunk, 0, 0, kDefaultPeelWave};
    while (sh.dom_chunk > kDomChunkMin && dom_items_of(n2, sh.dom_chunk) < 2ll * sms) sh.dom_chunk >>= 1;
    return sh;
}

Shape shape_for(int dev, int sms, int m, int64_t n2)
{
    static std::once_flag env_once;  // shapes tuned by earlier processes
    std::call_once(env_once, [] { load_tune_cache(std::getenv("EMO_AUTOTUNE_CACHE")); });
    Shape sh = default_shape(sms, n2);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(std::make_tuple(device_arch(dev), m, size_bucket(n2)));
        if (it != g_tune.end()) sh = it->second;
        if (g_force.assoc_bps > 0) sh.assoc_bps = g_force.assoc_bps;
        if (g_force.dom_chunk > 0) sh.dom_chunk = g_force.dom_chunk;
        if (g_force.cap_wide >= 0) sh.cap_wide = g_force.cap_wide;
        if (g_force.cap_narrow >= 0) sh.cap_narrow = g_force.cap_narrow;
        if (g_force.peel_wave >= 0) sh.peel_wave = g_force.peel_wave;
    }
    return sh;
}

emo_status run_niche_stages(std::vector<ProbIn>& ins, const DevInfo& di, Plan* plan, cudaStream_t s,
                            StageMarker& sm, bool finish);

// The selection stages after the peeling (statistics, association, niche
// counts, niching, survivors); with `finish`, also the survivors' stage. A
// population split over GPUs stops after the association of one GPU's points
// (SPLIT_ASSOC) or starts from the gathered association (SPLIT_NICHE).
emo_status run_selection_stages(std::vector<ProbIn>& ins, const DevInfo& di, Plan* plan, int dev, cudaStream_t s,
                                StageMarker& sm, bool finish = true, int split = SPLIT_NONE)
{
    const int nprob = (int)ins.size();
    if (split == SPLIT_NICHE) {
        if (coop((const void*)k_given_in, di.G, 0, s, plan) != cudaSuccess) return EMO_ERR_CUDA;
        sm.mark("given");
        return run_niche_stages(ins, di, plan, s, sm, finish);
    }
    if (coop((const void*)k_stats, di.G, 0, s, plan) != cudaSuccess) return EMO_ERR_CUDA;
    sm.mark("stats");
    std::vector<int> m_of(nprob);
    for (int p = 0; p < nprob; ++p) m_of[p] = ins[p].m;
    int big = 0;
    for (int p = 1; p < nprob; ++p)
        if (ins[p].n2 > ins[big].n2) big = p;
    const int bps = shape_for(dev, di.sms, ins[big].m, ins[big].n2).assoc_bps;
    if (launch_assoc(plan, nprob, m_of.data(), di.sms, bps, s) != cudaSuccess) return EMO_ERR_CUDA;
    sm.mark("assoc");
    k_rescan<<<di.sms * 2, 256, 0, s>>>(plan);
    if (cudaGetLastError() != cudaSuccess) return EMO_ERR_CUDA;
    sm.mark("rescan");
    if (split == SPLIT_ASSOC) {
        if (coop((const void*)k_assoc_out, di.G, 0, s, plan) != cudaSuccess) return EMO_ERR_CUDA;
        sm.mark("assoc_out");
        if (finish) {  // status and info
            if (coop((const void*)k_finish, di.G, 0, s, plan) != cudaSuccess) return EMO_ERR_CUDA;
            sm.mark("finish");
        }
        return EMO_OK;
    }
    return run_niche_stages(ins, di, plan, s, sm, finish);
}

// Niche counts and candidate lists, niching, survivors.
emo_status run_niche_stages(std::vector<ProbIn>& ins, const DevInfo& di, Plan* plan, cudaStream_t s,
                            StageMarker& sm, bool finish)
{
    if (coop((const void*)k_csr, di.G, 0, s, plan) != cudaSuccess) return EMO_ERR_CUDA;
    sm.mark("csr");
    bool any_exact = false, any_oneshot = false;
    for (const ProbIn& in : ins) {
        any_exact |= in.mode == MODE_SELECT && in.niche == EMO_NICHE_EXACT;
        any_oneshot |= in.mode == MODE_SELECT && in.niche == EMO_NICHE_ONESHOT;
    }
    if (any_exact && coop((const void*)k_niche, di.G, 0, s, plan) != cudaSuccess) return EMO_ERR_CUDA;
    if (any_oneshot && coop((const void*)k_niche_oneshot, di.G, 0, s, plan) != cudaSuccess) return EMO_ERR_CUDA;
    sm.mark("niche");
    if (finish) {
        if (coop((const void*)k_finish, di.G, 0, s, plan) != cudaSuccess) return EMO_ERR_CUDA;
        sm.mark("finish");
    }
    return EMO_OK;
}

// Launch the whole pipeline for problems already laid out in `ins` (ordered
// by objective count).
emo_status run(std::vector<ProbIn>& ins, void* ws, size_t ws_bytes, cudaStream_t s, const SplitArgs* split = nullptr)
{
    SplitArgs sp;
    std::memset(&sp, 0, sizeof(sp));
    if (split) sp = *split;
    if (sp.kind != SPLIT_NONE && (ins.size() != 1 || !ins[0].ranked)) return EMO_ERR_INVALID_ARG;
    DevInfo di = dev_info();
    if (!di.ok) return EMO_ERR_CUDA;
    const int nprob = (int)ins.size();
    if (nprob < 1 || nprob > kMaxBatch || nprob > di.G) return EMO_ERR_INVALID_ARG;
    if (!ws || !aligned(ws, 256)) return EMO_ERR_INVALID_ARG;
    int64_t off = kPlanBytes;
    int max_ncb = 1;
    bool any_select = false, any_hype = false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EMO_ERR_CUDA;
    for (auto& in : ins) {
        const Shape sh = shape_for(dev, di.sms, in.m, in.n2);
        in.dom_chunk = sh.dom_chunk;
        in.cap_wide = sh.cap_wide;
        in.cap_narrow = sh.cap_narrow;
        in.ws_off = (uint64_t)off;
        off += layout_problem(in, di.G, nullptr, nullptr);
        max_ncb = std::max<int>(max_ncb, (int)cdiv(in.n2, kColBlock));
        any_select |= in.mode == MODE_SELECT;
        any_hype |= in.mode == MODE_HYPE;
    }
    if ((int64_t)ws_bytes < off) return EMO_ERR_WORKSPACE;

    static thread_local SetupArgs args;
    std::memset(&args, 0, sizeof(args));
    args.nprob = nprob;
    args.G = di.G;
    args.spin_budget = spin_budget();
    for (int p = 0; p < nprob; ++p) args.in[p] = ins[p];
    Plan* plan = (Plan*)ws;
    char* base = (char*)ws;

    StageMarker sm(s);
    k_setup<<<1, 128, 0, s>>>(args, sp, plan, base);
    if (cudaGetLastError() != cudaSuccess) return EMO_ERR_CUDA;
    k_prep<<<dim3((unsigned)std::max(1, di.sms * 2 / nprob), nprob), 256, 0, s>>>(plan);
    if (cudaGetLastError() != cudaSuccess) return EMO_ERR_CUDA;
    sm.mark("prep");
    // (from given ranks only the references are ordered; the niching from a
    // given association has none)
    if (sp.kind != SPLIT_NICHE && coop((const void*)k_sort, di.G, 0, s, plan) != cudaSuccess) return EMO_ERR_CUDA;
    sm.mark("sort");
    if (nprob == 1 && ins[0].mode == MODE_DOM) {  // caller-order dominance matrix only
        const ProbIn& in = ins[0];
        const long long nitems = cdiv(in.n2, kColBlock) * cdiv(cdiv(in.n2, 32), in.dom_chunk);
        if (launch_dominance_caller(in.m, plan, di.sms, s, nitems, &plan->dom_ctr[0]) != cudaSuccess)
            return EMO_ERR_CUDA;
        sm.mark("dominance");
        // status word of the workspace and the sticky device status
        if (coop((const void*)k_finish, di.G, 0, s, plan) != cudaSuccess) return EMO_ERR_CUDA;
        sm.mark("finish");
        return EMO_OK;
    }
    if (nprob == 1 && ins[0].ranked) {  // the ranks are given: no dominance matrix, no peeling
        if (coop((const void*)k_rank_in, di.G, 0, s, plan) != cudaSuccess) return EMO_ERR_CUDA;
        sm.mark("rank_in");
        return run_selection_stages(ins, di, plan, dev, s, sm, true, sp.kind);
    }
    if (launch_colprep(plan, di.sms, s, nprob) != cudaSuccess) return EMO_ERR_CUDA;
    sm.mark("colprep");
    // dominance: one launch per objective count present
    long long item = 0;
    for (int p = 0; p < nprob;) {
        int q = p;
        long long hi = item;
        while (q < nprob && ins[q].m == ins[p].m) {
            hi += dom_items_of(ins[q].n2, ins[q].dom_chunk);
            ++q;
        }
        if (launch_dominance_tri_range(ins[p].m, plan, di.sms, s, item, hi, &plan->dom_ctr[ins[p].m], p, q) !=
            cudaSuccess)
            return EMO_ERR_CUDA;
        item = hi;
        p = q;
    }
    sm.mark("dominance");
    {
        int big = 0;
        for (int p = 1; p < nprob; ++p)
            if (ins[p].n2 > ins[big].n2) big = p;
        const bool wave = shape_for(dev, di.sms, ins[big].m, ins[big].n2).peel_wave != 0;
        const size_t smem = (size_t)(wave ? peel_wave_smem_bytes(max_ncb) : peel_smem_bytes(max_ncb));
        if (coop(wave ? (const void*)k_peel_wave : (const void*)k_peel, di.G, smem, s, plan) != cudaSuccess)
            return EMO_ERR_CUDA;
    }
    sm.mark("peel");
    if (any_select) {
        const emo_status st = run_selection_stages(ins, di, plan, dev, s, sm, false);
        if (st != EMO_OK) return st;
    }
    if (any_hype) {
        int hm = 2;
        for (const ProbIn& in : ins)
            if (in.mode == MODE_HYPE) hm = std::max(hm, (int)in.m);
        if (coop_phase((const void*)k_hype, di.G, 0, s, plan, 0) != cudaSuccess) return EMO_ERR_CUDA;
        sm.mark("hype_samples");
        k_hype_counts<<<di.sms, kCoopThreads, hype_counts_smem(hm), s>>>(plan);
        if (cudaGetLastError() != cudaSuccess) return EMO_ERR_CUDA;
        sm.mark("hype_counts");
        if (coop_phase((const void*)k_hype, di.G, 0, s, plan, 1) != cudaSuccess) return EMO_ERR_CUDA;
        sm.mark("hype");
    }
    if (coop((const void*)k_finish, di.G, 0, s, plan) != cudaSuccess) return EMO_ERR_CUDA;
    sm.mark("finish");
    return EMO_OK;
}

int64_t problem_bytes(const ProbIn& in)
{
    DevInfo di = dev_info();
    if (!di.ok) return -1;
    return layout_problem(in, di.G, nullptr, nullptr);
}

emo_status check_select_args(const float* F, int64_t n2, int32_t m, const float* R, int32_t n_r, int64_t n_keep,
                             int32_t* survivors)
{
    if (!F || !R || !survivors) return EMO_ERR_INVALID_ARG;
    if (!sizes_ok(n2, m) || n_r < 1 || n_keep < 1 || n_keep > n2) return EMO_ERR_INVALID_ARG;
    if (!aligned(F, 4) || !aligned(R, 4) || !aligned(survivors, 4)) return EMO_ERR_INVALID_ARG;
    return EMO_OK;
}

}  // namespace

extern "C" {

// Workspace of one generation: the merged decision vectors and objectives
// (2N rows), the survivor indices and the selection workspace. Returns the
// total bytes (0 when the sizes are out of range); fills `at` when given.
struct GenLayout {
    int64_t x2, f2, surv, sel, sel_bytes;
};
static size_t generation_layout(int64_t n, int32_t m, int32_t n_r, int64_t d, GenLayout* at)
{
    auto up = [](int64_t b) { return (b + 255) / 256 * 256; };
    if (n < 1 || !sizes_ok(2 * n, m) || n_r < 1 || d < m || d > (1 << 20)) return 0;
    const size_t sel = emo_workspace_size(EMO_OP_NSGA3_SELECT, 2 * n, m, n_r);
    if (sel == 0) return 0;
    GenLayout L;
    L.x2 = 0;
    L.f2 = up(8 * n * d);
    L.surv = up(L.f2 + 8 * n * m);
    L.sel = up(L.surv + 4 * n);
    L.sel_bytes = (int64_t)sel;
    if (at) *at = L;
    return (size_t)(L.sel + L.sel_bytes);
}

size_t emo_workspace_size(int op, int64_t n2, int32_t m, int32_t n_r)
{
    if (!sizes_ok(n2, m)) return 0;
    if (op == EMO_OP_DOMINANCE) return 0;
    if (op == EMO_OP_DOMINANCE_WS) {
        if (m > 5) return 0;  // the direct kernel needs no workspace
        ProbIn in = make_in(nullptr, nullptr, n2, m, 1, n2, 0, 0, nullptr, nullptr, MODE_DOM);
        const int64_t b = problem_bytes(in);
        return b < 0 ? 0 : (size_t)(kPlanBytes + b);
    }
    if (op == EMO_OP_SELECT_RANKED) {
        if (n_r < 1) return 0;
        ProbIn in = make_in(nullptr, nullptr, n2, m, n_r, n2, 0, 0, nullptr, nullptr, MODE_SELECT);
        in.ranked = 1;
        const int64_t b = problem_bytes(in);
        return b < 0 ? 0 : (size_t)(kPlanBytes + b);
    }
    if (op == EMO_OP_MOEAD_SELECT) return n_r >= 1 && n_r <= n2 ? (size_t)moead_layout(n2, m, n_r, nullptr, nullptr) : 0;
    if (op == EMO_OP_IGD) return (size_t)(n2 * 8);
    int mode = op == EMO_OP_ND_RANK ? MODE_RANK
               : op == EMO_OP_NSGA3_SELECT ? MODE_SELECT
               : op == EMO_OP_HYPE_SELECT ? MODE_HYPE
                                          : 0;
    if (!mode) return 0;
    if ((mode == MODE_SELECT || mode == MODE_HYPE) && n_r < 1) return 0;
    ProbIn in = make_in(nullptr, nullptr, n2, m, mode == MODE_RANK ? 1 : n_r, n2, 0, 0, nullptr, nullptr, mode);
    int64_t b = problem_bytes(in);
    return b < 0 ? 0 : (size_t)(kPlanBytes + b);
}

emo_status emo_dominance_cols(const float* F, int64_t n2, int32_t m, int64_t col_lo, int64_t col_hi, uint32_t* D,
                              int64_t ld_words, int32_t* dom_count, emo_stream_t stream)
{
    if (!F || !D || !sizes_ok(n2, m) || col_lo < 0 || col_hi > n2 || col_lo >= col_hi || col_lo % kColBlock != 0 ||
        ld_words < cdiv(col_hi - col_lo, 32))
        return EMO_ERR_INVALID_ARG;
    if (!aligned(F, 4) || !aligned(D, 4) || (dom_count && !aligned(dom_count, 4))) return EMO_ERR_INVALID_ARG;
    DevInfo di = dev_info();
    if (!di.ok) return EMO_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t ncols = col_hi - col_lo;
    if (dom_count && cudaMemsetAsync(dom_count, 0, (size_t)ncols * 4, s) != cudaSuccess) return EMO_ERR_CUDA;
    const int64_t wfull = cdiv(ncols, kColBlock) * 32;  // words the kernel writes per row
    if (ld_words > wfull &&
        cudaMemset2DAsync(D + wfull, (size_t)ld_words * 4, 0, (size_t)(ld_words - wfull) * 4, (size_t)n2, s) !=
            cudaSuccess)
        return EMO_ERR_CUDA;
    if (launch_dominance_full_c(F, n2, col_lo, col_hi, m, D, ld_words, dom_count, di.sms, s) != cudaSuccess)
        return EMO_ERR_CUDA;
    return EMO_OK;
}

emo_status emo_dominance_ws(const float* F, int64_t n2, int32_t m, uint32_t* D, int64_t ld_words, int32_t* dom_count,
                            void* ws, size_t ws_bytes, emo_stream_t stream)
{
    if (!F || !D || !sizes_ok(n2, m) || ld_words < cdiv(n2, 32)) return EMO_ERR_INVALID_ARG;
    if (m > 5) return emo_dominance_cols(F, n2, m, 0, n2, D, ld_words, dom_count, stream);
    if (!aligned(F, 4) || !aligned(D, 4) || (dom_count && !aligned(dom_count, 4))) return EMO_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (dom_count && cudaMemsetAsync(dom_count, 0, (size_t)n2 * 4, s) != cudaSuccess) return EMO_ERR_CUDA;
    const int64_t wfull = cdiv(n2, kColBlock) * 32;  // words the kernel writes per row
    if (ld_words > wfull &&
        cudaMemset2DAsync(D + wfull, (size_t)ld_words * 4, 0, (size_t)(ld_words - wfull) * 4, (size_t)n2, s) !=
            cudaSuccess)
        return EMO_ERR_CUDA;
    std::vector<ProbIn> ins(1, make_in(F, nullptr, n2, m, 1, n2, 0, 0, nullptr, nullptr, MODE_DOM));
    ins[0].dom_out = D;
    ins[0].dom_count = dom_count;
    ins[0].dom_ld = ld_words;
    return run(ins, ws, ws_bytes, s);
}

emo_status emo_dominance(const float* F, int64_t n2, int32_t m, uint32_t* D, int64_t ld_words, int32_t* dom_count,
                         emo_stream_t stream)
{
    if (!F || !D || !sizes_ok(n2, m) || ld_words < cdiv(n2, 32)) return EMO_ERR_INVALID_ARG;
    return emo_dominance_cols(F, n2, m, 0, n2, D, ld_words, dom_count, stream);
}

emo_status emo_nd_rank(const float* F, int64_t n2, int32_t m, int64_t n_keep, int32_t* rank, int32_t* last_rank,
                       void* ws, size_t ws_bytes, emo_stream_t stream)
{
    if (!F || !rank || !sizes_ok(n2, m) || n_keep < 0 || n_keep > n2) return EMO_ERR_INVALID_ARG;
    if (!aligned(F, 4) || !aligned(rank, 4) || (last_rank && !aligned(last_rank, 4))) return EMO_ERR_INVALID_ARG;
    std::vector<ProbIn> ins(1, make_in(F, nullptr, n2, m, 1, n_keep, 0, 0, nullptr, nullptr, MODE_RANK));
    ins[0].rank_out = rank;
    ins[0].last_rank_out = last_rank;
    return run(ins, ws, ws_bytes, (cudaStream_t)stream);
}

emo_status emo_hype_select(const float* F, int64_t n2, int32_t m, const float* v_ref, const float* U,
                           int32_t n_samples, int64_t n_keep, int32_t* survivors, emo_select_info* info,
                           double* hv, void* ws, size_t ws_bytes, emo_stream_t stream)
{
    emo_status st = check_select_args(F, n2, m, v_ref, n_samples, n_keep, survivors);
    if (st != EMO_OK) return st;
    if (!U || !aligned(U, 4) || (hv && !aligned(hv, 8))) return EMO_ERR_INVALID_ARG;
    std::vector<ProbIn> ins(1, make_in(F, v_ref, n2, m, n_samples, n_keep, 0, 0, survivors, info, MODE_HYPE));
    ins[0].U = U;
    ins[0].hv_out = hv;
    return run(ins, ws, ws_bytes, (cudaStream_t)stream);
}

emo_status emo_moead_select(const float* X, const float* F1, const float* O, const float* F2, int64_t n, int64_t d,
                            int32_t m, float* z, const float* W, const int32_t* I_nb, int32_t T, double theta,
                            float* X_next, float* F_next, int32_t* winner, int32_t* status_out, void* ws,
                            size_t ws_bytes, emo_stream_t stream)
{
    if (!X || !F1 || !O || !F2 || !z || !W || !I_nb || !X_next || !F_next || !ws) return EMO_ERR_INVALID_ARG;
    if (!sizes_ok(n, m) || d < 1 || T < 1 || T > n || T > 4096 || !std::isfinite(theta) || theta < 0.0)
        return EMO_ERR_INVALID_ARG;
    for (const void* p : {(const void*)X, (const void*)F1, (const void*)O, (const void*)F2, (const void*)z,
                          (const void*)W, (const void*)I_nb, (const void*)X_next, (const void*)F_next,
                          (const void*)winner, (const void*)status_out})
        if (p && !aligned(p, 4)) return EMO_ERR_INVALID_ARG;
    if (!aligned(ws, 256)) return EMO_ERR_INVALID_ARG;
    MoeadArgs a;
    std::memset(&a, 0, sizeof(a));
    if ((int64_t)ws_bytes < moead_layout(n, m, T, (char*)ws, &a)) return EMO_ERR_WORKSPACE;
    DevInfo di = dev_info();
    if (!di.ok) return EMO_ERR_CUDA;
    a.X = X;
    a.F1 = F1;
    a.O = O;
    a.F2 = F2;
    a.W = W;
    a.I_nb = I_nb;
    a.z = z;
    a.X_next = X_next;
    a.F_next = F_next;
    a.winner = winner;
    a.status_out = status_out;
    a.n = n;
    a.d = d;
    a.m = m;
    a.T = T;
    a.theta = theta;
    return launch_moead_select(a, di.sms, (cudaStream_t)stream) == cudaSuccess ? EMO_OK : EMO_ERR_CUDA;
}

size_t emo_generation_workspace_size(int64_t n, int64_t d, int32_t m, int32_t n_r)
{
    return generation_layout(n, m, n_r, d, nullptr);
}

emo_status emo_variation(const float* X, int64_t n, int64_t d, const float* lo, const float* hi, int64_t n_off,
                         uint64_t seed, uint64_t generation, double eta_c, double eta_m, double p_c, double p_m,
                         float* X_off, int32_t* parents, emo_stream_t stream)
{
    if (!X || !X_off || (!lo) != (!hi) || n < 1 || n > INT32_MAX || d < 1 || d > 0x00FFFFFF || n_off < 1 ||
        n_off > INT32_MAX || !(eta_c >= 0.0) || !(eta_m >= 0.0) || !std::isfinite(eta_c) || !std::isfinite(eta_m) ||
        std::isnan(p_c) || std::isnan(p_m))
        return EMO_ERR_INVALID_ARG;
    for (const void* p : {(const void*)X, (const void*)lo, (const void*)hi, (const void*)X_off, (const void*)parents})
        if (p && !aligned(p, 4)) return EMO_ERR_INVALID_ARG;
    DevInfo di = dev_info();
    if (!di.ok) return EMO_ERR_CUDA;
    VariationArgs a{X, lo, hi, X_off, parents, n, d, n_off, seed, generation, eta_c, eta_m, p_c, p_m};
    return launch_variation(a, di.sms, (cudaStream_t)stream) == cudaSuccess ? EMO_OK : EMO_ERR_CUDA;
}

emo_status emo_standin_objectives(const float* X, int64_t n, int64_t d, int32_t m, int32_t shape, float* F,
                                  emo_stream_t stream)
{
    if (!X || !F || n < 1 || m < 2 || m > kMaxM || d < m || (shape != EMO_SHAPE_LINEAR && shape != EMO_SHAPE_SPHERE))
        return EMO_ERR_INVALID_ARG;
    if (!aligned(X, 4) || !aligned(F, 4)) return EMO_ERR_INVALID_ARG;
    DevInfo di = dev_info();
    if (!di.ok) return EMO_ERR_CUDA;
    return launch_standin(X, n, d, m, shape, F, di.sms, (cudaStream_t)stream) == cudaSuccess ? EMO_OK : EMO_ERR_CUDA;
}

emo_status emo_igd(const float* F, int64_t n, int32_t m, const float* Ref, int64_t n_ref, double* igd_out, void* ws,
                   size_t ws_bytes, emo_stream_t stream)
{
    if (!F || !Ref || !igd_out || !ws || n < 1 || n_ref < 1 || m < 1 || m > kMaxM) return EMO_ERR_INVALID_ARG;
    if (!aligned(F, 4) || !aligned(Ref, 4) || !aligned(igd_out, 8) || !aligned(ws, 8)) return EMO_ERR_INVALID_ARG;
    if ((int64_t)ws_bytes < n_ref * 8) return EMO_ERR_WORKSPACE;
    DevInfo di = dev_info();
    if (!di.ok) return EMO_ERR_CUDA;
    return launch_igd(F, n, m, Ref, n_ref, (double*)ws, igd_out, di.sms, (cudaStream_t)stream) == cudaSuccess
               ? EMO_OK
               : EMO_ERR_CUDA;
}

emo_status emo_nsga3_generation(float* X, float* F, int64_t n, int64_t d, int32_t m, const float* R, int32_t n_r,
                                int32_t shape, uint64_t seed, uint64_t generation, double eta_c, double eta_m,
                                double p_c, double p_m, int32_t niche_mode, emo_select_info* info, void* ws,
                                size_t ws_bytes, emo_stream_t stream)
{
    if (!X || !F || !R || !ws || d < m || d > (1 << 20) || !aligned(ws, 256)) return EMO_ERR_INVALID_ARG;
    GenLayout L;
    const size_t need = generation_layout(n, m, n_r, d, &L);
    if (need == 0) return EMO_ERR_INVALID_ARG;
    if (ws_bytes < need) return EMO_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    char* base = (char*)ws;
    float* X2 = (float*)(base + L.x2);
    float* F2 = (float*)(base + L.f2);
    int32_t* surv = (int32_t*)(base + L.surv);
    DevInfo di = dev_info();
    if (!di.ok) return EMO_ERR_CUDA;
    if (cudaMemcpyAsync(X2, X, (size_t)(n * d) * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(F2, F, (size_t)(n * m) * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return EMO_ERR_CUDA;
    emo_status st = emo_variation(X, n, d, nullptr, nullptr, n, seed, generation, eta_c, eta_m, p_c, p_m, X2 + n * d,
                                  nullptr, stream);
    if (st != EMO_OK) return st;
    st = emo_standin_objectives(X2 + n * d, n, d, m, shape, F2 + n * m, stream);
    if (st != EMO_OK) return st;
    st = emo_nsga3_select_ex(F2, 2 * n, m, R, n_r, n, seed, generation, niche_mode, surv, info, nullptr,
                             base + L.sel, (size_t)L.sel_bytes, stream);
    if (st != EMO_OK) return st;
    if (launch_gather_rows(X2, surv, n, d, X, di.sms, s) != cudaSuccess ||
        launch_gather_rows(F2, surv, n, m, F, di.sms, s) != cudaSuccess)
        return EMO_ERR_CUDA;
    return EMO_OK;
}

emo_status emo_nsga3_select_ex(const float* F, int64_t n2, int32_t m, const float* R, int32_t n_r,
                               int64_t n_keep, uint64_t seed, uint64_t generation, int32_t niche_mode,
                               int32_t* survivors, emo_select_info* info, const emo_select_debug* dbg, void* ws,
                               size_t ws_bytes, emo_stream_t stream)
{
    emo_status st = check_select_args(F, n2, m, R, n_r, n_keep, survivors);
    if (st != EMO_OK) return st;
    if (niche_mode != EMO_NICHE_EXACT && niche_mode != EMO_NICHE_ONESHOT) return EMO_ERR_INVALID_ARG;
    std::vector<ProbIn> ins(1, make_in(F, R, n2, m, n_r, n_keep, seed, generation, survivors, info, MODE_SELECT));
    ins[0].niche = niche_mode;
    if (dbg) ins[0].dbg = *dbg;
    return run(ins, ws, ws_bytes, (cudaStream_t)stream);
}

emo_status emo_nsga3_select_ranked(const float* F, int64_t n2, int32_t m, const float* R, int32_t n_r,
                                   int64_t n_keep, uint64_t seed, uint64_t generation, const int32_t* rank,
                                   int32_t* survivors, emo_select_info* info, void* ws, size_t ws_bytes,
                                   emo_stream_t stream)
{
    emo_status st = check_select_args(F, n2, m, R, n_r, n_keep, survivors);
    if (st != EMO_OK) return st;
    if (!rank || !aligned(rank, 4)) return EMO_ERR_INVALID_ARG;
    std::vector<ProbIn> ins(1, make_in(F, R, n2, m, n_r, n_keep, seed, generation, survivors, info, MODE_SELECT));
    ins[0].ranked = 1;
    ins[0].rank_in = rank;
    return run(ins, ws, ws_bytes, (cudaStream_t)stream);
}

emo_status emo_nsga3_associate_range(const float* F, int64_t n2, int32_t m, const float* R, int32_t n_r,
                                     int64_t n_keep, const int32_t* rank, int64_t col_lo, int64_t col_hi, int32_t* pi,
                                     double* dist, int32_t* rho, emo_select_info* info, void* ws, size_t ws_bytes,
                                     emo_stream_t stream)
{
    if (!F || !R || !rank || !rho) return EMO_ERR_INVALID_ARG;
    if (!sizes_ok(n2, m) || n_r < 1 || n_keep < 1 || n_keep > n2) return EMO_ERR_INVALID_ARG;
    if (col_lo < 0 || col_lo > col_hi || col_hi > n2) return EMO_ERR_INVALID_ARG;
    if (col_hi > col_lo && (!pi || !dist)) return EMO_ERR_INVALID_ARG;
    if (!aligned(F, 4) || !aligned(R, 4) || !aligned(rank, 4) || !aligned(rho, 4) || !aligned(pi, 4) ||
        !aligned(dist, 8))
        return EMO_ERR_INVALID_ARG;
    std::vector<ProbIn> ins(1, make_in(F, R, n2, m, n_r, n_keep, 0, 0, nullptr, info, MODE_SELECT));
    ins[0].ranked = 1;
    ins[0].rank_in = rank;
    SplitArgs sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.kind = SPLIT_ASSOC;
    sp.col_lo = col_lo;
    sp.col_hi = col_hi;
    sp.pi_out = pi;
    sp.d_out = dist;
    sp.rho = rho;
    return run(ins, ws, ws_bytes, (cudaStream_t)stream, &sp);
}

emo_status emo_nsga3_niche_given(int64_t n2, int32_t n_r, int64_t n_keep, uint64_t seed, uint64_t generation,
                                 int32_t niche_mode, const int32_t* rank, const int32_t* rho, const int32_t* last,
                                 const int32_t* last_pi, const double* last_dist, int64_t n_last,
                                 int32_t* survivors, emo_select_info* info, void* ws, size_t ws_bytes,
                                 emo_stream_t stream)
{
    if (!rank || !rho || !last || !last_pi || !last_dist || !survivors) return EMO_ERR_INVALID_ARG;
    if (!sizes_ok(n2, 2) || n_r < 1 || n_keep < 1 || n_keep > n2 || n_last < 1 || n_last > n2)
        return EMO_ERR_INVALID_ARG;
    if (niche_mode != EMO_NICHE_EXACT && niche_mode != EMO_NICHE_ONESHOT) return EMO_ERR_INVALID_ARG;
    if (!aligned(rank, 4) || !aligned(rho, 4) || !aligned(last, 4) || !aligned(last_pi, 4) ||
        !aligned(last_dist, 8) || !aligned(survivors, 4))
        return EMO_ERR_INVALID_ARG;
    // no objectives: the layout of two (the smallest)
    std::vector<ProbIn> ins(1, make_in(nullptr, nullptr, n2, 2, n_r, n_keep, seed, generation, survivors, info,
                                       MODE_SELECT));
    ins[0].ranked = 1;
    ins[0].rank_in = rank;
    ins[0].niche = niche_mode;
    SplitArgs sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.kind = SPLIT_NICHE;
    sp.rho = const_cast<int32_t*>(rho);  // read only in this kind
    sp.last = last;
    sp.last_pi = last_pi;
    sp.last_d = last_dist;
    sp.n_last = n_last;
    return run(ins, ws, ws_bytes, (cudaStream_t)stream, &sp);
}

emo_status emo_front_counts(const uint32_t* D, int64_t ld_words, int64_t ncols, const int32_t* rows, int64_t n_rows,
                            int32_t* counts, uint8_t* next_front, emo_stream_t stream)
{
    if (!D || !counts || !next_front || ncols < 1 || ncols > kMaxN2 || ld_words < cdiv(ncols, 32) || n_rows < 0 ||
        n_rows > kMaxN2 || (n_rows > 0 && !rows))
        return EMO_ERR_INVALID_ARG;
    if (!aligned(D, 4) || !aligned(counts, 4) || (rows && !aligned(rows, 4))) return EMO_ERR_INVALID_ARG;
    DevInfo di = dev_info();
    if (!di.ok) return EMO_ERR_CUDA;
    return launch_front_counts(D, ld_words, ncols, rows, n_rows, counts, next_front, di.sms, (cudaStream_t)stream) ==
                   cudaSuccess
               ? EMO_OK
               : EMO_ERR_CUDA;
}

emo_status emo_nsga3_select_debug(const float* F, int64_t n2, int32_t m, const float* R, int32_t n_r,
                                  int64_t n_keep, uint64_t seed, uint64_t generation, int32_t* survivors,
                                  emo_select_info* info, const emo_select_debug* dbg, void* ws, size_t ws_bytes,
                                  emo_stream_t stream)
{
    return emo_nsga3_select_ex(F, n2, m, R, n_r, n_keep, seed, generation, EMO_NICHE_EXACT, survivors, info, dbg,
                               ws, ws_bytes, stream);
}

emo_status emo_nsga3_select(const float* F, int64_t n2, int32_t m, const float* R, int32_t n_r, int64_t n_keep,
                            uint64_t seed, uint64_t generation, int32_t* survivors, emo_select_info* info, void* ws,
                            size_t ws_bytes, emo_stream_t stream)
{
    return emo_nsga3_select_debug(F, n2, m, R, n_r, n_keep, seed, generation, survivors, info, nullptr, ws,
                                  ws_bytes, stream);
}

static bool batch_order(const emo_problem* descs, int32_t batch, std::vector<ProbIn>& ins)
{
    if (!descs || batch < 1 || batch > kMaxBatch) return false;
    ins.clear();
    for (int b = 0; b < batch; ++b) {
        const emo_problem& p = descs[b];
        if (check_select_args(p.F, p.n2, p.m, p.R, p.n_r, p.n_keep, p.survivors) != EMO_OK) return false;
        if (p.niche_mode != EMO_NICHE_EXACT && p.niche_mode != EMO_NICHE_ONESHOT) return false;
        ins.push_back(make_in(p.F, p.R, p.n2, p.m, p.n_r, p.n_keep, p.seed, p.generation, p.survivors, p.info,
                              MODE_SELECT));
        ins.back().niche = p.niche_mode;
    }
    std::stable_sort(ins.begin(), ins.end(), [](const ProbIn& a, const ProbIn& b) {
        return a.m != b.m ? a.m < b.m : a.n2 > b.n2;
    });
    return true;
}

size_t emo_batch_workspace_size(const emo_problem* descs, int32_t batch)
{
    std::vector<ProbIn> ins;
    if (!batch_order(descs, batch, ins)) return 0;
    int64_t total = kPlanBytes;
    for (auto& in : ins) {
        int64_t b = problem_bytes(in);
        if (b < 0) return 0;
        total += b;
    }
    return (size_t)total;
}

emo_status emo_nsga3_select_batch(const emo_problem* descs, int32_t batch, void* ws, size_t ws_bytes,
                                  emo_stream_t stream)
{
    std::vector<ProbIn> ins;
    if (!batch_order(descs, batch, ins)) return EMO_ERR_INVALID_ARG;
    return run(ins, ws, ws_bytes, (cudaStream_t)stream);
}

emo_status emo_workspace_status(const void* ws, emo_stream_t stream, int32_t* status_out)
{
    if (!ws || !status_out) return EMO_ERR_INVALID_ARG;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return EMO_ERR_CUDA;
    int32_t st = 0;
    if (cudaMemcpy(&st, &((const Plan*)ws)->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess)
        return EMO_ERR_CUDA;
    *status_out = st;
    return EMO_OK;
}

void emo_set_spin_budget(int64_t cycles) { g_spin_budget.store(cycles > 0 ? cycles : 0); }

emo_status emo_get_last_device_status(emo_stream_t stream, int32_t* status_out)
{
    if (!status_out) return EMO_ERR_INVALID_ARG;
    return sticky_status((cudaStream_t)stream, status_out, true) == cudaSuccess ? EMO_OK : EMO_ERR_CUDA;
}

emo_status emo_autotune(int32_t m, int64_t n2, const char* cache_path)
{
    if (!sizes_ok(n2, m) || n2 < 64) return EMO_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EMO_ERR_CUDA;
    const int arch = device_arch(dev);
    const auto key = std::make_tuple(arch, (int)m, size_bucket(n2));
    if (cache_path) {
        load_tune_cache(cache_path);
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (g_tune.count(key)) return EMO_OK;
    }
    // a synthetic population: a sphere-shaped front with a spread of
    // distances, and n2 / 2 directions drawn on the simplex (fixed seed)
    const int64_t n_r = std::max<int64_t>(1, std::min<int64_t>(n2 / 2, 1 << 20));
    std::vector<float> F((size_t)(n2 * m)), R((size_t)(n_r * m));
    uint64_t x = 0x9E3779B97F4A7C15ull;
    auto uni = [&]() {  // splitmix64 -> (0, 1)
        x += 0x9E3779B97F4A7C15ull;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    for (int64_t i = 0; i < n2; ++i) {
        double nrm = 0.0, v[kMaxM];
        for (int k = 0; k < m; ++k) { v[k] = -std::log(uni()); nrm += v[k] * v[k]; }
        const double scale = (1.0 + 0.5 * uni()) / std::sqrt(nrm);
        for (int k = 0; k < m; ++k) F[(size_t)(i * m + k)] = (float)(v[k] * scale);
    }
    for (int64_t j = 0; j < n_r; ++j) {
        double sum = 0.0, v[kMaxM];
        for (int k = 0; k < m; ++k) { v[k] = -std::log(uni()); sum += v[k]; }
        for (int k = 0; k < m; ++k) R[(size_t)(j * m + k)] = (float)(v[k] / sum);
    }
    const size_t wsb = emo_workspace_size(EMO_OP_NSGA3_SELECT, n2, m, (int32_t)n_r);
    if (wsb == 0) return EMO_ERR_INVALID_ARG;
    DevInfo di = dev_info();
    if (!di.ok) return EMO_ERR_CUDA;
    void *dF = nullptr, *dR = nullptr, *dS = nullptr, *dW = nullptr;
    emo_status st = EMO_OK;
    Shape best = default_shape(di.sms, n2);
    if (cudaMalloc(&dF, F.size() * 4) != cudaSuccess || cudaMalloc(&dR, R.size() * 4) != cudaSuccess ||
        cudaMalloc(&dS, (size_t)(n2 / 2 + 1) * 4) != cudaSuccess || cudaMalloc(&dW, wsb) != cudaSuccess ||
        cudaMemcpy(dF, F.data(), F.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dR, R.data(), R.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        st = EMO_ERR_CUDA;
    } else {
        const int prev_timing = g_timing.exchange(1);
        // Sum over three selections of the named stages' device times with
        // shape `sh` forced (the first selection also warms up), or +inf.
        auto timed = [&](const Shape& sh, std::initializer_list<const char*> stages) {
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                g_force = sh;
            }
            float best_ms = INFINITY;
            for (int rep = 0; rep < 4 && st == EMO_OK; ++rep) {
                st = emo_nsga3_select((const float*)dF, n2, m, (const float*)dR, (int32_t)n_r, n2 / 2, 1, rep,
                                      (int32_t*)dS, nullptr, dW, wsb, nullptr);
                float ms[32];
                const char* names[32];
                const int ns = st == EMO_OK ? emo_stage_times(ms, names, 32) : -1;
                if (ns < 0) {
                    if (st == EMO_OK) st = EMO_ERR_CUDA;
                    break;
                }
                float sum = 0.0f;
                for (int i = 0; i < ns; ++i)
                    for (const char* nm : stages)
                        if (std::strcmp(names[i], nm) == 0) sum += ms[i];
                if (rep > 0) best_ms = std::min(best_ms, sum);
            }
            return best_ms;
        };
        // coordinate search, one shape parameter at a time in pipeline order
        float bms = INFINITY;
        for (int c = kDomChunkMin; c <= kDomRowChunk && st == EMO_OK; c <<= 1) {
            Shape t = best;
            t.dom_chunk = c;
            const float v = timed(t, {"dominance"});
            if (v < bms) { bms = v; best.dom_chunk = c; }
        }
        bms = INFINITY;
        for (int w = 0; w <= 1 && st == EMO_OK; ++w) {
            Shape t = best;
            t.peel_wave = w;
            const float v = timed(t, {"peel"});
            if (v < bms) { bms = v; best.peel_wave = w; }
        }
        std::vector<int> caps = {0};
        for (int c = di.G / 2; c >= 1; c /= 2) caps.push_back(c);
        bms = INFINITY;
        for (int c : caps) {
            if (st != EMO_OK) break;
            Shape t = best;
            t.cap_wide = c;
            t.cap_narrow = 0;
            const float v = timed(t, {"peel"});
            if (v < bms) { bms = v; best.cap_wide = c; }
        }
        bms = INFINITY;
        for (int c : caps) {
            if (st != EMO_OK) break;
            if (best.cap_wide > 0 && (c == 0 || c > best.cap_wide)) continue;
            Shape t = best;
            t.cap_narrow = c;
            const float v = timed(t, {"sort", "stats", "csr", "niche", "finish"});
            if (v < bms) { bms = v; best.cap_narrow = c; }
        }
        bms = INFINITY;
        for (int c : {2, 4, 8, 16, 32}) {
            if (st != EMO_OK) break;
            Shape t = best;
            t.assoc_bps = c;
            const float v = timed(t, {"assoc"});
            if (v < bms) { bms = v; best.assoc_bps = c; }
        }
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_force = Shape{0, 0, -1, -1, -1};
        }
        g_timing.store(prev_timing);
    }
    cudaFree(dF); cudaFree(dR); cudaFree(dS); cudaFree(dW);
    if (st != EMO_OK) return st;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = best;
    }
    if (cache_path)
        if (FILE* fh = std::fopen(cache_path, "a")) {
            std::fprintf(fh, "%d %d %d %d %d %d %d %d\n", arch, (int)m, size_bucket(n2), best.assoc_bps,
                         best.dom_chunk, best.cap_wide, best.cap_narrow, best.peel_wave);
            std::fclose(fh);
        }
    return EMO_OK;
}

emo_status emo_launch_shape(int32_t m, int64_t n2, int32_t* shape_out)
{
    if (!sizes_ok(n2, m) || !shape_out) return EMO_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EMO_ERR_CUDA;
    DevInfo di = dev_info();
    if (!di.ok) return EMO_ERR_CUDA;
    const Shape sh = shape_for(dev, di.sms, m, n2);
    shape_out[0] = sh.assoc_bps;
    shape_out[1] = sh.dom_chunk;
    shape_out[2] = sh.cap_wide > 0 ? std::min(sh.cap_wide, di.G) : di.G;
    shape_out[3] = sh.cap_narrow > 0 ? std::min(sh.cap_narrow, shape_out[2]) : shape_out[2];
    shape_out[4] = sh.peel_wave;
    return EMO_OK;
}

void emo_autotune_reset(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
}

const char* emo_status_string(int status)
{
    switch (status) {
    case EMO_OK: return "ok";
    case EMO_ERR_INVALID_ARG: return "invalid argument";
    case EMO_ERR_NONFINITE: return "non-finite objective or zero/non-finite reference direction";
    case EMO_ERR_WORKSPACE: return "workspace too small";
    case EMO_ERR_CUDA: return "CUDA runtime error";
    case EMO_ERR_TIMEOUT: return "bounded device wait ran out";
    case EMO_ERR_NOT_IMPLEMENTED: return "not implemented";
    default: return "unknown status";
    }
}

int32_t emo_version(void) { return 100; }

int32_t emo_device_report(char* buf, int32_t len)
{
    if (!buf || len < 1) return -1;
    std::string out;
    int dev = -1, sms = 0, coop = 0;
    cudaError_t e = cudaGetDevice(&dev);
    out += "device " + std::to_string(dev) + (e == cudaSuccess ? "" : std::string(" error ") + cudaGetErrorString(e));
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    out += "; sms " + std::to_string(sms) + "; cooperative " + std::to_string(coop);
    DevInfo di = dev_info();  // also sets the dynamic shared memory limit of k_peel
    struct K { const char* name; const void* fn; int dyn; };
    const K ks[] = {{"k_sort", (const void*)k_sort, 0}, {"k_peel", (const void*)k_peel, kPeelDynSmem},
                    {"k_stats", (const void*)k_stats, 0}, {"k_csr", (const void*)k_csr, 0},
                    {"k_niche", (const void*)k_niche, 0}, {"k_niche_oneshot", (const void*)k_niche_oneshot, 0},
                    {"k_peel_wave", (const void*)k_peel_wave, kPeelWaveDynSmem},
                    {"k_hype", (const void*)k_hype, 0}, {"k_hype_counts", (const void*)k_hype_counts, hype_counts_smem(4)},
                    {"k_finish", (const void*)k_finish, 0}};
    for (const K& k : ks) {
        cudaFuncAttributes fa{};
        int occ = -1;
        cudaError_t e1 = cudaFuncGetAttributes(&fa, k.fn);
        cudaError_t e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k.fn, kCoopThreads, k.dyn);
        out += std::string("; ") + k.name + " regs " + std::to_string(fa.numRegs) + " smem " +
               std::to_string(fa.sharedSizeBytes) + " occ " + std::to_string(occ);
        if (e1 != cudaSuccess || e2 != cudaSuccess)
            out += std::string(" (") + cudaGetErrorString(e1 != cudaSuccess ? e1 : e2) + ")";
    }
    out += "; coop grid " + std::to_string(di.G) + (di.ok ? "" : " (unavailable)");
    std::snprintf(buf, (size_t)len, "%s", out.c_str());
    return (int32_t)out.size();
}

void emo_set_stage_timing(int32_t enable) { g_timing.store(enable ? 1 : 0); }

int32_t emo_stage_times(float* ms_out, const char** names_out, int32_t max_n)
{
    if (!g_st.created || g_st.n == 0) return 0;
    if (cudaEventSynchronize(g_st.ev[g_st.n]) != cudaSuccess) return -1;
    int n = std::min(g_st.n, (int)max_n);
    for (int i = 0; i < n; ++i) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, g_st.ev[i], g_st.ev[i + 1]) != cudaSuccess) return -1;
        if (ms_out) ms_out[i] = ms;
        if (names_out) names_out[i] = g_st.name[i];
    }
    return n;
}

}  // extern "C"
