// Pair schedules: which (target block, source range) items evaluate the dense
// sum of Eq. (2.30), and in what order their partial sums are added.
//
// The punctured kernel sum is symmetric in structure: the pair (i, j) needs
// r = |P_i - P_j|, e^{-kappa r}, the three dot products of d = P_i - P_j with
// n_i and n_j, and n_i . n_j, whichever of the two nodes is the target.  A
// symmetric item evaluates each pair of its (target block, source range) once
// for both orientations (pairkern.cuh, pair_item_sym); a one-sided item
// evaluates target rows only and masks the correction pairs N(i), which the
// dense sum omits.  N(i) is not symmetric (j in N(i) does not imply i in N(j)),
// so every block pair (I, J) in which some correction pair occurs in either
// direction is "near" and gets one-sided items from both sides; every other
// block pair with J > I gets symmetric items.  Since the correction nodes of i
// lie within a few h of P_i, near pairs form a band around the diagonal.
//
// Items are split to at most a quarter-wave of work each, and to at most
// kItemSeconds of one resident block's time, and sorted by cost for the
// atomic-counter scheduler.  Every item adds its sums into the nodes'
// exact accumulators (pairkern.cuh, fx_add: integer addition, so the order in
// which blocks add does not change a bit of the result).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <numeric>

#include "pairkern.cuh"

namespace ctr {

using namespace pk;

namespace {

constexpr int kItemsPerSlot = 4;     // items per resident block in a single-system launch
constexpr int kMaxBaseBlocks = 8192; // near-flag matrix side (bytes: its square)

// Relative cost of one symmetric pair evaluation (two orientations) against a
// one-sided one, per arithmetic: extra terms of the second orientation plus the
// in-warp transposed sums.
constexpr double kSymCost[3] = {1.25, 1.20, 1.15};

__global__ void near_flags_kernel(const int32_t* __restrict__ ptr, const int32_t* __restrict__ excl, int64_t M,
                                  int g0, int nb0, uint8_t* __restrict__ flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int bi = (int)(i / g0);
    flags[(size_t)bi * nb0 + bi] = 1;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
        const int bj = excl[e] / g0;
        flags[(size_t)bi * nb0 + bj] = 1;
        flags[(size_t)bj * nb0 + bi] = 1;
    }
}

template <typename Policy, int R, int V, int U>
__global__ void __launch_bounds__(kThreads, 2) sched_kernel(const typename Policy::Src* __restrict__ src, int M,
                                                         const int32_t* __restrict__ eptr,
                                                         const int32_t* __restrict__ excl,
                                                         const PairItem* __restrict__ items, int n_items,
                                                         int* __restrict__ counter,
                                                         unsigned long long* __restrict__ acc, PairConsts kc,
                                                         int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    PairSmem<Policy> sm(smem_raw);
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int cur;
    pair_block_init<Policy>(kc, sm.tab, bar);
    uint32_t gt = 0;
    for (;;) {
        if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
        __syncthreads();
        const int it = cur;
        __syncthreads();
        if (it >= n_items) break;
        if (!run_item<Policy, R, V, U>(items[it], src, M, eptr, excl, acc, kc, err, sm.ring, sm.jred, sm.tab, bar,
                                       gt))
            return;
    }
}

template <typename Policy, int R, int V, int U>
int sched_per_sm() {
    static int per_dev[64] = {0};   // resident blocks of this instantiation, per device (attribute set there)
    int dev = 0;
    CTR_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CTR_ERR_INVALID, "device index");
    int& per_sm = per_dev[dev];
    if (per_sm == 0) {
        int b = 0;
        // dynamic shared memory above the default 48 KB per block needs the kernel's opt-in
        CTR_CUDA_TRY(cudaFuncSetAttribute(sched_kernel<Policy, R, V, U>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)pair_smem_bytes<Policy>()));
        CTR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sched_kernel<Policy, R, V, U>, kThreads,
                                                                   pair_smem_bytes<Policy>()));
        per_sm = std::max(1, b);
    }
    return per_sm;
}

template <typename Policy, int R, int V, int U>
int sched_launch(ctr_ibim* s, int pol, const void* src, const PairConsts& kc, int sms) {
    const PairSchedule& p = s->sched[pol];
    if (p.items.empty()) return CTR_OK;
    const int per_sm = sched_per_sm<Policy, R, V, U>();
    if (per_sm < 0) return per_sm;
    const int grid = (int)std::min<int64_t>((int64_t)per_sm * sms, (int64_t)p.items.size());
    int* counter = s->counter.as<int>() + pol;
    CTR_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), s->stream));
    sched_kernel<Policy, R, V, U><<<grid, kThreads, pair_smem_bytes<Policy>(), s->stream>>>(
        reinterpret_cast<const typename Policy::Src*>(src), (int)s->M,
        s->tree ? s->tree->d_eptr.as<int32_t>() : s->corr_ptr.as<int32_t>(),
        s->tree ? s->tree->d_excl.as<int32_t>() : s->excl.as<int32_t>(), p.d_items.as<PairItem>(),
        (int)p.items.size(), counter, s->acc.as<unsigned long long>(), kc, s->err.as<int>());
    CTR_LAUNCHED();
    return CTR_OK;
}

// Items of one arithmetic for a system of M nodes with the given near-flag matrix.
void plan_schedule(PairSchedule& p, int64_t M, int R, int tile, double sym_cost, double item_cost,
                   const std::vector<uint8_t>& flags, int g0, int nb0, int slots) {
    p.R = R;
    p.BS = kThreads * R;
    p.tile = tile;
    const int BS = p.BS;
    const int nb = (int)((M + BS - 1) / BS);
    p.nb = nb;
    auto base_range = [&](int I, int& lo, int& hi) {
        lo = (int)((int64_t)I * BS / g0);
        hi = (int)std::min<int64_t>(nb0 - 1, (((int64_t)I + 1) * BS - 1) / g0);
    };
    auto near = [&](int I, int J) {
        int a0, a1, b0, b1;
        base_range(I, a0, a1);
        base_range(J, b0, b1);
        for (int a = a0; a <= a1; ++a)
            for (int b = b0; b <= b1; ++b)
                if (flags[(size_t)a * nb0 + b]) return true;
        return false;
    };
    struct Run {
        int I, j0, j1, sym;
    };
    std::vector<Run> runs;
    double total = 0.0;
    for (int I = 0; I < nb; ++I) {
        int J = 0;
        while (J < nb) {
            if (near(I, J)) {
                int J1 = J;
                while (J1 < nb && near(I, J1)) ++J1;
                runs.push_back(Run{I, (int)((int64_t)J * BS), (int)std::min<int64_t>(M, (int64_t)J1 * BS), 0});
                J = J1;
            } else if (J > I) {
                int J1 = J;
                while (J1 < nb && !near(I, J1)) ++J1;
                runs.push_back(Run{I, (int)((int64_t)J * BS), (int)std::min<int64_t>(M, (int64_t)J1 * BS), 1});
                J = J1;
            } else {
                ++J;
            }
        }
    }
    for (const Run& r : runs) total += (double)BS * (r.j1 - r.j0) * (r.sym ? sym_cost : 1.0);
    // split runs into items of at most a quarter-wave of work and kItemSeconds of one block (item_cost:
    // the arithmetic's rate x kItemSeconds; whole tiles, at least two when possible)
    const double nslots = (double)std::max(1, slots);
    const double cmax = std::max(1.0, std::min(total / ((double)kItemsPerSlot * nslots), item_cost / nslots));
    p.total_cost = total;
    p.items.clear();
    p.cost.clear();
    p.pairs_sym = p.pairs_one = 0;
    for (const Run& r : runs) {
        const int64_t len = r.j1 - r.j0;
        const double unit = (double)BS * (r.sym ? sym_cost : 1.0);
        int64_t pieces = std::max<int64_t>(1, (int64_t)std::ceil(unit * (double)len / cmax));
        int64_t plen = (len + pieces - 1) / pieces;
        plen = ((plen + tile - 1) / tile) * tile;
        plen = std::max<int64_t>(plen, std::min<int64_t>(len, 2 * (int64_t)tile));
        for (int64_t a = r.j0; a < r.j1; a += plen) {
            PairItem it{};
            it.I = r.I;
            it.j_begin = (int32_t)a;
            it.j_end = (int32_t)std::min<int64_t>(r.j1, a + plen);
            it.sym = r.sym;
            const int64_t tgt = std::min<int64_t>(BS, M - (int64_t)r.I * BS);
            if (r.sym) p.pairs_sym += tgt * (it.j_end - it.j_begin);
            else p.pairs_one += tgt * (it.j_end - it.j_begin);
            p.items.push_back(it);
            p.cost.push_back(unit * (double)(it.j_end - it.j_begin));
        }
    }
}

// Device copy of the items sorted by decreasing cost (afterwards the host copy is in that order too).
int upload_schedule(PairSchedule& p, int64_t M, cudaStream_t st) {
    std::vector<int> order(p.items.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return p.cost[a] > p.cost[b]; });
    std::vector<PairItem> sorted(p.items.size());
    std::vector<double> sorted_cost(p.items.size());
    for (size_t k = 0; k < order.size(); ++k) {
        sorted[k] = p.items[order[k]];
        sorted_cost[k] = p.cost[order[k]];
    }
    CTR_TRY(p.d_items.alloc(sizeof(PairItem) * std::max<size_t>(1, sorted.size())));
    if (!sorted.empty())
        CTR_CUDA_TRY(cudaMemcpyAsync(p.d_items.p, sorted.data(), sizeof(PairItem) * sorted.size(),
                                     cudaMemcpyHostToDevice, st));
    CTR_CUDA_TRY(cudaStreamSynchronize(st));   // the host vectors above go out of scope
    // the host copy follows the device order: the engine's work entries index the device list
    p.items.swap(sorted);
    p.cost.swap(sorted_cost);
    (void)M;
    return CTR_OK;
}

std::atomic<int> g_last_var32{-1};

struct PerSm {
    template <typename P, int R, int V, int U>
    int run() const { return sched_per_sm<P, R, V, U>(); }
};

struct SchedRun {
    ctr_ibim* s;
    const void* src;
    const PairConsts* kc;
    int sms;
    template <typename P, int R, int V, int U>
    int run() const { return sched_launch<P, R, V, U>(s, 0, src, *kc, sms); }
};

// The FP32 variant of a system: fixed by its options, else the one timed fastest on the first system
// of its size bucket (log2 M) on this device, cached for the process.  Timing: every variant's
// schedule for this system, one application each after a warm-up, with the right-hand side as the
// weights.  Leaves s->sched[0] planned for the chosen variant.
int plan_fp32(ctr_ibim* s, const std::vector<uint8_t>& flags, int g0, int nb0, int sms) {
    const int64_t M = s->M;
    auto plan = [&](int v) -> int {
        const int per = with_var32(v, PerSm{});
        if (per < 0) return per;
        plan_schedule(s->sched[0], M, kVar32[v].R * Fp32x2Policy::kPack, kVar32[v].tile, kSymCost[0],
                      kUnitRate[0] * kItemSeconds[0], flags, g0, nb0, per * sms);
        CTR_TRY(upload_schedule(s->sched[0], M, s->stream));
        s->sched[0].var = v;
        return CTR_OK;
    };
    const int want_bs = s->opt.fp32_block, want_tile = s->opt.fp32_tile;
    if (want_bs > 0 || want_tile > 0) {
        for (int v = 0; v < kNumVar32; ++v) {
            const int bs = kThreads * kVar32[v].R * Fp32x2Policy::kPack;
            if ((want_bs <= 0 || want_bs == bs) && (want_tile <= 0 || want_tile == kVar32[v].tile)) return plan(v);
        }
        return fail(CTR_ERR_INVALID, "fp32_block must be 512 or 1024 and fp32_tile 128 or 256");
    }
    static std::mutex mu;
    static std::map<std::pair<int, int>, int> cache;
    const int bucket = (int)std::floor(std::log2((double)std::max<int64_t>(M, 1)));
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find({s->device, bucket});
        if (it != cache.end()) {
            g_last_var32.store(it->second);
            return plan(it->second);
        }
    }
    CTR_TRY(pack_sources(s, s->rhs.as<double>(), CTR_FP32_REFINE));
    PairConsts kc;
    CTR_TRY(pair_consts(s, false, &kc));
    cudaEvent_t a = nullptr, b = nullptr;
    CTR_CUDA_TRY(cudaEventCreate(&a));
    CTR_CUDA_TRY(cudaEventCreate(&b));
    int best = 0;
    float best_ms = 1e30f;
    int st = CTR_OK;
    for (int v = 0; v < kNumVar32 && st == CTR_OK; ++v) {
        st = plan(v);
        const SchedRun r{s, s->src32.p, &kc, sms};
        if (st == CTR_OK && v == 0) st = with_var32(v, r);   // warm-up
        if (st == CTR_OK && cudaEventRecord(a, s->stream) != cudaSuccess) st = fail(CTR_ERR_CUDA, "event");
        if (st == CTR_OK) st = with_var32(v, r);
        if (st == CTR_OK && cudaEventRecord(b, s->stream) != cudaSuccess) st = fail(CTR_ERR_CUDA, "event");
        float ms = 0.f;
        if (st == CTR_OK && (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess))
            st = fail(CTR_ERR_CUDA, "event timing");
        if (st == CTR_OK && ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    CTR_TRY(st);
    CTR_TRY(check_device_error(s, "pair-kernel tuning"));
    // the timed applications added into the accumulators with no finish after them
    CTR_CUDA_TRY(cudaMemsetAsync(s->acc.p, 0, s->acc.bytes, s->stream));
    {
        std::lock_guard<std::mutex> lk(mu);
        best = cache.emplace(std::make_pair(s->device, bucket), best).first->second;   // first tuning wins
    }
    g_last_var32.store(best);
    return plan(best);
}

}  // namespace

int last_fp32_variant() { return g_last_var32.load(); }

int schedule_slots(int sms, int slots[3]) {
    const int a = with_var32(0, PerSm{});
    if (a < 0) return a;
    const int b = sched_per_sm<Df64Policy, kRdf, kChunkDf, 1>();
    if (b < 0) return b;
    const int c = sched_per_sm<Fp64Policy, kR64, kChunk64, 1>();
    if (c < 0) return c;
    slots[0] = a * sms;
    slots[1] = b * sms;
    slots[2] = c * sms;
    return CTR_OK;
}

int launch_schedule(ctr_ibim* s, int pol, const void* src, const PairConsts& kc) {
    CTR_TRY(ensure_schedule(s, pol));
    int sms = 0;
    CTR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
    if (pol == 0) return with_var32(s->sched[0].var, SchedRun{s, src, &kc, sms});
    if (pol == 1) return sched_launch<Df64Policy, kRdf, kChunkDf, 1>(s, 1, src, kc, sms);
    return sched_launch<Fp64Policy, kR64, kChunk64, 1>(s, 2, src, kc, sms);
}

// Near flags on base blocks of g0 nodes (the smallest target block, coarsened for huge systems).
static int near_flags(ctr_ibim* s, std::vector<uint8_t>& flags, int& g0, int& nb0) {
    const int64_t M = s->M;
    g0 = kThreads;
    while ((M + g0 - 1) / g0 > kMaxBaseBlocks) g0 *= 2;
    nb0 = (int)((M + g0 - 1) / g0);
    DevBuf d_flags;
    CTR_TRY(d_flags.alloc((size_t)nb0 * nb0));
    CTR_CUDA_TRY(cudaMemsetAsync(d_flags.p, 0, (size_t)nb0 * nb0, s->stream));
    near_flags_kernel<<<grid_for(M, 256), 256, 0, s->stream>>>(s->corr_ptr.as<int32_t>(), s->excl.as<int32_t>(), M,
                                                              g0, nb0, d_flags.as<uint8_t>());
    CTR_LAUNCHED();
    flags.assign((size_t)nb0 * nb0, 0);
    CTR_CUDA_TRY(cudaMemcpyAsync(flags.data(), d_flags.p, flags.size(), cudaMemcpyDeviceToHost, s->stream));
    CTR_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return CTR_OK;
}

// The float-float (pol 1) or FP64 (pol 2) schedule with its fixed shape.
static int plan_fixed(ctr_ibim* s, int pol, const std::vector<uint8_t>& flags, int g0, int nb0, const int slots[3]) {
    const int Rs[3] = {0, kRdf, kR64};   // targets per thread of the fixed shapes
    const int tiles[3] = {0, Df64Policy::kTile, Fp64Policy::kTile};
    plan_schedule(s->sched[pol], s->M, Rs[pol], tiles[pol], kSymCost[pol], kUnitRate[pol] * kItemSeconds[pol], flags,
                  g0, nb0, slots[pol]);
    CTR_TRY(upload_schedule(s->sched[pol], s->M, s->stream));
    s->sched[pol].planned = true;
    return CTR_OK;
}

// Setup: the FP32 schedule (tuned), and the float-float and FP64 ones if the handle's options use them
// (inner precision or refinement residual); an unused one is planned on first use (ensure_schedule).
int build_schedules(ctr_ibim* s, const int slots[3]) {
    std::vector<uint8_t> flags;
    int g0 = 0, nb0 = 0;
    CTR_TRY(near_flags(s, flags, g0, nb0));
    CTR_TRY(alloc_accumulators(s));
    CTR_TRY(s->counter.alloc(sizeof(int) * 4));
    const int prec = s->opt.precision;
    const bool uses[3] = {true, prec == CTR_DF64 || (prec == CTR_FP32_REFINE && s->opt.residual == CTR_DF64),
                          prec == CTR_FP64 || (prec == CTR_FP32_REFINE && s->opt.residual == CTR_FP64)};
    for (int p = 1; p < 3; ++p)
        if (uses[p]) CTR_TRY(plan_fixed(s, p, flags, g0, nb0, slots));
    int sms = 0;
    CTR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
    CTR_TRY(plan_fp32(s, flags, g0, nb0, sms));
    s->sched[0].planned = true;
    return CTR_OK;
}

int ensure_schedule(ctr_ibim* s, int pol) {
    if (pol < 0 || pol > 2) return fail(CTR_ERR_INVALID, "pair arithmetic");
    if (s->sched[pol].planned) return CTR_OK;
    if (pol == 0 || s->tree) return fail(CTR_ERR_INVALID, "schedule missing");   // planned at setup
    int sms = 0;
    CTR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
    int slots[3] = {0, 0, 0};
    CTR_TRY(schedule_slots(sms, slots));
    std::vector<uint8_t> flags;
    int g0 = 0, nb0 = 0;
    CTR_TRY(near_flags(s, flags, g0, nb0));
    return plan_fixed(s, pol, flags, g0, nb0, slots);
}

}  // namespace ctr
