// The operator of Eq. (2.30): punctured dense kernel sum + sparse correction + diagonal.
//
//   (A p)_1,i = lambda_1 rho1_i + h^3 sum_{j not in N(i)} W_j (K11 rho1_j - K12 rho2_j)
//               + sum_{m in N(i)} W_m (h^2 omega11 rho1_m - h^3 kappa/(4 pi) rho2_m)
//   (A p)_2,i = lambda_2 rho2_i + h^3 sum_{j not in N(i)} W_j (K21 rho1_j - K22 rho2_j)
//               + sum_{m in N(i)} W_m (h^2 omega21 rho1_m - h^2 omega22 rho2_m)
// (Eqs. 2.14-2.15), kernels K_ij of Eq. (1.4) at (P_i, n_i; P_j, n_j) (Eq. 2.11).
//
// Dense sum (the hot loop, M^2 pairs per application): one thread owns R
// targets (positions and normals in registers, per-tile partial sums folded
// into FP64 accumulators after every source tile).  Sources are packed per
// node as {P, a}{n, b} with a = h^3 W rho1/(4 pi), b = h^3 W rho2/(4 pi) and
// streamed through a two-stage shared-memory ring filled by bulk asynchronous
// copies (cp.async.bulk + mbarrier transaction counts); every thread of the
// block reads each source by broadcast.  The correction pairs N(i) (sorted
// per target) are skipped exactly: a warp takes a masked path only for tiles
// that contain one of its lanes' excluded nodes.  The work is a schedule of
// one-sided and symmetric items (schedule.cu): block pairs without correction
// pairs are evaluated once for both orientations, and each item adds its FP64
// sums into the nodes' exact accumulators (integer addition: the result does
// not depend on the order in which blocks add), read and cleared by the
// finishing kernel.
//
// Three pair arithmetics share this pipeline (policies below):
//   Fp32  FP32 terms, rsqrt and exp2 on the SFU (44 FP32-pipe ops per pair);
//   Fp64  IEEE FP64 (DFMA, 1/64 of the FP32 rate on this chip);
//   Df64  double-FP32 "float-float" terms (error-free sums and products with
//         FMA, rsqrt by one Newton step in df64, exp by two exact tables and
//         a degree-4 polynomial), ~2^-44 relative, on the FP32 pipe.
#include <atomic>
#include <cstring>
#include <mutex>

#include "pairkern.cuh"

namespace ctr {

using namespace pk;

namespace {

template <typename Policy, int R>
__global__ void __launch_bounds__(kThreads) pair_kernel(const typename Policy::Src* __restrict__ src, int M,
                                                        const int32_t* __restrict__ eptr,
                                                        const int32_t* __restrict__ excl, int src_per_split,
                                                        double* __restrict__ partial, PairConsts kc,
                                                        int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    PairSmem<Policy> sm(smem_raw);
    __shared__ __align__(8) uint64_t bar[2];
    pair_block_init<Policy>(kc, sm.tab, bar);
    const int j_begin = blockIdx.y * src_per_split;
    const int j_end = min(M, j_begin + src_per_split);
    uint32_t gt = 0;
    const RegionOut out{partial + (size_t)blockIdx.y * 2 * M, M, 0};
    (void)pair_item<Policy, R, 2, RegionOut>(src, M, eptr, excl, blockIdx.x, j_begin, j_end, out, kc, err, sm.ring,
                                             sm.tab, bar, gt);
}

// a = h^3 W rho1/(4 pi), b = h^3 W rho2/(4 pi) into the weight slots of the packed sources
// (at the node's tree position when the treecode has reordered the sources)
__global__ void pack_kernel(const double* __restrict__ x, const double* __restrict__ W, int64_t M, double scale,
                            float4* __restrict__ s32, double4* __restrict__ s64, float4* __restrict__ sdf,
                            const int32_t* __restrict__ tinv) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M) return;
    const double a = scale * W[t] * x[t];
    const double b = scale * W[t] * x[M + t];
    const int64_t j = tinv ? (int64_t)tinv[t] : t;
    if (s32) {   // duplicated pairs: a and -b
        s32[4 * j + 1].z = s32[4 * j + 1].w = (float)a;
        s32[4 * j + 3].z = s32[4 * j + 3].w = -(float)b;
    }
    if (s64) {
        s64[2 * j].w = a;
        s64[2 * j + 1].w = b;
    }
    if (sdf) {
        const float ah = (float)a, bh = (float)b;
        sdf[4 * j].w = ah;
        sdf[4 * j + 1].w = (float)(a - (double)ah);
        sdf[4 * j + 2].w = bh;
        sdf[4 * j + 3].w = (float)(b - (double)bh);
    }
}

// y = diag + the node's accumulated dense sum (read and cleared) + correction (FP64)
__global__ void finish_kernel(int64_t M, unsigned long long* __restrict__ acc, const double* __restrict__ x,
                              double* __restrict__ y, const double* __restrict__ W, const int32_t* __restrict__ ptr,
                              const int32_t* __restrict__ node, const double* __restrict__ w, int64_t E,
                              double lam1, double lam2, double h2, double h3, const int32_t* __restrict__ tinv) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    double s1, s2;
    fx_read(acc + (tinv ? (int64_t)tinv[i] : i), M, true, s1, s2);
    double c1 = 0.0, c2 = 0.0;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
        const int m = node[e];
        const double Wm = W[m], r1 = x[m], r2 = x[M + m];
        c1 += Wm * (h2 * w[e] * r1 - h3 * w[3 * E + e] * r2);
        c2 += Wm * (h2 * w[E + e] * r1 - h2 * w[2 * E + e] * r2);
    }
    y[i] = lam1 * x[i] + s1 + c1;
    y[M + i] = lam2 * x[M + i] + s2 + c2;
}

// float-float static source data {P.hi}{P.lo}{n.hi}{n.lo} (weights filled per application)
__global__ void df_static_kernel(NodeArrays na, int64_t M, float4* __restrict__ sdf) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    auto hi = [](double v) { return (float)v; };
    auto lo = [](double v) { return (float)(v - (double)(float)v); };
    sdf[4 * j] = make_float4(hi(na.Px[j]), hi(na.Py[j]), hi(na.Pz[j]), 0.f);
    sdf[4 * j + 1] = make_float4(lo(na.Px[j]), lo(na.Py[j]), lo(na.Pz[j]), 0.f);
    sdf[4 * j + 2] = make_float4(hi(na.nx[j]), hi(na.ny[j]), hi(na.nz[j]), 0.f);
    sdf[4 * j + 3] = make_float4(lo(na.nx[j]), lo(na.ny[j]), lo(na.nz[j]), 0.f);
}

}  // namespace

// Source splits for equal-work items (target block x source range) that fill
// whole waves of resident blocks: minimise ceil(items / slots) / splits, the
// time in units of a full-range item, and take the fewest splits within 5% of it.
PairPlan make_plan(int64_t M, int R, int tile, int slots) {
    PairPlan p;
    p.R = R;
    p.target_blocks = (int)((M + (int64_t)kThreads * R - 1) / ((int64_t)kThreads * R));
    const int max_splits = (int)std::max<int64_t>(1, std::min<int64_t>((M + tile - 1) / tile, 256));
    auto actual = [&](int S, int64_t& per) {
        per = (M + S - 1) / S;
        per = ((per + tile - 1) / tile) * tile;
        return (int)((M + per - 1) / per);
    };
    double best = 1e300;
    std::vector<double> cost(max_splits + 1, 1e300);
    for (int S = 1; S <= max_splits; ++S) {
        int64_t per;
        const int Sa = actual(S, per);
        const int64_t items = (int64_t)p.target_blocks * Sa;
        const int64_t waves = (items + slots - 1) / slots;
        cost[S] = (double)waves * (double)per / (double)M;
        best = std::min(best, cost[S]);
    }
    int pick = 1;
    for (int S = 1; S <= max_splits; ++S)
        if (cost[S] <= 1.05 * best) { pick = S; break; }
    int64_t per;
    p.splits = actual(pick, per);
    p.src_per_split = (int)per;
    return p;
}

// Dynamic shared memory of the one-sided grid launch: the source ring only (no symmetric items, no
// tables); the occupancy query and the launch use the same figure.
template <typename Policy>
constexpr size_t grid_launch_smem() {
    static_assert(!Policy::kTables, "the one-sided grid launch carries no exponential tables");
    return pair_ring_bytes<Policy>();
}

template <typename Policy, int R>
int resident_slots(int sms, int* slots) {
    int per_sm = 0;
    const size_t smem = grid_launch_smem<Policy>();
    CTR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_kernel<Policy, R>, kThreads, smem));
    *slots = std::max(1, per_sm) * sms;
    return CTR_OK;
}

// float-float table of e^{-k} (k < 64) and e^{-k/1024} (k < 1024), one per device
int exp_table(int dev, const float2** out) {
    static std::mutex mu;
    static DevBuf tabs[64];
    static bool ready[64] = {false};
    if (dev < 0 || dev >= 64) return fail(CTR_ERR_INVALID, "device index");
    std::lock_guard<std::mutex> lk(mu);
    if (!ready[dev]) {
        std::vector<float2> h(kExpHi + kExpLo);
        for (int k = 0; k < kExpHi; ++k) h[k] = split_ff(std::exp(-(double)k));
        for (int k = 0; k < kExpLo; ++k) h[kExpHi + k] = split_ff(std::exp(-(double)k / 1024.0));
        CTR_TRY(tabs[dev].alloc(sizeof(float2) * h.size()));
        CTR_CUDA_TRY(cudaMemcpy(tabs[dev].p, h.data(), sizeof(float2) * h.size(), cudaMemcpyHostToDevice));
        ready[dev] = true;
    }
    *out = tabs[dev].as<float2>();
    return CTR_OK;
}

// The f32x2 operands: each FP32 constant in both halves of a 64-bit word.
void set_packed_consts(PairConsts& kc) {
    auto dup = [](float f) {
        uint32_t b;
        std::memcpy(&b, &f, sizeof b);
        return ((unsigned long long)b << 32) | (unsigned long long)b;
    };
    kc.one2 = dup(1.f);
    kc.mone2 = dup(-1.f);
    kc.three2 = dup(3.f);
    kc.mthree2 = dup(-3.f);
    kc.c1x2 = dup(kc.c1f);
    kc.nc1x2 = dup(-kc.c1f);
    kc.c2x2 = dup(kc.c2f);
    kc.nc2x2 = dup(-kc.c2f);
    kc.kap2 = dup(kc.kappaf);
    kc.kl2x2 = dup(kc.kl2f);
}

namespace {
std::atomic<uint32_t> g_wait_limit{kWaitLimit};
}  // namespace

uint32_t wait_limit() { return g_wait_limit.load(std::memory_order_relaxed); }

int pair_consts(ctr_ibim* s, bool tables, PairConsts* out) {
    PairConsts kc{};
    kc.wait_limit = wait_limit();
    kc.c1 = s->eps_out / s->eps_in;
    kc.c2 = s->eps_in / s->eps_out;
    kc.kappa = s->kappa;
    kc.c1f = (float)kc.c1;
    kc.c2f = (float)kc.c2;
    kc.kappaf = (float)s->kappa;
    kc.kl2f = (float)(-s->kappa * 1.4426950408889634);
    kc.c1d = split_ff(kc.c1);
    kc.c2d = split_ff(kc.c2);
    kc.kappad = split_ff(kc.kappa);
    set_packed_consts(kc);
    kc.exp_tab = nullptr;
    if (tables) CTR_TRY(exp_table(s->device, &kc.exp_tab));
    *out = kc;
    return CTR_OK;
}

int pack_sources(ctr_ibim* s, const double* d_x, int precision) {
    const int64_t M = s->M;
    const double scale = s->h * s->h * s->h / (4.0 * kPi);
    float4* s32 = (precision == CTR_FP32_REFINE) ? s->src32.as<float4>() : nullptr;
    double4* s64 = (precision == CTR_FP64) ? s->src64.as<double4>() : nullptr;
    float4* sdf = (precision == CTR_DF64) ? s->srcdf.as<float4>() : nullptr;
    const int32_t* tinv = s->tree ? s->tree->d_tinv.as<int32_t>() : nullptr;
    pack_kernel<<<grid_for(M, 256), 256, 0, s->stream>>>(d_x, s->na.W, M, scale, s32, s64, sdf, tinv);
    CTR_LAUNCHED();
    return CTR_OK;
}

int alloc_accumulators(ctr_ibim* s) {
    const size_t bytes = sizeof(unsigned long long) * (size_t)kFxWords * (size_t)s->M;
    CTR_TRY(s->acc.alloc(bytes));
    CTR_CUDA_TRY(cudaMemsetAsync(s->acc.p, 0, bytes, s->stream));
    return CTR_OK;
}

int plan_pairs(ctr_ibim* s) {
    int sms = 0;
    CTR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
    int slots[3] = {0, 0, 0};
    CTR_TRY(schedule_slots(sms, slots));
    CTR_TRY(s->srcdf.alloc(sizeof(float4) * 4 * (size_t)s->M));
    df_static_kernel<<<grid_for(s->M, 256), 256, 0, s->stream>>>(s->na, s->M, s->srcdf.as<float4>());
    CTR_LAUNCHED();
    if (s->opt.farfield == CTR_FARFIELD_TREECODE) return build_tree_schedules(s, slots);
    return build_schedules(s, slots);
}

int apply_operator(ctr_ibim* s, const double* d_x, double* d_y, int precision) {
    return apply_operator_timed(s, d_x, d_y, precision, nullptr);
}

// The operator with, when ev is not NULL, events recorded on the handle's stream before packing, the
// pair items, the far field, the finish and after it (ev[0..4]).
int apply_operator_timed(ctr_ibim* s, const double* d_x, double* d_y, int precision, cudaEvent_t* ev) {
    const int64_t M = s->M;
    cudaStream_t st = s->stream;
    auto mark = [&](int k) -> int {
        if (ev) CTR_CUDA_TRY(cudaEventRecord(ev[k], st));
        return CTR_OK;
    };
    CTR_TRY(mark(0));
    const double scale = s->h * s->h * s->h / (4.0 * kPi);
    float4* s32 = (precision == CTR_FP32_REFINE) ? s->src32.as<float4>() : nullptr;
    double4* s64 = (precision == CTR_FP64) ? s->src64.as<double4>() : nullptr;
    float4* sdf = (precision == CTR_DF64) ? s->srcdf.as<float4>() : nullptr;
    const int32_t* tinv = s->tree ? s->tree->d_tinv.as<int32_t>() : nullptr;
    pack_kernel<<<grid_for(M, 256), 256, 0, st>>>(d_x, s->na.W, M, scale, s32, s64, sdf, tinv);
    CTR_LAUNCHED();
    PairConsts kc;
    CTR_TRY(pair_consts(s, precision == CTR_DF64, &kc));
    const int pol = (precision == CTR_FP32_REFINE) ? 0 : (precision == CTR_DF64 ? 1 : 2);
    const void* src = s32 ? (const void*)s32 : (sdf ? (const void*)sdf : (const void*)s64);
    CTR_TRY(mark(1));
    CTR_TRY(launch_schedule(s, pol, src, kc));
    CTR_TRY(mark(2));
    CTR_TRY(launch_tree(s, pol));
    CTR_TRY(mark(3));
    const double h2 = s->h * s->h;
    const double h3 = s->h * s->h * s->h;
    finish_kernel<<<grid_for(M, 256), 256, 0, st>>>(M, s->acc.as<unsigned long long>(), d_x, d_y, s->na.W,
                                                   s->corr_ptr.as<int32_t>(), s->corr_node.as<int32_t>(),
                                                   s->corr_w.as<double>(), s->E,
                                                   0.5 * (1.0 + s->eps_out / s->eps_in),
                                                   0.5 * (1.0 + s->eps_in / s->eps_out), h2, h3, tinv);
    CTR_LAUNCHED();
    CTR_TRY(mark(4));
    return CTR_OK;
}

}  // namespace ctr

extern "C" int ctr_set_wait_limit(int64_t polls) {
    if (polls > (int64_t)UINT32_MAX) return ctr::fail(CTR_ERR_INVALID, "polls must be < 2^32");
    ctr::g_wait_limit.store(polls < 0 ? ctr::pk::kWaitLimit : (uint32_t)polls, std::memory_order_relaxed);
    return CTR_OK;
}

namespace ctr {

// FP32 pair sum of caller-provided packed sources into caller-provided split
// scratch (partial, at most max_partial doubles); used by the entry point
// whose scratch is a fixed device array.  Returns the number of splits used.
int launch_fp32_pairs_external(const float4* src, int64_t M, const int32_t* eptr, const int32_t* excl,
                               double eps_ratio, double kappa, int64_t max_partial, double* partial, int* err,
                               cudaStream_t st, int* splits_out) {
    int dev = 0, sms = 0;
    CTR_CUDA_TRY(cudaGetDevice(&dev));
    CTR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int slots = 0;
    CTR_TRY((resident_slots<Fp32Policy, 2>(sms, &slots)));
    PairPlan p = make_plan(M, 2, Fp32Policy::kTile, slots);
    const int64_t cap = max_partial / (2 * M);
    if (cap < 1) return fail(CTR_ERR_CAPACITY, "scratch too small for this many nodes");
    if (p.splits > cap) {
        int64_t per = (M + cap - 1) / cap;
        per = ((per + Fp32Policy::kTile - 1) / Fp32Policy::kTile) * Fp32Policy::kTile;
        p.src_per_split = (int)per;
        p.splits = (int)((M + per - 1) / per);
    }
    PairConsts kc{};
    kc.c1 = eps_ratio;
    kc.c2 = 1.0 / eps_ratio;
    kc.kappa = kappa;
    kc.c1f = (float)kc.c1;
    kc.c2f = (float)kc.c2;
    kc.kappaf = (float)kappa;
    kc.kl2f = (float)(-kappa * 1.4426950408889634);
    set_packed_consts(kc);
    kc.wait_limit = wait_limit();
    const size_t smem = grid_launch_smem<Fp32Policy>();
    dim3 grid(p.target_blocks, p.splits);
    pair_kernel<Fp32Policy, 2><<<grid, kThreads, smem, st>>>(src, (int)M, eptr, excl, p.src_per_split, partial, kc,
                                                             err);
    CTR_LAUNCHED();
    *splits_out = p.splits;
    return CTR_OK;
}

}  // namespace ctr
