// The operator of Eq. (2.30): punctured dense kernel sum + sparse correction + diagonal.
//
//   (A p)_1,i = lambda_1 rho1_i + h^3 sum_{j not in N(i)} W_j (K11 rho1_j - K12 rho2_j)
//               + sum_{m in N(i)} W_m (h^2 omega11 rho1_m - h^3 kappa/(4 pi) rho2_m)
//   (A p)_2,i = lambda_2 rho2_i + h^3 sum_{j not in N(i)} W_j (K21 rho1_j - K22 rho2_j)
//               + sum_{m in N(i)} W_m (h^2 omega21 rho1_m - h^2 omega22 rho2_m)
// (Eqs. 2.14-2.15), kernels K_ij of Eq. (1.4) at (P_i, n_i; P_j, n_j) (Eq. 2.11).
//
// Dense sum (the hot loop, M^2 pairs per application): one thread owns R
// targets (positions and normals in registers, per-tile FP32 partial sums
// folded into FP64 accumulators after every source tile).  Sources are
// packed 32 B (FP32) or 64 B (FP64) per node as {P, a}{n, b} with
// a = h^3 W rho1 / (4 pi), b = h^3 W rho2 / (4 pi), and streamed through a
// two-stage shared-memory ring filled by bulk asynchronous copies
// (cp.async.bulk + mbarrier transaction counts); every thread of the block
// reads each source by broadcast.  rsqrt and exp2 run on the SFU.  The
// correction pairs N(i) (sorted per target) are skipped exactly: a warp takes
// a masked path only for tiles that contain one of its lanes' excluded nodes.
// Source ranges are split across blockIdx.y; each split writes FP64 partial
// sums, which the finishing kernel adds in a fixed order (deterministic).
#include "common.cuh"

namespace ctr {

namespace {

constexpr int kThreads = 256;
constexpr int kTile32 = 256;     // sources per tile, FP32 (8 KB)
constexpr int kTile64 = 128;     // sources per tile, FP64 (8 KB)
constexpr uint32_t kWaitLimit = 1u << 22;

struct PairConsts {
    float c1f, c2f, kappaf, kl2f;    // eps_E/eps_I, eps_I/eps_E, kappa, -kappa log2(e)
    double c1, c2, kappa;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false after kWaitLimit polls (each poll may suspend briefly).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ float rsqrt_sfu(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_sfu(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ------------------------------------------------------------------ pair terms
// Adds a*K11 - b*K12 to acc1 and a*K21 - b*K22 to acc2 (times 4 pi, folded into a, b).
// d = x - y; s = 1/r^3; E = e^{-kappa r}; E1 = E (1 + kappa r):
//   4pi K11 = (d.n_y) s (1 - (eps_E/eps_I) E1)
//   4pi K12 = (1 - E)/r
//   4pi K22 = -(d.n_x) s (1 - (eps_I/eps_E) E1)
//   4pi K21 = s [ (1 - E1) n_x.n_y - (3 - E (3 + 3 kappa r + kappa^2 r^2)) (d.n_x)(d.n_y)/r^2 ]
__device__ __forceinline__ void pair_terms(float px, float py, float pz, float qx, float qy, float qz,
                                           const float4 pa, const float4 nb, const PairConsts& k,
                                           float& acc1, float& acc2) {
    const float dx = px - pa.x, dy = py - pa.y, dz = pz - pa.z;
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    const float rinv = rsqrt_sfu(r2);
    const float r = r2 * rinv;
    const float E = ex2_sfu(k.kl2f * r);
    const float kr = k.kappaf * r;
    const float E1 = fmaf(E, kr, E);
    const float dny = fmaf(dz, nb.z, fmaf(dy, nb.y, dx * nb.x));
    const float dnx = fmaf(dz, qz, fmaf(dy, qy, dx * qx));
    const float nn = fmaf(qz, nb.z, fmaf(qy, nb.y, qx * nb.x));
    const float rinv2 = rinv * rinv;
    const float s = rinv2 * rinv;
    const float as = pa.w * s, bs = nb.w * s;
    const float t1 = fmaf(-k.c1f, E1, 1.f);
    acc1 = fmaf(as, dny * t1, acc1);
    const float om = fmaf(-rinv, E, rinv);
    acc1 = fmaf(-nb.w, om, acc1);
    const float t2 = fmaf(-k.c2f, E1, 1.f);
    acc2 = fmaf(bs, dnx * t2, acc2);
    const float u = 1.f - E1;
    const float q = fmaf(kr, kr + 3.f, 3.f);
    const float t3 = fmaf(-E, q, 3.f);
    const float B = t3 * dnx * dny * rinv2;
    acc2 = fmaf(as, fmaf(u, nn, -B), acc2);
}

__device__ __forceinline__ void pair_terms(double px, double py, double pz, double qx, double qy, double qz,
                                           const double4 pa, const double4 nb, const PairConsts& k,
                                           double& acc1, double& acc2) {
    const double dx = px - pa.x, dy = py - pa.y, dz = pz - pa.z;
    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    const double rinv = rsqrt(r2);
    const double r = r2 * rinv;
    const double E = exp(-k.kappa * r);
    const double kr = k.kappa * r;
    const double E1 = fma(E, kr, E);
    const double dny = fma(dz, nb.z, fma(dy, nb.y, dx * nb.x));
    const double dnx = fma(dz, qz, fma(dy, qy, dx * qx));
    const double nn = fma(qz, nb.z, fma(qy, nb.y, qx * nb.x));
    const double rinv2 = rinv * rinv;
    const double s = rinv2 * rinv;
    const double as = pa.w * s, bs = nb.w * s;
    const double t1 = fma(-k.c1, E1, 1.0);
    acc1 = fma(as, dny * t1, acc1);
    const double om = fma(-rinv, E, rinv);
    acc1 = fma(-nb.w, om, acc1);
    const double t2 = fma(-k.c2, E1, 1.0);
    acc2 = fma(bs, dnx * t2, acc2);
    const double u = 1.0 - E1;
    const double q = fma(kr, kr + 3.0, 3.0);
    const double t3 = fma(-E, q, 3.0);
    const double B = t3 * dnx * dny * rinv2;
    acc2 = fma(as, fma(u, nn, -B), acc2);
}

template <typename Src>
struct SrcTraits;
template <>
struct SrcTraits<float4> {
    using Real = float;
    static constexpr int kTile = kTile32;
};
template <>
struct SrcTraits<double4> {
    using Real = double;
    static constexpr int kTile = kTile64;
};

template <typename Src, int R>
__global__ void __launch_bounds__(kThreads) pair_kernel(const Src* __restrict__ src, int M,
                                                        const int32_t* __restrict__ eptr,
                                                        const int32_t* __restrict__ excl, int src_per_split,
                                                        double* __restrict__ partial, PairConsts kc,
                                                        int* __restrict__ err) {
    using Real = typename SrcTraits<Src>::Real;
    constexpr int TILE = SrcTraits<Src>::kTile;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Src* ring = reinterpret_cast<Src*>(smem_raw);   // [2][TILE][2]
    __shared__ __align__(8) uint64_t bar[2];

    const int tid = threadIdx.x;
    const int j_begin = blockIdx.y * src_per_split;
    const int j_end = min(M, j_begin + src_per_split);
    const int ntiles = (j_end > j_begin) ? (j_end - j_begin + TILE - 1) / TILE : 0;

    Real px[R], py[R], pz[R], qx[R], qy[R], qz[R];
    double s1[R], s2[R];
    int ti[R], epos[R], eend[R], enext[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        ti[r] = blockIdx.x * (kThreads * R) + r * kThreads + tid;
        const int t = min(ti[r], M - 1);
        const Src a = src[2 * t], b = src[2 * t + 1];
        px[r] = a.x; py[r] = a.y; pz[r] = a.z;
        qx[r] = b.x; qy[r] = b.y; qz[r] = b.z;
        s1[r] = 0.0;
        s2[r] = 0.0;
        int e = eptr[t], ee = eptr[t + 1];
        while (e < ee && excl[e] < j_begin) ++e;
        epos[r] = e;
        eend[r] = ee;
        enext[r] = (e < ee) ? excl[e] : INT_MAX;
    }

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int k) {
        const int j0 = j_begin + k * TILE;
        const int n = min(TILE, j_end - j0);
        const uint32_t bytes = (uint32_t)(n * 2 * sizeof(Src));
        Src* dst = ring + (k & 1) * TILE * 2;
        fence_proxy_async();
        mbar_expect_tx(&bar[k & 1], bytes);
        bulk_load(dst, src + 2 * (size_t)j0, bytes, &bar[k & 1]);
    };
    if (tid == 0 && ntiles > 0) issue(0);

    for (int k = 0; k < ntiles; ++k) {
        if (tid == 0 && k + 1 < ntiles) issue(k + 1);
        const bool ok = mbar_wait(&bar[k & 1], (uint32_t)((k >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            // give up: flag it, let the copy that may still be in flight land, return
            if (tid == 0) {
                atomicOr(err, kErrWait);
                if (k + 1 < ntiles) (void)mbar_wait(&bar[(k + 1) & 1], (uint32_t)(((k + 1) >> 1) & 1));
            }
            return;
        }
        const Src* tile = ring + (k & 1) * TILE * 2;
        const int j0 = j_begin + k * TILE;
        const int n = min(TILE, j_end - j0);
        bool need = false;
#pragma unroll
        for (int r = 0; r < R; ++r) need |= (enext[r] < j0 + n);
        Real a1[R], a2[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a1[r] = a2[r] = Real(0);
        if (!__any_sync(0xffffffffu, need)) {
#pragma unroll 4
            for (int q = 0; q < n; ++q) {
                const Src pa = tile[2 * q], nb = tile[2 * q + 1];
#pragma unroll
                for (int r = 0; r < R; ++r)
                    pair_terms(px[r], py[r], pz[r], qx[r], qy[r], qz[r], pa, nb, kc, a1[r], a2[r]);
            }
        } else {
            for (int q = 0; q < n; ++q) {
                const Src pa = tile[2 * q], nb = tile[2 * q + 1];
                const int j = j0 + q;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const bool ex = (j == enext[r]);
                    Src pa2 = pa, nb2 = nb;
                    if (ex) {
                        // excluded correction pair: a zero-weight source at distance 1 (no NaN)
                        pa2.x = px[r] + Real(1);
                        pa2.y = py[r];
                        pa2.z = pz[r];
                        pa2.w = Real(0);
                        nb2.w = Real(0);
                        ++epos[r];
                        enext[r] = (epos[r] < eend[r]) ? excl[epos[r]] : INT_MAX;
                    }
                    pair_terms(px[r], py[r], pz[r], qx[r], qy[r], qz[r], pa2, nb2, kc, a1[r], a2[r]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            s1[r] += (double)a1[r];
            s2[r] += (double)a2[r];
        }
        __syncthreads();   // the buffer of tile k is free for tile k + 2
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (ti[r] < M) {
            partial[((size_t)blockIdx.y * 2 + 0) * M + ti[r]] = s1[r];
            partial[((size_t)blockIdx.y * 2 + 1) * M + ti[r]] = s2[r];
        }
    }
}

// a = h^3 W rho1/(4 pi), b = h^3 W rho2/(4 pi) into the .w slots of the packed sources
__global__ void pack_kernel(const double* __restrict__ x, const double* __restrict__ W, int64_t M, double scale,
                            float4* __restrict__ s32, double4* __restrict__ s64) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const double a = scale * W[j] * x[j];
    const double b = scale * W[j] * x[M + j];
    if (s32) {
        s32[2 * j].w = (float)a;
        s32[2 * j + 1].w = (float)b;
    }
    if (s64) {
        s64[2 * j].w = a;
        s64[2 * j + 1].w = b;
    }
}

// y = diag + fixed-order sum of the split partials + correction (FP64)
__global__ void finish_kernel(int64_t M, int S, const double* __restrict__ partial, const double* __restrict__ x,
                              double* __restrict__ y, const double* __restrict__ W, const int32_t* __restrict__ ptr,
                              const int32_t* __restrict__ node, const double* __restrict__ w, int64_t E,
                              double lam1, double lam2, double h2, double h3w12) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    double s1 = 0.0, s2 = 0.0;
    for (int s = 0; s < S; ++s) {
        s1 += partial[((size_t)s * 2 + 0) * M + i];
        s2 += partial[((size_t)s * 2 + 1) * M + i];
    }
    double c1 = 0.0, c2 = 0.0;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
        const int m = node[e];
        const double Wm = W[m], r1 = x[m], r2 = x[M + m];
        c1 += Wm * (h2 * w[e] * r1 - h3w12 * r2);
        c2 += Wm * (h2 * w[E + e] * r1 - h2 * w[2 * E + e] * r2);
    }
    y[i] = lam1 * x[i] + s1 + c1;
    y[M + i] = lam2 * x[M + i] + s2 + c2;
}

template <typename Src, int R>
int launch_pairs(ctr_ibim* s, const Src* src, const PairPlan& p, const PairConsts& kc) {
    const int TILE = SrcTraits<Src>::kTile;
    const size_t smem = 2 * TILE * 2 * sizeof(Src);
    dim3 grid(p.target_blocks, p.splits);
    pair_kernel<Src, R><<<grid, kThreads, smem, s->stream>>>(src, (int)s->M, s->corr_ptr.as<int32_t>(),
                                                            s->excl.as<int32_t>(), p.src_per_split,
                                                            s->partial.as<double>(), kc, s->err.as<int>());
    CTR_CUDA_TRY(cudaGetLastError());
    return CTR_OK;
}

PairPlan make_plan(int64_t M, int R, int tile, int sms) {
    PairPlan p;
    p.R = R;
    p.target_blocks = (int)((M + (int64_t)kThreads * R - 1) / ((int64_t)kThreads * R));
    const int want = 4 * sms;   // blocks in flight for load balance
    int splits = (want + p.target_blocks - 1) / p.target_blocks;
    const int max_splits = (int)((M + tile - 1) / tile);
    splits = std::max(1, std::min(splits, max_splits));
    int64_t per = (M + splits - 1) / splits;
    per = ((per + tile - 1) / tile) * tile;
    p.src_per_split = (int)per;
    p.splits = (int)((M + per - 1) / per);
    return p;
}

}  // namespace

int plan_pairs(ctr_ibim* s) {
    int sms = 0;
    CTR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
    int R32 = s->opt.tile_targets;
    if (R32 != 1 && R32 != 2 && R32 != 4) R32 = 2;
    s->plan32 = make_plan(s->M, R32, kTile32, sms);
    s->plan64 = make_plan(s->M, 1, kTile64, sms);
    const int S = std::max(s->plan32.splits, s->plan64.splits);
    CTR_TRY(s->partial.alloc(sizeof(double) * 2 * (size_t)S * s->M));
    return CTR_OK;
}

int apply_operator(ctr_ibim* s, const double* d_x, double* d_y, int precision) {
    const int64_t M = s->M;
    cudaStream_t st = s->stream;
    const bool fp32 = (precision == CTR_FP32_REFINE);
    const double scale = s->h * s->h * s->h / (4.0 * kPi);
    pack_kernel<<<grid_for(M, 256), 256, 0, st>>>(d_x, s->na.W, M, scale, fp32 ? s->src32.as<float4>() : nullptr,
                                                 fp32 ? nullptr : s->src64.as<double4>());
    CTR_CUDA_TRY(cudaGetLastError());
    PairConsts kc;
    kc.c1 = s->eps_out / s->eps_in;
    kc.c2 = s->eps_in / s->eps_out;
    kc.kappa = s->kappa;
    kc.c1f = (float)kc.c1;
    kc.c2f = (float)kc.c2;
    kc.kappaf = (float)s->kappa;
    kc.kl2f = (float)(-s->kappa * 1.4426950408889634);
    const PairPlan& p = fp32 ? s->plan32 : s->plan64;
    if (fp32) {
        switch (p.R) {
            case 1: CTR_TRY((launch_pairs<float4, 1>(s, s->src32.as<float4>(), p, kc))); break;
            case 4: CTR_TRY((launch_pairs<float4, 4>(s, s->src32.as<float4>(), p, kc))); break;
            default: CTR_TRY((launch_pairs<float4, 2>(s, s->src32.as<float4>(), p, kc))); break;
        }
    } else {
        CTR_TRY((launch_pairs<double4, 1>(s, s->src64.as<double4>(), p, kc)));
    }
    const double h2 = s->h * s->h;
    const double h3w12 = s->h * s->h * s->h * s->kappa / (4.0 * kPi);
    finish_kernel<<<grid_for(M, 256), 256, 0, st>>>(M, p.splits, s->partial.as<double>(), d_x, d_y, s->na.W,
                                                   s->corr_ptr.as<int32_t>(), s->corr_node.as<int32_t>(),
                                                   s->corr_w.as<double>(), s->E,
                                                   0.5 * (1.0 + s->eps_out / s->eps_in),
                                                   0.5 * (1.0 + s->eps_in / s->eps_out), h2, h3w12);
    CTR_CUDA_TRY(cudaGetLastError());
    return CTR_OK;
}

}  // namespace ctr
