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
// that contain one of its lanes' excluded nodes.  Source ranges are split
// across blockIdx.y; each split writes FP64 partial sums, which the
// finishing kernel adds in a fixed order (deterministic).
//
// Three pair arithmetics share this pipeline (policies below):
//   Fp32  FP32 terms, rsqrt and exp2 on the SFU (44 FP32-pipe ops per pair);
//   Fp64  IEEE FP64 (DFMA, 1/64 of the FP32 rate on this chip);
//   Df64  double-FP32 "float-float" terms (error-free sums and products with
//         FMA, rsqrt by one Newton step in df64, exp by two exact tables and
//         a degree-4 polynomial), ~2^-44 relative, on the FP32 pipe.
#include "common.cuh"

namespace ctr {

namespace {

constexpr int kThreads = 256;
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr int kExpHi = 64;      // e^{-k}, k = 0..63
constexpr int kExpLo = 1024;    // e^{-k/1024}, k = 0..1023

struct PairConsts {
    float c1f, c2f, kappaf, kl2f;    // eps_E/eps_I, eps_I/eps_E, kappa, -kappa log2(e)
    double c1, c2, kappa;
    float2 c1d, c2d, kappad;         // float-float copies
    const float2* exp_tab;           // [kExpHi + kExpLo] float-float, global
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

// ------------------------------------------------------------------ float-float arithmetic
// A value is hi + lo with |lo| <= ulp(hi)/2.  Error-free transformations use
// explicitly rounded intrinsics so that nothing is fused or reassociated.
struct F2 {
    float hi, lo;
};
__device__ __forceinline__ F2 f2(float2 v) { return F2{v.x, v.y}; }
__device__ __forceinline__ F2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return F2{s, e};
}
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {   // |a| >= |b|, or a == 0
    const float s = __fadd_rn(a, b);
    return F2{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ F2 two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return F2{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ F2 neg(F2 a) { return F2{-a.hi, -a.lo}; }
__device__ __forceinline__ F2 add(F2 a, F2 b) {
    const F2 s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ F2 sub(F2 a, F2 b) { return add(a, neg(b)); }
__device__ __forceinline__ F2 add_f(F2 a, float b) {
    const F2 s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ F2 mul(F2 a, F2 b) {
    const F2 p = two_prod(a.hi, b.hi);
    return fast_two_sum(p.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo)));
}
// a0 b0 + a1 b1 + a2 b2
__device__ __forceinline__ F2 dot3(F2 a0, F2 a1, F2 a2, F2 b0, F2 b1, F2 b2) {
    const F2 p0 = two_prod(a0.hi, b0.hi), p1 = two_prod(a1.hi, b1.hi), p2 = two_prod(a2.hi, b2.hi);
    const F2 s = two_sum(p0.hi, p1.hi);
    const F2 t = two_sum(s.hi, p2.hi);
    float e = __fadd_rn(__fadd_rn(p0.lo, p1.lo), __fadd_rn(p2.lo, __fadd_rn(s.lo, t.lo)));
    e = __fmaf_rn(a0.hi, b0.lo, __fmaf_rn(a0.lo, b0.hi, e));
    e = __fmaf_rn(a1.hi, b1.lo, __fmaf_rn(a1.lo, b1.hi, e));
    e = __fmaf_rn(a2.hi, b2.lo, __fmaf_rn(a2.lo, b2.hi, e));
    return fast_two_sum(t.hi, e);
}
// 1/sqrt(x): SFU seed y0 (rel. err < 2^-22), one Newton step y0 + y0 (1 - x y0^2)/2 in float-float
__device__ __forceinline__ F2 rsqrt_ff(F2 x) {
    const float y0 = rsqrt_sfu(x.hi);
    const F2 t = mul(x, two_prod(y0, y0));
    const float e = __fsub_rn(__fsub_rn(1.0f, t.hi), t.lo);
    return fast_two_sum(y0, __fmul_rn(__fmul_rn(0.5f, y0), e));
}
// e^{-x}, x >= 0: x = k/1024 + f (k nearest), e^{-x} = e^{-(k>>10)} e^{-(k&1023)/1024} e^{-f},
// e^{-f} = 1 - f + f^2 (1/2 - f/6 + f^2/24) for |f| <= 1/2048 (truncation < 3e-19)
__device__ __forceinline__ F2 exp_neg_ff(F2 x, const float2* tab) {
    float xh = x.hi, xl = x.lo;
    if (xh > 63.9f) {
        xh = 63.9f;
        xl = 0.f;
    }
    const float t = __fmaf_rn(xh, 1024.f, 12582912.f);   // 1.5 * 2^23: round(x * 1024) in the mantissa
    const int k = min(max(__float_as_int(t) - 0x4B400000, 0), kExpHi * kExpLo - 1);   // in range for any input
    const float kf = __fsub_rn(t, 12582912.f);
    const F2 f = two_sum(__fmaf_rn(kf, -1.0f / 1024.f, xh), xl);   // the first term is exact
    const float fh = f.hi;
    const float poly = __fmaf_rn(__fmaf_rn(fh, 1.0f / 24.0f, -1.0f / 6.0f), fh, 0.5f);
    const float q = __fmul_rn(__fmul_rn(fh, fh), poly);
    const F2 omf = fast_two_sum(1.0f, -fh);
    const F2 ef = fast_two_sum(omf.hi, __fadd_rn(__fsub_rn(omf.lo, f.lo), q));
    return mul(mul(f2(tab[k >> 10]), f2(tab[kExpHi + (k & 1023)])), ef);
}

// ------------------------------------------------------------------ pair policies
// Fp32: 4 pi K terms, d = x - y, s = 1/r^3, E = e^{-kappa r}, E1 = E (1 + kappa r):
//   4pi K11 = (d.n_y) s (1 - (eps_E/eps_I) E1)
//   4pi K12 = (1 - E)/r
//   4pi K22 = -(d.n_x) s (1 - (eps_I/eps_E) E1)
//   4pi K21 = s [ (1 - E1) n_x.n_y - (3 - E (3 + 3 kappa r + kappa^2 r^2)) (d.n_x)(d.n_y)/r^2 ]
// and acc1 += a K11 - b K12, acc2 += a K21 - b K22.
struct Fp32Policy {
    using Src = float4;
    static constexpr int kVec = 2;    // Src per node
    static constexpr int kTile = 256; // nodes per tile (8 KB)
    static constexpr bool kTables = false;
    struct Tgt {
        float px, py, pz, qx, qy, qz;
    };
    struct Acc {
        float a1, a2;
    };
    __device__ static Tgt load(const Src* src, int t) {
        const float4 a = src[2 * t], b = src[2 * t + 1];
        return Tgt{a.x, a.y, a.z, b.x, b.y, b.z};
    }
    __device__ static void zero(Acc& c) { c.a1 = c.a2 = 0.f; }
    __device__ static void fold(const Acc& c, double& s1, double& s2) {
        s1 += (double)c.a1;
        s2 += (double)c.a2;
    }
    template <bool kMask>
    __device__ static void pair(const Tgt& T, const Src* S, const PairConsts& k, const float2*, Acc& acc, bool ex) {
        float4 pa = S[0], nb = S[1];
        if (kMask && ex) {   // excluded correction pair: a zero-weight source at distance 1
            pa = make_float4(T.px + 1.f, T.py, T.pz, 0.f);
            nb.w = 0.f;
        }
        const float dx = T.px - pa.x, dy = T.py - pa.y, dz = T.pz - pa.z;
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float rinv = rsqrt_sfu(r2);
        const float r = r2 * rinv;
        const float E = ex2_sfu(k.kl2f * r);
        const float kr = k.kappaf * r;
        const float E1 = fmaf(E, kr, E);
        const float dny = fmaf(dz, nb.z, fmaf(dy, nb.y, dx * nb.x));
        const float dnx = fmaf(dz, T.qz, fmaf(dy, T.qy, dx * T.qx));
        const float nn = fmaf(T.qz, nb.z, fmaf(T.qy, nb.y, T.qx * nb.x));
        const float rinv2 = rinv * rinv;
        const float s = rinv2 * rinv;
        const float as = pa.w * s, bs = nb.w * s;
        const float t1 = fmaf(-k.c1f, E1, 1.f);
        acc.a1 = fmaf(as, dny * t1, acc.a1);
        const float om = fmaf(-rinv, E, rinv);
        acc.a1 = fmaf(-nb.w, om, acc.a1);
        const float t2 = fmaf(-k.c2f, E1, 1.f);
        acc.a2 = fmaf(bs, dnx * t2, acc.a2);
        const float u = 1.f - E1;
        const float q = fmaf(kr, kr + 3.f, 3.f);
        const float t3 = fmaf(-E, q, 3.f);
        const float B = t3 * dnx * dny * rinv2;
        acc.a2 = fmaf(as, fmaf(u, nn, -B), acc.a2);
    }
};

struct Fp64Policy {
    using Src = double4;
    static constexpr int kVec = 2;
    static constexpr int kTile = 128;   // 8 KB
    static constexpr bool kTables = false;
    struct Tgt {
        double px, py, pz, qx, qy, qz;
    };
    struct Acc {
        double a1, a2;
    };
    __device__ static Tgt load(const Src* src, int t) {
        const double4 a = src[2 * t], b = src[2 * t + 1];
        return Tgt{a.x, a.y, a.z, b.x, b.y, b.z};
    }
    __device__ static void zero(Acc& c) { c.a1 = c.a2 = 0.0; }
    __device__ static void fold(const Acc& c, double& s1, double& s2) {
        s1 += c.a1;
        s2 += c.a2;
    }
    template <bool kMask>
    __device__ static void pair(const Tgt& T, const Src* S, const PairConsts& k, const float2*, Acc& acc, bool ex) {
        double4 pa = S[0], nb = S[1];
        if (kMask && ex) {
            pa = make_double4(T.px + 1.0, T.py, T.pz, 0.0);
            nb.w = 0.0;
        }
        const double dx = T.px - pa.x, dy = T.py - pa.y, dz = T.pz - pa.z;
        const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        const double rinv = rsqrt(r2);
        const double r = r2 * rinv;
        const double E = exp(-k.kappa * r);
        const double kr = k.kappa * r;
        const double E1 = fma(E, kr, E);
        const double dny = fma(dz, nb.z, fma(dy, nb.y, dx * nb.x));
        const double dnx = fma(dz, T.qz, fma(dy, T.qy, dx * T.qx));
        const double nn = fma(T.qz, nb.z, fma(T.qy, nb.y, T.qx * nb.x));
        const double rinv2 = rinv * rinv;
        const double s = rinv2 * rinv;
        const double as = pa.w * s, bs = nb.w * s;
        const double t1 = fma(-k.c1, E1, 1.0);
        acc.a1 = fma(as, dny * t1, acc.a1);
        const double om = fma(-rinv, E, rinv);
        acc.a1 = fma(-nb.w, om, acc.a1);
        const double t2 = fma(-k.c2, E1, 1.0);
        acc.a2 = fma(bs, dnx * t2, acc.a2);
        const double u = 1.0 - E1;
        const double q = fma(kr, kr + 3.0, 3.0);
        const double t3 = fma(-E, q, 3.0);
        const double B = t3 * dnx * dny * rinv2;
        acc.a2 = fma(as, fma(u, nn, -B), acc.a2);
    }
};

// Source node = 4 float4: {P.hi, a.hi} {P.lo, a.lo} {n.hi, b.hi} {n.lo, b.lo}.
struct Df64Policy {
    using Src = float4;
    static constexpr int kVec = 4;
    static constexpr int kTile = 128;   // 8 KB
    static constexpr bool kTables = true;
    struct Tgt {
        F2 px, py, pz, qx, qy, qz;
    };
    struct Acc {
        F2 a1, a2;
    };
    __device__ static Tgt load(const Src* src, int t) {
        const float4 a = src[4 * t], b = src[4 * t + 1], c = src[4 * t + 2], d = src[4 * t + 3];
        return Tgt{F2{a.x, b.x}, F2{a.y, b.y}, F2{a.z, b.z}, F2{c.x, d.x}, F2{c.y, d.y}, F2{c.z, d.z}};
    }
    __device__ static void zero(Acc& c) { c.a1 = c.a2 = F2{0.f, 0.f}; }
    __device__ static void fold(const Acc& c, double& s1, double& s2) {
        s1 += (double)c.a1.hi + (double)c.a1.lo;
        s2 += (double)c.a2.hi + (double)c.a2.lo;
    }
    template <bool kMask>
    __device__ static void pair(const Tgt& T, const Src* S, const PairConsts& k, const float2* tab, Acc& acc,
                                bool ex) {
        const float4 s0 = S[0], s1 = S[1], s2 = S[2], s3 = S[3];
        F2 Px{s0.x, s1.x}, Py{s0.y, s1.y}, Pz{s0.z, s1.z}, A{s0.w, s1.w};
        const F2 Nx{s2.x, s3.x}, Ny{s2.y, s3.y}, Nz{s2.z, s3.z};
        F2 Bw{s2.w, s3.w};
        if (kMask && ex) {
            Px = F2{T.px.hi + 1.f, T.px.lo};
            Py = T.py;
            Pz = T.pz;
            A = Bw = F2{0.f, 0.f};
        }
        const F2 dx = sub(T.px, Px), dy = sub(T.py, Py), dz = sub(T.pz, Pz);
        const F2 r2 = dot3(dx, dy, dz, dx, dy, dz);
        const F2 rinv = rsqrt_ff(r2);
        const F2 r = mul(r2, rinv);
        const F2 kr = mul(f2(k.kappad), r);
        const F2 E = exp_neg_ff(kr, tab);
        const F2 E1 = mul(E, add_f(kr, 1.f));
        const F2 dny = dot3(dx, dy, dz, Nx, Ny, Nz);
        const F2 dnx = dot3(dx, dy, dz, T.qx, T.qy, T.qz);
        const F2 nn = dot3(T.qx, T.qy, T.qz, Nx, Ny, Nz);
        const F2 rinv2 = mul(rinv, rinv);
        const F2 s = mul(rinv2, rinv);
        const F2 as = mul(A, s), bs = mul(Bw, s);
        const F2 t1 = add_f(neg(mul(E1, f2(k.c1d))), 1.f);
        acc.a1 = add(acc.a1, mul(as, mul(dny, t1)));
        const F2 om = mul(rinv, add_f(neg(E), 1.f));
        acc.a1 = sub(acc.a1, mul(Bw, om));
        const F2 t2 = add_f(neg(mul(E1, f2(k.c2d))), 1.f);
        acc.a2 = add(acc.a2, mul(bs, mul(dnx, t2)));
        const F2 u = add_f(neg(E1), 1.f);
        const F2 q = add_f(mul(kr, add_f(kr, 3.f)), 3.f);
        const F2 t3 = add_f(neg(mul(E, q)), 3.f);
        const F2 Bt = mul(mul(t3, mul(dnx, dny)), rinv2);
        acc.a2 = add(acc.a2, mul(as, sub(mul(u, nn), Bt)));
    }
};

template <typename Policy, int R>
__global__ void __launch_bounds__(kThreads) pair_kernel(const typename Policy::Src* __restrict__ src, int M,
                                                        const int32_t* __restrict__ eptr,
                                                        const int32_t* __restrict__ excl, int src_per_split,
                                                        double* __restrict__ partial, PairConsts kc,
                                                        int* __restrict__ err) {
    using Src = typename Policy::Src;
    constexpr int TILE = Policy::kTile;
    constexpr int VEC = Policy::kVec;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Src* ring = reinterpret_cast<Src*>(smem_raw);   // [2][TILE][VEC]
    float2* tab = reinterpret_cast<float2*>(smem_raw + 2 * TILE * VEC * sizeof(Src));
    __shared__ __align__(8) uint64_t bar[2];

    const int tid = threadIdx.x;
    const int j_begin = blockIdx.y * src_per_split;
    const int j_end = min(M, j_begin + src_per_split);
    const int ntiles = (j_end > j_begin) ? (j_end - j_begin + TILE - 1) / TILE : 0;

    typename Policy::Tgt tg[R];
    double s1[R], s2[R];
    int ti[R], epos[R], eend[R], enext[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        ti[r] = blockIdx.x * (kThreads * R) + r * kThreads + tid;
        const int t = min(ti[r], M - 1);
        tg[r] = Policy::load(src, t);
        s1[r] = 0.0;
        s2[r] = 0.0;
        int e = eptr[t], ee = eptr[t + 1];
        while (e < ee && excl[e] < j_begin) ++e;
        epos[r] = e;
        eend[r] = ee;
        enext[r] = (e < ee) ? excl[e] : INT_MAX;
    }
    if constexpr (Policy::kTables) {
        for (int q = tid; q < kExpHi + kExpLo; q += kThreads) tab[q] = kc.exp_tab[q];
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
        const uint32_t bytes = (uint32_t)(n * VEC * sizeof(Src));
        Src* dst = ring + (k & 1) * TILE * VEC;
        fence_proxy_async();
        mbar_expect_tx(&bar[k & 1], bytes);
        bulk_load(dst, src + (size_t)VEC * j0, bytes, &bar[k & 1]);
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
        const Src* tile = ring + (k & 1) * TILE * VEC;
        const int j0 = j_begin + k * TILE;
        const int n = min(TILE, j_end - j0);
        bool need = false;
#pragma unroll
        for (int r = 0; r < R; ++r) need |= (enext[r] < j0 + n);
        typename Policy::Acc acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) Policy::zero(acc[r]);
        if (!__any_sync(0xffffffffu, need)) {
#pragma unroll 2
            for (int q = 0; q < n; ++q) {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    Policy::template pair<false>(tg[r], tile + q * VEC, kc, tab, acc[r], false);
            }
        } else {
            for (int q = 0; q < n; ++q) {
                const int j = j0 + q;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const bool ex = (j == enext[r]);
                    if (ex) {
                        ++epos[r];
                        enext[r] = (epos[r] < eend[r]) ? excl[epos[r]] : INT_MAX;
                    }
                    Policy::template pair<true>(tg[r], tile + q * VEC, kc, tab, acc[r], ex);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) Policy::fold(acc[r], s1[r], s2[r]);
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

// a = h^3 W rho1/(4 pi), b = h^3 W rho2/(4 pi) into the weight slots of the packed sources
__global__ void pack_kernel(const double* __restrict__ x, const double* __restrict__ W, int64_t M, double scale,
                            float4* __restrict__ s32, double4* __restrict__ s64, float4* __restrict__ sdf) {
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
    if (sdf) {
        const float ah = (float)a, bh = (float)b;
        sdf[4 * j].w = ah;
        sdf[4 * j + 1].w = (float)(a - (double)ah);
        sdf[4 * j + 2].w = bh;
        sdf[4 * j + 3].w = (float)(b - (double)bh);
    }
}

// y = diag + fixed-order sum of the split partials + correction (FP64)
__global__ void finish_kernel(int64_t M, int S, const double* __restrict__ partial, const double* __restrict__ x,
                              double* __restrict__ y, const double* __restrict__ W, const int32_t* __restrict__ ptr,
                              const int32_t* __restrict__ node, const double* __restrict__ w, int64_t E,
                              double lam1, double lam2, double h2, double h3) {
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
        c1 += Wm * (h2 * w[e] * r1 - h3 * w[3 * E + e] * r2);
        c2 += Wm * (h2 * w[E + e] * r1 - h2 * w[2 * E + e] * r2);
    }
    y[i] = lam1 * x[i] + s1 + c1;
    y[M + i] = lam2 * x[M + i] + s2 + c2;
}

template <typename Policy, int R>
int launch_pairs(ctr_ibim* s, const typename Policy::Src* src, const PairPlan& p, const PairConsts& kc) {
    const size_t smem = 2 * Policy::kTile * Policy::kVec * sizeof(typename Policy::Src) +
                        (Policy::kTables ? (kExpHi + kExpLo) * sizeof(float2) : 0);
    dim3 grid(p.target_blocks, p.splits);
    pair_kernel<Policy, R><<<grid, kThreads, smem, s->stream>>>(src, (int)s->M, s->corr_ptr.as<int32_t>(),
                                                               s->excl.as<int32_t>(), p.src_per_split,
                                                               s->partial.as<double>(), kc, s->err.as<int>());
    CTR_LAUNCHED();
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

float2 split_ff(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

// float-float table of e^{-k} (k < 64) and e^{-k/1024} (k < 1024), one per device
int exp_table(ctr_ibim* s, const float2** out) {
    static DevBuf tabs[64];
    static bool ready[64] = {false};
    const int dev = s->device;
    if (dev < 0 || dev >= 64) return fail(CTR_ERR_INVALID, "device index");
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

int plan_pairs(ctr_ibim* s) {
    int sms = 0;
    CTR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
    int R32 = s->opt.tile_targets;
    if (R32 != 1 && R32 != 2 && R32 != 4) R32 = 2;
    s->plan32 = make_plan(s->M, R32, Fp32Policy::kTile, sms);
    s->plan64 = make_plan(s->M, 1, Fp64Policy::kTile, sms);
    s->plandf = make_plan(s->M, 1, Df64Policy::kTile, sms);
    const int S = std::max(s->plan32.splits, std::max(s->plan64.splits, s->plandf.splits));
    CTR_TRY(s->partial.alloc(sizeof(double) * 2 * (size_t)S * s->M));
    CTR_TRY(s->srcdf.alloc(sizeof(float4) * 4 * (size_t)s->M));
    df_static_kernel<<<grid_for(s->M, 256), 256, 0, s->stream>>>(s->na, s->M, s->srcdf.as<float4>());
    CTR_LAUNCHED();
    return CTR_OK;
}

int apply_operator(ctr_ibim* s, const double* d_x, double* d_y, int precision) {
    const int64_t M = s->M;
    cudaStream_t st = s->stream;
    const double scale = s->h * s->h * s->h / (4.0 * kPi);
    float4* s32 = (precision == CTR_FP32_REFINE) ? s->src32.as<float4>() : nullptr;
    double4* s64 = (precision == CTR_FP64) ? s->src64.as<double4>() : nullptr;
    float4* sdf = (precision == CTR_DF64) ? s->srcdf.as<float4>() : nullptr;
    pack_kernel<<<grid_for(M, 256), 256, 0, st>>>(d_x, s->na.W, M, scale, s32, s64, sdf);
    CTR_LAUNCHED();
    PairConsts kc;
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
    kc.exp_tab = nullptr;
    const PairPlan* p = nullptr;
    if (precision == CTR_FP32_REFINE) {
        p = &s->plan32;
        switch (p->R) {
            case 1: CTR_TRY((launch_pairs<Fp32Policy, 1>(s, s32, *p, kc))); break;
            case 4: CTR_TRY((launch_pairs<Fp32Policy, 4>(s, s32, *p, kc))); break;
            default: CTR_TRY((launch_pairs<Fp32Policy, 2>(s, s32, *p, kc))); break;
        }
    } else if (precision == CTR_DF64) {
        p = &s->plandf;
        CTR_TRY(exp_table(s, &kc.exp_tab));
        CTR_TRY((launch_pairs<Df64Policy, 1>(s, sdf, *p, kc)));
    } else {
        p = &s->plan64;
        CTR_TRY((launch_pairs<Fp64Policy, 1>(s, s64, *p, kc)));
    }
    const double h2 = s->h * s->h;
    const double h3 = s->h * s->h * s->h;
    finish_kernel<<<grid_for(M, 256), 256, 0, st>>>(M, p->splits, s->partial.as<double>(), d_x, d_y, s->na.W,
                                                   s->corr_ptr.as<int32_t>(), s->corr_node.as<int32_t>(),
                                                   s->corr_w.as<double>(), s->E,
                                                   0.5 * (1.0 + s->eps_out / s->eps_in),
                                                   0.5 * (1.0 + s->eps_in / s->eps_out), h2, h3);
    CTR_LAUNCHED();
    return CTR_OK;
}

}  // namespace ctr

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
    PairPlan p = make_plan(M, 2, Fp32Policy::kTile, sms);
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
    const size_t smem = 2 * Fp32Policy::kTile * Fp32Policy::kVec * sizeof(float4);
    dim3 grid(p.target_blocks, p.splits);
    pair_kernel<Fp32Policy, 2><<<grid, kThreads, smem, st>>>(src, (int)M, eptr, excl, p.src_per_split, partial, kc,
                                                             err);
    CTR_LAUNCHED();
    *splits_out = p.splits;
    return CTR_OK;
}

}  // namespace ctr
