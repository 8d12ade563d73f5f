// Dense pair-sum core shared by the single-system operator (pairsum.cu) and
// the multi-slot engine (engine.cu): kernel constants, bulk-copy/mbarrier
// helpers, float-float arithmetic, the three pair policies and one work item
// of the tiled pair sum.  Internal to the library.
#pragma once

#include "common.cuh"

namespace ctr {
namespace pk {

constexpr int kThreads = 256;
constexpr uint32_t kWaitLimit = 1u << 22;   // default polls of a bounded mbarrier wait
constexpr int kExpHi = 64;      // e^{-k}, k = 0..63
constexpr int kExpLo = 1024;    // e^{-k/1024}, k = 0..1023

struct PairConsts {
    float c1f, c2f, kappaf, kl2f;    // eps_E/eps_I, eps_I/eps_E, kappa, -kappa log2(e)
    double c1, c2, kappa;
    float2 c1d, c2d, kappad;         // float-float copies
    const float2* exp_tab;           // [kExpHi + kExpLo] float-float, global
    // the FP32 values duplicated into both halves of a 64-bit word (f32x2 operands)
    unsigned long long one2, mone2, three2, mthree2, c1x2, nc1x2, c2x2, nc2x2, kap2, kl2x2;
    uint32_t wait_limit;             // polls of a source-tile wait before the block gives up
    uint32_t pad_;
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
// Bounded wait: false after `limit` polls (each poll may suspend briefly).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = kWaitLimit) {
    for (uint32_t it = 0; it < limit; ++it)
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

// ------------------------------------------------------------------ f32x2 arithmetic
// Two FP32 values in one 64-bit register pair, one IEEE round-to-nearest operation per half
// (add/sub/mul/fma.rn.f32x2): half the issue slots of two scalar instructions.
using u64 = unsigned long long;
__device__ __forceinline__ u64 pk2(float a, float b) {
    u64 d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ void up2(u64 v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {   // a * b + c
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 rsqrt2(u64 v) {
    float a, b;
    up2(v, a, b);
    return pk2(rsqrt_sfu(a), rsqrt_sfu(b));
}
__device__ __forceinline__ u64 ex2_2(u64 v) {
    float a, b;
    up2(v, a, b);
    return pk2(ex2_sfu(a), ex2_sfu(b));
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
// Lazy forms for the symmetric pair terms.  A lazy value is hi + lo with |lo|
// a few ulp(hi) instead of at most ulp(hi)/2: it carries the same value to the
// same accuracy, and a product of two lazy values loses only the dropped
// lo * lo term (relative 2^-44 or less).  Results that meet a cancellation
// (differences, 1 - E, 3 - E q) go through the normalised add, whose two_sum
// is exact for any inputs.
__device__ __forceinline__ F2 mull(F2 a, F2 b) {
    const F2 p = two_prod(a.hi, b.hi);
    return F2{p.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo))};
}
// acc += x without renormalising acc: exact two_sum of the high parts, plain sum of the low parts
__device__ __forceinline__ void acc_add(F2& acc, F2 x) {
    const F2 s = two_sum(acc.hi, x.hi);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, x.lo));
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
// The same with lazy products (for the symmetric pair terms).
__device__ __forceinline__ F2 exp_neg_ffl(F2 x, const float2* tab) {
    float xh = x.hi, xl = x.lo;
    if (xh > 63.9f) {
        xh = 63.9f;
        xl = 0.f;
    }
    const float t = __fmaf_rn(xh, 1024.f, 12582912.f);
    const int k = min(max(__float_as_int(t) - 0x4B400000, 0), kExpHi * kExpLo - 1);
    const float kf = __fsub_rn(t, 12582912.f);
    const F2 f = two_sum(__fmaf_rn(kf, -1.0f / 1024.f, xh), xl);
    const float fh = f.hi;
    const float poly = __fmaf_rn(__fmaf_rn(fh, 1.0f / 24.0f, -1.0f / 6.0f), fh, 0.5f);
    const float q = __fmul_rn(__fmul_rn(fh, fh), poly);
    const F2 omf = fast_two_sum(1.0f, -fh);
    const F2 ef = fast_two_sum(omf.hi, __fadd_rn(__fsub_rn(omf.lo, f.lo), q));
    return mull(mull(f2(tab[k >> 10]), f2(tab[kExpHi + (k & 1023)])), ef);
}

// ------------------------------------------------------------------ exact node accumulators
// The dense sum's partial results (an item's target sums, a symmetric tile's source sums, a far item's
// sums) are added into per-node accumulators in whatever order the blocks run.  To keep the result
// independent of that order, each contribution v (FP64) is turned into the integer round(|v| 2^kFxFrac)
// and added exactly: the integer's 32-bit chunks go to 64-bit words by atomic addition (fewer than 2^31
// contributions per word cannot carry out of it), positive and negative contributions to separate sets
// of kFxChunks words, so a contribution touches at most the three words its 53 significant bits span.
// Reading a node's sum propagates the carries, subtracts the two sets and rounds once to FP64.
// Range: |v| < 2^(32 kFxChunks - kFxFrac) = 2^72; below 2^-kFxFrac a contribution is rounded to a
// multiple of 2^-kFxFrac = 7.5e-37.  A non-finite or out-of-range contribution marks the node
// (its last word), and the node then reads as NaN, as an FP64 sum of such a term would.
// Layout: word k of sign set g (0 positive, 1 negative) of sum c (0, 1) of node position p at
// acc[((2 c + g) kFxChunks + k) * stride + p], the mark at acc[4 kFxChunks * stride + p]:
// kFxWords 64-bit words per node.
constexpr int kFxChunks = 6;
constexpr int kFxFrac = 120;
constexpr int kFxWords = 4 * kFxChunks + 1;

__device__ __forceinline__ void fx_add(unsigned long long* __restrict__ acc, int64_t stride, int c, double v) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((bits >> 52) & 0x7ff);
    if (ex == 0x7ff) {   // not finite
        atomicOr(acc + (int64_t)(4 * kFxChunks) * stride, 1ull);
        return;
    }
    unsigned long long m = bits & ((1ull << 52) - 1);
    if (ex != 0) m |= 1ull << 52;
    if (m == 0) return;
    int sh = (ex != 0 ? ex - 1075 : -1074) + kFxFrac;   // |v| 2^kFxFrac = m 2^sh
    if (sh < 0) {                                       // below the resolution: round to nearest
        if (sh < -60) return;
        m = (m + (1ull << (-sh - 1))) >> (-sh);
        sh = 0;
        if (m == 0) return;
    }
    if (sh + 53 > 32 * kFxChunks) {   // out of range
        atomicOr(acc + (int64_t)(4 * kFxChunks) * stride, 1ull);
        return;
    }
    unsigned long long* base = acc + (int64_t)((2 * c + (int)(bits >> 63)) * kFxChunks) * stride;
    // m 2^sh spans the 32-bit chunks k0 .. k0 + 2 (m < 2^53)
    const int k0 = sh >> 5, r = sh & 31;
    const unsigned long long lo = m << r;                       // bits 0..63 of m 2^r
    const unsigned long long hi = r ? (m >> (64 - r)) : 0ull;   // bits 64.. (m 2^r < 2^85)
    const unsigned long long ch[3] = {lo & 0xffffffffull, lo >> 32, hi};
#pragma unroll
    for (int q = 0; q < 3; ++q)
        if (ch[q] != 0 && k0 + q < kFxChunks) atomicAdd(base + (int64_t)(k0 + q) * stride, ch[q]);
}

// One sum (c) of the node at acc (stride as in fx_add), rounded to FP64: carries of both sign sets,
// positive minus negative, one rounding.  The node's words of that sum are cleared when `clear`.
__device__ __forceinline__ double fx_read_one(unsigned long long* __restrict__ acc, int64_t stride, int c,
                                              bool clear) {
    uint32_t D[kFxChunks + 1];
    unsigned long long cp = 0, cn = 0;
    long long borrow = 0;
#pragma unroll
    for (int k = 0; k <= kFxChunks; ++k) {
        unsigned long long tp = cp, tn = cn;
        if (k < kFxChunks) {
            unsigned long long* ap = acc + (int64_t)((2 * c) * kFxChunks + k) * stride;
            unsigned long long* an = acc + (int64_t)((2 * c + 1) * kFxChunks + k) * stride;
            tp += *ap;
            tn += *an;
            if (clear) *ap = *an = 0ull;
        }
        cp = tp >> 32;
        cn = tn >> 32;
        const long long t = (long long)(tp & 0xffffffffull) - (long long)(tn & 0xffffffffull) - borrow;
        D[k] = (uint32_t)t;
        borrow = t < 0 ? 1 : 0;
    }
    const bool neg = borrow != 0;
    if (neg) {   // two's complement of the chunk string
        unsigned long long carry = 1;
#pragma unroll
        for (int k = 0; k <= kFxChunks; ++k) {
            const unsigned long long t = (unsigned long long)(uint32_t)~D[k] + carry;
            D[k] = (uint32_t)t;
            carry = t >> 32;
        }
    }
    double v = 0.0;
#pragma unroll
    for (int k = kFxChunks; k >= 0; --k) v = fma(v, 4294967296.0, (double)D[k]);
    v = ldexp(v, -kFxFrac);
    return neg ? -v : v;
}

// Both sums of the node at acc (NaN when a contribution was marked); clears the node's words when `clear`.
__device__ __forceinline__ void fx_read(unsigned long long* __restrict__ acc, int64_t stride, bool clear, double& s1,
                                        double& s2) {
    unsigned long long* mark = acc + (int64_t)(4 * kFxChunks) * stride;
    const bool bad = *mark != 0ull;
    s1 = fx_read_one(acc, stride, 0, clear);
    s2 = fx_read_one(acc, stride, 1, clear);
    if (clear) *mark = 0ull;
    if (bad) s1 = s2 = __longlong_as_double(0x7ff8000000000000ll);
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
    static constexpr int kSymStep = 32;   // symmetric chunk fully unrolled
    struct Tgt {
        float px, py, pz, qx, qy, qz, wa, wb;
    };
    struct Acc {
        float a1, a2;
    };
    using JAcc = Acc;
    using JAccR = Acc;                  // source-side sums while a source meets the thread's targets
    static constexpr int kPack = 1;     // targets per thread slot
    __device__ static JAcc jfinal(const JAccR& a) { return a; }   // source-side (transposed) sums of a symmetric tile
    __device__ static Tgt load(const Src* src, int t) {
        const float4 a = src[2 * t], b = src[2 * t + 1];
        return Tgt{a.x, a.y, a.z, b.x, b.y, b.z, a.w, b.w};
    }
    __device__ static void clear_w(Tgt& t) { t.wa = t.wb = 0.f; }
    __device__ static void zero(Acc& c) { c.a1 = c.a2 = 0.f; }
    __device__ static void fold(const Acc& c, double& s1, double& s2) {
        s1 += (double)c.a1;
        s2 += (double)c.a2;
    }
    __device__ static JAcc jadd(const JAcc& x, const JAcc& y) { return JAcc{x.a1 + y.a1, x.a2 + y.a2}; }
    __device__ static JAcc jshfl_xor(const JAcc& x, int m) {
        return JAcc{__shfl_xor_sync(0xffffffffu, x.a1, m), __shfl_xor_sync(0xffffffffu, x.a2, m)};
    }
    template <bool kMask>
    __device__ static void pair(const Tgt& T, const Src* S, const PairConsts& k, const float2*, Acc& acc, const bool* exv) {
        const bool ex = exv[0];
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

// Packed FP32: the Fp32 terms for two targets at once (lanes of f32x2 operations).  A thread slot
// holds targets a, b (lanes x, y); a source node is stored with every value duplicated,
// {(x,x),(y,y)} {(z,z),(a,a)} {(nx,nx),(ny,ny)} {(nz,nz),(-b,-b)} (64 B), so a broadcast
// shared-memory load gives ready operands.  Signs are arranged so that every step is a plain
// add/sub/mul or a*b + c (the f32x2 forms take no negated operands):
//   t1 = 1 - c1 E1, t1n = -t1, t2 = 1 - c2 E1, t2n = -t2, om = (1 - E)/r, u = 1 - E1,
//   t3n = E q - 3, Bn = t3n (d.n_x)(d.n_y)/r^2, X = u n_x.n_y + Bn,
//   target rows: a1 += a s (d.n_y) t1 + (-b) om,   a2 += (-b s)(d.n_x) t2n + a s X;
//   source rows: a1 += ((-a_t) s)(d.n_x) t1 + (-b_t) om,
//                -a2 += ((-b_t) s)(d.n_y) t2n + ((-a_t) s) X   (negated; jfinal restores the sign).
struct Fp32x2Policy {
    using Src = ulonglong2;
    static constexpr int kVec = 4;      // Src per node (64 B)
    static constexpr int kTile = 256;   // nodes per tile (16 KB)
    static constexpr bool kTables = false;
    static constexpr int kSymStep = 32;
    static constexpr int kPack = 2;
    struct Tgt {
        u64 px, py, pz, qx, qy, qz, nwa, nwb;
    };
    struct Acc {
        u64 a1, a2;
    };
    struct JAcc {
        float a1, a2;
    };
    using JAccR = Acc;
    __device__ static JAcc jfinal(const JAccR& j) {
        float x0, x1, y0, y1;
        up2(j.a1, x0, x1);
        up2(j.a2, y0, y1);
        return JAcc{x0 + x1, -(y0 + y1)};
    }
    __device__ static Tgt load_pack(const Src* src, int M, const int* ti) {
        float v[2][8];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int t = min(ti[h], M - 1);
            const ulonglong2 a = src[4 * t], b = src[4 * t + 1], c = src[4 * t + 2], d = src[4 * t + 3];
            float dummy;
            up2(a.x, v[h][0], dummy);
            up2(a.y, v[h][1], dummy);
            up2(b.x, v[h][2], dummy);
            up2(b.y, v[h][6], dummy);   // a
            up2(c.x, v[h][3], dummy);
            up2(c.y, v[h][4], dummy);
            up2(d.x, v[h][5], dummy);
            up2(d.y, v[h][7], dummy);   // -b
            v[h][6] = -v[h][6];                        // -a
            if (ti[h] >= M) v[h][6] = v[h][7] = 0.f;   // a padding target adds nothing to the sources
        }
        return Tgt{pk2(v[0][0], v[1][0]), pk2(v[0][1], v[1][1]), pk2(v[0][2], v[1][2]), pk2(v[0][3], v[1][3]),
                   pk2(v[0][4], v[1][4]), pk2(v[0][5], v[1][5]), pk2(v[0][6], v[1][6]), pk2(v[0][7], v[1][7])};
    }
    __device__ static void zero(Acc& c) { c.a1 = c.a2 = 0ull; }
    __device__ static void zero(JAcc& c) { c.a1 = c.a2 = 0.f; }
    __device__ static void fold_pack(const Acc& c, double* s1, double* s2) {
        float x0, x1, y0, y1;
        up2(c.a1, x0, x1);
        up2(c.a2, y0, y1);
        s1[0] += (double)x0;
        s1[1] += (double)x1;
        s2[0] += (double)y0;
        s2[1] += (double)y1;
    }
    __device__ static void fold(const JAcc& c, double& s1, double& s2) {
        s1 += (double)c.a1;
        s2 += (double)c.a2;
    }
    __device__ static JAcc jadd(const JAcc& x, const JAcc& y) { return JAcc{x.a1 + y.a1, x.a2 + y.a2}; }
    __device__ static JAcc jshfl_xor(const JAcc& x, int m) {
        return JAcc{__shfl_xor_sync(0xffffffffu, x.a1, m), __shfl_xor_sync(0xffffffffu, x.a2, m)};
    }
    // The terms shared by both orientations for the two targets of T and source S.
    struct Common {
        u64 dnx, dny, om, t1, t2n, X, s;
    };
    __device__ static Common common(const Tgt& T, u64 Sx, u64 Sy, u64 Sz, u64 Nx, u64 Ny, u64 Nz,
                                    const PairConsts& k) {
        const u64 dx = sub2(T.px, Sx), dy = sub2(T.py, Sy), dz = sub2(T.pz, Sz);
        const u64 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
        const u64 rinv = rsqrt2(r2);
        const u64 r = mul2(r2, rinv);
        const u64 E = ex2_2(mul2(k.kl2x2, r));
        const u64 kr = mul2(k.kap2, r);
        const u64 E1 = fma2(E, kr, E);
        Common c;
        c.dny = fma2(dz, Nz, fma2(dy, Ny, mul2(dx, Nx)));
        c.dnx = fma2(dz, T.qz, fma2(dy, T.qy, mul2(dx, T.qx)));
        const u64 nn = fma2(T.qz, Nz, fma2(T.qy, Ny, mul2(T.qx, Nx)));
        const u64 rinv2 = mul2(rinv, rinv);
        c.s = mul2(rinv2, rinv);
        c.t1 = fma2(k.nc1x2, E1, k.one2);
        c.t2n = fma2(k.c2x2, E1, k.mone2);
        c.om = mul2(rinv, sub2(k.one2, E));
        const u64 u = sub2(k.one2, E1);
        const u64 q = fma2(kr, add2(kr, k.three2), k.three2);
        const u64 t3n = fma2(E, q, k.mthree2);
        const u64 Bn = mul2(mul2(mul2(t3n, c.dnx), c.dny), rinv2);
        c.X = fma2(u, nn, Bn);
        return c;
    }
    __device__ static void target_terms(const Common& c, u64 Sa, u64 Snb, Acc& acc) {
        const u64 as = mul2(Sa, c.s), nbs = mul2(Snb, c.s);
        acc.a1 = fma2(mul2(as, c.dny), c.t1, acc.a1);
        acc.a1 = fma2(Snb, c.om, acc.a1);
        acc.a2 = fma2(mul2(nbs, c.dnx), c.t2n, acc.a2);
        acc.a2 = fma2(as, c.X, acc.a2);
    }
    template <bool kMask>
    __device__ static void pair(const Tgt& T, const Src* S, const PairConsts& k, const float2*, Acc& acc,
                                const bool* ex) {
        const ulonglong2 v0 = S[0], v1 = S[1], v2 = S[2], v3 = S[3];
        u64 Sx = v0.x, Sy = v0.y, Sz = v1.x, Sa = v1.y, Snb = v3.y;
        if (kMask && (ex[0] || ex[1])) {   // excluded correction pair: a zero-weight source at distance 1
            float x[2], y[2], z[2], a[2], b[2], tx[2], ty[2], tz[2];
            up2(Sx, x[0], x[1]);
            up2(Sy, y[0], y[1]);
            up2(Sz, z[0], z[1]);
            up2(Sa, a[0], a[1]);
            up2(Snb, b[0], b[1]);
            up2(T.px, tx[0], tx[1]);
            up2(T.py, ty[0], ty[1]);
            up2(T.pz, tz[0], tz[1]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (ex[h]) {
                    x[h] = tx[h] + 1.f;
                    y[h] = ty[h];
                    z[h] = tz[h];
                    a[h] = b[h] = 0.f;
                }
            }
            Sx = pk2(x[0], x[1]);
            Sy = pk2(y[0], y[1]);
            Sz = pk2(z[0], z[1]);
            Sa = pk2(a[0], a[1]);
            Snb = pk2(b[0], b[1]);
        }
        const Common c = common(T, Sx, Sy, Sz, v2.x, v2.y, v3.x, k);
        target_terms(c, Sa, Snb, acc);
    }
    // Both orientations: s is folded once into the factors the two share (s t1, s t2n, s X), which
    // saves one f32x2 operation per pair against forming a s, b s and the targets' (-a) s, (-b) s.
    template <bool kFirst>
    __device__ static void pair_sym(const Tgt& T, const Src* S, const PairConsts& k, const float2*, Acc& acc,
                                    JAccR& ja) {
        const ulonglong2 v0 = S[0], v1 = S[1], v2 = S[2], v3 = S[3];
        const Common c = common(T, v0.x, v0.y, v1.x, v2.x, v2.y, v3.x, k);
        const u64 st1 = mul2(c.s, c.t1), st2n = mul2(c.s, c.t2n), sX = mul2(c.s, c.X);
        const u64 Sa = v1.y, Snb = v3.y;
        acc.a1 = fma2(mul2(Sa, c.dny), st1, acc.a1);
        acc.a1 = fma2(Snb, c.om, acc.a1);
        acc.a2 = fma2(mul2(Snb, c.dnx), st2n, acc.a2);
        acc.a2 = fma2(Sa, sX, acc.a2);
        if constexpr (kFirst) {
            ja.a1 = mul2(mul2(T.nwa, c.dnx), st1);
            ja.a2 = mul2(mul2(T.nwb, c.dny), st2n);   // ja.a2 holds -a2 until jfinal
        } else {
            ja.a1 = fma2(mul2(T.nwa, c.dnx), st1, ja.a1);
            ja.a2 = fma2(mul2(T.nwb, c.dny), st2n, ja.a2);
        }
        ja.a1 = fma2(T.nwb, c.om, ja.a1);
        ja.a2 = fma2(T.nwa, sX, ja.a2);
    }
};

struct Fp64Policy {
    using Src = double4;
    static constexpr int kVec = 2;
    static constexpr int kTile = 128;   // 8 KB
    static constexpr bool kTables = false;
    static constexpr int kSymStep = 4;
    struct Tgt {
        double px, py, pz, qx, qy, qz, wa, wb;
    };
    struct Acc {
        double a1, a2;
    };
    using JAcc = Acc;
    using JAccR = Acc;                  // source-side sums while a source meets the thread's targets
    static constexpr int kPack = 1;     // targets per thread slot
    __device__ static JAcc jfinal(const JAccR& a) { return a; }
    __device__ static Tgt load(const Src* src, int t) {
        const double4 a = src[2 * t], b = src[2 * t + 1];
        return Tgt{a.x, a.y, a.z, b.x, b.y, b.z, a.w, b.w};
    }
    __device__ static void clear_w(Tgt& t) { t.wa = t.wb = 0.0; }
    __device__ static void zero(Acc& c) { c.a1 = c.a2 = 0.0; }
    __device__ static void fold(const Acc& c, double& s1, double& s2) {
        s1 += c.a1;
        s2 += c.a2;
    }
    __device__ static JAcc jadd(const JAcc& x, const JAcc& y) { return JAcc{x.a1 + y.a1, x.a2 + y.a2}; }
    __device__ static JAcc jshfl_xor(const JAcc& x, int m) {
        return JAcc{__shfl_xor_sync(0xffffffffu, x.a1, m), __shfl_xor_sync(0xffffffffu, x.a2, m)};
    }
    template <bool kFirst>
    __device__ static void pair_sym(const Tgt& T, const Src* S, const PairConsts& k, const float2*, Acc& acc,
                                    JAcc& ja) {
        const double4 pa = S[0], nb = S[1];
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
        const double om = fma(-rinv, E, rinv);
        const double t2 = fma(-k.c2, E1, 1.0);
        const double u = 1.0 - E1;
        const double q = fma(kr, kr + 3.0, 3.0);
        const double t3 = fma(-E, q, 3.0);
        const double B = t3 * dnx * dny * rinv2;
        const double X = fma(u, nn, -B);
        acc.a1 = fma(as, dny * t1, acc.a1);
        acc.a1 = fma(-nb.w, om, acc.a1);
        acc.a2 = fma(bs, dnx * t2, acc.a2);
        acc.a2 = fma(as, X, acc.a2);
        const double ast = T.wa * s, bst = T.wb * s;
        if constexpr (kFirst) {
            ja.a1 = -ast * (dnx * t1);
            ja.a2 = -bst * (dny * t2);
        } else {
            ja.a1 = fma(-ast, dnx * t1, ja.a1);
            ja.a2 = fma(-bst, dny * t2, ja.a2);
        }
        ja.a1 = fma(-T.wb, om, ja.a1);
        ja.a2 = fma(ast, X, ja.a2);
    }
    template <bool kMask>
    __device__ static void pair(const Tgt& T, const Src* S, const PairConsts& k, const float2*, Acc& acc, const bool* exv) {
        const bool ex = exv[0];
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
    static constexpr int kSymStep = 2;    // ~640 FP32 ops per symmetric pair: two per unrolled step
    struct Tgt {
        F2 px, py, pz, qx, qy, qz, wa, wb;
    };
    struct Acc {
        F2 a1, a2;
    };
    using JAcc = Acc;
    using JAccR = Acc;                  // source-side sums while a source meets the thread's targets
    static constexpr int kPack = 1;     // targets per thread slot
    __device__ static JAcc jfinal(const JAccR& a) { return a; }
    __device__ static Tgt load(const Src* src, int t) {
        const float4 a = src[4 * t], b = src[4 * t + 1], c = src[4 * t + 2], d = src[4 * t + 3];
        return Tgt{F2{a.x, b.x}, F2{a.y, b.y}, F2{a.z, b.z}, F2{c.x, d.x}, F2{c.y, d.y}, F2{c.z, d.z},
                   F2{a.w, b.w}, F2{c.w, d.w}};
    }
    __device__ static void clear_w(Tgt& t) { t.wa = t.wb = F2{0.f, 0.f}; }
    __device__ static void zero(Acc& c) { c.a1 = c.a2 = F2{0.f, 0.f}; }
    __device__ static void fold(const Acc& c, double& s1, double& s2) {
        s1 += (double)c.a1.hi + (double)c.a1.lo;
        s2 += (double)c.a2.hi + (double)c.a2.lo;
    }
    // unnormalised sums (exact two_sum of the high parts); the caller folds the result to FP64
    __device__ static JAcc jadd(const JAcc& x, const JAcc& y) {
        JAcc r = x;
        acc_add(r.a1, y.a1);
        acc_add(r.a2, y.a2);
        return r;
    }
    __device__ static JAcc jshfl_xor(const JAcc& x, int m) {
        return JAcc{F2{__shfl_xor_sync(0xffffffffu, x.a1.hi, m), __shfl_xor_sync(0xffffffffu, x.a1.lo, m)},
                    F2{__shfl_xor_sync(0xffffffffu, x.a2.hi, m), __shfl_xor_sync(0xffffffffu, x.a2.lo, m)}};
    }
    template <bool kMask>
    __device__ static void pair(const Tgt& T, const Src* S, const PairConsts& k, const float2* tab, Acc& acc,
                                const bool* exv) {
        const bool ex = exv[0];
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
        // lazy products and unnormalised accumulation as in pair_sym (the target rows of its terms); the
        // differences that can cancel (d, the dot products, 1 - E, 1 - E1, 3 - E q, X) stay normalised
        const F2 dx = sub(T.px, Px), dy = sub(T.py, Py), dz = sub(T.pz, Pz);
        const F2 r2 = dot3(dx, dy, dz, dx, dy, dz);
        const F2 rinv = rsqrt_ff(r2);
        const F2 r = mull(r2, rinv);
        const F2 kr = mull(f2(k.kappad), r);
        const F2 E = exp_neg_ffl(kr, tab);
        const F2 E1 = mull(E, add_f(kr, 1.f));
        const F2 dny = dot3(dx, dy, dz, Nx, Ny, Nz);
        const F2 dnx = dot3(dx, dy, dz, T.qx, T.qy, T.qz);
        const F2 nn = dot3(T.qx, T.qy, T.qz, Nx, Ny, Nz);
        const F2 rinv2 = mull(rinv, rinv);
        const F2 s = mull(rinv2, rinv);
        const F2 t1 = add_f(neg(mull(E1, f2(k.c1d))), 1.f);
        const F2 om = mull(rinv, add_f(neg(E), 1.f));
        const F2 t2 = add_f(neg(mull(E1, f2(k.c2d))), 1.f);
        const F2 u = add_f(neg(E1), 1.f);
        const F2 q = add_f(mull(kr, add_f(kr, 3.f)), 3.f);
        const F2 t3 = add_f(neg(mull(E, q)), 3.f);
        const F2 Bt = mull(mull(t3, mull(dnx, dny)), rinv2);
        const F2 X = sub(mull(u, nn), Bt);
        const F2 as = mull(A, s), bs = mull(Bw, s);
        acc_add(acc.a1, mull(as, mull(dny, t1)));
        acc_add(acc.a1, neg(mull(Bw, om)));
        acc_add(acc.a2, mull(bs, mull(dnx, t2)));
        acc_add(acc.a2, mull(as, X));
    }
    // Both orientations with lazy products (mull) and unnormalised accumulation (acc_add); the
    // differences that can cancel (d, the dot products, 1 - E, 1 - E1, 3 - E q, X) stay normalised.
    template <bool kFirst>
    __device__ static void pair_sym(const Tgt& T, const Src* S, const PairConsts& k, const float2* tab, Acc& acc,
                                    JAcc& ja) {
        const float4 s0 = S[0], s1 = S[1], s2 = S[2], s3 = S[3];
        const F2 Px{s0.x, s1.x}, Py{s0.y, s1.y}, Pz{s0.z, s1.z}, A{s0.w, s1.w};
        const F2 Nx{s2.x, s3.x}, Ny{s2.y, s3.y}, Nz{s2.z, s3.z}, Bw{s2.w, s3.w};
        const F2 dx = sub(T.px, Px), dy = sub(T.py, Py), dz = sub(T.pz, Pz);
        const F2 r2 = dot3(dx, dy, dz, dx, dy, dz);
        const F2 rinv = rsqrt_ff(r2);
        const F2 r = mull(r2, rinv);
        const F2 kr = mull(f2(k.kappad), r);
        const F2 E = exp_neg_ffl(kr, tab);
        const F2 E1 = mull(E, add_f(kr, 1.f));
        const F2 dny = dot3(dx, dy, dz, Nx, Ny, Nz);
        const F2 dnx = dot3(dx, dy, dz, T.qx, T.qy, T.qz);
        const F2 nn = dot3(T.qx, T.qy, T.qz, Nx, Ny, Nz);
        const F2 rinv2 = mull(rinv, rinv);
        const F2 s = mull(rinv2, rinv);
        const F2 t1 = add_f(neg(mull(E1, f2(k.c1d))), 1.f);
        const F2 om = mull(rinv, add_f(neg(E), 1.f));
        const F2 t2 = add_f(neg(mull(E1, f2(k.c2d))), 1.f);
        const F2 u = add_f(neg(E1), 1.f);
        const F2 q = add_f(mull(kr, add_f(kr, 3.f)), 3.f);
        const F2 t3 = add_f(neg(mull(E, q)), 3.f);
        const F2 Bt = mull(mull(t3, mull(dnx, dny)), rinv2);
        const F2 X = sub(mull(u, nn), Bt);
        const F2 as = mull(A, s), bs = mull(Bw, s);
        acc_add(acc.a1, mull(as, mull(dny, t1)));
        acc_add(acc.a1, neg(mull(Bw, om)));
        acc_add(acc.a2, mull(bs, mull(dnx, t2)));
        acc_add(acc.a2, mull(as, X));
        const F2 ast = mull(T.wa, s), bst = mull(T.wb, s);
        if constexpr (kFirst) {
            ja.a1 = neg(mull(ast, mull(dnx, t1)));
            ja.a2 = neg(mull(bst, mull(dny, t2)));
        } else {
            acc_add(ja.a1, neg(mull(ast, mull(dnx, t1))));
            acc_add(ja.a2, neg(mull(bst, mull(dny, t2))));
        }
        acc_add(ja.a1, neg(mull(T.wb, om)));
        acc_add(ja.a2, mull(ast, X));
    }
};

// Generic target handling for policies with kPack targets per thread slot: slot r of a thread holds
// targets tblock * BS + (r * kPack + h) * kThreads + tid, h < kPack.
template <typename Policy>
__device__ __forceinline__ typename Policy::Tgt load_targets(const typename Policy::Src* src, int M, const int* ti) {
    if constexpr (Policy::kPack == 1) {
        typename Policy::Tgt t = Policy::load(src, min(ti[0], M - 1));
        if (ti[0] >= M) Policy::clear_w(t);   // a padding target adds nothing to the sources
        return t;
    } else {
        return Policy::load_pack(src, M, ti);
    }
}
template <typename Policy>
__device__ __forceinline__ void fold_targets(const typename Policy::Acc& a, double* s1, double* s2) {
    if constexpr (Policy::kPack == 1) Policy::fold(a, s1[0], s2[0]);
    else Policy::fold_pack(a, s1, s2);
}

// Where a work item's sums go.  RegionOut: the sums of node i to out[c * cstride + (i - t0)], c = 0, 1
// (one region per item, added later in a fixed order); FxOut: added into the node's exact accumulators.
struct RegionOut {
    double* out;
    int64_t cstride, t0;
    __device__ __forceinline__ void put(int64_t i, double s1, double s2) const {
        out[i - t0] = s1;
        out[cstride + i - t0] = s2;
    }
};
struct FxOut {
    unsigned long long* acc;
    int64_t stride;
    __device__ __forceinline__ void put(int64_t i, double s1, double s2) const {
        fx_add(acc + i, stride, 0, s1);
        fx_add(acc + i, stride, 1, s2);
    }
};

// One one-sided work item of the dense pair sum: target block `tblock`
// (kThreads * R targets) against sources [j_begin, j_end), with the correction
// pairs masked; the sums of target i go to `out` (RegionOut or FxOut).
// Shared memory (ring, tables, barriers) is set up by the caller; `gt` counts
// the tiles this block has consumed so far (it fixes the mbarrier phase parity
// across items).  Returns false when a bounded wait expired (the error word is
// set; the caller must return).
template <typename Policy, int R, int U = 2, typename Out = FxOut>
__device__ __forceinline__ bool pair_item(const typename Policy::Src* __restrict__ src, int M,
                                          const int32_t* __restrict__ eptr, const int32_t* __restrict__ excl,
                                          int tblock, int j_begin, int j_end, const Out& out,
                                          const PairConsts& kc,
                                          int* __restrict__ err, typename Policy::Src* ring, const float2* tab,
                                          uint64_t* bar, uint32_t& gt) {
    using Src = typename Policy::Src;
    constexpr int TILE = Policy::kTile;
    constexpr int VEC = Policy::kVec;
    constexpr int P = Policy::kPack;
    constexpr int RP = R * P;
    const int tid = threadIdx.x;
    const int ntiles = (j_end > j_begin) ? (j_end - j_begin + TILE - 1) / TILE : 0;

    typename Policy::Tgt tg[R];
    double s1[RP], s2[RP];
    int ti[RP], epos[RP], eend[RP], enext[RP];
#pragma unroll
    for (int a = 0; a < RP; ++a) {
        ti[a] = tblock * (kThreads * RP) + a * kThreads + tid;
        const int t = min(ti[a], M - 1);
        s1[a] = 0.0;
        s2[a] = 0.0;
        int e = eptr[t], ee = eptr[t + 1];
        while (e < ee && excl[e] < j_begin) ++e;
        epos[a] = e;
        eend[a] = ee;
        enext[a] = (e < ee) ? excl[e] : INT_MAX;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) tg[r] = load_targets<Policy>(src, M, &ti[r * P]);
    auto issue = [&](int k) {
        const uint32_t g = gt + (uint32_t)k;
        const int j0 = j_begin + k * TILE;
        const int n = min(TILE, j_end - j0);
        const uint32_t bytes = (uint32_t)(n * VEC * sizeof(Src));
        Src* dst = ring + (g & 1) * TILE * VEC;
        fence_proxy_async();
        mbar_expect_tx(&bar[g & 1], bytes);
        bulk_load(dst, src + (size_t)VEC * j0, bytes, &bar[g & 1]);
    };
    if (tid == 0 && ntiles > 0) issue(0);

    for (int k = 0; k < ntiles; ++k) {
        const uint32_t g = gt + (uint32_t)k;
        if (tid == 0 && k + 1 < ntiles) issue(k + 1);
        const bool ok = mbar_wait(&bar[g & 1], (g >> 1) & 1, kc.wait_limit);
        if (__syncthreads_or(!ok)) {
            // give up: flag it, let the copies that may still be in flight (this tile's and the
            // next one's) land in this block's shared memory, return
            if (tid == 0) {
                atomicOr(err, kErrWait);
                (void)mbar_wait(&bar[g & 1], (g >> 1) & 1);
                if (k + 1 < ntiles) (void)mbar_wait(&bar[(g + 1) & 1], ((g + 1) >> 1) & 1);
            }
            return false;
        }
        const Src* tile = ring + (g & 1) * TILE * VEC;
        const int j0 = j_begin + k * TILE;
        const int n = min(TILE, j_end - j0);
        bool need = false;
#pragma unroll
        for (int a = 0; a < RP; ++a) need |= (enext[a] < j0 + n);
        typename Policy::Acc acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) Policy::zero(acc[r]);
        if (!__any_sync(0xffffffffu, need)) {
            const bool none[P] = {};
#pragma unroll U
            for (int q = 0; q < n; ++q) {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    Policy::template pair<false>(tg[r], tile + q * VEC, kc, tab, acc[r], none);
            }
        } else {
            for (int q = 0; q < n; ++q) {
                const int j = j0 + q;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    bool ex[P];
#pragma unroll
                    for (int h = 0; h < P; ++h) {
                        const int a = r * P + h;
                        ex[h] = (j == enext[a]);
                        if (ex[h]) {
                            ++epos[a];
                            enext[a] = (epos[a] < eend[a]) ? excl[epos[a]] : INT_MAX;
                        }
                    }
                    Policy::template pair<true>(tg[r], tile + q * VEC, kc, tab, acc[r], ex);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) fold_targets<Policy>(acc[r], &s1[r * P], &s2[r * P]);
        __syncthreads();   // the buffer of this tile is free for the tile after next
    }
    gt += (uint32_t)ntiles;
#pragma unroll
    for (int a = 0; a < RP; ++a)
        if (ti[a] < M) out.put(ti[a], s1[a], s2[a]);
    return true;
}

// In-warp transpose-and-sum of V per-lane values v[0..V) (V a power of two <= 32):
// afterwards every lane holds, in v[0], the sum over all 32 lanes of entry
// lane >> (5 - log2 V).  Each exchange stage halves the entries a lane keeps
// (it sends the half its partner keeps); the remaining stages are a plain
// butterfly.  The summation tree is the hypercube order 16, 8, 4, 2, 1 for any V.
template <typename Policy, int V>
__device__ __forceinline__ void transpose_sum(typename Policy::JAcc (&v)[V], int lane) {
    using J = typename Policy::JAcc;
    int cnt = V;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        if (cnt > 1) {
            const bool upper = (lane & m) != 0;
            const int h = cnt / 2;
#pragma unroll
            for (int i = 0; i < V / 2; ++i) {
                if (i < h) {
                    const J send = upper ? v[i] : v[i + h];
                    const J keep = upper ? v[i + h] : v[i];
                    v[i] = Policy::jadd(keep, Policy::jshfl_xor(send, m));
                }
            }
            cnt = h;
        } else {
            v[0] = Policy::jadd(v[0], Policy::jshfl_xor(v[0], m));
        }
    }
}

// One symmetric work item: target block `tblock` against sources
// [j_begin, j_end), no correction pair among them (the schedule guarantees it).
// Every pair is evaluated once for both orientations (Policy::pair_sym).  The
// target sums (at the item's end) and the source sums (per tile) are added
// into the nodes' exact accumulators (`out`).  Sources are read by
// broadcast as in the one-sided item; a thread accumulates the source-side
// terms of a chunk of V sources over its R targets, the warp transposes and
// sums them (transpose_sum), and the kWarps warp sums of a tile are added in
// warp order in shared memory (jred: kWarps * TILE entries).  The chunk loop
// is unrolled S sources at a time (S = V: fully); with S < V the chunk's
// accumulators shift by S registers per step, which keeps the code of long
// pair arithmetics within the instruction cache.
template <typename Policy, int R, int V, int U, int S = V>
__device__ __forceinline__ bool pair_item_sym(const typename Policy::Src* __restrict__ src, int M, int tblock,
                                              int j_begin, int j_end, const FxOut& out, const PairConsts& kc,
                                              int* __restrict__ err, typename Policy::Src* ring,
                                              typename Policy::JAcc* jred, const float2* tab, uint64_t* bar,
                                              uint32_t& gt) {
    using Src = typename Policy::Src;
    using J = typename Policy::JAcc;
    constexpr int TILE = Policy::kTile;
    constexpr int VEC = Policy::kVec;
    constexpr int P = Policy::kPack;
    constexpr int RP = R * P;
    constexpr int BS = kThreads * RP;
    constexpr int kWarps = kThreads / 32;
    constexpr int kShift = (V == 32) ? 0 : (V == 16) ? 1 : (V == 8) ? 2 : (V == 4) ? 3 : (V == 2) ? 4 : 5;
    static_assert(TILE % V == 0 && TILE <= kThreads, "tile layout");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int len = j_end - j_begin;
    const int ntiles = (len + TILE - 1) / TILE;

    typename Policy::Tgt tg[R];
    double s1[RP], s2[RP];
    int ti[RP];
#pragma unroll
    for (int a = 0; a < RP; ++a) {
        ti[a] = tblock * BS + a * kThreads + tid;
        s1[a] = 0.0;
        s2[a] = 0.0;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) tg[r] = load_targets<Policy>(src, M, &ti[r * P]);
    auto issue = [&](int k) {
        const uint32_t g = gt + (uint32_t)k;
        const int j0 = j_begin + k * TILE;
        const int n = min(TILE, j_end - j0);
        const uint32_t bytes = (uint32_t)(n * VEC * sizeof(Src));
        Src* dst = ring + (g & 1) * TILE * VEC;
        fence_proxy_async();
        mbar_expect_tx(&bar[g & 1], bytes);
        bulk_load(dst, src + (size_t)VEC * j0, bytes, &bar[g & 1]);
    };
    if (tid == 0 && ntiles > 0) issue(0);

    for (int k = 0; k < ntiles; ++k) {
        const uint32_t g = gt + (uint32_t)k;
        if (tid == 0 && k + 1 < ntiles) issue(k + 1);
        const bool ok = mbar_wait(&bar[g & 1], (g >> 1) & 1, kc.wait_limit);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {   // as in pair_item: flag, drain both copies in flight, return
                atomicOr(err, kErrWait);
                (void)mbar_wait(&bar[g & 1], (g >> 1) & 1);
                if (k + 1 < ntiles) (void)mbar_wait(&bar[(g + 1) & 1], ((g + 1) >> 1) & 1);
            }
            return false;
        }
        const Src* tile = ring + (g & 1) * TILE * VEC;
        const int j0 = j_begin + k * TILE;
        const int n = min(TILE, j_end - j0);
        typename Policy::Acc acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) Policy::zero(acc[r]);
#pragma unroll U
        for (int c0 = 0; c0 < n; c0 += V) {
            J ja[V];
#pragma unroll
            for (int q = 0; q < V; ++q) Policy::zero(ja[q]);
            if constexpr (S == V) {
                if (c0 + V <= n) {
#pragma unroll
                    for (int q = 0; q < V; ++q) {
                        typename Policy::JAccR jr;
                        Policy::template pair_sym<true>(tg[0], tile + (c0 + q) * VEC, kc, tab, acc[0], jr);
#pragma unroll
                        for (int r = 1; r < R; ++r)
                            Policy::template pair_sym<false>(tg[r], tile + (c0 + q) * VEC, kc, tab, acc[r], jr);
                        ja[q] = Policy::jfinal(jr);
                    }
                } else {   // ragged end of the item: warp-uniform skip
#pragma unroll
                    for (int q = 0; q < V; ++q) {
                        if (c0 + q < n) {
                            typename Policy::JAccR jr;
                            Policy::template pair_sym<true>(tg[0], tile + (c0 + q) * VEC, kc, tab, acc[0], jr);
#pragma unroll
                            for (int r = 1; r < R; ++r)
                                Policy::template pair_sym<false>(tg[r], tile + (c0 + q) * VEC, kc, tab, acc[r], jr);
                            ja[q] = Policy::jfinal(jr);
                        }
                    }
                }
            } else {
                // S sources per step; afterwards ja[k] holds source V - S (k / S + 1) + k % S of the chunk
#pragma unroll 1
                for (int q0 = 0; q0 < V; q0 += S) {
                    J cur[S];
#pragma unroll
                    for (int t = 0; t < S; ++t) {
                        Policy::zero(cur[t]);
                        const int q = c0 + q0 + t;
                        if (q < n) {   // warp-uniform
                            typename Policy::JAccR jr;
                            Policy::template pair_sym<true>(tg[0], tile + q * VEC, kc, tab, acc[0], jr);
#pragma unroll
                            for (int r = 1; r < R; ++r)
                                Policy::template pair_sym<false>(tg[r], tile + q * VEC, kc, tab, acc[r], jr);
                            cur[t] = Policy::jfinal(jr);
                        }
                    }
#pragma unroll
                    for (int k = V - 1; k >= S; --k) ja[k] = ja[k - S];
#pragma unroll
                    for (int t = 0; t < S; ++t) ja[t] = cur[t];
                }
            }
            transpose_sum<Policy, V>(ja, lane);
            const int e = lane >> kShift;
            const int qs = V - S * (e / S + 1) + e % S;
            if ((lane & ((1 << kShift) - 1)) == 0 && c0 + qs < n) jred[warp * TILE + c0 + qs] = ja[0];
        }
#pragma unroll
        for (int r = 0; r < R; ++r) fold_targets<Policy>(acc[r], &s1[r * P], &s2[r * P]);
        __syncthreads();   // all warp sums of this tile are in jred
        if (tid < n) {
            J t = jred[tid];
#pragma unroll
            for (int w = 1; w < kWarps; ++w) t = Policy::jadd(t, jred[w * TILE + tid]);
            double d1 = 0.0, d2 = 0.0;
            Policy::fold(t, d1, d2);
            out.put(j0 + tid, d1, d2);
        }
        __syncthreads();   // jred and the buffer of this tile are free again
    }
    gt += (uint32_t)ntiles;
#pragma unroll
    for (int a = 0; a < RP; ++a)
        if (ti[a] < M) out.put(ti[a], s1[a], s2[a]);
    return true;
}

// Runs one item of a schedule (dispatch on its kind); its sums go into the nodes' exact accumulators
// (acc, M words per accumulator word, fx_add).
template <typename Policy, int R, int V, int U>
__device__ __forceinline__ bool run_item(const PairItem& it, const typename Policy::Src* __restrict__ src, int M,
                                         const int32_t* __restrict__ eptr, const int32_t* __restrict__ excl,
                                         unsigned long long* __restrict__ acc, const PairConsts& kc,
                                         int* __restrict__ err, typename Policy::Src* ring,
                                         typename Policy::JAcc* jred, const float2* tab, uint64_t* bar,
                                         uint32_t& gt) {
    constexpr int S = Policy::kSymStep < V ? Policy::kSymStep : V;
    const FxOut out{acc, (int64_t)M};
    if (it.sym)
        return pair_item_sym<Policy, R, V, U, S>(src, M, it.I, it.j_begin, it.j_end, out, kc, err, ring, jred, tab,
                                                 bar, gt);
    return pair_item<Policy, R, U>(src, M, eptr, excl, it.I, it.j_begin, it.j_end, out, kc, err, ring, tab, bar, gt);
}

// Shared-memory bytes of a pair block: the two-stage source ring, the warp
// sums of a symmetric tile and, for the float-float policy, the exponential
// tables (in that order; each part a multiple of 16 bytes).
template <typename Policy>
constexpr size_t pair_ring_bytes() {
    return 2 * Policy::kTile * Policy::kVec * sizeof(typename Policy::Src);
}
template <typename Policy>
constexpr size_t pair_jred_bytes() {
    return (size_t)(kThreads / 32) * Policy::kTile * sizeof(typename Policy::JAcc);
}
template <typename Policy>
constexpr size_t pair_smem_bytes() {
    return pair_ring_bytes<Policy>() + pair_jred_bytes<Policy>() +
           (Policy::kTables ? (kExpHi + kExpLo) * sizeof(float2) : 0);
}
// The dynamic shared memory of a pair block, carved in the order above.
template <typename Policy>
struct PairSmem {
    typename Policy::Src* ring;
    typename Policy::JAcc* jred;
    float2* tab;
    __device__ explicit PairSmem(unsigned char* raw)
        : ring(reinterpret_cast<typename Policy::Src*>(raw)),
          jred(reinterpret_cast<typename Policy::JAcc*>(raw + pair_ring_bytes<Policy>())),
          tab(reinterpret_cast<float2*>(raw + pair_ring_bytes<Policy>() + pair_jred_bytes<Policy>())) {}
};

// Launch shapes of the schedules: thread slots (x the policy's kPack targets) and sources per
// transposed chunk.  R and the tile fix the target blocks and the per-tile sums, hence the summation
// order: they are a property of a system's schedule (set when the system is set up), the same
// wherever the system runs.  The float-float and FP64 shapes are fixed; kR32 is the default FP32 one.
constexpr int kR32 = 2, kRdf = 1, kR64 = 1;   // thread slots (FP32: 2 packed pairs = 4 targets)
constexpr int kChunkDf = 8, kChunk64 = 8;

// The packed FP32 policy with another source tile (sources per shared-memory stage).
template <int TILE>
struct Fp32x2T : Fp32x2Policy {
    static constexpr int kTile = TILE;
};

// FP32 schedule-kernel variants, one of which each system's FP32 schedule uses: thread slots R (R x 2
// targets per thread: 512 or 1024 per block), source tile, sources per transposed chunk V and unroll
// U of the chunk loop.  Variant 0 is the default shape (the treecode's near items always use it).
struct Var32 {
    int R, tile, V, U;
};
constexpr int kNumVar32 = 6;
constexpr Var32 kVar32[kNumVar32] = {{2, 256, 8, 1}, {2, 256, 8, 2}, {1, 256, 8, 2},
                                     {2, 128, 8, 2}, {1, 128, 8, 2}, {2, 256, 4, 2}};

// f.template run<Policy, R, V, U>() for FP32 variant v (a functor with a member template `run`)
template <typename F>
inline int with_var32(int v, const F& f) {
    switch (v) {
        case 1: return f.template run<Fp32x2T<256>, 2, 8, 2>();
        case 2: return f.template run<Fp32x2T<256>, 1, 8, 2>();
        case 3: return f.template run<Fp32x2T<128>, 2, 8, 2>();
        case 4: return f.template run<Fp32x2T<128>, 1, 8, 2>();
        case 5: return f.template run<Fp32x2T<256>, 2, 4, 2>();
        default: return f.template run<Fp32x2T<256>, 2, 8, 1>();
    }
}

// Per-block setup shared by every pair kernel: exponential tables and the two mbarriers.
template <typename Policy>
__device__ __forceinline__ void pair_block_init(const PairConsts& kc, float2* tab, uint64_t* bar) {
    if constexpr (Policy::kTables) {
        for (int q = threadIdx.x; q < kExpHi + kExpLo; q += kThreads) tab[q] = kc.exp_tab[q];
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
}

inline float2 split_ff(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}
__device__ __forceinline__ float2 split_ff_dev(double v) {
    const float hi = __double2float_rn(v);
    return make_float2(hi, __double2float_rn(v - (double)hi));
}

}  // namespace pk

// float-float table of e^{-k} (k < 64) and e^{-k/1024} (k < 1024) on a device
int exp_table(int device, const float2** out);
// Splits of the source range for equal-work items filling whole waves of `slots` resident blocks
// (one-sided grid launch of the fixed-scratch entry point)
PairPlan make_plan(int64_t M, int R, int tile, int slots);
// Resident blocks of the schedule kernels of the three arithmetics: [0] FP32 (default variant),
// [1] float-float, [2] FP64
int schedule_slots(int sms, int slots[3]);
// The FP32 variant of the most recent tuning in this process (-1 before any)
int last_fp32_variant();
// Runs a handle's schedule of one arithmetic (policy index 0 FP32, 1 float-float, 2 FP64) on its stream
int launch_schedule(ctr_ibim* s, int pol, const void* src, const pk::PairConsts& kc);
// Fill the f32x2 copies of a PairConsts from its FP32 fields
void set_packed_consts(pk::PairConsts& kc);
// Pair constants of a handle (kernel-ratio terms, kappa, tables when needed)
int pair_consts(ctr_ibim* s, bool tables, pk::PairConsts* out);
// Polls of the pair kernels' bounded waits for launches prepared from now on (ctr_set_wait_limit)
uint32_t wait_limit();

}  // namespace ctr
