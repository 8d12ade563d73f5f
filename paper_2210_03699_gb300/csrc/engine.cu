// Multi-slot solver engine: many CTR-IBIM systems advanced together on one GPU.
//
// Each slot holds one system (a ctr_ibim handle) and its solver state on the
// device.  The solver is right-preconditioned GMRES(m) (CGS2, FP64 Givens) on
// the operator of Eq. (2.30); every cycle ends by recomputing the true
// residual r = g - A x with the residual pair arithmetic and starting the next
// cycle from it.  With FP32 inner pairs and an FP64-accurate residual this is
// GMRES-based iterative refinement; with the same precision inside and out it
// is plain restarted GMRES.
//
// One engine step, captured once as a CUDA graph and replayed:
//   inner half   (slots in state INNER)  one Arnoldi iteration:
//                z = Lambda^-1 V_j, pack, pairs, finish w = A z, CGS2 (two passes
//                of batched dot products and updates), norm, Givens, scale, advance;
//   update half  (slots in state UPDATE) x += Lambda^-1 V y, pack, pairs,
//                finish r = g - A x, norm, decide (done / next cycle), start cycle.
// The dense pair sums of all slots run in persistent kernels (one per pair
// arithmetic and half) whose blocks take work entries (slot, item of that
// slot's pair schedule: target block, source range, one-sided or symmetric)
// from a list sorted by cost through an atomic counter; entries of slots in
// another state return at once.  A slot's items, partial-sum layout,
// reduction chunks and scalar updates are exactly those of the slot alone, so
// a system's result does not depend on what else the engine holds.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>

#include "engine.cuh"
#include "pairkern.cuh"
#include "tree.cuh"

namespace ctr {

using namespace pk;

namespace {

constexpr int kVecThreads = 256;
constexpr double kUpdateGate = 1e-4;   // |r| / |g| below which refinement residuals are updated
// Work entries carry (slot, item | part << kPartShift): items of a schedule < 2^24, parts <= kMaxParts.
constexpr int kPartShift = 24;
constexpr int kItemMask = (1 << kPartShift) - 1;
constexpr int kMaxParts = 127;
constexpr int kMinItemsPerPart = 64;

__device__ __forceinline__ double block_sum_d(double v) {
    __shared__ double sh[kVecThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kVecThreads / 32; ++w) t += sh[w];
    __syncthreads();
    return t;
}

__device__ __forceinline__ bool inner_active(const SlotDev& s) { return s.stat.state == kSlotInner; }
__device__ __forceinline__ bool update_active(const SlotDev& s) { return s.stat.state == kSlotUpdate; }
// Pair arithmetic of a slot's residual in this cycle: the residual arithmetic for g - A x, the inner
// one for an update r - A d of a small correction d.
__device__ __forceinline__ int res_arith(const SlotDev& s) { return s.upd ? s.inner_prec : s.res_prec; }

// ---------------------------------------------------------------- packing
__device__ __forceinline__ void pack_weights(const SlotDev& s, int prec, int64_t t, double a, double b) {
    if (prec == CTR_FP32_REFINE) {
        s.src32[4 * t + 1].z = s.src32[4 * t + 1].w = (float)a;   // duplicated pairs: a and -b
        s.src32[4 * t + 3].z = s.src32[4 * t + 3].w = -(float)b;
    } else if (prec == CTR_FP64) {
        s.src64[2 * t].w = a;
        s.src64[2 * t + 1].w = b;
    } else {
        const float ah = (float)a, bh = (float)b;
        s.srcdf[4 * t].w = ah;
        s.srcdf[4 * t + 1].w = (float)(a - (double)ah);
        s.srcdf[4 * t + 2].w = bh;
        s.srcdf[4 * t + 3].w = (float)(b - (double)bh);
    }
}

// inner: z = Lambda^-1 V_j and the weights of z
__global__ void k_prep_inner(SlotDev* S) {
    const SlotDev& s = S[blockIdx.y];
    if (!inner_active(s) || s.part != 0) return;   // later parts reuse the packed weights
    const int64_t M = s.M;
    const double* v = s.V + (size_t)s.j * s.n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < M; t += (int64_t)gridDim.x * blockDim.x) {
        const double z1 = v[t] * s.il1, z2 = v[M + t] * s.il2;
        s.z[t] = z1;
        s.z[M + t] = z2;
        pack_weights(s, s.inner_prec, s.tinv ? (int64_t)s.tinv[t] : t, s.scale * s.W[t] * z1, s.scale * s.W[t] * z2);
    }
}

// update: d = Lambda^-1 V y (k columns), x += d, and the weights of x (residual g - A x) or, for a
// residual update, d kept in z and its weights in the inner arithmetic (residual r - A d)
__global__ void k_update_x(SlotDev* S) {
    const SlotDev& s = S[blockIdx.y];
    if (!update_active(s) || s.part != 0) return;
    const int64_t M = s.M, n = s.n;
    const int k = s.kdone;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < M; t += (int64_t)gridDim.x * blockDim.x) {
        double v1 = 0.0, v2 = 0.0;
        for (int i = 0; i < k; ++i) {
            v1 += s.V[(size_t)i * n + t] * s.y[i];
            v2 += s.V[(size_t)i * n + M + t] * s.y[i];
        }
        const double d1 = v1 * s.il1, d2 = v2 * s.il2;
        const double x1 = s.x[t] + d1, x2 = s.x[M + t] + d2;
        s.x[t] = x1;
        s.x[M + t] = x2;
        const int64_t pos = s.tinv ? (int64_t)s.tinv[t] : t;
        if (s.upd) {
            s.z[t] = d1;
            s.z[M + t] = d2;
            pack_weights(s, s.inner_prec, pos, s.scale * s.W[t] * d1, s.scale * s.W[t] * d2);
        } else {
            pack_weights(s, s.res_prec, pos, s.scale * s.W[t] * x1, s.scale * s.W[t] * x2);
        }
    }
}

// ---------------------------------------------------------------- persistent pair kernels
// Work entries (slot, item of that slot's schedule), sorted by decreasing cost.  kShared: every slot
// of this arithmetic has the same pair constants, passed as the launch parameter `pkc` (read from the
// constant bank, no registers); otherwise each item takes its slot's constants.
template <typename Policy, int R, int V, int U, bool kShared>
__global__ void __launch_bounds__(kThreads, 2) k_pairs(SlotDev* S, const int2* __restrict__ items,
                                                    const int* __restrict__ n_items, int* __restrict__ counter,
                                                    int half, int prec, int pol, const float2* __restrict__ exp_tab,
                                                    int* __restrict__ err, const PairConsts pkc,
                                                    const int* __restrict__ need) {
    using Src = typename Policy::Src;
    if (need[pol] == 0) return;   // no slot in this half uses this arithmetic: skip the whole list
    extern __shared__ __align__(128) unsigned char smem_raw[];
    PairSmem<Policy> sm(smem_raw);
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int cur;
    __shared__ PairConsts kc;
    if (threadIdx.x == 0) kc.exp_tab = exp_tab;   // one table per device, shared by every slot
    __syncthreads();
    pair_block_init<Policy>(kc, sm.tab, bar);
    uint32_t gt = 0;
    const int total = *n_items;
    for (;;) {
        if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
        __syncthreads();
        const int it = cur;
        __syncthreads();
        if (it >= total) break;
        const int2 w = items[it];   // slot, item | part << kPartShift
        const SlotDev& s = S[w.x];
        const bool want = half == 0 ? (inner_active(s) && s.inner_prec == prec)
                                    : (update_active(s) && res_arith(s) == prec);
        const int pe = w.y >> kPartShift;
        if (!want || pe < s.part || pe >= s.part + s.span) continue;
        const int item = w.y & kItemMask;
        const Src* src = reinterpret_cast<const Src*>(prec == CTR_FP32_REFINE ? (const void*)s.src32
                                                      : prec == CTR_DF64 ? (const void*)s.srcdf
                                                                         : (const void*)s.src64);
        if constexpr (kShared) {
            if (!run_item<Policy, R, V, U>(s.items[pol][item], src, s.M, s.eptr, s.excl, s.acc, pkc, err, sm.ring,
                                           sm.jred, sm.tab, bar, gt))
                return;
        } else {
            if (threadIdx.x == 0) {
                const float2* t = kc.exp_tab;
                kc = s.kc;
                kc.exp_tab = t;
            }
            __syncthreads();
            const PairConsts k = kc;   // block-uniform register copy: no shared loads in the pair loops
            if (!run_item<Policy, R, V, U>(s.items[pol][item], src, s.M, s.eptr, s.excl, s.acc, k, err, sm.ring,
                                           sm.jred, sm.tab, bar, gt))
                return;
        }
        __syncthreads();
    }
}

// finish: diag + the node's accumulated dense sum (read and cleared) + correction of the applied vector;
// inner: w = V_{j+1} = A z;   update: r = g - A x, or r = r - A d (residual update, d in z)
__global__ void k_finish(SlotDev* S, int half) {
    const SlotDev& s = S[blockIdx.y];
    if (half == 0 ? !inner_active(s) : !update_active(s)) return;
    const int64_t M = s.M, E = s.E;
    const bool upd = (half == 1) && s.upd;
    const double* x = (half == 0 || upd) ? s.z : s.x;
    double* out = (half == 0) ? s.V + (size_t)(s.j + 1) * s.n : s.r;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        double s1, s2;
        fx_read(s.acc + (s.tinv ? (int64_t)s.tinv[i] : i), M, true, s1, s2);
        double c1 = 0.0, c2 = 0.0;
        for (int e = s.cptr[i]; e < s.cptr[i + 1]; ++e) {
            const int m = s.cnode[e];
            const double Wm = s.W[m], r1 = x[m], r2 = x[M + m];
            c1 += Wm * (s.h2 * s.cw[e] * r1 - s.h3 * s.cw[3 * E + e] * r2);
            c2 += Wm * (s.h2 * s.cw[E + e] * r1 - s.h2 * s.cw[2 * E + e] * r2);
        }
        const double y1 = s.lam1 * x[i] + s1 + c1;
        const double y2 = s.lam2 * x[M + i] + s2 + c2;
        if (half == 0) {
            out[i] = y1;
            out[M + i] = y2;
        } else if (upd) {   // out is r: each thread updates its own two entries
            out[i] -= y1;
            out[M + i] -= y2;
        } else {
            out[i] = s.g[i] - y1;
            out[M + i] = s.g[M + i] - y2;
        }
    }
}

// ---------------------------------------------------------------- batched reductions (same chunking as alone)
// mode 0/1: c = V[0..j] . w (first / second Gram-Schmidt pass), 2: |w|^2, 3: |r|^2
__global__ void k_dots_partial(SlotDev* S, int mode) {
    const SlotDev& s = S[blockIdx.y];
    const bool act = (mode == 3) ? update_active(s) : inner_active(s);
    if (!act || (int)blockIdx.x >= s.nblk) return;
    const int64_t n = s.n;
    const int64_t chunk = (n + s.nblk - 1) / s.nblk;
    const int64_t t0 = (int64_t)blockIdx.x * chunk, t1 = min(n, t0 + chunk);
    const double* w = (mode == 3) ? s.r : s.V + (size_t)(s.j + 1) * n;
    const int count = (mode <= 1) ? s.j + 1 : 1;
    for (int i = 0; i < count; ++i) {
        const double* a = (mode <= 1) ? s.V + (size_t)i * n : w;
        double v = 0.0;
        for (int64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) v += a[t] * w[t];
        v = block_sum_d(v);
        if (threadIdx.x == 0) s.dpart[(size_t)i * s.nblk + blockIdx.x] = v;
    }
}

__global__ void k_dots_final(SlotDev* S, int mode) {
    const SlotDev& s = S[blockIdx.y];
    const bool act = (mode == 3) ? update_active(s) : inner_active(s);
    if (!act) return;
    const int count = (mode <= 1) ? s.j + 1 : 1;
    const int i = blockIdx.x;
    if (i >= count) return;
    double v = 0.0;
    for (int b = threadIdx.x; b < s.nblk; b += blockDim.x) v += s.dpart[(size_t)i * s.nblk + b];
    v = block_sum_d(v);
    if (threadIdx.x == 0) {
        double* out = (mode == 0) ? s.cgs : (mode == 1) ? s.cgs2 : (mode == 2) ? s.scal : s.scal + 1;
        out[i] = v;
    }
}

// w -= V[0..j] c   (pass: 0 first coefficients, 1 second)
__global__ void k_sub(SlotDev* S, int pass) {
    const SlotDev& s = S[blockIdx.y];
    if (!inner_active(s)) return;
    const int64_t n = s.n;
    double* w = s.V + (size_t)(s.j + 1) * n;
    const double* c = pass ? s.cgs2 : s.cgs;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double v = w[t];
        for (int i = 0; i <= s.j; ++i) v -= s.V[(size_t)i * n + t] * c[i];
        w[t] = v;
    }
}

// Givens update of Hessenberg column j (one thread per slot)
__global__ void k_givens(SlotDev* S, int cap) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cap) return;
    SlotDev& s = S[q];
    if (!inner_active(s)) return;
    const int j = s.j, ldh = s.m + 1;
    double* col = s.H + (size_t)j * ldh;
    for (int i = 0; i <= j; ++i) col[i] = s.cgs[i] + s.cgs2[i];
    const double hn = sqrt(s.scal[0]);
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        const double t = s.cs[i] * col[i] + s.sn[i] * col[i + 1];
        col[i + 1] = -s.sn[i] * col[i] + s.cs[i] * col[i + 1];
        col[i] = t;
    }
    const double den = hypot(col[j], col[j + 1]);
    s.cs[j] = col[j] / den;
    s.sn[j] = col[j + 1] / den;
    col[j] = den;
    col[j + 1] = 0.0;
    s.sv[j + 1] = -s.sn[j] * s.sv[j];
    s.sv[j] = s.cs[j] * s.sv[j];
    s.scal[2] = hn;
    s.stat.iterations++;
    if (s.inner_prec == CTR_FP32_REFINE) s.stat.matvecs_fp32++; else s.stat.matvecs_fp64++;
    s.budget--;
    const double est = fabs(s.sv[j + 1]);
    if (!isfinite(est)) s.stat.numeric_error = 1;
    s.cycle_end = (est <= s.tol_cycle || j + 1 == s.m || s.budget <= 0 || hn == 0.0 || !isfinite(est)) ? 1 : 0;
}

__global__ void k_scale_next(SlotDev* S) {
    const SlotDev& s = S[blockIdx.y];
    if (!inner_active(s)) return;
    double* w = s.V + (size_t)(s.j + 1) * s.n;
    const double f = 1.0 / s.scal[2];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < s.n; t += (int64_t)gridDim.x * blockDim.x)
        w[t] *= f;
}

// advance (one thread per slot): next Arnoldi index, or end of cycle -> update state
__global__ void k_advance(SlotDev* S, int cap) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cap) return;
    SlotDev& s = S[q];
    if (!inner_active(s)) return;
    if (s.cycle_end) {
        s.kdone = s.j + 1;
        s.stat.state = kSlotUpdate;
    } else {
        s.j += 1;
    }
}

// back substitution R y = s (one thread per slot in UPDATE)
__global__ void k_upper_solve(SlotDev* S, int cap) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cap) return;
    SlotDev& s = S[q];
    if (!update_active(s) || s.part != 0) return;
    const int k = s.kdone, ldh = s.m + 1;
    for (int i = k - 1; i >= 0; --i) {
        double v = s.sv[i];
        for (int l = i + 1; l < k; ++l) v -= s.H[(size_t)l * ldh + i] * s.y[l];
        s.y[i] = v / s.H[(size_t)i * ldh + i];
    }
}

// after the residual: converged, out of budget, or the next cycle from r
__global__ void k_decide(SlotDev* S, int cap) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cap) return;
    SlotDev& s = S[q];
    if (!update_active(s)) return;
    if (s.upd) s.stat.matvecs_fp32++; else s.stat.matvecs_fp64++;
    s.stat.refinements++;
    const double rn = sqrt(s.scal[1]);
    s.stat.residual = (s.gnorm > 0.0) ? rn / s.gnorm : 0.0;
    if (!isfinite(rn)) {
        s.stat.numeric_error = 1;
        s.stat.state = kSlotDone;
        return;
    }
    const bool conv = rn <= s.tol_out * s.gnorm;
    const bool out = s.budget <= 0 || (s.refine && s.stat.refinements >= s.max_refine);
    if (conv || out) {
        s.stat.converged = conv ? 1 : 0;
        s.stat.state = kSlotDone;
        return;
    }
    s.beta = rn;
    s.tol_cycle = s.refine ? s.inner_tol * rn : s.tol_out * s.gnorm;
    // The next residual may be updated as r - A d in the inner arithmetic once r is small: the inner
    // operator's error on d (about 1e-7 |A| |d|, |d| ~ |A^-1| |r|) then stays orders of magnitude
    // below the tolerance, while g - A x would need the residual arithmetic at full magnitude.
    s.upd = (s.refine && s.res_update && rn <= kUpdateGate * s.gnorm) ? 1 : 0;
    s.stat.state = kSlotStart;
}

// V[0] = r / beta for slots starting a cycle
__global__ void k_start_vec(SlotDev* S) {
    const SlotDev& s = S[blockIdx.y];
    if (s.stat.state != kSlotStart) return;
    const double f = 1.0 / s.beta;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < s.n; t += (int64_t)gridDim.x * blockDim.x)
        s.V[t] = s.r[t] * f;
}

__global__ void k_start_scalars(SlotDev* S, int cap) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cap) return;
    SlotDev& s = S[q];
    if (s.stat.state != kSlotStart) return;
    for (int i = 0; i <= s.m; ++i) s.sv[i] = 0.0;
    s.sv[0] = s.beta;
    s.j = 0;
    s.stat.state = kSlotInner;
}

__device__ __forceinline__ int arith_index(int prec) { return prec == CTR_FP32_REFINE ? 0 : (prec == CTR_DF64 ? 1 : 2); }

// Estimated pair work of a slot in the step ahead (seconds), and its arithmetic.
__device__ __forceinline__ float step_work(const SlotDev& s, int& a) {
    if (s.stat.state == kSlotInner) a = arith_index(s.inner_prec);
    else if (s.stat.state == kSlotUpdate) a = arith_index(res_arith(s));
    else return 0.f;
    return s.part_s[a];
}

// Start of a step (one block): slots between two parts of an application resume; every slot whose
// application is split gets its span of parts for this step: one, or as many as fit in the pair work of
// all other slots in the step.  A large system thus takes about half of a busy step and one part of an
// otherwise idle one, and the other slots' steps grow by at most that much.
__global__ void k_plan_step(SlotDev* S, int cap) {
    __shared__ float red[kVecThreads];
    float w = 0.f;
    for (int q = threadIdx.x; q < cap; q += blockDim.x) {
        SlotDev& s = S[q];
        if (s.stat.state == kSlotInnerWait) s.stat.state = kSlotInner;
        else if (s.stat.state == kSlotUpdateWait) s.stat.state = kSlotUpdate;
        int a = 0;
        w += step_work(s, a);
    }
    red[threadIdx.x] = w;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const float total = red[0];
    for (int q = threadIdx.x; q < cap; q += blockDim.x) {
        SlotDev& s = S[q];
        int a = 0;
        const float mine = step_work(s, a);
        s.span = 1;
        if (mine > 0.f && s.nparts[a] > 1) {
            const float fit = floorf((total - mine) / mine);
            s.span = max(1, min(s.nparts[a] - s.part, (int)fminf(fit, (float)kMaxParts)));
        }
    }
}

// Before a half's pair launches (one block): which pair arithmetics any slot applies in this half (the
// inner arithmetic of slots in INNER, the residual arithmetic of slots in UPDATE).  The persistent pair
// kernels of the others return at once instead of walking their whole work lists.
__global__ void k_need(const SlotDev* S, int cap, int half, int* need) {
    __shared__ int f[3];
    if (threadIdx.x < 3) f[threadIdx.x] = 0;
    __syncthreads();
    for (int q = threadIdx.x; q < cap; q += blockDim.x) {
        const SlotDev& s = S[q];
        if (half == 0 ? inner_active(s) : update_active(s))
            f[arith_index(half == 0 ? s.inner_prec : res_arith(s))] = 1;
    }
    __syncthreads();
    if (threadIdx.x < 3) need[threadIdx.x] = f[threadIdx.x];
}

// After a half's pair launches: a slot whose application has parts left waits for the next step (the
// rest of this step skips it); one that ran its last part goes on to finish the application.
__global__ void k_part(SlotDev* S, int cap, int half) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cap) return;
    SlotDev& s = S[q];
    if (half == 0 ? !inner_active(s) : !update_active(s)) return;
    const int np = s.nparts[arith_index(half == 0 ? s.inner_prec : res_arith(s))];
    if (s.part + s.span < np) {
        s.part += s.span;
        s.stat.state = half == 0 ? kSlotInnerWait : kSlotUpdateWait;
    } else {
        s.part = 0;
        s.span = 1;   // a residual started later in this step runs one part
    }
}

__global__ void k_stats(const SlotDev* S, int cap, SlotStat* out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < cap) out[q] = S[q].stat;
}

constexpr int kNV = kNumVar32;   // work lists per arithmetic

template <typename Policy, int R, int V, int U, bool kShared>
int launch_persistent_k(Engine* e, int pol, int var, int half, int prec) {
    const size_t smem = pair_smem_bytes<Policy>();
    static int per_dev[64] = {0};   // resident blocks of this instantiation, per device (attribute set there)
    int dev = 0;
    CTR_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CTR_ERR_INVALID, "device index");
    int& per_sm = per_dev[dev];
    if (per_sm == 0) {
        int b = 0;
        // dynamic shared memory above the default 48 KB per block needs the kernel's opt-in
        CTR_CUDA_TRY(cudaFuncSetAttribute(k_pairs<Policy, R, V, U, kShared>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        CTR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pairs<Policy, R, V, U, kShared>, kThreads,
                                                                   smem));
        per_sm = std::max(1, b);
    }
    const int list = pol * kNV + var;
    k_pairs<Policy, R, V, U, kShared><<<per_sm * e->sms, kThreads, smem, e->stream>>>(
        e->slots.as<SlotDev>(), e->items[pol][var].as<int2>(), e->n_items.as<int>() + list,
        e->counters.as<int>() + 2 * list + half, half, prec, pol, e->exp_tab, e->err.as<int>(), e->kc_val[pol],
        e->need.as<int>());
    CTR_LAUNCHED();
    return CTR_OK;
}

template <typename Policy, int R, int V, int U>
int launch_persistent(Engine* e, int pol, int var, int half, int prec) {
    return e->kc_shared[pol] ? launch_persistent_k<Policy, R, V, U, true>(e, pol, var, half, prec)
                             : launch_persistent_k<Policy, R, V, U, false>(e, pol, var, half, prec);
}

struct PersistentRun {
    Engine* e;
    int var, half;
    template <typename P, int R, int V, int U>
    int run() const { return launch_persistent<P, R, V, U>(e, 0, var, half, CTR_FP32_REFINE); }
};

// Treecode entries of a slot in this half's arithmetic (filtered by the slot's state at run time).
struct EngineTreeAcc {
    const SlotDev* S;
    int half, prec;
    __device__ const TreeView* view(int q) const {
        const SlotDev& s = S[q];
        const bool want = half == 0 ? (inner_active(s) && s.inner_prec == prec) : (update_active(s) && res_arith(s) == prec);
        return (want && s.tv.on) ? &s.tv : nullptr;
    }
};

template <typename Real, int R, int NT>
int launch_tree_engine(Engine* e, int pol, int half, int prec) {
    static std::map<std::pair<int, int>, int> cache;
    const EngineTreeAcc acc{e->slots.as<SlotDev>(), half, prec};
    const int* cnt = e->tree_cnt.as<int>() + 3 * pol;
    int* ctr = e->tree_counters.as<int>() + 4 * pol + 2 * half;
    k_tree_mom<Real, EngineTreeAcc><<<2 * e->sms, kThreads, 0, e->stream>>>(acc, e->tree_ent[pol][0].as<int2>(), cnt,
                                                                          ctr, pol);
    CTR_LAUNCHED();
    k_tree_momred<Real, EngineTreeAcc><<<4 * e->sms, kThreads, 0, e->stream>>>(acc, e->tree_ent[pol][1].as<int2>(),
                                                                             cnt + 1, pol);
    CTR_LAUNCHED();
    if constexpr (sizeof(Real) == 8 && R == kTreeR[1] && NT == kTreeNT[1]) {   // float-float far field
        auto kern = k_tree_far_ff<R, NT, EngineTreeAcc>;
        const int smem = (int)tree_farff_smem(std::max(1, e->tree_np[pol]));   // the largest proxy count admitted
        const int per_sm = far_per_sm(kern, NT, smem, (int)tree_farff_smem(), cache);
        if (per_sm < 0) return per_sm;
        kern<<<per_sm * e->sms, NT, smem, e->stream>>>(acc, e->tree_ent[pol][2].as<int2>(), cnt + 2, ctr + 1);
    } else if constexpr (sizeof(Real) == 4) {
        auto kern = k_tree_far2<R / 2, NT, EngineTreeAcc>;
        const int smem = (int)tree_far2_smem(std::max(1, e->tree_np[pol]));   // the largest proxy count admitted
        const int per_sm = far_per_sm(kern, NT, smem, (int)tree_far2_smem(), cache);
        if (per_sm < 0) return per_sm;
        kern<<<per_sm * e->sms, NT, smem, e->stream>>>(acc, e->tree_ent[pol][2].as<int2>(), cnt + 2, ctr + 1, pol);
    } else {
        auto kern = k_tree_far<Real, R, NT, EngineTreeAcc>;
        const int per_sm = far_per_sm(kern, NT, (int)tree_far_smem<Real>(), (int)tree_far_smem<Real>(), cache);
        if (per_sm < 0) return per_sm;
        kern<<<per_sm * e->sms, NT, tree_far_smem<Real>(), e->stream>>>(acc, e->tree_ent[pol][2].as<int2>(),
                                                                       cnt + 2, ctr + 1, pol);
    }
    CTR_LAUNCHED();
    return CTR_OK;
}

int launch_trees(Engine* e, int half) {
    if (!e->any_tree) return CTR_OK;
    CTR_TRY((launch_tree_engine<float, kTreeR[0], kTreeNT[0]>(e, 0, half, CTR_FP32_REFINE)));
    CTR_TRY((launch_tree_engine<double, kTreeR[1], kTreeNT[1]>(e, 1, half, CTR_DF64)));
    CTR_TRY((launch_tree_engine<double, kTreeR[2], kTreeNT[2]>(e, 2, half, CTR_FP64)));
    return CTR_OK;
}

// One persistent FP32 launch per kernel variant among the occupied slots
int launch_fp32(Engine* e, int half) {
    for (int v = 0; v < kNV; ++v)
        if (e->var_used[v]) CTR_TRY(with_var32(v, PersistentRun{e, v, half}));
    return CTR_OK;
}

}  // namespace

// ---------------------------------------------------------------- host side
static int policy_index(int prec) { return prec == CTR_FP32_REFINE ? 0 : (prec == CTR_DF64 ? 1 : 2); }

Engine::~Engine() {
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    if (stream) {
        cudaStreamSynchronize(stream);
        cudaStreamDestroy(stream);
    }
}

int engine_create(int device, int cap, Engine** out) {
    Engine* e = new Engine();
    e->device = device;
    e->cap = cap;
    if (cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete e;
        return fail(CTR_ERR_CUDA, "stream create");
    }
    cudaStream_t stream = e->stream;
    e->host.assign(cap, SlotDev{});
    e->owner.assign(cap, nullptr);
    auto bad = [&](int st) {
        delete e;
        return st;
    };
    int st;
    if ((st = e->slots.alloc(sizeof(SlotDev) * cap)) < 0) return bad(st);
    if ((st = e->stats.alloc(sizeof(SlotStat) * cap)) < 0) return bad(st);
    if ((st = e->n_items.alloc(sizeof(int) * 3 * kNV)) < 0) return bad(st);
    if ((st = e->counters.alloc(sizeof(int) * 2 * 3 * kNV)) < 0) return bad(st);
    if ((st = e->tree_cnt.alloc(sizeof(int) * 9)) < 0) return bad(st);
    if ((st = e->tree_counters.alloc(sizeof(int) * 12)) < 0) return bad(st);
    if (cudaMemsetAsync(e->tree_cnt.p, 0, sizeof(int) * 9, stream) != cudaSuccess)
        return bad(fail(CTR_ERR_CUDA, "memset"));
    if ((st = e->err.alloc(sizeof(int))) < 0) return bad(st);
    if ((st = e->need.alloc(sizeof(int) * 3)) < 0) return bad(st);
    if (cudaMemsetAsync(e->err.p, 0, sizeof(int), stream) != cudaSuccess) return bad(fail(CTR_ERR_CUDA, "memset"));
    if (cudaMemsetAsync(e->n_items.p, 0, sizeof(int) * 3 * kNV, stream) != cudaSuccess)
        return bad(fail(CTR_ERR_CUDA, "memset"));
    for (int q = 0; q < cap; ++q) e->host[q].stat.state = kSlotEmpty;
    if (cudaMemcpyAsync(e->slots.p, e->host.data(), sizeof(SlotDev) * cap, cudaMemcpyHostToDevice, stream) !=
        cudaSuccess)
        return bad(fail(CTR_ERR_CUDA, "slot upload"));
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return bad(fail(CTR_ERR_CUDA, "attribute"));
    e->sms = sms;
    if ((st = exp_table(device, &e->exp_tab)) < 0) return bad(st);
    if (cudaStreamSynchronize(stream) != cudaSuccess) return bad(fail(CTR_ERR_CUDA, "sync"));
    *out = e;
    return CTR_OK;
}

// Treecode work lists per pair arithmetic (moment chunks, far clusters, far items of every occupied
// treecode slot), sorted by decreasing cost like the pair items.
static int rebuild_tree_items(Engine* e) {
    bool any = false;
    int counts[9] = {0};
    int np_max[3] = {0, 0, 0};
    for (int p = 0; p < 3; ++p) {
        struct It {
            int2 v;
            double cost;
        };
        std::vector<It> lists[3];
        for (int q = 0; q < e->cap; ++q) {
            ctr_ibim* h = e->owner[q];
            if (!h || !h->tree) continue;
            any = true;
            const SlotDev& s = e->host[q];
            if (policy_index(s.inner_prec) != p && policy_index(s.res_prec) != p) continue;
            const TreeData::Pol& P = h->tree->pol[p];
            np_max[p] = std::max(np_max[p], P.np);
            for (size_t k = 0; k < P.chunks.size(); ++k) lists[0].push_back(It{make_int2(q, (int)k), P.chunk_cost[k]});
            for (int k = 0; k < P.nq; ++k) lists[1].push_back(It{make_int2(q, k), 1.0});
            for (size_t k = 0; k < P.far.size(); ++k) lists[2].push_back(It{make_int2(q, (int)k), P.far_cost[k]});
        }
        for (int k = 0; k < 3; ++k) {
            std::stable_sort(lists[k].begin(), lists[k].end(), [](const It& a, const It& b) { return a.cost > b.cost; });
            std::vector<int2> v(lists[k].size());
            for (size_t i = 0; i < v.size(); ++i) v[i] = lists[k][i].v;
            if ((int64_t)v.size() > e->tree_cap[p][k] || !e->tree_ent[p][k].p) {
                const int64_t capn = std::max<int64_t>(256, (int64_t)v.size() * 2);
                CTR_TRY(e->tree_ent[p][k].alloc(sizeof(int2) * capn));
                e->tree_cap[p][k] = capn;
                e->graph_dirty = true;   // the entry buffer moved
            }
            if (!v.empty())
                CTR_CUDA_TRY(cudaMemcpyAsync(e->tree_ent[p][k].p, v.data(), sizeof(int2) * v.size(),
                                             cudaMemcpyHostToDevice, e->stream));
            counts[3 * p + k] = (int)v.size();
        }
    }
    CTR_CUDA_TRY(cudaMemcpyAsync(e->tree_cnt.p, counts, sizeof(counts), cudaMemcpyHostToDevice, e->stream));
    CTR_CUDA_TRY(cudaStreamSynchronize(e->stream));
    if (any != e->any_tree) {
        e->any_tree = any;
        e->graph_dirty = true;   // the step gains or loses the treecode launches
    }
    for (int p = 0; p < 3; ++p)
        if (np_max[p] != e->tree_np[p]) {
            e->tree_np[p] = np_max[p];
            e->graph_dirty = true;   // the far kernels' shared memory changes
        }
    return CTR_OK;
}

// Rebuild the work lists (every item of every occupied slot's schedule, one list per arithmetic and
// kernel variant; each entry is filtered by its slot's state and part at run time), in decreasing cost
// for the atomic-counter scheduler: each slot's items are already in that order, so the lists are a
// merge of the slots' sequences (ties: lower slot, then lower item first).  A slot whose application
// is split gets its items dealt to the parts in that order, back and forth (0, 1, .., n-1, n-1, .., 0),
// which balances the parts' costs.
static int rebuild_items(Engine* e) {
    bool used[kNV] = {};
    for (int p = 0; p < 3; ++p) {
        struct Seq {
            int q, np;
            const std::vector<double>* cost;
        };
        std::vector<Seq> seqs[kNV];
        for (int q = 0; q < e->cap; ++q) {
            if (!e->owner[q]) continue;
            const SlotDev& s = e->host[q];
            const bool uses = (policy_index(s.inner_prec) == p) || (policy_index(s.res_prec) == p);
            if (!uses) continue;
            const PairSchedule& sc = e->owner[q]->sched[p];
            if (sc.items.size() > (size_t)kItemMask) return fail(CTR_ERR_CAPACITY, "engine: schedule too long");
            const int var = (p == 0) ? sc.var : 0;
            if (p == 0) used[var] = true;
            seqs[var].push_back(Seq{q, std::max(1, s.nparts[p]), &sc.cost});
        }
        // one set of pair constants for every slot of this arithmetic: pass it as a launch parameter
        bool shared = true, any = false;
        PairConsts val{};
        for (int q = 0; q < e->cap && shared; ++q) {
            if (!e->owner[q]) continue;
            const SlotDev& s = e->host[q];
            if (policy_index(s.inner_prec) != p && policy_index(s.res_prec) != p) continue;
            PairConsts c = s.kc;
            c.exp_tab = e->exp_tab;
            if (!any) {
                val = c;
                any = true;
            } else if (std::memcmp(&val, &c, sizeof(PairConsts)) != 0) {
                shared = false;
            }
        }
        if (!any) val.exp_tab = e->exp_tab;
        if (shared != e->kc_shared[p] || std::memcmp(&val, &e->kc_val[p], sizeof(PairConsts)) != 0) {
            e->kc_shared[p] = shared;
            e->kc_val[p] = val;
            e->graph_dirty = true;   // the captured launches carry the constants
        }
        for (int v = 0; v < kNV; ++v) {
            size_t total = 0;
            for (const Seq& a : seqs[v]) total += a.cost->size();
            std::vector<int2> ent;
            ent.reserve(total);
            std::vector<size_t> pos(seqs[v].size(), 0);
            auto later = [&](int a, int b) {   // heap order: the entry to take next on top
                const double ca = (*seqs[v][a].cost)[pos[a]], cb = (*seqs[v][b].cost)[pos[b]];
                return ca != cb ? ca < cb : a > b;
            };
            std::vector<int> heap;
            for (int a = 0; a < (int)seqs[v].size(); ++a)
                if (!seqs[v][a].cost->empty()) heap.push_back(a);
            std::make_heap(heap.begin(), heap.end(), later);
            while (!heap.empty()) {
                std::pop_heap(heap.begin(), heap.end(), later);
                const int a = heap.back();
                const Seq& sq = seqs[v][a];
                const size_t k = pos[a];
                const int round = (int)(k / (size_t)sq.np), at = (int)(k % (size_t)sq.np);
                const int part = (round & 1) ? sq.np - 1 - at : at;
                ent.push_back(make_int2(sq.q, (int)k | (part << kPartShift)));
                if (++pos[a] < sq.cost->size()) std::push_heap(heap.begin(), heap.end(), later);
                else heap.pop_back();
            }
            if ((int64_t)ent.size() > e->item_cap[p][v]) {
                const int64_t capn = std::max<int64_t>(1024, (int64_t)ent.size() * 2);
                CTR_TRY(e->items[p][v].alloc(sizeof(int2) * capn));
                e->item_cap[p][v] = capn;
                e->graph_dirty = true;   // the item buffer moved
            }
            if (!ent.empty())
                CTR_CUDA_TRY(cudaMemcpyAsync(e->items[p][v].p, ent.data(), sizeof(int2) * ent.size(),
                                             cudaMemcpyHostToDevice, e->stream));
            const int cnt = (int)ent.size();
            CTR_CUDA_TRY(cudaMemcpyAsync(e->n_items.as<int>() + p * kNV + v, &cnt, sizeof(int), cudaMemcpyHostToDevice,
                                         e->stream));
        }
        CTR_CUDA_TRY(cudaStreamSynchronize(e->stream));
    }
    for (int v = 0; v < kNV; ++v)
        if (used[v] != e->var_used[v]) {
            e->var_used[v] = used[v];
            e->graph_dirty = true;   // the step gains or loses a variant's launches
        }
    return rebuild_tree_items(e);
}

// The kernels of one engine step, in stream order (captured into the graph).
static int enqueue_step(Engine* e) {
    cudaStream_t st = e->stream;
    SlotDev* S = e->slots.as<SlotDev>();
    const int cap = e->cap;
    const int mx = e->max_nblk;
    const dim3 vec(e->vec_blocks, cap);
    const unsigned one = grid_for(cap, 128);
    k_plan_step<<<1, kVecThreads, 0, st>>>(S, cap);
    CTR_LAUNCHED();
    // ---- inner half: one Arnoldi iteration
    k_prep_inner<<<vec, kVecThreads, 0, st>>>(S);
    CTR_LAUNCHED();
    CTR_CUDA_TRY(cudaMemsetAsync(e->counters.p, 0, sizeof(int) * 2 * 3 * kNV, st));
    if (e->any_tree) CTR_CUDA_TRY(cudaMemsetAsync(e->tree_counters.p, 0, sizeof(int) * 12, st));
    k_need<<<1, kVecThreads, 0, st>>>(S, cap, 0, e->need.as<int>());
    CTR_LAUNCHED();
    CTR_TRY(launch_fp32(e, 0));
    CTR_TRY((launch_persistent<Df64Policy, kRdf, kChunkDf, 1>(e, 1, 0, 0, CTR_DF64)));
    CTR_TRY((launch_persistent<Fp64Policy, kR64, kChunk64, 1>(e, 2, 0, 0, CTR_FP64)));
    CTR_TRY(launch_trees(e, 0));
    k_part<<<one, 128, 0, st>>>(S, cap, 0);
    CTR_LAUNCHED();
    k_finish<<<vec, kVecThreads, 0, st>>>(S, 0);
    CTR_LAUNCHED();
    for (int pass = 0; pass < 2; ++pass) {
        k_dots_partial<<<dim3(mx, cap), kVecThreads, 0, st>>>(S, pass);
        CTR_LAUNCHED();
        k_dots_final<<<dim3(e->max_m + 1, cap), kVecThreads, 0, st>>>(S, pass);
        CTR_LAUNCHED();
        k_sub<<<vec, kVecThreads, 0, st>>>(S, pass);
        CTR_LAUNCHED();
    }
    k_dots_partial<<<dim3(mx, cap), kVecThreads, 0, st>>>(S, 2);
    CTR_LAUNCHED();
    k_dots_final<<<dim3(1, cap), kVecThreads, 0, st>>>(S, 2);
    CTR_LAUNCHED();
    k_givens<<<one, 128, 0, st>>>(S, cap);
    CTR_LAUNCHED();
    k_scale_next<<<vec, kVecThreads, 0, st>>>(S);
    CTR_LAUNCHED();
    k_advance<<<one, 128, 0, st>>>(S, cap);
    CTR_LAUNCHED();
    // ---- update half: x, true residual, next cycle
    k_upper_solve<<<one, 128, 0, st>>>(S, cap);
    CTR_LAUNCHED();
    k_update_x<<<vec, kVecThreads, 0, st>>>(S);
    CTR_LAUNCHED();
    k_need<<<1, kVecThreads, 0, st>>>(S, cap, 1, e->need.as<int>());
    CTR_LAUNCHED();
    CTR_TRY(launch_fp32(e, 1));
    CTR_TRY((launch_persistent<Df64Policy, kRdf, kChunkDf, 1>(e, 1, 0, 1, CTR_DF64)));
    CTR_TRY((launch_persistent<Fp64Policy, kR64, kChunk64, 1>(e, 2, 0, 1, CTR_FP64)));
    CTR_TRY(launch_trees(e, 1));
    k_part<<<one, 128, 0, st>>>(S, cap, 1);
    CTR_LAUNCHED();
    k_finish<<<vec, kVecThreads, 0, st>>>(S, 1);
    CTR_LAUNCHED();
    k_dots_partial<<<dim3(mx, cap), kVecThreads, 0, st>>>(S, 3);
    CTR_LAUNCHED();
    k_dots_final<<<dim3(1, cap), kVecThreads, 0, st>>>(S, 3);
    CTR_LAUNCHED();
    k_decide<<<one, 128, 0, st>>>(S, cap);
    CTR_LAUNCHED();
    k_start_vec<<<vec, kVecThreads, 0, st>>>(S);
    CTR_LAUNCHED();
    k_start_scalars<<<one, 128, 0, st>>>(S, cap);
    CTR_LAUNCHED();
    k_stats<<<one, 128, 0, st>>>(S, cap, e->stats.as<SlotStat>());
    CTR_LAUNCHED();
    return CTR_OK;
}

static int ensure_graph(Engine* e) {
    if (e->graph_exec && !e->graph_dirty) return CTR_OK;
    if (e->graph_exec) {
        cudaGraphExecDestroy(e->graph_exec);
        e->graph_exec = nullptr;
    }
    if (!e->use_graph) return CTR_OK;
    cudaGraph_t g = nullptr;
    const int64_t before = ctr_kernel_launches();
    CTR_CUDA_TRY(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
    const int st = enqueue_step(e);
    e->kernels_per_step = ctr_kernel_launches() - before;
    cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
    if (st < 0) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (ce != cudaSuccess) return fail(CTR_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&e->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return fail(CTR_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
    e->graph_dirty = false;
    return CTR_OK;
}

int engine_admit(Engine* e, ctr_ibim* s, int* slot_out) {
    int q = -1;
    for (int i = 0; i < e->cap; ++i)
        if (!e->owner[i]) {
            q = i;
            break;
        }
    if (q < 0) return fail(CTR_ERR_CAPACITY, "no free engine slot");
    CTR_TRY(engine_prepare_handle(s));
    SlotDev d{};
    d.M = (int)s->M;
    d.n = 2 * s->M;
    d.E = (int)s->E;
    d.m = s->kr.m;
    d.nblk = s->kr.nblk;
    d.W = s->na.W;
    d.cptr = s->corr_ptr.as<int32_t>();
    d.cnode = s->corr_node.as<int32_t>();
    d.cw = s->corr_w.as<double>();
    d.excl = s->tree ? s->tree->d_excl.as<int32_t>() : s->excl.as<int32_t>();
    d.eptr = s->tree ? s->tree->d_eptr.as<int32_t>() : s->corr_ptr.as<int32_t>();
    d.tinv = s->tree ? s->tree->d_tinv.as<int32_t>() : nullptr;
    if (s->tree) d.tv = s->tree->view;
    d.src32 = s->src32.as<float4>();
    d.src64 = s->src64.as<double4>();
    d.srcdf = s->srcdf.as<float4>();
    d.acc = s->acc.as<unsigned long long>();
    d.g = s->rhs.as<double>();
    d.lam1 = 0.5 * (1.0 + s->eps_out / s->eps_in);
    d.lam2 = 0.5 * (1.0 + s->eps_in / s->eps_out);
    d.il1 = 2.0 / (1.0 + s->eps_out / s->eps_in);
    d.il2 = 2.0 / (1.0 + s->eps_in / s->eps_out);
    d.h2 = s->h * s->h;
    d.h3 = s->h * s->h * s->h;
    d.scale = s->h * s->h * s->h / (4.0 * kPi);
    d.refine = (s->opt.precision == CTR_FP32_REFINE) ? 1 : 0;
    d.inner_prec = s->opt.precision;
    d.res_prec = d.refine ? s->opt.residual : s->opt.precision;
    // a treecode handle's FP32 operator carries its own approximation error (degree 6): its refinement
    // residuals are always formed in full with the residual arithmetic
    d.res_update = (d.refine && s->opt.residual_mode == CTR_RESIDUAL_UPDATE && !s->tree) ? 1 : 0;
    // the slot's two arithmetics were planned at setup from the same options: these are guards
    CTR_TRY(ensure_schedule(s, policy_index(d.inner_prec)));
    CTR_TRY(ensure_schedule(s, policy_index(d.res_prec)));
    d.upd = 0;
    d.part = 0;
    for (int p = 0; p < 3; ++p) {   // parts of one application (treecode handles: always whole)
        const PairSchedule& sc = s->sched[p];
        int64_t np = 1;
        if (e->quantum_s > 0.0 && !s->tree) {
            // a part lasts at least as long as its longest item runs on one block (kItemSeconds): keep
            // every part at twice that or more, and at kMinItemsPerPart items or more
            const double t = sc.total_cost / kUnitRate[p];
            np = (int64_t)std::ceil(t / e->quantum_s);
            np = std::min<int64_t>(np, (int64_t)(t / (2.0 * kItemSeconds[p])));
            np = std::min<int64_t>(np, (int64_t)sc.items.size() / kMinItemsPerPart);
        }
        d.nparts[p] = (int)std::max<int64_t>(1, std::min<int64_t>(np, kMaxParts));
        d.part_s[p] = (float)(sc.total_cost / kUnitRate[p] / d.nparts[p]);
    }
    d.span = 1;
    CTR_TRY(pair_consts(s, true, &d.kc));
    for (int p = 0; p < 3; ++p) {
        d.items[p] = s->sched[p].d_items.as<PairItem>();
        d.BS[p] = s->sched[p].BS;
    }
    double* b = s->vecs.as<double>();
    const int64_t n = d.n;
    d.x = b;
    d.r = b + n;
    d.z = b + 2 * n;
    d.V = s->kr.V.as<double>();
    d.H = s->kr.H.as<double>();
    d.cs = s->kr.cs.as<double>();
    d.sn = s->kr.sn.as<double>();
    d.sv = s->kr.s.as<double>();
    d.y = s->kr.y.as<double>();
    d.cgs = s->kr.y.as<double>() + (d.m + 1);
    d.cgs2 = s->kr.y.as<double>() + 2 * (d.m + 1);
    d.dpart = s->kr.part.as<double>();
    d.scal = s->kr.scal.as<double>();
    d.tol_out = s->opt.tol;
    d.inner_tol = s->opt.inner_tol;
    d.max_refine = s->opt.max_refine;
    d.budget = s->opt.max_iter;
    // initial residual r = g (x = 0) and its norm
    CTR_CUDA_TRY(cudaStreamSynchronize(s->stream));   // the handle's setup work is complete
    CTR_CUDA_TRY(cudaMemsetAsync(d.x, 0, sizeof(double) * n, e->stream));
    CTR_CUDA_TRY(cudaMemcpyAsync(d.r, d.g, sizeof(double) * n, cudaMemcpyDeviceToDevice, e->stream));
    double gn2 = 0.0;
    CTR_TRY(device_dot(s, d.g, d.g, n, &gn2));
    d.gnorm = std::sqrt(gn2);
    d.beta = d.gnorm;
    d.tol_cycle = d.refine ? d.inner_tol * d.gnorm : d.tol_out * d.gnorm;
    d.stat = SlotStat{};
    if (d.gnorm == 0.0) {
        d.stat.state = kSlotDone;
        d.stat.converged = 1;
    } else {
        d.stat.state = kSlotStart;
    }
    e->host[q] = d;
    e->owner[q] = s;
    CTR_CUDA_TRY(cudaMemcpyAsync(e->slots.as<SlotDev>() + q, &d, sizeof(SlotDev), cudaMemcpyHostToDevice, e->stream));
    CTR_CUDA_TRY(cudaMemcpyAsync(e->stats.as<SlotStat>() + q, &d.stat, sizeof(SlotStat), cudaMemcpyHostToDevice,
                                 e->stream));
    if (d.stat.state == kSlotStart) {
        k_start_vec<<<dim3(e->vec_blocks, e->cap), kVecThreads, 0, e->stream>>>(e->slots.as<SlotDev>());
        CTR_LAUNCHED();
        k_start_scalars<<<grid_for(e->cap, 128), 128, 0, e->stream>>>(e->slots.as<SlotDev>(), e->cap);
        CTR_LAUNCHED();
    }
    if (d.nblk > e->max_nblk) {   // launch shapes of the captured step change
        e->max_nblk = d.nblk;
        e->graph_dirty = true;
    }
    if (d.m > e->max_m) {
        e->max_m = d.m;
        e->graph_dirty = true;
    }
    const int vb = (int)std::min<int64_t>(grid_for(s->M, kVecThreads), 1024);
    if (vb > e->vec_blocks) {
        e->vec_blocks = vb;
        e->graph_dirty = true;
    }
    e->lists_dirty = true;   // the work lists gain its items before the next step
    *slot_out = q;
    return CTR_OK;
}

int engine_retire(Engine* e, int q, ctr_solve_info* info) {
    if (q < 0 || q >= e->cap || !e->owner[q]) return fail(CTR_ERR_INVALID, "bad slot");
    SlotStat st;
    CTR_CUDA_TRY(cudaMemcpyAsync(&st, e->stats.as<SlotStat>() + q, sizeof(SlotStat), cudaMemcpyDeviceToHost, e->stream));
    CTR_CUDA_TRY(cudaStreamSynchronize(e->stream));
    if (st.state == kSlotInnerWait || st.state == kSlotUpdateWait) {
        // retired between two parts of an application (cancelled): its node accumulators hold partial
        // sums; clear them so the handle's next application starts from zero
        ctr_ibim* h = e->owner[q];
        CTR_CUDA_TRY(cudaMemsetAsync(h->acc.p, 0, h->acc.bytes, e->stream));
        CTR_CUDA_TRY(cudaStreamSynchronize(e->stream));
    }
    if (info) {
        info->iterations = st.iterations;
        info->refinements = st.refinements;
        info->matvecs_fp32 = st.matvecs_fp32;
        info->matvecs_fp64 = st.matvecs_fp64;
        info->residual = st.residual;
        info->converged = st.converged;
    }
    SlotDev empty{};
    empty.stat.state = kSlotEmpty;
    e->host[q] = empty;
    e->owner[q] = nullptr;
    CTR_CUDA_TRY(cudaMemcpyAsync(e->slots.as<SlotDev>() + q, &empty, sizeof(SlotDev), cudaMemcpyHostToDevice, e->stream));
    e->lists_dirty = true;   // its entries are inert (an empty slot matches no state) until the next rebuild
    return st.numeric_error ? fail(CTR_ERR_NUMERIC, "non-finite residual") : CTR_OK;
}

int engine_step(Engine* e, std::vector<SlotStat>* stats) {
    if (e->lists_dirty) {   // one rebuild for all admissions and retirements since the last step
        CTR_TRY(rebuild_items(e));
        e->lists_dirty = false;
    }
    CTR_TRY(ensure_graph(e));
    if (e->graph_exec) {
        CTR_CUDA_TRY(cudaGraphLaunch(e->graph_exec, e->stream));
        count_launches(e->kernels_per_step);   // kernels run by the replay
    } else {
        CTR_TRY(enqueue_step(e));
    }
    stats->resize(e->cap);
    CTR_CUDA_TRY(cudaMemcpyAsync(stats->data(), e->stats.p, sizeof(SlotStat) * e->cap, cudaMemcpyDeviceToHost, e->stream));
    CTR_CUDA_TRY(cudaStreamSynchronize(e->stream));
    int herr = 0;
    CTR_CUDA_TRY(cudaMemcpyAsync(&herr, e->err.p, sizeof(int), cudaMemcpyDeviceToHost, e->stream));
    CTR_CUDA_TRY(cudaStreamSynchronize(e->stream));
    if (herr) return fail(CTR_ERR_DEVICE_WAIT, "engine: a bounded device wait expired");
    e->steps++;
    return CTR_OK;
}

// The handle's solver workspace, sized for the engine (Krylov basis, vectors).
int engine_prepare_handle(ctr_ibim* s) {
    CTR_TRY(ensure_krylov_public(s));
    return CTR_OK;
}

// Solve every handle to completion in one engine (all slots admitted at once).
int engine_solve_all(ctr_ibim* const* hs, int64_t n, int use_graph, std::vector<ctr_solve_info>* infos,
                     int64_t* steps) {
    if (n <= 0) return CTR_OK;
    Engine* e = nullptr;
    CTR_TRY(engine_create(hs[0]->device, (int)n, &e));
    std::unique_ptr<Engine> guard(e);
    e->use_graph = use_graph != 0;
    e->vec_blocks = 1;
    for (int64_t i = 0; i < n; ++i)
        e->vec_blocks = std::max<int>(e->vec_blocks, (int)std::min<int64_t>(grid_for(hs[i]->M, kVecThreads), 1024));
    std::vector<int> slot(n);
    for (int64_t i = 0; i < n; ++i) CTR_TRY(engine_admit(e, hs[i], &slot[i]));
    infos->assign(n, ctr_solve_info{});
    std::vector<int> state(n);
    for (int64_t i = 0; i < n; ++i) state[i] = e->host[slot[i]].stat.state == kSlotDone ? kSlotDone : kSlotInner;
    std::vector<char> done(n, 0);
    std::vector<SlotStat> st;
    int first_error = CTR_OK;
    for (;;) {
        for (int64_t i = 0; i < n; ++i) {
            if (!done[i] && state[i] == kSlotDone) {
                const int r = engine_retire(e, slot[i], &(*infos)[i]);
                if (r < 0 && first_error == CTR_OK) first_error = r;
                done[i] = 1;
            }
        }
        bool left = false;
        for (int64_t i = 0; i < n; ++i) left |= !done[i];
        if (!left) break;
        CTR_TRY(engine_step(e, &st));
        for (int64_t i = 0; i < n; ++i)
            if (!done[i]) state[i] = st[slot[i]].state;
    }
    if (steps) *steps = e->steps;
    return first_error;
}

}  // namespace ctr
