// Far-field acceleration of the dense sum (the fast summation of K v inside
// GMRES, Sec. 2.5): the device kernels of the particle-cluster treecode.
//
// A far cluster C of a target block is replaced by the tensor Chebyshev
// points s_k of its box (k = (k3 n1 + k2) n1 + k1) carrying the charges of
// the interpolated source variable, G(x, y) ~ sum_k G(x, s_k) L_k(y):
//   Dk = sum_j a_j n_j . grad L_k(P_j),   Sk = sum_j b_j L_k(P_j)
//   (a = h^3 W rho1 / 4 pi, b = h^3 W rho2 / 4 pi, the packed source weights),
//   Q0 = Dk - Sk,  Qk = -(eps_E/eps_I) Dk + Sk,  Qk' = -Dk + (eps_I/eps_E) Sk,
// and a target (x, n_x) of the block receives, from K11..K22 of Eq. (1.4),
//   out1 += sum_k Q0/r + Qk e^{-kappa r}/r,
//   out2 += sum_k -(d . n_x)/r^3 (Q0 + (1 + kappa r) e^{-kappa r} Qk'),
// with d = x - s_k, r = |d|.  Three kernels per pair arithmetic:
//   k_tree_mom     Dk, Sk of one chunk of a cluster's sources (per-source
//                  barycentric basis and derivative in shared memory; each
//                  thread owns one (k2, k3) row of proxies);
//   k_tree_momred  the chunks of a cluster added in a fixed order, Q formed;
//   k_tree_far2    far items (target block x a run of its far clusters) of the
//                  FP32 operator: FP32 charges, two targets per f32x2
//                  instruction; the cluster's proxies and charges in shared
//                  memory, FP32 sums per cluster folded into FP64 per target,
//                  added into the nodes' exact accumulators like a pair item's;
//   k_tree_far_ff  the same for the float-float operator: FP64 moments of the
//                  full float-float sources, charges and proxies split into
//                  float-float, every evaluation in float-float arithmetic
//                  (about 2^-44 relative, like its pair terms);
//   k_tree_far     the same in scalar FP64 arithmetic (FP64 operator).
// The blocks of each kernel take work entries (handle, index) from a list
// through an atomic counter; `Acc` maps an entry's handle to its TreeView (or
// to nothing when that handle is not in this pass).
#pragma once

#include <map>
#include <mutex>

#include "common.cuh"
#include "pairkern.cuh"

namespace ctr {

using pk::kThreads;

constexpr int kMomTile = 32;      // sources per shared tile of the moment kernel
// far kernel shape per pair arithmetic: R targets per thread x NT threads = the target block
// (FP32 charges: packed pairs of targets, R / 2 per thread; FP64: scalar)
constexpr int kTreeR[3] = {4, 2, 1};
constexpr int kTreeNT[3] = {256, 128, 256};
constexpr int kChunkSrc = 2048;   // sources per moment chunk

// Float-float sums of two values that cannot cancel (same sign), left unnormalised like pk::mull's
// products: exact two_sum of the high parts, plain sum of the low parts.
__device__ __forceinline__ pk::F2 ff_addl(pk::F2 a, pk::F2 b) {
    const pk::F2 s = pk::two_sum(a.hi, b.hi);
    return pk::F2{s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo))};
}
__device__ __forceinline__ pk::F2 ff_add_fl(pk::F2 a, float b) {
    const pk::F2 s = pk::two_sum(a.hi, b);
    return pk::F2{s.hi, __fadd_rn(s.lo, a.lo)};
}

template <typename Real>
__device__ __forceinline__ void tree_source(const TreeView& t, int pol, int64_t p, Real P[3], Real n[3], Real& a,
                                            Real& b) {
    if (pol == 2) {
        const double4 u = t.src64[2 * p], v = t.src64[2 * p + 1];
        P[0] = (Real)u.x, P[1] = (Real)u.y, P[2] = (Real)u.z, a = (Real)u.w;
        n[0] = (Real)v.x, n[1] = (Real)v.y, n[2] = (Real)v.z, b = (Real)v.w;
    } else if (pol == 1) {   // float-float sources: hi + lo in FP64, the leading floats in FP32
        const float4 u = t.srcdf[4 * p], v = t.srcdf[4 * p + 2];
        P[0] = (Real)u.x, P[1] = (Real)u.y, P[2] = (Real)u.z, a = (Real)u.w;
        n[0] = (Real)v.x, n[1] = (Real)v.y, n[2] = (Real)v.z, b = (Real)v.w;
        if constexpr (sizeof(Real) == 8) {
            const float4 ul = t.srcdf[4 * p + 1], vl = t.srcdf[4 * p + 3];
            P[0] += (Real)ul.x, P[1] += (Real)ul.y, P[2] += (Real)ul.z, a += (Real)ul.w;
            n[0] += (Real)vl.x, n[1] += (Real)vl.y, n[2] += (Real)vl.z, b += (Real)vl.w;
        }
    } else {                 // duplicated f32x2 layout {x,x,y,y}{z,z,a,a}{nx,nx,ny,ny}{nz,nz,-b,-b}
        const float4 u0 = t.src32[4 * p], u1 = t.src32[4 * p + 1], u2 = t.src32[4 * p + 2],
                     u3 = t.src32[4 * p + 3];
        P[0] = (Real)u0.x, P[1] = (Real)u0.z, P[2] = (Real)u1.x, a = (Real)u1.z;
        n[0] = (Real)u2.x, n[1] = (Real)u2.z, n[2] = (Real)u3.x, b = -(Real)u3.z;
    }
}

// The next work entry of this block from the atomic counter (block-uniform).
__device__ __forceinline__ int tree_next(int* counter, int* cur) {
    if (threadIdx.x == 0) *cur = atomicAdd(counter, 1);
    __syncthreads();
    const int it = *cur;
    __syncthreads();
    return it;
}

// ---------------------------------------------------------------- moments of one chunk
template <typename Real, class Acc>
__global__ void __launch_bounds__(kThreads) k_tree_mom(Acc acc, const int2* __restrict__ ent,
                                                    const int* __restrict__ n_ent, int* __restrict__ counter,
                                                    int pol) {
    __shared__ Real xr[kTreeMaxN1], bw[kTreeMaxN1], dr[kTreeMaxN1 * kTreeMaxN1];
    __shared__ Real L[3][kMomTile][kTreeMaxN1], G[3][kMomTile][kTreeMaxN1], BL[kMomTile][kTreeMaxN1];
    __shared__ int cur;
    const int tid = threadIdx.x;
    const int total = *n_ent;
    for (;;) {
        const int it = tree_next(counter, &cur);
        if (it >= total) break;
        const int2 w = ent[it];
        const TreeView* tp = acc.view(w.x);
        if (!tp) continue;   // block-uniform
        const TreeView& t = *tp;
        const int n1 = t.n1[pol], np = t.np[pol];
        const MomChunk ch = t.chunks[pol][w.y];
        for (int i = tid; i < n1; i += kThreads) {
            xr[i] = (Real)t.xref[pol][i];
            bw[i] = (Real)t.bw[pol][i];
        }
        for (int i = tid; i < n1 * n1; i += kThreads) dr[i] = (Real)t.dref[pol][i];
        const double* bx = t.box[pol] + 6 * (int64_t)ch.q;
        Real accD[kTreeMaxN1], accS[kTreeMaxN1];
#pragma unroll
        for (int k = 0; k < kTreeMaxN1; ++k) accD[k] = accS[k] = (Real)0;
        const int row = tid;                  // proxy row (k2, k3) = (row % n1, row / n1)
        const bool owner = row < n1 * n1;
        const int k2 = owner ? row % n1 : 0, k3 = owner ? row / n1 : 0;
        __syncthreads();
        for (int j0 = ch.j0; j0 < ch.j1; j0 += kMomTile) {
            const int nt = min(kMomTile, ch.j1 - j0);
            if (tid < 3 * kMomTile) {
                const int s = tid % kMomTile, ax = tid / kMomTile;
                Real l[kTreeMaxN1];
                Real coef = (Real)0, bcoef = (Real)0;
#pragma unroll
                for (int m = 0; m < kTreeMaxN1; ++m) l[m] = (Real)0;
                if (s < nt) {
                    Real P[3], n[3], a, b;
                    tree_source<Real>(t, pol, j0 + s, P, n, a, b);
                    const Real c = (Real)bx[ax], wd = (Real)bx[3 + ax];
                    const Real u = (P[ax] - c) / wd;
                    int hit = -1;
#pragma unroll
                    for (int m = 0; m < kTreeMaxN1; ++m)
                        if (m < n1 && u == xr[m]) hit = m;
                    if (hit >= 0) {
#pragma unroll
                        for (int m = 0; m < kTreeMaxN1; ++m) l[m] = (m == hit) ? (Real)1 : (Real)0;
                    } else {
                        Real den = (Real)0;
#pragma unroll
                        for (int m = 0; m < kTreeMaxN1; ++m)
                            if (m < n1) {
                                l[m] = bw[m] / (u - xr[m]);
                                den += l[m];
                            }
#pragma unroll
                        for (int m = 0; m < kTreeMaxN1; ++m)
                            if (m < n1) l[m] = l[m] / den;
                    }
                    coef = a * n[ax] / wd;
                    bcoef = b;
                }
                // basis, derivative (l' = l D / w, weighted by a n_ax) and b-weighted basis
#pragma unroll
                for (int q = 0; q < kTreeMaxN1; ++q) {
                    if (q >= n1) break;
                    Real gq = (Real)0;
#pragma unroll
                    for (int m = 0; m < kTreeMaxN1; ++m)
                        if (m < n1) gq += l[m] * dr[m * n1 + q];
                    L[ax][s][q] = l[q];
                    G[ax][s][q] = coef * gq;
                    if (ax == 0) BL[s][q] = bcoef * l[q];
                }
            }
            __syncthreads();
            if (owner) {
                for (int s = 0; s < nt; ++s) {
                    const Real l1 = L[1][s][k2], g1 = G[1][s][k2], l2 = L[2][s][k3], g2 = G[2][s][k3];
                    const Real y12 = l1 * l2;
                    const Real tt = g1 * l2 + l1 * g2;
#pragma unroll
                    for (int k1 = 0; k1 < kTreeMaxN1; ++k1) {
                        if (k1 < n1) {
                            accS[k1] += BL[s][k1] * y12;
                            accD[k1] += G[0][s][k1] * y12 + L[0][s][k1] * tt;
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (owner) {
            Real* out = static_cast<Real*>(t.mpart[pol]) + (size_t)w.y * 2 * np;
#pragma unroll
            for (int k1 = 0; k1 < kTreeMaxN1; ++k1) {
                if (k1 < n1) {
                    out[row * n1 + k1] = accD[k1];
                    out[np + row * n1 + k1] = accS[k1];
                }
            }
        }
    }
}

// ---------------------------------------------------------------- chunk sums -> charges
template <typename Real, class Acc>
__global__ void __launch_bounds__(kThreads) k_tree_momred(Acc acc, const int2* __restrict__ ent,
                                                       const int* __restrict__ n_ent, int pol) {
    const int total = *n_ent;
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int2 w = ent[it];
        const TreeView* tp = acc.view(w.x);
        if (!tp) continue;
        const TreeView& t = *tp;
        const int np = t.np[pol], q = w.y;
        const int c0 = t.cptr[pol][q], c1 = t.cptr[pol][q + 1];
        const Real* mp = static_cast<const Real*>(t.mpart[pol]);
        Real* Q = static_cast<Real*>(t.mom[pol]) + (size_t)q * 3 * np;
        for (int k = threadIdx.x; k < np; k += blockDim.x) {
            double D = 0.0, S = 0.0;
            for (int c = c0; c < c1; ++c) {
                D += (double)mp[(size_t)c * 2 * np + k];
                S += (double)mp[(size_t)c * 2 * np + np + k];
            }
            Q[k] = (Real)(D - S);
            Q[np + k] = (Real)(-t.c1 * D + S);
            Q[2 * np + k] = (Real)(-D + t.c2 * S);
        }
    }
}

// ---------------------------------------------------------------- far items
template <typename Real>
__device__ __forceinline__ void far_terms(Real dx, Real ryz, Real dyzn, Real nx, Real q0, Real qk, Real qk2,
                                          Real kappa, Real kl2, Real& a1, Real& a2) {
    const Real r2 = fma(dx, dx, ryz);
    const Real dn = fma(dx, nx, dyzn);
    Real ri, E;
    if constexpr (sizeof(Real) == 4) {
        ri = pk::rsqrt_sfu(r2);
        E = pk::ex2_sfu(kl2 * (r2 * ri));
    } else {
        ri = rsqrt(r2);
        E = exp(-kappa * (r2 * ri));
    }
    const Real r = r2 * ri;
    a1 = fma(ri, fma(E, qk, q0), a1);
    const Real f = E * fma(kappa, r, (Real)1);
    a2 = fma(-dn * (ri * ri * ri), fma(f, qk2, q0), a2);
}

template <typename Real>
constexpr size_t tree_far_smem() {
    return sizeof(Real) * (3 * kTreeMaxN1 + 3 * kTreeMaxNp);
}

// NT threads x R targets per thread cover one target block (NT * R = the arithmetic's block size).
template <typename Real, int R, int NT, class Acc>
__global__ void __launch_bounds__(NT) k_tree_far(Acc acc, const int2* __restrict__ ent,
                                              const int* __restrict__ n_ent, int* __restrict__ counter, int pol) {
    extern __shared__ __align__(16) unsigned char tree_smem[];
    Real* sx = reinterpret_cast<Real*>(tree_smem);         // [3][kTreeMaxN1]
    Real* sq = sx + 3 * kTreeMaxN1;                        // [3][np]
    __shared__ int cur;
    const int tid = threadIdx.x;
    const int total = *n_ent;
    for (;;) {
        const int it = tree_next(counter, &cur);
        if (it >= total) break;
        const int2 w = ent[it];
        const TreeView* tp = acc.view(w.x);
        if (!tp) continue;
        const TreeView& t = *tp;
        const int n1 = t.n1[pol], np = t.np[pol], M = t.M, BS = t.BS[pol];
        const FarItem f = t.far[pol][w.y];
        const Real kappa = (Real)t.kappa;
        const Real kl2 = (Real)(-t.kappa * 1.4426950408889634);
        Real px[R], py[R], pz[R], nx[R], ny[R], nz[R];
        double o1[R], o2[R];
        int64_t pp[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            pp[r] = (int64_t)f.I * BS + r * NT + tid;
            Real P[3], n[3], a, b;
            tree_source<Real>(t, pol, min(pp[r], (int64_t)M - 1), P, n, a, b);
            px[r] = P[0], py[r] = P[1], pz[r] = P[2];
            nx[r] = n[0], ny[r] = n[1], nz[r] = n[2];
            o1[r] = 0.0, o2[r] = 0.0;
        }
        for (int l = f.l0; l < f.l1; ++l) {
            const int q = t.flist[pol][l];
            __syncthreads();   // the previous cluster's proxies are no longer read
            const double* bx = t.box[pol] + 6 * (int64_t)q;
            for (int i = tid; i < 3 * n1; i += NT) {
                const int ax = i / n1, m = i % n1;
                sx[ax * kTreeMaxN1 + m] = (Real)(bx[ax] + bx[3 + ax] * t.xref[pol][m]);
            }
            const Real* Q = static_cast<const Real*>(t.mom[pol]) + (size_t)q * 3 * np;
            for (int i = tid; i < 3 * np; i += NT) sq[i] = Q[i];
            __syncthreads();
            Real a1[R], a2[R];
#pragma unroll
            for (int r = 0; r < R; ++r) a1[r] = a2[r] = (Real)0;
            for (int k3 = 0; k3 < n1; ++k3) {
                const Real sz = sx[2 * kTreeMaxN1 + k3];
                Real dz2[R], dzn[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const Real dz = pz[r] - sz;
                    dz2[r] = dz * dz;
                    dzn[r] = dz * nz[r];
                }
                for (int k2 = 0; k2 < n1; ++k2) {
                    const Real sy = sx[kTreeMaxN1 + k2];
                    Real ryz[R], dyzn[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const Real dy = py[r] - sy;
                        ryz[r] = fma(dy, dy, dz2[r]);
                        dyzn[r] = fma(dy, ny[r], dzn[r]);
                    }
                    const int kb = (k3 * n1 + k2) * n1;
                    for (int k1 = 0; k1 < n1; ++k1) {
                        const Real sxk = sx[k1];
                        const Real q0 = sq[kb + k1], qk = sq[np + kb + k1], qk2 = sq[2 * np + kb + k1];
#pragma unroll
                        for (int r = 0; r < R; ++r)
                            far_terms<Real>(px[r] - sxk, ryz[r], dyzn[r], nx[r], q0, qk, qk2, kappa, kl2, a1[r],
                                            a2[r]);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                o1[r] += (double)a1[r];
                o2[r] += (double)a2[r];
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (pp[r] < M) {
                pk::fx_add(t.acc + pp[r], M, 0, o1[r]);
                pk::fx_add(t.acc + pp[r], M, 1, o2[r]);
            }
        }
    }
}

// FP32 far items with two targets per f32x2 register pair (RP pairs per thread): the
// FMA-pipe work of two evaluations in one instruction, rsqrt and ex2 per half on
// the SFU; proxies and charges are duplicated into 64-bit words in shared memory.
// Dynamic shared memory of k_tree_far2 for clusters of np proxies.
constexpr size_t tree_far2_smem(int np = kTreeMaxNp) { return sizeof(unsigned long long) * (3 * kTreeMaxN1 + 3 * np); }

template <int RP, int NT, class Acc>
__global__ void __launch_bounds__(NT) k_tree_far2(Acc acc, const int2* __restrict__ ent,
                                               const int* __restrict__ n_ent, int* __restrict__ counter, int pol) {
    using pk::u64;
    extern __shared__ __align__(16) unsigned char tree_smem[];
    u64* sx = reinterpret_cast<u64*>(tree_smem);   // [3][kTreeMaxN1]
    u64* sq = sx + 3 * kTreeMaxN1;                 // [3][np]
    __shared__ int cur;
    const int tid = threadIdx.x;
    const int total = *n_ent;
    for (;;) {
        const int it = tree_next(counter, &cur);
        if (it >= total) break;
        const int2 w = ent[it];
        const TreeView* tp = acc.view(w.x);
        if (!tp) continue;
        const TreeView& t = *tp;
        const int n1 = t.n1[pol], np = t.np[pol], M = t.M, BS = t.BS[pol];
        const FarItem f = t.far[pol][w.y];
        const float kap = (float)t.kappa;
        const float kl2 = (float)(-t.kappa * 1.4426950408889634);
        const u64 kap2 = pk::pk2(kap, kap), kl2x2 = pk::pk2(kl2, kl2), one2 = pk::pk2(1.f, 1.f);
        u64 px[RP], py[RP], pz[RP], nx[RP], ny[RP], nz[RP];
        double o1[2 * RP], o2[2 * RP];
        int64_t pp[2 * RP];
#pragma unroll
        for (int j = 0; j < RP; ++j) {
            float P[2][3], n[2][3];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = 2 * j + h;
                pp[r] = (int64_t)f.I * BS + r * NT + tid;
                float a, b;
                tree_source<float>(t, pol, pp[r] < M ? pp[r] : (int64_t)M - 1, P[h], n[h], a, b);
                o1[r] = 0.0, o2[r] = 0.0;
            }
            px[j] = pk::pk2(P[0][0], P[1][0]), py[j] = pk::pk2(P[0][1], P[1][1]), pz[j] = pk::pk2(P[0][2], P[1][2]);
            nx[j] = pk::pk2(n[0][0], n[1][0]), ny[j] = pk::pk2(n[0][1], n[1][1]), nz[j] = pk::pk2(n[0][2], n[1][2]);
        }
        for (int l = f.l0; l < f.l1; ++l) {
            const int q = t.flist[pol][l];
            __syncthreads();   // the previous cluster's proxies are no longer read
            const double* bx = t.box[pol] + 6 * (int64_t)q;
            for (int i = tid; i < 3 * n1; i += NT) {
                const int ax = i / n1, m = i % n1;
                const float v = (float)(bx[ax] + bx[3 + ax] * t.xref[pol][m]);
                sx[ax * kTreeMaxN1 + m] = pk::pk2(v, v);
            }
            const float* Q = static_cast<const float*>(t.mom[pol]) + (size_t)q * 3 * np;
            for (int i = tid; i < 3 * np; i += NT) {
                const float v = Q[i];
                sq[i] = pk::pk2(v, v);
            }
            __syncthreads();
            u64 a1[RP], a2[RP];
#pragma unroll
            for (int j = 0; j < RP; ++j) a1[j] = a2[j] = 0ull;   // +0.0f in both halves
            for (int k3 = 0; k3 < n1; ++k3) {
                const u64 sz = sx[2 * kTreeMaxN1 + k3];
                u64 dz2[RP], dzn[RP];
#pragma unroll
                for (int j = 0; j < RP; ++j) {
                    const u64 dz = pk::sub2(pz[j], sz);
                    dz2[j] = pk::mul2(dz, dz);
                    dzn[j] = pk::mul2(dz, nz[j]);
                }
                for (int k2 = 0; k2 < n1; ++k2) {
                    const u64 sy = sx[kTreeMaxN1 + k2];
                    u64 ryz[RP], dyzn[RP];
#pragma unroll
                    for (int j = 0; j < RP; ++j) {
                        const u64 dy = pk::sub2(py[j], sy);
                        ryz[j] = pk::fma2(dy, dy, dz2[j]);
                        dyzn[j] = pk::fma2(dy, ny[j], dzn[j]);
                    }
                    const int kb = (k3 * n1 + k2) * n1;
                    for (int k1 = 0; k1 < n1; ++k1) {
                        const u64 sxk = sx[k1];
                        const u64 q0 = sq[kb + k1], qk = sq[np + kb + k1], qkp = sq[2 * np + kb + k1];
#pragma unroll
                        for (int j = 0; j < RP; ++j) {
                            const u64 dx = pk::sub2(px[j], sxk);
                            const u64 r2 = pk::fma2(dx, dx, ryz[j]);
                            const u64 dn = pk::fma2(dx, nx[j], dyzn[j]);
                            const u64 ri = pk::rsqrt2(r2);
                            const u64 r = pk::mul2(r2, ri);
                            const u64 E = pk::ex2_2(pk::mul2(kl2x2, r));
                            a1[j] = pk::fma2(ri, pk::fma2(E, qk, q0), a1[j]);
                            const u64 Ef = pk::mul2(E, pk::fma2(kap2, r, one2));
                            const u64 ri3 = pk::mul2(pk::mul2(ri, ri), ri);
                            a2[j] = pk::fma2(pk::mul2(dn, ri3), pk::fma2(Ef, qkp, q0), a2[j]);   // -(out2)
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < RP; ++j) {
                float x0, x1, y0, y1;
                pk::up2(a1[j], x0, x1);
                pk::up2(a2[j], y0, y1);
                o1[2 * j] += (double)x0, o1[2 * j + 1] += (double)x1;
                o2[2 * j] -= (double)y0, o2[2 * j + 1] -= (double)y1;
            }
        }
#pragma unroll
        for (int r = 0; r < 2 * RP; ++r) {
            if (pp[r] < M) {
                pk::fx_add(t.acc + pp[r], M, 0, o1[r]);
                pk::fx_add(t.acc + pp[r], M, 1, o2[r]);
            }
        }
    }
}

// Float-float far items (the float-float operator): R targets per thread x NT threads = a 256-node block.
// Dynamic shared memory: the cluster's proxy coordinates and charges as float-float pairs, then the
// exponential tables.
constexpr size_t tree_farff_smem(int np = kTreeMaxNp) {
    return sizeof(float2) * (3 * kTreeMaxN1 + 3 * np + pk::kExpHi + pk::kExpLo);
}

template <int R, int NT, class Acc>
__global__ void __launch_bounds__(NT) k_tree_far_ff(Acc acc, const int2* __restrict__ ent,
                                                  const int* __restrict__ n_ent, int* __restrict__ counter) {
    using pk::F2;
    constexpr int pol = 1;
    extern __shared__ __align__(16) unsigned char tree_smem[];
    float2* sx = reinterpret_cast<float2*>(tree_smem);   // [3][kTreeMaxN1]
    float2* sq = sx + 3 * kTreeMaxN1;                     // [3][np]
    __shared__ int cur;
    __shared__ const float2* tab_src;
    const int tid = threadIdx.x;
    const int total = *n_ent;
    bool tab_ready = false;
    for (;;) {
        const int it = tree_next(counter, &cur);
        if (it >= total) break;
        const int2 w = ent[it];
        const TreeView* tp = acc.view(w.x);
        if (!tp) continue;
        const TreeView& t = *tp;
        const int n1 = t.n1[pol], np = t.np[pol], M = t.M, BS = t.BS[pol];
        float2* tab = sq + 3 * np;
        if (!tab_ready) {   // block-uniform; every handle's table is the same device table
            if (tid == 0) tab_src = t.exp_tab;
            __syncthreads();
            for (int q = tid; q < pk::kExpHi + pk::kExpLo; q += NT) tab[q] = tab_src[q];
            tab_ready = true;
        }
        const FarItem f = t.far[pol][w.y];
        const F2 kap = pk::f2(pk::split_ff_dev(t.kappa));
        F2 px[R], py[R], pz[R], nx[R], ny[R], nz[R];
        double o1[R], o2[R];
        int64_t pp[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            pp[r] = (int64_t)f.I * BS + r * NT + tid;
            const int64_t p = pp[r] < M ? pp[r] : (int64_t)M - 1;
            const float4 u = t.srcdf[4 * p], ul = t.srcdf[4 * p + 1], v = t.srcdf[4 * p + 2],
                         vl = t.srcdf[4 * p + 3];
            px[r] = F2{u.x, ul.x}, py[r] = F2{u.y, ul.y}, pz[r] = F2{u.z, ul.z};
            nx[r] = F2{v.x, vl.x}, ny[r] = F2{v.y, vl.y}, nz[r] = F2{v.z, vl.z};
            o1[r] = 0.0, o2[r] = 0.0;
        }
        for (int l = f.l0; l < f.l1; ++l) {
            const int q = t.flist[pol][l];
            __syncthreads();   // the previous cluster's proxies are no longer read (and the table is in)
            const double* bx = t.box[pol] + 6 * (int64_t)q;
            for (int i = tid; i < 3 * n1; i += NT) {
                const int ax = i / n1, m = i % n1;
                sx[ax * kTreeMaxN1 + m] = pk::split_ff_dev(bx[ax] + bx[3 + ax] * t.xref[pol][m]);
            }
            const double* Q = static_cast<const double*>(t.mom[pol]) + (size_t)q * 3 * np;
            for (int i = tid; i < 3 * np; i += NT) sq[i] = pk::split_ff_dev(Q[i]);
            __syncthreads();
            F2 a1[R], a2[R];
#pragma unroll
            for (int r = 0; r < R; ++r) a1[r] = a2[r] = F2{0.f, 0.f};
            for (int k3 = 0; k3 < n1; ++k3) {
                const F2 sz = pk::f2(sx[2 * kTreeMaxN1 + k3]);
                F2 dz2[R], dzn[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const F2 dz = pk::sub(pz[r], sz);
                    dz2[r] = pk::mull(dz, dz);
                    dzn[r] = pk::mul(dz, nz[r]);
                }
                for (int k2 = 0; k2 < n1; ++k2) {
                    const F2 sy = pk::f2(sx[kTreeMaxN1 + k2]);
                    F2 ryz[R], dyzn[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const F2 dy = pk::sub(py[r], sy);
                        ryz[r] = ff_addl(pk::mull(dy, dy), dz2[r]);
                        dyzn[r] = pk::add(pk::mul(dy, ny[r]), dzn[r]);
                    }
                    const int kb = (k3 * n1 + k2) * n1;
                    for (int k1 = 0; k1 < n1; ++k1) {
                        const F2 sxk = pk::f2(sx[k1]);
                        const F2 q0 = pk::f2(sq[kb + k1]), qk = pk::f2(sq[np + kb + k1]),
                                 qkp = pk::f2(sq[2 * np + kb + k1]);
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            // lazy (unnormalised) values wherever no cancellation can follow: the squares
                            // and r^2, kappa r, the exponential, 1 + kappa r and the products; the
                            // differences, the dot product and the two charge combinations stay normalised
                            const F2 dx = pk::sub(px[r], sxk);
                            const F2 r2 = ff_addl(pk::mull(dx, dx), ryz[r]);
                            const F2 dn = pk::add(pk::mul(dx, nx[r]), dyzn[r]);
                            const F2 ri = pk::rsqrt_ff(r2);
                            const F2 kr = pk::mull(kap, pk::mull(r2, ri));
                            const F2 E = pk::exp_neg_ffl(kr, tab);
                            pk::acc_add(a1[r], pk::mull(ri, pk::add(pk::mull(E, qk), q0)));
                            const F2 Ef = pk::mull(E, ff_add_fl(kr, 1.f));
                            const F2 ri3 = pk::mull(pk::mull(ri, ri), ri);
                            pk::acc_add(a2[r], pk::mull(pk::mull(dn, ri3), pk::add(pk::mull(Ef, qkp), q0)));   // -(out2)
                        }
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                o1[r] += (double)a1[r].hi + (double)a1[r].lo;
                o2[r] -= (double)a2[r].hi + (double)a2[r].lo;
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (pp[r] < M) {
                pk::fx_add(t.acc + pp[r], M, 0, o1[r]);
                pk::fx_add(t.acc + pp[r], M, 1, o2[r]);
            }
        }
    }
}

// Work entries of one handle alone: every entry belongs to it.
struct OneTreeAcc {
    const TreeView* t;
    __device__ const TreeView* view(int) const { return t; }
};

// Resident blocks per SM of a far kernel instantiation with `smem` bytes of dynamic shared memory (host):
// the kernel's opt-in to `smem_max` (above 48 KB) is set once per device; results are cached per
// (device, smem) in `cache`.
template <typename K>
int far_per_sm(K kernel, int threads, int smem, int smem_max, std::map<std::pair<int, int>, int>& cache) {
    static std::mutex mu;
    int dev = 0;
    CTR_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find({dev, smem});
    if (it != cache.end()) return it->second;
    if (cache.find({dev, -1}) == cache.end()) {
        CTR_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
        cache[{dev, -1}] = 1;
    }
    int b = 0;
    CTR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem));
    b = std::max(1, b);
    cache[{dev, smem}] = b;
    return b;
}

}  // namespace ctr
