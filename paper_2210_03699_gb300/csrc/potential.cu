// Reaction potential at arbitrary points (Eq. 2.31) as a tiled pair sum: potential maps and the
// polarization energy (Eq. 3.3).
//
//   psi_rxn(z) = h^3 sum_j W_j [ ((eps_E/eps_I) dGk/dn_y - dG0/dn_y)(z, P_j) psi_j + (G0 - Gk)(z, P_j) dpsi_j ]
//
// by the plain trapezoidal rule on the tube (z away from the surface).  With a_j = h^3 W_j psi_j / (4 pi),
// b_j = h^3 W_j dpsi_j / (4 pi), d = z - P_j, s = 1/r^3, E = e^{-kappa r}, E1 = E (1 + kappa r):
//
//   psi_rxn(z) = sum_j [ a_j (d.n_j) s ((eps_E/eps_I) E1 - 1) + b_j (1 - E) / r ].
//
// The points are the targets (registers), the tube nodes the sources: the packed source arrays of the
// operator (their weight slots rewritten with a, b) streamed through the same two-stage shared-memory
// ring (cp.async.bulk + mbarrier) as the operator's pair items.  A grid of (target block, source split)
// blocks writes per-split FP64 partial sums (per-tile sums folded into FP64), added in split order by a
// second kernel: the result does not depend on scheduling.  Three arithmetics:
//   Fp32x2  two points per f32x2 instruction, 22 FMA-pipe lane operations + 2 SFU per pair;
//   Df64    float-float (the operator's residual arithmetic), one point per thread;
//   Fp64    IEEE FP64 (the energy of ctr_ibim_energy).
// The split partials live in a workspace the handle keeps and grows (no allocation once it is large
// enough).
#include "pairkern.cuh"

namespace ctr {

using namespace pk;

namespace {

// ---------------------------------------------------------------- map policies
struct MapFp32x2 {
    using Src = ulonglong2;   // the operator's packed FP32 node {(x,x),(y,y)} {(z,z),(a,a)} {(nx,nx),(ny,ny)} {(nz,nz),(-b,-b)}
    static constexpr int kVec = 4;
    static constexpr int kTile = 256;
    static constexpr int kPack = 2;
    static constexpr int kR = 2;
    static constexpr bool kTables = false;
    struct Tgt {
        u64 x, y, z;
    };
    using Acc = u64;
    __device__ static Tgt load(const double* xyz, int64_t n, const int64_t* p) {
        float v[2][3];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t q = min(p[h], n - 1);
#pragma unroll
            for (int c = 0; c < 3; ++c) v[h][c] = (float)xyz[3 * q + c];
        }
        return Tgt{pk2(v[0][0], v[1][0]), pk2(v[0][1], v[1][1]), pk2(v[0][2], v[1][2])};
    }
    __device__ static void zero(Acc& a) { a = 0ull; }
    __device__ static void fold(const Acc& a, double* s) {
        float x, y;
        up2(a, x, y);
        s[0] += (double)x;
        s[1] += (double)y;
    }
    // acc += a s (d.n) (c1 E1 - 1) + (-b) (E - 1)/r  (= b (1 - E)/r)
    __device__ static void pair(const Tgt& T, const Src* S, const PairConsts& k, const float2*, Acc& acc) {
        const ulonglong2 v0 = S[0], v1 = S[1], v2 = S[2], v3 = S[3];
        const u64 dx = sub2(T.x, v0.x), dy = sub2(T.y, v0.y), dz = sub2(T.z, v1.x);
        const u64 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
        const u64 rinv = rsqrt2(r2);
        const u64 r = mul2(r2, rinv);
        const u64 E = ex2_2(mul2(k.kl2x2, r));
        const u64 E1 = fma2(E, mul2(k.kap2, r), E);
        const u64 dny = fma2(dz, v3.x, fma2(dy, v2.y, mul2(dx, v2.x)));
        const u64 s = mul2(mul2(rinv, rinv), rinv);
        const u64 t = fma2(k.c1x2, E1, k.mone2);
        acc = fma2(mul2(mul2(v1.y, s), dny), t, acc);
        acc = fma2(v3.y, mul2(rinv, sub2(E, k.one2)), acc);
    }
};

// float-float node {P.hi, a.hi} {P.lo, a.lo} {n.hi, b.hi} {n.lo, b.lo}
struct MapDf64 {
    using Src = float4;
    static constexpr int kVec = 4;
    static constexpr int kTile = 128;
    static constexpr int kPack = 1;
    static constexpr int kR = 1;
    static constexpr bool kTables = true;
    struct Tgt {
        F2 x, y, z;
    };
    using Acc = F2;
    __device__ static Tgt load(const double* xyz, int64_t n, const int64_t* p) {
        const int64_t q = min(p[0], n - 1);
        F2 c[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double v = xyz[3 * q + i];
            const float hi = (float)v;
            c[i] = F2{hi, (float)(v - (double)hi)};
        }
        return Tgt{c[0], c[1], c[2]};
    }
    __device__ static void zero(Acc& a) { a = F2{0.f, 0.f}; }
    __device__ static void fold(const Acc& a, double* s) { s[0] += (double)a.hi + (double)a.lo; }
    __device__ static void pair(const Tgt& T, const Src* S, const PairConsts& k, const float2* tab, Acc& acc) {
        const float4 s0 = S[0], s1 = S[1], s2 = S[2], s3 = S[3];
        const F2 dx = sub(T.x, F2{s0.x, s1.x}), dy = sub(T.y, F2{s0.y, s1.y}), dz = sub(T.z, F2{s0.z, s1.z});
        const F2 r2 = dot3(dx, dy, dz, dx, dy, dz);
        const F2 rinv = rsqrt_ff(r2);
        const F2 r = mul(r2, rinv);
        const F2 kr = mul(f2(k.kappad), r);
        const F2 E = exp_neg_ff(kr, tab);
        const F2 E1 = mul(E, add_f(kr, 1.f));
        const F2 dny = dot3(dx, dy, dz, F2{s2.x, s3.x}, F2{s2.y, s3.y}, F2{s2.z, s3.z});
        const F2 s = mul(mul(rinv, rinv), rinv);
        const F2 t = add_f(mul(E1, f2(k.c1d)), -1.f);
        acc = add(acc, mul(mul(F2{s0.w, s1.w}, s), mul(dny, t)));
        acc = add(acc, mul(F2{s2.w, s3.w}, mul(rinv, add_f(neg(E), 1.f))));
    }
};

// FP64 node {P, a} {n, b}
struct MapFp64 {
    using Src = double4;
    static constexpr int kVec = 2;
    static constexpr int kTile = 128;
    static constexpr int kPack = 1;
    static constexpr int kR = 1;
    static constexpr bool kTables = false;
    struct Tgt {
        double x, y, z;
    };
    using Acc = double;
    __device__ static Tgt load(const double* xyz, int64_t n, const int64_t* p) {
        const int64_t q = min(p[0], n - 1);
        return Tgt{xyz[3 * q], xyz[3 * q + 1], xyz[3 * q + 2]};
    }
    __device__ static void zero(Acc& a) { a = 0.0; }
    __device__ static void fold(const Acc& a, double* s) { s[0] += a; }
    __device__ static void pair(const Tgt& T, const Src* S, const PairConsts& k, const float2*, Acc& acc) {
        const double4 pa = S[0], nb = S[1];
        const double dx = T.x - pa.x, dy = T.y - pa.y, dz = T.z - pa.z;
        const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        const double rinv = rsqrt(r2);
        const double r = r2 * rinv;
        const double E = exp(-k.kappa * r);
        const double E1 = fma(E, k.kappa * r, E);
        const double dny = fma(dz, nb.z, fma(dy, nb.y, dx * nb.x));
        const double s = rinv * rinv * rinv;
        acc = fma(pa.w * s * dny, fma(k.c1, E1, -1.0), acc);
        acc = fma(nb.w, (1.0 - E) * rinv, acc);
    }
};

// One block: points [blockIdx.x * BS, +BS) against sources [j_begin, j_end) of its split; the sums go to
// part[split * n + point].
template <typename Pol>
__global__ void __launch_bounds__(kThreads) map_kernel(const typename Pol::Src* __restrict__ src, int M,
                                                       const double* __restrict__ xyz, int64_t n, int per_split,
                                                       double* __restrict__ part, PairConsts kc,
                                                       int* __restrict__ err) {
    using Src = typename Pol::Src;
    constexpr int TILE = Pol::kTile, VEC = Pol::kVec, P = Pol::kPack, R = Pol::kR, RP = R * P;
    constexpr int BS = kThreads * RP;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Src* ring = reinterpret_cast<Src*>(smem_raw);
    float2* tab = reinterpret_cast<float2*>(smem_raw + 2 * TILE * VEC * sizeof(Src));
    __shared__ __align__(8) uint64_t bar[2];
    if constexpr (Pol::kTables) {
        for (int q = threadIdx.x; q < kExpHi + kExpLo; q += kThreads) tab[q] = kc.exp_tab[q];
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int tid = threadIdx.x;
    const int j_begin = blockIdx.y * per_split;
    const int j_end = min(M, j_begin + per_split);
    const int ntiles = (j_end > j_begin) ? (j_end - j_begin + TILE - 1) / TILE : 0;
    int64_t pi[RP];
    double s[RP];
    typename Pol::Tgt tg[R];
#pragma unroll
    for (int a = 0; a < RP; ++a) {
        pi[a] = (int64_t)blockIdx.x * BS + a * kThreads + tid;
        s[a] = 0.0;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) tg[r] = Pol::load(xyz, n, &pi[r * P]);
    auto issue = [&](int k) {
        const int j0 = j_begin + k * TILE;
        const uint32_t bytes = (uint32_t)(min(TILE, j_end - j0) * VEC * sizeof(Src));
        fence_proxy_async();
        mbar_expect_tx(&bar[k & 1], bytes);
        bulk_load(ring + (k & 1) * TILE * VEC, src + (size_t)VEC * j0, bytes, &bar[k & 1]);
    };
    if (tid == 0 && ntiles > 0) issue(0);
    for (int k = 0; k < ntiles; ++k) {
        if (tid == 0 && k + 1 < ntiles) issue(k + 1);
        const bool ok = mbar_wait(&bar[k & 1], (k >> 1) & 1, kc.wait_limit);
        if (__syncthreads_or(!ok)) {   // give up: flag, let both copies in flight land, return
            if (tid == 0) {
                atomicOr(err, kErrWait);
                (void)mbar_wait(&bar[k & 1], (k >> 1) & 1);
                if (k + 1 < ntiles) (void)mbar_wait(&bar[(k + 1) & 1], ((k + 1) >> 1) & 1);
            }
            return;
        }
        const Src* tile = ring + (k & 1) * TILE * VEC;
        const int cnt = min(TILE, j_end - (j_begin + k * TILE));
        typename Pol::Acc acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) Pol::zero(acc[r]);
#pragma unroll 2
        for (int q = 0; q < cnt; ++q) {
#pragma unroll
            for (int r = 0; r < R; ++r) Pol::pair(tg[r], tile + q * VEC, kc, tab, acc[r]);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) Pol::fold(acc[r], &s[r * P]);
        __syncthreads();   // this buffer is free for the tile after next
    }
#pragma unroll
    for (int a = 0; a < RP; ++a)
        if (pi[a] < n) part[(size_t)blockIdx.y * n + pi[a]] = s[a];
}

// out[p] = sum over splits of part[split * n + p], in split order
__global__ void map_sum_kernel(const double* __restrict__ part, int splits, int64_t n, double* __restrict__ out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double v = 0.0;
    for (int q = 0; q < splits; ++q) v += part[(size_t)q * n + p];
    out[p] = v;
}

// a = h^3 W psi / (4 pi), b = h^3 W dpsi / (4 pi) into the weight slots of one packed source array
__global__ void map_pack_kernel(const double* __restrict__ psi, const double* __restrict__ dpsi,
                                const double* __restrict__ W, int64_t M, double scale, int prec,
                                float4* __restrict__ s32, double4* __restrict__ s64, float4* __restrict__ sdf,
                                const int32_t* __restrict__ tinv) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M) return;
    const double a = scale * W[t] * psi[t], b = scale * W[t] * dpsi[t];
    const int64_t j = tinv ? (int64_t)tinv[t] : t;
    if (prec == CTR_FP32_REFINE) {
        s32[4 * j + 1].z = s32[4 * j + 1].w = (float)a;
        s32[4 * j + 3].z = s32[4 * j + 3].w = -(float)b;
    } else if (prec == CTR_FP64) {
        s64[2 * j].w = a;
        s64[2 * j + 1].w = b;
    } else {
        const float ah = (float)a, bh = (float)b;
        sdf[4 * j].w = ah;
        sdf[4 * j + 1].w = (float)(a - (double)ah);
        sdf[4 * j + 2].w = bh;
        sdf[4 * j + 3].w = (float)(b - (double)bh);
    }
}

template <typename Pol>
constexpr size_t map_smem() {
    return 2 * Pol::kTile * Pol::kVec * sizeof(typename Pol::Src) +
           (Pol::kTables ? (kExpHi + kExpLo) * sizeof(float2) : 0);
}

template <typename Pol>
int map_launch(ctr_ibim* s, const void* src, const double* d_xyz, int64_t n, const PairConsts& kc, int* splits_out) {
    constexpr int BS = kThreads * Pol::kR * Pol::kPack;
    static int per_dev[64] = {0};   // resident blocks per SM of this instantiation, per device
    int dev = 0, sms = 0;
    CTR_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CTR_ERR_INVALID, "device index");
    CTR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = map_smem<Pol>();
    if (per_dev[dev] == 0) {
        int b = 0;
        CTR_CUDA_TRY(cudaFuncSetAttribute(map_kernel<Pol>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        CTR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, map_kernel<Pol>, kThreads, smem));
        per_dev[dev] = std::max(1, b);
    }
    const int64_t M = s->M;
    const int64_t tblocks = (n + BS - 1) / BS;
    if (n > (int64_t)INT32_MAX) return fail(CTR_ERR_CAPACITY, "more than 2^31 - 1 points");
    // source splits: about two waves of resident blocks, whole tiles, at least four tiles per split
    const int64_t want = std::max<int64_t>(1, 2LL * per_dev[dev] * sms / std::max<int64_t>(1, tblocks));
    const int64_t max_splits = std::max<int64_t>(1, M / (4 * Pol::kTile));
    int64_t splits = std::min<int64_t>({want, max_splits, 4096});
    int64_t per = (M + splits - 1) / splits;
    per = ((per + Pol::kTile - 1) / Pol::kTile) * Pol::kTile;
    splits = (M + per - 1) / per;
    CTR_TRY(s->map_ws.alloc(sizeof(double) * (size_t)(splits * n)));
    dim3 grid((unsigned)tblocks, (unsigned)splits);
    map_kernel<Pol><<<grid, kThreads, smem, s->stream>>>(reinterpret_cast<const typename Pol::Src*>(src), (int)M,
                                                         d_xyz, n, (int)per, s->map_ws.as<double>(), kc,
                                                         s->err.as<int>());
    CTR_LAUNCHED();
    *splits_out = (int)splits;
    return CTR_OK;
}

}  // namespace

int potential_map(ctr_ibim* s, const double* d_psi, const double* d_dpsi, int64_t n, const double* d_xyz,
                  double* d_out, int precision) {
    if (n <= 0) return CTR_OK;
    const int64_t M = s->M;
    const double scale = s->h * s->h * s->h / (4.0 * kPi);
    const int32_t* tinv = s->tree ? s->tree->d_tinv.as<int32_t>() : nullptr;
    map_pack_kernel<<<grid_for(M, 256), 256, 0, s->stream>>>(d_psi, d_dpsi, s->na.W, M, scale, precision,
                                                            s->src32.as<float4>(), s->src64.as<double4>(),
                                                            s->srcdf.as<float4>(), tinv);
    CTR_LAUNCHED();
    PairConsts kc;
    CTR_TRY(pair_consts(s, precision == CTR_DF64, &kc));
    int splits = 0;
    if (precision == CTR_FP32_REFINE) CTR_TRY(map_launch<MapFp32x2>(s, s->src32.p, d_xyz, n, kc, &splits));
    else if (precision == CTR_DF64) CTR_TRY(map_launch<MapDf64>(s, s->srcdf.p, d_xyz, n, kc, &splits));
    else CTR_TRY(map_launch<MapFp64>(s, s->src64.p, d_xyz, n, kc, &splits));
    map_sum_kernel<<<grid_for(n, 256), 256, 0, s->stream>>>(s->map_ws.as<double>(), splits, n, d_out);
    CTR_LAUNCHED();
    return CTR_OK;
}

}  // namespace ctr
