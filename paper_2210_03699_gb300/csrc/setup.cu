// Tube extraction, finite-difference geometry and right-hand side (Sec. 2.1, Eq. 2.12).
//
// Every step runs on the device.  Values that decide an integer downstream
// (tube membership, the node coordinates y, normals n and closest points P
// that fix the correction planes and nodes) are computed with explicitly
// rounded FP64 operations (__dadd_rn, __dmul_rn, ...) in a fixed order, so no
// multiply-add is fused and the result is the IEEE value of the written
// expression:  y = origin + h*i;  g_c = (d[+c] - d[-c]) / (2h);
// |g| = sqrt((g0*g0 + g1*g1) + g2*g2);  n_c = g_c / |g|;  P_c = y_c - d*n_c.
#include "common.cuh"

namespace ctr {

namespace {

constexpr int kChunk = 4096;      // grid nodes per block in the tube scan
constexpr int kScanThreads = 256;

__device__ __forceinline__ bool in_tube(double d, double eps) { return fabs(d) < eps; }

// Tube nodes per chunk of the grid; a non-finite signed distance anywhere sets kErrNumeric.
__global__ void tube_count_kernel(const double* __restrict__ sd, int64_t total, double eps,
                                  int32_t* __restrict__ counts, int* __restrict__ err) {
    int64_t base = (int64_t)blockIdx.x * kChunk;
    int c = 0;
    bool bad = false;
    for (int t = threadIdx.x; t < kChunk; t += blockDim.x) {
        int64_t g = base + t;
        if (g < total) {
            const double v = sd[g];
            bad |= !isfinite(v);
            if (in_tube(v, eps)) ++c;
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, kErrNumeric);
    __shared__ int warp_sum[kScanThreads / 32];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) s += warp_sum[w];
        counts[blockIdx.x] = s;
    }
}

__global__ void tube_compact_kernel(const double* __restrict__ sd, int64_t total, double eps,
                                    const int32_t* __restrict__ offsets, int64_t* __restrict__ lin,
                                    int32_t* __restrict__ node_of) {
    int64_t base = (int64_t)blockIdx.x * kChunk;
    __shared__ int warp_tot[kScanThreads / 32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = offsets[blockIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t0 = 0; t0 < kChunk; t0 += kScanThreads) {
        int64_t g = base + t0 + threadIdx.x;
        bool f = (g < total) && in_tube(sd[g], eps);
        unsigned b = __ballot_sync(0xffffffffu, f);
        int pre = __popc(b & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[warp] = __popc(b);
        __syncthreads();
        int off = carry;
        for (int w = 0; w < warp; ++w) off += warp_tot[w];
        if (f) {
            int id = off + pre;
            lin[id] = g;
            node_of[g] = id;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int s = 0;
            for (int w = 0; w < kScanThreads / 32; ++w) s += warp_tot[w];
            carry += s;
        }
        __syncthreads();
    }
}

// Single-block exclusive scan of n counts (any n), offsets[n] = total.
__global__ void scan_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n) {
    __shared__ int32_t buf[1024];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < n; b += 1024) {
        int64_t i = b + threadIdx.x;
        int32_t v = (i < n) ? in[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            int32_t t = (threadIdx.x >= (unsigned)o) ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < n) out[i] = carry + buf[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += buf[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = carry;
}

__device__ __forceinline__ double phi_avg(double x) {
    // averaging kernel of Sec. 2.6: (1 + cos(pi x))/2 on |x| <= 1
    return fabs(x) <= 1.0 ? 0.5 * (1.0 + cospi(x)) : 0.0;
}

__global__ void geometry_kernel(const double* __restrict__ sd, const int64_t* __restrict__ lin, int64_t M,
                                int64_t nx, int64_t ny, int64_t nz, double ox, double oy, double oz,
                                double h, double eps, int kreg_all, NodeArrays na, uint8_t* __restrict__ bad,
                                float4* __restrict__ src32, double4* __restrict__ src64, int* __restrict__ err) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int64_t g = lin[m];
    const int64_t i = g % nx, j = (g / nx) % ny, k = g / (nx * ny);
    if (i < 2 || j < 2 || k < 2 || i > nx - 3 || j > ny - 3 || k > nz - 3) {
        atomicOr(err, kErrMargin);
        return;
    }
    const int64_t sx = 1, sy = nx, sz = nx * ny;
    auto D = [&](int di, int dj, int dk) { return sd[g + di * sx + dj * sy + dk * sz]; };
    const double two_h = 2.0 * h;
    const double g0 = __ddiv_rn(__dsub_rn(D(1, 0, 0), D(-1, 0, 0)), two_h);
    const double g1 = __ddiv_rn(__dsub_rn(D(0, 1, 0), D(0, -1, 0)), two_h);
    const double g2 = __ddiv_rn(__dsub_rn(D(0, 0, 1), D(0, 0, -1)), two_h);
    const double gn = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(g0, g0), __dmul_rn(g1, g1)), __dmul_rn(g2, g2)));
    const double n0 = __ddiv_rn(g0, gn), n1 = __ddiv_rn(g1, gn), n2 = __ddiv_rn(g2, gn);
    const double dd = D(0, 0, 0);
    const double y0 = __dadd_rn(ox, __dmul_rn(h, (double)i));
    const double y1 = __dadd_rn(oy, __dmul_rn(h, (double)j));
    const double y2 = __dadd_rn(oz, __dmul_rn(h, (double)k));
    const double P0 = __dsub_rn(y0, __dmul_rn(dd, n0));
    const double P1 = __dsub_rn(y1, __dmul_rn(dd, n1));
    const double P2 = __dsub_rn(y2, __dmul_rn(dd, n2));

    // Hessian: central difference of the central-difference gradient (5 nodes per axis)
    const double inv4h2 = 1.0 / (4.0 * h * h);
    double H[3][3];
    H[0][0] = (D(2, 0, 0) - 2.0 * dd + D(-2, 0, 0)) * inv4h2;
    H[1][1] = (D(0, 2, 0) - 2.0 * dd + D(0, -2, 0)) * inv4h2;
    H[2][2] = (D(0, 0, 2) - 2.0 * dd + D(0, 0, -2)) * inv4h2;
    H[0][1] = H[1][0] = (D(1, 1, 0) - D(1, -1, 0) - D(-1, 1, 0) + D(-1, -1, 0)) * inv4h2;
    H[0][2] = H[2][0] = (D(1, 0, 1) - D(1, 0, -1) - D(-1, 0, 1) + D(-1, 0, -1)) * inv4h2;
    H[1][2] = H[2][1] = (D(0, 1, 1) - D(0, 1, -1) - D(0, -1, 1) + D(0, -1, -1)) * inv4h2;

    // tangent basis e1 = n x e_c (c: smallest |n_c|), e2 = n x e1
    const double nv[3] = {n0, n1, n2};
    int c = 0;
    if (fabs(nv[1]) < fabs(nv[c])) c = 1;
    if (fabs(nv[2]) < fabs(nv[c])) c = 2;
    double ec[3] = {0, 0, 0};
    ec[c] = 1.0;
    double e1[3] = {nv[1] * ec[2] - nv[2] * ec[1], nv[2] * ec[0] - nv[0] * ec[2], nv[0] * ec[1] - nv[1] * ec[0]};
    const double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    e1[0] /= l1; e1[1] /= l1; e1[2] /= l1;
    const double e2[3] = {nv[1] * e1[2] - nv[2] * e1[1], nv[2] * e1[0] - nv[0] * e1[2], nv[0] * e1[1] - nv[1] * e1[0]};
    double He1[3], He2[3];
    for (int a = 0; a < 3; ++a) {
        He1[a] = H[a][0] * e1[0] + H[a][1] * e1[1] + H[a][2] * e1[2];
        He2[a] = H[a][0] * e2[0] + H[a][1] * e2[1] + H[a][2] * e2[2];
    }
    const double s00 = (e1[0] * He1[0] + e1[1] * He1[1] + e1[2] * He1[2]) / gn;
    const double s11 = (e2[0] * He2[0] + e2[1] * He2[1] + e2[2] * He2[2]) / gn;
    const double s01 = 0.5 * ((e1[0] * He2[0] + e1[1] * He2[1] + e1[2] * He2[2]) +
                              (e2[0] * He1[0] + e2[1] * He1[1] + e2[2] * He1[2])) / gn;
    // 2x2 symmetric eigenproblem: level-set principal curvatures kp1 <= kp2
    const double mean = 0.5 * (s00 + s11), half = 0.5 * (s00 - s11);
    const double rad = hypot(half, s01);
    const double kp1 = mean - rad, kp2 = mean + rad;
    const double th = 0.5 * atan2(2.0 * s01, s00 - s11);   // eigenvector of kp2: (cos th, sin th)
    const double ct = cos(th), st = sin(th);
    const double t2[3] = {ct * e1[0] + st * e2[0], ct * e1[1] + st * e2[1], ct * e1[2] + st * e2[2]};
    const double t1[3] = {-st * e1[0] + ct * e2[0], -st * e1[1] + ct * e2[1], -st * e1[2] + ct * e2[2]};
    // Jacobian (Eq. 2.8 with d > 0 outside), surface curvatures and M = diag(-k1, -k2)
    double J = (1.0 - dd * kp1) * (1.0 - dd * kp2);
    const double k1 = kp1 / (1.0 - dd * kp1), k2 = kp2 / (1.0 - dd * kp2);
    // hybrid classification (Sec. 3.2): untrustworthy curvature -> bad node, J = 1 (Eq. 3.2)
    const bool finite = isfinite(J) && isfinite(k1) && isfinite(k2) && isfinite(t1[0] + t1[1] + t1[2]) &&
                        isfinite(t2[0] + t2[1] + t2[2]);
    const bool is_bad = kreg_all || !finite || fmax(fabs(k1), fabs(k2)) * (eps + h) >= 0.8;
    if (is_bad) J = 1.0;
    const double W = J * phi_avg(dd / eps) / eps;
    if (!isfinite(W) || !isfinite(P0 + P1 + P2) || !(gn > 0.0)) atomicOr(err, kErrNumeric);
    bad[m] = is_bad ? 1 : 0;

    na.Px[m] = P0; na.Py[m] = P1; na.Pz[m] = P2;
    na.nx[m] = n0; na.ny[m] = n1; na.nz[m] = n2;
    na.W[m] = W; na.d[m] = dd;
    na.t1x[m] = t1[0]; na.t1y[m] = t1[1]; na.t1z[m] = t1[2];
    na.t2x[m] = t2[0]; na.t2y[m] = t2[1]; na.t2z[m] = t2[2];
    na.m1[m] = -k1; na.m2[m] = -k2;
    src32[4 * m] = make_float4((float)P0, (float)P0, (float)P1, (float)P1);
    src32[4 * m + 1] = make_float4((float)P2, (float)P2, 0.f, 0.f);
    src32[4 * m + 2] = make_float4((float)n0, (float)n0, (float)n1, (float)n1);
    src32[4 * m + 3] = make_float4((float)n2, (float)n2, 0.f, 0.f);
    src64[2 * m] = make_double4(P0, P1, P2, 0.0);
    src64[2 * m + 1] = make_double4(n0, n1, n2, 0.0);
}

// g1 = sum_k q_k/eps_I G0(P, z_k), g2 = sum_k q_k/eps_I dG0/dn_x(P, z_k)   (Eq. 2.12)
__global__ void rhs_kernel(NodeArrays na, int64_t M, const double* __restrict__ ch, int64_t nc,
                           double eps_in, double* __restrict__ g) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const double px = na.Px[m], py = na.Py[m], pz = na.Pz[m];
    const double qx = na.nx[m], qy = na.ny[m], qz = na.nz[m];
    double g1 = 0.0, g2 = 0.0;
    const double inv4pi = 1.0 / (4.0 * kPi);
    for (int64_t c = 0; c < nc; ++c) {
        const double dx = px - ch[c], dy = py - ch[nc + c], dz = pz - ch[2 * nc + c];
        const double q = ch[3 * nc + c] / eps_in;
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double rinv = 1.0 / sqrt(r2);
        g1 += q * inv4pi * rinv;
        g2 -= q * inv4pi * (dx * qx + dy * qy + dz * qz) * rinv * rinv * rinv;
    }
    g[m] = g1;
    g[M + m] = g2;
}

}  // namespace

int exclusive_scan_i32(const int32_t* d_counts, int32_t* d_offsets, int64_t n, cudaStream_t st,
                       DevBuf& /*scratch*/) {
    scan_kernel<<<1, 1024, 0, st>>>(d_counts, d_offsets, n);
    CTR_LAUNCHED();
    return CTR_OK;
}

int check_device_error(ctr_ibim* s, const char* where) {
    int herr = 0;
    CTR_CUDA_TRY(cudaMemcpyAsync(&herr, s->err.p, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CTR_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (herr == 0) return CTR_OK;
    CTR_CUDA_TRY(cudaMemsetAsync(s->err.p, 0, sizeof(int), s->stream));
    std::string w(where);
    if (herr & kErrMargin) return fail(CTR_ERR_GRID_MARGIN, w + ": a tube node lies within 2 nodes of the grid boundary");
    if (herr & kErrNumeric) return fail(CTR_ERR_NUMERIC, w + ": non-finite value");
    if (herr & kErrCapacity) return fail(CTR_ERR_CAPACITY, w + ": fixed capacity exceeded");
    return fail(CTR_ERR_DEVICE_WAIT, w + ": a bounded device wait expired");
}

int setup_tube_and_geometry(ctr_ibim* s, const double* d_sdist) {
    const int64_t total = s->n[0] * s->n[1] * s->n[2];
    const int64_t nchunks = (total + kChunk - 1) / kChunk;
    cudaStream_t st = s->stream;
    DevBuf counts, offsets, node_of, scratch;
    CTR_TRY(counts.alloc(sizeof(int32_t) * nchunks));
    CTR_TRY(offsets.alloc(sizeof(int32_t) * (nchunks + 1)));
    tube_count_kernel<<<(unsigned)nchunks, kScanThreads, 0, st>>>(d_sdist, total, s->eps, counts.as<int32_t>(),
                                                                  s->err.as<int>());
    CTR_LAUNCHED();
    CTR_TRY(exclusive_scan_i32(counts.as<int32_t>(), offsets.as<int32_t>(), nchunks, st, scratch));
    int32_t Mh = 0;
    CTR_CUDA_TRY(cudaMemcpyAsync(&Mh, offsets.as<int32_t>() + nchunks, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CTR_CUDA_TRY(cudaStreamSynchronize(st));
    CTR_TRY(check_device_error(s, "signed distance"));
    if (Mh <= 0) return fail(CTR_ERR_EMPTY_TUBE, "no grid node with |d| < eps");
    const int64_t M = Mh;
    s->M = M;
    CTR_TRY(s->lin.alloc(sizeof(int64_t) * M));
    CTR_TRY(node_of.alloc(sizeof(int32_t) * total));
    CTR_CUDA_TRY(cudaMemsetAsync(node_of.p, 0xff, sizeof(int32_t) * total, st));
    tube_compact_kernel<<<(unsigned)nchunks, kScanThreads, 0, st>>>(d_sdist, total, s->eps, offsets.as<int32_t>(),
                                                                    s->lin.as<int64_t>(), node_of.as<int32_t>());
    CTR_LAUNCHED();

    CTR_TRY(s->nodes.alloc(sizeof(double) * NodeArrays::kCount * M));
    double* b = s->nodes.as<double>();
    double** f[NodeArrays::kCount] = {&s->na.Px, &s->na.Py, &s->na.Pz, &s->na.nx, &s->na.ny, &s->na.nz,
                                      &s->na.W, &s->na.d, &s->na.t1x, &s->na.t1y, &s->na.t1z,
                                      &s->na.t2x, &s->na.t2y, &s->na.t2z, &s->na.m1, &s->na.m2};
    for (int q = 0; q < NodeArrays::kCount; ++q) *f[q] = b + (size_t)q * M;
    CTR_TRY(s->src32.alloc(sizeof(float4) * 4 * M));
    CTR_TRY(s->src64.alloc(sizeof(double4) * 2 * M));
    CTR_TRY(s->bad.alloc(M));
    geometry_kernel<<<grid_for(M, 128), 128, 0, st>>>(d_sdist, s->lin.as<int64_t>(), M, s->n[0], s->n[1], s->n[2],
                                                     s->origin[0], s->origin[1], s->origin[2], s->h, s->eps,
                                                     s->opt.method == CTR_METHOD_KREG ? 1 : 0, s->na,
                                                     s->bad.as<uint8_t>(), s->src32.as<float4>(),
                                                     s->src64.as<double4>(), s->err.as<int>());
    CTR_LAUNCHED();
    CTR_TRY(check_device_error(s, "geometry"));

    // correction-weight tables (Ewald, computed once per device), then the correction matrix
    const double* tab = nullptr;
    CTR_TRY(weight_tables_cached(s->device, st, &tab));
    CTR_TRY(setup_corrections(s, tab, node_of.as<int32_t>()));
    CTR_CUDA_TRY(cudaStreamSynchronize(st));   // temporaries are freed on return
    return CTR_OK;
}

int setup_rhs(ctr_ibim* s) {
    CTR_TRY(s->rhs.alloc(sizeof(double) * 2 * s->M));
    rhs_kernel<<<grid_for(s->M, 128), 128, 0, s->stream>>>(s->na, s->M, s->charges.as<double>(), s->nc, s->eps_in,
                                                          s->rhs.as<double>());
    CTR_LAUNCHED();
    return CTR_OK;
}

}  // namespace ctr
