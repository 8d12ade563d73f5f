// Correction weights (Sec. 2.4): tables of Sec. 2.4.2 and the correction matrix Omega.
//
// Tables.  The paper defines omega[s; alpha, beta] as the limit of Eq. (2.29)
// and evaluates it by refining h.  For s = |y|^-1 e^{i k psi} that limit is
// minus the regularised punctured lattice sum
//     -Z(alpha) = -( sum'_{n != 0} f(n - (alpha, beta)) )_reg,   f(x) = (x1 + i x2)^k |x|^-(k+1),
// which this file evaluates by Ewald splitting instead of by refinement:
// with s = (k+1)/2 and the Mellin form |x|^-2s = pi^s/Gamma(s) int t^{s-1} e^{-pi t|x|^2} dt
// split at t = 1, the t >= 1 part is a rapidly convergent real-space sum with
// Q(s, pi|x|^2) = Gamma(s, pi|x|^2)/Gamma(s), and the t < 1 part is
// Poisson-summed (Hecke's identity: the Fourier transform of a solid harmonic
// times a Gaussian is (-i)^k the same harmonic times a Gaussian):
//   Z = sum_{n != 0} e^{ik psi(n-a)}/|n-a| Q(s, pi|n-a|^2)
//       - (x1 + i x2)^k pi^s [gamma(s, pi|a|^2)/(pi|a|^2)^s] / Gamma(s)     (n = 0 minus f(-a); x = -a)
//       + (-i)^k sum_{m != 0} e^{ik psi(m)}/|m| Q(s, pi|m|^2) e^{-2 pi i m.a}
//       - 2 [k = 0]                                                          (analytic continuation of m = 0)
// Both routes give the same numbers (to ~1e-14); refinement needs ~10^5
// lattice points per value, Ewald a few hundred.
//
// K-reg rows (Sec. 2.3) replace CTR2 at targets the hybrid classification
// marks bad (Sec. 3.2): every tube node y in the cylinder around the normal
// line of radius tau = 2h (distance of the tangent-plane projections of y and
// x, computed unfused as v = y - P, s = (v0 n0 + v1 n1) + v2 n2,
// t = v - s n, (t0 t0 + t1 t1) + t2 t2 < tau^2), in ascending node order, with
// weights C11 = C21 = C22 = 0 and C12 = (e^{-kappa tau} - 1 + kappa tau)/(2 pi kappa tau^2).
//
// Correction matrix (per target node y_i, Sec. 2.4): the planes t_k of the
// dominant axis, the singular line of Eq. (2.19), the nearest node and shift
// (alpha, beta), the angular functions of the theorem in Sec. 2.4.1 (Eq. 2.28,
// with kappa^2 in s0^(21)), their even Fourier coefficients by a direct DFT of
// 64 samples, and the tensor Lagrange (degree 5) interpolation of the tables.
#include <mutex>

#include "common.cuh"

namespace ctr {

namespace {

__constant__ double c_cos64[kSamples];
__constant__ double c_sin64[kSamples];

// Q(q + 1/2, x) = Gamma(q+1/2, x)/Gamma(q+1/2) = erfc(sqrt x) + sum_{j<q} x^{j+1/2} e^{-x} / Gamma(j + 3/2)
__device__ double reg_upper_gamma_half(int q, double x) {
    double Q = erfc(sqrt(x));
    double term = sqrt(x) * exp(-x) / (0.5 * sqrt(kPi));   // x^{1/2} e^{-x} / Gamma(3/2)
    for (int j = 0; j < q; ++j) {
        Q += term;
        term *= x / (j + 1.5);                              // x^{j+3/2}/Gamma(j+5/2)
    }
    return Q;
}

// gamma(s, x) / x^s = e^{-x} sum_{j>=0} x^j / (s (s+1) ... (s+j))
__device__ double lower_gamma_scaled(double s, double x) {
    double term = 1.0 / s, sum = term;
    for (int j = 1; j < 200; ++j) {
        term *= x / (s + j);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return exp(-x) * sum;
}

__device__ double gamma_half(int q) {   // Gamma(q + 1/2)
    double g = sqrt(kPi);
    for (int j = 0; j < q; ++j) g *= (j + 0.5);
    return g;
}

__device__ void cpow(double c, double s, int k, double& re, double& im) {
    double pr = 1.0, pi = 0.0;
    for (int j = 0; j < k; ++j) {
        double nr = pr * c - pi * s, ni = pr * s + pi * c;
        pr = nr; pi = ni;
    }
    re = pr; im = pi;
}

__global__ void ewald_tables_kernel(double* __restrict__ T) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= kModes * kTabN * kTabN) return;
    const int q = idx / (kTabN * kTabN);
    const int ia = (idx / kTabN) % kTabN, ib = idx % kTabN;
    const int k = 2 * q;
    const double s = 0.5 * (k + 1);
    const double a0 = (ia - kTabHalf) * kTabSpacing, a1 = (ib - kTabHalf) * kTabSpacing;
    constexpr int R = 7;
    double zr = 0.0, zi = 0.0;
    // real space, n != 0
    for (int n2 = -R; n2 <= R; ++n2)
        for (int n1 = -R; n1 <= R; ++n1) {
            if (n1 == 0 && n2 == 0) continue;
            const double x1 = n1 - a0, x2 = n2 - a1;
            const double r = sqrt(x1 * x1 + x2 * x2);
            double er, ei;
            cpow(x1 / r, x2 / r, k, er, ei);
            const double w = reg_upper_gamma_half(q, kPi * r * r) / r;
            zr += w * er;
            zi += w * ei;
        }
    // n = 0 term minus f(-a)
    {
        const double x1 = -a0, x2 = -a1;
        double pr, pi;
        cpow(x1, x2, k, pr, pi);   // (x1 + i x2)^k
        const double x = kPi * (x1 * x1 + x2 * x2);
        const double f = pow(kPi, s) * lower_gamma_scaled(s, x) / gamma_half(q);
        zr -= pr * f;
        zi -= pi * f;
    }
    // reciprocal space, m != 0: (-i)^k = (-1)^(k/2) for even k
    const double sgn = (q & 1) ? -1.0 : 1.0;
    double rr = 0.0, ri = 0.0;
    for (int m2 = -R; m2 <= R; ++m2)
        for (int m1 = -R; m1 <= R; ++m1) {
            if (m1 == 0 && m2 == 0) continue;
            const double r = sqrt((double)(m1 * m1 + m2 * m2));
            double er, ei;
            cpow(m1 / r, m2 / r, k, er, ei);
            const double w = reg_upper_gamma_half(q, kPi * r * r) / r;
            double sp, cp;
            sincospi(-2.0 * (m1 * a0 + m2 * a1), &sp, &cp);
            rr += w * (er * cp - ei * sp);
            ri += w * (er * sp + ei * cp);
        }
    zr += sgn * rr;
    zi += sgn * ri;
    if (k == 0) zr -= 2.0;
    T[((0 * kModes + q) * kTabN + ia) * kTabN + ib] = -zr;
    T[((1 * kModes + q) * kTabN + ia) * kTabN + ib] = -zi;
}

struct PlaneCtx {
    int64_t nx, ny, nz;
    double origin[3];
    double h, eps;
    int K;       // planes on each side
    int Kc;      // K-reg cylinder search half-width (grid nodes)
    double tau;  // K-reg radius
};

// Visits the K-reg cylinder nodes of target i in ascending node order.
template <typename F>
__device__ void visit_cylinder(const PlaneCtx& c, const NodeArrays& na, const int64_t* lin,
                               const int32_t* node_of, int64_t i, F&& fn) {
    const double P[3] = {na.Px[i], na.Py[i], na.Pz[i]};
    const double n[3] = {na.nx[i], na.ny[i], na.nz[i]};
    const int64_t g = lin[i];
    const int64_t ci = g % c.nx, cj = (g / c.nx) % c.ny, ck = g / (c.nx * c.ny);
    const double tau2 = __dmul_rn(c.tau, c.tau);
    for (int64_t k = max((int64_t)0, ck - c.Kc); k <= min(c.nz - 1, ck + c.Kc); ++k)
        for (int64_t j = max((int64_t)0, cj - c.Kc); j <= min(c.ny - 1, cj + c.Kc); ++j)
            for (int64_t q = max((int64_t)0, ci - c.Kc); q <= min(c.nx - 1, ci + c.Kc); ++q) {
                const int32_t m = node_of[q + c.nx * (j + c.ny * k)];
                if (m < 0) continue;
                const double y0 = __dadd_rn(c.origin[0], __dmul_rn(c.h, (double)q));
                const double y1 = __dadd_rn(c.origin[1], __dmul_rn(c.h, (double)j));
                const double y2 = __dadd_rn(c.origin[2], __dmul_rn(c.h, (double)k));
                const double v0 = __dsub_rn(y0, P[0]), v1 = __dsub_rn(y1, P[1]), v2 = __dsub_rn(y2, P[2]);
                const double sdot = __dadd_rn(__dadd_rn(__dmul_rn(v0, n[0]), __dmul_rn(v1, n[1])), __dmul_rn(v2, n[2]));
                const double t0 = __dsub_rn(v0, __dmul_rn(sdot, n[0]));
                const double t1 = __dsub_rn(v1, __dmul_rn(sdot, n[1]));
                const double t2 = __dsub_rn(v2, __dmul_rn(sdot, n[2]));
                const double q2 = __dadd_rn(__dadd_rn(__dmul_rn(t0, t0), __dmul_rn(t1, t1)), __dmul_rn(t2, t2));
                if (q2 < tau2) fn(m, 0.0, 0.0, 0.0);
            }
}

// Visits the correction nodes of target i in ascending plane order.
// fn(m, alpha, beta, eta) is called for each tube node found.
template <typename F>
__device__ void visit_planes(const PlaneCtx& c, const NodeArrays& na, const int64_t* lin,
                             const int32_t* node_of, int64_t i, F&& fn) {
    const double P[3] = {na.Px[i], na.Py[i], na.Pz[i]};
    const double n[3] = {na.nx[i], na.ny[i], na.nz[i]};
    int a = 0;
    if (fabs(n[1]) > fabs(n[a])) a = 1;
    if (fabs(n[2]) > fabs(n[a])) a = 2;
    const int b = (a == 0) ? 1 : 0;
    const int cc = (a == 2) ? 1 : 2;
    const int64_t g = lin[i];
    const int64_t ijk[3] = {g % c.nx, (g / c.nx) % c.ny, g / (c.nx * c.ny)};
    const int64_t dims[3] = {c.nx, c.ny, c.nz};
    const double lim = __dadd_rn(c.eps, c.h);
    for (int64_t ka = ijk[a] - c.K; ka <= ijk[a] + c.K; ++ka) {
        const double t = __dadd_rn(c.origin[a], __dmul_rn(c.h, (double)ka));
        const double eta = __ddiv_rn(__dsub_rn(t, P[a]), n[a]);
        if (fabs(eta) > lim) continue;
        const double u0b = __dadd_rn(P[b], __dmul_rn(eta, n[b]));
        const double u0c = __dadd_rn(P[cc], __dmul_rn(eta, n[cc]));
        const double sb = __ddiv_rn(__dsub_rn(u0b, c.origin[b]), c.h);
        const double sc = __ddiv_rn(__dsub_rn(u0c, c.origin[cc]), c.h);
        const double kb = floor(__dadd_rn(sb, 0.5));
        const double kc = floor(__dadd_rn(sc, 0.5));
        const double alpha = __dsub_rn(sb, kb), beta = __dsub_rn(sc, kc);
        int64_t idx[3];
        idx[a] = ka;
        idx[b] = (int64_t)kb;
        idx[cc] = (int64_t)kc;
        if (idx[0] < 0 || idx[1] < 0 || idx[2] < 0 || idx[0] >= dims[0] || idx[1] >= dims[1] || idx[2] >= dims[2])
            continue;
        const int32_t m = node_of[idx[0] + c.nx * (idx[1] + c.ny * idx[2])];
        if (m < 0) continue;
        fn(m, alpha, beta, eta);
    }
}

__global__ void corr_count_kernel(PlaneCtx c, NodeArrays na, const int64_t* __restrict__ lin,
                                  const int32_t* __restrict__ node_of, const uint8_t* __restrict__ bad, int64_t M,
                                  int32_t* __restrict__ counts) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    int cnt = 0;
    auto inc = [&](int32_t, double, double, double) { ++cnt; };
    if (bad[i]) visit_cylinder(c, na, lin, node_of, i, inc);
    else visit_planes(c, na, lin, node_of, i, inc);
    counts[i] = cnt;
}

__global__ void corr_fill_kernel(PlaneCtx c, NodeArrays na, const int64_t* __restrict__ lin,
                                 const int32_t* __restrict__ node_of, const uint8_t* __restrict__ bad, int64_t M,
                                 const int32_t* __restrict__ ptr, int32_t* __restrict__ node,
                                 double* __restrict__ ab_eta, int64_t E, int32_t* __restrict__ excl) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    int e = ptr[i];
    const int e0 = e;
    auto put = [&](int32_t m, double alpha, double beta, double eta) {
        node[e] = m;
        ab_eta[e] = alpha;
        ab_eta[E + e] = beta;
        ab_eta[2 * E + e] = eta;
        ++e;
    };
    if (bad[i]) visit_cylinder(c, na, lin, node_of, i, put);
    else visit_planes(c, na, lin, node_of, i, put);
    // sorted copy (insertion sort; at most a few entries) for the dense-sum exclusion
    for (int p = e0; p < e; ++p) {
        int32_t v = node[p];
        int q = p;
        while (q > e0 && excl[q - 1] > v) {
            excl[q] = excl[q - 1];
            --q;
        }
        excl[q] = v;
    }
}

__device__ void lagrange6(double x, int& i0, double cw[6]) {
    const int f = (int)floor(x * 32.0);
    i0 = f - 2;
    double xs[6];
    for (int l = 0; l < 6; ++l) xs[l] = (i0 + l) * kTabSpacing;
    for (int mm = 0; mm < 6; ++mm) {
        double v = 1.0;
        for (int l = 0; l < 6; ++l)
            if (l != mm) v *= (x - xs[l]) / (xs[mm] - xs[l]);
        cw[mm] = v;
    }
}

__global__ void corr_weight_kernel(NodeArrays na, const uint8_t* __restrict__ bad, const int32_t* __restrict__ ptr,
                                   int64_t M, const double* __restrict__ ab_eta, int64_t E,
                                   const double* __restrict__ T, double c11, double c22, double kappa2,
                                   double w12_ctr, double w12_kreg, double* __restrict__ w, int* __restrict__ err) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    // target of entry e: binary search in ptr
    int64_t lo = 0, hi = M;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) / 2;
        if (ptr[mid] <= e) lo = mid; else hi = mid;
    }
    const int64_t i = lo;
    if (bad[i]) {   // K-reg row: only the constant C12 (Sec. 2.3)
        w[e] = w[E + e] = w[2 * E + e] = 0.0;
        w[3 * E + e] = w12_kreg;
        return;
    }
    w[3 * E + e] = w12_ctr;
    const double alpha = ab_eta[e], beta = ab_eta[E + e], eta = ab_eta[2 * E + e];
    const double n[3] = {na.nx[i], na.ny[i], na.nz[i]};
    int a = 0;
    if (fabs(n[1]) > fabs(n[a])) a = 1;
    if (fabs(n[2]) > fabs(n[a])) a = 2;
    const int b = (a == 0) ? 1 : 0;
    const int cc = (a == 2) ? 1 : 2;
    const double t1[3] = {na.t1x[i], na.t1y[i], na.t1z[i]};
    const double t2[3] = {na.t2x[i], na.t2y[i], na.t2z[i]};
    const double A00 = t1[b], A01 = t1[cc], A10 = t2[b], A11 = t2[cc];   // rows Q tau_1, Q tau_2 (Eq. 2.26)
    const double m1 = na.m1[i], m2 = na.m2[i];
    const double D1 = 1.0 / (1.0 - eta * m1), D2 = 1.0 / (1.0 - eta * m2);   // D0 = (I - eta M)^-1
    double aA[kModes], bA[kModes], aB[kModes], bB[kModes];
    for (int q = 0; q < kModes; ++q) aA[q] = bA[q] = aB[q] = bB[q] = 0.0;
    const double inv8pi = 1.0 / (8.0 * kPi);
    for (int j = 0; j < kSamples; ++j) {
        const double ct = c_cos64[j], st = c_sin64[j];
        const double v1 = D1 * (A00 * ct + A01 * st);
        const double v2 = D2 * (A10 * ct + A11 * st);
        const double vv = v1 * v1 + v2 * v2;
        const double vn = sqrt(vv);
        const double lA = (m1 * v1 * v1 + m2 * v2 * v2) * inv8pi / (vv * vn);
        const double lB = inv8pi / vn;
        for (int q = 0; q < kModes; ++q) {
            const int jk = (j * 2 * q) & (kSamples - 1);
            aA[q] += lA * c_cos64[jk];
            bA[q] += lA * c_sin64[jk];
            aB[q] += lB * c_cos64[jk];
            bB[q] += lB * c_sin64[jk];
        }
    }
    const double sc0 = 1.0 / kSamples, sc = 2.0 / kSamples;
    aA[0] *= sc0; aB[0] *= sc0; bA[0] = bB[0] = 0.0;
    for (int q = 1; q < kModes; ++q) { aA[q] *= sc; bA[q] *= sc; aB[q] *= sc; bB[q] *= sc; }
    int i0, j0;
    double ca[6], cb[6];
    lagrange6(alpha, i0, ca);
    lagrange6(beta, j0, cb);
    if (i0 + kTabHalf < 0 || j0 + kTabHalf < 0 || i0 + 5 + kTabHalf >= kTabN || j0 + 5 + kTabHalf >= kTabN) {
        atomicOr(err, kErrCapacity);   // shift outside the tabulated range (cannot happen for |alpha| <= 1/2)
        w[e] = w[E + e] = w[2 * E + e] = w[3 * E + e] = 0.0;
        return;
    }
    double wA = 0.0, wB = 0.0;
    for (int p = 0; p < 6; ++p)
        for (int r = 0; r < 6; ++r) {
            const int ia = i0 + p + kTabHalf, ib = j0 + r + kTabHalf;
            double tA = 0.0, tB = 0.0;
            for (int q = 0; q < kModes; ++q) {
                const double Tc = T[((0 * kModes + q) * kTabN + ia) * kTabN + ib];
                const double Ts = T[((1 * kModes + q) * kTabN + ia) * kTabN + ib];
                tA += aA[q] * Tc + bA[q] * Ts;
                tB += aB[q] * Tc + bB[q] * Ts;
            }
            wA += ca[p] * cb[r] * tA;
            wB += ca[p] * cb[r] * tB;
        }
    w[e] = c11 * wA;           // omega11
    w[E + e] = kappa2 * wB;    // omega21
    w[2 * E + e] = c22 * wA;   // omega22
}

bool g_trig_ready[64] = {false};

int upload_trig(int device) {
    if (device >= 0 && device < 64 && g_trig_ready[device]) return CTR_OK;
    double c[kSamples], s[kSamples];
    for (int j = 0; j < kSamples; ++j) {
        c[j] = cos(2.0 * kPi * j / kSamples);
        s[j] = sin(2.0 * kPi * j / kSamples);
    }
    CTR_CUDA_TRY(cudaMemcpyToSymbol(c_cos64, c, sizeof(c)));
    CTR_CUDA_TRY(cudaMemcpyToSymbol(c_sin64, s, sizeof(s)));
    if (device >= 0 && device < 64) g_trig_ready[device] = true;
    return CTR_OK;
}

}  // namespace

int weight_tables_device(double* d_tables, cudaStream_t st) {
    const int n = kModes * kTabN * kTabN;
    ewald_tables_kernel<<<grid_for(n, 128), 128, 0, st>>>(d_tables);
    CTR_LAUNCHED();
    return CTR_OK;
}

// The tables depend on nothing but their grid: computed once per device (complete before use).
int weight_tables_cached(int dev, cudaStream_t st, const double** out) {
    static std::mutex mu;
    static DevBuf tabs[64];
    static bool ready[64] = {false};
    if (dev < 0 || dev >= 64) return fail(CTR_ERR_INVALID, "device index");
    std::lock_guard<std::mutex> lk(mu);
    if (!ready[dev]) {
        CTR_TRY(tabs[dev].alloc(sizeof(double) * kTabSize));
        CTR_TRY(weight_tables_device(tabs[dev].as<double>(), st));
        CTR_CUDA_TRY(cudaStreamSynchronize(st));
        ready[dev] = true;
    }
    *out = tabs[dev].as<double>();
    return CTR_OK;
}

int setup_corrections(ctr_ibim* s, const double* d_tables, const int32_t* d_node_of) {
    cudaStream_t st = s->stream;
    const int64_t M = s->M;
    CTR_TRY(upload_trig(s->device));
    PlaneCtx c;
    c.nx = s->n[0]; c.ny = s->n[1]; c.nz = s->n[2];
    for (int q = 0; q < 3; ++q) c.origin[q] = s->origin[q];
    c.h = s->h;
    c.eps = s->eps;
    c.K = (int)ceil(2.0 * s->eps / s->h) + 2;
    c.tau = 2.0 * s->h;
    c.Kc = (int)ceil((s->eps + c.tau) / s->h) + 1;
    DevBuf counts, scratch, abeta;
    CTR_TRY(counts.alloc(sizeof(int32_t) * M));
    CTR_TRY(s->corr_ptr.alloc(sizeof(int32_t) * (M + 1)));
    corr_count_kernel<<<grid_for(M, 128), 128, 0, st>>>(c, s->na, s->lin.as<int64_t>(), d_node_of,
                                                       s->bad.as<uint8_t>(), M, counts.as<int32_t>());
    CTR_LAUNCHED();
    CTR_TRY(exclusive_scan_i32(counts.as<int32_t>(), s->corr_ptr.as<int32_t>(), M, st, scratch));
    int32_t Eh = 0;
    CTR_CUDA_TRY(cudaMemcpyAsync(&Eh, s->corr_ptr.as<int32_t>() + M, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CTR_CUDA_TRY(cudaStreamSynchronize(st));
    const int64_t E = Eh;
    s->E = E;
    CTR_TRY(s->corr_node.alloc(sizeof(int32_t) * (E > 0 ? E : 1)));
    CTR_TRY(s->excl.alloc(sizeof(int32_t) * (E > 0 ? E : 1)));
    CTR_TRY(s->corr_w.alloc(sizeof(double) * 4 * (E > 0 ? E : 1)));
    CTR_TRY(abeta.alloc(sizeof(double) * 3 * (E > 0 ? E : 1)));
    corr_fill_kernel<<<grid_for(M, 128), 128, 0, st>>>(c, s->na, s->lin.as<int64_t>(), d_node_of,
                                                      s->bad.as<uint8_t>(), M, s->corr_ptr.as<int32_t>(),
                                                      s->corr_node.as<int32_t>(), abeta.as<double>(), E,
                                                      s->excl.as<int32_t>());
    CTR_LAUNCHED();
    if (E > 0) {
        const double c11 = 1.0 - s->eps_out / s->eps_in;
        const double c22 = 1.0 - s->eps_in / s->eps_out;
        const double tau = 2.0 * s->h;
        const double k = s->kappa;
        const double w12_kreg = (k == 0.0) ? 0.0 : (exp(-k * tau) - 1.0 + k * tau) / (2.0 * kPi * k * tau * tau);
        corr_weight_kernel<<<grid_for(E, 128), 128, 0, st>>>(s->na, s->bad.as<uint8_t>(), s->corr_ptr.as<int32_t>(), M,
                                                            abeta.as<double>(), E, d_tables, c11, c22, k * k,
                                                            k / (4.0 * kPi), w12_kreg, s->corr_w.as<double>(),
                                                            s->err.as<int>());
        CTR_LAUNCHED();
    }
    CTR_CUDA_TRY(cudaStreamSynchronize(st));
    return CTR_OK;
}

}  // namespace ctr
