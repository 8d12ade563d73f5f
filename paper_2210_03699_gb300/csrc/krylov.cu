// GMRES on the device (Sec. 2.5: "standard GMRES") and FP64 iterative refinement.
//
// Arnoldi uses classical Gram-Schmidt applied twice (CGS2: as stable as
// modified Gram-Schmidt, but two batched passes instead of j+1 dependent
// ones); the Hessenberg columns, Givens rotations, the least-squares right
// side and the triangular solve are FP64 device scalars updated by one
// thread.  All reductions sum per-block partials in a fixed order, so a
// solve is bitwise reproducible run to run.
//
// Right preconditioning by the diagonal Lambda = diag(lambda_1 I, lambda_2 I)
// of Eq. (2.30): GMRES runs on A Lambda^-1 u = b and returns x = Lambda^-1 u.
// It minimises the same residual |b - A x| and cuts the iteration count about
// threefold (the two blocks of unknowns differ in scale by eps_E/eps_I).
//
// Precision modes:
//   CTR_FP64/DF64    GMRES on the FP64 (or float-float) pair operator, x0 = 0.
//   CTR_FP32_REFINE  x = 0; repeat { r = g - A x (pairs in opt.residual: float-float
//                    or FP64); stop if |r| <= tol |g|; GMRES on A32 d = r to
//                    inner_tol; x += d }   (A32: FP32 pairs, FP64 everything else).
#include <cmath>

#include "common.cuh"

namespace ctr {

namespace {

constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[kRedThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kRedThreads / 32; ++w) t += sh[w];
    __syncthreads();
    return t;   // valid in thread 0
}

// part[i * nblk + b] = sum over block b's chunk of A[i][t] * w[t], i < count
__global__ void dots_partial_kernel(const double* __restrict__ A, int64_t lda, int count,
                                    const double* __restrict__ w, int64_t n, int64_t chunk,
                                    double* __restrict__ part, int nblk) {
    const int64_t t0 = (int64_t)blockIdx.x * chunk;
    const int64_t t1 = min(n, t0 + chunk);
    for (int i = 0; i < count; ++i) {
        const double* a = A + (size_t)i * lda;
        double v = 0.0;
        for (int64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) v += a[t] * w[t];
        v = block_sum(v);
        if (threadIdx.x == 0) part[(size_t)i * nblk + blockIdx.x] = v;
    }
}

// out[i] (+)= sum_b part[i * nblk + b]
__global__ void dots_final_kernel(const double* __restrict__ part, int nblk, double* __restrict__ out, int accumulate) {
    const int i = blockIdx.x;
    double v = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) v += part[(size_t)i * nblk + b];
    v = block_sum(v);
    if (threadIdx.x == 0) out[i] = accumulate ? out[i] + v : v;
}

// w[t] -= sum_i A[i][t] c[i]
__global__ void sub_multi_kernel(const double* __restrict__ A, int64_t lda, int count, const double* __restrict__ c,
                                 double* __restrict__ w, int64_t n) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double v = w[t];
    for (int i = 0; i < count; ++i) v -= A[(size_t)i * lda + t] * c[i];
    w[t] = v;
}

// x[t] += sum_i A[i][t] c[i]
__global__ void add_multi_kernel(const double* __restrict__ A, int64_t lda, int count, const double* __restrict__ c,
                                 double* __restrict__ x, int64_t n) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double v = x[t];
    for (int i = 0; i < count; ++i) v += A[(size_t)i * lda + t] * c[i];
    x[t] = v;
}

__global__ void scale_kernel(const double* __restrict__ a, const double* __restrict__ sc, int inv, double* __restrict__ out,
                             int64_t n) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double f = inv ? 1.0 / sc[0] : sc[0];
    out[t] = a[t] * f;
}

// out = Lambda^-1 a (first M entries / lambda_1, last M / lambda_2)
__global__ void diag_inv_kernel(const double* __restrict__ a, double* __restrict__ out, int64_t M, double il1,
                                double il2) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * M) return;
    out[t] = a[t] * (t < M ? il1 : il2);
}

// x[t] += Lambda^-1 (sum_i A[i][t] c[i])
__global__ void add_multi_prec_kernel(const double* __restrict__ A, int64_t lda, int count, const double* __restrict__ c,
                                      double* __restrict__ x, int64_t M, double il1, double il2) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * M) return;
    double v = 0.0;
    for (int i = 0; i < count; ++i) v += A[(size_t)i * lda + t] * c[i];
    x[t] += v * (t < M ? il1 : il2);
}

__global__ void axpby_kernel(double alpha, const double* __restrict__ a, double beta, const double* __restrict__ b,
                             double* __restrict__ out, int64_t n) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    out[t] = alpha * a[t] + beta * b[t];
}

// Scalars layout (device): sc[0] = |w| (then beta), sc[1] = residual estimate |s_{j+1}|,
// sc[2] = converged flag (0/1), sc[3] = breakdown flag.
// Hcol: c[0..j] from the two Gram-Schmidt passes (already summed), nrm2 = |w|^2.
__global__ void givens_kernel(double* __restrict__ H, int ldh, int j, const double* __restrict__ c,
                              const double* __restrict__ nrm2, double* __restrict__ cs, double* __restrict__ sn,
                              double* __restrict__ sv, double* __restrict__ sc, double tol_abs) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double* col = H + (size_t)j * ldh;
    for (int i = 0; i <= j; ++i) col[i] = c[i];
    const double hn = sqrt(nrm2[0]);
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
    }
    const double den = hypot(col[j], col[j + 1]);
    cs[j] = col[j] / den;
    sn[j] = col[j + 1] / den;
    col[j] = den;
    col[j + 1] = 0.0;
    sv[j + 1] = -sn[j] * sv[j];
    sv[j] = cs[j] * sv[j];
    sc[0] = hn;
    sc[1] = fabs(sv[j + 1]);
    sc[2] = (fabs(sv[j + 1]) <= tol_abs) ? 1.0 : 0.0;
    sc[3] = (hn == 0.0 || !isfinite(hn)) ? 1.0 : 0.0;
}

__global__ void init_rhs_kernel(double* __restrict__ sv, int m, double beta) {
    int i = threadIdx.x + blockIdx.x * blockDim.x;
    if (i <= m) sv[i] = (i == 0) ? beta : 0.0;
}

// back substitution R y = s (R upper triangular in H, k columns)
__global__ void upper_solve_kernel(const double* __restrict__ H, int ldh, int k, const double* __restrict__ sv,
                                   double* __restrict__ y) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double v = sv[i];
        for (int l = i + 1; l < k; ++l) v -= H[(size_t)l * ldh + i] * y[l];
        y[i] = v / H[(size_t)i * ldh + i];
    }
}

struct Vecs {
    double *x, *r, *w, *d, *t, *u;
};

Vecs vecs_of(ctr_ibim* s) {
    double* b = s->vecs.as<double>();
    const int64_t n = 2 * s->M;
    return Vecs{b, b + n, b + 2 * n, b + 3 * n, b + 4 * n, b + 5 * n};
}

int ensure_krylov(ctr_ibim* s) {
    Krylov& k = s->kr;
    const int64_t n = 2 * s->M;
    int m = s->opt.restart;
    if (k.m == m && k.n == n) return CTR_OK;
    k.m = m;
    k.n = n;
    k.nblk = (int)std::min<int64_t>(std::max<int64_t>(1, (n + 4095) / 4096), 608);
    CTR_TRY(k.V.alloc(sizeof(double) * (size_t)(m + 1) * n));
    CTR_TRY(k.H.alloc(sizeof(double) * (size_t)(m + 1) * m));
    CTR_TRY(k.cs.alloc(sizeof(double) * m));
    CTR_TRY(k.sn.alloc(sizeof(double) * m));
    CTR_TRY(k.s.alloc(sizeof(double) * (m + 1)));
    CTR_TRY(k.y.alloc(sizeof(double) * (m + 1) * 3));   // y, c (GS coefficients), tmp
    CTR_TRY(k.part.alloc(sizeof(double) * (size_t)(m + 1) * k.nblk));
    CTR_TRY(k.scal.alloc(sizeof(double) * 8));
    return CTR_OK;
}

// out[i] = <A_i, w> for i < count (A rows of length n with stride lda); accumulate: out += ...
int dots(ctr_ibim* s, const double* A, int64_t lda, int count, const double* w, int64_t n, double* out,
         int accumulate) {
    Krylov& k = s->kr;
    const int64_t chunk = (n + k.nblk - 1) / k.nblk;
    dots_partial_kernel<<<k.nblk, kRedThreads, 0, s->stream>>>(A, lda, count, w, n, chunk, k.part.as<double>(), k.nblk);
    CTR_LAUNCHED();
    dots_final_kernel<<<count, kRedThreads, 0, s->stream>>>(k.part.as<double>(), k.nblk, out, accumulate);
    CTR_LAUNCHED();
    return CTR_OK;
}

int read_scalars(ctr_ibim* s, double* h, int count) {
    CTR_CUDA_TRY(cudaMemcpyAsync(h, s->kr.scal.p, sizeof(double) * count, cudaMemcpyDeviceToHost, s->stream));
    CTR_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return CTR_OK;
}

// GMRES for A x = b with x0 = 0 (x overwritten).  tol_rel relative to |b|.
int gmres(ctr_ibim* s, int precision, const double* b, double* x, double tol_rel, int64_t& budget,
          ctr_solve_info* info, bool& converged) {
    Krylov& k = s->kr;
    const int64_t n = 2 * s->M;
    const int m = k.m;
    double* V = k.V.as<double>();
    double* H = k.H.as<double>();
    double* c = k.y.as<double>() + (m + 1);
    double* nrm = k.y.as<double>() + 2 * (m + 1);
    double* sc = k.scal.as<double>();
    Vecs v = vecs_of(s);
    const unsigned gb = grid_for(n, 256);
    cudaStream_t st = s->stream;
    const double il1 = 2.0 / (1.0 + s->eps_out / s->eps_in);   // 1 / lambda_1
    const double il2 = 2.0 / (1.0 + s->eps_in / s->eps_out);   // 1 / lambda_2
    converged = false;
    CTR_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    double bnorm = 0.0;
    CTR_TRY(device_dot(s, b, b, n, &bnorm));
    bnorm = std::sqrt(bnorm);
    if (bnorm == 0.0) {
        converged = true;
        return CTR_OK;
    }
    const double tol_abs = tol_rel * bnorm;
    double beta = bnorm;
    const double* start = b;
    while (budget > 0) {
        // V[0] = start / beta
        axpby_kernel<<<gb, 256, 0, st>>>(1.0 / beta, start, 0.0, start, V, n);
        CTR_LAUNCHED();
        init_rhs_kernel<<<1, 1024, 0, st>>>(k.s.as<double>(), m, beta);
        CTR_LAUNCHED();
        int kdone = 0;
        double hsc[4] = {0, 0, 0, 0};
        for (int j = 0; j < m && budget > 0; ++j) {
            double* w = V + (size_t)(j + 1) * n;   // build the next vector in place
            diag_inv_kernel<<<gb, 256, 0, st>>>(V + (size_t)j * n, v.w, s->M, il1, il2);
            CTR_LAUNCHED();
            CTR_TRY(apply_operator(s, v.w, w, precision));
            if (precision == CTR_FP32_REFINE) info->matvecs_fp32++; else info->matvecs_fp64++;
            // CGS2
            CTR_TRY(dots(s, V, n, j + 1, w, n, c, 0));
            sub_multi_kernel<<<gb, 256, 0, st>>>(V, n, j + 1, c, w, n);
            CTR_LAUNCHED();
            CTR_TRY(dots(s, V, n, j + 1, w, n, nrm + 1, 0));   // second pass coefficients in nrm[1..]
            sub_multi_kernel<<<gb, 256, 0, st>>>(V, n, j + 1, nrm + 1, w, n);
            CTR_LAUNCHED();
            axpby_kernel<<<grid_for(j + 1, 128), 128, 0, st>>>(1.0, c, 1.0, nrm + 1, c, j + 1);
            CTR_LAUNCHED();
            CTR_TRY(dots(s, w, n, 1, w, n, nrm, 0));
            givens_kernel<<<1, 1, 0, st>>>(H, m + 1, j, c, nrm, k.cs.as<double>(), k.sn.as<double>(),
                                           k.s.as<double>(), sc, tol_abs);
            CTR_LAUNCHED();
            scale_kernel<<<gb, 256, 0, st>>>(w, sc, 1, w, n);
            CTR_LAUNCHED();
            CTR_TRY(read_scalars(s, hsc, 4));
            kdone = j + 1;
            --budget;
            info->iterations++;
            if (!std::isfinite(hsc[1])) return fail(CTR_ERR_NUMERIC, "GMRES: non-finite residual");
            if (hsc[2] != 0.0 || hsc[3] != 0.0) break;
        }
        upper_solve_kernel<<<1, 1, 0, st>>>(H, m + 1, kdone, k.s.as<double>(), k.y.as<double>());
        CTR_LAUNCHED();
        add_multi_prec_kernel<<<gb, 256, 0, st>>>(V, n, kdone, k.y.as<double>(), x, s->M, il1, il2);
        CTR_LAUNCHED();
        if (hsc[2] != 0.0 || hsc[3] != 0.0) {
            converged = true;
            break;
        }
        if (budget <= 0) break;
        // restart from the true residual
        CTR_TRY(apply_operator(s, x, v.u, precision));
        if (precision == CTR_FP32_REFINE) info->matvecs_fp32++; else info->matvecs_fp64++;
        axpby_kernel<<<gb, 256, 0, st>>>(1.0, b, -1.0, v.u, v.t, n);
        CTR_LAUNCHED();
        double rn = 0.0;
        CTR_TRY(device_dot(s, v.t, v.t, n, &rn));
        beta = std::sqrt(rn);
        if (beta <= tol_abs) {
            converged = true;
            break;
        }
        start = v.t;
    }
    return CTR_OK;
}

}  // namespace

int device_dot(ctr_ibim* s, const double* a, const double* b, int64_t n, double* h_out) {
    CTR_TRY(ensure_krylov(s));
    double* tmp = s->kr.scal.as<double>() + 4;
    CTR_TRY(dots(s, a, n, 1, b, n, tmp, 0));
    CTR_CUDA_TRY(cudaMemcpyAsync(h_out, tmp, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CTR_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return CTR_OK;
}

int solve_system(ctr_ibim* s, double* d_psi, double* d_dpsi, ctr_solve_info* info) {
    CTR_TRY(ensure_krylov(s));
    const int64_t M = s->M, n = 2 * M;
    cudaStream_t st = s->stream;
    Vecs v = vecs_of(s);
    const unsigned gb = grid_for(n, 256);
    const double* g = s->rhs.as<double>();
    double gnorm2 = 0.0;
    CTR_TRY(device_dot(s, g, g, n, &gnorm2));
    const double gnorm = std::sqrt(gnorm2);
    int64_t budget = s->opt.max_iter;
    bool conv = false;
    if (s->opt.precision != CTR_FP32_REFINE) {
        CTR_TRY(gmres(s, s->opt.precision, g, v.x, s->opt.tol, budget, info, conv));
        CTR_TRY(apply_operator(s, v.x, v.u, s->opt.precision));
        info->matvecs_fp64++;
        axpby_kernel<<<gb, 256, 0, st>>>(1.0, g, -1.0, v.u, v.r, n);
        CTR_LAUNCHED();
    } else {
        CTR_CUDA_TRY(cudaMemsetAsync(v.x, 0, sizeof(double) * n, st));
        CTR_CUDA_TRY(cudaMemcpyAsync(v.r, g, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        for (int it = 0;; ++it) {
            double rn2 = 0.0;
            CTR_TRY(device_dot(s, v.r, v.r, n, &rn2));
            if (!std::isfinite(rn2)) return fail(CTR_ERR_NUMERIC, "refinement: non-finite residual");
            if (std::sqrt(rn2) <= s->opt.tol * gnorm || it >= s->opt.max_refine || budget <= 0) break;
            bool inner = false;
            CTR_TRY(gmres(s, CTR_FP32_REFINE, v.r, v.d, s->opt.inner_tol, budget, info, inner));
            axpby_kernel<<<gb, 256, 0, st>>>(1.0, v.x, 1.0, v.d, v.x, n);
            CTR_LAUNCHED();
            CTR_TRY(apply_operator(s, v.x, v.u, s->opt.residual));
            info->matvecs_fp64++;
            info->refinements++;
            axpby_kernel<<<gb, 256, 0, st>>>(1.0, g, -1.0, v.u, v.r, n);
            CTR_LAUNCHED();
        }
    }
    double rn2 = 0.0;
    CTR_TRY(device_dot(s, v.r, v.r, n, &rn2));
    info->residual = (gnorm > 0) ? std::sqrt(rn2) / gnorm : 0.0;
    info->converged = (info->residual <= s->opt.tol) ? 1 : 0;
    if (!std::isfinite(info->residual)) return fail(CTR_ERR_NUMERIC, "solve: non-finite residual");
    CTR_CUDA_TRY(cudaMemcpyAsync(d_psi, v.x, sizeof(double) * M, cudaMemcpyDeviceToDevice, st));
    CTR_CUDA_TRY(cudaMemcpyAsync(d_dpsi, v.x + M, sizeof(double) * M, cudaMemcpyDeviceToDevice, st));
    CTR_TRY(check_device_error(s, "solve"));
    return info->converged ? CTR_OK : CTR_NOT_CONVERGED;
}

}  // namespace ctr
