// Krylov workspace of a handle and FP64 dot products (the solver itself is the
// multi-slot engine, engine.cu).
//
// GMRES on the device (Sec. 2.5: "standard GMRES"): Arnoldi uses classical
// Gram-Schmidt applied twice (CGS2: as stable as modified Gram-Schmidt, but
// two batched passes instead of j+1 dependent ones); the Hessenberg columns,
// Givens rotations, the least-squares right side and the triangular solve are
// FP64 device scalars updated by one thread.  All reductions sum per-block
// partials in a fixed order, so a solve is bitwise reproducible run to run.
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

}  // namespace

int ensure_krylov_public(ctr_ibim* s) { return ensure_krylov(s); }

int device_dot(ctr_ibim* s, const double* a, const double* b, int64_t n, double* h_out) {
    CTR_TRY(ensure_krylov(s));
    double* tmp = s->kr.scal.as<double>() + 4;
    CTR_TRY(dots(s, a, n, 1, b, n, tmp, 0));
    CTR_CUDA_TRY(cudaMemcpyAsync(h_out, tmp, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CTR_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return CTR_OK;
}

}  // namespace ctr
