// Reaction potential (Eq. 2.31) and polarization energy (Eq. 3.3).
//
// psi_rxn(z) = h^3 sum_j W_j [ ((eps_E/eps_I) dGk/dn_y - dG0/dn_y)(z, P_j) psi_j + (G0 - Gk)(z, P_j) dpsi_j ]
// by the plain trapezoidal rule on the tube (z is away from the surface).
// FP64; per-block partial sums over source chunks, added in a fixed order.
#include "common.cuh"

namespace ctr {

namespace {

constexpr int kThreads = 256;

__global__ void rxn_partial_kernel(NodeArrays na, int64_t M, const double* __restrict__ psi,
                                   const double* __restrict__ dpsi, const double* __restrict__ z, int64_t npts,
                                   double h3, double kappa, double ratio, int64_t chunk, double* __restrict__ part) {
    const int64_t p = blockIdx.x;
    const int b = blockIdx.y;
    const double zx = z[3 * p], zy = z[3 * p + 1], zz = z[3 * p + 2];
    const int64_t j0 = (int64_t)b * chunk, j1 = min(M, j0 + chunk);
    const double inv4pi = 1.0 / (4.0 * kPi);
    double acc = 0.0;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const double dx = zx - na.Px[j], dy = zy - na.Py[j], dz = zz - na.Pz[j];
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double rinv = rsqrt(r2);
        const double r = r2 * rinv;
        const double E = exp(-kappa * r);
        const double dny = dx * na.nx[j] + dy * na.ny[j] + dz * na.nz[j];
        const double s3 = rinv * rinv * rinv;
        const double dG0 = dny * s3;                       // 4 pi dG0/dn_y
        const double dGk = E * (1.0 + kappa * r) * dny * s3;
        const double K12 = (1.0 - E) * rinv;                // 4 pi (G0 - Gk)
        acc += h3 * na.W[j] * inv4pi * ((ratio * dGk - dG0) * psi[j] + K12 * dpsi[j]);
    }
    __shared__ double sh[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += sh[w];
        part[p * gridDim.y + b] = t;
    }
}

__global__ void rxn_final_kernel(const double* __restrict__ part, int nb, int64_t npts, double* __restrict__ out) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npts) return;
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += part[p * nb + b];
    out[p] = t;
}

}  // namespace

int reaction_potential(ctr_ibim* s, const double* d_psi, const double* d_dpsi, int64_t npts, const double* d_xyz,
                       double* d_out) {
    if (npts <= 0) return CTR_OK;
    int sms = 0;
    CTR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
    int nb = (int)std::max<int64_t>(1, std::min<int64_t>((s->M + 4095) / 4096,
                                                         std::max<int64_t>(1, 4 * sms / std::max<int64_t>(1, npts))));
    nb = std::min(nb, 65535);
    const int64_t chunk = (s->M + nb - 1) / nb;
    DevBuf part;
    CTR_TRY(part.alloc(sizeof(double) * (size_t)npts * nb));
    dim3 grid((unsigned)npts, (unsigned)nb);
    rxn_partial_kernel<<<grid, kThreads, 0, s->stream>>>(s->na, s->M, d_psi, d_dpsi, d_xyz, npts,
                                                        s->h * s->h * s->h, s->kappa, s->eps_out / s->eps_in, chunk,
                                                        part.as<double>());
    CTR_LAUNCHED();
    rxn_final_kernel<<<grid_for(npts, 128), 128, 0, s->stream>>>(part.as<double>(), nb, npts, d_out);
    CTR_LAUNCHED();
    CTR_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return CTR_OK;
}

}  // namespace ctr
