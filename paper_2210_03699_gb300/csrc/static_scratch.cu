// FP32 dense pair sum whose scratch is a fixed device array: for callers that
// cannot allocate device memory (see ctr_pair_sum_fp32_static in ctr_ibim.h).
//
// The split partial sums live in g_scratch, a file-scope __device__ array
// that every GPU loading the library holds until the process exits.  Host
// code must not pass the symbol itself to a kernel (in host code it names a
// host-side stand-in); the device address comes from cudaGetSymbolAddress,
// taken once per device, with that device current, by the first call made
// on it.  All calls share the array, so calls that overlap on the GPU race.
#include <mutex>

#include "common.cuh"

namespace ctr {
int launch_fp32_pairs_external(const float4* src, int64_t M, const int32_t* eptr, const int32_t* excl,
                               double eps_ratio, double kappa, int64_t max_partial, double* partial, int* err,
                               cudaStream_t st, int* splits_out);
}

namespace {

constexpr int64_t kScratchDoubles = 2 * (int64_t)CTR_STATIC_SCRATCH_NODES;   // 16 MiB

__device__ __align__(256) double g_scratch[kScratchDoubles];
__device__ __align__(256) int g_wait_flag[64];

struct DevicePtrs {
    double* scratch = nullptr;
    int* flag = nullptr;
};

std::mutex g_lock;
DevicePtrs g_ptrs[64];

int device_ptrs(DevicePtrs* out) {
    int dev = 0;
    CTR_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return ctr::fail(CTR_ERR_INVALID, "device index out of range");
    std::lock_guard<std::mutex> guard(g_lock);
    DevicePtrs& p = g_ptrs[dev];
    if (!p.scratch) {
        void* s = nullptr;
        void* f = nullptr;
        CTR_CUDA_TRY(cudaGetSymbolAddress(&s, g_scratch));
        CTR_CUDA_TRY(cudaGetSymbolAddress(&f, g_wait_flag));
        p.scratch = static_cast<double*>(s);
        p.flag = static_cast<int*>(f);
    }
    *out = p;
    return CTR_OK;
}

// out[c*M + i] = sum over splits of partial[(s*2 + c)*M + i], in split order
__global__ void sum_splits_kernel(const double* __restrict__ partial, int S, int64_t M, double* __restrict__ out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * M) return;
    const int c = (int)(t / M);
    const int64_t i = t - (int64_t)c * M;
    double v = 0.0;
    for (int s = 0; s < S; ++s) v += partial[((size_t)s * 2 + c) * M + i];
    out[t] = v;
}

}  // namespace

extern "C" int ctr_pair_sum_fp32_static(int64_t M, const float* src, const int32_t* row_ptr,
                                        const int32_t* excluded, double eps_ratio, double kappa, double* out,
                                        void* stream) {
    using namespace ctr;
    if (M <= 0 || !src || !row_ptr || !excluded || !out) return fail(CTR_ERR_INVALID, "bad argument");
    if (M > CTR_STATIC_SCRATCH_NODES)
        return fail(CTR_ERR_CAPACITY, "more nodes than the fixed scratch holds (CTR_STATIC_SCRATCH_NODES)");
    if (!(eps_ratio > 0.0) || !(kappa >= 0.0)) return fail(CTR_ERR_INVALID, "eps_ratio must be > 0, kappa >= 0");
    if ((reinterpret_cast<uintptr_t>(src) & 15) != 0) return fail(CTR_ERR_INVALID, "src must be 16-byte aligned");
    DevicePtrs p;
    CTR_TRY(device_ptrs(&p));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CTR_CUDA_TRY(cudaMemsetAsync(p.flag, 0, sizeof(int), st));
    int splits = 0;
    CTR_TRY(launch_fp32_pairs_external(reinterpret_cast<const float4*>(src), M, row_ptr, excluded, eps_ratio, kappa,
                                       kScratchDoubles, p.scratch, p.flag, st, &splits));
    sum_splits_kernel<<<grid_for(2 * M, 256), 256, 0, st>>>(p.scratch, splits, M, out);
    CTR_LAUNCHED();
    int flag = 0;
    CTR_CUDA_TRY(cudaMemcpyAsync(&flag, p.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CTR_CUDA_TRY(cudaStreamSynchronize(st));
    if (flag) return fail(CTR_ERR_DEVICE_WAIT, "pair kernel: a bounded wait expired");
    return CTR_OK;
}
