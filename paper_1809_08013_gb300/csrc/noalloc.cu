// noalloc.cu -- the time-step reduction for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: code embedded in a host that owns all
// device memory through its own pool (a serving runtime or a framework
// plugin with a fixed memory budget), or a latency-critical loop where an
// allocation may synchronise the device. sph_dt_noalloc computes the same
// time step as sph_forces, but from arrays the caller already holds, and
// keeps its block partial minima in a file-scope device array instead of a
// context buffer. The array (SPH_NOALLOC_MAX_N / 256 doubles, 64 KiB) is
// part of the library image: every GPU that loads the library holds it until
// the process exits.
#include "sph_internal.cuh"

namespace sph {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocMaxBlocks = (int)(SPH_NOALLOC_MAX_N / kNoAllocThreads);
static_assert((int64_t)kNoAllocMaxBlocks * kNoAllocThreads == SPH_NOALLOC_MAX_N,
              "SPH_NOALLOC_MAX_N must be a multiple of the block size");

// Shared by every call on a device: one partial minimum per block.
static __device__ __align__(256) double g_noalloc_dt_part[kNoAllocMaxBlocks];

// Candidate h_i / (c_i + 1.2 (alpha c_i + beta mumax_i)) per particle, block minimum.
__global__ void __launch_bounds__(kNoAllocThreads)
k_noalloc_dt_partial(int64_t n, double alpha, double beta, const double* __restrict__ h,
                     const double* __restrict__ c, const double* __restrict__ mumax,
                     double* __restrict__ part) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 1.0 / 0.0;
    if (i < n) {
        const double ci = c[i];
        const double mu = mumax ? mumax[i] : 0.0;
        v = h[i] / (ci + 1.2 * (alpha * ci + beta * mu));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    __shared__ double sh[kNoAllocThreads / 32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = sh[0];
        for (int w = 1; w < kNoAllocThreads / 32; ++w) m = fmin(m, sh[w]);
        part[blockIdx.x] = m;
    }
}

// dt = cfl * min over the first nb partials (nb = 0 gives +inf).
__global__ void __launch_bounds__(kNoAllocThreads)
k_noalloc_dt_finish(const double* __restrict__ part, int nb, double cfl, double* __restrict__ dt) {
    double m = 1.0 / 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) m = fmin(m, part[k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double sh[kNoAllocThreads / 32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = sh[0];
        for (int w = 1; w < kNoAllocThreads / 32; ++w) r = fmin(r, sh[w]);
        *dt = cfl * r;
    }
}

// Device address of g_noalloc_dt_part in the current context. In host code
// the array's name is only a host-side handle, never a device address. The
// address belongs to a CUDA context, not to a device number, so it is asked
// for on every call rather than cached: after a device reset, or with another
// context made current, a cached address could point at freed memory or into
// another context. The first lookup in a context may load the library's
// module there, which is why the first call should come before any capture.
static cudaError_t noalloc_scratch(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_dt_part);
    *out = (double*)p;
    return e;
}

}  // namespace sph

extern "C" sph_status sph_dt_noalloc(const sph_params* prm, int64_t n, const double* h,
                                     const double* c, const double* mumax, double* dt,
                                     void* stream) {
    using namespace sph;
    if (!prm || !dt || n < 0 || !(prm->cfl > 0.0)) return SPH_E_INVAL;
    if (n > SPH_NOALLOC_MAX_N) return SPH_E_INVAL;  // beyond the static scratch
    if (n > 0 && (!h || !c)) return SPH_E_INVAL;
    // An error left pending by the caller's earlier work is reported, not
    // cleared, so the caller's own check still sees it.
    if (cudaPeekAtLastError() != cudaSuccess) return SPH_E_CUDA;
    double* part = nullptr;
    if (noalloc_scratch(&part) != cudaSuccess) {
        cudaGetLastError();  // this call's own failure
        return SPH_E_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)((n + kNoAllocThreads - 1) / kNoAllocThreads);
    if (nb > 0) {
        k_noalloc_dt_partial<<<nb, kNoAllocThreads, 0, s>>>(n, prm->alpha, prm->beta, h, c, mumax,
                                                            part);
        if (cudaGetLastError() != cudaSuccess) return SPH_E_CUDA;
    }
    k_noalloc_dt_finish<<<1, kNoAllocThreads, 0, s>>>(part, nb, prm->cfl, dt);
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_E_CUDA;
}
