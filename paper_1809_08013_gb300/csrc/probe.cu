// probe.cu -- FMA throughput probe used for the roofline denominator of the
// FP64 pair kernels (not part of the SPH path). Each thread runs CH
// independent register-resident FMA chains; the result is folded into a
// file-scope sink so the work cannot be removed.
#include <math_constants.h>

#include "sph_internal.cuh"

namespace sph {

static __device__ double g_sink_d;
static __device__ float g_sink_f;

template <typename T, int CH>
__global__ void __launch_bounds__(256) k_fma_probe(T a, T b, int reps) {
    T x[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) x[k] = (T)(threadIdx.x & 7) * (T)0.001 + (T)k;
    for (int r = 0; r < reps; ++r) {
#pragma unroll
        for (int it = 0; it < 64; ++it) {
#pragma unroll
            for (int k = 0; k < CH; ++k) x[k] = fma(x[k], a, b);
        }
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < CH; ++k) s += x[k];
    if (s == (T)-1.2345) {
        if (sizeof(T) == 8) g_sink_d = (double)s;
        else g_sink_f = (float)s;
    }
}

}  // namespace sph

extern "C" sph_status sph_probe_fma_peak(int device, int fp64, void* stream, double* flops_per_s) {
    using namespace sph;
    if (!flops_per_s) return SPH_E_INVAL;
    *flops_per_s = 0.0;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return SPH_E_CUDA;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        cudaGetLastError();
        return SPH_E_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = prop.multiProcessorCount * 8, threads = 256, CH = 8;
    const int reps = fp64 ? 24 : 1024;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 0.0f;
    for (int trial = 0; trial < 3; ++trial) {
        cudaEventRecord(e0, s);
        if (fp64) k_fma_probe<double, CH><<<blocks, threads, 0, s>>>(0.9999999, 1e-7, reps);
        else k_fma_probe<float, CH><<<blocks, threads, 0, s>>>(0.9999f, 1e-4f, reps);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (trial > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (prev >= 0) cudaSetDevice(prev);
    if (cudaGetLastError() != cudaSuccess || best <= 0.0f) return SPH_E_CUDA;
    const double fmas = (double)blocks * threads * CH * 64.0 * reps;
    *flops_per_s = 2.0 * fmas / (best * 1e-3);
    return SPH_OK;
}
