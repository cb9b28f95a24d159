// scan.cu -- device-wide exclusive prefix sums (reduce, scan partials, apply).
// Used for the radix-sort digit offsets and for the neighbour-list row offsets.
#include "sph_internal.cuh"

namespace sph {

int64_t scan_parts(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

// Exclusive scan of one value per thread over a 256-thread block; *total gets
// the block sum.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* total) {
    __shared__ T warp_tot[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < kThreads / 32 ? warp_tot[lane] : T(0);
        T wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < kThreads / 32) warp_tot[lane] = wi - w;  // exclusive warp offsets
        if (lane == kThreads / 32 - 1) *total = wi;
    }
    __syncthreads();
    T r = warp_tot[warp] + inc - v;
    __syncthreads();
    return r;
}

// gate / mask: when gate is given, the kernels do nothing unless *gate & mask
// (a device flag decides whether the scan is needed; the launches stay fixed).
__device__ __forceinline__ bool gated_off(const unsigned* gate, unsigned mask) {
    return gate && !(*(volatile const unsigned*)gate & mask);
}

template <typename In, typename Acc>
__global__ void __launch_bounds__(kThreads) k_scan_reduce(const In* __restrict__ in, int64_t n,
                                                          Acc* __restrict__ part,
                                                          const unsigned* gate, unsigned mask) {
    if (gated_off(gate, mask)) return;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * 8;
    Acc s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if (base + k < n) s += (Acc)in[base + k];
    __shared__ Acc tot;
    block_excl_scan<Acc>(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Single block, exclusive scan in place over np partials.
template <typename Acc>
__global__ void __launch_bounds__(kThreads) k_scan_partials(Acc* part, int64_t np,
                                                            const unsigned* gate, unsigned mask) {
    if (gated_off(gate, mask)) return;
    const int64_t per = (np + kThreads - 1) / kThreads;
    const int64_t b = (int64_t)threadIdx.x * per;
    Acc s = 0;
    for (int64_t k = 0; k < per; ++k)
        if (b + k < np) s += part[b + k];
    __shared__ Acc tot;
    Acc off = block_excl_scan<Acc>(s, &tot);
    for (int64_t k = 0; k < per; ++k)
        if (b + k < np) {
            Acc v = part[b + k];
            part[b + k] = off;
            off += v;
        }
}

template <typename In, typename Out>
__global__ void __launch_bounds__(kThreads) k_scan_apply(const In* in, int64_t n,
                                                         const Out* __restrict__ part, Out* out,
                                                         int write_total, const unsigned* gate,
                                                         unsigned mask) {
    if (gated_off(gate, mask)) return;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * 8;
    Out v[8];
    Out s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        v[k] = (base + k < n) ? (Out)in[base + k] : Out(0);
        s += v[k];
    }
    __shared__ Out tot;
    Out run = block_excl_scan<Out>(s, &tot) + part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (base + k < n) {
            out[base + k] = run;
            run += v[k];
            if (write_total && base + k == n - 1) out[n] = run;
        }
    }
}

void launch_scan_i32_i64(const int32_t* in, int64_t n, int64_t* out, int64_t* part,
                         cudaStream_t s, const unsigned* gate, unsigned mask) {
    if (n <= 0) {
        cudaMemsetAsync(out, 0, sizeof(int64_t), s);
        return;
    }
    const int64_t np = scan_parts(n);
    k_scan_reduce<int32_t, int64_t><<<(unsigned)np, kThreads, 0, s>>>(in, n, part, gate, mask);
    k_scan_partials<int64_t><<<1, kThreads, 0, s>>>(part, np, gate, mask);
    k_scan_apply<int32_t, int64_t><<<(unsigned)np, kThreads, 0, s>>>(in, n, part, out, 1, gate,
                                                                      mask);
}

void launch_scan_u32(uint32_t* data, int64_t n, uint32_t* part, cudaStream_t s) {
    if (n <= 0) return;
    const int64_t np = scan_parts(n);
    k_scan_reduce<uint32_t, uint32_t><<<(unsigned)np, kThreads, 0, s>>>(data, n, part, nullptr, 0u);
    k_scan_partials<uint32_t><<<1, kThreads, 0, s>>>(part, np, nullptr, 0u);
    k_scan_apply<uint32_t, uint32_t><<<(unsigned)np, kThreads, 0, s>>>(data, n, part, data, 0,
                                                                        nullptr, 0u);
}

}  // namespace sph
