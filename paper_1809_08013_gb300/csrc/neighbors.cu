// neighbors.cu -- Algorithm 1 step 2 ("find neighbours and smoothing length").
//
// Pair test. The definition is the FP64 test r_ij^2 < (2h)^2 with
// r^2 = (dx dx + dy dy) + dz dz, each operation rounded on its own (minimum
// image along z when periodic). GB300's FP64 pipe is narrow, so candidates are
// first classified in FP32 from float copies of the positions:
//   r2f < Tin   -> certainly inside,   r2f > Tout -> certainly outside,
//   otherwise   -> the exact FP64 test above decides.
// Tin/Tout are derived per particle from a rigorous bound on the FP32 error
// (see thresholds()), so every decision equals the FP64 one bit for bit and
// the neighbour sets are exact.
//
// h search (reading of the Section 2 footnote: h follows a target neighbour
// count): bracketing search using only correctly rounded * and +,
//   n < target - tol: lo = h; h = (hi == inf) ? 1.25 h : (lo + hi) / 2
//   n > target + tol: hi = h; h = (lo == 0)   ? 0.8 h  : (lo + hi) / 2
// for at most max_h_iter counts; the result is the last h counted.
//
// Symmetric set S_i = { j != i : r_ij < 2h_i or r_ij < 2h_j } as CSR: row i
// holds N_i (r_ij < 2h_i) first, then the rest.
#include <math_constants.h>

#include "sph_internal.cuh"

namespace sph {

struct Thr {
    float tin, tout;
    double r2;  // (2h)^2 in FP64, the exact threshold
};

// FP32 classification thresholds for radius R = 2h.
// |xf - x| <= 2^-24 X for each coordinate (X = max |coordinate|); the FP32
// difference, the periodic shift by lzf and the rounding of r2f add at most
// 2^-24 (2X + 2.02 R + 2 lz) per component and 3 * 2^-24 relative on the sum
// of squares, so the FP32 norm is within d = sqrt(3) e of the norm of the FP64
// difference vector, whose rounded square differs from it by < 2^-50 relative.
__device__ __forceinline__ Thr thresholds(double h, const Grid* __restrict__ g) {
    const double R = 2.0 * h;
    Thr t;
    t.r2 = __dmul_rn(R, R);
    const double u24 = 5.9604644775390625e-08;  // 2^-24
    const double per = g->periodic_z ? 2.0 * g->lz : 0.0;
    const double e = u24 * (4.0 * g->X + 2.02 * R + per) * 1.0001 + 1e-37;
    const double d = 1.7320508075688772 * e * 1.000001;
    const double a = R * (1.0 - 8.8817841970012523e-16) - d;
    const double b = R * (1.0 + 8.8817841970012523e-16) + d;
    t.tin = a > 0.0 ? __double2float_rd(a * a * (1.0 - 3.0 * u24) * (1.0 - 9.094947017729282e-13))
                    : -1.0f;
    t.tout = __double2float_ru(b * b * (1.0 + 3.0 * u24) * (1.0 + 9.094947017729282e-13));
    if (g->periodic_z && R > 0.25 * g->lz) {  // wrap decisions may differ: exact path only
        t.tin = -1.0f;
        t.tout = CUDART_INF_F;
    }
    return t;
}

__device__ __forceinline__ float f_r2(const float4& a, const float4& b, const Grid* __restrict__ g) {
    const float dx = a.x - b.x, dy = a.y - b.y;
    float dz = a.z - b.z;
    if (g->periodic_z) {
        if (dz > g->halflzf) dz -= g->lzf;
        else if (dz < -g->halflzf) dz += g->lzf;
    }
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

// The defining FP64 squared distance, operation by operation.
__device__ __forceinline__ double exact_r2(const double4_32a& a, const double4_32a& b,
                                           const Grid* __restrict__ g) {
    const double dx = __dsub_rn(a.x, b.x), dy = __dsub_rn(a.y, b.y);
    double dz = __dsub_rn(a.z, b.z);
    if (g->periodic_z) {
        const double half = __dmul_rn(0.5, g->lz);
        if (dz > half) dz = __dsub_rn(dz, g->lz);
        else if (dz < -half) dz = __dadd_rn(dz, g->lz);
    }
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__device__ __forceinline__ int wrapi(int k, int n) {
    int r = k % n;
    return r < 0 ? r + n : r;
}

// Cell index range overlapping [a, b] along axis d (clamped); along the
// periodic z axis the range may be unclamped (wrapped by the caller) or the
// whole axis (*all = true).
__device__ __forceinline__ void box_range(float a, float b, const Grid* __restrict__ g, int d,
                                          int& k0, int& k1, bool& all) {
    const float lo = g->lof[d], inv = g->invwf[d], s = g->slop[d];
    const int n = g->n[d];
    all = false;
    if (d == 2 && g->periodic_z) {
        const float fa = floorf((a - s + g->halflzf) * inv);
        const float fb = floorf((b + s + g->halflzf) * inv);
        if (!(fb - fa + 1.0f < (float)n)) {
            k0 = 0;
            k1 = n - 1;
            all = true;
            return;
        }
        k0 = (int)fa;
        k1 = (int)fb;
        return;
    }
    float fa = floorf((a - s - lo) * inv);
    float fb = floorf((b + s - lo) * inv);
    fa = fminf(fmaxf(fa, 0.0f), (float)n);
    fb = fmaxf(fminf(fb, (float)(n - 1)), -1.0f);
    k0 = (int)fa;
    k1 = (int)fb;
}

// Distance from v to the slab of cell k along axis d (0 inside), inflated by slop.
__device__ __forceinline__ float axis_gap(float v, int k, const Grid* __restrict__ g, int d) {
    const float a = g->lof[d] + (float)k * g->wf[d] - g->slop[d];
    const float b = g->lof[d] + (float)(k + 1) * g->wf[d] + g->slop[d];
    return fmaxf(0.0f, fmaxf(a - v, v - b));
}

__device__ __forceinline__ float wmin(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float wmax(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Warp-cooperative candidate walk. The 32 lanes of a warp query the union of
// their boxes [q - R, q + R] (inactive lanes contribute nothing); cells are
// visited in warp-uniform loops, each cell's particles are staged 32 at a
// time in shared memory, and every lane sees every staged candidate:
//   keep(cell, kx, ky, kz) -> bool  per-lane wish to visit a cell (any lane
//                                    wanting it makes the warp visit it)
//   visit(j, fj, tinj)               per lane, per staged candidate
// All 32 lanes must call this together.
template <class Keep, class Visit>
__device__ __forceinline__ void warp_walk(const Grid* __restrict__ g, const int2* __restrict__ cells,
                                          const float4* __restrict__ fpos,
                                          const float* __restrict__ tin, float4* s_f, float* s_t,
                                          const float4& q, float R, bool active, Keep&& keep,
                                          Visit&& visit) {
    const int lane = threadIdx.x & 31;
    const float lx = wmin(active ? q.x - R : CUDART_INF_F), hx = wmax(active ? q.x + R : -CUDART_INF_F);
    if (!(lx <= hx)) return;  // no active lane
    const float ly = wmin(active ? q.y - R : CUDART_INF_F), hy = wmax(active ? q.y + R : -CUDART_INF_F);
    const float lz = wmin(active ? q.z - R : CUDART_INF_F), hz = wmax(active ? q.z + R : -CUDART_INF_F);
    int x0, x1, y0, y1, z0, z1;
    bool ax, ay, az;
    box_range(lx, hx, g, 0, x0, x1, ax);
    box_range(ly, hy, g, 1, y0, y1, ay);
    box_range(lz, hz, g, 2, z0, z1, az);
    const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
    const bool per = g->periodic_z != 0;
    for (int kz = z0; kz <= z1; ++kz) {
        const int cz = per ? wrapi(kz, nz) : kz;
        for (int ky = y0; ky <= y1; ++ky) {
            const long long row = ((long long)cz * ny + ky) * nx;
            for (int kx = x0; kx <= x1; ++kx) {
                const int2 se = __ldg(&cells[row + kx]);
                if (se.y <= se.x) continue;
                if (!__any_sync(0xffffffffu, active && keep(row + kx, kx, ky, kz))) continue;
                for (int base = se.x; base < se.y; base += 32) {
                    const int j = base + lane;
                    if (j < se.y) {
                        s_f[lane] = __ldg(&fpos[j]);
                        if (tin) s_t[lane] = __ldg(&tin[j]);
                    }
                    __syncwarp();
                    const int cnt = min(32, se.y - base);
                    for (int k = 0; k < cnt; ++k) visit(base + k, s_f[k], tin ? s_t[k] : 0.0f);
                    __syncwarp();
                }
            }
        }
    }
}

// ------------------------------------------------------------ h search
// One warp per 32 consecutive particles. Each pass counts |N_i(h)| for every
// still-searching lane; the warp repeats passes until all lanes are done.
__global__ void __launch_bounds__(kThreads)
k_h_iterate(int64_t n, const Grid* __restrict__ g, KParams kp, double4_32a* posh,
            const float4* __restrict__ fpos, const int2* __restrict__ cells,
            int32_t* __restrict__ nnb, unsigned* __restrict__ status) {
    __shared__ float4 s_f[kThreads / 32][32];
    const int warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    double4_32a pi = make_double4_32a(0.0, 0.0, 0.0, 1.0);
    float4 fi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
        pi = posh[i];
        fi = fpos[i];
    }
    double h = pi.w, lo = 0.0, hi = CUDART_INF;
    const int lowb = kp.n_target - kp.n_tol, highb = kp.n_target + kp.n_tol;
    int cnt = 0, it = 0;
    bool active = valid && kp.max_h_iter > 0, conv = false;
    while (__any_sync(0xffffffffu, active)) {
        const Thr t = thresholds(h, g);
        const float R = (float)(2.0 * h) * 1.0001f;
        int c = 0;
        warp_walk(
            g, cells, fpos, nullptr, s_f[warp], nullptr, fi, R, active,
            [&](long long, int, int, int) { return true; },
            [&](int j, const float4& fj, float) {
                const float r2f = f_r2(fi, fj, g);
                if (r2f < t.tin) {
                    c += (j != i);
                } else if (r2f <= t.tout && j != i && active) {
                    c += exact_r2(pi, posh[j], g) < t.r2;
                }
            });
        if (active) {
            cnt = c;
            ++it;
            if (cnt >= lowb && cnt <= highb) {
                conv = true;
                active = false;
            } else if (it >= kp.max_h_iter) {
                active = false;
            } else if (cnt < lowb) {
                lo = h;
                h = isinf(hi) ? __dmul_rn(h, 1.25) : __dmul_rn(0.5, __dadd_rn(lo, hi));
            } else {
                hi = h;
                h = (lo == 0.0) ? __dmul_rn(h, 0.8) : __dmul_rn(0.5, __dadd_rn(lo, hi));
            }
        }
    }
    if (!valid) return;
    posh[i].w = h;
    nnb[i] = cnt;
    if (!conv) {
        atomicOr(&status[0], (unsigned)ST_HNOCONV);
        atomicAdd(&status[1], 1u);
    }
}

// Per-particle FP32 thresholds at the final h.
__global__ void __launch_bounds__(kThreads)
k_finalize_h(int64_t n, const Grid* __restrict__ g, const double4_32a* __restrict__ posh,
             float4* __restrict__ fpos, float* __restrict__ tin) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Thr t = thresholds(posh[i].w, g);
    fpos[i].w = t.tout;
    tin[i] = t.tin;
}

// Per-cell max h, and the global max (one atomic per block).
__global__ void __launch_bounds__(kThreads)
k_cell_hmax(const Grid* __restrict__ gc, Grid* gw, const int2* __restrict__ cells,
            const double4_32a* __restrict__ posh, unsigned long long* __restrict__ cell_hmax) {
    const long long nc = gc->ncells;
    double bmax = 0.0;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < nc;
         c += (long long)gridDim.x * blockDim.x) {
        const int2 se = cells[c];
        double m = 0.0;
        for (int k = se.x; k < se.y; ++k) m = fmax(m, posh[k].w);
        cell_hmax[c] = (unsigned long long)__double_as_longlong(m);
        bmax = fmax(bmax, m);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
    __shared__ double sh[kThreads / 32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = bmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = sh[0];
        for (int w = 1; w < kThreads / 32; ++w) m = fmax(m, sh[w]);
        atomicMax(&gw->hmax_bits, (unsigned long long)__double_as_longlong(m));
    }
}

// ------------------------------------------------------------ CSR
// FILL = false: rowlen[i] = |S_i|, ngather[i] = |N_i|.
// FILL = true : write row i at offsets[i] (N_i first); rows are skipped when
//               the total exceeds the capacity (status bit raised).
// One warp per 32 consecutive particles; a cell is visited when some lane
// can reach it: its box lies within 2 max(h_i, max h of the cell).
template <bool FILL>
__global__ void __launch_bounds__(kThreads)
k_csr(int64_t n, const Grid* __restrict__ g, const double4_32a* __restrict__ posh,
      const float4* __restrict__ fpos, const float* __restrict__ tin,
      const int2* __restrict__ cells, const unsigned long long* __restrict__ cell_hmax,
      int32_t* __restrict__ rowlen, int32_t* __restrict__ ngather,
      const int64_t* __restrict__ offsets, int32_t* __restrict__ idx, int64_t nnzcap,
      unsigned* __restrict__ status) {
    __shared__ float4 s_f[kThreads / 32][32];
    __shared__ float s_t[kThreads / 32][32];
    const int warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (FILL) {
        const int64_t tot = offsets[n];
        if (tot > nnzcap) {
            if (i == 0) atomicOr(&status[0], (unsigned)ST_CAPACITY);
            return;  // whole grid returns: no warp-collective call is left waiting
        }
    }
    const bool valid = i < n;
    double4_32a pi = make_double4_32a(0.0, 0.0, 0.0, 1.0);
    float4 fi = make_float4(0.f, 0.f, 0.f, 0.f);
    float tin_i = -1.0f;
    if (valid) {
        pi = posh[i];
        fi = fpos[i];
        tin_i = tin[i];
    }
    const double r2i = thresholds(pi.w, g).r2;
    const double hmaxg = __longlong_as_double((long long)g->hmax_bits);
    const float Rbig = (float)(2.0 * fmax(pi.w, hmaxg)) * 1.0001f;
    int64_t pg = 0, po = 0, pg_end = 0, po_end = 0;
    if (FILL && valid) {
        pg = offsets[i];
        pg_end = po = pg + ngather[i];
        po_end = offsets[i + 1];
    }
    int cg = 0, co = 0;
    const bool per = g->periodic_z != 0;
    warp_walk(
        g, cells, fpos, tin, s_f[warp], s_t[warp], fi, Rbig, valid,
        [&](long long cell, int kx, int ky, int kz) {
            const double hc = __longlong_as_double((long long)__ldg(&cell_hmax[cell]));
            const float reach = (float)(2.0 * fmax(pi.w, hc)) * 1.0001f;
            const float gx = axis_gap(fi.x, kx, g, 0), gy = axis_gap(fi.y, ky, g, 1);
            const float gz = per ? 0.0f : axis_gap(fi.z, kz, g, 2);
            return fmaf(gz, gz, fmaf(gy, gy, gx * gx)) < reach * reach;
        },
        [&](int j, const float4& fj, float tinj) {
            if (!valid || j == i) return;
            const float r2f = f_r2(fi, fj, g);
            bool in_i, have = false;
            double er2 = 0.0;
            if (r2f < tin_i) {
                in_i = true;
            } else if (r2f > fi.w) {
                in_i = false;
            } else {
                er2 = exact_r2(pi, posh[j], g);
                have = true;
                in_i = er2 < r2i;
            }
            if (in_i) {
                if (FILL && pg < pg_end) idx[pg++] = j;
                ++cg;
                return;
            }
            if (r2f > fj.w) return;
            bool in_j;
            if (r2f < tinj) {
                in_j = true;
            } else {
                const double4_32a pj = posh[j];
                if (!have) er2 = exact_r2(pi, pj, g);
                const double Rj = 2.0 * pj.w;
                in_j = er2 < __dmul_rn(Rj, Rj);
            }
            if (in_j) {
                if (FILL && po < po_end) idx[po++] = j;
                ++co;
            }
        });
    if (!FILL && valid) {
        rowlen[i] = cg + co;
        ngather[i] = cg;
    }
}

void launch_h_search(sph_ctx* c, const KParams& kp, cudaStream_t s) {
    const int64_t n = c->n;
    if (n == 0) return;
    const unsigned nb = (unsigned)((n + kThreads - 1) / kThreads);
    double4_32a* posh = c->posh[c->cur];
    c->launches += 3;
    k_h_iterate<<<nb, kThreads, 0, s>>>(n, c->grid, kp, posh, c->fpos, c->cells, c->nnb,
                                        c->status);
    k_finalize_h<<<nb, kThreads, 0, s>>>(n, c->grid, posh, c->fpos, c->tin);
    k_cell_hmax<<<kReduceBlocks, kThreads, 0, s>>>(c->grid, c->grid, c->cells, posh, c->cell_hmax);
}

void launch_csr(sph_ctx* c, cudaStream_t s) {
    const int64_t n = c->n;
    if (n == 0) {
        c->launches += 1;
        cudaMemsetAsync(c->offsets, 0, sizeof(int64_t), s);
        return;
    }
    const unsigned nb = (unsigned)((n + kThreads - 1) / kThreads);
    double4_32a* posh = c->posh[c->cur];
    c->launches += 5;
    k_csr<false><<<nb, kThreads, 0, s>>>(n, c->grid, posh, c->fpos, c->tin, c->cells,
                                         c->cell_hmax, c->rowlen, c->ngather, nullptr, nullptr,
                                         c->nnzcap, c->status);
    launch_scan_i32_i64(c->rowlen, n, c->offsets, c->row_part, s);
    k_csr<true><<<nb, kThreads, 0, s>>>(n, c->grid, posh, c->fpos, c->tin, c->cells,
                                        c->cell_hmax, c->rowlen, c->ngather, c->offsets, c->idx,
                                        c->nnzcap, c->status);
}

}  // namespace sph
