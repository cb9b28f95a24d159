// sort.cu -- Algorithm 1 step 1 (the tree build), done as Morton-sorted cell
// lists: bounding box and cell grid on the device, 24-bit Morton key of each
// particle's cell, a stable LSD radix sort (3 passes of 8 bits, one more for
// the instance id of a batch), the permutation of the particle state into
// sorted order, and the [start, end) range of every occupied cell.
//
// The keys are sorted in caller order (each particle at its "rank" roff[k] +
// its index within its instance), not in the order the previous step left,
// so particles of one cell always end up ordered by caller index: the
// internal order -- and with it every summation order -- depends only on the
// positions, and a run split into several calls gives the same bits as one.
#include <math_constants.h>

#include "df.cuh"
#include "sph_internal.cuh"

namespace sph {

// ------------------------------------------------------------------ state I/O
// Caller arrays (instances back to back) into the slot layout: instance k's
// particle r goes to slot ioff[k] + r; empty slots get an inert state and
// order = -1.
__global__ void __launch_bounds__(kThreads)
k_load_state(int64_t n, Batch B, const int64_t* __restrict__ coff, const double* __restrict__ x,
             const double* __restrict__ y, const double* __restrict__ z,
             const double* __restrict__ h, const double* __restrict__ vx,
             const double* __restrict__ vy, const double* __restrict__ vz,
             const double* __restrict__ m, const double* __restrict__ u,
             double4_32a* __restrict__ posh, double4_32a* __restrict__ velm,
             double* __restrict__ ue, int32_t* __restrict__ order, double4_32a* __restrict__ posh2,
             double4_32a* __restrict__ velm2, double* __restrict__ ue2, int32_t* __restrict__ order2) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int inst = slot_inst(B, k);
    const int64_t r = k - __ldg(&B.ioff[inst]);
    if (r >= __ldg(&B.icnt[inst])) {  // empty slot, inert in both buffers (never permuted)
        posh[k] = posh2[k] = make_double4_32a(0.0, 0.0, 0.0, 1.0);
        velm[k] = velm2[k] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        ue[k] = ue2[k] = 0.0;
        order[k] = order2[k] = -1;
        return;
    }
    const int64_t c = __ldg(&coff[inst]) + r;
    posh[k] = make_double4_32a(x[c], y[c], z[c], h[c]);
    velm[k] = make_double4_32a(vx ? vx[c] : 0.0, vy ? vy[c] : 0.0, vz ? vz[c] : 0.0, m ? m[c] : 0.0);
    ue[k] = u ? u[c] : 0.0;
    order[k] = (int32_t)c;
}

void launch_load_state(sph_ctx* c, const sph_particles* P, cudaStream_t s) {
    const int64_t n = c->n;
    if (n == 0) return;
    const int b = c->cur;
    c->launches += 1;
    k_load_state<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        n, batch_of(c), c->coff, P->x, P->y, P->z, P->h, P->vx, P->vy, P->vz, P->m, P->u,
        c->posh[b], c->velm[b], c->ue[b], c->order[b], c->posh[1 - b], c->velm[1 - b],
        c->ue[1 - b], c->order[1 - b]);
}

// Pack of the double-float pair kernels for particle k: the fixed-point chunks
// of its position (dfl::to_fx, exponents of its instance) and its mass, both
// in the pair kernels' units of the instance,
//   xpk[3k] = (x.c2, y.c2, z.c2, m.hi), xpk[3k+1] = (x.c1, y.c1, z.c1, m.lo),
//   xpk[3k+2] = (x.c0, y.c0, z.c0, 0).
__device__ __forceinline__ void write_xpk(float4* __restrict__ xpk, int64_t k, const double4_32a& p,
                                          double mass, const Grid& g) {
    const int f = g.fxk + g.uL;
    const dfl::fx3 X = dfl::to_fx(p.x, g.fxk, f), Y = dfl::to_fx(p.y, g.fxk, f);
    const dfl::fx3 Z = dfl::to_fx(p.z, g.fxk, f);
    const dfl::df m = dfl::from_double_fp64(mass * p2d(-g.uM));
    xpk[3 * k + 0] = make_float4(X.c2, Y.c2, Z.c2, m.hi);
    xpk[3 * k + 1] = make_float4(X.c1, Y.c1, Z.c1, m.lo);
    xpk[3 * k + 2] = make_float4(X.c0, Y.c0, Z.c0, 0.0f);
}

// Velocity of particle k as float pairs in the velocity unit 2^uV of its
// instance (the double-float force kernels' view of it).
__device__ __forceinline__ void write_vpk(float4* __restrict__ vpa, float2* __restrict__ vpb,
                                          int64_t k, const double4_32a& v, const Grid& g) {
    const double sv = p2d(-g.uV);
    const dfl::df x = dfl::from_double_fp64(v.x * sv), y = dfl::from_double_fp64(v.y * sv);
    const dfl::df z = dfl::from_double_fp64(v.z * sv);
    vpa[k] = make_float4(x.hi, x.lo, y.hi, y.lo);
    vpb[k] = make_float2(z.hi, z.lo);
}

// Re-read the caller's arrays into the sorted order of the last build and
// derive the per-particle quantities the pair kernels load for j.
__global__ void __launch_bounds__(kThreads)
k_gather_state(int64_t n, int what, int precision, double alpha, const int32_t* __restrict__ order,
               const double* __restrict__ x, const double* __restrict__ y,
               const double* __restrict__ z, const double* __restrict__ h,
               const double* __restrict__ vx, const double* __restrict__ vy,
               const double* __restrict__ vz, const double* __restrict__ m,
               const double* __restrict__ rho, const double* __restrict__ p,
               const double* __restrict__ cs, double4_32a* __restrict__ posh,
               double4_32a* __restrict__ velm, double4_32a* __restrict__ therm,
               double2* __restrict__ kern, double* __restrict__ cint, float4* __restrict__ dpk,
               float4* __restrict__ xpk, float4* __restrict__ vpa, float2* __restrict__ vpb,
               const Grid* __restrict__ grid, unsigned* status) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t o = order[k];
    if (o < 0) return;  // empty slot
    const double hh = h[o];
    const double4_32a ps = make_double4_32a(x[o], y[o], z[o], hh);
    posh[k] = ps;
    const double mm = m[o];
    const Grid& g = grid[0];  // a single problem: instance 0
    write_xpk(xpk, k, ps, mm, g);
    if (what == GATHER_DENSITY) {
        velm[k] = make_double4_32a(0.0, 0.0, 0.0, mm);
    } else {
        const double4_32a vv = make_double4_32a(vx[o], vy[o], vz[o], mm);
        velm[k] = vv;
        if (precision == PREC_FP64) write_vpk(vpa, vpb, k, vv, g);
        const double r = rho[o], c = cs[o];
        const double hinv = 1.0 / hh;
        const double h2 = hinv * hinv;
        const double A = p[o] / (r * r);
        therm[k] = make_double4_32a(0.5 * r, A, 0.5 * alpha * c, 0.5 * hh);
        kern[k] = make_double2(hinv, h2 * h2);
        if (precision == PREC_FP64)  // the double-float kernels' pack
            dfl::write_pack(dpk, k, hinv, A, hh, r, alpha, c, dfl::pair_units(g.uL, g.uM, g.uV),
                            status, ST_RANGE);
        cint[k] = c;
    }
}

void launch_gather_state(sph_ctx* c, const sph_particles* P, const KParams& kp, int what,
                         cudaStream_t s) {
    const int64_t n = c->n;
    if (n == 0) return;
    const int b = c->cur;
    c->launches += 1;
    k_gather_state<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        n, what, kp.precision, kp.alpha, c->order[b], P->x, P->y, P->z, P->h, P->vx, P->vy, P->vz, P->m,
        P->rho, P->p, P->c, c->posh[b], c->velm[b], c->therm, c->kern, c->cint, c->dpk, c->xpk,
        c->vpa, c->vpb, c->grid, c->status);
}

// ------------------------------------------------------------ bbox and grid
// Min / max of doubles as signed 64-bit integer min / max of order-preserving
// keys (GB300's FP64 pipe is narrow; integer compares are not on it).
__device__ __forceinline__ long long okey(double x) {
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double okey_inv(long long k) {
    return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffLL));
}

constexpr long long kKeyMax = 0x7fffffffffffffffLL, kKeyMin = -kKeyMax - 1;

// Bounding-box partials: min x, y, z and max x, y, z, h, m, |v| (largest
// component), u (as keys) and the sum of h over the particles of each group
// of kSlotAlign slots (one instance), one block of kSlotAlign / kBoxWarpSlots
// warps per group, reduced in a fixed
// order; with candidate lists also the largest displacement since the last
// list build, the smallest list slack (list radius - 2h), and the largest and
// smallest build stamp. Stored as kBoxStride doubles per group: mn[3],
// mx[11], hs.
constexpr int kBoxMax = 11;
enum { BX_D = 7, BX_NSLACK = 8, BX_STAMP = 9, BX_NSTAMP = 10 };

struct BoxPart {
    long long mn[3], mx[kBoxMax];
    double hs;
};

__device__ __forceinline__ void box_init(BoxPart& b) {
    for (int d = 0; d < 3; ++d) b.mn[d] = kKeyMax;
    for (int d = 0; d < kBoxMax; ++d) b.mx[d] = kKeyMin;
    b.hs = 0.0;
}

// Fixed-order warp reduction of the first NMAX maxima (the others untouched).
template <int NMAX = kBoxMax>
__device__ __forceinline__ void box_warp_reduce(BoxPart& b) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const long long v = __shfl_xor_sync(0xffffffffu, b.mn[d], o);
            b.mn[d] = v < b.mn[d] ? v : b.mn[d];
        }
#pragma unroll
        for (int d = 0; d < NMAX; ++d) {
            const long long v = __shfl_xor_sync(0xffffffffu, b.mx[d], o);
            b.mx[d] = v > b.mx[d] ? v : b.mx[d];
        }
        b.hs += __shfl_xor_sync(0xffffffffu, b.hs, o);
    }
}

static_assert(kSlotAlign % kBoxWarpSlots == 0 && kBoxWarpSlots % 32 == 0, "bbox groups");
constexpr int kBoxThreads = kSlotAlign / kBoxWarpSlots * 32;  // one block per group

// LISTS: some instance keeps candidate lists (their statistics are gathered).
template <bool LISTS>
__global__ void __launch_bounds__(kBoxThreads)
k_bbox(int64_t n, Batch B, const double4_32a* __restrict__ posh,
       const double4_32a* __restrict__ velm, const double* __restrict__ ue,
       const int32_t* __restrict__ order, const LMeta* __restrict__ lmeta,
       double* __restrict__ part, unsigned* __restrict__ status) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t grp = blockIdx.x;  // group of kSlotAlign slots (< n: one block per group)
    const int64_t w0 = grp * kSlotAlign + (int64_t)warp * kBoxWarpSlots;
    const int inst = slot_inst(B, grp * kSlotAlign);
    const int64_t end = __ldg(&B.ioff[inst]) + __ldg(&B.icnt[inst]);
    const KParams& kp = B.kp[inst];
    const bool lists = LISTS && kp.list_skin > 0.0;
    const bool per = kp.periodic_z != 0;
    const float lzf = (float)kp.lz, hlzf = 0.5f * lzf;
    BoxPart b;
    box_init(b);
    bool bad = false;
#pragma unroll
    for (int q = 0; q < kBoxWarpSlots / 32; ++q) {
        const int64_t k = w0 + q * 32 + lane;
        if (k < end) {
            // a particle outside the geometry range (NaN, infinity, beyond the
            // FP32 range) is reported and kept out of the box and the means:
            // the cells, the search and the units stay those of the others
            const double4_32a p = posh[k];
            const double4_32a v = velm[k];
            const double uk = ue[k];
            const bool geo = coord_ok(p.x) && coord_ok(p.y) && coord_ok(p.z) && h_ok(p.w);
            const bool fin = finite_bits(v.x) && finite_bits(v.y) && finite_bits(v.z) &&
                             finite_bits(v.w) && finite_bits(uk);
            if (lists && geo) {
                // since the last list build: the displacement (truncated floats,
                // the minimum image along a periodic z), the list's slack at the
                // current h, the build stamp
                const int32_t id = order[k];
                const float4 m0 = __ldg(reinterpret_cast<const float4*>(lmeta) + 2 * id);
                const int4 m1 = __ldg(reinterpret_cast<const int4*>(lmeta) + 2 * id + 1);
                const float dx = dfl::from_double(p.x).hi - m0.x;
                const float dy = dfl::from_double(p.y).hi - m0.y;
                float dz = dfl::from_double(p.z).hi - m0.z;
                if (per) {
                    if (dz > hlzf) dz -= lzf;
                    else if (dz < -hlzf) dz += lzf;
                }
                const long long kd = __float_as_int(sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx))));
                b.mx[BX_D] = kd > b.mx[BX_D] ? kd : b.mx[BX_D];  // NaN keys above +inf
                if (m1.z > 0) {
                    const long long ks = fkey(reach_f32(p.w) - m0.w);
                    b.mx[BX_NSLACK] = ks > b.mx[BX_NSLACK] ? ks : b.mx[BX_NSLACK];
                }
                b.mx[BX_STAMP] = m1.x > b.mx[BX_STAMP] ? m1.x : b.mx[BX_STAMP];
                b.mx[BX_NSTAMP] = -(long long)m1.x > b.mx[BX_NSTAMP] ? -(long long)m1.x : b.mx[BX_NSTAMP];
            }
            bad |= !(geo && fin);
            if (!(geo && fin)) continue;
            const long long kx = okey(p.x), ky = okey(p.y), kz = okey(p.z), kh = okey(p.w);
            b.mn[0] = kx < b.mn[0] ? kx : b.mn[0];
            b.mn[1] = ky < b.mn[1] ? ky : b.mn[1];
            b.mn[2] = kz < b.mn[2] ? kz : b.mn[2];
            b.mx[0] = kx > b.mx[0] ? kx : b.mx[0];
            b.mx[1] = ky > b.mx[1] ? ky : b.mx[1];
            b.mx[2] = kz > b.mx[2] ? kz : b.mx[2];
            b.mx[3] = kh > b.mx[3] ? kh : b.mx[3];
            b.hs += p.w;
            const long long km = okey(v.w), ku = okey(uk);
            const long long kv = okey(fmax(fabs(v.x), fmax(fabs(v.y), fabs(v.z))));
            b.mx[4] = km > b.mx[4] ? km : b.mx[4];
            b.mx[5] = kv > b.mx[5] ? kv : b.mx[5];
            b.mx[6] = ku > b.mx[6] ? ku : b.mx[6];
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, (unsigned)ST_NONFINITE);
    // without lists the list fields are neither reduced nor written (nothing reads them)
    constexpr int NMAX = LISTS ? kBoxMax : BX_D;
    box_warp_reduce<NMAX>(b);
    __shared__ BoxPart wb[kBoxThreads / 32];
    if (lane == 0) wb[warp] = b;
    __syncthreads();
    if (threadIdx.x == 0) {  // the block's warps in order: a fixed summation order
        BoxPart a = wb[0];
        for (int w = 1; w < kBoxThreads / 32; ++w) {
            for (int d = 0; d < 3; ++d) a.mn[d] = wb[w].mn[d] < a.mn[d] ? wb[w].mn[d] : a.mn[d];
            for (int d = 0; d < NMAX; ++d) a.mx[d] = wb[w].mx[d] > a.mx[d] ? wb[w].mx[d] : a.mx[d];
            a.hs += wb[w].hs;
        }
        double* o = part + grp * kBoxStride;
        for (int d = 0; d < 3; ++d) o[d] = __longlong_as_double(a.mn[d]);
        for (int d = 0; d < NMAX; ++d) o[3 + d] = __longlong_as_double(a.mx[d]);
        o[3 + kBoxMax] = a.hs;
    }
}

__device__ __forceinline__ int grid_count(double ext, double w, double* wout) {
    double c = floor(ext / w) + 1.0;
    if (c > (double)kMaxCellsPerAxis) c = (double)kMaxCellsPerAxis;
    if (!(c >= 1.0)) c = 1.0;  // also a NaN extent: never an empty axis
    double ww = w;
    if (c * ww <= ext) ww = ext / (c - 0.5);
    *wout = ww;
    return (int)c;
}

// One block per instance: reduce the instance's bbox partials (fixed order:
// thread t takes partials t, t + 1024, ..., then a fixed tree) and derive its
// cell grid. The cell width is 2 <h> cell_scale (<h> the mean smoothing
// length), widened while the grid would exceed the instance's cell budget;
// the neighbour sets do not depend on it, only the candidates visited do.
constexpr int kGridThreads = 1024;

__global__ void __launch_bounds__(kGridThreads)
k_grid_setup(const double* __restrict__ part, Batch B, Grid* __restrict__ grid,
             unsigned* __restrict__ status, unsigned long long* __restrict__ wctr,
             unsigned* __restrict__ lctr) {
    const int inst = blockIdx.x;
    const int64_t n = B.icnt[inst];
    const int64_t b0 = B.ioff[inst] / kSlotAlign;
    const int64_t nbk = (n + kSlotAlign - 1) / kSlotAlign;
    // field f = t % 16 of every 64th partial from partial t / 16 on: each
    // load instruction of a warp reads two whole partials. Fields 0-2 are
    // minima, 3 .. 3 + kBoxMax - 1 maxima, 3 + kBoxMax the sum of h.
    static_assert(kBoxStride == 16 && 3 + kBoxMax < kBoxStride, "bbox partial layout");
    const int f = threadIdx.x & 15;
    const bool fmin_ = f < 3, fsum = f == 3 + kBoxMax;
    long long acc = fmin_ ? kKeyMax : kKeyMin;
    double hsum = 0.0;
    const double* base = part + b0 * kBoxStride + f;
    for (int64_t b = threadIdx.x >> 4; b < nbk; b += kGridThreads / 16) {
        const double v = base[b * kBoxStride];
        const long long k = __double_as_longlong(v);
        if (fmin_) acc = k < acc ? k : acc;
        else acc = k > acc ? k : acc;
        if (fsum) hsum += v;
    }
    // lanes l and l + 16 hold the same field: combine, lower lane first (a
    // fixed order), then the warps in order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    {
        const long long ok = __shfl_xor_sync(0xffffffffu, acc, 16);
        const double oh = __shfl_xor_sync(0xffffffffu, hsum, 16);
        acc = fmin_ ? (ok < acc ? ok : acc) : (ok > acc ? ok : acc);
        hsum = lane < 16 ? hsum + oh : oh + hsum;
    }
    __shared__ long long wk[kGridThreads / 32][16];
    __shared__ double wh[kGridThreads / 32];
    if (lane < 16) wk[warp][lane] = acc;
    if (lane == 3 + kBoxMax) wh[warp] = hsum;
    __syncthreads();
    __shared__ double r[11];
    __shared__ long long lk[4];  // list keys: displacement, -slack, stamp, -stamp
    if (threadIdx.x == 0) {
        BoxPart a;
        box_init(a);
        for (int w = 0; w < kGridThreads / 32; ++w) {
            for (int d = 0; d < 3; ++d) a.mn[d] = wk[w][d] < a.mn[d] ? wk[w][d] : a.mn[d];
            for (int d = 0; d < kBoxMax; ++d) a.mx[d] = wk[w][3 + d] > a.mx[d] ? wk[w][3 + d] : a.mx[d];
            a.hs += wh[w];
        }
        // the layout the grid derivation below reads: min x, y, z, -max x, y, z, -max h, sum h
        for (int d = 0; d < 3; ++d) {
            r[d] = okey_inv(a.mn[d]);
            r[3 + d] = -okey_inv(a.mx[d]);
        }
        r[6] = -okey_inv(a.mx[3]);
        r[7] = a.hs;
        r[8] = okey_inv(a.mx[4]);   // max m
        r[9] = okey_inv(a.mx[5]);   // max |v| component
        r[10] = okey_inv(a.mx[6]);  // max u
        for (int q = 0; q < 4; ++q) lk[q] = a.mx[BX_D + q];
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const KParams kp = B.kp[inst];
    Grid* g = grid + inst;
    const long long cellcap = g->cap;
    double mn[3] = {r[0], r[1], r[2]};
    double mx[3] = {-r[3], -r[4], -r[5]};
    for (int d = 0; d < 3; ++d)  // no particle, or none inside the geometry range
        if (n == 0 || !(mn[d] <= mx[d])) { mn[d] = 0.0; mx[d] = 0.0; }
    if (inst == 0) {
        status[2] = 0u;
        status[3] = 0u;
        wctr[0] = 0ull;
    }
    const double hmean = n > 0 ? r[7] / (double)n : 1.0;
    double w = 2.0 * hmean * kp.cell_scale;
    if (!(w > 0.0) || !isfinite(w)) w = 1.0;
    const bool per = kp.periodic_z != 0;
    double X = 0.0;
    for (int d = 0; d < 3; ++d) X = fmax(X, fmax(fabs(mn[d]), fabs(mx[d])));
    if (per) X = fmax(X, 0.5 * kp.lz);
    // Candidate lists of the h search. The instance keeps its lists while
    // every particle carries the same build stamp and twice the largest
    // displacement since that build (bounded with the truncation errors of
    // both positions) is below every list's slack at the current h: then any
    // j within 2 h of i now was within the list radius at the build, and is
    // listed. Otherwise this step rebuilds them under a new stamp. While they
    // are kept, so are the build's cell geometry and (through the sort keys)
    // its cells, whose walks then reach further by the displacement bound.
    bool keep = false;
    float dm2 = CUDART_INF_F;
    if (kp.list_skin > 0.0 && n > 0) {
        const long long smax = lk[2], smin = -lk[3];
        const bool epoch = smax == smin && smin > 0;
        const float D = lk[0] == kKeyMin ? 0.0f : __int_as_float((int)lk[0]);
        const double Dm = (double)D * (1.0 + 0x1p-20) + 0x1p-20 * (X + (double)D);
        dm2 = (float)(2.0 * Dm * (1.0 + 0x1p-20));
        const float slack = lk[1] == kKeyMin ? CUDART_INF_F : -fkey_inv(lk[1]);
        keep = epoch && g->gvalid && dm2 < slack;  // false for a NaN displacement
        g->lstamp = keep ? (int)smin : (int)((atomicAdd(lctr, 1u) & 0x3fffffffu) + 1u);
    } else {
        g->lstamp = 0;
    }
    g->lbuild = kp.list_skin > 0.0 && n > 0 && !keep ? 1 : 0;
    g->dm2 = dm2;
    int cnt[3];
    double ww[3], lo[3];
    for (int tries = 0; tries < 200 && !keep; ++tries) {
        for (int d = 0; d < 3; ++d) {
            lo[d] = mn[d];
            cnt[d] = grid_count(mx[d] - mn[d], w, &ww[d]);
        }
        if (per) {
            double c = floor(kp.lz / w);
            if (c < 1.0) c = 1.0;
            if (c > (double)kMaxCellsPerAxis) c = (double)kMaxCellsPerAxis;
            cnt[2] = (int)c;
            lo[2] = -0.5 * kp.lz;
            ww[2] = kp.lz / c;
        }
        if ((long long)cnt[0] * cnt[1] * cnt[2] <= cellcap) break;
        w *= 1.25;
    }
    if (!keep) {
        for (int d = 0; d < 3; ++d) {
            g->lo[d] = lo[d];
            g->w[d] = ww[d];
            g->inv_w[d] = 1.0 / ww[d];
            g->n[d] = cnt[d];
            g->lof[d] = (float)lo[d];
            g->wf[d] = (float)ww[d];
            g->invwf[d] = (float)(1.0 / ww[d]);
        }
        g->ncells = (long long)cnt[0] * cnt[1] * cnt[2];
        g->gvalid = 1;
    }
    for (int d = 0; d < 3; ++d)
        g->slop[d] = (float)(1e-3 * g->w[d] + 1.2e-7 * X + (keep ? 0.5 * 1.001 * dm2 : 0.0));
    g->periodic_z = per ? 1 : 0;
    g->lz = kp.lz;
    g->lzf = (float)kp.lz;
    g->halflzf = (float)(0.5 * kp.lz);
    g->X = X;
    // |fl32 difference - FP64 difference| <= 2^-24 (4X + 2.02R + 2 lz) per
    // component (conversions of both coordinates, the FP32 subtraction, the
    // periodic shift); 1.0001 and the upward rounding keep it an upper bound
    const double u24 = 5.9604644775390625e-08;
    g->eC = __double2float_ru(u24 * (4.0 * X + (per ? 2.0 * kp.lz : 0.0)) * 1.0001 + 1e-37);
    g->eR = __double2float_ru(u24 * 2.02 * 1.0001);
    // Units of the pair kernels (Grid::uL, uM, uV): the power of two at or
    // just above the mean h, the largest mass and a velocity scale (the
    // largest |v| component, or the sound speed the parameters imply if that
    // is larger: c0 for Tait, sqrt(gamma (gamma - 1) max u) for an ideal gas).
    auto unit_exp = [](double v) {
        int e = 0;
        if (!(v > 0.0) || !isfinite(v)) return 0;
        frexp(v, &e);  // v < 2^e
        return e < -300 ? -300 : (e > 300 ? 300 : e);
    };
    double vs = n > 0 ? r[9] : 0.0;
    if (kp.eos == 0) vs = fmax(vs, fabs(kp.c0));
    else if (n > 0 && r[10] > 0.0) vs = fmax(vs, sqrt(kp.gamma * (kp.gamma - 1.0) * r[10]));
    g->uL = unit_exp(hmean);
    g->uM = unit_exp(n > 0 ? r[8] : 0.0);
    g->uV = unit_exp(vs);
    // fixed-point exponent of the coordinate chunks (dfl::to_fx): |x| 2^k < 2^61,
    // and the chunks' float exponent k + uL must keep them normal floats
    int ex = 0;
    frexp(X, &ex);  // X < 2^ex
    int k = X > 0.0 && isfinite(X) ? 61 - ex : 61;
    k = k < -1000 ? -1000 : (k > 1000 ? 1000 : k);
    if (k + g->uL > 100 || k + g->uL < -60) {  // coordinates out of all proportion to h
        k = k + g->uL > 100 ? 100 - g->uL : -60 - g->uL;
        if (kp.precision == PREC_FP64) atomicOr(&status[0], (unsigned)ST_RANGE);
    }
    g->fxk = k;
    const dfl::fx3 L = dfl::to_fx(per ? kp.lz : 0.0, k, k + g->uL);
    g->lzc[0] = L.c2;
    g->lzc[1] = L.c1;
    g->lzc[2] = L.c0;
    g->hlzc = (float)(0.5 * kp.lz * p2d(-g->uL));
    g->hmean = hmean;
    g->hmax_bits = 0ull;
}

// ----------------------------------------------------------- Morton keys
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t compact3(uint32_t v) {
    v &= 0x09249249u;
    v = (v | (v >> 2)) & 0x030c30c3u;
    v = (v | (v >> 4)) & 0x0300f00fu;
    v = (v | (v >> 8)) & 0x030000ffu;
    v = (v | (v >> 16)) & 0x000003ffu;
    return v;
}

// Cell index along one axis, in FP32 from the truncated float of v (integer
// operations, no FP64 pipe). The neighbour search widens every query box by
// the grid's slop (>= 1e-3 cell widths), far more than these roundings, so
// any particle within reach of a query lies in a cell the query visits.
__device__ __forceinline__ int cell_coord(double v, float lo, float inv, int n) {
    const float f = floorf((dfl::from_double(v).hi - lo) * inv);
    const int top = n > 1 ? n - 1 : 0;
    if (!(f >= 0.0f)) return 0;  // also catches NaN
    if (f > (float)top) return top;
    return (int)f;
}

// key = instance (top 8 bits) | 24-bit Morton code of the particle's cell in
// its instance's grid, stored at the particle's rank roff[k] + (caller index
// - coff[k]) with its current slot as the value.
// While the instance keeps its candidate lists, the code is the particle's
// code at the list build, so the sort gives every particle its slot of then;
// a build step records the codes it sorts by.
__global__ void __launch_bounds__(kThreads)
k_keys(int64_t n, Batch B, const int64_t* __restrict__ coff, const int64_t* __restrict__ roff,
       const double4_32a* __restrict__ posh, const int32_t* __restrict__ order,
       uint32_t* __restrict__ keys, int32_t* __restrict__ vals, LMeta* __restrict__ lmeta) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int inst = slot_inst(B, k);
    if (!slot_real(B, inst, k)) return;
    const Grid* g = B.grid + inst;
    const bool lists = B.kp[inst].list_skin > 0.0;
    const int32_t id = order[k];
    uint32_t code;
    if (lists && !g->lbuild) {
        code = lmeta[id].code;
    } else {
        const double4_32a p = posh[k];
        const int kx = cell_coord(p.x, g->lof[0], g->invwf[0], g->n[0]);
        const int ky = cell_coord(p.y, g->lof[1], g->invwf[1], g->n[1]);
        const int kz = cell_coord(p.z, g->lof[2], g->invwf[2], g->n[2]);
        code = spread3(kx) | (spread3(ky) << 1) | (spread3(kz) << 2);
        if (lists) lmeta[id].code = code;
    }
    const int64_t q = __ldg(&roff[inst]) + ((int64_t)id - __ldg(&coff[inst]));
    keys[q] = ((uint32_t)inst << 24) | code;
    vals[q] = (int32_t)k;
}

// --------------------------------------------------------- stable radix sort
__global__ void __launch_bounds__(kThreads)
k_radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift, uint32_t* __restrict__ hist,
             int nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
#pragma unroll
    for (int k = 0; k < kRadixItems; ++k) {
        const int64_t i = base + k * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Each warp ranks a contiguous run of 256 keys in (iteration, lane) order, so
// the rank of a key among equal digits follows its input position: stable.
__global__ void __launch_bounds__(kThreads)
k_radix_scatter(const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin, int64_t n,
                int shift, const uint32_t* __restrict__ hist, int nblocks,
                uint32_t* __restrict__ kout, int32_t* __restrict__ vout) {
    __shared__ uint32_t cnt[kThreads / 32][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = threadIdx.x; q < (kThreads / 32) * 256; q += kThreads) (&cnt[0][0])[q] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile + warp * (32 * kRadixItems);
    uint32_t key[kRadixItems];
    int32_t val[kRadixItems];
    uint32_t rank[kRadixItems];
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int it = 0; it < kRadixItems; ++it) {
        const int64_t i = base + it * 32 + lane;
        const bool ok = i < n;
        key[it] = ok ? kin[i] : 0u;
        val[it] = ok ? vin[i] : 0;
        const uint32_t d = ok ? ((key[it] >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t b = ok ? cnt[warp][d] : 0u;
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) cnt[warp][d] = b + __popc(peers);
        __syncwarp();
        rank[it] = b + __popc(peers & lt);
    }
    __syncthreads();
    {
        const int d = threadIdx.x;  // one digit per thread
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            const uint32_t c = cnt[w][d];
            cnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kRadixItems; ++it) {
        const int64_t i = base + it * 32 + lane;
        if (i < n) {
            const uint32_t d = (key[it] >> shift) & 255u;
            const uint32_t pos = hist[(int64_t)d * nblocks + blockIdx.x] + cnt[warp][d] + rank[it];
            kout[pos] = key[it];
            vout[pos] = val[it];
        }
    }
}

// ------------------------------------------------------ permute and cells
// Sorted rank p of instance i goes to slot ioff[i] + (p - roff[i]).
__global__ void __launch_bounds__(kThreads)
k_permute(int64_t ntot, Batch B, const int64_t* __restrict__ roff,
          const uint32_t* __restrict__ keys, const int32_t* __restrict__ perm,
          const double4_32a* __restrict__ posh_in,
          const double4_32a* __restrict__ velm_in, const double* __restrict__ u_in,
          const int32_t* __restrict__ order_in, double4_32a* __restrict__ posh_out,
          double4_32a* __restrict__ velm_out, double* __restrict__ u_out,
          int32_t* __restrict__ order_out, float4* __restrict__ fpos, float4* __restrict__ xpk,
          float4* __restrict__ vpa, float2* __restrict__ vpb) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ntot) return;
    const int inst = (int)(keys[r] >> 24);
    const int64_t k = __ldg(&B.ioff[inst]) + (r - __ldg(&roff[inst]));
    const int64_t o = perm[r];
    const double4_32a p = posh_in[o];
    posh_out[k] = p;
    const double4_32a v = velm_in[o];
    velm_out[k] = v;
    write_xpk(xpk, k, p, v.w, B.grid[inst]);
    if (B.kp[inst].precision == PREC_FP64) write_vpk(vpa, vpb, k, v, B.grid[inst]);
    u_out[k] = u_in[o];
    order_out[k] = order_in[o];
    fpos[k] = make_float4((float)p.x, (float)p.y, (float)p.z, 0.0f);
}

// Clear each instance's cells (blockIdx.y = instance).
__global__ void __launch_bounds__(kThreads)
k_cells_clear(Batch B, int2* __restrict__ cells, unsigned long long* __restrict__ cell_hmax) {
    const Grid* g = B.grid + blockIdx.y;
    const long long nc = g->ncells, cb = g->cbase;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < nc;
         c += (long long)gridDim.x * blockDim.x) {
        cells[cb + c] = make_int2(0, 0);
        cell_hmax[cb + c] = 0ull;
    }
}

// Cell ranges (in slots) from the sorted keys (in ranks).
__global__ void __launch_bounds__(kThreads)
k_cells_mark(int64_t ntot, Batch B, const int64_t* __restrict__ roff,
             const uint32_t* __restrict__ keys, int2* __restrict__ cells) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ntot) return;
    const uint32_t key = keys[r];
    const int inst = (int)(key >> 24);
    const int64_t a = __ldg(&roff[inst]), e = a + __ldg(&B.icnt[inst]);
    const bool first = (r == a) || keys[r - 1] != key;
    const bool last = (r == e - 1) || keys[r + 1] != key;
    if (!(first || last)) return;
    const int64_t k = __ldg(&B.ioff[inst]) + (r - a);
    const Grid* g = B.grid + inst;
    const uint32_t code = key & 0xffffffu;
    const int kx = compact3(code), ky = compact3(code >> 1), kz = compact3(code >> 2);
    const long long lin = g->cbase + ((long long)kz * g->n[1] + ky) * g->n[0] + kx;
    if (first) cells[lin].x = (int)k;
    if (last) cells[lin].y = (int)(k + 1);
}

void launch_build_cells(sph_ctx* c, cudaStream_t s) {
    const int64_t n = c->n;
    const unsigned nb = (unsigned)((n + kThreads - 1) / kThreads);
    const Batch B = batch_of(c);
    c->launches += 1;
    if (nb > 0) {  // one block per group of kSlotAlign slots
        c->launches += 1;
        const unsigned gb = (unsigned)((n + kSlotAlign - 1) / kSlotAlign);
        if (c->any_lists)
            k_bbox<true><<<gb, kBoxThreads, 0, s>>>(n, B, c->posh[c->cur], c->velm[c->cur],
                                                 c->ue[c->cur], c->order[c->cur], c->lmeta,
                                                 c->red_part, c->status);
        else
            k_bbox<false><<<gb, kBoxThreads, 0, s>>>(n, B, c->posh[c->cur], c->velm[c->cur],
                                                  c->ue[c->cur], c->order[c->cur], c->lmeta,
                                                  c->red_part, c->status);
    }
    k_grid_setup<<<c->ninst, kGridThreads, 0, s>>>(c->red_part, B, c->grid, c->status, c->wctr,
                                                    c->lctr);
    if (n == 0) return;
    const int64_t nt = c->ntot;
    if (nt == 0) return;
    const unsigned nbt = (unsigned)((nt + kThreads - 1) / kThreads);
    const int passes = c->ninst > 1 ? 4 : 3;
    c->launches += 1 + passes * 5 + 3;
    k_keys<<<nb, kThreads, 0, s>>>(n, B, c->coff, c->roff, c->posh[c->cur], c->order[c->cur],
                                   c->keys[0], c->vals[0], c->lmeta);
    const int nsb = (int)((nt + kRadixTile - 1) / kRadixTile);
    int src = 0;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        k_radix_hist<<<nsb, kThreads, 0, s>>>(c->keys[src], nt, shift, c->hist, nsb);
        launch_scan_u32(c->hist, (int64_t)256 * nsb, c->hist_part, s);
        k_radix_scatter<<<nsb, kThreads, 0, s>>>(c->keys[src], c->vals[src], nt, shift, c->hist,
                                                  nsb, c->keys[1 - src], c->vals[1 - src]);
        src = 1 - src;
    }
    // sorted keys / permutation now in keys[src], vals[src]
    const int a = c->cur, b = 1 - c->cur;
    k_permute<<<nbt, kThreads, 0, s>>>(nt, B, c->roff, c->keys[src], c->vals[src], c->posh[a],
                                        c->velm[a], c->ue[a], c->order[a], c->posh[b], c->velm[b],
                                        c->ue[b], c->order[b], c->fpos, c->xpk, c->vpa, c->vpb);
    c->cur = b;
    k_cells_clear<<<dim3(64, (unsigned)c->ninst), kThreads, 0, s>>>(B, c->cells, c->cell_hmax);
    k_cells_mark<<<nbt, kThreads, 0, s>>>(nt, B, c->roff, c->keys[src], c->cells);
}

}  // namespace sph
