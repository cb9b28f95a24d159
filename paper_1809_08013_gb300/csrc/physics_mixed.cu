// physics_mixed.cu -- density and forces (Algorithm 1 step 3) in mixed
// precision: FP32 pair arithmetic on relative coordinates, FP32 kernel and
// gradient terms, sums accumulated in double-float (about 48 bits). Positions,
// the h / neighbour-count iteration, the time step and the integration stay
// FP64 (the neighbour sets are the exact FP64 ones). Definitions as in
// physics.cu; results are within ~1e-6 of the FP64 evaluation.
//
// Relative coordinates without the FP64 pipe: each FP64 position (and
// velocity) is split once per step into a float pair hi + lo; for a pair,
// (hi_i - hi_j) is exact when the two highs are within a factor of two (and
// within 2^-24 |dx| otherwise), so dx = (hi_i - hi_j) + (lo_i - lo_j) carries
// a relative error of a few 2^-24. Along the periodic z axis the wrap is
// applied to the exact high difference (see rel_z).
//
// Every quantity of the pack is in the instance's pair units (Grid::uL, uM,
// uV; powers of two near the mean h, the largest mass and a velocity scale),
// so FP32 holds it whatever units the caller uses; the sums go back to the
// caller's units exactly when they are written out.
//
// Per-particle pack, five float4 (80 B):
//   mpk[5k]   = (x_hi, y_hi, z_hi, m)      mpk[5k+1] = (x_lo, y_lo, z_lo, 1/h)
//   mpk[5k+2] = (vx_hi, vy_hi, vz_hi, 1/h^4)  mpk[5k+3] = (vx_lo, vy_lo, vz_lo, p/rho^2)
//   mpk[5k+4] = (h/2, rho/2, alpha c/2, 0)
#include <math_constants.h>

#include "df.cuh"
#include "sph_internal.cuh"

namespace sph {

using dfl::df;

namespace {

constexpr float kInvPiF = 0.318309886f;

__device__ __forceinline__ void split2(double d, float& hi, float& lo) {
    hi = __double2float_rn(d);
    lo = __double2float_rn(d - (double)hi);
}

// relative coordinate a_i - a_j from float pairs
__device__ __forceinline__ float rel(float hi_i, float lo_i, float hi_j, float lo_j) {
    return __fsub_rn(hi_i, hi_j) + __fsub_rn(lo_i, lo_j);
}

// Periodic z: the high difference is formed exactly (TwoSum) and wrapped by
// the high part of lz, which is exact for |dz_hi| in [lz/2, lz] (Sterbenz);
// the rounding error, the low parts and lz's low part go into the correction.
struct ZWrap {
    bool per;
    float half, lzh, lzl;
};

__device__ __forceinline__ ZWrap make_zwrap(const KParams& kp, const Grid& g) {
    ZWrap w;
    w.per = kp.periodic_z != 0;
    const double lz = kp.lz * p2d(-g.uL);  // in the length unit
    w.lzh = __double2float_rn(lz);
    w.lzl = __double2float_rn(lz - (double)w.lzh);
    w.half = 0.5f * w.lzh;
    return w;
}

__device__ __forceinline__ float rel_z(float hi_i, float lo_i, float hi_j, float lo_j,
                                       const ZWrap& w) {
    if (!w.per) return rel(hi_i, lo_i, hi_j, lo_j);
    const df t = dfl::two_sum(hi_i, -hi_j);
    float d = t.hi, corr = __fadd_rn(t.lo, __fsub_rn(lo_i, lo_j));
    if (d > w.half) {
        d = __fsub_rn(d, w.lzh);
        corr = __fsub_rn(corr, w.lzl);
    } else if (d < -w.half) {
        d = __fadd_rn(d, w.lzh);
        corr = __fadd_rn(corr, w.lzl);
    }
    return __fadd_rn(d, corr);
}

__device__ __forceinline__ float rsqrt_f(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y * fmaf(-0.5f * x * y, y, 1.5f);  // one Newton step
}

__device__ __forceinline__ float rcp_f(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y * fmaf(-x, y, 2.0f);
}

// pi h^3 W(q) and pi h^4 dW/dr (q) for q >= 0
__device__ __forceinline__ float w_shape_f(float q) {
    const float win = fmaf(q * q, fmaf(0.75f, q, -1.5f), 1.0f);
    const float t = 2.0f - q;
    const float wout = 0.25f * t * t * t;
    return q < 1.0f ? win : (q < 2.0f ? wout : 0.0f);
}

__device__ __forceinline__ float dw_shape_f(float q) {
    const float fin = q * fmaf(2.25f, q, -3.0f);
    const float t = 2.0f - q;
    const float fout = -0.75f * t * t;
    return q < 1.0f ? fin : (q < 2.0f ? fout : 0.0f);
}

__device__ __forceinline__ void eos_m(const KParams& kp, double rho, double u, double& p, double& c) {
    if (kp.eos == 0) {
        const double x = rho * kp.inv_rho0;  // within an ulp of rho / rho0
        const double x2 = x * x;
        const double x4 = x2 * x2;
        const double x7 = (x4 * x2) * x;
        p = kp.tait_k * (x7 - 1.0);
        c = kp.c0 * (x2 * x);
    } else {
        p = (kp.gamma - 1.0) * rho * u;
        c = sqrt(kp.gamma * (kp.gamma - 1.0) * u);
    }
}

}  // namespace

// Thermodynamic part of the pack (1/h^4, p/rho^2, h/2, rho/2, alpha c/2), in
// the pair units; a particle outside dfl::pack_in_range raises ST_RANGE.
__device__ __forceinline__ void pack_thermo(float4* __restrict__ mpk, int64_t k, double h,
                                            double rho, double A, double alpha, double c,
                                            const dfl::PairUnits& U, unsigned* status) {
    const double hu = U.iL / h;
    const double h2 = hu * hu;
    const double Au = A * U.A;
    const double ru = 0.5 * rho * U.rho;
    const double cu = 0.5 * alpha * c * U.V;
    if (!dfl::pack_in_range(hu, 2.0 * ru, Au, 2.0 * cu)) atomicOr(status, (unsigned)ST_RANGE);
    mpk[5 * k + 2].w = (float)(h2 * h2);
    mpk[5 * k + 3].w = (float)Au;
    mpk[5 * k + 4] = make_float4((float)(0.5 * h * U.L), (float)ru, (float)cu, 0.0f);
}

// Position / velocity / mass / 1/h part of the pack from the sorted state;
// with THERMO also the thermodynamic part from therm = (rho/2, p/rho^2,
// alpha c/2, h/2) (a standalone force call, where density ran elsewhere).
template <bool THERMO>
__global__ void __launch_bounds__(kThreads)
k_pack_mx(int64_t n, Batch B, const double4_32a* __restrict__ posh,
          const double4_32a* __restrict__ velm, const double4_32a* __restrict__ therm,
          float4* __restrict__ mpk, unsigned* status) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const Grid& g = B.grid[slot_inst(B, k)];
    const dfl::PairUnits U = dfl::pair_units(g.uL, g.uM, g.uV);
    const double4_32a p = posh[k];
    const double4_32a v = velm[k];
    float xh, xl, yh, yl, zh, zl, ah, al, bh, bl, ch, cl;
    split2(p.x * U.L, xh, xl);
    split2(p.y * U.L, yh, yl);
    split2(p.z * U.L, zh, zl);
    split2(v.x * U.V, ah, al);
    split2(v.y * U.V, bh, bl);
    split2(v.z * U.V, ch, cl);
    const double hinv = U.iL / p.w;
    mpk[5 * k + 0] = make_float4(xh, yh, zh, (float)(v.w * U.M));
    mpk[5 * k + 1] = make_float4(xl, yl, zl, (float)hinv);
    if (THERMO) {
        const double4_32a t = therm[k];
        mpk[5 * k + 2] = make_float4(ah, bh, ch, 0.0f);
        mpk[5 * k + 3] = make_float4(al, bl, cl, 0.0f);
        pack_thermo(mpk, k, p.w, 2.0 * t.x, t.y, 1.0, 2.0 * t.z, U, status);
    } else {
        mpk[5 * k + 2] = make_float4(ah, bh, ch, 0.0f);
        mpk[5 * k + 3] = make_float4(al, bl, cl, 0.0f);
    }
}

// T lanes per particle: lane s of particle i takes row entries s, s + T, ...
// OUTER: as k_density_df, the kernel also records in omask the gather entries
// j of row i with i not in N_j. The FP32 relative coordinates put r^2 within
// ~2^-21 of the defining FP64 value and 1/h_j is packed as a float, so
// r^2 / h_j^2 below / above 4 by more than 2^-18 decides; the band between,
// and a periodic axis shorter than 8 h_j, take the FP64 test itself.
template <bool FUSE, int T, bool OUTER>
__global__ void __launch_bounds__(kThreads)
k_density_mx(int64_t n, Batch B, const double4_32a* __restrict__ posh,
             const double* __restrict__ ue, float4* __restrict__ mpk,
             Rows R, double4_32a* __restrict__ therm,
             double* __restrict__ pint, double* __restrict__ cint, unsigned* status,
             unsigned long long* __restrict__ omask) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / T;
    const int sub = (int)(threadIdx.x % T);
    const int inst = slot_inst(B, ((int64_t)blockIdx.x * blockDim.x) / T);
    const int32_t* ent = nullptr;
    int len = 0;
    const bool act = i < n && slot_real(B, inst, i) && row_of(R, n, i, true, ent, len);
    if (T == 1 && !act) return;
    const KParams& kp = B.kp[inst];
    df acc = {0.0f, 0.0f};
    unsigned long long om0 = 0ull, om1 = 0ull;  // OUTER: bits of the gather entries
    if (act) {
    const float4 a0 = mpk[5 * i], a1 = mpk[5 * i + 1];
    const float hinv = a1.w;
    const ZWrap zw = make_zwrap(kp, B.grid[inst]);
    if (sub == 0) acc = df{a0.w, 0.0f};  // self term m_i W(0, h_i): shape 1
    // rows read from the CSR (a gather set overflowed) are complete already
    const bool append = OUTER && !(R.status[2] & IF_SLAB_OVF);
    for (int e = sub; e < len; e += T) {
        const int j = __ldg(&ent[e]);
        const float4 b0 = __ldg(&mpk[5 * j]), b1 = __ldg(&mpk[5 * j + 1]);
        const float dx = rel(a0.x, a1.x, b0.x, b1.x), dy = rel(a0.y, a1.y, b0.y, b1.y);
        const float dz = rel_z(a0.z, a1.z, b0.z, b1.z, zw);
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float q = r2 > 0.0f ? r2 * rsqrt_f(r2) * hinv : 0.0f;
        acc = dfl::addf(acc, b0.w * w_shape_f(q));
        if (append) {
            const float t = r2 * b1.w * b1.w;  // (r / h_j)^2
            bool in_j;
            if (!(zw.per && b1.w * zw.lzh < 8.0f) && t < 4.0f * 0.99999619f) {
                in_j = true;
            } else if (!(zw.per && b1.w * zw.lzh < 8.0f) && t > 4.0f * 1.00000381f) {
                in_j = false;
            } else {
                const double4_32a pj = posh[j];
                const double Rj = 2.0 * pj.w;
                in_j = exact_r2_def(posh[i], pj, zw.per, kp.lz) < __dmul_rn(Rj, Rj);
            }
            if (!in_j) {  // i belongs in the outer part of row j
                if (e < 64) om0 |= 1ull << e;
                else om1 |= 1ull << (e - 64);
            }
        }
    }
    }
    if (T > 1) {
        acc = dfl::lane_sum<T>(acc);
        if (OUTER) {
#pragma unroll
            for (int o = 1; o < T; o <<= 1) {
                om0 |= __shfl_xor_sync(0xffffffffu, om0, o);
                om1 |= __shfl_xor_sync(0xffffffffu, om1, o);
            }
        }
        if (!act || sub != 0) return;
    }
    if (OUTER) {
        omask[2 * i] = om0;
        omask[2 * i + 1] = om1;
    }
    const Grid& g = B.grid[inst];
    const double hd = posh[i].w;
    const double hid = 1.0 / hd;
    const double rho = dfl::to_double(acc) * p2d(g.uM) * (hid * hid * hid * 0.31830988618379067154);
    if (FUSE) {
        double p, c;
        eos_m(kp, rho, ue[i], p, c);
        const double A = p / (rho * rho);
        therm[i] = make_double4_32a(0.5 * rho, A, 0.5 * kp.alpha * c, 0.5 * hd);
        pack_thermo(mpk, i, hd, rho, A, kp.alpha, c, dfl::pair_units(g.uL, g.uM, g.uV), status);
        pint[i] = p;
        cint[i] = c;
    } else {
        therm[i].x = 0.5 * rho;
    }
}

template <int T>
__global__ void __launch_bounds__(kThreads)
k_forces_mx(int64_t n, Batch B, const double4_32a* __restrict__ posh,
            const float4* __restrict__ mpk, const double* __restrict__ cint,
            Rows R,
            double4_32a* __restrict__ acc, double* __restrict__ mumax,
            double* __restrict__ dt_part) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / T;
    const int sub = (int)(threadIdx.x % T);
    const int inst = slot_inst(B, ((int64_t)blockIdx.x * blockDim.x) / T);
    const int32_t* ent = nullptr;
    int len = 0;
    const bool act = i < n && slot_real(B, inst, i) && row_of(R, n, i, false, ent, len);
    double dtc = CUDART_INF;
    df sx = {0.f, 0.f}, sy = {0.f, 0.f}, sz = {0.f, 0.f}, sp = {0.f, 0.f}, sv = {0.f, 0.f};
    float mum = 0.0f;
    if (act) {
        const KParams& kp = B.kp[inst];
        const float4 a0 = mpk[5 * i], a1 = mpk[5 * i + 1], a2 = mpk[5 * i + 2];
        const float4 a3 = mpk[5 * i + 3], a4 = mpk[5 * i + 4];
        const ZWrap zw = make_zwrap(kp, B.grid[inst]);
        const float eta2 = (float)kp.eta2, beta = (float)kp.beta;
        const float cpi = 0.5f * kInvPiF;
        for (int e = sub; e < len; e += T) {
            const int j = __ldg(&ent[e]);
            const float4 b0 = __ldg(&mpk[5 * j]), b1 = __ldg(&mpk[5 * j + 1]);
            const float4 b2 = __ldg(&mpk[5 * j + 2]), b3 = __ldg(&mpk[5 * j + 3]);
            const float4 b4 = __ldg(&mpk[5 * j + 4]);
            const float dx = rel(a0.x, a1.x, b0.x, b1.x), dy = rel(a0.y, a1.y, b0.y, b1.y);
            const float dz = rel_z(a0.z, a1.z, b0.z, b1.z, zw);
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (!(r2 > 0.0f)) continue;  // coincident particles exert no force
            const float rinv = rsqrt_f(r2);
            const float r = r2 * rinv;
            const float fa = dw_shape_f(r * a1.w), fb = dw_shape_f(r * b1.w);
            const float Fb = fmaf(a2.w, fa, b2.w * fb) * (cpi * rinv);
            const float wx = rel(a2.x, a3.x, b2.x, b3.x), wy = rel(a2.y, a3.y, b2.y, b3.y);
            const float wz = rel(a2.z, a3.z, b2.z, b3.z);
            const float vr = fmaf(wz, dz, fmaf(wy, dy, wx * dx));
            float Pi = 0.0f;
            if (vr < 0.0f) {
                const float hb = a4.x + b4.x;
                const float d1 = fmaf(eta2 * hb, hb, r2);
                const float rb = a4.y + b4.y;
                const float R = rcp_f(d1 * rb);
                const float mu = hb * vr * rb * R;
                Pi = mu * fmaf(beta, mu, -(a4.z + b4.z)) * (d1 * R);
                mum = fmaxf(mum, -mu);
            }
            const float mF = b0.w * Fb;
            const float g = mF * ((a3.w + b3.w) + Pi);
            sx = dfl::addf(sx, g * dx);
            sy = dfl::addf(sy, g * dy);
            sz = dfl::addf(sz, g * dz);
            const float mFv = mF * vr;
            sp = dfl::addf(sp, mFv);
            sv = dfl::addf(sv, mFv * Pi);
        }
    }
    if (T > 1) {
        sx = dfl::lane_sum<T>(sx);
        sy = dfl::lane_sum<T>(sy);
        sz = dfl::lane_sum<T>(sz);
        sp = dfl::lane_sum<T>(sp);
        sv = dfl::lane_sum<T>(sv);
#pragma unroll
        for (int o = 1; o < T; o <<= 1) mum = fmaxf(mum, __shfl_xor_sync(0xffffffffu, mum, o));
    }
    if (act && sub == 0) {
        // back to the caller's units: a ~ V^2 / L, du ~ V^3 / L, mu ~ V
        const int ins = slot_inst(B, ((int64_t)blockIdx.x * blockDim.x) / T);
        const Grid& gu = B.grid[ins];
        const double sa = p2d(2 * gu.uV - gu.uL), su = p2d(3 * gu.uV - gu.uL);
        const double Aid = (double)mpk[5 * i + 3].w;
        acc[i] = make_double4_32a(-dfl::to_double(sx) * sa, -dfl::to_double(sy) * sa,
                                  -dfl::to_double(sz) * sa,
                                  fma(Aid, dfl::to_double(sp), 0.5 * dfl::to_double(sv)) * su);
        const double mu_max = (double)mum * p2d(gu.uV);
        mumax[i] = mu_max;
        const double ci = cint[i];
        // parameters re-read here rather than kept in registers across the loop
        const KParams& ke = B.kp[ins];
        dtc = posh[i].w / (ci + 1.2 * (ke.alpha * ci + ke.beta * mu_max));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dtc = fmin(dtc, __shfl_xor_sync(0xffffffffu, dtc, o));
    __shared__ double sh[kThreads / 32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = dtc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = sh[0];
        for (int w = 1; w < kThreads / 32; ++w) m = fmin(m, sh[w]);
        dt_part[blockIdx.x] = m;
    }
}

void launch_pack_mx(sph_ctx* c, bool thermo, cudaStream_t s) {
    const int64_t n = c->n;
    if (n == 0) return;
    const unsigned nb = (unsigned)((n + kThreads - 1) / kThreads);
    const int b = c->cur;
    c->launches += 1;
    if (thermo)
        k_pack_mx<true><<<nb, kThreads, 0, s>>>(n, batch_of(c), c->posh[b], c->velm[b], c->therm,
                                                c->mpk, c->status);
    else
        k_pack_mx<false><<<nb, kThreads, 0, s>>>(n, batch_of(c), c->posh[b], c->velm[b], c->therm,
                                                 c->mpk, c->status);
}

template <bool FUSE, int T, bool OUTER>
static void density_mx_t(sph_ctx* c, cudaStream_t s) {
    const int64_t n = c->n;
    const unsigned nb = (unsigned)((n * T + kThreads - 1) / kThreads);
    const int b = c->cur;
    k_density_mx<FUSE, T, OUTER><<<nb, kThreads, 0, s>>>(
        n, batch_of(c), c->posh[b], c->ue[b], c->mpk, OUTER ? rows_gather(c) : rows_of(c),
        c->therm, c->pint, c->cint, c->status, c->omask);
}

template <bool FUSE, bool OUTER>
static void density_mx_f(sph_ctx* c, cudaStream_t s) {
    switch (c->tpp) {
        case 2: density_mx_t<FUSE, 2, OUTER>(c, s); break;
        case 4: density_mx_t<FUSE, 4, OUTER>(c, s); break;
        case 8: density_mx_t<FUSE, 8, OUTER>(c, s); break;
        default: density_mx_t<FUSE, 1, OUTER>(c, s); break;
    }
}

void launch_density_mx(sph_ctx* c, bool fuse_eos, cudaStream_t s, bool outer) {
    if (c->n == 0) return;
    c->launches += 1;
    if (fuse_eos && outer) density_mx_f<true, true>(c, s);
    else if (fuse_eos) density_mx_f<true, false>(c, s);
    else density_mx_f<false, false>(c, s);
}

template <int T>
static void forces_mx_t(sph_ctx* c, cudaStream_t s) {
    const int64_t n = c->n;
    const unsigned nb = (unsigned)((n * T + kThreads - 1) / kThreads);
    const int b = c->cur;
    k_forces_mx<T><<<nb, kThreads, 0, s>>>(n, batch_of(c), c->posh[b], c->mpk, c->cint,
                                           rows_of(c), c->acc, c->mumax,
                                           c->dt_part);
}

void launch_forces_mx(sph_ctx* c, cudaStream_t s) {
    if (c->n == 0) return;
    c->launches += 1;
    switch (c->tpp) {
        case 2: forces_mx_t<2>(c, s); break;
        case 4: forces_mx_t<4>(c, s); break;
        case 8: forces_mx_t<8>(c, s); break;
        default: forces_mx_t<1>(c, s); break;
    }
}

}  // namespace sph
