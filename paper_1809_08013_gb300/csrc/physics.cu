// physics.cu -- Algorithm 1 steps 3, 5 and 6: density summation, equation of
// state, momentum and energy with Monaghan artificial viscosity, the new time
// step, and the kick-drift update. All arithmetic is FP64.
//
// M4 cubic spline (Table 1) in branch-free form: with q = r/h,
// t = max(2 - q, 0) and s = max(1 - q, 0),
//   W(r, h)     = (1/(pi h^3)) (t^3/4 - s^3)
//   dW/dr(r, h) = (1/(pi h^4)) (3 s^2 - 3 t^2/4)
// which equals the piecewise definition on [0,1), [1,2) and [2, inf).
#include <math_constants.h>

#include "sph_internal.cuh"

namespace sph {

// ---- FP64-pipe economy helpers. GB300 issues FP64 arithmetic at 1/64 of
// the FP32 rate, so compares, selects, sign tests and clamps are done with
// integer operations on the IEEE bit patterns (which order non-negative
// doubles like their values), and divisions / square roots start from the
// hardware approximations refined by Newton-Raphson.
__device__ __forceinline__ long long bits(double v) { return __double_as_longlong(v); }

// 1/sqrt(x), x > 0 normal: rsqrt.approx.f64 seed, two Newton-Raphson steps
// y <- y (3/2 - x/2 y^2) (quadratic convergence; a few ulp in the end).
__device__ __forceinline__ double rsqrt_nr(double x) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double hx = 0.5 * x;
    y = y * fma(-hx, y * y, 1.5);
    y = y * fma(-hx, y * y, 1.5);
    return y;
}

// 1/d, d > 0 normal: rcp.approx.ftz.f64 seed, two Newton-Raphson steps
// y <- y + y (1 - d y).
__device__ __forceinline__ double rcp_nr(double d) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
    double e = fma(-d, y, 1.0);
    y = fma(y, e, y);
    e = fma(-d, y, 1.0);
    y = fma(y, e, y);
    return y;
}

// Minimum image along z: |dz| > lz/2 (integer compare of |dz|'s bits) shifts
// dz by -sign(dz) lz, the same two-sided rule as the definition.
__device__ __forceinline__ double wrap_z(double dz, long long half_bits, double lz) {
    if ((bits(dz) & 0x7fffffffffffffffLL) > half_bits) dz -= copysign(lz, dz);
    return dz;
}

constexpr long long kOneBits = 0x3ff0000000000000LL;  // bits of 1.0
constexpr long long kTwoBits = 0x4000000000000000LL;  // bits of 2.0

// Cubic-spline shape g(q) = pi h^3 W: 1 - 1.5 q^2 + 0.75 q^3 (q < 1),
// (2 - q)^3 / 4 (1 <= q < 2), 0 beyond; q >= 0.
__device__ __forceinline__ double w_shape(double q) {
    const double q2 = q * q;
    const double win = fma(q2, fma(0.75, q, -1.5), 1.0);
    const double t = 2.0 - q;
    const double wout = (0.25 * t) * (t * t);
    const long long qb = bits(q);
    return qb < kOneBits ? win : (qb < kTwoBits ? wout : 0.0);
}

// Derivative shape f(q) = pi h^4 dW/dr: q (2.25 q - 3) (q < 1),
// -0.75 (2 - q)^2 (1 <= q < 2), 0 beyond; q >= 0.
__device__ __forceinline__ double dw_shape(double q) {
    const double fin = q * fma(2.25, q, -3.0);
    const double t = 2.0 - q;
    const double fout = (-0.75 * t) * t;
    const long long qb = bits(q);
    return qb < kOneBits ? fin : (qb < kTwoBits ? fout : 0.0);
}

// ---- Table 1 kernel variants, as shapes g (W = wnorm h^-3 g(q)) and f
// (dW/dr = dnorm h^-4 f(q)), zero from q = 2 on:
//   Wendland C2: g = (1 - q/2)^4 (1 + 2q), f = -q (1 - q/2)^3
//     (wnorm = 21/(16 pi), dnorm = 105/(16 pi));
//   sinc: with x = pi q / 2 and S = sin x / x, g = S^n and
//     f = n S^(n-1) (x cos x - sin x) / x^2 (wnorm = B_n, dnorm = B_n pi / 2).
__device__ __forceinline__ double ipow(double v, int k) {
    double r = 1.0;
    for (int e = 0; e < k; ++e) r *= v;
    return r;
}

template <int KER>
__device__ __forceinline__ double kw(double q, int sn) {
    if (KER == KER_M4) return w_shape(q);
    if (!(bits(q) < kTwoBits)) return 0.0;
    if (KER == KER_WENDLAND) {
        const double t = 1.0 - 0.5 * q;
        const double t2 = t * t;
        return (t2 * t2) * (1.0 + 2.0 * q);
    }
    const double x = (0.5 * kPi) * q;
    return bits(x) == 0 ? 1.0 : ipow(sin(x) / x, sn);
}

template <int KER>
__device__ __forceinline__ double kdw(double q, int sn) {
    if (KER == KER_M4) return dw_shape(q);
    if (!(bits(q) < kTwoBits)) return 0.0;
    if (KER == KER_WENDLAND) {
        const double t = 1.0 - 0.5 * q;
        return -(q * ((t * t) * t));
    }
    const double x = (0.5 * kPi) * q;
    if (bits(x) == 0) return 0.0;
    double sx, cx;
    sincos(x, &sx, &cx);
    const double S = sx / x;
    return ((double)sn * ipow(S, sn - 1)) * ((x * cx - sx) / (x * x));
}

__device__ __forceinline__ void eos(const KParams& kp, double rho, double u, double& p, double& c) {
    if (kp.eos == 0) {
        const double x = rho / kp.rho0;
        const double x2 = x * x;
        const double x4 = x2 * x2;
        const double x7 = (x4 * x2) * x;
        p = (kp.c0 * kp.c0 * kp.rho0 / 7.0) * (x7 - 1.0);
        c = kp.c0 * (x2 * x);
    } else {
        p = (kp.gamma - 1.0) * rho * u;
        c = sqrt(kp.gamma * (kp.gamma - 1.0) * u);
    }
}

// ------------------------------------------------------------ density
// rho_i = m_i W(0, h_i) + sum_{j in N_i} m_j W(r_ij, h_i). With FUSE the EOS
// follows in the same thread and the pair kernels' per-particle packs are
// written: therm = (rho/2, p/rho^2, alpha c/2, h/2), kern = (1/h, 1/h^4).
template <bool FUSE, int KER>
__global__ void __launch_bounds__(kThreads)
k_density(int64_t n, Batch B, const double4_32a* __restrict__ posh,
          const double4_32a* __restrict__ velm, const double* __restrict__ ue,
          Rows R, double4_32a* __restrict__ therm,
          double2* __restrict__ kern, double* __restrict__ pint, double* __restrict__ cint) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int inst = slot_inst(B, (int64_t)blockIdx.x * blockDim.x);
    const int32_t* ent = nullptr;
    int len = 0;
    if (i >= n || !slot_real(B, inst, i) || !row_of(R, n, i, true, ent, len)) return;
    const KParams& kp = B.kp[inst];
    const double4_32a pi = posh[i];
    const double hinv = 1.0 / pi.w;
    const long long half_bits = bits(0.5 * kp.lz);
    const bool per = kp.periodic_z != 0;
    const double lz = kp.lz;
    const int sn = kp.sinc_n;
    double acc = 0.0;
    for (int e = 0; e < len; ++e) {
        const int j = __ldg(&ent[e]);
        const double4_32a pj = posh[j];
        const double mj = velm[j].w;
        const double dx = pi.x - pj.x, dy = pi.y - pj.y;
        double dz = pi.z - pj.z;
        if (per) dz = wrap_z(dz, half_bits, lz);
        const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        // r2 > 0 for j != i unless two particles coincide; r = r2 / sqrt(r2)
        const double q = bits(r2) > 0 ? r2 * rsqrt_nr(r2) * hinv : 0.0;
        acc = fma(mj, kw<KER>(q, sn), acc);
    }
    const double sigma = hinv * hinv * hinv * (KER == KER_M4 ? kInvPi : B.kp[inst].wnorm);
    const double rho = (velm[i].w + acc) * sigma;  // g(0) = 1 for every kernel
    if (FUSE) {
        double p, c;
        eos(kp, rho, ue[i], p, c);
        therm[i] = make_double4_32a(0.5 * rho, p / (rho * rho), 0.5 * kp.alpha * c, 0.5 * pi.w);
        const double h2 = hinv * hinv;
        kern[i] = make_double2(hinv, h2 * h2);
        pint[i] = p;
        cint[i] = c;
    } else {
        therm[i].x = 0.5 * rho;
    }
}

void launch_density(sph_ctx* c, bool fuse_eos, cudaStream_t s, bool outer) {
    if (c->prec == PREC_MIXED) {
        launch_pack_mx(c, false, s);
        launch_density_mx(c, fuse_eos, s, outer);
        return;
    }
    if (!native_pairs(c)) {
        launch_density_df(c, fuse_eos, s, outer);
        return;
    }
    const int64_t n = c->n;
    if (n == 0) return;
    const unsigned nb = (unsigned)((n + kThreads - 1) / kThreads);
    const int b = c->cur;
    const Batch B = batch_of(c);
    c->launches += 1;
    auto go = [&](auto kern_fn) {
        kern_fn<<<nb, kThreads, 0, s>>>(n, B, c->posh[b], c->velm[b], c->ue[b], rows_of(c),
                                        c->therm, c->kern, c->pint, c->cint);
    };
    switch (c->kern_kind * 2 + (fuse_eos ? 1 : 0)) {
        case 0: go(k_density<false, KER_M4>); break;
        case 1: go(k_density<true, KER_M4>); break;
        case 2: go(k_density<false, KER_WENDLAND>); break;
        case 3: go(k_density<true, KER_WENDLAND>); break;
        case 4: go(k_density<false, KER_SINC>); break;
        default: go(k_density<true, KER_SINC>); break;
    }
}

// ------------------------------------------------------------ EOS (caller arrays)
__global__ void __launch_bounds__(kThreads)
k_eos_caller(int64_t n, KParams kp, const double* __restrict__ rho, const double* __restrict__ u,
             double* __restrict__ p, double* __restrict__ c) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double pp, cc;
    eos(kp, rho[i], u ? u[i] : 0.0, pp, cc);
    p[i] = pp;
    c[i] = cc;
}

void launch_eos_caller(const KParams& kp, const sph_particles* P, cudaStream_t s) {
    if (P->n == 0) return;
    k_eos_caller<<<(unsigned)((P->n + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        P->n, kp, P->rho, P->u, P->p, P->c);
}

// ------------------------------------------------------------ forces + dt
// For j in S_i, r_ij = r_i - r_j, v_ij = v_i - v_j:
//   Fbar = (dW/dr(r, h_i) + dW/dr(r, h_j)) / (2 r)
//   mu   = hb v.r / (r^2 + eta2 hb^2), Pi = (-alpha cb mu + beta mu^2) / rhob  if v.r < 0
//   a_i  = -sum m_j (A_i + A_j + Pi) Fbar r_ij
//   du_i = A_i sum m_j Fbar v.r + 1/2 sum m_j Pi Fbar v.r
// and the time-step candidate h_i / (c_i + 1.2 (alpha c_i + beta mumax_i)).
// Algebra used: Fbar = (0.5/pi) (f(q_i)/h_i^4 + f(q_j)/h_j^4) / r with the
// shape f above; both divisions of the viscosity share one reciprocal,
// R = 1 / ((r^2 + eta2 hb^2) rhob): mu = hb v.r rhob R and 1/rhob = (r^2 +
// eta2 hb^2) R; Pi = mu (beta mu - alpha cb) / rhob.
template <int KER>
__global__ void __launch_bounds__(kThreads)
k_forces(int64_t n, Batch B, const double4_32a* __restrict__ posh,
         const double4_32a* __restrict__ velm, const double4_32a* __restrict__ therm,
         const double2* __restrict__ kern, const double* __restrict__ cint,
         Rows R,
         double4_32a* __restrict__ acc, double* __restrict__ mumax, double* __restrict__ dt_part) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int inst = slot_inst(B, (int64_t)blockIdx.x * blockDim.x);
    double dtc = CUDART_INF;
    const int32_t* ent = nullptr;
    int len = 0;
    if (i < n && slot_real(B, inst, i) && row_of(R, n, i, false, ent, len)) {
        const KParams& kp = B.kp[inst];
        const double4_32a pi = posh[i];
        const double4_32a vi = velm[i];
        const double4_32a ti = therm[i];
        const double2 ki = kern[i];
        const long long half_bits = bits(0.5 * kp.lz);
        const bool per = kp.periodic_z != 0;
        const double lz = kp.lz;
        const double eta2 = kp.eta2, beta = kp.beta;
        const int sn = kp.sinc_n;
        const double cpi = 0.5 * (KER == KER_M4 ? kInvPi : kp.dnorm);
        double sx = 0.0, sy = 0.0, sz = 0.0, sp = 0.0, sv = 0.0;
        long long mum = 0;  // bits of max |mu| (non-negative doubles order as integers)
        for (int e = 0; e < len; ++e) {
            const int j = __ldg(&ent[e]);
            const double4_32a pj = posh[j];
            const double4_32a vj = velm[j];
            const double4_32a tj = therm[j];
            const double2 kj = __ldg(&kern[j]);
            const double dx = pi.x - pj.x, dy = pi.y - pj.y;
            double dz = pi.z - pj.z;
            if (per) dz = wrap_z(dz, half_bits, lz);
            const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
            if (bits(r2) == 0) continue;  // coincident particles exert no force
            const double rinv = rsqrt_nr(r2);
            const double r = r2 * rinv;
            const double fa = kdw<KER>(r * ki.x, sn), fb = kdw<KER>(r * kj.x, sn);
            const double Fb = fma(ki.y, fa, kj.y * fb) * (cpi * rinv);
            const double wx = vi.x - vj.x, wy = vi.y - vj.y, wz = vi.z - vj.z;
            const double vr = fma(wz, dz, fma(wy, dy, wx * dx));
            double Pi = 0.0;
            if (__double2hiint(vr) < 0) {  // v.r < 0 (a -0 gives mu = Pi = 0 as well)
                const double hb = ti.w + tj.w;
                const double d1 = fma(eta2 * hb, hb, r2);
                const double rb = ti.x + tj.x;
                const double R = rcp_nr(d1 * rb);
                const double mu = ((hb * vr) * rb) * R;
                Pi = (mu * fma(beta, mu, -(ti.z + tj.z))) * (d1 * R);
                const long long ab = bits(mu) & 0x7fffffffffffffffLL;
                mum = ab > mum ? ab : mum;
            }
            const double mF = vj.w * Fb;
            const double g = mF * ((ti.y + tj.y) + Pi);
            sx = fma(g, dx, sx);
            sy = fma(g, dy, sy);
            sz = fma(g, dz, sz);
            const double mFv = mF * vr;
            sp += mFv;
            sv = fma(mFv, Pi, sv);
        }
        const double mu_max = __longlong_as_double(mum);
        acc[i] = make_double4_32a(-sx, -sy, -sz, fma(ti.y, sp, 0.5 * sv));
        mumax[i] = mu_max;
        const double ci = cint[i];
        // parameters re-read here rather than kept in registers across the loop
        const KParams& ke = B.kp[slot_inst(B, (int64_t)blockIdx.x * blockDim.x)];
        dtc = pi.w / (ci + 1.2 * (ke.alpha * ci + ke.beta * mu_max));
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

// ------------------------------------------------------------ IAD (Table 1)
// Volume elements V_i = m_i / rho_i, once per particle (rho from the force
// pack, therm.x = rho / 2), so that the matrix pass reads one number per
// neighbour and divides nowhere.
__global__ void __launch_bounds__(kThreads)
k_volume(int64_t n, Batch B, const double4_32a* __restrict__ velm,
         const double4_32a* __restrict__ therm, double* __restrict__ vol) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int inst = slot_inst(B, i);
    if (!slot_real(B, inst, i)) return;
    vol[i] = velm[i].w / (2.0 * therm[i].x);
}

// tau_i = sum_{j in N_i} V_j W(r_ij, h_i) (r_j - r_i)(r_j - r_i)^T and
// C_i = tau_i^-1 by the adjugate (C_i = 0 when det tau_i = 0); after the
// density (V_j needs rho_j).
template <int KER>
__global__ void __launch_bounds__(kThreads)
k_iad(int64_t n, Batch B, const double4_32a* __restrict__ posh,
      const double* __restrict__ vol, Rows R,
      double4_32a* __restrict__ ca, double2* __restrict__ cb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int inst = slot_inst(B, (int64_t)blockIdx.x * blockDim.x);
    const int32_t* ent = nullptr;
    int len = 0;
    if (i >= n || !slot_real(B, inst, i) || !row_of(R, n, i, true, ent, len)) return;
    const KParams& kp = B.kp[inst];
    const double4_32a pi = posh[i];
    const double hinv = 1.0 / pi.w;
    const long long half_bits = bits(0.5 * kp.lz);
    const bool per = kp.periodic_z != 0;
    const double lz = kp.lz;
    const int sn = kp.sinc_n;
    double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0, t4 = 0.0, t5 = 0.0;
    for (int e = 0; e < len; ++e) {
        const int j = __ldg(&ent[e]);
        const double4_32a pj = posh[j];
        const double dx = pi.x - pj.x, dy = pi.y - pj.y;
        double dz = pi.z - pj.z;
        if (per) dz = wrap_z(dz, half_bits, lz);
        const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        const double q = bits(r2) > 0 ? r2 * rsqrt_nr(r2) * hinv : 0.0;
        const double w = __ldg(&vol[j]) * kw<KER>(q, sn);
        const double wx = w * dx, wy = w * dy;
        t0 = fma(wx, dx, t0);
        t1 = fma(wx, dy, t1);
        t2 = fma(wx, dz, t2);
        t3 = fma(wy, dy, t3);
        t4 = fma(wy, dz, t4);
        t5 = fma(w * dz, dz, t5);
    }
    const double sg = hinv * hinv * hinv * (KER == KER_M4 ? kInvPi : B.kp[inst].wnorm);
    t0 *= sg; t1 *= sg; t2 *= sg; t3 *= sg; t4 *= sg; t5 *= sg;
    // cofactors of [[t0 t1 t2] [t1 t3 t4] [t2 t4 t5]]
    const double c00 = t3 * t5 - t4 * t4, c01 = t2 * t4 - t1 * t5, c02 = t1 * t4 - t2 * t3;
    const double c11 = t0 * t5 - t2 * t2, c12 = t1 * t2 - t0 * t4, c22 = t0 * t3 - t1 * t1;
    const double det = t0 * c00 + t1 * c01 + t2 * c02;
    if (det == 0.0) {
        ca[i] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        cb[i] = make_double2(0.0, 0.0);
        return;
    }
    ca[i] = make_double4_32a(c00 / det, c01 / det, c02 / det, c11 / det);
    cb[i] = make_double2(c12 / det, c22 / det);
}

// Forces with IAD gradients: the pair gradient Fbar r_ij becomes
//   G_ij = (W(r, h_i) C_i + W(r, h_j) C_j) (r_j - r_i) / 2
// in the momentum and energy sums (viscosity, mu and dt as in k_forces):
//   a_i  = -sum m_j (A_i + A_j + Pi) G_ij
//   du_i = A_i sum m_j G_ij . v_ij + 1/2 sum m_j Pi G_ij . v_ij
// With W = wnorm h^-3 g(q): G_ij = -(wnorm/2) (h_i^-3 g_i C_i + h_j^-3 g_j C_j) r_ij.
template <int KER>
__global__ void __launch_bounds__(kThreads)
k_forces_iad(int64_t n, Batch B, const double4_32a* __restrict__ posh,
             const double4_32a* __restrict__ velm, const double4_32a* __restrict__ therm,
             const double2* __restrict__ kern, const double* __restrict__ cint,
             const double4_32a* __restrict__ ca, const double2* __restrict__ cb, Rows R,
             double4_32a* __restrict__ acc, double* __restrict__ mumax,
             double* __restrict__ dt_part) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int inst = slot_inst(B, (int64_t)blockIdx.x * blockDim.x);
    double dtc = CUDART_INF;
    const int32_t* ent = nullptr;
    int len = 0;
    if (i < n && slot_real(B, inst, i) && row_of(R, n, i, false, ent, len)) {
        const KParams& kp = B.kp[inst];
        const double4_32a pi = posh[i];
        const double4_32a vi = velm[i];
        const double4_32a ti = therm[i];
        const double hi = kern[i].x;
        const double hi3 = hi * hi * hi;
        const double4_32a ci = ca[i];
        const double2 ci2 = cb[i];
        const long long half_bits = bits(0.5 * kp.lz);
        const bool per = kp.periodic_z != 0;
        const double lz = kp.lz;
        const double eta2 = kp.eta2, beta = kp.beta;
        const int sn = kp.sinc_n;
        const double kg = -0.5 * (KER == KER_M4 ? kInvPi : kp.wnorm);
        double sx = 0.0, sy = 0.0, sz = 0.0, sp = 0.0, sv = 0.0;
        long long mum = 0;
        for (int e = 0; e < len; ++e) {
            const int j = __ldg(&ent[e]);
            const double4_32a pj = posh[j];
            const double4_32a vj = velm[j];
            const double4_32a tj = therm[j];
            const double hj = __ldg(&kern[j].x);
            const double4_32a cj = ca[j];
            const double2 cj2 = cb[j];
            const double dx = pi.x - pj.x, dy = pi.y - pj.y;
            double dz = pi.z - pj.z;
            if (per) dz = wrap_z(dz, half_bits, lz);
            const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
            if (bits(r2) == 0) continue;
            const double r = r2 * rsqrt_nr(r2);
            const double wi = hi3 * kw<KER>(r * hi, sn);
            const double wj = (hj * hj * hj) * kw<KER>(r * hj, sn);
            // M = wi C_i + wj C_j (symmetric), G = kg M r_ij
            const double m00 = fma(wi, ci.x, wj * cj.x), m01 = fma(wi, ci.y, wj * cj.y);
            const double m02 = fma(wi, ci.z, wj * cj.z), m11 = fma(wi, ci.w, wj * cj.w);
            const double m12 = fma(wi, ci2.x, wj * cj2.x), m22 = fma(wi, ci2.y, wj * cj2.y);
            const double gx = kg * fma(m02, dz, fma(m01, dy, m00 * dx));
            const double gy = kg * fma(m12, dz, fma(m11, dy, m01 * dx));
            const double gz = kg * fma(m22, dz, fma(m12, dy, m02 * dx));
            const double wx = vi.x - vj.x, wy = vi.y - vj.y, wz = vi.z - vj.z;
            const double vr = fma(wz, dz, fma(wy, dy, wx * dx));
            double Pi = 0.0;
            if (__double2hiint(vr) < 0) {
                const double hb = ti.w + tj.w;
                const double d1 = fma(eta2 * hb, hb, r2);
                const double rb = ti.x + tj.x;
                const double Rr = rcp_nr(d1 * rb);
                const double mu = ((hb * vr) * rb) * Rr;
                Pi = (mu * fma(beta, mu, -(ti.z + tj.z))) * (d1 * Rr);
                const long long ab = bits(mu) & 0x7fffffffffffffffLL;
                mum = ab > mum ? ab : mum;
            }
            const double gv = fma(gz, wz, fma(gy, wy, gx * wx));
            const double g = vj.w * ((ti.y + tj.y) + Pi);
            sx = fma(g, gx, sx);
            sy = fma(g, gy, sy);
            sz = fma(g, gz, sz);
            const double mgv = vj.w * gv;
            sp += mgv;
            sv = fma(mgv, Pi, sv);
        }
        const double mu_max = __longlong_as_double(mum);
        acc[i] = make_double4_32a(-sx, -sy, -sz, fma(ti.y, sp, 0.5 * sv));
        mumax[i] = mu_max;
        const double c = cint[i];
        const KParams& ke = B.kp[slot_inst(B, (int64_t)blockIdx.x * blockDim.x)];
        dtc = pi.w / (c + 1.2 * (ke.alpha * c + ke.beta * mu_max));
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

// One block per instance: dt[k] = cfl_k * min over the instance's block
// partials; time[k] += dt[k] when time is given. The force kernel ran with
// tpp lanes per particle, so a block covered kThreads / tpp particles.
__global__ void __launch_bounds__(kThreads)
k_dt_finish(const double* __restrict__ part, Batch B, int tpp, double* __restrict__ dt_out,
            double* __restrict__ time) {
    const int inst = blockIdx.x;
    const int64_t per_block = kThreads / tpp;
    const int64_t b0 = B.ioff[inst] / per_block;
    const int64_t nbk = (B.icnt[inst] + per_block - 1) / per_block;
    double m = CUDART_INF;
    for (int64_t k = threadIdx.x; k < nbk; k += blockDim.x) m = fmin(m, part[b0 + k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double sh[kThreads / 32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = sh[0];
        for (int w = 1; w < kThreads / 32; ++w) r = fmin(r, sh[w]);
        const double dt = B.kp[inst].cfl * r;
        dt_out[inst] = dt;
        if (time) time[inst] = time[inst] + dt;
    }
}

void launch_forces(sph_ctx* c, double* dt_out, double* time_inout, cudaStream_t s) {
    const int64_t n = c->n;
    const unsigned nb = (unsigned)((n + kThreads - 1) / kThreads);
    const int b = c->cur;
    const Batch B = batch_of(c);
    c->launches += 1;
    if (c->prec == PREC_MIXED)
        launch_forces_mx(c, s);
    else if (!native_pairs(c) && c->grad_kind == 1)
        launch_forces_iad_df(c, s);
    else if (!native_pairs(c))
        launch_forces_df(c, s);
    else if (n > 0 && c->grad_kind == 1) {
        c->launches += 3;
        const Rows R = rows_of(c);
        k_volume<<<nb, kThreads, 0, s>>>(n, B, c->velm[b], c->therm, c->vol);
        auto go = [&](auto iad_fn, auto forces_fn) {
            iad_fn<<<nb, kThreads, 0, s>>>(n, B, c->posh[b], c->vol, R, c->iad_a, c->iad_b);
            forces_fn<<<nb, kThreads, 0, s>>>(n, B, c->posh[b], c->velm[b], c->therm, c->kern,
                                              c->cint, c->iad_a, c->iad_b, R, c->acc, c->mumax,
                                              c->dt_part);
        };
        if (c->kern_kind == KER_WENDLAND) go(k_iad<KER_WENDLAND>, k_forces_iad<KER_WENDLAND>);
        else if (c->kern_kind == KER_SINC) go(k_iad<KER_SINC>, k_forces_iad<KER_SINC>);
        else go(k_iad<KER_M4>, k_forces_iad<KER_M4>);
    } else if (n > 0) {
        c->launches += 1;
        auto go = [&](auto forces_fn) {
            forces_fn<<<nb, kThreads, 0, s>>>(n, B, c->posh[b], c->velm[b], c->therm, c->kern,
                                              c->cint, rows_of(c), c->acc, c->mumax, c->dt_part);
        };
        if (c->kern_kind == KER_WENDLAND) go(k_forces<KER_WENDLAND>);
        else if (c->kern_kind == KER_SINC) go(k_forces<KER_SINC>);
        else go(k_forces<KER_M4>);
    }
    k_dt_finish<<<c->ninst, kThreads, 0, s>>>(c->dt_part, B, native_pairs(c) ? 1 : c->tpp,
                                              dt_out, time_inout);
}

// ------------------------------------------------------------ leapfrog
// Kick-drift (reading of Algorithm 1 step 6): v += dt a, u += dt du,
// x += dt v (new v); z wrapped into [-lz/2, lz/2) when periodic.
__global__ void __launch_bounds__(kThreads)
k_leapfrog(int64_t n, Batch B, const double* __restrict__ dtp, double4_32a* __restrict__ posh,
           double4_32a* __restrict__ velm, double* __restrict__ ue, const double4_32a* __restrict__ acc) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int inst = slot_inst(B, k);
    if (!slot_real(B, inst, k)) return;
    const KParams& kp = B.kp[inst];
    const double dt = dtp[inst];
    double4_32a p = posh[k];
    double4_32a v = velm[k];
    const double4_32a a = acc[k];
    v.x += dt * a.x;
    v.y += dt * a.y;
    v.z += dt * a.z;
    ue[k] += dt * a.w;
    p.x += dt * v.x;
    p.y += dt * v.y;
    p.z += dt * v.z;
    if (kp.periodic_z) {
        const double half = 0.5 * kp.lz;
        if (p.z >= half) p.z -= kp.lz;
        else if (p.z < -half) p.z += kp.lz;
    }
    posh[k] = p;
    velm[k] = v;
}

void launch_leapfrog(sph_ctx* c, const double* dt, cudaStream_t s) {
    const int64_t n = c->n;
    if (n == 0) return;
    const int b = c->cur;
    c->launches += 1;
    k_leapfrog<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        n, batch_of(c), dt, c->posh[b], c->velm[b], c->ue[b], c->acc);
}

// ------------------------------------------------------------ scatter
struct ScatterSrc {
    const int32_t* order;
    const double4_32a *posh, *velm, *therm, *acc;
    const double *ue, *pint, *cint, *mumax;
    const int32_t* nnb;
};

__global__ void __launch_bounds__(kThreads)
k_scatter(int64_t n, unsigned f, ScatterSrc S, sph_particles P) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t o = S.order[k];
    if (o < 0) return;  // empty slot
    if (f & (SC_POS | SC_H)) {
        const double4_32a p = S.posh[k];
        if (f & SC_POS) { P.x[o] = p.x; P.y[o] = p.y; P.z[o] = p.z; }
        if (f & SC_H) P.h[o] = p.w;
    }
    if (f & SC_VEL) {
        const double4_32a v = S.velm[k];
        P.vx[o] = v.x; P.vy[o] = v.y; P.vz[o] = v.z;
    }
    if (f & SC_U) P.u[o] = S.ue[k];
    if (f & SC_RHO) P.rho[o] = 2.0 * S.therm[k].x;
    if (f & SC_PC) {
        P.p[o] = S.pint[k];
        P.c[o] = S.cint[k];
    }
    if (f & SC_ACC) {
        const double4_32a a = S.acc[k];
        P.ax[o] = a.x; P.ay[o] = a.y; P.az[o] = a.z; P.du[o] = a.w;
    }
    if ((f & SC_MUMAX) && P.mumax) P.mumax[o] = S.mumax[k];
    if ((f & SC_NNB) && P.nnb) P.nnb[o] = S.nnb[k];
}

void launch_scatter(sph_ctx* c, const sph_particles* P, unsigned fields, cudaStream_t s) {
    const int64_t n = c->n;
    if (n == 0) return;
    const int b = c->cur;
    c->launches += 1;
    ScatterSrc S{c->order[b], c->posh[b], c->velm[b], c->therm, c->acc, c->ue[b], c->pint,
                 c->cint, c->mumax, c->nnb};
    k_scatter<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(n, fields, S, *P);
}

}  // namespace sph
