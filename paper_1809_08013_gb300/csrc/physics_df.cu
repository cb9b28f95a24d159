// physics_df.cu -- density and forces (Algorithm 1 step 3) with the pair
// arithmetic in double-float on the FP32 pipes.
//
// Same definitions as physics.cu (cubic-spline gather density; momentum and
// energy with Monaghan viscosity over S_i; time-step candidate). GB300 issues
// FP64 at 1/64 of the FP32 rate, so the pair loops keep off the FP64 pipe
// almost entirely. Position differences come from the exact fixed-point
// chunks of each particle's coordinates (dfl::to_fx, written once per step):
// three exact FP32 subtractions and one double-float sum per component. The
// velocities are float pairs (written once per step), and their differences
// double-float subtractions. Everything else -- r^2, 1/r,
// the kernel polynomials, the viscosity, the sums -- runs in ~48-bit
// double-float (df.cuh). Per-particle inputs (1/h, 1/h^4, p/rho^2, h/2, rho/2,
// alpha c/2, m) are converted once per step into float packs read for every
// neighbour. Everything the pair loops hold is in the instance's pair units
// (Grid::uL, uM, uV: powers of two near the mean h, the largest mass and a
// velocity scale), so the float exponent range holds it whatever units the
// caller uses; the sums are taken back to the caller's units exactly, by
// powers of two, when they are written out.
#include <math_constants.h>

#include "df.cuh"
#include "sph_internal.cuh"

namespace sph {

using dfl::df;

namespace {

// pi h^3 W as a function of q >= 0 (cubic spline). In the outer piece,
// 1 <= q.hi <= 2, 2 - q.hi is exact (Sterbenz) and a multiple of ulp(q.hi),
// so Fast2Sum with -q.lo gives 2 - q exactly, normalised.
__device__ __forceinline__ df w_shape(df q) {
    const df q2 = dfl::sqr(q);
    const df a = dfl::addf(dfl::mulf(q, 0.75f), -1.5f);
    const df win = dfl::addf(dfl::mul(q2, a), 1.0f);  // 1 - 1.5 q^2 + 0.75 q^3
    const df t = dfl::fast_two_sum(__fsub_rn(2.0f, q.hi), -q.lo);
    const df wout = dfl::scale2(dfl::mul(dfl::sqr(t), t), 0.25f);  // (2 - q)^3 / 4
    const df zero = {0.0f, 0.0f};
    return q.hi < 1.0f ? win : (q.hi < 2.0f ? wout : zero);
}

// pi h^4 dW/dr as a function of q >= 0. Both pieces are one product
// (q + a)(b q + c) with the coefficients of q's piece:
//   q < 1:      q (2.25 q - 3)                        (a, b, c) = (0, 2.25, -3)
//   1 <= q < 2: (q - 2)(1.5 - 0.75 q) = -0.75 (2 - q)^2    (a, b, c) = (-2, -0.75, 1.5)
// q + a is exact: for q < 1 it is q; for 1 <= q.hi <= 2, q.hi - 2 is exact
// (Sterbenz) and a multiple of ulp(q.hi), so Fast2Sum with q.lo gives q - 2
// exactly, normalised. Near q = 2 both factors are small with an absolute
// error ~2^-47, so the product's absolute error stays ~2^-47 |2 - q|.
__device__ __forceinline__ df dw_shape(df q) {
    const bool in = q.hi < 1.0f;
    const df u = in ? q : dfl::fast_two_sum(__fsub_rn(q.hi, 2.0f), q.lo);
    const df v = dfl::addf(dfl::mulf(q, in ? 2.25f : -0.75f), in ? -3.0f : 1.5f);
    const df f = dfl::mul(u, v);
    const df zero = {0.0f, 0.0f};
    return q.hi < 2.0f ? f : zero;
}

// ---- Sinc kernel in double-float. With x = pi q / 2 <= pi and y = x^2,
//   S(x) = sin x / x = sum_k (-1)^k y^k / (2k+1)!           (k = 0..14)
//   S'(x) = x Q(y),  Q(y) = sum_k (-1)^k 2k y^(k-1) / (2k+1)!  (k = 1..14)
// (the Taylor series of sin x / x and its term-by-term derivative; the
// first omitted terms are below 3e-19 at x = pi, and neither form cancels at
// small x). Coefficients as float pairs, computed at compile time.
struct F2 {
    float hi, lo;
};

constexpr F2 split_f2(double v) {
    return F2{static_cast<float>(v), static_cast<float>(v - static_cast<double>(static_cast<float>(v)))};
}

constexpr int kSincTerms = 15;

struct SincTab {
    F2 p[kSincTerms];
    F2 q[kSincTerms - 1];
};

constexpr SincTab make_sinc_tab() {
    SincTab t{};
    double inv = 1.0;  // 1 / (2k+1)!
    for (int k = 0; k < kSincTerms; ++k) {
        if (k > 0) inv = inv / ((2.0 * k) * (2.0 * k + 1.0));
        const double sgn = (k % 2) ? -1.0 : 1.0;
        t.p[k] = split_f2(sgn * inv);
        if (k > 0) t.q[k - 1] = split_f2(sgn * 2.0 * k * inv);
    }
    return t;
}

__constant__ SincTab kSinc = make_sinc_tab();
constexpr F2 kHalfPi = split_f2(0.5 * kPi);

template <int M>
__device__ __forceinline__ df horner(const F2* c, df y) {
    df acc = {c[M - 1].hi, c[M - 1].lo};
#pragma unroll
    for (int k = M - 2; k >= 0; --k) acc = dfl::add(dfl::mul(acc, y), df{c[k].hi, c[k].lo});
    return acc;
}

__device__ __forceinline__ df ipow_df(df v, int k) {
    df r = {1.0f, 0.0f};
    for (int e = 0; e < k; ++e) r = dfl::mul(r, v);
    return r;
}

// Kernel shapes by kind (sn: the sinc exponent), zero from q = 2 on; the
// normalisations (wnorm, dnorm) are applied by the caller.
//   Wendland C2 (Table 1): g = (1 - q/2)^4 (1 + 2q), f = -q (1 - q/2)^3;
//   sinc: g = S^n, f = n S^(n-1) S'(x) (dW/dr takes pi/2 into dnorm).
template <int KER>
__device__ __forceinline__ df w_shape_k(df q, int sn) {
    if (KER == KER_M4) return w_shape(q);
    const df zero = {0.0f, 0.0f};
    if (KER == KER_SINC) {
        if (!(q.hi < 2.0f)) return zero;
        const df x = dfl::mul(q, df{kHalfPi.hi, kHalfPi.lo});
        return ipow_df(horner<kSincTerms>(kSinc.p, dfl::sqr(x)), sn);
    }
    const df t = dfl::addf(dfl::scale2(dfl::neg(q), 0.5f), 1.0f);
    const df t2 = dfl::sqr(t);
    const df g = dfl::mul(dfl::sqr(t2), dfl::addf(dfl::scale2(q, 2.0f), 1.0f));
    return q.hi < 2.0f ? g : zero;
}

template <int KER>
__device__ __forceinline__ df dw_shape_k(df q, int sn) {
    if (KER == KER_M4) return dw_shape(q);
    const df zero = {0.0f, 0.0f};
    if (KER == KER_SINC) {
        if (!(q.hi < 2.0f)) return zero;
        const df x = dfl::mul(q, df{kHalfPi.hi, kHalfPi.lo});
        const df y = dfl::sqr(x);
        const df S = horner<kSincTerms>(kSinc.p, y);
        const df dS = dfl::mul(x, horner<kSincTerms - 1>(kSinc.q, y));
        return dfl::mul(dfl::mulf(ipow_df(S, sn - 1), (float)sn), dS);
    }
    const df t = dfl::addf(dfl::scale2(dfl::neg(q), 0.5f), 1.0f);
    const df f = dfl::neg(dfl::mul(q, dfl::mul(dfl::sqr(t), t)));
    return q.hi < 2.0f ? f : zero;
}

// Minimum image along z on the chunk differences (dfl::to_fx): when |dz| >
// lz/2 (decided on the leading chunk, which is within ~2^-18 |x|max of dz and
// so unambiguous for any pair of a row), subtract sign(dz) lz chunk by chunk;
// each chunk difference stays exact.
__device__ __forceinline__ void wrap_fx(float& z2, float& z1, float& z0, float hlz, float L2,
                                        float L1, float L0) {
    if (fabsf(z2) > hlz) {
        const float sg = copysignf(1.0f, z2);
        z2 = __fsub_rn(z2, sg * L2);
        z1 = __fsub_rn(z1, sg * L1);
        z0 = __fsub_rn(z0, sg * L0);
    }
}

__device__ __forceinline__ void eos_d(const KParams& kp, double rho, double u, double& p, double& c) {
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

// ------------------------------------------------------------ density
// T lanes per particle: lane s of particle i takes row entries s, s + T, ...
// KER: the M4 spline, the Wendland C2 or the sinc kernel.
// OUTER: the kernel also decides, for each j of N_i, whether i is in N_j --
// r_ij^2 < (2 h_j)^2 by the defining FP64 test -- and records the entries
// where it is not as bits of omask (bit e for gather entry e of row i);
// k_append_outer then appends those i to the outer parts of the rows j. The
// pair's double-float r^2 is within ~2^-45 of the defining FP64 value and
// (2 h_j)^2 is packed as a float (within 2^-24), so r^2 below / above it by
// more than 2^-20 decides; the band between takes the FP64 test itself. The
// sets are the exact ones, as built by k_outer.
template <bool FUSE, int T, int KER, bool OUTER>
__global__ void __launch_bounds__(kThreads)
k_density_df(int64_t n, Batch B, const double4_32a* __restrict__ posh,
             const float4* __restrict__ xpk, const double* __restrict__ ue,
             Rows R, double4_32a* __restrict__ therm,
             double2* __restrict__ kern, float4* __restrict__ dpk, double* __restrict__ pint,
             double* __restrict__ cint, unsigned* status,
             unsigned long long* __restrict__ omask) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / T;
    const int sub = (int)(threadIdx.x % T);
    const int inst = slot_inst(B, ((int64_t)blockIdx.x * blockDim.x) / T);
    const int32_t* ent = nullptr;
    int len = 0;
    const bool act = i < n && slot_real(B, inst, i) && row_of(R, n, i, true, ent, len);
    if (T == 1 && !act) return;
    const KParams& kp = B.kp[inst];
    double4_32a pi = make_double4_32a(0.0, 0.0, 0.0, 1.0);
    df acc = {0.0f, 0.0f};
    unsigned long long om0 = 0ull, om1 = 0ull;  // OUTER: bits of the gather entries
    if (act) {
    pi = posh[i];
    const Grid& g = B.grid[inst];
    const double hinv = 1.0 / pi.w;
    const int sn = kp.sinc_n;
    const df Hi = dfl::from_double_fp64(hinv * p2d(g.uL));  // 1/h in the length unit
    const bool per = kp.periodic_z != 0;
    const float hlz = g.hlzc, L2 = g.lzc[0], L1 = g.lzc[1], L0 = g.lzc[2];
    const float4 I0 = xpk[3 * i], I1 = xpk[3 * i + 1], I2 = xpk[3 * i + 2];
    if (sub == 0) acc = df{I0.w, I1.w};  // self term m_i W(0, h_i): shape 1
    // rows read from the CSR (a gather set overflowed) are complete already
    const bool append = OUTER && !(R.status[2] & IF_SLAB_OVF);
    for (int e = sub; e < len; e += T) {
        const int j = __ldg(&ent[e]);
        const float4 J0 = __ldg(&xpk[3 * j]), J1 = __ldg(&xpk[3 * j + 1]);
        const float4 J2 = __ldg(&xpk[3 * j + 2]);
        const df mj = {J0.w, J1.w};
        float z2 = __fsub_rn(I0.z, J0.z), z1 = __fsub_rn(I1.z, J1.z), z0 = __fsub_rn(I2.z, J2.z);
        if (per) wrap_fx(z2, z1, z0, hlz, L2, L1, L0);
        const df X = dfl::fx_sum(__fsub_rn(I0.x, J0.x), __fsub_rn(I1.x, J1.x), __fsub_rn(I2.x, J2.x));
        const df Y = dfl::fx_sum(__fsub_rn(I0.y, J0.y), __fsub_rn(I1.y, J1.y), __fsub_rn(I2.y, J2.y));
        const df Z = dfl::fx_sum(z2, z1, z0);
        const df r2 = dfl::add(dfl::add_same(dfl::sqr(X), dfl::sqr(Y)), dfl::sqr(Z));
        df w = {1.0f, 0.0f};  // coincident particles: q = 0
        if (r2.hi > 0.0f) {
            const df q = dfl::mul(dfl::mul(r2, dfl::rsqrt(r2)), Hi);
            w = w_shape_k<KER>(q, sn);
        }
        acc = dfl::add(acc, dfl::mul(mj, w));
        if (append) {
            const float tj = J2.w;  // (2 h_j)^2 in the length unit (NaN: exact test only)
            bool in_j;
            if (r2.hi < tj * 0.99999905f) {
                in_j = true;
            } else if (r2.hi > tj * 1.00000095f) {
                in_j = false;
            } else {
                const double4_32a pj = posh[j];
                const double Rj = 2.0 * pj.w;
                in_j = exact_r2_def(pi, pj, per, kp.lz) < __dmul_rn(Rj, Rj);
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
    if (OUTER && !act) return;
    if (OUTER) {
        omask[2 * i] = om0;
        omask[2 * i + 1] = om1;
    }
    const Grid& g = B.grid[inst];
    const double hinv = 1.0 / pi.w;
    const double sigma = hinv * hinv * hinv * (KER == KER_M4 ? kInvPi : kp.wnorm);
    const double rho = dfl::to_double(acc) * p2d(g.uM) * sigma;  // masses back from the mass unit
    if (FUSE) {
        double p, c;
        eos_d(kp, rho, ue[i], p, c);
        const double A = p / (rho * rho);
        // (the FP64-pipe kernels' kern pack is not needed at this precision)
        therm[i] = make_double4_32a(0.5 * rho, A, 0.5 * kp.alpha * c, 0.5 * pi.w);
        dfl::write_pack(dpk, i, hinv, A, pi.w, rho, kp.alpha, c, dfl::pair_units(g.uL, g.uM, g.uV),
                        status, ST_RANGE);
        pint[i] = p;
        cint[i] = c;
    } else {
        therm[i].x = 0.5 * rho;
    }
}

template <bool FUSE, int T, bool OUTER>
static void density_df_t(sph_ctx* c, cudaStream_t s) {
    const int64_t n = c->n;
    const unsigned nb = (unsigned)((n * T + kThreads - 1) / kThreads);
    const int b = c->cur;
    const Rows R = OUTER ? rows_gather(c) : rows_of(c);
    auto go = [&](auto kernel_fn) {
        kernel_fn<<<nb, kThreads, 0, s>>>(n, batch_of(c), c->posh[b], c->xpk, c->ue[b], R,
                                          c->therm, c->kern, c->dpk, c->pint, c->cint, c->status,
                                          c->omask);
    };
    if (c->kern_kind == KER_WENDLAND) go(k_density_df<FUSE, T, KER_WENDLAND, OUTER>);
    else if (c->kern_kind == KER_SINC) go(k_density_df<FUSE, T, KER_SINC, OUTER>);
    else go(k_density_df<FUSE, T, KER_M4, OUTER>);
}

template <bool FUSE, bool OUTER>
static void density_df_f(sph_ctx* c, cudaStream_t s) {
    switch (c->tpp) {
        case 2: density_df_t<FUSE, 2, OUTER>(c, s); break;
        case 4: density_df_t<FUSE, 4, OUTER>(c, s); break;
        case 8: density_df_t<FUSE, 8, OUTER>(c, s); break;
        default: density_df_t<FUSE, 1, OUTER>(c, s); break;
    }
}

void launch_density_df(sph_ctx* c, bool fuse_eos, cudaStream_t s, bool outer) {
    if (c->n == 0) return;
    c->launches += 1;
    if (fuse_eos && outer) density_df_f<true, true>(c, s);
    else if (fuse_eos) density_df_f<true, false>(c, s);
    else density_df_f<false, false>(c, s);
}

// ------------------------------------------------------------ forces + dt
// Definitions as in physics.cu; algebra: Fbar = (0.5/pi)(f(q_i)/h_i^4 +
// f(q_j)/h_j^4)/r, one shared reciprocal R = 1/((r^2 + eta2 hb^2) rhob) for the
// viscosity, mu = hb v.r rhob R, 1/rhob = (r^2 + eta2 hb^2) R. Every sum is
// linear in Fbar, so its constant factor (0.5/pi, or dnorm/2) is applied once
// per particle, in FP64, when the sums are written out.
template <int T, int KER>
__global__ void __launch_bounds__(kThreads, KER == KER_SINC ? 2 : 3)
k_forces_df(int64_t n, Batch B, const double4_32a* __restrict__ posh,
            const float4* __restrict__ vpa, const float2* __restrict__ vpb,
            const float4* __restrict__ dpk,
            const float4* __restrict__ xpk, const double* __restrict__ cint,
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
    df mumx = {0.f, 0.f};
    if (act) {
        const KParams& kp = B.kp[inst];
        const float4 va = vpa[i];
        const float2 vb = vpb[i];
        const df VXi = {va.x, va.y}, VYi = {va.z, va.w}, VZi = {vb.x, vb.y};
        const float4 I0 = xpk[3 * i], I1 = xpk[3 * i + 1], I2 = xpk[3 * i + 2];
        const float4 a0 = dpk[3 * i], a1 = dpk[3 * i + 1], a2 = dpk[3 * i + 2];
        const df Hi = {a0.x, a0.y}, Ki = {a0.z, a0.w}, Ai = {a1.x, a1.y}, hhi = {a1.z, a1.w};
        const df rhi = {a2.x, a2.y}, cai = {a2.z, a2.w};
        const Grid& gr = B.grid[inst];
        const bool per = kp.periodic_z != 0;
        const float hlz = gr.hlzc, L2 = gr.lzc[0], L1 = gr.lzc[1], L0 = gr.lzc[2];
        const int sn = kp.sinc_n;
        const df eta2 = dfl::from_double_fp64(kp.eta2);
        const df betad = dfl::from_double_fp64(kp.beta);
        for (int e = sub; e < len; e += T) {
            const int j = __ldg(&ent[e]);
            const float4 J0 = __ldg(&xpk[3 * j]), J1 = __ldg(&xpk[3 * j + 1]);
            const float4 J2 = __ldg(&xpk[3 * j + 2]);
            const float4 wa = __ldg(&vpa[j]);
            const float2 wb = __ldg(&vpb[j]);
            const float4 b0 = __ldg(&dpk[3 * j]), b1 = __ldg(&dpk[3 * j + 1]);
            const float4 b2 = __ldg(&dpk[3 * j + 2]);
            float z2 = __fsub_rn(I0.z, J0.z), z1 = __fsub_rn(I1.z, J1.z), z0 = __fsub_rn(I2.z, J2.z);
            if (per) wrap_fx(z2, z1, z0, hlz, L2, L1, L0);
            const df X = dfl::fx_sum(__fsub_rn(I0.x, J0.x), __fsub_rn(I1.x, J1.x), __fsub_rn(I2.x, J2.x));
            const df Y = dfl::fx_sum(__fsub_rn(I0.y, J0.y), __fsub_rn(I1.y, J1.y), __fsub_rn(I2.y, J2.y));
            const df Z = dfl::fx_sum(z2, z1, z0);
            const df r2 = dfl::add(dfl::add_same(dfl::sqr(X), dfl::sqr(Y)), dfl::sqr(Z));
            if (!(r2.hi > 0.0f)) continue;  // coincident particles exert no force
            const df rinv = dfl::rsqrt(r2);
            const df r = dfl::mul(r2, rinv);
            const df fa = dw_shape_k<KER>(dfl::mul(r, Hi), sn);
            const df fb = dw_shape_k<KER>(dfl::mul(r, df{b0.x, b0.y}), sn);
            const df Fb = dfl::mul(dfl::add(dfl::mul(Ki, fa), dfl::mul(df{b0.z, b0.w}, fb)), rinv);
            const df WX = dfl::sub(VXi, df{wa.x, wa.y}), WY = dfl::sub(VYi, df{wa.z, wa.w});
            const df WZ = dfl::sub(VZi, df{wb.x, wb.y});
            const df vr = dfl::add(dfl::add(dfl::mul(WX, X), dfl::mul(WY, Y)), dfl::mul(WZ, Z));
            df Pi = {0.f, 0.f};
            if (vr.hi < 0.0f) {
                const df hb = dfl::add(hhi, df{b1.z, b1.w});
                const df d1 = dfl::add(r2, dfl::mul(dfl::mul(eta2, hb), hb));
                const df rb = dfl::add(rhi, df{b2.x, b2.y});
                const df R = dfl::rcp(dfl::mul(d1, rb));
                const df mu = dfl::mul(dfl::mul(dfl::mul(hb, vr), rb), R);
                const df cb = dfl::add(cai, df{b2.z, b2.w});
                const df t = dfl::add(dfl::mul(betad, mu), dfl::neg(cb));
                Pi = dfl::mul(dfl::mul(mu, t), dfl::mul(d1, R));
                if (-mu.hi > mumx.hi) mumx = dfl::neg(mu);
            }
            const df mF = dfl::mul(df{J0.w, J1.w}, Fb);
            const df g = dfl::mul(mF, dfl::add(dfl::add(Ai, df{b1.x, b1.y}), Pi));
            sx = dfl::add(sx, dfl::mul(g, X));
            sy = dfl::add(sy, dfl::mul(g, Y));
            sz = dfl::add(sz, dfl::mul(g, Z));
            const df mFv = dfl::mul(mF, vr);
            sp = dfl::add(sp, mFv);
            sv = dfl::add(sv, dfl::mul(mFv, Pi));
        }
    }
    if (T > 1) {
        sx = dfl::lane_sum<T>(sx);
        sy = dfl::lane_sum<T>(sy);
        sz = dfl::lane_sum<T>(sz);
        sp = dfl::lane_sum<T>(sp);
        sv = dfl::lane_sum<T>(sv);
#pragma unroll
        for (int o = 1; o < T; o <<= 1) {  // largest (hi, lo): a total order
            const df w = {__shfl_xor_sync(0xffffffffu, mumx.hi, o),
                          __shfl_xor_sync(0xffffffffu, mumx.lo, o)};
            if (w.hi > mumx.hi || (w.hi == mumx.hi && w.lo > mumx.lo)) mumx = w;
        }
    }
    if (act && sub == 0) {
        // back to the caller's units: a ~ V^2 / L, du ~ V^3 / L, mu ~ V; and the
        // constant factor of Fbar
        const int ins = slot_inst(B, ((int64_t)blockIdx.x * blockDim.x) / T);
        const Grid& gu = B.grid[ins];
        const double cF = 0.5 * (KER == KER_M4 ? kInvPi : B.kp[ins].dnorm);
        const double sa = p2d(2 * gu.uV - gu.uL) * cF, su = p2d(3 * gu.uV - gu.uL) * cF;
        const double Aid = (double)dpk[3 * i + 1].x + (double)dpk[3 * i + 1].y;
        acc[i] = make_double4_32a(-dfl::to_double(sx) * sa, -dfl::to_double(sy) * sa,
                                  -dfl::to_double(sz) * sa,
                                  fma(Aid, dfl::to_double(sp), 0.5 * dfl::to_double(sv)) * su);
        const double mu_max = dfl::to_double(mumx) * p2d(gu.uV);
        mumax[i] = mu_max;
        const double ci = cint[i];
        // parameters re-read here rather than kept in registers across the loop
        const KParams& ke = B.kp[slot_inst(B, ((int64_t)blockIdx.x * blockDim.x) / T)];
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

template <int T>
static void forces_df_t(sph_ctx* c, cudaStream_t s) {
    const int64_t n = c->n;
    const unsigned nb = (unsigned)((n * T + kThreads - 1) / kThreads);
    const int b = c->cur;
    if (c->kern_kind == KER_WENDLAND)
        k_forces_df<T, KER_WENDLAND><<<nb, kThreads, 0, s>>>(
            n, batch_of(c), c->posh[b], c->vpa, c->vpb, c->dpk, c->xpk, c->cint, rows_of(c), c->acc,
            c->mumax, c->dt_part);
    else if (c->kern_kind == KER_SINC)
        k_forces_df<T, KER_SINC><<<nb, kThreads, 0, s>>>(
            n, batch_of(c), c->posh[b], c->vpa, c->vpb, c->dpk, c->xpk, c->cint, rows_of(c), c->acc,
            c->mumax, c->dt_part);
    else
        k_forces_df<T, KER_M4><<<nb, kThreads, 0, s>>>(
            n, batch_of(c), c->posh[b], c->vpa, c->vpb, c->dpk, c->xpk, c->cint, rows_of(c), c->acc,
            c->mumax, c->dt_part);
}

void launch_forces_df(sph_ctx* c, cudaStream_t s) {
    if (c->n == 0) return;
    c->launches += 1;
    switch (c->tpp) {
        case 2: forces_df_t<2>(c, s); break;
        case 4: forces_df_t<4>(c, s); break;
        case 8: forces_df_t<8>(c, s); break;
        default: forces_df_t<1>(c, s); break;
    }
}

// ------------------------------------------------------------ IAD (Table 1)
// The double-float IAD path (M4 and Wendland C2; definitions as in physics.cu).
// Volume elements V = m / rho as float pairs, once per particle.
__global__ void __launch_bounds__(kThreads)
k_volume_df(int64_t n, Batch B, const double4_32a* __restrict__ velm,
            const double4_32a* __restrict__ therm, float2* __restrict__ vdf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int inst = slot_inst(B, i);
    if (!slot_real(B, inst, i)) return;
    // m / rho (a volume, L^3) in the length unit
    const df v = dfl::from_double_fp64(velm[i].w / (2.0 * therm[i].x) * p2d(-3 * B.grid[inst].uL));
    vdf[i] = make_float2(v.hi, v.lo);
}

// tau_i = sum_{j in N_i} V_j W(r_ij, h_i) (r_j - r_i)(r_j - r_i)^T summed in
// double-float (T lanes per particle, fixed butterfly), then scaled, inverted
// in FP64 by the adjugate (C_i = 0 if singular) and stored as float pairs:
//   cpk[3i] = (C00, C01), cpk[3i+1] = (C02, C11), cpk[3i+2] = (C12, C22).
template <int T, int KER>
__global__ void __launch_bounds__(kThreads)
k_iad_df(int64_t n, Batch B, const double4_32a* __restrict__ posh,
         const float4* __restrict__ xpk, const float2* __restrict__ vdf, Rows R,
         float4* __restrict__ cpk) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / T;
    const int sub = (int)(threadIdx.x % T);
    const int inst = slot_inst(B, ((int64_t)blockIdx.x * blockDim.x) / T);
    const int32_t* ent = nullptr;
    int len = 0;
    const bool act = i < n && slot_real(B, inst, i) && row_of(R, n, i, true, ent, len);
    if (T == 1 && !act) return;
    df t[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) t[k] = df{0.0f, 0.0f};
    double hinv = 1.0;  // in the length unit: tau and C then come out in it too
    if (act) {
        const Grid& g = B.grid[inst];
        hinv = 1.0 / posh[i].w * p2d(g.uL);
        const int sn = B.kp[inst].sinc_n;
        const df Hi = dfl::from_double_fp64(hinv);
        const bool per = B.kp[inst].periodic_z != 0;
        const float hlz = g.hlzc, L2 = g.lzc[0], L1 = g.lzc[1], L0 = g.lzc[2];
        const float4 I0 = xpk[3 * i], I1 = xpk[3 * i + 1], I2 = xpk[3 * i + 2];
        for (int e = sub; e < len; e += T) {
            const int j = __ldg(&ent[e]);
            const float4 J0 = __ldg(&xpk[3 * j]), J1 = __ldg(&xpk[3 * j + 1]);
            const float4 J2 = __ldg(&xpk[3 * j + 2]);
            const float2 vj = __ldg(&vdf[j]);
            float z2 = __fsub_rn(I0.z, J0.z), z1 = __fsub_rn(I1.z, J1.z), z0 = __fsub_rn(I2.z, J2.z);
            if (per) wrap_fx(z2, z1, z0, hlz, L2, L1, L0);
            const df X = dfl::fx_sum(__fsub_rn(I0.x, J0.x), __fsub_rn(I1.x, J1.x), __fsub_rn(I2.x, J2.x));
            const df Y = dfl::fx_sum(__fsub_rn(I0.y, J0.y), __fsub_rn(I1.y, J1.y), __fsub_rn(I2.y, J2.y));
            const df Z = dfl::fx_sum(z2, z1, z0);
            const df r2 = dfl::add(dfl::add_same(dfl::sqr(X), dfl::sqr(Y)), dfl::sqr(Z));
            if (!(r2.hi > 0.0f)) continue;  // r = 0 adds nothing to tau
            const df q = dfl::mul(dfl::mul(r2, dfl::rsqrt(r2)), Hi);
            const df w = dfl::mul(df{vj.x, vj.y}, w_shape_k<KER>(q, sn));
            const df wx = dfl::mul(w, X), wy = dfl::mul(w, Y);
            t[0] = dfl::add(t[0], dfl::mul(wx, X));
            t[1] = dfl::add(t[1], dfl::mul(wx, Y));
            t[2] = dfl::add(t[2], dfl::mul(wx, Z));
            t[3] = dfl::add(t[3], dfl::mul(wy, Y));
            t[4] = dfl::add(t[4], dfl::mul(wy, Z));
            t[5] = dfl::add(t[5], dfl::mul(dfl::mul(w, Z), Z));
        }
    }
    if (T > 1) {
#pragma unroll
        for (int k = 0; k < 6; ++k) t[k] = dfl::lane_sum<T>(t[k]);
        if (!act || sub != 0) return;
    }
    const double sg = hinv * hinv * hinv * (KER == KER_M4 ? kInvPi : B.kp[inst].wnorm);
    double a[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) a[k] = dfl::to_double(t[k]) * sg;
    const double c00 = a[3] * a[5] - a[4] * a[4], c01 = a[2] * a[4] - a[1] * a[5];
    const double c02 = a[1] * a[4] - a[2] * a[3], c11 = a[0] * a[5] - a[2] * a[2];
    const double c12 = a[1] * a[2] - a[0] * a[4], c22 = a[0] * a[3] - a[1] * a[1];
    const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    const double id = det == 0.0 ? 0.0 : 1.0 / det;
    const df C[6] = {dfl::from_double_fp64(c00 * id), dfl::from_double_fp64(c01 * id),
                     dfl::from_double_fp64(c02 * id), dfl::from_double_fp64(c11 * id),
                     dfl::from_double_fp64(c12 * id), dfl::from_double_fp64(c22 * id)};
    cpk[3 * i + 0] = make_float4(C[0].hi, C[0].lo, C[1].hi, C[1].lo);
    cpk[3 * i + 1] = make_float4(C[2].hi, C[2].lo, C[3].hi, C[3].lo);
    cpk[3 * i + 2] = make_float4(C[4].hi, C[4].lo, C[5].hi, C[5].lo);
}

// symmetric 3x3 (in the cpk order) times a vector, in double-float
__device__ __forceinline__ void symv_df(const df* M, const df& x, const df& y, const df& z, df& ox,
                                        df& oy, df& oz) {
    ox = dfl::add(dfl::add(dfl::mul(M[0], x), dfl::mul(M[1], y)), dfl::mul(M[2], z));
    oy = dfl::add(dfl::add(dfl::mul(M[1], x), dfl::mul(M[3], y)), dfl::mul(M[4], z));
    oz = dfl::add(dfl::add(dfl::mul(M[2], x), dfl::mul(M[4], y)), dfl::mul(M[5], z));
}

// Forces with IAD gradients: as k_forces_df with F r_ij replaced by
// G_ij = -(wnorm / 2) (h_i^-3 g(q_i) C_i + h_j^-3 g(q_j) C_j) r_ij.
template <int T, int KER>
__global__ void __launch_bounds__(kThreads, 2)
k_forces_iad_df(int64_t n, Batch B, const double4_32a* __restrict__ posh,
                const float4* __restrict__ vpa, const float2* __restrict__ vpb,
                const float4* __restrict__ dpk,
                const float4* __restrict__ xpk, const float4* __restrict__ cpk,
                const double* __restrict__ cint, Rows R, double4_32a* __restrict__ acc,
                double* __restrict__ mumax, double* __restrict__ dt_part) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / T;
    const int sub = (int)(threadIdx.x % T);
    const int inst = slot_inst(B, ((int64_t)blockIdx.x * blockDim.x) / T);
    const int32_t* ent = nullptr;
    int len = 0;
    const bool act = i < n && slot_real(B, inst, i) && row_of(R, n, i, false, ent, len);
    double dtc = CUDART_INF;
    df sx = {0.f, 0.f}, sy = {0.f, 0.f}, sz = {0.f, 0.f}, sp = {0.f, 0.f}, sv = {0.f, 0.f};
    df mumx = {0.f, 0.f};
    if (act) {
        const KParams& kp = B.kp[inst];
        const float4 va = vpa[i];
        const float2 vb = vpb[i];
        const df VXi = {va.x, va.y}, VYi = {va.z, va.w}, VZi = {vb.x, vb.y};
        const float4 I0 = xpk[3 * i], I1 = xpk[3 * i + 1], I2 = xpk[3 * i + 2];
        const float4 a0 = dpk[3 * i], a1 = dpk[3 * i + 1], a2 = dpk[3 * i + 2];
        const df Hi = {a0.x, a0.y}, Ai = {a1.x, a1.y}, hhi = {a1.z, a1.w};
        const df rhi = {a2.x, a2.y}, cai = {a2.z, a2.w};
        const df Hi3 = dfl::mul(Hi, dfl::sqr(Hi));
        const float4 c0 = cpk[3 * i], c1 = cpk[3 * i + 1], c2 = cpk[3 * i + 2];
        const df Ci[6] = {{c0.x, c0.y}, {c0.z, c0.w}, {c1.x, c1.y},
                          {c1.z, c1.w}, {c2.x, c2.y}, {c2.z, c2.w}};
        const Grid& gr = B.grid[inst];
        const bool per = kp.periodic_z != 0;
        const float hlz = gr.hlzc, L2 = gr.lzc[0], L1 = gr.lzc[1], L0 = gr.lzc[2];
        const int sn = kp.sinc_n;
        const df kg = dfl::from_double_fp64(-0.5 * (KER == KER_M4 ? kInvPi : kp.wnorm));
        const df eta2 = dfl::from_double_fp64(kp.eta2);
        const df betad = dfl::from_double_fp64(kp.beta);
        for (int e = sub; e < len; e += T) {
            const int j = __ldg(&ent[e]);
            const float4 J0 = __ldg(&xpk[3 * j]), J1 = __ldg(&xpk[3 * j + 1]);
            const float4 J2 = __ldg(&xpk[3 * j + 2]);
            const float4 wa = __ldg(&vpa[j]);
            const float2 wb = __ldg(&vpb[j]);
            const float4 b0 = __ldg(&dpk[3 * j]), b1 = __ldg(&dpk[3 * j + 1]);
            const float4 b2 = __ldg(&dpk[3 * j + 2]);
            float z2 = __fsub_rn(I0.z, J0.z), z1 = __fsub_rn(I1.z, J1.z), z0 = __fsub_rn(I2.z, J2.z);
            if (per) wrap_fx(z2, z1, z0, hlz, L2, L1, L0);
            const df X = dfl::fx_sum(__fsub_rn(I0.x, J0.x), __fsub_rn(I1.x, J1.x), __fsub_rn(I2.x, J2.x));
            const df Y = dfl::fx_sum(__fsub_rn(I0.y, J0.y), __fsub_rn(I1.y, J1.y), __fsub_rn(I2.y, J2.y));
            const df Z = dfl::fx_sum(z2, z1, z0);
            const df r2 = dfl::add(dfl::add_same(dfl::sqr(X), dfl::sqr(Y)), dfl::sqr(Z));
            if (!(r2.hi > 0.0f)) continue;  // coincident particles exert no force
            const df r = dfl::mul(r2, dfl::rsqrt(r2));
            const df Hj = {b0.x, b0.y};
            const df wi = dfl::mul(Hi3, w_shape_k<KER>(dfl::mul(r, Hi), sn));
            const df wj = dfl::mul(dfl::mul(Hj, dfl::sqr(Hj)), w_shape_k<KER>(dfl::mul(r, Hj), sn));
            df M[6];
            {
                const float4 d0 = __ldg(&cpk[3 * j]), d1 = __ldg(&cpk[3 * j + 1]);
                const float4 d2 = __ldg(&cpk[3 * j + 2]);
                const df Cj[6] = {{d0.x, d0.y}, {d0.z, d0.w}, {d1.x, d1.y},
                                  {d1.z, d1.w}, {d2.x, d2.y}, {d2.z, d2.w}};
#pragma unroll
                for (int k = 0; k < 6; ++k) M[k] = dfl::add(dfl::mul(wi, Ci[k]), dfl::mul(wj, Cj[k]));
            }
            df Gx, Gy, Gz;
            symv_df(M, X, Y, Z, Gx, Gy, Gz);
            Gx = dfl::mul(kg, Gx);
            Gy = dfl::mul(kg, Gy);
            Gz = dfl::mul(kg, Gz);
            const df WX = dfl::sub(VXi, df{wa.x, wa.y}), WY = dfl::sub(VYi, df{wa.z, wa.w});
            const df WZ = dfl::sub(VZi, df{wb.x, wb.y});
            const df vr = dfl::add(dfl::add(dfl::mul(WX, X), dfl::mul(WY, Y)), dfl::mul(WZ, Z));
            df Pi = {0.f, 0.f};
            if (vr.hi < 0.0f) {
                const df hb = dfl::add(hhi, df{b1.z, b1.w});
                const df d1 = dfl::add(r2, dfl::mul(dfl::mul(eta2, hb), hb));
                const df rb = dfl::add(rhi, df{b2.x, b2.y});
                const df Rr = dfl::rcp(dfl::mul(d1, rb));
                const df mu = dfl::mul(dfl::mul(dfl::mul(hb, vr), rb), Rr);
                const df cb = dfl::add(cai, df{b2.z, b2.w});
                const df tt = dfl::add(dfl::mul(betad, mu), dfl::neg(cb));
                Pi = dfl::mul(dfl::mul(mu, tt), dfl::mul(d1, Rr));
                if (-mu.hi > mumx.hi) mumx = dfl::neg(mu);
            }
            const df mj = {J0.w, J1.w};
            const df g = dfl::mul(mj, dfl::add(dfl::add(Ai, df{b1.x, b1.y}), Pi));
            sx = dfl::add(sx, dfl::mul(g, Gx));
            sy = dfl::add(sy, dfl::mul(g, Gy));
            sz = dfl::add(sz, dfl::mul(g, Gz));
            const df Gv = dfl::add(dfl::add(dfl::mul(Gx, WX), dfl::mul(Gy, WY)), dfl::mul(Gz, WZ));
            const df mGv = dfl::mul(mj, Gv);
            sp = dfl::add(sp, mGv);
            sv = dfl::add(sv, dfl::mul(mGv, Pi));
        }
    }
    if (T > 1) {
        sx = dfl::lane_sum<T>(sx);
        sy = dfl::lane_sum<T>(sy);
        sz = dfl::lane_sum<T>(sz);
        sp = dfl::lane_sum<T>(sp);
        sv = dfl::lane_sum<T>(sv);
#pragma unroll
        for (int o = 1; o < T; o <<= 1) {
            const df w = {__shfl_xor_sync(0xffffffffu, mumx.hi, o),
                          __shfl_xor_sync(0xffffffffu, mumx.lo, o)};
            if (w.hi > mumx.hi || (w.hi == mumx.hi && w.lo > mumx.lo)) mumx = w;
        }
    }
    if (act && sub == 0) {
        // back to the caller's units: a ~ V^2 / L, du ~ V^3 / L, mu ~ V
        const Grid& gu = B.grid[slot_inst(B, ((int64_t)blockIdx.x * blockDim.x) / T)];
        const double sa = p2d(2 * gu.uV - gu.uL), su = p2d(3 * gu.uV - gu.uL);
        const double Aid = (double)dpk[3 * i + 1].x + (double)dpk[3 * i + 1].y;
        acc[i] = make_double4_32a(-dfl::to_double(sx) * sa, -dfl::to_double(sy) * sa,
                                  -dfl::to_double(sz) * sa,
                                  fma(Aid, dfl::to_double(sp), 0.5 * dfl::to_double(sv)) * su);
        const double mu_max = dfl::to_double(mumx) * p2d(gu.uV);
        mumax[i] = mu_max;
        const double ci = cint[i];
        const KParams& ke = B.kp[slot_inst(B, ((int64_t)blockIdx.x * blockDim.x) / T)];
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

template <int T, int KER>
static void iad_df_t(sph_ctx* c, cudaStream_t s) {
    const int64_t n = c->n;
    const unsigned nb = (unsigned)((n * T + kThreads - 1) / kThreads);
    const int b = c->cur;
    const Batch B = batch_of(c);
    const Rows R = rows_of(c);
    k_iad_df<T, KER><<<nb, kThreads, 0, s>>>(n, B, c->posh[b], c->xpk, c->vdf, R, c->cpk);
    k_forces_iad_df<T, KER><<<nb, kThreads, 0, s>>>(n, B, c->posh[b], c->vpa, c->vpb, c->dpk, c->xpk,
                                                    c->cpk, c->cint, R, c->acc, c->mumax,
                                                    c->dt_part);
}

template <int KER>
static void iad_df_k(sph_ctx* c, cudaStream_t s) {
    switch (c->tpp) {
        case 2: iad_df_t<2, KER>(c, s); break;
        case 4: iad_df_t<4, KER>(c, s); break;
        case 8: iad_df_t<8, KER>(c, s); break;
        default: iad_df_t<1, KER>(c, s); break;
    }
}

void launch_forces_iad_df(sph_ctx* c, cudaStream_t s) {
    const int64_t n = c->n;
    if (n == 0) return;
    c->launches += 3;
    const int b = c->cur;
    k_volume_df<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        n, batch_of(c), c->velm[b], c->therm, c->vdf);
    if (c->kern_kind == KER_WENDLAND) iad_df_k<KER_WENDLAND>(c, s);
    else if (c->kern_kind == KER_SINC) iad_df_k<KER_SINC>(c, s);
    else iad_df_k<KER_M4>(c, s);
}

}  // namespace sph
