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

constexpr double kInvPi = 0.31830988618379067154;

__device__ __forceinline__ void pair_vec(const double4_32a& a, const double4_32a& b, const KParams& kp,
                                         double& dx, double& dy, double& dz) {
    dx = a.x - b.x;
    dy = a.y - b.y;
    dz = a.z - b.z;
    if (kp.periodic_z) {
        const double half = 0.5 * kp.lz;
        if (dz > half) dz -= kp.lz;
        else if (dz < -half) dz += kp.lz;
    }
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
// follows in the same thread and therm[i] = (rho, p/rho^2, c, 1/h) is written.
template <bool FUSE>
__global__ void __launch_bounds__(kThreads)
k_density(int64_t n, KParams kp, const double4_32a* __restrict__ posh,
          const double4_32a* __restrict__ velm, const double* __restrict__ ue,
          const int64_t* __restrict__ offsets, const int32_t* __restrict__ ngather,
          const int32_t* __restrict__ idx, int64_t nnzcap, double4_32a* __restrict__ therm,
          double* __restrict__ pint) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || offsets[n] > nnzcap) return;
    const double4_32a pi = posh[i];
    const double hinv = 1.0 / pi.w;
    double acc = 0.0;
    const int64_t e0 = offsets[i], e1 = e0 + ngather[i];
    for (int64_t e = e0; e < e1; ++e) {
        const int j = __ldg(&idx[e]);
        const double4_32a pj = posh[j];
        const double mj = velm[j].w;
        double dx, dy, dz;
        pair_vec(pi, pj, kp, dx, dy, dz);
        const double q = sqrt(dx * dx + dy * dy + dz * dz) * hinv;
        const double t = fmax(2.0 - q, 0.0), s = fmax(1.0 - q, 0.0);
        acc += mj * (0.25 * t * t * t - s * s * s);
    }
    const double sigma = hinv * hinv * hinv * kInvPi;
    const double rho = (velm[i].w + acc) * sigma;
    if (FUSE) {
        double p, c;
        eos(kp, rho, ue[i], p, c);
        therm[i] = make_double4_32a(rho, p / (rho * rho), c, hinv);
        pint[i] = p;
    } else {
        therm[i].x = rho;
    }
}

void launch_density(sph_ctx* c, const KParams& kp, bool fuse_eos, cudaStream_t s) {
    const int64_t n = c->n;
    if (n == 0) return;
    const unsigned nb = (unsigned)((n + kThreads - 1) / kThreads);
    const int b = c->cur;
    c->launches += 1;
    if (fuse_eos)
        k_density<true><<<nb, kThreads, 0, s>>>(n, kp, c->posh[b], c->velm[b], c->ue[b],
                                                c->offsets, c->ngather, c->idx, c->nnzcap,
                                                c->therm, c->pint);
    else
        k_density<false><<<nb, kThreads, 0, s>>>(n, kp, c->posh[b], c->velm[b], c->ue[b],
                                                 c->offsets, c->ngather, c->idx, c->nnzcap,
                                                 c->therm, c->pint);
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
__global__ void __launch_bounds__(kThreads)
k_forces(int64_t n, KParams kp, const double4_32a* __restrict__ posh, const double4_32a* __restrict__ velm,
         const double4_32a* __restrict__ therm, const int64_t* __restrict__ offsets,
         const int32_t* __restrict__ idx, int64_t nnzcap, double4_32a* __restrict__ acc,
         double* __restrict__ mumax, double* __restrict__ dt_part) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double dtc = CUDART_INF;
    if (i < n && offsets[n] <= nnzcap) {
        const double4_32a pi = posh[i];
        const double4_32a vi = velm[i];
        const double4_32a ti = therm[i];
        const double hi2 = ti.w * ti.w;
        const double Ki = hi2 * hi2;
        double sx = 0.0, sy = 0.0, sz = 0.0, sp = 0.0, sv = 0.0, mum = 0.0;
        const int64_t e0 = offsets[i], e1 = offsets[i + 1];
        for (int64_t e = e0; e < e1; ++e) {
            const int j = __ldg(&idx[e]);
            const double4_32a pj = posh[j];
            const double4_32a vj = velm[j];
            const double4_32a tj = therm[j];
            double dx, dy, dz;
            pair_vec(pi, pj, kp, dx, dy, dz);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) continue;
            const double rinv = rsqrt(r2);
            const double r = r2 * rinv;
            const double qi = r * ti.w, qj = r * tj.w;
            const double ta = fmax(2.0 - qi, 0.0), sa = fmax(1.0 - qi, 0.0);
            const double tb = fmax(2.0 - qj, 0.0), sb = fmax(1.0 - qj, 0.0);
            const double fa = 3.0 * sa * sa - 0.75 * ta * ta;
            const double fb = 3.0 * sb * sb - 0.75 * tb * tb;
            const double hj2 = tj.w * tj.w;
            const double Fb = (Ki * fa + (hj2 * hj2) * fb) * (0.5 * kInvPi) * rinv;
            const double wx = vi.x - vj.x, wy = vi.y - vj.y, wz = vi.z - vj.z;
            const double vr = wx * dx + wy * dy + wz * dz;
            double Pi = 0.0, mu = 0.0;
            if (vr < 0.0) {
                const double hb = 0.5 * (pi.w + pj.w);
                const double cb = 0.5 * (ti.z + tj.z);
                const double rb = 0.5 * (ti.x + tj.x);
                mu = hb * vr / (r2 + kp.eta2 * hb * hb);
                Pi = (-kp.alpha * cb * mu + kp.beta * mu * mu) / rb;
            }
            const double g = vj.w * (ti.y + tj.y + Pi) * Fb;
            sx += g * dx;
            sy += g * dy;
            sz += g * dz;
            const double mFv = vj.w * Fb * vr;
            sp += mFv;
            sv += mFv * Pi;
            mum = fmax(mum, fabs(mu));
        }
        acc[i] = make_double4_32a(-sx, -sy, -sz, ti.y * sp + 0.5 * sv);
        mumax[i] = mum;
        dtc = pi.w / (ti.z + 1.2 * (kp.alpha * ti.z + kp.beta * mum));
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

// dt = cfl * min over the block partials; optionally time += dt.
__global__ void __launch_bounds__(kThreads)
k_dt_finish(const double* __restrict__ part, int np, double cfl, double* __restrict__ dt_out,
            double* __restrict__ time) {
    double m = CUDART_INF;
    for (int k = threadIdx.x; k < np; k += blockDim.x) m = fmin(m, part[k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double sh[kThreads / 32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = sh[0];
        for (int w = 1; w < kThreads / 32; ++w) r = fmin(r, sh[w]);
        const double dt = cfl * r;
        *dt_out = dt;
        if (time) *time = *time + dt;
    }
}

void launch_forces(sph_ctx* c, const KParams& kp, double* dt_out, double* time_inout,
                   cudaStream_t s) {
    const int64_t n = c->n;
    const unsigned nb = (unsigned)((n + kThreads - 1) / kThreads);
    const int b = c->cur;
    c->launches += (n > 0) ? 2 : 1;
    if (n > 0)
        k_forces<<<nb, kThreads, 0, s>>>(n, kp, c->posh[b], c->velm[b], c->therm, c->offsets,
                                         c->idx, c->nnzcap, c->acc, c->mumax, c->dt_part);
    k_dt_finish<<<1, kThreads, 0, s>>>(c->dt_part, n > 0 ? (int)nb : 0, kp.cfl, dt_out,
                                       time_inout);
}

// ------------------------------------------------------------ leapfrog
// Kick-drift (reading of Algorithm 1 step 6): v += dt a, u += dt du,
// x += dt v (new v); z wrapped into [-lz/2, lz/2) when periodic.
__global__ void __launch_bounds__(kThreads)
k_leapfrog(int64_t n, KParams kp, const double* __restrict__ dtp, double4_32a* __restrict__ posh,
           double4_32a* __restrict__ velm, double* __restrict__ ue, const double4_32a* __restrict__ acc) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double dt = *dtp;
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

void launch_leapfrog(sph_ctx* c, const KParams& kp, const double* dt, cudaStream_t s) {
    const int64_t n = c->n;
    if (n == 0) return;
    const int b = c->cur;
    c->launches += 1;
    k_leapfrog<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        n, kp, dt, c->posh[b], c->velm[b], c->ue[b], c->acc);
}

// ------------------------------------------------------------ scatter
struct ScatterSrc {
    const int32_t* order;
    const double4_32a *posh, *velm, *therm, *acc;
    const double *ue, *pint, *mumax;
    const int32_t* nnb;
};

__global__ void __launch_bounds__(kThreads)
k_scatter(int64_t n, unsigned f, ScatterSrc S, sph_particles P) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t o = S.order[k];
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
    if (f & (SC_RHO | SC_PC)) {
        const double4_32a t = S.therm[k];
        if (f & SC_RHO) P.rho[o] = t.x;
        if (f & SC_PC) { P.p[o] = S.pint[k]; P.c[o] = t.z; }
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
                 c->mumax, c->nnb};
    k_scatter<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(n, fields, S, *P);
}

}  // namespace sph
