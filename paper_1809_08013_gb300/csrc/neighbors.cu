// neighbors.cu -- Algorithm 1 step 2: the neighbours and the smoothing length.
//
// Pair test. The definition is the FP64 test r_ij^2 < (2h)^2 with
// r^2 = (dx dx + dy dy) + dz dz, each operation rounded on its own (minimum
// image along z when periodic). GB300 issues FP64 at 1/64 of the FP32 rate,
// so candidates are classified in FP32 from float copies of the positions:
//   r2f < Tin   -> certainly inside,   r2f > Tout -> certainly outside,
//   otherwise   -> the exact FP64 test above decides.
// Tin/Tout come from a rigorous bound on the FP32 error evaluated with
// directed-rounding FP32 operations (thresholds()), so every decision equals
// the FP64 one and the neighbour sets are exact.
//
// h search (reading of the Section 3 footnote: h follows a target neighbour
// count): bracketing search using only correctly rounded * and +,
//   n < target - tol: lo = h; h = (hi == inf) ? 1.25 h : (lo + hi) / 2
//   n > target + tol: hi = h; h = (lo == 0)   ? 0.8 h  : (lo + hi) / 2
// for at most max_h_iter counts; the result is the last h counted.
//
// Symmetric set S_i = { j != i : r_ij < 2h_i or r_ij < 2h_j } as CSR: row i
// holds N_i (r_ij < 2h_i) first, then the rest.
//
// Work decomposition: one warp per particle. The lanes take 32 candidates of
// a cell at a time (coalesced loads), counts come from ballots and row
// entries are compacted with ballot prefix counts, so the particle's own
// iteration count never stalls other particles.
#include <math_constants.h>

#include <algorithm>

#include "df.cuh"
#include "sph_internal.cuh"

namespace sph {

constexpr unsigned kFull = 0xffffffffu;

struct Thr {
    float tin, tout;
};

// FP32 classification thresholds for radius R = 2h (R > 0).
// The FP32 norm of a pair differs from the norm of the FP64 difference vector
// by at most d = sqrt(3) e, e = eC + eR R (see k_grid_setup); the FP32 sum of
// squares adds at most 3 * 2^-24 relative; the FP64 square differs from the
// FP64 norm squared by < 2^-50 relative. All operations round outward.
__device__ __forceinline__ Thr thresholds(double R, const Grid* __restrict__ g) {
    float Rl, Rh;
    f32_bounds(R, Rl, Rh);
    const float e = __fmaf_ru(g->eR, Rh, g->eC);
    const float d = __fmul_ru(1.7320525f, e);
    Thr t;
    const float a = __fsub_rd(__fmul_rd(Rl, 0.99999905f), d);  // Rl (1 - 2^-20) - d
    t.tin = a > 0.0f ? __fmul_rd(__fmul_rd(a, a), 0.9999997f) : -1.0f;
    const float b = __fadd_ru(__fmul_ru(Rh, 1.00000096f), d);   // Rh (1 + 2^-20) + d
    t.tout = __fmul_ru(__fmul_ru(b, b), 1.0000003f);
    if (g->periodic_z && Rh > 0.25f * g->lzf) {  // wrap decisions may differ: exact path only
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
    return exact_r2_def(a, b, g->periodic_z != 0, g->lz);
}

__device__ __forceinline__ int wrapi(int k, int n) {
    int r = k % n;
    return r < 0 ? r + n : r;
}

// Cell index range overlapping [v - R, v + R] along axis d (clamped); along the
// periodic z axis an unclamped range (wrapped by the caller) or the whole axis.
// A non-finite v or R (a particle outside the geometry range) gets no cells;
// a periodic range far from the box (|index| >= 2^30) takes the whole axis,
// so the callers' int loops never come near overflow.
__device__ __forceinline__ void axis_range(float v, float R, const Grid* __restrict__ g, int d,
                                           int& k0, int& k1) {
    const float inv = g->invwf[d], s = g->slop[d];
    const int n = g->n[d];
    if (!(fabsf(v) < CUDART_INF_F) || !(R < CUDART_INF_F)) {
        k0 = 0;
        k1 = -1;
        return;
    }
    if (d == 2 && g->periodic_z) {
        const float fa = floorf((v - R - s + g->halflzf) * inv);
        const float fb = floorf((v + R + s + g->halflzf) * inv);
        if (!(fb - fa + 1.0f < (float)n) || !(fabsf(fa) < 1.0e9f && fabsf(fb) < 1.0e9f)) {
            k0 = 0;
            k1 = n - 1;
            return;
        }
        k0 = (int)fa;
        k1 = (int)fb;
        return;
    }
    const float lo = g->lof[d];
    float fa = floorf((v - R - s - lo) * inv);
    float fb = floorf((v + R + s - lo) * inv);
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

// Cell index range overlapping [a, b] along axis d (clamped); along the
// periodic z axis an unclamped range (wrapped by the caller) or the whole axis.
// Non-finite bounds and far periodic ranges as in axis_range.
__device__ __forceinline__ void box_range(float a, float b, const Grid* __restrict__ g, int d,
                                          int& k0, int& k1) {
    const float inv = g->invwf[d], s = g->slop[d];
    const int n = g->n[d];
    if (!(fabsf(a) < CUDART_INF_F) || !(fabsf(b) < CUDART_INF_F)) {
        k0 = 0;
        k1 = -1;
        return;
    }
    if (d == 2 && g->periodic_z) {
        const float fa = floorf((a - s + g->halflzf) * inv);
        const float fb = floorf((b + s + g->halflzf) * inv);
        if (!(fb - fa + 1.0f < (float)n) || !(fabsf(fa) < 1.0e9f && fabsf(fb) < 1.0e9f)) {
            k0 = 0;
            k1 = n - 1;
            return;
        }
        k0 = (int)fa;
        k1 = (int)fb;
        return;
    }
    const float lo = g->lof[d];
    float fa = floorf((a - s - lo) * inv);
    float fb = floorf((b + s - lo) * inv);
    fa = fminf(fmaxf(fa, 0.0f), (float)n);
    fb = fmaxf(fminf(fb, (float)(n - 1)), -1.0f);
    k0 = (int)fa;
    k1 = (int)fb;
}

__device__ __forceinline__ float wmin(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
__device__ __forceinline__ float wmax(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// One warp, one particle: enumerate the candidates of every cell overlapping
// the box [q - R, q + R] as one flat list. Up to 32 cells are fetched at once
// (one per lane), a warp scan of their sizes gives each cell's offset, and the
// list is handed out 32 candidates at a time: chunk(valid, j) is called by
// all lanes together, lane l receiving candidate j (valid = false past the
// end). PRUNE = 1 drops a cell whose box lies farther than R from the
// particle; PRUNE = 2 drops it unless its box lies within
// 2 max(h_i, max h of the cell) of the particle (hib = bits of h_i).
template <int PRUNE, class Chunk>
__device__ __forceinline__ void particle_pass(const Grid* __restrict__ g,
                                              const int2* __restrict__ cells,
                                              const unsigned long long* __restrict__ cell_hmax,
                                              const float4& q, float R, long long hib,
                                              int* s_start, int* s_pref, Chunk&& chunk) {
    const int lane = threadIdx.x & 31;
    int x0, x1, y0, y1, z0, z1;
    axis_range(q.x, R, g, 0, x0, x1);
    axis_range(q.y, R, g, 1, y0, y1);
    axis_range(q.z, R, g, 2, z0, z1);
    const int nxr = x1 - x0 + 1, nyr = y1 - y0 + 1, nzr = z1 - z0 + 1;
    if (nxr <= 0 || nyr <= 0 || nzr <= 0) return;
    const int C = nxr * nyr * nzr;
    const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
    const bool per = g->periodic_z != 0;
    for (int c0 = 0; c0 < C; c0 += 32) {
        const int c = c0 + lane;
        int start = 0, cnt = 0;
        if (c < C) {
            const int kx = x0 + c % nxr;
            const int rr = c / nxr;
            const int ky = y0 + rr % nyr;
            const int kz = z0 + rr / nyr;
            const int cz = per ? wrapi(kz, nz) : kz;
            const long long lin = ((long long)cz * ny + ky) * nx + kx;
            const int2 se = __ldg(&cells[lin]);
            start = se.x;
            cnt = se.y - se.x;
            if (PRUNE && cnt > 0) {
                float reach = R;
                if (PRUNE == 2) {
                    const long long hcb = (long long)__ldg(&cell_hmax[lin]);
                    reach = reach_f32(__longlong_as_double(hcb > hib ? hcb : hib));
                }
                const float gx = axis_gap(q.x, kx, g, 0), gy = axis_gap(q.y, ky, g, 1);
                const float gz = per ? 0.0f : axis_gap(q.z, kz, g, 2);
                if (fmaf(gz, gz, fmaf(gy, gy, gx * gx)) >= reach * reach) cnt = 0;
            }
        }
        int inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += v;
        }
        const int total = __shfl_sync(kFull, inc, 31);
        s_start[lane] = start;
        s_pref[lane] = inc - cnt;  // exclusive offset; lanes past C hold total
        __syncwarp();
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int t = t0 + lane;
            const bool valid = t < total;
            int j = -1;
            if (valid) {
                int k = 0;  // last cell whose offset is <= t
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (s_pref[k + step] <= t) k += step;
                j = s_start[k] + (t - s_pref[k]);
            }
            chunk(valid, j);
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------ h search
// Phase 1: one warp per 32 consecutive (Morton-sorted) particles, one lane
// per particle. Each pass counts N_i(h) for every still-searching lane over
// the union of their query boxes (candidates staged once for the warp) and
// records the gather set in the slab. While more than defer_lanes lanes are
// still searching the warp keeps going; the stragglers are then handed, with
// their bisection state, to the per-particle kernel below through a worklist.

// Cell index of a (float) coordinate along axis d, clamped to the grid; only
// used to cluster the lanes of a warp, so FP32 rounding is harmless.
__device__ __forceinline__ int lane_cell(float v, const Grid* __restrict__ g, int d) {
    const float lo = (d == 2 && g->periodic_z) ? -g->halflzf : g->lof[d];
    const int k = (int)floorf((v - lo) * g->invwf[d]);
    return min(max(k, 0), g->n[d] - 1);
}

// Test the 32 staged candidates of a warp against every lane's particle and
// fold the outcome into that lane's count and gather slab. Candidates are
// (float x, y, z) already moved to the lane's periodic image; sidx holds
// their particle indices. Padding slots sit far away.
// rec: instead of counting, record (r^2 in FP32, j) of every candidate that
// may lie within the thresholds' radius (r2 <= Tout) in recb (up to kRec),
// except those with r2 < tin_lo, certainly within 2 lo (lo the bisection's
// lower bound, so within 2 h for every h still to be tried): those go to the
// gather slab and the count c at once.
// BL: also append to the lane's candidate list (slots, entries 32 apart from
// lrow on; nl of them) every staged candidate with r^2 <= tL. Padding slots
// (sidx -1) are never counted, recorded or listed.
template <bool BL>
__device__ __forceinline__ void union_chunk(const float4* __restrict__ st, const int* __restrict__ sidx,
                                            const float4& fi, const Thr& t, bool active, bool rec,
                                            float tin_lo, int64_t i, double h, double& R2,
                                            const double4_32a* posh, const Grid* __restrict__ g,
                                            int32_t* slab, int& c, int2* recb, int& nrec,
                                            float tL, int32_t* __restrict__ lrow, int& nl) {
    unsigned in = 0u, bd = 0u, lb = 0u;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const float4 q = st[k];
        const float dx = fi.x - q.x, dy = fi.y - q.y, dz = fi.z - q.z;
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        if (r2 < t.tin) in |= 1u << k;
        if (r2 <= t.tout) bd |= 1u << k;
        if (BL && r2 <= tL) lb |= 1u << k;
    }
    if (!active) return;
    if (BL) {
        while (lb) {
            const int k = __ffs(lb) - 1;
            lb &= lb - 1u;
            const int j = sidx[k];
            if (j == i || j < 0) continue;
            if (nl < kList) lrow[nl * 32] = j;
            ++nl;
        }
    }
    if (rec) {
        while (bd) {
            const int k = __ffs(bd) - 1;
            bd &= bd - 1u;
            const int j = sidx[k];
            if (j == i || j < 0) continue;
            const float4 q = st[k];
            const float dx = fi.x - q.x, dy = fi.y - q.y, dz = fi.z - q.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (r2 < tin_lo) {
                if (c < kGSlab) slab[c] = j;
                ++c;
                continue;
            }
            if (nrec < kRec) recb[nrec] = make_int2(__float_as_int(r2), j);
            ++nrec;
        }
        return;
    }
    bd &= ~in;
    while (bd) {  // the ~1e-5-wide border band: exact FP64 test (rare: reloads p_i)
        const int k = __ffs(bd) - 1;
        bd &= bd - 1u;
        const int j = sidx[k];
        if (j == i || j < 0) continue;
        if (R2 < 0.0) {
            const double R = 2.0 * h;
            R2 = __dmul_rn(R, R);
        }
        if (exact_r2(posh[i], posh[j], g) < R2) in |= 1u << k;
    }
    while (in) {
        const int k = __ffs(in) - 1;
        in &= in - 1u;
        const int j = sidx[k];
        if (j == i || j < 0) continue;
        if (c < kGSlab) slab[c] = j;
        ++c;
    }
}

// N_i(h) from a candidate list (slots, ln entries 32 apart from L on): the
// same FP32 decisions with the exact FP64 band as a cell walk, the members
// written to the slab in list order. The list must hold every j within 2 h of
// i (the caller checks that it still does).
__device__ __forceinline__ int list_count(const int32_t* __restrict__ L, int ln,
                                          const float4* __restrict__ fpos, const float4& fi,
                                          const Thr& t, int64_t i, double h,
                                          const double4_32a* posh, const Grid* __restrict__ g,
                                          int32_t* slab) {
    int c = 0;
    double R2 = -1.0;
    constexpr int G = 4;  // entries in flight per group (loads first, then the tests)
    for (int e0 = 0; e0 < ln; e0 += G) {
        int j[G];
        float4 f[G];
#pragma unroll
        for (int k = 0; k < G; ++k) j[k] = e0 + k < ln ? __ldg(&L[(e0 + k) * 32]) : -1;
#pragma unroll
        for (int k = 0; k < G; ++k) f[k] = j[k] >= 0 ? __ldg(&fpos[j[k]]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < G; ++k) {
            if (j[k] < 0) continue;
            const float r2 = f_r2(fi, f[k], g);
            bool in = r2 < t.tin;
            if (!in && r2 <= t.tout) {
                if (R2 < 0.0) {
                    const double R = 2.0 * h;
                    R2 = __dmul_rn(R, R);
                }
                in = exact_r2(posh[i], posh[j[k]], g) < R2;
            }
            if (in) {
                if (c < kGSlab) slab[c] = j[k];
                ++c;
            }
        }
    }
    return c;
}

// |N_i(hh)| from the c0 neighbours certainly within 2 lo <= 2 hh (already in
// the slab) and the records of a record pass made at a radius >= 2 hh, with
// the same decisions as a counting pass (FP32 thresholds, exact FP64 test in
// the band between them); with slab, the recorded members of N_i(hh) are
// appended after the first c0, in record order.
__device__ int count_records(const int2* recb, int nrec, double hh, const Grid* __restrict__ g,
                             const double4_32a* posh, int64_t i, int32_t* slab, int c0) {
    const double R = 2.0 * hh;
    const Thr t = thresholds(R, g);
    double R2 = -1.0;
    int c = c0;
    for (int q = 0; q < nrec; ++q) {
        const int2 e = recb[q];
        const float r2 = __int_as_float(e.x);
        bool in = r2 < t.tin;
        if (!in && r2 <= t.tout) {
            if (R2 < 0.0) R2 = __dmul_rn(R, R);
            in = exact_r2(posh[i], posh[e.y], g) < R2;
        }
        if (in) {
            if (slab && c < kGSlab) slab[c] = e.y;
            ++c;
        }
    }
    return c;
}

// The 32 particles i0 .. i0 + 31 (one per lane; all of one instance).
// LISTS: the batch has instances with candidate lists (else their code is
// compiled out).
template <bool LISTS>
__device__ __forceinline__ void union_group(
    int64_t i0, int64_t n, const Batch& B, double4_32a* posh, const float4* __restrict__ fpos,
    const int2* __restrict__ cells, int32_t* __restrict__ nnb, int32_t* __restrict__ ngather,
    int32_t* __restrict__ rslab, double* __restrict__ hs_lo, double* __restrict__ hs_hi,
    int32_t* __restrict__ hs_it, int32_t* __restrict__ wl, unsigned* __restrict__ status,
    float4* st, int* sidx, int2* recb, const int32_t* __restrict__ order,
    int32_t* __restrict__ lst, LMeta* __restrict__ lmeta) {
    const int lane = threadIdx.x & 31;
    const int64_t i = i0 + lane;
    const int inst = slot_inst(B, i0);
    const Grid* __restrict__ g = B.grid + inst;
    const KParams& kp = B.kp[inst];
    cells += g->cbase;
    const bool inb = i < n;
    const bool valid = inb && slot_real(B, inst, i);
    float4 fi = make_float4(0.f, 0.f, 0.f, 0.f);
    double h = 1.0, lo = 0.0, hi = CUDART_INF;
    if (valid) {
        h = posh[i].w;
        fi = fpos[i];
    }
    // a particle outside the geometry range (reported by the bounding box)
    // does not search: no neighbours, h unchanged
    const bool geo = valid && isfinite(fi.x) && isfinite(fi.y) && isfinite(fi.z) && h_ok(h);
    const int lowb = kp.n_target - kp.n_tol, highb = kp.n_target + kp.n_tol;
    const int max_it = kp.max_h_iter;
    const int defer = kp.defer_lanes;
    int cnt = 0, it = 0;
    bool active = geo && max_it > 0, conv = false, deferred = false;
    int32_t* slab = rslab + (valid ? i : 0) * kRSlab;
    const bool per = g->periodic_z != 0;
    const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
    const unsigned lt = (1u << lane) - 1u;
    // Candidate lists: a lane with a kept list was served by k_h_lists. A
    // build step walks every lane, recording its list (every candidate within
    // 2 h (1 + skin)) in the first walk.
    const bool build = LISTS && kp.list_skin > 0.0 && g->lbuild != 0;
    const int32_t id = LISTS && valid && kp.list_skin > 0.0 ? __ldg(&order[i]) : 0;
    int32_t* lrow = lst + (i >> 5) * (int64_t)kList * 32 + (i & 31);
    int nl = 0;
    bool listed = false;
    if (build && valid) {  // the list build's record of the particle (its list comes with the walk)
        const double4_32a p = posh[i];
        reinterpret_cast<float4*>(lmeta)[2 * id] =
            make_float4(dfl::from_double(p.x).hi, dfl::from_double(p.y).hi,
                        dfl::from_double(p.z).hi, 0.0f);
        lmeta[id].stamp = g->lstamp;  // (the cell code was recorded by the sort)
        lmeta[id].cnt = 0;
    } else if (LISTS && kp.list_skin > 0.0 && active && lmeta[id].cnt > 0) {
        listed = true;
        active = false;
    }
    for (int pass = 0;; ++pass) {  // pass is warp-uniform; it (per lane) stops at convergence
        const unsigned am = __ballot_sync(kFull, active);
        if (!am) break;
        // Pass 0 counts N_i(h). Later passes record every candidate within 2 hs,
        // hs = the largest h the bisection can still test without growing (hi, or
        // h while hi is unbounded), and resolve the following counts from the
        // records: a search from a poor initial h takes ~2 passes, not ~8.
        const bool rec = pass > 0;
        const double hs = rec && !isinf(hi) ? hi : h;
        const Thr t = thresholds(2.0 * hs, g);
        const float tin_lo = rec && lo > 0.0 ? thresholds(2.0 * lo, g).tin : -1.0f;
        const bool blist = build && pass == 0;  // list radius RL = 2 hs (1 + skin)
        const double RL = blist ? 2.0 * hs * (1.0 + kp.list_skin) : 0.0;
        const float tL = blist ? thresholds(RL, g).tout : 0.0f;
        const float Rq = blist ? reach_f32(0.5 * RL) : reach_f32(hs);
        const float lzz = wmin(active ? fi.z - Rq : CUDART_INF_F), hzz = wmax(active ? fi.z + Rq : -CUDART_INF_F);
        // Periodic z: candidates are moved to the image nearest a reference lane's
        // z, which is each lane's minimum image while the lanes' z span S and
        // reach R satisfy R + S < lz/2 (a candidate within R of lane i is then
        // within lz/2 of the reference lane). A warp with S + 2R > lz/4 hands
        // its particles to the per-particle kernel: correct up to ~lz/2, but
        // measured faster there (27k periodic patch: 0.47 ms per step at lz/4,
        // 0.52 at 0.45 lz; the 1M patch the same within 1%).
        const bool wide = per && (hzz - lzz > 0.25f * g->lzf);
        if ((pass > 0 && __popc(am) <= defer) || wide) {
            if (active) {
                deferred = true;
                active = false;
                posh[i].w = h;
                hs_lo[i] = lo;
                hs_hi[i] = hi;
                hs_it[i] = it;
                wl[atomicAdd(&status[3], 1u)] = (int32_t)i;
            }
            break;
        }
        // The active lanes are served in clusters: the first remaining lane and
        // every remaining lane whose cell is within one cell of it. A warp whose
        // particles straddle a jump of the Morton curve thus searches two
        // compact boxes instead of one box spanning both places.
        const int mcx = lane_cell(fi.x, g, 0), mcy = lane_cell(fi.y, g, 1);
        const int mcz = lane_cell(fi.z, g, 2);
        double R2 = -1.0;
        int c = 0, nrec = 0;
        unsigned todo = am;
        while (todo) {
            const int a = __ffs(todo) - 1;
            const int ax = __shfl_sync(kFull, mcx, a), ay = __shfl_sync(kFull, mcy, a);
            const int az = __shfl_sync(kFull, mcz, a);
            int dzc = abs(mcz - az);
            if (per) dzc = min(dzc, nz - dzc);
            const bool mine = ((todo >> lane) & 1u) && abs(mcx - ax) <= 1 && abs(mcy - ay) <= 1 &&
                              dzc <= 1;
            todo &= ~__ballot_sync(kFull, mine);
            const float sx0 = wmin(mine ? fi.x - Rq : CUDART_INF_F), sx1 = wmax(mine ? fi.x + Rq : -CUDART_INF_F);
            const float sy0 = wmin(mine ? fi.y - Rq : CUDART_INF_F), sy1 = wmax(mine ? fi.y + Rq : -CUDART_INF_F);
            const float sz0 = wmin(mine ? fi.z - Rq : CUDART_INF_F), sz1 = wmax(mine ? fi.z + Rq : -CUDART_INF_F);
            const float zc = __shfl_sync(kFull, fi.z, a);
            int x0, x1, y0, y1, z0, z1;
            box_range(sx0, sx1, g, 0, x0, x1);
            box_range(sy0, sy1, g, 1, y0, y1);
            box_range(sz0, sz1, g, 2, z0, z1);
            int fill = 0;  // staged candidates (warp-uniform)
            const float Rq2 = Rq * Rq;
            // Query box of the cluster: a candidate within 2h_i (FP64) of one of its
            // lanes lies inside it. The slop (>= 1e-3 cell widths + 1.2e-7 X)
            // covers the FP32 rounding of both coordinates and of the periodic shift.
            const float bx0 = sx0 - g->slop[0], bx1 = sx1 + g->slop[0];
            const float by0 = sy0 - g->slop[1], by1 = sy1 + g->slop[1];
            const float bz0 = sz0 - g->slop[2], bz1 = sz1 + g->slop[2];
            // and in a ball around the cluster's centre o: |q - o| <= |q - p_i| + |p_i - o|
            // <= Rq_i + |p_i - o| for a candidate q within reach of lane i
            const float ox = 0.5f * (wmin(mine ? fi.x : CUDART_INF_F) + wmax(mine ? fi.x : -CUDART_INF_F));
            const float oy = 0.5f * (wmin(mine ? fi.y : CUDART_INF_F) + wmax(mine ? fi.y : -CUDART_INF_F));
            const float oz = 0.5f * (wmin(mine ? fi.z : CUDART_INF_F) + wmax(mine ? fi.z : -CUDART_INF_F));
            float rb = 0.0f;
            if (mine) {
                const float ex = fi.x - ox, ey = fi.y - oy, ez = fi.z - oz;
                rb = sqrtf(fmaf(ez, ez, fmaf(ey, ey, ex * ex))) + Rq;
            }
            rb = wmax(rb) * 1.00001f + fmaxf(g->slop[0], fmaxf(g->slop[1], g->slop[2]));
            const float rb2 = rb * rb;
            for (int kz = z0; kz <= z1; ++kz) {
                const int cz = per ? wrapi(kz, nz) : kz;
                const float gz = per ? 0.0f : axis_gap(fi.z, kz, g, 2);
                for (int ky = y0; ky <= y1; ++ky) {
                    const long long row = ((long long)cz * ny + ky) * nx;
                    const float gy = axis_gap(fi.y, ky, g, 1);
                    for (int kx = x0; kx <= x1; ++kx) {
                        const int2 se = __ldg(&cells[row + kx]);
                        if (se.y <= se.x) continue;
                        const float gx = axis_gap(fi.x, kx, g, 0);
                        if (!__any_sync(kFull, mine && fmaf(gz, gz, fmaf(gy, gy, gx * gx)) < Rq2))
                            continue;
                        // append the cell's particles that lie in the query box to the
                        // staging buffer (ballot-compacted, so the order of the kept
                        // candidates is unchanged); run full chunks
                        for (int s0 = se.x; s0 < se.y; s0 += 32) {
                            const int j = s0 + lane;
                            bool ok = j < se.y;
                            float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (ok) {
                                f = __ldg(&fpos[j]);
                                if (per) {
                                    const float d = f.z - zc;
                                    if (d > g->halflzf) f.z -= g->lzf;
                                    else if (d < -g->halflzf) f.z += g->lzf;
                                }
                                const float qx = f.x - ox, qy = f.y - oy, qz = f.z - oz;
                                ok = f.x >= bx0 && f.x <= bx1 && f.y >= by0 && f.y <= by1 &&
                                     f.z >= bz0 && f.z <= bz1 &&
                                     fmaf(qz, qz, fmaf(qy, qy, qx * qx)) <= rb2;
                            }
                            const unsigned m = __ballot_sync(kFull, ok);
                            if (!m) continue;
                            const int r = __popc(m & lt), cnt = __popc(m), room = 32 - fill;
                            if (ok && r < room) {
                                st[fill + r] = f;
                                sidx[fill + r] = j;
                            }
                            if (cnt < room) {
                                fill += cnt;
                                continue;
                            }
                            __syncwarp();
                            if (blist)
                                union_chunk<true>(st, sidx, fi, t, mine, rec, tin_lo, i, h, R2,
                                                  posh, g, slab, c, recb, nrec, tL, lrow, nl);
                            else
                                union_chunk<false>(st, sidx, fi, t, mine, rec, tin_lo, i, h, R2,
                                                   posh, g, slab, c, recb, nrec, tL, lrow, nl);
                            __syncwarp();
                            if (ok && r >= room) {
                                st[r - room] = f;
                                sidx[r - room] = j;
                            }
                            fill = cnt - room;
                        }
                    }
                }
            }
            if (fill > 0) {  // last partial chunk: pad with far-away slots
                if (lane >= fill) {
                    st[lane] = make_float4(3.0e30f, 3.0e30f, 3.0e30f, 0.0f);
                    sidx[lane] = -1;
                }
                __syncwarp();
                if (blist)
                    union_chunk<true>(st, sidx, fi, t, mine, rec, tin_lo, i, h, R2, posh, g, slab,
                                      c, recb, nrec, tL, lrow, nl);
                else
                    union_chunk<false>(st, sidx, fi, t, mine, rec, tin_lo, i, h, R2, posh, g, slab,
                                       c, recb, nrec, tL, lrow, nl);
                __syncwarp();
            }
        }
        if (blist && active) {  // the list of this walk, complete unless it overflowed
            float lo_r, hi_r;
            f32_bounds(RL, lo_r, hi_r);
            lmeta[id].rad = lo_r * 0.999999f;
            lmeta[id].cnt = nl <= kList ? nl : 0;
        }
        if (active && rec && nrec > kRec) {  // too many to record: one warp of its own
            deferred = true;
            active = false;
            posh[i].w = h;
            hs_lo[i] = lo;
            hs_hi[i] = hi;
            hs_it[i] = it;
            wl[atomicAdd(&status[3], 1u)] = (int32_t)i;
        }
        // counts of this pass (or from its records) and the bisection updates
        const int cbase = rec ? c : 0;  // a record pass: the neighbours within 2 lo
        for (bool counted = !rec; active;) {
            if (rec) {
                if (h > hs) break;  // beyond the recorded radius: another pass
                c = count_records(recb, nrec, h, g, posh, i, nullptr, cbase);
            } else if (counted) {
                counted = false;  // c holds this pass's count
            } else {
                break;
            }
            cnt = c;
            ++it;
            if (cnt >= lowb && cnt <= highb) {
                conv = true;
                active = false;
            } else if (it >= max_it) {
                active = false;
            } else if (cnt < lowb) {
                lo = h;
                h = isinf(hi) ? __dmul_rn(h, 1.25) : __dmul_rn(0.5, __dadd_rn(lo, hi));
            } else {
                hi = h;
                h = (lo == 0.0) ? __dmul_rn(h, 0.8) : __dmul_rn(0.5, __dadd_rn(lo, hi));
            }
            if (!rec) break;
            if (!active) count_records(recb, nrec, h, g, posh, i, slab, cbase);  // N_i(final h)
        }
    }
    if (!valid) {
        if (inb) {  // empty slot: empty row
            nnb[i] = 0;
            ngather[i] = 0;
        }
        return;
    }
    if (deferred || listed) return;
    posh[i].w = h;
    nnb[i] = cnt;
    ngather[i] = cnt;
    if (cnt > kGSlab) atomicOr(&status[2], (unsigned)IF_SLAB_OVF);
    if (!conv) {
        atomicOr(&status[0], (unsigned)ST_HNOCONV);
        atomicAdd(&status[1], 1u);
    }
}

// The first count of the particles with a kept candidate list (one thread
// per slot; the others are left to k_h_union): one scan of the list at the
// current h, while the list still covers 2h (its radius at the build minus
// twice the largest displacement since), with the cell walk's decisions. A
// particle that converges is done; one that must go on bisecting (or whose
// list does not cover 2h) is handed, with its bisection state, to
// k_h_iterate, which takes its records from the list while it covers them:
// the same sequence of h and the same neighbour set as the cell walk.
__global__ void __launch_bounds__(kThreads)
k_h_lists(int64_t n, Batch B, double4_32a* posh, const float4* __restrict__ fpos,
          int32_t* __restrict__ nnb, int32_t* __restrict__ ngather, int32_t* __restrict__ rslab,
          double* __restrict__ hs_lo, double* __restrict__ hs_hi, int32_t* __restrict__ hs_it,
          int32_t* __restrict__ wl, unsigned* __restrict__ status,
          const int32_t* __restrict__ order, const int32_t* __restrict__ lst,
          const LMeta* __restrict__ lmeta) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int inst = slot_inst(B, i);
    if (!slot_real(B, inst, i)) return;
    const KParams& kp = B.kp[inst];
    const Grid* __restrict__ g = B.grid + inst;
    if (!(kp.list_skin > 0.0) || g->lbuild || kp.max_h_iter < 1) return;
    const int32_t id = order[i];
    const int ln = lmeta[id].cnt;
    if (ln <= 0) return;
    double h = posh[i].w;
    const float4 fi = fpos[i];
    if (!(isfinite(fi.x) && isfinite(fi.y) && isfinite(fi.z) && h_ok(h))) return;
    const float lrad = lmeta[id].rad, dm2 = g->dm2;
    const int lowb = kp.n_target - kp.n_tol, highb = kp.n_target + kp.n_tol;
    const int max_it = kp.max_h_iter;
    const int32_t* L = lst + (i >> 5) * (int64_t)kList * 32 + (i & 31);
    int32_t* slab = rslab + i * kRSlab;
    double lo = 0.0, hi = CUDART_INF;
    int cnt = 0, it = 0;
    bool conv = false;
    // one count at the current h, from the list if it still covers 2h; a
    // particle that has to go on bisecting (or whose list no longer covers
    // 2h) continues in k_h_iterate, which records its candidates once
    const bool covered = reach_f32(h) + dm2 <= lrad;
    if (covered) {
        cnt = list_count(L, ln, fpos, fi, thresholds(2.0 * h, g), i, h, posh, g, slab);
        it = 1;
        conv = cnt >= lowb && cnt <= highb;
    }
    if (!covered || (!conv && it < max_it)) {
        if (covered) {
            if (cnt < lowb) {
                lo = h;
                h = __dmul_rn(h, 1.25);  // no upper bound yet
            } else {
                hi = h;
                h = __dmul_rn(h, 0.8);  // no lower bound yet
            }
        }
        posh[i].w = h;
        hs_lo[i] = lo;
        hs_hi[i] = hi;
        hs_it[i] = it;
        wl[atomicAdd(&status[3], 1u)] = (int32_t)i;
        return;
    }
    posh[i].w = h;
    nnb[i] = cnt;
    ngather[i] = cnt;
    if (cnt > kGSlab) atomicOr(&status[2], (unsigned)IF_SLAB_OVF);
    if (!conv) {
        atomicOr(&status[0], (unsigned)ST_HNOCONV);
        atomicAdd(&status[1], 1u);
    }
}

// Persistent: warps take groups of 32 particles from a counter, so a group
// whose particles straddle far-apart cells (a jump of the Morton curve: a
// large query box, many candidates) delays one warp, not a whole wave.
template <bool LISTS>
__global__ void __launch_bounds__(kThreads, kUnionBlocksPerSM)
k_h_union(int64_t n, Batch B, double4_32a* posh, const float4* __restrict__ fpos,
          const int2* __restrict__ cells,
          int32_t* __restrict__ nnb, int32_t* __restrict__ ngather, int32_t* __restrict__ rslab,
          double* __restrict__ hs_lo, double* __restrict__ hs_hi, int32_t* __restrict__ hs_it,
          int32_t* __restrict__ wl, unsigned* __restrict__ status,
          unsigned long long* __restrict__ wctr, int2* __restrict__ recs,
          const int32_t* __restrict__ order, int32_t* __restrict__ lst,
          LMeta* __restrict__ lmeta) {
    __shared__ float4 s_f[kThreads / 32][32];
    __shared__ int s_i[kThreads / 32][32];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const long long ngroups = (n + 31) / 32;
    for (;;) {
        long long gi = 0;
        if (lane == 0) gi = (long long)atomicAdd(wctr, 1ull);
        gi = __shfl_sync(kFull, gi, 0);
        if (gi >= ngroups) break;
        union_group<LISTS>(gi * 32, n, B, posh, fpos, cells, nnb, ngather, rslab, hs_lo, hs_hi, hs_it,
                    wl, status, s_f[warp], s_i[warp],
                    recs + ((int64_t)(blockIdx.x * (kThreads / 32) + warp) * 32 + lane) * kRec,
                    order, lst, lmeta);
    }
}

// The candidates of a list (ln entries 32 apart from L on), 32 at a time:
// chunk(valid, j) is called by all lanes together, lane l receiving entry
// e0 + l (valid = false past the end), as particle_pass hands out a walk's.
template <class Chunk>
__device__ __forceinline__ void list_pass(const int32_t* __restrict__ L, int ln, Chunk&& chunk) {
    const int lane = threadIdx.x & 31;
    for (int e0 = 0; e0 < ln; e0 += 32) {
        const int e = e0 + lane;
        const bool valid = e < ln;
        chunk(valid, valid ? __ldg(&L[e * 32]) : -1);
    }
}

// Phase 2: one warp per handed-over particle (persistent grid over the
// worklist), continuing its bisection where phase 1 stopped. A walk over the
// cells records, in shared memory and in walk order, every candidate that may
// lie within 2 hs, hs = the largest h the bisection can still test without a
// new walk (hi once bracketed; 1.25 h, the next growth step, before); the
// counts at every h <= hs then come from the records with the same FP32 /
// exact FP64 decisions as a walk, and the gather set is written in the order
// a walk at h would find it. Only growth beyond hs (or more candidates than
// the record buffer holds) walks the cells again.
constexpr int kRecW = 512;  // records per warp

template <bool LISTS>
__global__ void __launch_bounds__(kThreads)
k_h_iterate(Batch B, double4_32a* posh, const float4* __restrict__ fpos,
            const int2* __restrict__ cells,
            int32_t* __restrict__ nnb, int32_t* __restrict__ ngather,
            int32_t* __restrict__ rslab, const double* __restrict__ hs_lo,
            const double* __restrict__ hs_hi, const int32_t* __restrict__ hs_it,
            const int32_t* __restrict__ wl, unsigned* __restrict__ status,
            const int32_t* __restrict__ order, const int32_t* __restrict__ lst,
            const LMeta* __restrict__ lmeta) {
    __shared__ int s_start[kThreads / 32][32], s_pref[kThreads / 32][32];
    __shared__ int2 s_rec[kThreads / 32][kRecW];  // (FP32 r^2 bits, j)
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const unsigned count = *(volatile unsigned*)&status[3];
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const unsigned lt = (1u << lane) - 1u;
    int2* rec = s_rec[warp];
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < count; w += nwarps) {
        const int64_t i = wl[w];
        const int inst = slot_inst(B, i);
        const Grid* __restrict__ g = B.grid + inst;
        const KParams& kp = B.kp[inst];
        const int2* __restrict__ cl = cells + g->cbase;
        const int lowb = kp.n_target - kp.n_tol, highb = kp.n_target + kp.n_tol;
        const int max_it = kp.max_h_iter;
        const double4_32a pi = posh[i];
        const float4 fi = fpos[i];
        double h = pi.w, lo = hs_lo[i], hi = hs_hi[i];
        int cnt = 0;
        bool conv = false;
        int32_t* slab = rslab + i * kRSlab;
        double hs = -1.0;  // radius / 2 the records cover (none yet)
        int nrec = 0;
        // the particle's kept candidate list, while it covers a radius 2 hq
        // (then it replaces the cell walk: the same candidates within 2 hq)
        const bool lists = LISTS && kp.list_skin > 0.0 && !g->lbuild;
        const int ln = lists ? lmeta[order[i]].cnt : 0;
        const float lrad = ln > 0 ? lmeta[order[i]].rad : 0.0f;
        const int32_t* L = lst + (i >> 5) * (int64_t)kList * 32 + (i & 31);
        auto list_covers = [&](double hq) { return ln > 0 && reach_f32(hq) + g->dm2 <= lrad; };
        for (int it = hs_it[i]; it < max_it; ++it) {
            const double R = 2.0 * h;
            const Thr t = thresholds(R, g);
            double R2 = -1.0;  // (2h)^2 in FP64, formed on first use
            int c = 0;
            if (!(h <= hs)) {
                // walk the cells once more and record everything that may lie
                // within 2 hs of the particle
                hs = isinf(hi) ? __dmul_rn(h, 1.25) : hi;
                const float tout_s = thresholds(2.0 * hs, g).tout;
                nrec = 0;
                auto record = [&](bool valid, int j) {
                    float r2f = 0.0f;
                    bool keep = false;
                    if (valid && j != i) {
                        r2f = f_r2(fi, __ldg(&fpos[j]), g);
                        keep = r2f <= tout_s;
                    }
                    const unsigned m = __ballot_sync(kFull, keep);
                    if (keep) {
                        const int q = nrec + __popc(m & lt);
                        if (q < kRecW) rec[q] = make_int2(__float_as_int(r2f), j);
                    }
                    nrec += __popc(m);
                };
                if (list_covers(hs)) list_pass(L, ln, record);
                else particle_pass<1>(g, cl, nullptr, fi, reach_f32(hs), 0, s_start[warp], s_pref[warp],
                                      record);
                __syncwarp();
                if (nrec > kRecW) hs = -1.0;  // too many to keep: count by walking
            }
            if (h <= hs) {
                for (int q0 = 0; q0 < nrec; q0 += 32) {
                    const int q = q0 + lane;
                    bool in = false, bd = false;
                    int j = -1;
                    if (q < nrec) {
                        const int2 e = rec[q];
                        const float r2f = __int_as_float(e.x);
                        j = e.y;
                        in = r2f < t.tin;
                        bd = !in && r2f <= t.tout;
                    }
                    if (__any_sync(kFull, bd) && bd) {
                        if (R2 < 0.0) R2 = __dmul_rn(R, R);
                        in = exact_r2(pi, posh[j], g) < R2;
                    }
                    const unsigned m = __ballot_sync(kFull, in);
                    if (in) {
                        const int qq = c + __popc(m & lt);
                        if (qq < kGSlab) slab[qq] = j;
                    }
                    c += __popc(m);
                }
            } else {
                auto count = [&](bool valid, int j) {
                    bool in = false, bd = false;
                    if (valid && j != i) {
                        const float r2f = f_r2(fi, __ldg(&fpos[j]), g);
                        in = r2f < t.tin;
                        bd = !in && r2f <= t.tout;
                    }
                    if (__any_sync(kFull, bd) && bd) {
                        if (R2 < 0.0) R2 = __dmul_rn(R, R);
                        in = exact_r2(pi, posh[j], g) < R2;
                    }
                    const unsigned m = __ballot_sync(kFull, in);
                    if (in) {
                        const int q = c + __popc(m & lt);
                        if (q < kGSlab) slab[q] = j;
                    }
                    c += __popc(m);
                };
                if (list_covers(h)) list_pass(L, ln, count);
                else particle_pass<1>(g, cl, nullptr, fi, reach_f32(h), 0, s_start[warp], s_pref[warp],
                                      count);
            }
            cnt = c;
            if (cnt >= lowb && cnt <= highb) {
                conv = true;
                break;
            }
            if (it == max_it - 1) break;
            if (cnt < lowb) {
                lo = h;
                h = isinf(hi) ? __dmul_rn(h, 1.25) : __dmul_rn(0.5, __dadd_rn(lo, hi));
            } else {
                hi = h;
                h = (lo == 0.0) ? __dmul_rn(h, 0.8) : __dmul_rn(0.5, __dadd_rn(lo, hi));
            }
        }
        __syncwarp();  // the records are reused by this warp's next particle
        if (lane == 0) {
            posh[i].w = h;
            nnb[i] = cnt;
            ngather[i] = cnt;
            if (cnt > kGSlab) atomicOr(&status[2], (unsigned)IF_SLAB_OVF);
            if (!conv) {
                atomicOr(&status[0], (unsigned)ST_HNOCONV);
                atomicAdd(&status[1], 1u);
            }
        }
    }
}

// Per-particle FP32 thresholds at the final h, and (2h)^2 in the length unit
// of the double-float pair kernels in the spare float of the position pack
// (NaN where the periodic wrap could decide differently: exact test only).
__global__ void __launch_bounds__(kThreads)
k_finalize_h(int64_t n, Batch B, const double4_32a* __restrict__ posh,
             float4* __restrict__ fpos, float* __restrict__ tin, int32_t* __restrict__ ocnt,
             float4* __restrict__ xpk) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    ocnt[i] = 0;
    const int inst = slot_inst(B, i);
    if (!slot_real(B, inst, i)) return;
    const Grid* g = B.grid + inst;
    const double h = posh[i].w;
    const Thr t = thresholds(2.0 * h, g);
    fpos[i].w = t.tout;
    tin[i] = t.tin;
    const double R = 2.0 * h * p2d(-g->uL);
    xpk[3 * i + 2].w = (g->periodic_z && 2.0 * h > 0.25 * g->lz) ? CUDART_NAN_F : (float)(R * R);
}

// Per-cell max h, and the instance's max (one atomic per block); blockIdx.y
// is the instance.
__global__ void __launch_bounds__(kThreads)
k_cell_hmax(Batch B, Grid* gw, const int2* __restrict__ cells,
            const double4_32a* __restrict__ posh, unsigned long long* __restrict__ cell_hmax) {
    const int inst = blockIdx.y;
    const long long nc = B.grid[inst].ncells, cb = B.grid[inst].cbase;
    cells += cb;
    cell_hmax += cb;
    long long bmax = 0;  // bits of positive doubles order like their values
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < nc;
         c += (long long)gridDim.x * blockDim.x) {
        const int2 se = cells[c];
        long long m = 0;
        for (int k = se.x; k < se.y; ++k) {
            const long long b = __double_as_longlong(posh[k].w);
            m = (b > m && b <= kHMaxBits) ? b : m;  // h outside the geometry range: not counted
        }
        cell_hmax[c] = (unsigned long long)m;
        bmax = m > bmax ? m : bmax;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long v = __shfl_xor_sync(kFull, bmax, o);
        bmax = v > bmax ? v : bmax;
    }
    __shared__ long long sh[kThreads / 32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = bmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long m = sh[0];
        for (int w = 1; w < kThreads / 32; ++w) m = sh[w] > m ? sh[w] : m;
        atomicMax(&gw[inst].hmax_bits, (unsigned long long)m);
    }
}

// ------------------------------------------------------------ CSR
// Slab path (normal case). The h search left N_i at the start of row i of the
// row slab. The rest of S_i is the transpose of the non-mutual gather pairs:
// S_j \ N_j = { i : j in N_i and i not in N_j }: k_outer scans the gather
// sets and appends such i after N_j (atomic slot, so unordered),
// k_rowlen_sort sorts each outer part by index (deterministic rows) and forms
// |S_i|; k_compose copies the rows into a CSR when a caller asks for the
// neighbour list.
__global__ void __launch_bounds__(kThreads)
k_outer(int64_t n, Batch B, const double4_32a* __restrict__ posh,
        const float4* __restrict__ fpos, const float* __restrict__ tin,
        const int32_t* __restrict__ ngather, int32_t* __restrict__ rslab,
        int32_t* __restrict__ ocnt, unsigned* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n || (status[2] & IF_SLAB_OVF)) return;
    const int inst = slot_inst(B, i);
    if (!slot_real(B, inst, i)) return;
    const Grid* __restrict__ g = B.grid + inst;
    const int ng = ngather[i];
    const float4 fi = fpos[i];
    // the slab row is read up front so the dependent loads of the entries overlap
    constexpr int kPer = kGSlab / 32;
    int jj[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int s = k * 32 + lane;
        jj[k] = s < ng ? rslab[i * kRSlab + s] : -1;
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int j = jj[k];
        if (j < 0) continue;
        const float4 fj = __ldg(&fpos[j]);
        const float r2f = f_r2(fi, fj, g);
        bool in_j;
        if (r2f < __ldg(&tin[j])) {
            in_j = true;
        } else if (r2f > fj.w) {
            in_j = false;
        } else {
            const double4_32a pj = posh[j];
            const double Rj = 2.0 * pj.w;
            in_j = exact_r2(posh[i], pj, g) < __dmul_rn(Rj, Rj);
        }
        if (!in_j) {  // i joins the outer part of row j, after j's gather set
            const int q = __ldg(&ngather[j]) + atomicAdd(&ocnt[j], 1);
            if (q < kRSlab) rslab[(int64_t)j * kRSlab + q] = (int32_t)i;
            else atomicOr(&status[2], (unsigned)IF_SLAB_OVF);
        }
    }
}

// After the precision 0 density kernel (k_density_df with OUTER): i joins the
// outer part of row j for every gather entry e of row i whose bit is set in
// omask (i is not in N_j). One thread per row; the rows' gather parts are
// only read and their outer parts only written, so nothing overlaps.
__global__ void __launch_bounds__(kThreads)
k_append_outer(int64_t n, Batch B, const unsigned long long* __restrict__ omask,
               const int32_t* __restrict__ ngather, int32_t* __restrict__ rslab,
               int32_t* __restrict__ ocnt, unsigned* __restrict__ status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (status[2] & IF_SLAB_OVF)) return;  // the CSR holds the whole rows
    const int inst = slot_inst(B, i);
    if (!slot_real(B, inst, i)) return;
    // up to four appends in flight per thread: their loads, then their atomic
    // slots, then their stores (each append is a chain of three memory steps)
    constexpr int kBatch = 4;
    const int32_t* row = rslab + i * kRSlab;
    unsigned long long m0 = omask[2 * i], m1 = omask[2 * i + 1];
    while (m0 | m1) {
        int e[kBatch], j[kBatch], q[kBatch];
#pragma unroll
        for (int b = 0; b < kBatch; ++b) {
            e[b] = -1;
            if (m0) {
                e[b] = __ffsll((long long)m0) - 1;
                m0 &= m0 - 1ull;
            } else if (m1) {
                e[b] = 64 + __ffsll((long long)m1) - 1;
                m1 &= m1 - 1ull;
            }
        }
#pragma unroll
        for (int b = 0; b < kBatch; ++b) j[b] = e[b] >= 0 ? row[e[b]] : 0;
#pragma unroll
        for (int b = 0; b < kBatch; ++b)
            q[b] = e[b] >= 0 ? __ldg(&ngather[j[b]]) + atomicAdd(&ocnt[j[b]], 1) : 0;
#pragma unroll
        for (int b = 0; b < kBatch; ++b) {
            if (e[b] < 0) continue;
            if (q[b] < kRSlab) rslab[(int64_t)j[b] * kRSlab + q[b]] = (int32_t)i;
            else atomicOr(&status[2], (unsigned)IF_OUTER_OVF);
        }
    }
}

// Row lengths, and the outer part of each row (appended in atomic order)
// sorted by index in place, one thread per row (rows hold a few outer
// entries): the rows, and every sum over them, become deterministic.
__global__ void __launch_bounds__(kThreads)
k_rowlen_sort(int64_t n, const int32_t* __restrict__ ngather, const int32_t* __restrict__ ocnt,
              int32_t* __restrict__ rowlen, int32_t* __restrict__ rslab,
              const unsigned* __restrict__ status, unsigned mask) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (status[2] & mask)) return;
    const int ng = ngather[i], no = ocnt[i];
    rowlen[i] = ng + no;
    int32_t* row = rslab + i * kRSlab + ng;
    for (int a = 1; a < no; ++a) {  // insertion sort
        const int32_t v = row[a];
        int b = a - 1;
        while (b >= 0 && row[b] > v) {
            row[b + 1] = row[b];
            --b;
        }
        row[b + 1] = v;
    }
}

// The rows as a CSR (for callers of the neighbour list): a copy of each row.
__global__ void __launch_bounds__(kThreads)
k_compose(int64_t n, const int32_t* __restrict__ rowlen, const int32_t* __restrict__ rslab,
          const int64_t* __restrict__ offsets, int32_t* __restrict__ idx, int64_t nnzcap,
          unsigned* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (status[2] & (IF_SLAB_OVF | IF_OUTER_OVF)) return;  // the fallback wrote the CSR
    if (offsets[n] > nnzcap) {
        if (i == 0 && lane == 0) atomicOr(&status[0], (unsigned)ST_CAPACITY);
        return;
    }
    if (i >= n) return;
    const int64_t off = offsets[i];
    const int len = rowlen[i];
    for (int s = lane; s < len; s += 32) idx[off + s] = __ldg(&rslab[i * kRSlab + s]);
}

// Fallback (a row overflowed a slab): the full two-pass build below.
// FILL = false: rowlen[i] = |S_i|, ngather[i] = |N_i|.
// FILL = true : write row i at offsets[i] (N_i first) with ballot-compacted,
//               coalesced stores; nothing is written when the total exceeds
//               the capacity (status bit raised).
// A cell is visited when its box lies within 2 max(h_i, max h of the cell).
template <bool FILL>
__global__ void __launch_bounds__(kThreads)
k_csr(int64_t n, Batch B, const double4_32a* __restrict__ posh,
      const float4* __restrict__ fpos, const float* __restrict__ tin,
      const int2* __restrict__ cells, const unsigned long long* __restrict__ cell_hmax,
      int32_t* __restrict__ rowlen, int32_t* __restrict__ ngather,
      const int64_t* __restrict__ offsets, int32_t* __restrict__ idx, int64_t nnzcap,
      unsigned* __restrict__ status, unsigned mask) {
    __shared__ int s_start[kThreads / 32][32], s_pref[kThreads / 32][32];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (!(status[2] & mask)) return;  // the slab path built the list
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (FILL && offsets[n] > nnzcap) {
        if (gw == 0 && lane == 0) atomicOr(&status[0], (unsigned)ST_CAPACITY);
        return;
    }
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = gw; i < n; i += nwarps) {  // persistent: one warp per particle in turn
    const int inst = slot_inst(B, i);
    if (!slot_real(B, inst, i)) {
        if (!FILL && lane == 0) {
            rowlen[i] = 0;
            ngather[i] = 0;
        }
        continue;
    }
    const Grid* __restrict__ g = B.grid + inst;
    const int2* __restrict__ cl = cells + g->cbase;
    const unsigned long long* __restrict__ chm = cell_hmax + g->cbase;
    const double4_32a pi = posh[i];
    const float4 fi = fpos[i];
    const float tin_i = tin[i];
    const long long hib = __double_as_longlong(pi.w);
    const long long hgb = (long long)g->hmax_bits;
    const float Rbig = reach_f32(__longlong_as_double(hgb > hib ? hgb : hib));
    double R2i = -1.0;
    const unsigned lt = (1u << lane) - 1u;
    int64_t pg = 0, po = 0, pg_end = 0, po_end = 0;
    if (FILL) {
        pg = offsets[i];
        pg_end = po = pg + ngather[i];
        po_end = offsets[i + 1];
    }
    int cg = 0, co = 0;
    particle_pass<2>(g, cl, chm, fi, Rbig, hib, s_start[warp], s_pref[warp],
                        [&](bool valid, int j) {
        bool in_i = false, in_j = false;
        if (valid && j != i) {
            const float4 fj = __ldg(&fpos[j]);
            const float r2f = f_r2(fi, fj, g);
            bool bd_i = false;
            if (r2f < tin_i) in_i = true;
            else if (r2f <= fi.w) bd_i = true;
            double er2 = -1.0;
            if (bd_i) {
                if (R2i < 0.0) R2i = __dmul_rn(2.0 * pi.w, 2.0 * pi.w);
                er2 = exact_r2(pi, posh[j], g);
                in_i = er2 < R2i;
            }
            if (!in_i && r2f <= fj.w) {
                if (r2f < __ldg(&tin[j])) {
                    in_j = true;
                } else {
                    const double4_32a pj = posh[j];
                    if (er2 < 0.0) er2 = exact_r2(pi, pj, g);
                    const double Rj = 2.0 * pj.w;
                    in_j = er2 < __dmul_rn(Rj, Rj);
                }
            }
        }
        const unsigned gm = __ballot_sync(kFull, in_i);
        const unsigned om = __ballot_sync(kFull, in_j);
        if (FILL) {
            if (in_i) {
                const int64_t q = pg + cg + __popc(gm & lt);
                if (q < pg_end) idx[q] = j;
            } else if (in_j) {
                const int64_t q = po + co + __popc(om & lt);
                if (q < po_end) idx[q] = j;
            }
        }
        cg += __popc(gm);
        co += __popc(om);
    });
    if (!FILL && lane == 0) {
        rowlen[i] = cg + co;
        ngather[i] = cg;
    }
    }
}

void launch_h_search(sph_ctx* c, cudaStream_t s) {
    const int64_t n = c->n;
    if (n == 0) return;
    const unsigned nb = (unsigned)((n + kThreads - 1) / kThreads);
    double4_32a* posh = c->posh[c->cur];
    const Batch B = batch_of(c);
    c->launches += 4;
    if (c->any_lists) {
        c->launches += 1;
        k_h_lists<<<nb, kThreads, 0, s>>>(n, B, posh, c->fpos, c->nnb, c->ngather, c->rslab,
                                          c->hs_lo, c->hs_hi, c->hs_it, c->wl, c->status,
                                          c->order[c->cur], c->lst, c->lmeta);
    }
    const int64_t nbu = std::min<int64_t>((int64_t)c->nsm * kUnionBlocksPerSM, ((n + 31) / 32 + 7) / 8);
    if (c->any_lists) {
        k_h_union<true><<<(unsigned)nbu, kThreads, 0, s>>>(
            n, B, posh, c->fpos, c->cells, c->nnb, c->ngather, c->rslab, c->hs_lo, c->hs_hi,
            c->hs_it, c->wl, c->status, c->wctr, c->recs, c->order[c->cur], c->lst, c->lmeta);
        k_h_iterate<true><<<kReduceBlocks * 4, kThreads, 0, s>>>(
            B, posh, c->fpos, c->cells, c->nnb, c->ngather, c->rslab, c->hs_lo, c->hs_hi,
            c->hs_it, c->wl, c->status, c->order[c->cur], c->lst, c->lmeta);
    } else {
        k_h_union<false><<<(unsigned)nbu, kThreads, 0, s>>>(
            n, B, posh, c->fpos, c->cells, c->nnb, c->ngather, c->rslab, c->hs_lo, c->hs_hi,
            c->hs_it, c->wl, c->status, c->wctr, c->recs, c->order[c->cur], c->lst, c->lmeta);
        k_h_iterate<false><<<kReduceBlocks * 4, kThreads, 0, s>>>(
            B, posh, c->fpos, c->cells, c->nnb, c->ngather, c->rslab, c->hs_lo, c->hs_hi,
            c->hs_it, c->wl, c->status, c->order[c->cur], c->lst, c->lmeta);
    }
    k_finalize_h<<<nb, kThreads, 0, s>>>(n, B, posh, c->fpos, c->tin, c->ocnt, c->xpk);
    const unsigned gx = (unsigned)std::max(2, kReduceBlocks / c->ninst);
    k_cell_hmax<<<dim3(gx, (unsigned)c->ninst), kThreads, 0, s>>>(B, c->grid, c->cells, posh,
                                                                  c->cell_hmax);
}

// The two-pass CSR build, for the rows flagged in status[2] & mask (launched
// every step; without the flag its kernels return at once).
static void csr_fallback(sph_ctx* c, cudaStream_t s, unsigned mask) {
    const int64_t n = c->n;
    double4_32a* posh = c->posh[c->cur];
    const Batch B = batch_of(c);
    c->launches += 5;  // two build passes and the three kernels of the scan
    k_csr<false><<<kReduceBlocks * 4, kThreads, 0, s>>>(n, B, posh, c->fpos, c->tin, c->cells,
                                                        c->cell_hmax, c->rowlen, c->ngather,
                                                        nullptr, nullptr, c->nnzcap, c->status,
                                                        mask);
    launch_scan_i32_i64(c->rowlen, n, c->offsets, c->row_part, s, c->status + 2, mask);
    k_csr<true><<<kReduceBlocks * 4, kThreads, 0, s>>>(n, B, posh, c->fpos, c->tin, c->cells,
                                                       c->cell_hmax, c->rowlen, c->ngather,
                                                       c->offsets, c->idx, c->nnzcap, c->status,
                                                       mask);
}

void launch_csr(sph_ctx* c, cudaStream_t s, bool outer_later) {
    const int64_t n = c->n;
    c->csr_ready = false;
    if (n == 0) {
        c->launches += 1;
        cudaMemsetAsync(c->offsets, 0, sizeof(int64_t), s);
        return;
    }
    const unsigned nb = (unsigned)((n + kThreads - 1) / kThreads);
    const unsigned nbw = (unsigned)((n * 32 + kThreads - 1) / kThreads);
    double4_32a* posh = c->posh[c->cur];
    const Batch B = batch_of(c);
    if (!outer_later) {
        c->launches += 2;
        k_outer<<<nbw, kThreads, 0, s>>>(n, B, posh, c->fpos, c->tin, c->ngather, c->rslab,
                                         c->ocnt, c->status);
        k_rowlen_sort<<<nb, kThreads, 0, s>>>(n, c->ngather, c->ocnt, c->rowlen, c->rslab,
                                              c->status, (unsigned)IF_SLAB_OVF);
    }
    // fallback (a row did not fit its slab): the full two-pass build into the CSR
    csr_fallback(c, s, (unsigned)IF_SLAB_OVF);
}

// After a density kernel that recorded the outer entries: append and sort
// them, and build the CSR instead if one of them overflowed its slab.
void launch_rows_finish(sph_ctx* c, cudaStream_t s) {
    const int64_t n = c->n;
    if (n == 0) return;
    const unsigned nb = (unsigned)((n + kThreads - 1) / kThreads);
    c->launches += 2;
    k_append_outer<<<nb, kThreads, 0, s>>>(n, batch_of(c), c->omask, c->ngather, c->rslab,
                                           c->ocnt, c->status);
    k_rowlen_sort<<<nb, kThreads, 0, s>>>(n, c->ngather, c->ocnt, c->rowlen, c->rslab, c->status,
                                          (unsigned)(IF_SLAB_OVF | IF_OUTER_OVF));
    csr_fallback(c, s, (unsigned)IF_OUTER_OVF);
}

void launch_compose(sph_ctx* c, cudaStream_t s) {
    const int64_t n = c->n;
    c->csr_ready = true;
    if (n == 0) return;
    const unsigned nbw = (unsigned)((n * 32 + kThreads - 1) / kThreads);
    c->launches += 4;
    // row offsets of the slab rows (the steps scan them only for the fallback)
    launch_scan_i32_i64(c->rowlen, n, c->offsets, c->row_part, s);
    k_compose<<<nbw, kThreads, 0, s>>>(n, c->rowlen, c->rslab, c->offsets, c->idx, c->nnzcap,
                                       c->status);
}

}  // namespace sph
