// sph_abi.cu -- the extern "C" entry points declared in include/sph.h:
// argument checks, context allocation, and the launch sequence of each call.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "sph_internal.cuh"

using namespace sph;

namespace {

void set_err(sph_ctx* c, const char* fmt, ...) {
    if (!c) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
}

// Switch to the context's device for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

sph_status check_launch(sph_ctx* c, const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_err(c, "%s: %s", where, cudaGetErrorString(e));
        return SPH_E_CUDA;
    }
    return SPH_OK;
}

sph_status ensure_lists(sph_ctx* c);

sph_status check_params(sph_ctx* c, const sph_params* p) {
    if (!p) { set_err(c, "params is NULL"); return SPH_E_INVAL; }
    if (p->eos != 0 && p->eos != 1) { set_err(c, "eos must be 0 or 1"); return SPH_E_INVAL; }
    if (p->precision < 0 || p->precision > 2) {
        set_err(c, "precision must be 0 (FP64-accurate), 1 (mixed) or 2 (FP64 pipe)");
        return SPH_E_INVAL;
    }
    if (!(p->pair_threads == 0 || p->pair_threads == 1 || p->pair_threads == 2 ||
          p->pair_threads == 4 || p->pair_threads == 8)) {
        set_err(c, "pair_threads must be 0, 1, 2, 4 or 8");
        return SPH_E_INVAL;
    }
    if (p->defer_lanes < 0 || p->defer_lanes > 32) {
        set_err(c, "defer_lanes must be in [0, 32]");
        return SPH_E_INVAL;
    }
    if (p->max_h_iter < 1 || p->n_target < 1 || p->n_tol < 0) {
        set_err(c, "bad h-search parameters");
        return SPH_E_INVAL;
    }
    if (p->kernel < KER_M4 || p->kernel > KER_SINC) {
        set_err(c, "kernel must be 0 (M4), 1 (Wendland C2) or 2 (sinc)");
        return SPH_E_INVAL;
    }
    if (p->kernel == KER_SINC && (p->sinc_n < 2 || p->sinc_n > 12)) {
        set_err(c, "sinc_n must be in [2, 12]");
        return SPH_E_INVAL;
    }
    if (p->gradients != 0 && p->gradients != 1) {
        set_err(c, "gradients must be 0 (kernel derivatives) or 1 (IAD)");
        return SPH_E_INVAL;
    }
    if (p->precision == PREC_MIXED && (p->kernel != KER_M4 || p->gradients != 0)) {
        set_err(c, "the Table 1 variants need precision 0 or 2");
        return SPH_E_INVAL;
    }
    if (p->periodic_z && !(p->lz > 0.0)) { set_err(c, "periodic_z needs lz > 0"); return SPH_E_INVAL; }
    if (!(p->list_skin <= 1.0)) { set_err(c, "list_skin must be at most 1"); return SPH_E_INVAL; }
    if (!(p->cfl > 0.0)) { set_err(c, "cfl must be > 0"); return SPH_E_INVAL; }
    if (p->list_skin > 0.0) return ensure_lists(c);
    return SPH_OK;
}

sph_status check_particles(sph_ctx* c, const sph_particles* P) {
    if (!P) { set_err(c, "particles is NULL"); return SPH_E_INVAL; }
    if (P->n < 0 || P->n > c->ncap) {
        set_err(c, "n = %lld outside [0, capacity %lld]", (long long)P->n, (long long)c->ncap);
        return SPH_E_INVAL;
    }
    return SPH_OK;
}

#define NEED(ptr)                                              \
    do {                                                       \
        if (!(ptr)) {                                          \
            set_err(c, "required array " #ptr " is NULL");     \
            return SPH_E_INVAL;                                \
        }                                                      \
    } while (0)

template <class T>
bool dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, count * sizeof(T)) == cudaSuccess;
}

// The buffers of the h search's candidate lists, allocated (and cleared) by
// the first call whose parameters turn the lists on: kList entries and a
// 32-byte record per slot, ~800 B per particle of capacity.
sph_status ensure_lists(sph_ctx* c) {
    if (c->lmeta) return SPH_OK;
    const size_t N = (size_t)std::max<int64_t>(c->nslots, 1);
    DeviceGuard dg(c->device);
    const bool ok = dalloc(&c->lst, (N + 31) / 32 * 32 * kList) && dalloc(&c->lmeta, N) &&
                    dalloc(&c->lctr, 1) &&
                    cudaMemset(c->lmeta, 0, N * sizeof(LMeta)) == cudaSuccess &&
                    cudaMemset(c->lctr, 0, sizeof(unsigned)) == cudaSuccess &&
                    cudaDeviceSynchronize() == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        if (c->lst) cudaFree(c->lst);
        if (c->lmeta) cudaFree(c->lmeta);
        if (c->lctr) cudaFree(c->lctr);
        c->lst = nullptr;
        c->lmeta = nullptr;
        c->lctr = nullptr;
        set_err(c, "candidate lists: device allocation failed");
        return SPH_E_NOMEM;
    }
    return SPH_OK;
}

void free_all(sph_ctx* c) {
    void* ptrs[] = {c->posh[0], c->posh[1], c->velm[0], c->velm[1], c->ue[0], c->ue[1],
                    c->therm, c->kern, c->acc, c->pint, c->cint, c->dpk, c->mpk, c->mumax, c->fpos, c->tin, c->order[0],
                    c->order[1], c->keys[0], c->keys[1], c->vals[0], c->vals[1], c->hist,
                    c->hist_part, c->cells, c->cell_hmax, c->nnb, c->ngather, c->rowlen,
                    c->offsets, c->row_part, c->idx, c->rslab, c->ocnt, c->omask, c->hs_lo, c->hs_hi, c->hs_it, c->wl, c->red_part, c->dt_part, c->grid,
                    c->status, c->scratch_scalar, c->blk, c->ioff, c->icnt, c->coff, c->kpi,
                    c->tune_dt, c->roff, c->wctr, c->recs, c->iad_a, c->iad_b, c->vol, c->xpk, c->vpa, c->vpb,
                    c->stage, c->stage_nnb, c->vdf, c->cpk, c->lst, c->lmeta, c->lctr};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->status_host) cudaFreeHost(c->status_host);
}

// Record a timing marker closing `phase` (or opening a call when phase < 0).
void mark(sph_ctx* c, int phase, cudaStream_t s) {
    if (!c->timing) return;
    if (phase >= 0) c->phase_launches[phase] += c->launches - c->mark_launches;
    c->mark_launches = c->launches;
    if (c->ev_used >= c->ev_cap) return;  // pool full: later markers are dropped
    if (cudaEventRecord(c->ev[c->ev_used], s) != cudaSuccess) return;
    c->ev_phase[c->ev_used++] = phase;
}

void free_events(sph_ctx* c) {
    if (c->ev) {
        for (int k = 0; k < c->ev_cap; ++k) cudaEventDestroy(c->ev[k]);
        delete[] c->ev;
        delete[] c->ev_phase;
    }
    c->ev = nullptr;
    c->ev_phase = nullptr;
    c->ev_cap = c->ev_used = 0;
}

// per-instance budgets instance_cell_cap(n_k) sum to at most this
int64_t cell_capacity(int64_t ncap, int64_t max_instances) {
    return std::min<int64_t>(2 * ncap + (int64_t)kMinInstanceCells * max_instances,
                             max_instances * kMaxCellsPerAxis * kMaxCellsPerAxis *
                                 kMaxCellsPerAxis);
}

// Device allocations of a context, listed once: with dry = true only their
// total size is computed (sph_ctx_bytes).
struct Allocator {
    bool dry;
    size_t bytes;
    template <class T>
    bool operator()(T** p, size_t count) {
        if (count == 0) count = 1;
        bytes += (count * sizeof(T) + 255) / 256 * 256;
        if (dry) {
            *p = nullptr;
            return true;
        }
        return dalloc(p, count);
    }
};

bool allocate_all(sph_ctx* c, int64_t nslots, Allocator& al) {
    const int64_t max_instances = c->maxinst;
    const int64_t nnzcap = c->nnzcap;
    const size_t N = (size_t)std::max<int64_t>(nslots, 1);
    const size_t nsb = (N + kRadixTile - 1) / kRadixTile;
    const size_t nfb = (N + kThreads - 1) / kThreads;
    bool ok = true;
    for (int b = 0; b < 2; ++b) {
        ok = ok && al(&c->posh[b], N) && al(&c->velm[b], N) && al(&c->ue[b], N) &&
             al(&c->order[b], N) && al(&c->keys[b], N) && al(&c->vals[b], N);
    }
    ok = ok && al(&c->therm, N) && al(&c->kern, N) && al(&c->acc, N) &&
         al(&c->pint, N) && al(&c->cint, N) && al(&c->dpk, 3 * N) &&
         al(&c->xpk, 3 * N) && al(&c->vpa, N) && al(&c->vpb, N) && al(&c->mpk, 5 * N) &&
         al(&c->mumax, N) && al(&c->iad_a, N) && al(&c->iad_b, N) && al(&c->vol, N) && al(&c->vdf, N) &&
         al(&c->cpk, 3 * N) &&
         al(&c->fpos, N) && al(&c->tin, N) &&
         al(&c->hist, 256 * nsb) && al(&c->hist_part, (size_t)scan_parts(256 * nsb) + 1) &&
         al(&c->cells, (size_t)c->cellcap) && al(&c->cell_hmax, (size_t)c->cellcap) &&
         al(&c->nnb, N) && al(&c->ngather, N) && al(&c->rowlen, N) &&
         al(&c->offsets, N + 1) && al(&c->row_part, (size_t)scan_parts(N) + 1) &&
         al(&c->idx, (size_t)nnzcap) && al(&c->red_part, (N + kSlotAlign - 1) / kSlotAlign * kBoxStride) &&
         al(&c->dt_part, nfb * kMaxPairThreads) && al(&c->grid, (size_t)max_instances) &&
         al(&c->status, 4) && al(&c->blk, nfb) &&
         al(&c->ioff, (size_t)max_instances + 1) && al(&c->icnt, (size_t)max_instances) &&
         al(&c->coff, (size_t)max_instances + 1) && al(&c->kpi, (size_t)max_instances) &&
         al(&c->roff, (size_t)max_instances + 1) &&
         al(&c->rslab, N * kRSlab) && al(&c->ocnt, N) && al(&c->omask, 2 * N) &&
         al(&c->hs_lo, N) && al(&c->hs_hi, N) && al(&c->hs_it, N) && al(&c->wl, N) &&
         al(&c->scratch_scalar, 2) && al(&c->tune_dt, 2 * (size_t)max_instances) &&
         al(&c->wctr, 4) &&
         al(&c->recs, (size_t)c->nsm * kUnionBlocksPerSM * kThreads * kRec);
    return ok;
}

}  // namespace

namespace sph {

// B_n = 1 / (4 pi int_0^2 q^2 (sin x / x)^n dq), x = pi q / 2, by 16-point
// Gauss-Legendre quadrature on 64 equal panels (the integrand is analytic, so
// this is exact to rounding). The nodes are the roots of the Legendre
// polynomial P_16, found by Newton's method on its three-term recurrence
// (k P_k = (2k - 1) t P_{k-1} - (k - 1) P_{k-2}) from the Chebyshev-like
// guesses cos(pi (i - 1/4) / (m + 1/2)); the weights are
// 2 / ((1 - t^2) P_16'(t)^2).
double sinc_norm(int n) {
    constexpr int m = 16, panels = 64;
    double t[m], w[m];
    for (int i = 0; i < m; ++i) {
        double z = cos(kPi * (i + 0.75) / (m + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= m; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = m * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        t[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    const double hp = 2.0 / panels;
    double sum = 0.0;
    for (int a = 0; a < panels; ++a) {
        double ps = 0.0;
        for (int i = 0; i < m; ++i) {
            const double q = hp * (a + 0.5 * (t[i] + 1.0));
            const double x = 0.5 * kPi * q;
            const double sx = sin(x) / x;
            double pw = 1.0;
            for (int e = 0; e < n; ++e) pw *= sx;
            ps += w[i] * q * q * pw;
        }
        sum += 0.5 * hp * ps;
    }
    return 1.0 / (4.0 * kPi * sum);
}

// Batch-of-one descriptors for a single problem of n particles, written on the
// stream (kernel arguments are captured at launch, so back-to-back calls with
// different parameters cannot overwrite each other's).
__global__ void __launch_bounds__(kThreads)
k_set_single(KParams kp, int64_t n, long long cap, int64_t nblk, int32_t* __restrict__ blk,
             int64_t* __restrict__ ioff, int64_t* __restrict__ icnt, int64_t* __restrict__ coff,
             int64_t* __restrict__ roff, KParams* __restrict__ kpi, Grid* __restrict__ grid) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t b = t; b < nblk; b += (int64_t)gridDim.x * blockDim.x) blk[b] = 0;
    if (t == 0) {
        kpi[0] = kp;
        ioff[0] = 0;
        ioff[1] = n;
        icnt[0] = n;
        coff[0] = 0;
        coff[1] = n;
        roff[0] = 0;
        roff[1] = n;
        grid[0].cbase = 0;
        grid[0].cap = cap;
    }
}

// The candidate lists of the h search and their records belong to an
// instance's caller range: an instance whose range (first, count) was not one
// of the previous batch's starts without them (its records are cleared, so
// its next step builds its lists). A range kept from one call to the next
// keeps its lists; whether they still hold is checked on the device.
// [first, first + count) is a non-empty range within [0, the capacity)
// (compared without forming first + count, which could overflow).
static bool in_capacity(const sph_ctx* c, int64_t first, int64_t count) {
    return count > 0 && first >= 0 && count <= c->ncap && first <= c->ncap - count;
}

void lists_for_layout(sph_ctx* c, int ninst, const int64_t* first, const int64_t* cnt,
                      cudaStream_t s) {
    for (int k = 0; k < ninst && c->lmeta; ++k) {
        bool seen = false;
        for (int q = 0; q < c->lay_n && !seen; ++q)
            seen = c->lay_first[q] == first[k] && c->lay_cnt[q] == cnt[k];
        if (!seen && in_capacity(c, first[k], cnt[k]))
            cudaMemsetAsync(c->lmeta + first[k], 0, (size_t)cnt[k] * sizeof(LMeta), s);
    }
    c->lay_n = ninst;
    for (int k = 0; k < ninst; ++k) {
        c->lay_first[k] = first[k];
        c->lay_cnt[k] = cnt[k];
    }
}

// Clear the list records of every instance of the current layout (their next
// step builds).
void lists_clear(sph_ctx* c, cudaStream_t s) {
    for (int k = 0; k < c->lay_n && c->lmeta; ++k)
        if (in_capacity(c, c->lay_first[k], c->lay_cnt[k]))
            cudaMemsetAsync(c->lmeta + c->lay_first[k], 0, (size_t)c->lay_cnt[k] * sizeof(LMeta), s);
}

void launch_set_single(sph_ctx* c, const KParams& kp, int64_t n, cudaStream_t s) {
    const int64_t zero = 0;
    lists_for_layout(c, 1, &zero, &n, s);
    c->any_lists = kp.list_skin > 0.0;
    c->n = n;
    c->ntot = n;
    c->cext = n;
    c->ninst = 1;
    c->prec = kp.precision;
    c->kern_kind = kp.kernel;
    c->grad_kind = kp.gradients;
    c->tpp = native_pairs(c) ? 1 : kp.pair_threads;
    const int64_t nblk = (n + kSlotAlign - 1) / kSlotAlign;
    const unsigned nb = (unsigned)std::min<int64_t>(std::max<int64_t>((nblk + kThreads - 1) / kThreads, 1), 1024);
    c->launches += 1;
    k_set_single<<<nb, kThreads, 0, s>>>(kp, n, instance_cell_cap(n), nblk, c->blk, c->ioff,
                                         c->icnt, c->coff, c->roff, c->kpi, c->grid);
}

// One step of the current batch on the state held in the context (Algorithm
// 1 steps 1-6); dt and time are device arrays of ninst entries.
void launch_step(sph_ctx* c, double* dt, double* time, cudaStream_t s) {
    launch_build_cells(c, s);
    mark(c, SPH_PHASE_CELLS, s);
    launch_h_search(c, s);
    mark(c, SPH_PHASE_HSEARCH, s);
    // at precision 0 the density kernel completes the rows (outer parts)
    const bool fo = fused_outer(c);
    launch_csr(c, s, fo);
    mark(c, SPH_PHASE_CSR, s);
    launch_density(c, true, s, fo);
    mark(c, SPH_PHASE_DENSITY, s);
    if (fo) {
        launch_rows_finish(c, s);
        mark(c, SPH_PHASE_CSR, s);
    }
    launch_forces(c, dt, time, s);
    mark(c, SPH_PHASE_FORCES, s);
    launch_leapfrog(c, dt, s);
}

void drop_step_graphs(sph_ctx* c) {
    for (auto& g : c->sg) {
        if (g.valid) cudaGraphExecDestroy(g.exec);
        g.valid = false;
    }
}

// One step of the current batch through the cached graph of its parity,
// captured (on the context's private stream) when missing or when anything
// the launches bake in has changed. Returns false, with nothing enqueued,
// when a graph cannot be made or launched: the caller then launches the step
// directly. Replaying gives the same kernels in the same order as launching
// them, so the results are the same bits.
bool step_graph(sph_ctx* c, double* dt, double* time, cudaStream_t s) {
    const int par = c->cur;
    const int64_t key[10] = {c->n, c->ntot, c->ninst, c->prec, c->tpp, c->kern_kind, c->grad_kind,
                             (int64_t)(intptr_t)dt, (int64_t)(intptr_t)time, c->any_lists ? 1 : 0};
    sph_ctx::StepGraph& g = c->sg[par];
    if (!g.valid || memcmp(g.key, key, sizeof key) != 0) {
        if (g.valid) cudaGraphExecDestroy(g.exec);
        g.valid = false;
        if (!c->gstream && cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking) != cudaSuccess) {
            c->gstream = nullptr;
            cudaGetLastError();
            return false;
        }
        const int64_t l0 = c->launches;
        if (cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        launch_step(c, dt, time, c->gstream);  // recorded, not run
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->gstream, &graph);
        const int64_t nl = c->launches - l0;
        c->launches = l0;
        c->cur = par;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        g.valid = true;
        g.launches = nl;
        memcpy(g.key, key, sizeof key);
    }
    if (cudaGraphLaunch(g.exec, s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    c->cur = 1 - par;  // what the step's sort does to the state buffers
    c->launches += g.launches;
    c->csr_ready = false;
    return true;
}

// nsteps steps of the current batch: the caller's arrays (those of `in` when
// given, else P's) are read into the slot layout, and the final state is
// written back to P's after the last step.
// Each step replays the step graph of its parity, unless per-phase timing is
// on (events between the phases) or the stream is being captured already
// (the caller is recording the launches into a graph of its own).
void run_steps(sph_ctx* c, sph_particles* P, int nsteps, cudaStream_t s,
               const sph_particles* in = nullptr) {
    mark(c, -1, s);
    launch_load_state(c, in ? in : P, s);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;  // unknown: launch directly
    }
    const bool graphs = !c->timing && c->n > 0 && cs == cudaStreamCaptureStatusNone;
    for (int k = 0; k < nsteps; ++k) {
        if (!(graphs && step_graph(c, P->dt, P->time, s))) launch_step(c, P->dt, P->time, s);
        if (k == nsteps - 1)
            launch_scatter(c, P, SC_POS | SC_VEL | SC_H | SC_U | SC_RHO | SC_PC | SC_ACC |
                                     SC_MUMAX | SC_NNB, s);
        mark(c, SPH_PHASE_UPDATE, s);
        if (c->timing) c->timed_steps += 1;
    }
}

// Device buffers out to host memory that the GPU reaches in place
// (blockIdx.y = buffer). Every buffer is an array of doubles or int32: 16-byte
// loads and stores where both ends are 16-byte aligned, else 4-byte words.
// Four loads go out before their stores, so each thread keeps several
// transfers over the host link in flight.
constexpr int kHostCopyMax = 20;
struct HostCopy {
    const void* src[kHostCopyMax];
    void* dst[kHostCopyMax];
    int64_t bytes[kHostCopyMax];
};

template <typename T>
__device__ __forceinline__ void copy_strided(const T* __restrict__ s, T* __restrict__ d, int64_t n,
                                             int64_t t, int64_t st) {
    int64_t i = t;
    for (; i + 3 * st < n; i += 4 * st) {
        const T a = s[i], b = s[i + st], e = s[i + 2 * st], f = s[i + 3 * st];
        d[i] = a;
        d[i + st] = b;
        d[i + 2 * st] = e;
        d[i + 3 * st] = f;
    }
    for (; i < n; i += st) d[i] = s[i];
}

__global__ void __launch_bounds__(kThreads) k_to_host(HostCopy C) {
    const int f = blockIdx.y;
    const char* s = (const char*)C.src[f];
    char* d = (char*)C.dst[f];
    const int64_t nb = C.bytes[f];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t st = (int64_t)gridDim.x * blockDim.x;
    int64_t done = 0;
    if ((((uintptr_t)s | (uintptr_t)d) & 15) == 0) {
        done = nb & ~(int64_t)15;
        copy_strided((const int4*)s, (int4*)d, done >> 4, t, st);
    }
    copy_strided((const int32_t*)(s + done), (int32_t*)(d + done), (nb - done) >> 2, t, st);
}

void launch_to_host(sph_ctx* c, const HostCopy& C, int nbuf, int64_t maxbytes, cudaStream_t s) {
    if (nbuf == 0) return;
    const int64_t per_block = (int64_t)kThreads * 4 * 16;
    const int64_t want = std::max<int64_t>(1, (maxbytes + per_block - 1) / per_block);
    const int64_t cap = std::max(1, 16 * 152 / nbuf);
    c->launches += 1;
    k_to_host<<<dim3((unsigned)std::min(want, cap), (unsigned)nbuf), kThreads, 0, s>>>(C);
}

}  // namespace sph

extern "C" {

int64_t sph_launch_count(const sph_ctx* c) { return c ? c->launches : 0; }

int64_t sph_neighbor_rows(const sph_ctx* c) { return c ? c->n : 0; }

sph_status sph_lists_clear(sph_ctx* c, int64_t first, int64_t count, void* stream) {
    if (!c) return SPH_E_INVAL;
    if (first < 0 || count < 0 || first > c->ncap || count > c->ncap - first) {
        set_err(c, "sph_lists_clear: %lld entries from %lld outside [0, %lld)", (long long)count,
                (long long)first, (long long)c->ncap);
        return SPH_E_INVAL;
    }
    if (count == 0 || !c->lmeta) return SPH_OK;  // no lists yet: nothing to forget
    DeviceGuard dg(c->device);
    const cudaError_t e = cudaMemsetAsync(c->lmeta + first, 0, (size_t)count * sizeof(LMeta),
                                          (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_err(c, "sph_lists_clear: %s", cudaGetErrorString(e));
        return SPH_E_CUDA;
    }
    return SPH_OK;
}

sph_status sph_list_builds(sph_ctx* c, int64_t* builds, void* stream) {
    if (!c || !builds) return SPH_E_INVAL;
    *builds = 0;
    if (!c->lctr) return SPH_OK;  // lists never turned on
    DeviceGuard dg(c->device);
    unsigned v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, c->lctr, sizeof v, cudaMemcpyDeviceToHost,
                                    (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_err(c, "sph_list_builds: %s", cudaGetErrorString(e));
        return SPH_E_CUDA;
    }
    *builds = (int64_t)v;
    return SPH_OK;
}

sph_status sph_timing_enable(sph_ctx* c, int enable) {
    if (!c) return SPH_E_INVAL;
    DeviceGuard dg(c->device);
    free_events(c);
    c->timing = 0;
    memset(c->phase_launches, 0, sizeof(c->phase_launches));
    c->timed_steps = 0;
    c->mark_launches = c->launches;
    if (!enable) return SPH_OK;
    const int cap = 8 * 1024;
    c->ev = new (std::nothrow) cudaEvent_t[cap];
    c->ev_phase = new (std::nothrow) int[cap];
    if (!c->ev || !c->ev_phase) {
        delete[] c->ev;
        delete[] c->ev_phase;
        c->ev = nullptr;
        c->ev_phase = nullptr;
        return SPH_E_NOMEM;
    }
    for (int k = 0; k < cap; ++k) {
        if (cudaEventCreate(&c->ev[k]) != cudaSuccess) {
            c->ev_cap = k;
            free_events(c);
            cudaGetLastError();
            set_err(c, "cudaEventCreate failed");
            return SPH_E_CUDA;
        }
    }
    c->ev_cap = cap;
    c->timing = 1;
    return SPH_OK;
}

sph_status sph_timing_read(sph_ctx* c, double* ms, int64_t* launches, int64_t* steps) {
    if (!c) return SPH_E_INVAL;
    DeviceGuard dg(c->device);
    double acc[SPH_NPHASES] = {0};
    if (c->ev_used > 0 && cudaEventSynchronize(c->ev[c->ev_used - 1]) != cudaSuccess) {
        cudaGetLastError();
        set_err(c, "sph_timing_read: event wait failed");
        return SPH_E_CUDA;
    }
    for (int k = 1; k < c->ev_used; ++k) {
        const int ph = c->ev_phase[k];
        if (ph < 0) continue;
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, c->ev[k - 1], c->ev[k]) == cudaSuccess) acc[ph] += t;
        else cudaGetLastError();
    }
    for (int p = 0; p < SPH_NPHASES; ++p) {
        if (ms) ms[p] = acc[p];
        if (launches) launches[p] = c->phase_launches[p];
    }
    if (steps) *steps = c->timed_steps;
    c->ev_used = 0;
    memset(c->phase_launches, 0, sizeof(c->phase_launches));
    c->timed_steps = 0;
    c->mark_launches = c->launches;
    return SPH_OK;
}

const char* sph_version(void) { return "libsph 0.1 (sm_103a, FP64)"; }

const char* sph_last_error(const sph_ctx* c) { return c ? c->err : "context is NULL"; }

int64_t sph_last_hnoconv(const sph_ctx* c) { return c ? c->last_hnoconv : 0; }

int64_t sph_ctx_bytes(int64_t ncap, int64_t nnzcap, int32_t max_instances) {
    if (ncap < 0 || ncap > (int64_t)INT32_MAX || nnzcap < 0 || max_instances < 1 ||
        max_instances > SPH_MAX_INSTANCES)
        return -1;
    sph_ctx c;
    memset(&c, 0, sizeof(c));
    c.ncap = ncap;
    c.nnzcap = nnzcap;
    c.maxinst = max_instances;
    c.cellcap = cell_capacity(ncap, max_instances);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c.nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        c.nsm < 1) {
        cudaGetLastError();
        c.nsm = 256;  // no device to ask: an upper bound for the per-SM scratch
    }
    Allocator A{true, 0};
    allocate_all(&c, ncap + (int64_t)(kSlotAlign - 1) * (max_instances - 1), A);
    return (int64_t)A.bytes;
}

sph_status sph_ctx_create(sph_ctx** out, int64_t ncap, int64_t nnzcap, int device) {
    return sph_ctx_create_batch(out, ncap, nnzcap, 1, device);
}

sph_status sph_ctx_create_batch(sph_ctx** out, int64_t ncap, int64_t nnzcap, int32_t max_instances,
                                int device) {
    if (!out) return SPH_E_INVAL;
    *out = nullptr;
    if (max_instances < 1 || max_instances > SPH_MAX_INSTANCES) return SPH_E_INVAL;
    if (ncap < 0 || ncap > (int64_t)INT32_MAX || nnzcap < 0 || nnzcap > ((int64_t)1 << 40))
        return SPH_E_INVAL;
    // slots: the particles plus the gaps that start every instance on a block boundary
    const int64_t nslots = ncap + (int64_t)(kSlotAlign - 1) * (max_instances - 1);
    if (nslots > (int64_t)INT32_MAX - 1) return SPH_E_INVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return SPH_E_CUDA;
    }
    DeviceGuard dg(device);
    if (!dg.ok) return SPH_E_CUDA;
    sph_ctx* c = new (std::nothrow) sph_ctx;
    if (!c) return SPH_E_NOMEM;
    memset(c, 0, sizeof(*c));
    c->device = device;
    c->ncap = ncap;
    c->nnzcap = nnzcap;
    c->maxinst = max_instances;
    c->ninst = 1;
    c->cellcap = cell_capacity(ncap, max_instances);
    c->nslots = nslots;
    if (cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        c->nsm < 1) {
        cudaGetLastError();
        c->nsm = 1;
    }
    Allocator A{false, 0};
    bool ok = allocate_all(c, nslots, A);
    ok = ok && cudaMallocHost((void**)&c->status_host, 2 * sizeof(unsigned)) == cudaSuccess;
    ok = ok && cudaMemset(c->status, 0, 4 * sizeof(unsigned)) == cudaSuccess &&
         cudaMemset(c->offsets, 0, sizeof(int64_t)) == cudaSuccess &&
         cudaMemset(c->grid, 0, (size_t)max_instances * sizeof(Grid)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return SPH_E_NOMEM;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return SPH_E_CUDA;
    }
    *out = c;
    return SPH_OK;
}

void sph_ctx_destroy(sph_ctx* c) {
    if (!c) return;
    DeviceGuard dg(c->device);
    cudaDeviceSynchronize();
    drop_step_graphs(c);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    free_events(c);
    free_all(c);
    delete c;
}

sph_status sph_build_neighbors(sph_ctx* c, const sph_params* prm, sph_particles* P,
                               sph_neighbors* out, void* stream) {
    if (!c) return SPH_E_INVAL;
    sph_status st;
    if ((st = check_params(c, prm)) != SPH_OK || (st = check_particles(c, P)) != SPH_OK) return st;
    if (P->n > 0) { NEED(P->x); NEED(P->y); NEED(P->z); NEED(P->h); }
    DeviceGuard dg(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const KParams kp = kparams(prm);
    launch_set_single(c, kp, P->n, s);
    launch_load_state(c, P, s);
    launch_build_cells(c, s);
    launch_h_search(c, s);
    launch_csr(c, s);
    launch_compose(c, s);
    launch_scatter(c, P, SC_H | SC_NNB, s);
    if ((st = check_launch(c, "sph_build_neighbors")) != SPH_OK) return st;
    if (out) {
        out->n = c->n;
        out->offsets = c->offsets;
        out->idx = c->idx;
        out->ngather = c->ngather;
        out->order = c->order[c->cur];
        out->nnz_dev = c->offsets + c->n;
    }
    return SPH_OK;
}

static sph_status need_build(sph_ctx* c, const sph_particles* P) {
    if (c->ninst != 1) {
        set_err(c, "the last build was a batch of %d instances: use sph_batch_step", c->ninst);
        return SPH_E_INVAL;
    }
    if (P->n != c->n) {
        set_err(c, "n = %lld differs from the last sph_build_neighbors (n = %lld)",
                (long long)P->n, (long long)c->n);
        return SPH_E_INVAL;
    }
    return SPH_OK;
}

sph_status sph_density(sph_ctx* c, const sph_params* prm, sph_particles* P, void* stream) {
    if (!c) return SPH_E_INVAL;
    sph_status st;
    if ((st = check_params(c, prm)) != SPH_OK || (st = check_particles(c, P)) != SPH_OK ||
        (st = need_build(c, P)) != SPH_OK)
        return st;
    if (P->n > 0) { NEED(P->x); NEED(P->y); NEED(P->z); NEED(P->h); NEED(P->m); NEED(P->rho); }
    DeviceGuard dg(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const KParams kp = kparams(prm);
    launch_set_single(c, kp, P->n, s);
    launch_gather_state(c, P, kp, GATHER_DENSITY, s);
    launch_density(c, false, s);
    launch_scatter(c, P, SC_RHO, s);
    return check_launch(c, "sph_density");
}

sph_status sph_eos(sph_ctx* c, const sph_params* prm, sph_particles* P, void* stream) {
    if (!c) return SPH_E_INVAL;
    sph_status st;
    if ((st = check_params(c, prm)) != SPH_OK || (st = check_particles(c, P)) != SPH_OK) return st;
    if (P->n > 0) {
        NEED(P->rho); NEED(P->p); NEED(P->c);
        if (prm->eos == 1) NEED(P->u);
    }
    DeviceGuard dg(c->device);
    launch_eos_caller(kparams(prm), P, (cudaStream_t)stream);
    return check_launch(c, "sph_eos");
}

sph_status sph_forces(sph_ctx* c, const sph_params* prm, sph_particles* P, void* stream) {
    if (!c) return SPH_E_INVAL;
    sph_status st;
    if ((st = check_params(c, prm)) != SPH_OK || (st = check_particles(c, P)) != SPH_OK ||
        (st = need_build(c, P)) != SPH_OK)
        return st;
    NEED(P->dt);
    if (P->n > 0) {
        NEED(P->x); NEED(P->y); NEED(P->z); NEED(P->vx); NEED(P->vy); NEED(P->vz);
        NEED(P->m); NEED(P->h); NEED(P->rho); NEED(P->p); NEED(P->c);
        NEED(P->ax); NEED(P->ay); NEED(P->az); NEED(P->du);
    }
    DeviceGuard dg(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const KParams kp = kparams(prm);
    launch_set_single(c, kp, P->n, s);
    launch_gather_state(c, P, kp, GATHER_FORCES, s);
    if (kp.precision == PREC_MIXED) launch_pack_mx(c, true, s);
    launch_forces(c, P->dt, nullptr, s);
    launch_scatter(c, P, SC_ACC | SC_MUMAX, s);
    return check_launch(c, "sph_forces");
}

sph_status sph_step(sph_ctx* c, const sph_params* prm, sph_particles* P, int nsteps,
                    void* stream) {
    if (!c) return SPH_E_INVAL;
    sph_status st;
    if ((st = check_params(c, prm)) != SPH_OK || (st = check_particles(c, P)) != SPH_OK) return st;
    if (nsteps < 0) { set_err(c, "nsteps < 0"); return SPH_E_INVAL; }
    NEED(P->dt); NEED(P->time);
    if (P->n > 0) {
        NEED(P->x); NEED(P->y); NEED(P->z); NEED(P->vx); NEED(P->vy); NEED(P->vz);
        NEED(P->m); NEED(P->h); NEED(P->u); NEED(P->rho); NEED(P->p); NEED(P->c);
        NEED(P->ax); NEED(P->ay); NEED(P->az); NEED(P->du);
    }
    DeviceGuard dg(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    launch_set_single(c, kparams(prm), P->n, s);
    run_steps(c, P, nsteps, s);
    return check_launch(c, "sph_step");
}

// The device address of a host array the GPU can reach in place (page-locked
// or registered host memory, or managed memory), else NULL (pageable memory,
// or nothing known about the pointer).
static void* device_view(const void* p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeManaged) ? a.devicePointer
                                                                              : nullptr;
}

sph_status sph_step_host(sph_ctx* c, const sph_params* prm, sph_particles* H, int nsteps,
                         void* stream) {
    if (!c) return SPH_E_INVAL;
    sph_status st;
    if ((st = check_params(c, prm)) != SPH_OK || (st = check_particles(c, H)) != SPH_OK) return st;
    if (nsteps < 0) { set_err(c, "nsteps < 0"); return SPH_E_INVAL; }
    NEED(H->dt); NEED(H->time);
    const int64_t n = H->n;
    if (n > 0) {
        NEED(H->x); NEED(H->y); NEED(H->z); NEED(H->vx); NEED(H->vy); NEED(H->vz);
        NEED(H->m); NEED(H->h); NEED(H->u);
    }
    if (nsteps == 0) return SPH_OK;
    DeviceGuard dg(c->device);
    const size_t N = (size_t)std::max<int64_t>(c->ncap, 1);
    if (!c->stage) {
        if (cudaMalloc((void**)&c->stage, (17 * N + 2) * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void**)&c->stage_nnb, N * sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            if (c->stage) cudaFree(c->stage);
            c->stage = nullptr;
            c->stage_nnb = nullptr;
            set_err(c, "sph_step_host: staging allocation failed");
            return SPH_E_NOMEM;
        }
    }
    // Device view D: the staging buffer, the state fields first (in and out),
    // then the outputs. The inputs I: a state array the GPU reaches in place
    // (pinned host memory) is read by the call's first kernel directly, in the
    // caller's order, over the host link; any other is copied to D's buffer
    // first. The last step writes every output through the sort permutation
    // into D (scattered 8-byte stores to host memory would waste most of each
    // transfer); from there one copy kernel streams the pinned arrays out over
    // the link, and the copy engines take the others.
    double* sg = c->stage;
    double** hf[17] = {&H->x, &H->y, &H->z, &H->vx, &H->vy, &H->vz, &H->m, &H->h, &H->u,
                       &H->rho, &H->p, &H->c, &H->ax, &H->ay, &H->az, &H->du, &H->mumax};
    sph_particles D;
    memset(&D, 0, sizeof D);
    D.n = n;
    double** df[17] = {&D.x, &D.y, &D.z, &D.vx, &D.vy, &D.vz, &D.m, &D.h, &D.u,
                       &D.rho, &D.p, &D.c, &D.ax, &D.ay, &D.az, &D.du, &D.mumax};
    void* view[17];
    for (int f = 0; f < 17; ++f) {
        view[f] = n > 0 ? device_view(*hf[f]) : nullptr;
        *df[f] = sg + (size_t)f * N;
    }
    if (!H->mumax) D.mumax = nullptr;
    D.nnb = H->nnb ? c->stage_nnb : nullptr;
    void* nnb_view = n > 0 ? device_view(H->nnb) : nullptr;
    D.time = sg + 17 * N;
    D.dt = sg + 17 * N + 1;
    sph_particles I = D;
    double** in[9] = {&I.x, &I.y, &I.z, &I.vx, &I.vy, &I.vz, &I.m, &I.h, &I.u};
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = (size_t)n * sizeof(double);
    cudaError_t e = cudaSuccess;
    for (int f = 0; f < 9 && e == cudaSuccess && n > 0; ++f) {
        if (view[f]) *in[f] = (double*)view[f];
        else e = cudaMemcpyAsync(*df[f], *hf[f], bytes, cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(D.time, H->time, sizeof(double), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_err(c, "sph_step_host: %s", cudaGetErrorString(e));
        return SPH_E_CUDA;
    }
    launch_set_single(c, kparams(prm), n, s);
    run_steps(c, &D, nsteps, s, &I);
    HostCopy hc;
    int nhc = 0;
    for (int f = 0; f < 17 && e == cudaSuccess && n > 0; ++f) {
        if (!*hf[f] || f == 6) continue;  // m is read, never written
        if (view[f]) {
            hc.src[nhc] = *df[f];
            hc.dst[nhc] = view[f];
            hc.bytes[nhc++] = (int64_t)bytes;
        } else {
            e = cudaMemcpyAsync(*hf[f], *df[f], bytes, cudaMemcpyDeviceToHost, s);
        }
    }
    if (e == cudaSuccess && H->nnb && n > 0) {
        if (nnb_view) {
            hc.src[nhc] = D.nnb;
            hc.dst[nhc] = nnb_view;
            hc.bytes[nhc++] = n * (int64_t)sizeof(int32_t);
        } else {
            e = cudaMemcpyAsync(H->nnb, D.nnb, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        }
    }
    if (e == cudaSuccess) launch_to_host(c, hc, nhc, (int64_t)bytes, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(H->time, D.time, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(H->dt, D.dt, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_err(c, "sph_step_host: %s", cudaGetErrorString(e));
        return SPH_E_CUDA;
    }
    return check_launch(c, "sph_step_host");
}

static sph_status batch_set(sph_ctx* c, int32_t ninst, const int64_t* counts, const int64_t* first,
                            const sph_params* params, void* stream);

// (the host tables of a batch are std::vector: no exception leaves the ABI)
sph_status sph_batch_set(sph_ctx* c, int32_t ninst, const int64_t* counts, const int64_t* first,
                         const sph_params* params, void* stream) {
    if (!c) return SPH_E_INVAL;
    try {
        return batch_set(c, ninst, counts, first, params, stream);
    } catch (const std::bad_alloc&) {
        set_err(c, "sph_batch_set: host memory for the batch tables");
        return SPH_E_NOMEM;
    }
}

static sph_status batch_set(sph_ctx* c, int32_t ninst, const int64_t* counts, const int64_t* first,
                            const sph_params* params, void* stream) {
    if (ninst < 1 || ninst > c->maxinst || !counts || !params) {
        set_err(c, "ninst = %d outside [1, %d] or NULL arrays", (int)ninst, c->maxinst);
        return SPH_E_INVAL;
    }
    std::vector<int64_t> ioff(ninst + 1), coff(ninst + 1), roff(ninst + 1), icnt(ninst);
    std::vector<KParams> kpi(ninst);
    std::vector<Grid> grid(ninst);
    int64_t slots = 0, tot = 0;
    long long cells = 0;
    for (int k = 0; k < ninst; ++k) {
        sph_status st = check_params(c, &params[k]);
        if (st != SPH_OK) return st;
        if (params[k].precision != params[0].precision ||
            params[k].pair_threads != params[0].pair_threads ||
            params[k].kernel != params[0].kernel || params[k].gradients != params[0].gradients ||
            (params[k].kernel == KER_SINC && params[k].sinc_n != params[0].sinc_n)) {
            set_err(c, "instances of a batch must share precision, pair_threads, kernel, "
                       "gradients and sinc_n");
            return SPH_E_INVAL;
        }
        if (counts[k] < 0) {
            set_err(c, "counts[%d] < 0", k);
            return SPH_E_INVAL;
        }
        if (first && first[k] < 0) {
            set_err(c, "first[%d] < 0", k);
            return SPH_E_INVAL;
        }
        // caller indices are held as int32: every instance ends below 2^31
        // (compared without forming first + count, which could overflow)
        if (counts[k] > (int64_t)INT32_MAX || (first && first[k] > (int64_t)INT32_MAX - counts[k])) {
            set_err(c, "instance %d reaches past 2^31 - 1 caller entries", k);
            return SPH_E_INVAL;
        }
        ioff[k] = slots;
        roff[k] = tot;
        coff[k] = first ? first[k] : tot;
        icnt[k] = counts[k];
        tot += counts[k];
        slots += counts[k];
        if (k + 1 < ninst) slots = (slots + kSlotAlign - 1) / kSlotAlign * kSlotAlign;
        kpi[k] = kparams(&params[k]);
        // the candidate lists' records are kept by caller index, up to the capacity
        // (compared without forming coff + count, which could overflow)
        if (counts[k] > c->ncap || coff[k] > c->ncap - counts[k]) kpi[k].list_skin = 0.0;
        memset(&grid[k], 0, sizeof(Grid));
        grid[k].cbase = cells;
        grid[k].cap = instance_cell_cap(counts[k]);
        cells += grid[k].cap;
    }
    ioff[ninst] = slots;
    roff[ninst] = tot;
    int64_t ext = tot;
    if (first) {  // the instances' caller ranges must not overlap
        std::vector<int> ord(ninst);
        for (int k = 0; k < ninst; ++k) ord[k] = k;
        std::sort(ord.begin(), ord.end(), [&](int a, int b) { return coff[a] < coff[b]; });
        ext = 0;
        for (int q = 0; q < ninst; ++q) {
            const int k = ord[q];
            if (q > 0 && counts[k] > 0 && coff[k] < ext) {
                set_err(c, "instance %d overlaps an earlier one in the caller arrays", k);
                return SPH_E_INVAL;
            }
            if (counts[k] > 0) ext = std::max(ext, coff[k] + counts[k]);
        }
    }
    coff[ninst] = ext;
    if (tot > c->ncap || cells > c->cellcap) {
        set_err(c, "batch of %lld particles exceeds the capacity %lld", (long long)tot,
                (long long)c->ncap);
        return SPH_E_INVAL;
    }
    const int64_t nblk = (slots + kSlotAlign - 1) / kSlotAlign;
    std::vector<int32_t> blk((size_t)std::max<int64_t>(nblk, 1), 0);
    for (int k = 0; k < ninst; ++k)
        for (int64_t b = ioff[k] / kSlotAlign; b < (ioff[k] + icnt[k] + kSlotAlign - 1) / kSlotAlign; ++b)
            blk[(size_t)b] = k;
    DeviceGuard dg(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    lists_for_layout(c, ninst, coff.data(), icnt.data(), s);
    c->any_lists = false;
    for (int k = 0; k < ninst; ++k) c->any_lists = c->any_lists || kpi[k].list_skin > 0.0;
    cudaError_t e = cudaMemcpyAsync(c->ioff, ioff.data(), (ninst + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->coff, coff.data(), (ninst + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->icnt, icnt.data(), ninst * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->roff, roff.data(), (ninst + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->kpi, kpi.data(), ninst * sizeof(KParams), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->grid, grid.data(), ninst * sizeof(Grid), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nblk > 0)
        e = cudaMemcpyAsync(c->blk, blk.data(), nblk * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host arrays die with this call
    if (e != cudaSuccess) {
        set_err(c, "sph_batch_set: %s", cudaGetErrorString(e));
        cudaGetLastError();
        return SPH_E_CUDA;
    }
    c->n = slots;
    c->ntot = tot;
    c->cext = ext;
    c->ninst = ninst;
    c->prec = params[0].precision;
    c->kern_kind = params[0].kernel;
    c->grad_kind = params[0].gradients;
    c->tpp = native_pairs(c) ? 1 : kpi[0].pair_threads;
    return SPH_OK;
}

sph_status sph_batch_step(sph_ctx* c, sph_particles* P, int nsteps, void* stream) {
    if (!c) return SPH_E_INVAL;
    if (!P) { set_err(c, "particles is NULL"); return SPH_E_INVAL; }
    if (nsteps < 0) { set_err(c, "nsteps < 0"); return SPH_E_INVAL; }
    if (P->n < c->cext) {
        set_err(c, "n = %lld: the batch's instances extend to index %lld of the arrays",
                (long long)P->n, (long long)c->cext);
        return SPH_E_INVAL;
    }
    NEED(P->dt); NEED(P->time);
    if (P->n > 0) {
        NEED(P->x); NEED(P->y); NEED(P->z); NEED(P->vx); NEED(P->vy); NEED(P->vz);
        NEED(P->m); NEED(P->h); NEED(P->u); NEED(P->rho); NEED(P->p); NEED(P->c);
        NEED(P->ax); NEED(P->ay); NEED(P->az); NEED(P->du);
    }
    DeviceGuard dg(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    run_steps(c, P, nsteps, s);
    return check_launch(c, "sph_batch_step");
}

sph_status sph_neighbors_to_host(sph_ctx* c, int64_t* offsets, int32_t* idx,
                                 int64_t idx_capacity, int32_t* ngather, int32_t* order,
                                 void* stream) {
    if (!c) return SPH_E_INVAL;
    DeviceGuard dg(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = c->n;
    if (!c->csr_ready) launch_compose(c, s);  // rows of the last step are in slab form
    int64_t nnz = 0;
    cudaError_t e = cudaMemcpyAsync(&nnz, c->offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && offsets)
        e = cudaMemcpy(offsets, c->offsets, (size_t)(n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && ngather && n > 0)
        e = cudaMemcpy(ngather, c->ngather, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && order && n > 0)
        e = cudaMemcpy(order, c->order[c->cur], (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        set_err(c, "sph_neighbors_to_host: %s", cudaGetErrorString(e));
        cudaGetLastError();
        return SPH_E_CUDA;
    }
    if (idx) {
        if (nnz > idx_capacity || nnz > c->nnzcap) {
            set_err(c, "neighbour list has %lld entries; buffer holds %lld (context capacity %lld)",
                    (long long)nnz, (long long)idx_capacity, (long long)c->nnzcap);
            return SPH_E_INVAL;
        }
        if (nnz > 0) {
            e = cudaMemcpy(idx, c->idx, (size_t)nnz * sizeof(int32_t), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                set_err(c, "sph_neighbors_to_host: %s", cudaGetErrorString(e));
                cudaGetLastError();
                return SPH_E_CUDA;
            }
        }
    }
    return SPH_OK;
}

sph_status sph_neighbors_to_host_caller(sph_ctx* c, int64_t ncaller, int64_t* offsets,
                                        int32_t* idx, int64_t idx_capacity, int32_t* ngather,
                                        void* stream) {
    if (!c) return SPH_E_INVAL;
    if (!offsets || ncaller < c->cext) {
        set_err(c, "sph_neighbors_to_host_caller: offsets NULL or ncaller %lld below the caller "
                   "arrays' extent %lld", (long long)ncaller, (long long)c->cext);
        return SPH_E_INVAL;
    }
    // the internal rows on the host, then permuted to caller order there (host
    // memory in proportion to the list; an allocation failure is a status)
    try {
        const int64_t n = c->n;
        std::vector<int64_t> off((size_t)n + 1);
        std::vector<int32_t> ng((size_t)std::max<int64_t>(n, 1)), ord((size_t)std::max<int64_t>(n, 1));
        sph_status st = sph_neighbors_to_host(c, off.data(), nullptr, 0, ng.data(), ord.data(), stream);
        if (st != SPH_OK) return st;
        const int64_t nnz = off[(size_t)n];
        if (idx && nnz > idx_capacity) {
            set_err(c, "neighbour list has %lld entries; buffer holds %lld", (long long)nnz,
                    (long long)idx_capacity);
            return SPH_E_INVAL;
        }
        std::vector<int32_t> in((size_t)std::max<int64_t>(idx ? nnz : 0, 1));
        if (idx && (st = sph_neighbors_to_host(c, nullptr, in.data(), nnz, nullptr, nullptr,
                                               stream)) != SPH_OK)
            return st;
        // row lengths by caller index (indices that hold no particle: empty rows),
        // then their running sum
        for (int64_t r = 0; r <= ncaller; ++r) offsets[r] = 0;
        if (ngather)
            for (int64_t r = 0; r < ncaller; ++r) ngather[r] = 0;
        for (int64_t k = 0; k < n; ++k) {
            const int32_t o = ord[(size_t)k];
            if (o < 0) continue;  // an empty slot between instances
            offsets[o + 1] = off[(size_t)k + 1] - off[(size_t)k];
            if (ngather) ngather[o] = ng[(size_t)k];
        }
        for (int64_t r = 0; r < ncaller; ++r) offsets[r + 1] += offsets[r];
        if (!idx) return SPH_OK;
        for (int64_t k = 0; k < n; ++k) {
            const int32_t o = ord[(size_t)k];
            if (o < 0) continue;
            int32_t* dst = idx + offsets[o];
            const int64_t a = off[(size_t)k], b = off[(size_t)k + 1];
            for (int64_t e = a; e < b; ++e) dst[e - a] = ord[(size_t)in[(size_t)e]];
            // each part in ascending caller index: independent of the internal order
            std::sort(dst, dst + ng[(size_t)k]);
            std::sort(dst + ng[(size_t)k], dst + (b - a));
        }
        return SPH_OK;
    } catch (const std::bad_alloc&) {
        set_err(c, "sph_neighbors_to_host_caller: host memory for the permutation");
        return SPH_E_NOMEM;
    }
}

sph_status sph_sync(sph_ctx* c, void* stream) {
    if (!c) return SPH_E_INVAL;
    DeviceGuard dg(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(c->status_host, c->status, 2 * sizeof(unsigned),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, 2 * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_err(c, "sph_sync: %s", cudaGetErrorString(e));
        cudaGetLastError();
        return SPH_E_CUDA;
    }
    const unsigned bits = c->status_host[0];
    c->last_hnoconv = (int64_t)c->status_host[1];
    if (bits & ST_NONFINITE) {
        set_err(c, "a particle's state was non-finite or outside the geometry range "
                   "(|x|, |y|, |z| <= FLT_MAX, 0 <= h <= 2^100)");
        return SPH_E_NONFINITE;
    }
    if (bits & ST_CAPACITY) {
        set_err(c, "neighbour list exceeded nnz capacity %lld", (long long)c->nnzcap);
        return SPH_E_CAPACITY;
    }
    if (bits & ST_RANGE) {
        set_err(c, "a per-particle quantity of the float-pair pair kernels left their range "
                   "(use precision 2 for this input)");
        return SPH_E_RANGE;
    }
    if (bits & ST_HNOCONV) {
        set_err(c, "%lld particle(s) did not reach the target neighbour count",
                (long long)c->last_hnoconv);
        return SPH_E_HNOCONV;
    }
    return SPH_OK;
}

}  // extern "C"
