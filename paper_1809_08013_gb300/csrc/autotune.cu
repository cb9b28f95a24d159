// autotune.cu -- choice of the performance knobs of a batch by measurement.
//
// Three knobs change only the speed of a step, never which neighbours or h
// are found: the cell width factor (cell width = 2 <h> cell_scale; larger
// cells mean fewer cells to visit but more candidates to test), the lanes
// per particle of the density and force sums (more lanes shorten the longest
// row a warp waits for and coalesce the row reads, at the price of a
// cross-lane reduction), and the h-search hand-over threshold (how few
// particles of a warp may still be searching before each gets a warp of its
// own). The tuner times trial runs of the current batch from the caller's
// state and keeps, knob by knob, the fastest value (one coordinate-descent
// pass, in the order lanes, cell width, hand-over).
#include <string.h>


#include "sph_internal.cuh"

namespace sph {

__global__ void k_set_knobs(KParams* __restrict__ kpi, int ninst, double cell_scale,
                            int pair_threads, int defer_lanes) {
    for (int k = threadIdx.x; k < ninst; k += blockDim.x) {
        kpi[k].cell_scale = cell_scale;
        kpi[k].pair_threads = pair_threads;
        kpi[k].defer_lanes = defer_lanes;
    }
}

namespace {

struct Knobs {
    double cs;
    int tpp, defer;
};

void set_knobs(sph_ctx* c, const Knobs& k, cudaStream_t s) {
    c->launches += 1;
    k_set_knobs<<<1, 256, 0, s>>>(c->kpi, c->ninst, k.cs, k.tpp, k.defer);
    c->tpp = native_pairs(c) ? 1 : k.tpp;
}

// Device milliseconds per step of nsteps steps after one untimed step, from
// the caller's state (which is not modified); < 0 on a CUDA error.
float trial(sph_ctx* c, const sph_particles* P, const Knobs& k, int nsteps, cudaEvent_t e0,
            cudaEvent_t e1, cudaStream_t s) {
    set_knobs(c, k, s);
    double* dt = c->tune_dt;
    double* tm = c->tune_dt + c->maxinst;
    lists_clear(c, s);  // every trial starts without candidate lists
    launch_load_state(c, P, s);
    launch_step(c, dt, tm, s);
    cudaEventRecord(e0, s);
    for (int q = 0; q < nsteps; ++q) launch_step(c, dt, tm, s);
    cudaEventRecord(e1, s);
    float ms = -1.0f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        cudaGetLastError();
        return -1.0f;
    }
    return ms / (float)nsteps;
}

}  // namespace
}  // namespace sph

using namespace sph;

extern "C" sph_status sph_autotune(sph_ctx* c, sph_particles* P, int nsteps,
                                   const sph_tune_space* space, sph_tune_result* out,
                                   void* stream) {
    if (!c || !P || !out || nsteps < 1) return SPH_E_INVAL;
    if (P->n < c->cext) return SPH_E_INVAL;
    if (P->n > 0 && (!P->x || !P->y || !P->z || !P->h || !P->m)) return SPH_E_INVAL;
    static const double kCs[] = {0.875, 1.0, 1.25};
    static const int32_t kTpp[] = {1, 2, 4};
    static const int32_t kDefer[] = {8, 16};
    sph_tune_space d = {kCs, 3, kTpp, 3, kDefer, 2};
    const sph_tune_space& sp = space ? *space : d;
    if (sp.n_cell_scales < 0 || sp.n_pair_threads < 0 || sp.n_defer_lanes < 0 ||
        sp.n_cell_scales + sp.n_pair_threads + sp.n_defer_lanes > SPH_TUNE_MAX_TRIALS)
        return SPH_E_INVAL;
    for (int q = 0; q < sp.n_cell_scales; ++q)
        if (!(sp.cell_scales[q] > 0.0)) return SPH_E_INVAL;
    for (int q = 0; q < sp.n_pair_threads; ++q) {
        const int t = sp.pair_threads[q];
        if (!(t == 1 || t == 2 || t == 4 || t == 8)) return SPH_E_INVAL;
    }
    for (int q = 0; q < sp.n_defer_lanes; ++q)
        if (sp.defer_lanes[q] < 1 || sp.defer_lanes[q] > 32) return SPH_E_INVAL;

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPH_E_CUDA;
    const bool swap = dev != c->device;
    if (swap && cudaSetDevice(c->device) != cudaSuccess) return SPH_E_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    // the batch's current knobs (all instances carry the same ones)
    KParams k0;
    sph_status st = SPH_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMemcpyAsync(&k0, c->kpi, sizeof(KParams), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        st = SPH_E_CUDA;
    }
    Knobs best = {k0.cell_scale, k0.pair_threads, k0.defer_lanes};
    memset(out, 0, sizeof(*out));
    float best_ms = -1.0f;
    int nt = 0;
    auto run = [&](const Knobs& k) {
        if (st != SPH_OK) return;
        for (int q = 0; q < nt; ++q)  // a setting already timed
            if (out->trials[q].cell_scale == k.cs && out->trials[q].pair_threads == k.tpp &&
                out->trials[q].defer_lanes == k.defer)
                return;
        const float ms = trial(c, P, k, nsteps, e0, e1, s);
        if (ms < 0.0f) {
            st = SPH_E_CUDA;
            return;
        }
        out->trials[nt].cell_scale = k.cs;
        out->trials[nt].pair_threads = k.tpp;
        out->trials[nt].defer_lanes = k.defer;
        out->trials[nt].ms_per_step = ms;
        ++nt;
        if (best_ms < 0.0f || ms < best_ms) {
            best_ms = ms;
            best = k;
        }
    };
    run(best);  // the starting point
    for (int q = 0; q < sp.n_pair_threads; ++q) {
        const Knobs b = best;
        if (sp.pair_threads[q] != b.tpp) run(Knobs{b.cs, sp.pair_threads[q], b.defer});
    }
    for (int q = 0; q < sp.n_cell_scales; ++q) {
        const Knobs b = best;
        if (sp.cell_scales[q] != b.cs) run(Knobs{sp.cell_scales[q], b.tpp, b.defer});
    }
    for (int q = 0; q < sp.n_defer_lanes; ++q) {
        const Knobs b = best;
        if (sp.defer_lanes[q] != b.defer) run(Knobs{b.cs, b.tpp, sp.defer_lanes[q]});
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    lists_clear(c, s);  // the caller's next steps start as they would untuned
    if (st == SPH_OK) {
        set_knobs(c, best, s);  // the batch keeps the chosen knobs
        out->cell_scale = best.cs;
        out->pair_threads = best.tpp;
        out->defer_lanes = best.defer;
        out->ms_per_step = best_ms;
        out->n_trials = nt;
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            st = SPH_E_CUDA;
        }
    }
    if (swap) cudaSetDevice(dev);
    return st;
}
