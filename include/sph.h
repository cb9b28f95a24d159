/*
 * sph.h -- C ABI of libsph, the GB300 (sm_103a) implementation of the SPH
 * time-step hot path of "Towards a Mini-App for Smoothed Particle
 * Hydrodynamics at Exascale" (arXiv 1809.08013), Section 3, Algorithm 1:
 *
 *   1. build tree            -> Morton-sorted uniform cell lists
 *   2. find neighbours and h -> sph_build_neighbors
 *   3. SPH kernels           -> sph_density, sph_eos, sph_forces
 *   5. new time step         -> sph_forces (writes dt)
 *   6. update v, x           -> sph_step (steps 1-6, nsteps times)
 *
 * Step 4 (self-gravity) is not part of this library.
 *
 * Conventions for every call:
 *  - Pointers in sph_particles are DEVICE pointers to float64 (or int32)
 *    arrays of length n, owned by the caller (e.g. torch CUDA tensors), in
 *    the caller's particle order. Scalars time and dt are device pointers to
 *    one double each.
 *  - `stream` is a cudaStream_t passed as a plain pointer (NULL = the legacy
 *    default stream). All work is enqueued asynchronously on it; no call
 *    synchronises the host except sph_sync and sph_ctx_create/destroy.
 *  - Arguments are validated on the host before any launch: a null context
 *    or params, n < 0, n > the context's capacity, or a null required array
 *    returns SPH_E_INVAL and launches nothing.
 *  - Conditions found on the device (CSR capacity exceeded, h iteration not
 *    converged) are recorded in a device status word; sph_sync returns them.
 *    Calls never abort or throw across the ABI.
 *  - A context is not thread-safe; use one context per host thread/stream.
 */
#ifndef SPH_H
#define SPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sph_ctx sph_ctx;

typedef enum {
    SPH_OK = 0,
    SPH_E_INVAL = 1,     /* bad argument; nothing was launched */
    SPH_E_NOMEM = 2,     /* device allocation failed in sph_ctx_create */
    SPH_E_CUDA = 3,      /* a CUDA runtime call or launch failed; see sph_last_error */
    SPH_E_CAPACITY = 4,  /* neighbour list longer than nnz_capacity: outputs of the
                            affected step are not valid; recreate with more capacity */
    SPH_E_HNOCONV = 5,   /* some particle's h search ended outside n_target +- n_tol;
                            results are still computed with its last h */
    SPH_E_TIMEOUT = 6,   /* reserved for bounded device waits */
    SPH_E_RANGE = 7,     /* precision 0 or 1: some per-particle quantity of the pair
                            kernels lies outside the range they hold (see below); the
                            density and force outputs of the affected step are not
                            valid at their stated accuracy. Precision 2 never raises it */
    SPH_E_NONFINITE = 8  /* a particle's state held a NaN or an infinity, or lay outside
                            the geometry range of the neighbour search (|x|, |y|, |z| <=
                            FLT_MAX, 0 <= h <= 2^100). The step still runs to its end
                            without touching memory out of bounds: such a particle gets
                            no neighbours of its own (a NaN or an infinite position also
                            keeps it out of every other particle's sets) and is left out
                            of the cell grid and the units; every output of its instance
                            for that step is undefined */
} sph_status;

/* Range of the pair kernels at precision 0 (float pairs) and 1 (FP32).
 * Those kernels work in units of their own, chosen per instance and per step
 * as powers of two: length 2^uL at or just above the mean h, mass 2^uM at or
 * just above the largest m, velocity 2^uV at or just above a velocity scale
 * (the largest |v| component, or c0 for Tait, or sqrt(gamma (gamma - 1)
 * max u) for an ideal gas, whichever is larger). Scaling by powers of two is
 * exact, so the caller's choice of units (SI, cgs, code units) does not
 * change the results; in those units every quantity a pair term needs is
 * O(1). The step reports SPH_E_RANGE (through sph_sync) when, in them, some
 * particle has 1/h outside [2^-15, 2^15] (h more than 2^15 away from the
 * mean h of its instance), rho outside [2^-60, 2^60], alpha c above 2^60 or
 * |p/rho^2| above 2^64, or when
 * the coordinates span more than about 2^120 smoothing lengths: input
 * outside what float-pair arithmetic can hold at FP64 accuracy. Use
 * precision 2 for such input. */

/* Physical and numerical parameters (Section 5.1 workloads). */
typedef struct {
    int32_t eos;         /* 0 = Tait (square patch), 1 = ideal gas (Evrard) */
    int32_t n_target;    /* target neighbour count, e.g. 100 */
    int32_t n_tol;       /* accepted |n - n_target|, e.g. 5 */
    int32_t max_h_iter;  /* h-search counts per particle, >= 1 */
    int32_t periodic_z;  /* 1: minimum image along z with period lz, z kept in [-lz/2, lz/2) */
    int32_t precision;   /* arithmetic of the pair sums (density, forces); positions, h,
                            neighbour sets, dt and the integration are FP64 in all three:
                            0 = FP64-accurate (double-float pair arithmetic, ~1e-14),
                            1 = mixed: FP32 relative coordinates, kernel, gradient and
                                viscosity terms, sums kept in double-float (~1e-7),
                            2 = the same sums with native FP64 arithmetic.
                            Other values: SPH_E_INVAL. */
    int32_t pair_threads; /* lanes per particle in the density and force sums: 1, 2, 4
                             or 8 (0 selects 2); the lanes of a
                             particle split its
                             neighbour row and combine their sums in a fixed order.
                             Ignored by precision 2. A tuning knob (sph_autotune): the
                             sums round differently for each value */
    int32_t defer_lanes;  /* h search: a warp of 32 particles hands its particles still
                             searching to one warp each once at most this many remain
                             (0 selects 16; at most 32). A tuning knob: h and the
                             neighbour sets do not depend on it */
    double rho0, c0;     /* Tait: p = c0^2 rho0 / 7 ((rho/rho0)^7 - 1), c = c0 (rho/rho0)^3 */
    double gamma;        /* ideal gas: p = (gamma - 1) rho u, c = sqrt(gamma (gamma - 1) u) */
    double alpha, beta;  /* Monaghan artificial viscosity */
    double eta2;         /* eta^2 in mu_ij = hb v.r / (r^2 + eta^2 hb^2), e.g. 0.01 */
    double cfl;          /* dt = cfl * min h / (c + 1.2 (alpha c + beta mumax)) */
    double lz;           /* period along z when periodic_z = 1 */
    double cell_scale;   /* cell width = 2 <h> cell_scale (0 selects the default 1.0); a tuning
                            knob of the neighbour search: h and the neighbour sets do not
                            depend on it */
    /* Variants of Table 1 (support 2h for all kernels, q = r/h). They run in
       the double-float pair kernels at precision 0 and on the FP64 pipe at
       precision 2; with precision 1 any choice but (0, 0) is SPH_E_INVAL. The
       neighbour search does not depend on them. */
    int32_t kernel;      /* SPH_KERNEL_*: 0 = M4 cubic spline (1/(pi h^3)) (t^3/4 - s^3),
                            t = max(2-q, 0), s = max(1-q, 0);
                            1 = Wendland C2, 21/(16 pi h^3) (1 - q/2)^4 (1 + 2q) for q < 2;
                            2 = sinc, B_n/h^3 (sin x / x)^n, x = pi q / 2, q < 2, with
                            B_n = 1 / (4 pi int_0^2 q^2 (sin x / x)^n dq) */
    int32_t gradients;   /* SPH_GRAD_*: 0 = kernel derivatives; 1 = IAD, integral approach
                            to derivatives: C_i = tau_i^-1 with tau_i = sum_{j in N_i}
                            (m_j/rho_j) W(r_ij, h_i) (r_j - r_i)(r_j - r_i)^T (C_i = 0 if
                            tau_i is singular), and the symmetrised pair gradient
                            G_ij = (W(r_ij, h_i) C_i + W(r_ij, h_j) C_j)(r_j - r_i) / 2
                            in place of Fbar_ij r_ij in the momentum and energy sums */
    int32_t sinc_n;      /* exponent n of the sinc kernel, 2..12 (read when kernel = 2) */
    double list_skin;    /* h search with candidate lists (opt in; 0 or negative: off,
                            every count walks the cells): every particle keeps across
                            steps the list of all particles within 2 h (1 + list_skin)
                            of it at the last list build and counts its neighbours from
                            that list while it still holds them all (no particle has
                            moved far enough since); the instance rebuilds its lists
                            when one no longer covers its particle's 2 h. Above 1:
                            SPH_E_INVAL. On GB300 the cell walk, which loads each
                            candidate once for a warp of 32 particles, is the faster of
                            the two for the benchmark workloads. The first call that
                            turns the lists on allocates their buffers (about 800 B per
                            particle of capacity, not counted by sph_ctx_bytes; that call
                            synchronises the device and is not capturable, SPH_E_NOMEM
                            if the allocation fails). Their records are kept per
                            caller index: a batch instance whose caller range reaches
                            past the context's capacity runs without them. A tuning
                            knob: h and the neighbour sets do not depend on it (the
                            order within a gather set does) */
} sph_params;

#define SPH_KERNEL_M4 0
#define SPH_KERNEL_WENDLAND_C2 1
#define SPH_KERNEL_SINC 2
#define SPH_GRAD_KERNEL 0
#define SPH_GRAD_IAD 1

/* Caller-owned particle arrays (device pointers, caller order, length n). */
typedef struct {
    int64_t n;
    double *x, *y, *z;       /* position */
    double *vx, *vy, *vz;    /* velocity */
    double *m;               /* mass */
    double *h;               /* smoothing length: input guess, output converged value */
    double *u;               /* specific internal energy */
    double *rho, *p, *c;     /* density, pressure, sound speed */
    double *ax, *ay, *az;    /* acceleration */
    double *du;              /* du/dt */
    double *mumax;           /* optional (may be NULL): max_j |mu_ij| */
    int32_t *nnb;            /* optional (may be NULL): gather neighbour count n_i */
    double *time;            /* device scalar: simulated time, advanced by sph_step */
    double *dt;              /* device scalar: last time step */
} sph_particles;

/* View of the context-owned neighbour list, valid until the next call that
 * rebuilds it. Rows are in the library's internal (Morton cell) order:
 * internal row k belongs to caller particle order[k], and every idx entry is
 * an internal row number. After a batch step (sph_batch_step) the rows are
 * the slots of all instances; the empty slots between instances have
 * order[k] = -1 and empty rows. Row k lists first its gather set
 * N_k = { j : r_kj < 2 h_k } (ngather[k] entries), then the rest of the
 * symmetric set S_k = { j : r_kj < 2 max(h_k, h_j) }. Entry order within each
 * part is unspecified. All pointers are device pointers; *nnz_dev is the
 * number of entries (offsets[n]). */
typedef struct {
    int64_t n;
    const int64_t *offsets;  /* n + 1 */
    const int32_t *idx;      /* offsets[n] */
    const int32_t *ngather;  /* n */
    const int32_t *order;    /* n: caller index of internal row k */
    const int64_t *nnz_dev;  /* = offsets + n */
} sph_neighbors;

/* Create a context on CUDA device `device` for up to n_capacity particles and
 * nnz_capacity neighbour-list entries (about 1.1 x 105 per particle for the
 * 100-neighbour workloads). Allocates all scratch once; later calls allocate
 * nothing. On failure *out is NULL. The steps keep each particle's row of
 * S_i in a fixed slab of 224 entries (at most 128 of them the gather set);
 * the nnz_capacity-entry CSR is written for sph_build_neighbors and
 * sph_neighbors_to_host, and by a step only when some row does not fit its
 * slab (then SPH_E_CAPACITY if the CSR does not fit either). SPH_E_INVAL for
 * a negative capacity, n_capacity (plus the batch gaps below) above
 * 2^31 - 2 (slots are int32) or nnz_capacity above 2^40; SPH_E_CUDA for a
 * device that does not exist. */
sph_status sph_ctx_create(sph_ctx **out, int64_t n_capacity, int64_t nnz_capacity, int device);

/* Largest number of instances of one batch (the instance id takes the top 8
 * bits of the 32-bit sort key). */
#define SPH_MAX_INSTANCES 256

/* As sph_ctx_create, for batches of up to max_instances independent
 * problems with n_capacity particles in total (sph_batch_set / _step).
 * Internally every instance starts on a 256-slot boundary, so up to
 * 255 (max_instances - 1) extra slots are allocated. max_instances outside
 * [1, SPH_MAX_INSTANCES] returns SPH_E_INVAL. The paper runs one problem per
 * job; batching independent problems on one GPU has no counterpart in it. */
sph_status sph_ctx_create_batch(sph_ctx **out, int64_t n_capacity, int64_t nnz_capacity,
                                int32_t max_instances, int device);

/* Device bytes a context of these capacities allocates on the current device
 * (each allocation rounded up to 256 bytes; a few buffers scale with the
 * device's SM count), without allocating; -1 for invalid sizes. Lets a
 * caller fit contexts into a memory budget. */
int64_t sph_ctx_bytes(int64_t n_capacity, int64_t nnz_capacity, int32_t max_instances);

/* Free the context and its device memory (synchronises the device). NULL is a no-op. */
void sph_ctx_destroy(sph_ctx *ctx);

/* Algorithm 1 steps 1-2 (Section 3 and its footnote: h follows a target
 * neighbour count). Reads x, y, z, h (and m, v, u, which it also copies into
 * the context); sorts the particles by the Morton code of their cell; runs
 * the bracketing h search per particle (count of N_i(h) must reach
 * n_target +- n_tol); writes the final h (and nnb if given) back to the
 * caller arrays and builds the symmetric neighbour list. `out` may be NULL. */
sph_status sph_build_neighbors(sph_ctx *ctx, const sph_params *prm, sph_particles *P,
                               sph_neighbors *out, void *stream);

/* Algorithm 1 step 3, density: rho_i = m_i W(0, h_i) + sum_{j in N_i} m_j W(r_ij, h_i)
 * with the M4 cubic spline (Table 1). Uses the neighbour list of the last
 * sph_build_neighbors and the caller's current x, y, z, m, h; writes rho. */
sph_status sph_density(sph_ctx *ctx, const sph_params *prm, sph_particles *P, void *stream);

/* Algorithm 1 step 3, equation of state: reads rho, u; writes p, c. Elementwise. */
sph_status sph_eos(sph_ctx *ctx, const sph_params *prm, sph_particles *P, void *stream);

/* Algorithm 1 steps 3 and 5: momentum and energy equations with Monaghan
 * artificial viscosity over S_i, and the new time step. Reads x, y, z, vx,
 * vy, vz, m, h, rho, p, c; writes ax, ay, az, du, mumax (if given) and *dt. */
sph_status sph_forces(sph_ctx *ctx, const sph_params *prm, sph_particles *P, void *stream);

/* Algorithm 1, nsteps full iterations: neighbours and h, density, EOS,
 * forces, dt, then the kick-drift update v += dt a, u += dt du, x += dt v
 * (z wrapped when periodic), time += dt. State is kept in the context's
 * sorted order between steps and written back to the caller arrays at the
 * end, together with h, rho, p, c, a, du, mumax, nnb of the last step. */
sph_status sph_step(sph_ctx *ctx, const sph_params *prm, sph_particles *P, int nsteps,
                    void *stream);

/* sph_step on HOST arrays: the same nsteps iterations, with every pointer of
 * P a host pointer (any host memory works). The state x, y, z, vx, vy, vz, m,
 * h, u is read at the start and written back at the end, with *time, *dt and
 * each of rho, p, c, ax, ay, az, du, mumax, nnb that is not NULL (only the
 * state fields and time, dt are required). An array in page-locked (pinned)
 * or registered host memory is read and written in place by the call's first
 * and last kernels, over the link to host memory; any other array is copied
 * on the stream to device staging buffers owned by the context and back. The staging (17 doubles and one int32 per particle of capacity)
 * is allocated by the first call (SPH_E_NOMEM if that fails) and freed with
 * the context; sph_ctx_bytes does not include it. Asynchronous like
 * sph_step: the host arrays hold the results after sph_sync (or a stream
 * synchronisation). nsteps = 0 copies nothing. */
sph_status sph_step_host(sph_ctx *ctx, const sph_params *prm, sph_particles *P, int nsteps,
                         void *stream);

/* Describe a batch of ninst independent problems for sph_batch_step.
 * counts[k] (host array) is the number of particles of instance k, held in
 * the caller's arrays at [first[k], first[k] + counts[k]) (first: host array,
 * ranges must not overlap; NULL = back to back from index 0). params[k]
 * (host array) are its parameters; all instances must share `precision`
 * and `pair_threads`. Instances never
 * interact: each has its own cell grid, neighbour sets, time step and time.
 * An instance's results are bit-identical to a single-problem sph_step of it
 * with the same parameters. Copies the descriptors to the device and waits
 * for the copy (synchronises `stream`). SPH_E_INVAL for ninst outside
 * [1, max_instances], a negative count or first, overlapping ranges, a range
 * reaching past caller index 2^31 - 1, invalid params, or more particles
 * than the capacity. Any single-problem call replaces the batch. */
sph_status sph_batch_set(sph_ctx *ctx, int32_t ninst, const int64_t *counts,
                         const int64_t *first, const sph_params *params, void *stream);

/* sph_step for every instance of the batch: P holds all instances' arrays
 * (P->n = their length, at least the end of the last instance; entries
 * outside the instances are not touched); P->dt and P->time are device
 * arrays of ninst doubles (per-instance time step and time). Enqueues only
 * kernel launches, so it can be captured in a CUDA graph and replayed while
 * the batch is unchanged. SPH_E_INVAL if P->n is too short. Splitting a run
 * into several calls gives the same bits as one call. */
sph_status sph_batch_step(sph_ctx *ctx, sph_particles *P, int nsteps, void *stream);

/* Rows of the current neighbour list (the n of sph_neighbors): the particle
 * count of a single problem; for a batch, the slots of all instances. */
int64_t sph_neighbor_rows(const sph_ctx *ctx);

/* Search space of sph_autotune (host arrays of candidate values). */
#define SPH_TUNE_MAX_TRIALS 16
typedef struct {
    const double *cell_scales;   int32_t n_cell_scales;   /* each > 0 */
    const int32_t *pair_threads; int32_t n_pair_threads;  /* each 1, 2, 4 or 8 */
    const int32_t *defer_lanes;  int32_t n_defer_lanes;   /* each in [1, 32] */
} sph_tune_space;

typedef struct {
    double cell_scale;
    int32_t pair_threads, defer_lanes;
    double ms_per_step;
} sph_tune_trial;

typedef struct {
    double cell_scale;           /* the chosen knobs ... */
    int32_t pair_threads, defer_lanes;
    double ms_per_step;          /* ... and their device time per step */
    int32_t n_trials;
    sph_tune_trial trials[SPH_TUNE_MAX_TRIALS];  /* every setting timed, in order */
} sph_tune_result;

/* Choose the performance knobs of the current batch (or single problem of
 * the last call) by timing: for each candidate, the caller's state P is
 * loaded, one step runs untimed and nsteps steps are timed with CUDA events
 * on `stream`. One coordinate-descent pass from the current knobs, in the
 * order pair_threads, cell_scale, defer_lanes, keeps the fastest value of
 * each. The knobs change neither h nor the neighbour sets; the sums round
 * differently with pair_threads. P is not modified (dt and time of the
 * trials go to context scratch); the context keeps the chosen knobs for
 * sph_batch_step until the next sph_batch_set, and a single-problem call
 * takes them from its sph_params. space = NULL uses cell_scale {0.875, 1,
 * 1.25}, pair_threads {1, 2, 4}, defer_lanes {8, 16}. Synchronises the
 * stream (not capturable). SPH_E_INVAL for nsteps < 1, P->n too short for
 * the batch, invalid candidates or more than SPH_TUNE_MAX_TRIALS of them.
 * Device conditions of the trial runs (h non-convergence) stay in the
 * status word for the next sph_sync. This knob search has no counterpart in
 * the paper (its codes are tuned per machine by hand). */
sph_status sph_autotune(sph_ctx *ctx, sph_particles *P, int nsteps, const sph_tune_space *space,
                        sph_tune_result *out, void *stream);

/* Copy the neighbour list of the last sph_build_neighbors (or last step of
 * sph_step) into caller HOST buffers, synchronously after the stream's work:
 * offsets (n + 1), ngather (n), order (n) and, if idx is not NULL, idx (up to
 * idx_capacity entries; SPH_E_INVAL if offsets[n] > idx_capacity). Any of the
 * pointers may be NULL to skip that array. Layout as in sph_neighbors. */
sph_status sph_neighbors_to_host(sph_ctx *ctx, int64_t *offsets, int32_t *idx,
                                 int64_t idx_capacity, int32_t *ngather, int32_t *order,
                                 void *stream);

/* The same neighbour list in CALLER order, on the host: row r belongs to
 * the caller's particle r (r < ncaller, which must cover the caller arrays:
 * n for a single problem, the batch's extent otherwise; rows of indices that
 * hold no particle are empty) and lists caller indices: first its gather set
 * N_r (ngather[r] entries), then the rest of S_r, each part in ascending
 * caller index (so the rows do not depend on the library's internal order).
 * offsets (ncaller + 1, required), idx (up to idx_capacity entries;
 * SPH_E_INVAL if the list is longer) and ngather (ncaller) are host arrays;
 * idx and ngather may be NULL. Permuted on the host after the copies of
 * sph_neighbors_to_host (synchronises `stream`; host memory of about 4
 * bytes per entry and 16 per particle, SPH_E_NOMEM if it cannot be had). */
sph_status sph_neighbors_to_host_caller(sph_ctx *ctx, int64_t ncaller, int64_t *offsets,
                                        int32_t *idx, int64_t idx_capacity, int32_t *ngather,
                                        void *stream);

/* Phases of sph_step timed by sph_timing_read. */
enum {
    SPH_PHASE_CELLS = 0,    /* load, bounding box, Morton keys, radix sort, permute, cell ranges */
    SPH_PHASE_HSEARCH = 1,  /* h search, FP32 thresholds, per-cell max h */
    SPH_PHASE_CSR = 2,      /* rows of S_i: outer sets, sorted; lengths */
    SPH_PHASE_DENSITY = 3,  /* density with the equation of state fused */
    SPH_PHASE_FORCES = 4,   /* momentum, energy, viscosity, dt partials and dt */
    SPH_PHASE_UPDATE = 5,   /* kick-drift update and the final write-back */
    SPH_NPHASES = 6
};

/* Enable (1) or disable (0) per-phase timing of sph_step with CUDA events
 * recorded on the call's stream; enabling clears the accumulators and
 * creates the event pool (host-side objects, up to 1024 steps per read). */
sph_status sph_timing_enable(sph_ctx *ctx, int enable);

/* Wait for the recorded events and return, per phase, the accumulated device
 * milliseconds (ms[SPH_NPHASES]) and kernel launches (launches[SPH_NPHASES])
 * since the last read or enable; *steps receives the number of timed steps.
 * Any output pointer may be NULL. Clears the accumulators. */
sph_status sph_timing_read(sph_ctx *ctx, double *ms, int64_t *launches, int64_t *steps);

/* Forget the h search's candidate lists (sph_params.list_skin) of the
 * particles [first, first + count) of the caller arrays, on the stream: the
 * next step of their instance rebuilds its lists. h and the neighbour sets
 * never depend on the lists; the order of the pair sums does, so a context
 * carries, from one call to the next, lists that can change the last bits of
 * the sums. Contexts with the same history of calls give the same bits, and
 * an instance whose caller range (first, count) is new to the batch starts
 * without lists. A caller that writes a new problem into a range the last
 * batch already had, and wants the bits of a fresh context, calls this first.
 * SPH_E_INVAL for a range outside [0, the context's capacity). */
sph_status sph_lists_clear(sph_ctx *ctx, int64_t first, int64_t count, void *stream);

/* Number of candidate-list builds of this context so far (one per instance
 * and rebuilding step), after the stream's work (synchronises the stream):
 * a measure of how long the lists last for a given list_skin. */
sph_status sph_list_builds(sph_ctx *ctx, int64_t *builds, void *stream);

/* Total kernel launches issued by this context since creation. */
int64_t sph_launch_count(const sph_ctx *ctx);

/* Wait for the stream, then return and clear the device status: SPH_OK, or
 * the most severe of SPH_E_NONFINITE, SPH_E_CAPACITY, SPH_E_RANGE and
 * SPH_E_HNOCONV (in that order) raised since the last sph_sync. */
sph_status sph_sync(sph_ctx *ctx, void *stream);

/* Number of particles whose h search did not converge since the last
 * sph_sync (valid after sph_sync returned; reset by the next sph_sync). */
int64_t sph_last_hnoconv(const sph_ctx *ctx);

/* Text of the last error on this context ("" if none). Never NULL. */
const char *sph_last_error(const sph_ctx *ctx);

/* Largest n accepted by sph_dt_noalloc (its static scratch holds one partial
 * minimum per 256 particles: 8192 doubles, 64 KiB per device). */
#define SPH_NOALLOC_MAX_N ((int64_t)2097152)

/* The time step of sph_forces, dt = cfl * min_i h_i / (c_i + 1.2 (alpha c_i +
 * beta mumax_i)), computed from caller-held device arrays without any device
 * allocation. The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc -- code running under a host that owns
 * all device memory through its own pool (a serving runtime, a framework
 * plugin with a fixed budget), or a latency-critical loop where an
 * allocation may synchronise the device.
 *  - h, c, mumax (mumax may be NULL = all zero) are device arrays of length n;
 *    *dt is a device scalar written on `stream` (the current device's).
 *  - Its scratch is a static device array inside the library, which every GPU
 *    that loads the library holds until the process exits. Each call looks up
 *    that array's device address in the current context (cudaGetSymbolAddress);
 *    the first lookup in a context may load the library's device code there,
 *    so make the first call before any stream capture. No call allocates.
 *  - n > SPH_NOALLOC_MAX_N, n < 0, cfl <= 0 or a NULL required pointer returns
 *    SPH_E_INVAL and launches nothing; n = 0 writes +inf.
 *  - A CUDA error already pending when the call starts (from the caller's
 *    earlier work) returns SPH_E_CUDA with nothing launched and is left
 *    pending for the caller's own check; SPH_E_CUDA otherwise means this
 *    call's lookup or launch failed.
 *  - All calls on a device share the scratch: calls that may overlap on the
 *    GPU (different streams without ordering) race; serialise them. */
sph_status sph_dt_noalloc(const sph_params *prm, int64_t n, const double *h, const double *c,
                          const double *mumax, double *dt, void *stream);

/* Measurement utility, not part of the SPH path: run a register-resident
 * FMA-chain kernel on `stream` of `device` and return the achieved rate as
 * *flops_per_s = 2 x FMAs per second, FP64 when fp64 != 0, else FP32. This is
 * the denominator of the FP64 pair kernels' roofline. Synchronous. */
sph_status sph_probe_fma_peak(int device, int fp64, void *stream, double *flops_per_s);

/* Version string of the library. */
const char *sph_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPH_H */
