// sph_internal.cuh -- internal types and launchers of libsph (not part of the ABI).
//
// Data layout in HBM (internal, Morton-cell order, one entry per particle):
//   posh[k]   = (x, y, z, h)              32 B (double4, 32-byte aligned)
//   velm[k]   = (vx, vy, vz, m)           32 B
//   therm[k]  = (rho/2, A, alpha c/2, h/2) 32 B, A = p / rho^2
//   kern[k]   = (1/h, 1/h^4)              16 B
//   acc[k]    = (ax, ay, az, du)          32 B
//   ue[k], pint[k], cint[k], mumax[k]     u, p, c and max_j |mu_ij| (double)
//   fpos[k]   = (xf, yf, zf, Tout)  float4, 16 B: FP32 copy of the position and
//               the upper FP32 threshold of the (2h)^2 test (see neighbors.cu)
//   tin[k]    = Tin                 float: lower FP32 threshold
// The j-side loads of the pair kernels therefore touch one or three 32-byte
// sectors per neighbour instead of up to eleven scattered arrays.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "../../include/sph.h"

namespace sph {

constexpr int kMortonBits = 8;                      // bits per axis -> 24-bit keys
constexpr int kMaxCellsPerAxis = 1 << kMortonBits;  // 256
constexpr int kThreads = 256;
constexpr int kRadixItems = 8;                      // keys per thread in the sort
constexpr int kRadixTile = kThreads * kRadixItems;  // 2048 keys per block
constexpr int kScanTile = kThreads * 8;             // elements per block in scans
constexpr int kReduceBlocks = 304;                  // 2 x 152 SMs
constexpr int kMaxPairThreads = 8;                  // lanes per particle in the pair kernels
constexpr int kBoxStride = 16;                      // doubles per bounding-box partial
constexpr int kBoxWarpSlots = 64;                   // bounding box: slots per warp (4 per partial)

// device status word
enum : unsigned {
    ST_CAPACITY = 1u,   // neighbour list exceeded nnz capacity
    ST_HNOCONV = 2u,    // some h search did not converge
    ST_RANGE = 4u,      // a float-pair quantity left the range of the pair kernels
    ST_NONFINITE = 8u,  // a particle's state was non-finite or outside the geometry range
};

// Geometry range of a particle (integer tests on the bits, no FP64 pipe): the
// neighbour search works on FP32 coordinates and FP32 reaches, so |x|, |y|,
// |z| <= FLT_MAX and 0 <= h <= 2^100 (false for NaN and infinities).
constexpr long long kF32MaxBits = 0x47EFFFFFE0000000LL;  // FLT_MAX as a double
constexpr long long kHMaxBits = 0x4630000000000000LL;    // 2^100
__device__ __forceinline__ bool coord_ok(double x) {
    return (__double_as_longlong(x) & 0x7fffffffffffffffLL) <= kF32MaxBits;
}
__device__ __forceinline__ bool h_ok(double h) {
    const long long b = __double_as_longlong(h);
    return b >= 0 && b <= kHMaxBits;
}
__device__ __forceinline__ bool finite_bits(double x) {
    return (__double_as_longlong(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}

// Lower and upper FP32 bounds of a positive double from its bit pattern
// (truncation is rounding toward zero; integer operations only).
__device__ __forceinline__ void f32_bounds(double x, float& lo, float& hi) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)(b >> 52) - 1023 + 127;
    if (e <= 0) {
        lo = 0.0f;
        hi = 1.17549435e-38f;
    } else if (e >= 255) {
        lo = 3.40282347e+38f;
        hi = CUDART_INF_F;
    } else {
        const unsigned lb = ((unsigned)e << 23) | ((unsigned)(b >> 29) & 0x7fffffu);
        lo = __int_as_float((int)lb);
        hi = (b & 0x1fffffffull) ? __int_as_float((int)(lb + 1)) : lo;
    }
}

// Upper FP32 bound of 2 x (a positive double), widened by 1e-4 relative.
__device__ __forceinline__ float reach_f32(double h) {
    float lo, hi;
    f32_bounds(h, lo, hi);
    return 2.0f * hi * 1.0001f;
}

// Order-preserving integer key of a float (and back): signed integer order of
// the keys is the order of the values.
__device__ __forceinline__ long long fkey(float f) {
    const int b = __float_as_int(f);
    return (long long)(b >= 0 ? b : (b ^ 0x7fffffff));
}
__device__ __forceinline__ float fkey_inv(long long k) {
    const int b = (int)k;
    return __int_as_float(b >= 0 ? b : (b ^ 0x7fffffff));
}
// internal flags (status[2], cleared at every build)
enum : unsigned {
    IF_SLAB_OVF = 1u,   // a row did not fit the gather/outer slabs: full CSR kernels run
    IF_OUTER_OVF = 2u,  // an outer part overflowed while the density kernel appended it:
                        // the CSR kernels run after the density, before the forces
};
constexpr int kGSlab = 128;  // gather-set slots per particle (>= n_target + n_tol)
constexpr int kRec = 256;    // h search: candidates recorded per lane in flight
constexpr int kUnionBlocksPerSM = 4;  // resident blocks of the persistent h search
// Candidate lists of the h search, kept across steps (neighbors.cu). While an
// instance keeps its lists, its particles keep the slots of the list build:
// the sort orders them by the cell codes of that build, not by their current
// cells (the cell tables then hold the build's cells, and every cell walk
// widens its reach by the largest displacement since). A list holds the slots
// of every particle within 2 h (1 + skin) of its particle at the build; the
// lists of the 32 slots of a warp are stored interleaved (entry e of slot i at
// ((i / 32) kList + e) 32 + i % 32), so a warp reads 32 entries at once.
constexpr int kList = 192;                    // list entries per particle
struct LMeta {     // per caller index, written by the instance's last list build
    float x, y, z;   // the particle's position then (truncated floats)
    float rad;       // list radius (a lower bound): all j within it then are listed
    int32_t stamp;   // that build (0: none; builds of one context are numbered)
    uint32_t code;   // the particle's cell code (Morton) in the build's grid
    int32_t cnt;     // list length (0: no usable list)
    int32_t pad;
};
constexpr int kRSlab = 224;  // row slots per particle: gather set, then the outer set
                             // (outer sets: patch max ~40, Evrard ~64)

// Cell grid, computed on the device from the particle bounding box each build.
struct Grid {
    double lo[3];
    double w[3];
    double inv_w[3];
    int n[3];
    int periodic_z;
    double lz;
    double X;        // max |coordinate| (bounds the FP32 rounding error)
    double hmean;
    unsigned long long hmax_bits;  // bits of max h after the h search
    long long ncells;
    long long cbase;  // first entry of this instance's cells in the cell tables
    long long cap;    // cells this instance may use (sets the smallest cell width)
    float lof[3], wf[3], invwf[3];
    float lzf, halflzf;
    float slop[3];   // absolute slack added to query boxes (FP32 rounding cover)
    float eC, eR;    // FP32-error bound of a coordinate difference: e(R) <= eC + eR * R
    int fxk;         // fixed-point exponent of the coordinate chunks: |x| 2^fxk < 2^61
    float lzc[3];    // lz as chunks, in the pair kernels' length unit
    float hlzc;      // lz / 2 in that unit (the wrap test on chunk differences)
    // Units of the float-pair (precision 0) and FP32 (precision 1) pair
    // kernels: length 2^uL, mass 2^uM, velocity 2^uV, powers of two taken
    // from the instance's mean h, largest m and a velocity scale, so that the
    // quantities those kernels hold are O(1) whatever units the caller uses.
    // Multiplying by a power of two is exact, and every operation of the pair
    // sums commutes with it while its operands stay in the normal float
    // range, so in units where everything is already O(1) the results are
    // the same bits as without the rescaling.
    int uL, uM, uV;
    // Candidate lists (set per step by the grid setup): lbuild = 1 when this
    // step's h search rebuilds the instance's lists (stamped lstamp); else the
    // lists of build lstamp hold, and dm2 bounds twice any particle's
    // displacement since that build.
    int lbuild, lstamp;
    float dm2;
    int gvalid;  // the geometry above is that of a list build (kept while the lists are)
};

// 2^e as a double, exactly (e in [-1022, 1023]); integer operations only.
__host__ __device__ __forceinline__ double p2d(int e) {
    union { long long i; double d; } u;
    u.i = (long long)(1023 + e) << 52;
    return u.d;
}

// Parameters copied by value into kernels.
// kernel / gradients select the Table 1 variants; wnorm and dnorm are the
// kernel's normalisations, W = wnorm h^-3 g(q) and dW/dr = dnorm h^-4 f(q)
// with the shapes g and f of physics.cu.
struct KParams {
    int eos, n_target, n_tol, max_h_iter, periodic_z, precision, pair_threads, defer_lanes;
    int kernel, gradients, sinc_n;
    double rho0, c0, gamma, alpha, beta, eta2, cfl, lz, cell_scale;
    double wnorm, dnorm;
    double inv_rho0, tait_k;  // 1 / rho0 and c0^2 rho0 / 7, for the per-particle EOS
    double list_skin;         // candidate lists' skin (0: no lists)
};

enum { KER_M4 = 0, KER_WENDLAND = 1, KER_SINC = 2 };
enum { PREC_FP64 = 0, PREC_MIXED = 1, PREC_FP64_NATIVE = 2 };
constexpr double kPi = 3.14159265358979323846;
constexpr double kInvPi = 0.31830988618379067154;  // 1/pi
// B_n of the sinc kernel (host; Gauss-Legendre quadrature)
double sinc_norm(int n);

// Instances of a batch. Instance k holds the internal slots
// [ioff[k], ioff[k] + icnt[k]); ioff[k] is a multiple of kSlotAlign and the
// slots between the end of one instance and the start of the next are empty
// (skipped by every kernel). blk[b] is the instance of the slots
// [b kSlotAlign, (b + 1) kSlotAlign), so a 256-thread block, and each of its
// warps, belongs to one instance. A single problem is a batch of one with
// ioff[0] = 0: an instance is processed identically alone and in a batch.
constexpr int kSlotAlign = 256;
constexpr int kMaxInstances = 256;  // instance id = top 8 bits of the 32-bit sort key
constexpr int kMinInstanceCells = 4096;

struct Batch {
    const int32_t* blk;
    const int64_t* ioff;
    const int64_t* icnt;
    const Grid* grid;
    const KParams* kp;
};

__device__ __forceinline__ int slot_inst(const Batch& B, int64_t i) {
    return __ldg(&B.blk[i / kSlotAlign]);
}
__device__ __forceinline__ bool slot_real(const Batch& B, int inst, int64_t i) {
    return i - __ldg(&B.ioff[inst]) < __ldg(&B.icnt[inst]);
}

// Cells an instance of n particles may use.
inline long long instance_cell_cap(int64_t n) {
    const long long m = (long long)kMaxCellsPerAxis * kMaxCellsPerAxis * kMaxCellsPerAxis;
    long long c = 2 * (long long)n;
    if (c < kMinInstanceCells) c = kMinInstanceCells;
    return c < m ? c : m;
}

inline KParams kparams(const sph_params* p) {
    KParams k;
    k.eos = p->eos; k.n_target = p->n_target; k.n_tol = p->n_tol;
    k.max_h_iter = p->max_h_iter; k.periodic_z = p->periodic_z; k.precision = p->precision;
    k.rho0 = p->rho0; k.c0 = p->c0; k.gamma = p->gamma; k.alpha = p->alpha;
    k.beta = p->beta; k.eta2 = p->eta2; k.cfl = p->cfl; k.lz = p->lz;
    k.cell_scale = p->cell_scale > 0.0 ? p->cell_scale : 1.0;
    k.pair_threads = p->pair_threads > 0 ? p->pair_threads : 2;
    k.defer_lanes = p->defer_lanes > 0 ? p->defer_lanes : 16;
    k.kernel = p->kernel;
    k.gradients = p->gradients;
    k.sinc_n = p->sinc_n;
    k.inv_rho0 = p->rho0 != 0.0 ? 1.0 / p->rho0 : 0.0;
    k.tait_k = p->c0 * p->c0 * p->rho0 / 7.0;
    k.list_skin = p->list_skin > 0.0 ? p->list_skin : 0.0;
    if (p->kernel == KER_WENDLAND) {
        k.wnorm = 21.0 / (16.0 * kPi);
        k.dnorm = 105.0 / (16.0 * kPi);
    } else if (p->kernel == KER_SINC) {
        k.wnorm = sinc_norm(p->sinc_n);
        k.dnorm = k.wnorm * (0.5 * kPi);
    } else {
        k.wnorm = k.dnorm = kInvPi;
    }
    return k;
}

}  // namespace sph

struct sph_ctx {
    int device;
    int64_t ncap, nnzcap, cellcap;
    int64_t n;              // internal slots of the current batch (particles, plus the
                            // empty slots between instances)
    int64_t ntot;           // particles of the current batch
    int ninst, maxinst;     // instances of the current batch / capacity
    int prec;               // precision of the current batch
    int kern_kind, grad_kind;  // Table 1 variants of the current batch (KER_*, 0/1)
    int tpp;                // lanes per particle of the pair kernels (1, 2, 4, 8)
    int32_t* blk;           // instance of each block of kSlotAlign slots
    int64_t *ioff, *icnt, *coff;  // per instance: first slot, particles, first caller index
    int64_t* roff;          // per instance: first sort rank (sum of the earlier counts)
    int64_t cext;           // caller arrays must hold this many entries (max coff + icnt)
    sph::KParams* kpi;      // per-instance parameters
    int cur;                // current buffer of the double-buffered state
    double4_32a *posh[2], *velm[2];     // permuted with the particles (double-buffered)
    double* ue[2];                  // specific internal energy u
    double4_32a* therm;                 // recomputed every step after the sort
    double2* kern;
    double4_32a* acc;
    double* pint;
    double* cint;
    float4* dpk;            // 3 per particle: double-float pack of the force kernel
    float4* xpk;            // 3 per particle: exact fixed-point chunks of the position
                            // and the mass as a float pair (double-float pair kernels)
    float4* vpa;            // velocity as float pairs in the velocity unit of the pair
    float2* vpb;            // kernels: (vx.hi, vx.lo, vy.hi, vy.lo) and (vz.hi, vz.lo)
    float4* mpk;            // 5 per particle: pack of the mixed-precision pair kernels
    double* mumax;
    double4_32a* iad_a;     // IAD matrices C_i: (xx, xy, xz, yy) ...
    double2* iad_b;         // ... and (yz, zz)
    double* vol;            // IAD volume elements m / rho
    float2* vdf;            // the same as float pairs (double-float IAD)
    float4* cpk;            // 3 per particle: IAD matrix C_i as float pairs
    float4* fpos;
    float* tin;
    int32_t* order[2];
    uint32_t* keys[2];
    int32_t* vals[2];
    uint32_t* hist;         // 256 x sort blocks
    uint32_t* hist_part;    // scan partials of hist
    int2* cells;            // (start, end) per linear cell id
    unsigned long long* cell_hmax;  // per cell, bits of max h (h > 0)
    int32_t *nnb, *ngather, *rowlen;
    int64_t* offsets;
    int64_t* row_part;      // scan partials of the row lengths
    int32_t* idx;
    int32_t* rslab;         // kRSlab per particle: row i of S_i = the gather set of the last
                            // h-search count (ngather[i]), then the outer set (ocnt[i],
                            // r < 2 h_j only, sorted); rowlen[i] = ngather[i] + ocnt[i]
    bool csr_ready;         // offsets / idx hold the rows as a CSR
    int32_t* ocnt;          // outer-set sizes
    unsigned long long* omask;  // 2 per particle: bit e set when gather entry e of row i
                                // is a j with i not in N_j (the density kernel's
                                // record for the outer parts of precision 0)
    double *hs_lo, *hs_hi;  // bisection bracket of particles handed to the per-particle search
    int32_t* hs_it;         // counts already done for them
    int32_t* wl;            // their indices (count in status[3])
    double* red_part;       // bbox partials: kBoxStride per group of kSlotAlign slots
    double* dt_part;        // per force block (kMaxPairThreads per kThreads slots)
    sph::Grid* grid;        // per instance
    unsigned long long* wctr;  // work counters of persistent kernels (zeroed per build)
    int2* recs;             // h search records: kRec per lane of the persistent grid
    int64_t nslots;         // slot capacity (particles plus the gaps between instances)
    int32_t* lst;           // candidate lists: kList per slot (warp-interleaved); these
    sph::LMeta* lmeta;      // three are allocated by the first call that turns lists on;
    unsigned* lctr;         // their records per caller index; list builds so far
    bool any_lists;         // some instance of the current batch uses candidate lists
    int lay_n;              // instances of the last batch layout (first, count) ...
    int64_t lay_first[sph::kMaxInstances], lay_cnt[sph::kMaxInstances];  // ... and theirs
    int nsm;                // streaming multiprocessors of the device
    unsigned* status;       // [0] bits, [1] non-converged count, [2] internal flags,
                            // [3] h-search worklist length
    unsigned* status_host;  // pinned mirror
    double* scratch_scalar; // [0] internal dt, [1] internal time
    double* tune_dt;        // 2 x maxinst: dt and time of the autotuner's trial runs
    double* stage;          // sph_step_host staging: 17 x ncap doubles + time, dt (lazy)
    int32_t* stage_nnb;     // and ncap int32
    int64_t last_hnoconv;
    // launch accounting and optional per-phase event timing
    int64_t launches;
    int timing;
    cudaEvent_t* ev;        // event pool (ev_cap entries) when timing is on
    int* ev_phase;          // phase of each recorded marker (-1 = start of a call)
    int ev_cap, ev_used;
    int64_t mark_launches;  // launches at the previous marker
    int64_t phase_launches[SPH_NPHASES];
    int64_t timed_steps;
    // One step of the current batch as a CUDA graph, per parity of the
    // double-buffered state (cur at the start of the step), replayed by
    // sph_step / sph_batch_step instead of its ~35 separate launches.
    struct StepGraph {
        bool valid;
        int64_t key[10];         // what the launches bake in (sizes, kinds, dt/time pointers,
                                 // the bounding-box variant)
        cudaGraphExec_t exec;
        int64_t launches;        // kernels of one step
    } sg[2];
    cudaStream_t gstream;   // private stream the step graphs are captured on (lazy)
    char err[512];
};

namespace sph {

inline Batch batch_of(const sph_ctx* c) { return Batch{c->blk, c->ioff, c->icnt, c->grid, c->kpi}; }

// The pair sums run in the native FP64 kernels at precision 2; at precision
// 0 every kernel and gradient variant runs in double-float.
inline bool native_pairs(const sph_ctx* c) { return c->prec == PREC_FP64_NATIVE; }

// Rows of S_i for the pair kernels: the row slab unless a row overflowed it
// (device flag IF_SLAB_OVF), in which case the CSR built by the fallback.
struct Rows {
    const int32_t* rslab;
    const int32_t* idx;
    const int64_t* offsets;
    const int32_t* rowlen;   // |S_i| (either form)
    const int32_t* ngather;  // |N_i|: the first ngather[i] entries of a row
    const unsigned* status;
    int64_t nnzcap;
    unsigned mask;           // internal flags that send the reads to the CSR
};

// Rows of S_i once complete (either overflow flag selects the CSR).
inline Rows rows_of(const sph_ctx* c) {
    return Rows{c->rslab, c->idx, c->offsets, c->rowlen, c->ngather, c->status, c->nnzcap,
                (unsigned)(IF_SLAB_OVF | IF_OUTER_OVF)};
}

// Gather parts only, for the density kernel that completes the outer parts
// itself: an outer overflow raised while it runs must not switch its reads.
inline Rows rows_gather(const sph_ctx* c) {
    Rows r = rows_of(c);
    r.mask = IF_SLAB_OVF;
    return r;
}

// At precision 0 and 1 the step's density kernel also decides the outer parts
// of the rows (k_density_df / k_density_mx with OUTER, then k_append_outer);
// at precision 2 and outside a step, k_outer builds them before the density.
inline bool fused_outer(const sph_ctx* c) { return c->prec == PREC_FP64 || c->prec == PREC_MIXED; }

// The defining FP64 squared distance, operation by operation (minimum image
// along z when periodic): (dx dx + dy dy) + dz dz, each operation rounded.
__device__ __forceinline__ double exact_r2_def(const double4_32a& a, const double4_32a& b,
                                               bool periodic_z, double lz) {
    const double dx = __dsub_rn(a.x, b.x), dy = __dsub_rn(a.y, b.y);
    double dz = __dsub_rn(a.z, b.z);
    if (periodic_z) {
        const double half = __dmul_rn(0.5, lz);
        if (dz > half) dz = __dsub_rn(dz, lz);
        else if (dz < -half) dz = __dadd_rn(dz, lz);
    }
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Entries and length of row i (the whole row, or its gather part); false when
// the rows cannot be read (a fallback CSR over capacity).
__device__ __forceinline__ bool row_of(const Rows& R, int64_t n, int64_t i, bool gather_only,
                                       const int32_t*& ent, int& len) {
    if (!(R.status[2] & R.mask)) {
        ent = R.rslab + i * kRSlab;
    } else {
        if (R.offsets[n] > R.nnzcap) return false;
        ent = R.idx + R.offsets[i];
    }
    len = gather_only ? R.ngather[i] : R.rowlen[i];
    return true;
}

// ---- sph_abi.cu
// Describe a single problem of n particles (a batch of one) on the stream.
void launch_set_single(sph_ctx* c, const KParams& kp, int64_t n, cudaStream_t s);
void lists_for_layout(sph_ctx* c, int ninst, const int64_t* first, const int64_t* cnt,
                      cudaStream_t s);
void lists_clear(sph_ctx* c, cudaStream_t s);
// One step of the current batch on the context's state (dt, time: ninst each).
void launch_step(sph_ctx* c, double* dt, double* time, cudaStream_t s);

// ---- sort.cu
void launch_load_state(sph_ctx* c, const sph_particles* P, cudaStream_t s);
void launch_gather_state(sph_ctx* c, const sph_particles* P, const KParams& kp, int what,
                         cudaStream_t s);
void launch_build_cells(sph_ctx* c, cudaStream_t s);

// ---- neighbors.cu
void launch_h_search(sph_ctx* c, cudaStream_t s);
// the rows of S_i (slab form; the full two-pass CSR build if a row overflows);
// with outer_later the outer parts are left to the density kernel, and
// launch_rows_finish completes the rows after it
void launch_csr(sph_ctx* c, cudaStream_t s, bool outer_later = false);
void launch_rows_finish(sph_ctx* c, cudaStream_t s);
// the rows as a CSR in offsets / idx (a copy in slab form; nothing after a fallback)
void launch_compose(sph_ctx* c, cudaStream_t s);

// ---- physics.cu
enum { GATHER_DENSITY = 1, GATHER_FORCES = 2 };
void launch_density(sph_ctx* c, bool fuse_eos, cudaStream_t s, bool outer = false);
// ---- physics_df.cu (precision 0)
void launch_density_df(sph_ctx* c, bool fuse_eos, cudaStream_t s, bool outer = false);
void launch_forces_df(sph_ctx* c, cudaStream_t s);
void launch_forces_iad_df(sph_ctx* c, cudaStream_t s);  // IAD: volumes, matrices, forces
// ---- physics_mixed.cu (precision 1)
void launch_pack_mx(sph_ctx* c, bool thermo, cudaStream_t s);
void launch_density_mx(sph_ctx* c, bool fuse_eos, cudaStream_t s, bool outer = false);
void launch_forces_mx(sph_ctx* c, cudaStream_t s);
void launch_eos_caller(const KParams& kp, const sph_particles* P, cudaStream_t s);
// forces, then per instance dt[k] = cfl min_i (...) and time[k] += dt[k]
// (dt_out, time_inout: device arrays of ninst entries; time_inout may be NULL)
void launch_forces(sph_ctx* c, double* dt_out, double* time_inout, cudaStream_t s);
void launch_leapfrog(sph_ctx* c, const double* dt, cudaStream_t s);
void launch_scatter(sph_ctx* c, const sph_particles* P, unsigned fields, cudaStream_t s);

enum : unsigned {
    SC_POS = 1u, SC_VEL = 2u, SC_H = 4u, SC_U = 8u, SC_RHO = 16u, SC_PC = 32u,
    SC_ACC = 64u, SC_MUMAX = 128u, SC_NNB = 256u,
};

// ---- scan.cu
// exclusive scan of n int32 into n+1 int64 (out[n] = total); with gate, only
// when *gate & mask is set on the device when the kernels run
void launch_scan_i32_i64(const int32_t* in, int64_t n, int64_t* out, int64_t* part,
                         cudaStream_t s, const unsigned* gate = nullptr, unsigned mask = 0u);
// exclusive scan in place over n uint32
void launch_scan_u32(uint32_t* data, int64_t n, uint32_t* part, cudaStream_t s);
int64_t scan_parts(int64_t n);

}  // namespace sph
