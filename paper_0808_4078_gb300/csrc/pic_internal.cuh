// pic_internal.cuh -- device-side data structures shared by the libpic kernels.
//
// Layout in HBM (all carved from the caller's arena):
//   particles  binned by unit (2D: a cell; 3D: a tile of the 3D particle kernel): species s
//              keeps, per unit, a slot range of fixed capacity cap[s] holding that unit's
//              particles (SoA: offsets float x ndim, momenta float x 3, optional id int32, and in
//              3D the particle's cell within its tile) plus per-unit counts.  In 2D the cell
//              index is implied by the slot.  Two buffers: every step reads buffer `parity` and
//              writes each particle into its new unit's slots of the other buffer (a counting
//              sort fused into the push).  Particles that find their new unit full go to a
//              per-species spill list (cell index stored), processed by its own kernel.
//   fields     E[3], B[3] float per cell; J[3] int64 fixed point per cell.
//   drag       per cell: sum u (3 x int64, fixed point 2^20), count int32, and the cell-mean
//              momentum <u> (3 x float) of the previous step used by the Krook drag.
//   diag       FP64 per-CTA field-energy partials, int64 kinetic/momentum accumulators, history.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define PIC_NS 2                 // species slots
#define PIC_BLK 32               // slots per block of the particle arrays
#define PIC_MOM_SHIFT 20         // fixed-point shift of the drag moments
#define PIC_KIN_SHIFT 32         // fixed-point shift of the kinetic/momentum diagnostics

namespace pic {

// Error flags (device word, sticky)
enum : int { ERR_BADPART = 1, ERR_OVERFLOW = 2, ERR_TIMEOUT = 4, ERR_SPILL_FULL = 8, ERR_BOUNDS = 16 };

// Index checks of the bounds-checked debug build (compiled with -DPIC_DEBUG_BOUNDS): a failed
// check sets ERR_BOUNDS and the caller skips the access.  In the normal build every check is
// true at compile time and costs nothing.
#ifdef PIC_DEBUG_BOUNDS
__device__ __forceinline__ bool dbg_in(long long i, long long n, int* err) {
    const bool ok = i >= 0 && i < n;
    if (!ok) atomicOr(err, ERR_BOUNDS);
    return ok;
}
#else
__device__ __forceinline__ constexpr bool dbg_in(long long, long long, int*) { return true; }
#endif

struct SpeciesParams {
    float qmdt2;        // q dt / (2 m)
    float jx, jy, jz;   // -q w (dx/dt) 2^S, -q w (dy/dt) 2^S, (-q w (dz/dt) 2^S in 3D | q w 2^S in 2D)
    float dragf;        // 1 - exp(-nu dt); 0 = no drag
    float w;            // weight (density per macro-particle)
    int drag;           // accumulate cell moments and apply the drag
    int active;         // species loaded
    int coll;           // binary electron-ion collisions on
    float coll_sigma;   // sqrt(nu_coll dt / 2): standard deviation of tan(theta / 2)
    unsigned seed_lo, seed_hi;   // key of the collision draws
};

struct RunDev {
    int nx, ny, nz;
    int ntx, nty, ntz;      // tiles per axis
    int work_off;           // global index of the run's first tile (= its first work item)
    int cell_off;           // offset of this run's cells in the global cell space
    int shift;              // fixed-point shift S of J
    float dtdx, dtdy, dtdz; // dt / dx: displacement in cells per unit velocity per step
    float cx, cy, cz;       // dt / dx for the Yee curls
    float jscale;           // 2^-S
    float* E[3];
    float* B[3];
    long long* J[3];
    long long* Jlast[3];    // copy of the last step's J (test mode), or null
    long long* Jf[3];       // binomially filtered J (weights summing to 4^ndim), or null
    float jfscale;          // 2^-S / 4^ndim
    long long* msum[3];     // drag moments being accumulated (this step)
    int* mcnt;
    float* ubar[3];         // previous step's cell-mean momentum
    float* dragmap[PIC_NS]; // per-cell drag factor 1 - exp(-nu_c dt) replacing sp[s].dragf, or null
    SpeciesParams sp[PIC_NS];
};


// One species in one buffer.  A unit's cap slots are a stay area [0, cap_stay), filled by the
// CTA that owns the unit's tile (count = its fill: in 2D the cell's stayers and the particles
// that reach it from other cells of the same tile; in 3D every particle that ends the step in
// the tile it started in), and an immigrant area [cap_stay, cap) that the other particles
// arriving in the unit claim with an atomic counter (icount).  Counters may exceed their area;
// readers clamp them (the excess went to the spill list).  A unit is a cell in 2D and a tile in
// 3D (unit index = global tile index = the tile's work item; lc holds each particle's cell
// within the tile, x fastest).
// Slot arrays are stored in blocks of PIC_BLK consecutive slots: a block holds PIC_BLK values of
// each array in turn (o_x, o_y[, o_z], u_x, u_y, u_z[, id]), so that one address per particle
// reaches all its values and a warp reading 32 consecutive slots reads whole 128-byte lines.  Slot
// q of array X is X[slot_elt(S, q)]; o[d], u[d] and id point at their array in block 0.
struct Slots {
    float* o[3];     // offsets (x, y[, z])
    float* u[3];     // momenta
    int* id;         // or null
    int* lc;         // 3D: cell of the particle within its tile; null in 2D
    long long bstride;   // floats per block (PIC_BLK x arrays)
    int* count;      // [nunit] stay-area fill
    int* icount;     // [nunit] immigrant-area fill
    // spill list (particles whose cell was full)
    int* scell;      // global cell index
    float* so[3];
    float* su[3];
    int* sid;
    int* sn;         // number of spilled particles
};

// Device control block (lives in the arena, updated by kernels)
struct Ctl {
    long long step;              // steps completed
    int parity;                  // particle buffer read by the next step
    int err;                     // sticky error flags
    int staged[PIC_NS];          // particles in the staging area after the last compaction
    int spill_base[PIC_NS];      // spill-list fill right after the last re-sort
};

struct DiagRec {                 // mirrors pic_diag_rec
    long long step;
    double t;
    double WE[3], WB[3];
    double Ekin[PIC_NS];
    double P[3];
    int flags;
    int reserved;
};

struct Args {
    Ctl* ctl;
    const RunDev* runs;
    const int2* work;            // (run, tile) per CTA of the tiled kernels, runs in order
    const int* work_off;         // [nruns + 1] first work item of each run
    long long* kin;              // [nruns][PIC_NS][4] kinetic energy + momentum (diag steps)
    int nwork;
    int tx, ty, tz;              // tile shape of the tiled kernels (cells per axis)
    int push_variant;            // which compiled variant of the particle kernel runs (0 = default)
    int anydrag;                 // some run has a Krook-drag species (host copy of the run table)
    int nspecies;
    int nruns;
    int ndim;
    Slots slot[PIC_NS][2];
    int cap[PIC_NS];             // slots per unit (2D: cell, 3D: tile)
    int cap_stay[PIC_NS];        // of which the stay area
    int spill_cap[PIC_NS];
    long long ncell;             // total cells (all runs)
    long long nunit;             // total units (2D: ncell, 3D: nwork)
    double* partials;            // [nwork][8] field-energy partials of a diag step
    DiagRec* hist;               // [nruns][hist_cap]
    int hist_cap;
    int diag_interval;
    double dt;
    double dV;
    int* scan_tmp;               // block sums of the scan
    int* start;                  // [ncell + 1] exclusive scan of clamped counts (compaction)
    int* gate;                   // device flag of the conditional re-sort
    // Staging area of species s when buffer b is the current one: the slot memory of the OTHER
    // buffer viewed as flat arrays of stage_n[s] entries: cell, o[ndim], u[3], id.
    char* stage[PIC_NS][2];
    long long stage_n[PIC_NS];
    // 2D particle kernel: crossers of a cell edge are deposited after a CTA's main loop.  CTA b
    // queues them in xq + b * xq_cap entries (Crosser); past xq_cap they go to the overflow list
    // xo (xo_cap entries, fill *xo_n, cleared every step), deposited by the spill kernel.
    struct Crosser* xq;
    int xq_cap;
    struct CrosserX* xo;
    int* xo_n;
    int xo_cap;
};

// A particle that crossed a cell edge, pushed: old and new offsets, u^{n+1/2}, v_z, and a meta
// word (species bit 0, tile cell bits 1-10, x and y cell steps + 1 bits 11-12 and 13-14, bad
// bit 15), id.  A bad particle (non-finite push) carries its old state and no steps.
struct __align__(16) Crosser {
    float4 o;      // ox, oy, nox, noy
    float4 u;      // ux, uy, uz, vz
    int2 m;        // meta, id
    int2 pad;
};
// Overflow entry: the crosser and its old cell (global index).
struct __align__(16) CrosserX {
    Crosser c;
    int cell;
    int pad[3];
};

// Flat staging arrays (see Args::stage).
struct Stage {
    int* cell;
    float* o[3];
    float* u[3];
    int* id;
};
__host__ __device__ inline Stage stage_of(const Args& a, int s, int par) {
    Stage t;
    char* b = a.stage[s][par];
    const long long n = a.stage_n[s];
    t.cell = reinterpret_cast<int*>(b);
    for (int d = 0; d < 3; ++d) t.o[d] = d < a.ndim ? reinterpret_cast<float*>(b + 4 * n * (1 + d)) : nullptr;
    for (int d = 0; d < 3; ++d) t.u[d] = reinterpret_cast<float*>(b + 4 * n * (1 + a.ndim + d));
    t.id = reinterpret_cast<int*>(b + 4 * n * (4 + a.ndim));
    return t;
}

// Particles of unit c: n = stay part + immigrant part; element k lives in slot slot_of(k).
struct CellRange {
    int ns, n;
};
__device__ __forceinline__ CellRange cell_range(const Slots& S, int cap, int cap_stay, long long c) {
    CellRange r;
    r.ns = min(S.count[c], cap_stay);
    r.n = r.ns + min(S.icount[c], cap - cap_stay);
    return r;
}
__device__ __forceinline__ size_t slot_of(long long c, int cap, int cap_stay, int ns, int k) {
    return (size_t)c * cap + (k < ns ? k : cap_stay + (k - ns));
}
// Element of slot q in the slot arrays (see Slots).
__host__ __device__ __forceinline__ size_t slot_elt(const Slots& S, long long q) {
    return (size_t)(q / PIC_BLK) * (size_t)S.bstride + (size_t)(q % PIC_BLK);
}

__device__ __forceinline__ int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Run holding global cell g (runs are stored in cell order).
__device__ __forceinline__ int run_of_cell(const Args& a, long long g) {
    int lo = 0, hi = a.nruns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.runs[mid].cell_off <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}
// Run holding global tile (unit) T.
__device__ __forceinline__ int run_of_unit(const Args& a, long long T) {
    int lo = 0, hi = a.nruns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.runs[mid].work_off <= T) lo = mid; else hi = mid - 1;
    }
    return lo;
}
// Unit of global cell g and, in 3D, the cell's index within its tile (*lc).
__device__ __forceinline__ long long unit_of_cell(const Args& a, long long g, int* lc) {
    if (a.ndim != 3) {
        *lc = 0;
        return g;
    }
    const RunDev& R = a.runs[run_of_cell(a, g)];
    const long long l = g - R.cell_off;
    const long long nxy = (long long)R.nx * R.ny;
    const int z = (int)(l / nxy), rem = (int)(l - (long long)z * nxy);
    const int y = rem / R.nx, x = rem - y * R.nx;
    const int tx = x / a.tx, ty = y / a.ty, tz = z / a.tz;
    *lc = ((z - tz * a.tz) * a.ty + (y - ty * a.ty)) * a.tx + (x - tx * a.tx);
    return R.work_off + ((long long)tz * R.nty + ty) * R.ntx + tx;
}
// Global cell of the particle with in-tile cell lc in 3D unit T of run R.
__device__ __forceinline__ long long cell_of_unit(const Args& a, const RunDev& R, long long T, int lc) {
    const long long t = T - R.work_off;
    const int tx = (int)(t % R.ntx), ty = (int)((t / R.ntx) % R.nty), tz = (int)(t / ((long long)R.ntx * R.nty));
    lc %= a.tx * a.ty * a.tz;
    const int lx = lc % a.tx, ly = (lc / a.tx) % a.ty, lz = lc / (a.tx * a.ty);
    return R.cell_off + ((long long)(tz * a.tz + lz) * R.ny + (ty * a.ty + ly)) * R.nx + (tx * a.tx + lx);
}

// Round a*b to the nearest integer (ties to even) for |a*b| < 2^22 with one FFMA: adding
// 1.5*2^23 leaves the integer in the low mantissa bits.
__device__ __forceinline__ int round_small(float a, float b) {
    float t = __fmaf_rn(a, b, 12582912.0f);
    return __float_as_int(t) - 0x4B400000;
}

}  // namespace pic

// Host-side launchers (defined in the .cu files)
namespace pic {
// Load every kernel of the module now (lazy loading would otherwise add the first launch's
// load time to whatever step first uses a kernel).
cudaError_t preload_push2d();
cudaError_t preload_push3d();
cudaError_t preload_bins();
cudaError_t preload_fields();
cudaError_t launch_push2d(const Args& a, cudaStream_t s);
// Compiled variants of the 2D particle kernel: index for a tile shape and CTAs per SM (minb 0:
// the default, 3), or -1; count; shape of variant v.
int push2d_variant(int tx, int ty, int minb);
int push2d_num_variants();
void push2d_variant_info(int v, int* tx, int* ty, int* minb);
cudaError_t launch_push3d(const Args& a, cudaStream_t s);
bool has_push3d();
void push3d_tile(int t[3]);   // the 3D particle kernel's tile shape (cells per axis)
cudaError_t launch_spill2d(const Args& a, cudaStream_t s);
cudaError_t launch_spill3d(const Args& a, cudaStream_t s);
cudaError_t launch_yee2d(const Args& a, const RunDev* host_runs, int nruns, cudaStream_t s);
cudaError_t launch_yee3d(const Args& a, const RunDev* host_runs, int nruns, cudaStream_t s);
cudaError_t launch_finalize(const Args& a, cudaStream_t s);   // per-run records, then step++, flip
cudaError_t launch_clear_next(const Args& a, cudaStream_t s);
// Counting sort into the per-unit slots and its inverse.  All use the device parity: the
// current buffer's slots and the staging area in the other buffer's memory.  `gate` (device int,
// may be null) makes the kernels return at once when it holds 0.
//   launch_bin:     staging (n particles; n < 0: the count of the last compaction), or the
//                   device-addressable arrays *src when src is given, -> slots of the current
//                   buffer; staged cells are cell_base + value, valid if value is in
//                   [0, ncell_lim); ids kept if with_ids, else the staging index
//   launch_compact: the slots of units [c0, c0 + nc) and the spill entries of cells
//                   [cell_lo, cell_lo + ncells) of the current buffer -> staging in unit order,
//                   cell values written minus cell_base
cudaError_t launch_bin(const Args& a, int species, long long n, bool with_ids, long long cell_base,
                       long long ncell_lim, const int* gate, cudaStream_t s, const Stage* src = nullptr);
cudaError_t launch_compact(const Args& a, int species, long long c0, long long nc, long long cell_lo,
                           long long ncells, long long cell_base, const int* gate, cudaStream_t s);
cudaError_t launch_spill_gate(const Args& a, cudaStream_t s);
cudaError_t launch_clear_current(const Args& a, int species, const int* gate, cudaStream_t s);
// Standalone counting sort by cell (pic_bin_cells): scratch = count/cursor[ncell] + block sums.
size_t bin_cells_scratch_bytes(long long ncell);
cudaError_t launch_bin_cells(const int* cell, long long n, int ncell, int* start, int* order, int* scratch,
                             cudaStream_t s);
// Device address of the fixed scratch array of pic_bin_cells_noalloc (current device).
cudaError_t noalloc_bin_scratch(int** out);
// Full re-sort of every species (compact, clear, bin) when any particle is in a spill list.
cudaError_t launch_resort(const Args& a, cudaStream_t s, int* launches);
// Drag moments of the loaded particles of `species` in run `run` (units [u0, u0 + nu) of the
// current buffer and the run's spill entries).
cudaError_t launch_moments_init(const Args& a, int species, int run, long long u0, long long nu,
                                cudaStream_t s);
cudaError_t launch_moments_finalize(const Args& a, int run, long long ncell, cudaStream_t s);
// Moment recorder (moments.cu): scratch bytes for nc coarse cells and ncol columns, and the
// launch (psum cleared, particle and spill sums, field columns, finalisation into out).
size_t moments_scratch_bytes(long long nc, long long ncol);
cudaError_t launch_moments(const Args& a, const RunDev& host_run, int run, int bx, int by, float q_bg,
                           float nu_bg, float* out, void* scratch, cudaStream_t s);
cudaError_t preload_moments();
// Closure network (mlp.cu): per-feature normalisation x' = (x - mu) * inv_sigma of the first nin
// inputs (the others are 0).
struct MlpNorm {
    float mu[9];
    float inv_sigma[9];
    int nin;
};
size_t mlp_train_scratch_bytes();
cudaError_t launch_mlp_forward(const float* params, const MlpNorm& norm, const float* x, long long ldx, long long n,
                               float* y, cudaStream_t s);
cudaError_t launch_mlp_train(float* params, float* am, float* av, int t, float lr, const MlpNorm& norm,
                             const float* x, long long ldx, const float* target, long long n, float* loss,
                             void* scratch, cudaStream_t s);
cudaError_t mlp_status(int* err, bool clear);
// Closure training samples and the network's input normalisation (closure.cu).
size_t closure_samples_scratch_bytes(long long m);
cudaError_t launch_closure_samples(const float* rows, int nsnap, long long nc, int window, float nu_p, float uz_min,
                                   float* feat, float* label, long long cap, long long* n_out, void* scratch,
                                   cudaStream_t s);
cudaError_t launch_fit_norm(const float* x, long long ldx, long long n, int nin, float* mu_sigma, cudaStream_t s);
// One CTA waiting on a barrier nothing arrives on, giving up after `polls` polls (test hook).
cudaError_t launch_mlp_wait_test(long long polls, cudaStream_t s);
// cudaFuncAttributeMaxDynamicSharedMemorySize of kernel fn, set once per device (the attribute
// is per device).
cudaError_t smem_attr_once(const void* fn, int bytes);
cudaError_t preload_mlp();
// Per-cell drag factors of run `run` from per-coarse-cell rates nu (bx x by blocks).
cudaError_t launch_drag_map(const RunDev& host_run, float* map, const float* nu, int bx, int by, double dt,
                            cudaStream_t s);
// Growth rates of the collisional filamentation dispersion relation (dispersion.cu).
cudaError_t launch_dispersion(const double* params, int nsets, double kmin, double kmax, int nk, double* gamma,
                              double* kstar, cudaStream_t s);
// Error text of a failed context-free call (pic_last_error(NULL)).
void set_call_error(const char* msg);
cudaError_t launch_fit(const Args& a, int run, long long first, int nrec, int width, double t_noise,
                       double start_factor, double end_factor, double* out3, cudaStream_t s);
}  // namespace pic
