// pic_internal.cuh -- device-side data structures shared by the libpic kernels.
//
// Layout in HBM (all carved from the caller's arena):
//   particles  per species, two buffers (sort ping-pong), SoA: cell int32, offset float x ndim,
//              u float x 3, optional id int32.  The cell index is the run-global index
//              (run cell offset + local index, x fastest).
//   fields     E[3], B[3] float per cell; J[3] int64 fixed point per cell.
//   drag       per cell: sum u (3 x int64, fixed point 2^20), count int32, and the cell-mean
//              momentum <u> (3 x float) of the previous step used by the Krook drag.
//   sort       count / start / cursor int32 per key; keys are tile-major cell indices so a
//              tile's particles are contiguous after a sort.
//   diag       FP64 per-CTA field-energy partials, int64 kinetic/momentum accumulators, history.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define PIC_NS 2                 // species slots
#define PIC_MOM_SHIFT 20         // fixed-point shift of the drag moments (u * 2^20 as int32)
#define PIC_KIN_SHIFT 32         // fixed-point shift of the kinetic/momentum diagnostics

namespace pic {

// Error flags (device word, sticky)
enum : int { ERR_BADPART = 1, ERR_OVERFLOW = 2, ERR_TIMEOUT = 4 };

struct SpeciesParams {
    float qmdt2;        // q dt / (2 m)
    float jx, jy, jz;   // -q w (dx/dt) 2^S, -q w (dy/dt) 2^S, (-q w (dz/dt) 2^S in 3D | q w 2^S in 2D)
    float dragf;        // 1 - exp(-nu dt); 0 = no drag
    float w;            // weight (density per macro-particle)
    int drag;           // accumulate cell moments and apply the drag
    int active;         // species loaded
};

struct RunDev {
    int nx, ny, nz;
    int ntx, nty, ntz;      // tiles per axis
    int cell_off;           // offset of this run's cells/keys in the global key space
    int shift;              // fixed-point shift S of J
    float dtdx, dtdy, dtdz; // dt / dx: displacement in cells per unit velocity per step
    float cx, cy, cz;       // dt / dx for the Yee curls
    float jscale;           // 2^-S
    float* E[3];
    float* B[3];
    long long* J[3];
    long long* Jlast[3];    // copy of the last step's J (test mode), or null
    long long* msum[3];     // drag moments being accumulated (this step)
    int* mcnt;
    float* ubar[3];         // previous step's cell-mean momentum
    SpeciesParams sp[PIC_NS];
};

struct SpeciesBuf {
    int* cell;
    float* o[3];
    float* u[3];
    int* id;
};

// Device control block (lives in the arena, updated by kernels)
struct Ctl {
    long long step;              // steps completed
    int parity[PIC_NS];          // which particle buffer is current
    int err;                     // sticky error flags
    int pad;
    long long kin[PIC_NS][4];    // kinetic energy + momentum accumulators (diag steps)
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
    const int2* work;            // (run, tile) per CTA of the tiled kernels
    int nwork;
    int nspecies;
    SpeciesBuf buf[PIC_NS][2];
    int* start[PIC_NS];          // exclusive scan of per-key counts (tile ranges)
    int* count[PIC_NS];
    int* cursor[PIC_NS];
    long long nkeys;             // total keys (= total cells)
    long long npart[PIC_NS];     // loaded particles per species (all runs)
    double* partials;            // [nwork][8] field-energy partials of a diag step
    DiagRec* hist;
    int hist_cap;
    int diag_interval;
    double dt;
    double dV;
    int* scan_tmp;               // block sums of the scan
    int ndim;
    int nruns;
};

__device__ __forceinline__ int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Round x to the nearest integer (ties to even) for |x| < 2^22 with one FFMA: adding 1.5*2^23
// leaves the integer in the low mantissa bits.
__device__ __forceinline__ int round_small(float a, float b) {
    float t = __fmaf_rn(a, b, 12582912.0f);
    return __float_as_int(t) - 0x4B400000;
}

}  // namespace pic

// Host-side launchers (defined in the .cu files)
namespace pic {
cudaError_t launch_push2d(const Args& a, cudaStream_t s);
cudaError_t launch_push3d(const Args& a, cudaStream_t s);
bool has_push3d();
cudaError_t launch_yee2d(const Args& a, const RunDev* host_runs, int nruns, cudaStream_t s);
cudaError_t launch_yee3d(const Args& a, const RunDev* host_runs, int nruns, cudaStream_t s);
cudaError_t launch_finalize(const Args& a, cudaStream_t s);
cudaError_t launch_sort(const Args& a, int species, int tile_x, int tile_y, int tile_z,
                        cudaStream_t s);
int sort_launches(long long n);
cudaError_t launch_moments_init(const Args& a, int species, cudaStream_t s);
cudaError_t launch_moments_finalize(const Args& a, const RunDev* host_runs, int nruns,
                                    cudaStream_t s);
cudaError_t launch_validate(const Args& a, int species, long long first, long long n,
                            int run, cudaStream_t s);
cudaError_t launch_fit(const Args& a, long long first, int nrec, int width, double t_noise,
                       double start_factor, double end_factor, double* out3, cudaStream_t s);
}  // namespace pic
