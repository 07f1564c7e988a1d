/*
 * pic.h -- C ABI of libpic, a single-GPU (sm_103a) electromagnetic particle-in-cell engine for
 * the relativistic-electron-beam Weibel / filamentation problem of Karmakar, Kumar, Shvets,
 * Polomarov & Pukhov, "On collisions driven negative energy waves and Weibel instability of a
 * relativistic electron beam in a quasi-neutral plasma" (arXiv:0808.4078).
 *
 * Physics covered (paper passages):
 *   - 2D geometry: the plane transverse to a beam along z, no z dependence; 3D runs with the
 *     beam along z (simulation section);
 *   - beam and background (return-current) electrons, immobile ions of density n0, initial
 *     current neutralisation (simulation section);
 *   - collisional friction on the return current, Eq. (3) (d v_pz/dt + nu v_pz = ...), applied
 *     as a per-cell relaxation of the drag species' mean momentum at rate nu (Krook reading);
 *   - field-energy diagnostic, integral of F_i^2 dx dy per component (simulation section);
 *   - growth rate of the exponential stage of the magnetic energy (results section).
 * The paper gives no PIC algorithm; the discretisation is CIC gather + relativistic Boris push,
 * charge-conserving Esirkepov current deposit, Yee FDTD, periodic boundaries.
 *
 * Units: time 1/w_p, length c/w_p, momentum u = gamma v / c, fields m c w_p / e, density n0,
 * current e n0 c.  A particle is a cell (x fastest) plus FP32 in-cell offsets in [0, 1) and FP32
 * momenta; on the device particles are binned per cell (the cell index is implied by the slot)
 * and re-binned every step; push and gather are FP32; the current is accumulated in int64 fixed
 * point (bit-reproducible); global energy/momentum reductions are FP64.
 *
 * Conventions
 *   - Every function returns PIC_OK (0) or a negative PIC_E* code; pic_last_error() gives text.
 *     No C++ exception crosses this boundary.
 *   - Device memory: the caller allocates ONE device arena of pic_required_bytes() bytes and
 *     keeps it (and the CUDA stream) alive until pic_free().  The library never calls
 *     cudaMalloc for state; it carves the arena.  Host buffers passed in are copied during the
 *     call; host buffers passed out are written before the call returns.
 *   - All GPU work is issued on the caller's stream, asynchronously, except where a function
 *     says it synchronises.  Device-side error flags are sticky and reported by the next call
 *     that synchronises (pic_sync, pic_diag, pic_get_*).
 *   - Arrays of fields are [nz][ny][nx] (x fastest).  Yee staggering (2D):
 *     Ex(i+1/2,j) Ey(i,j+1/2) Ez(i,j) Bx(i,j+1/2) By(i+1/2,j) Bz(i+1/2,j+1/2); J like E.
 *     3D: Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2) Bx(i,j+1/2,k+1/2) By(i+1/2,j,k+1/2)
 *     Bz(i+1/2,j+1/2,k).
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_OK 0
#define PIC_EINVAL (-1)     /* bad argument or configuration */
#define PIC_ENOMEM (-2)     /* arena smaller than pic_required_bytes(), capacity exceeded, or (device,
                               sticky) a species' spill list full: raise cell_capacity */
#define PIC_ECUDA (-3)      /* a CUDA runtime call failed */
#define PIC_EOVERFLOW (-4)  /* fixed-point headroom exceeded.  Reserved: the per-run shift S bounds
                               every current term by 2^21 (|v| < c), so no int32 warp sum or int64
                               node sum can overflow and this version never returns it */
#define PIC_EBADPART (-5)   /* non-finite or out-of-range particle data at load (nothing is
                               loaded), or on the device a particle whose new position would lie
                               a cell or more away (a non-finite momentum, e.g. from non-finite
                               fields; the Courant check at init excludes it otherwise): the
                               particle stays where it was, unmoved and not deposited, and the
                               sticky flag fails the next synchronising call */
#define PIC_ETIMEOUT (-6)   /* a bounded device wait gave up */
#define PIC_ESTATE (-7)     /* call not valid in the current state */
#define PIC_EBOUNDS (-8)    /* (bounds-checked debug build, libpic_debug.so, only) a kernel's
                               shared-tile or halo index fell outside its array: the access was
                               skipped and the sticky flag fails the next synchronising call */

#define PIC_MAX_SPECIES 2

/* Flags for pic_config.flags */
#define PIC_FLAG_PROFILE 1   /* time each kernel phase with CUDA events (disables graphs) */
#define PIC_FLAG_NO_GRAPH 2  /* launch steps directly instead of replaying a CUDA graph */
#define PIC_FLAG_KEEP_J 4    /* keep a copy of the last step's J for pic_get_fields (tests) */
#define PIC_FLAG_NVTX 8      /* NVTX ranges: one per pic_step call and one per phase of every step
                                (push_deposit, yee, finalize, sort); launches steps directly so
                                that every phase is visible (no graph) */

typedef struct pic_ctx pic_ctx;

typedef struct pic_config {
    int32_t ndim;              /* 2 (2D3V) or 3 (3D3V) */
    int32_t nx, ny, nz;        /* cells per axis; nz = 1 in 2D; multiples of the tile sizes */
    double dx, dy, dz, dt;     /* cell sizes (c/w_p) and time step (1/w_p); Yee Courant limit */
    int32_t nspecies;          /* 1..PIC_MAX_SPECIES */
    int64_t capacity[PIC_MAX_SPECIES];      /* particle capacity per species (< 2^31) */
    int32_t cell_capacity[PIC_MAX_SPECIES]; /* particle slots per cell per species; 0 = automatic
                                               (2D: 8 x the mean per cell, multiple of 32,
                                               >= 32; 3D: 3 x the mean, multiple of 8, >= 16);
                                               must be >= 2 x capacity / cells.  In 3D the
                                               slots of a tile's cells form one range per tile
                                               (a particle may sit anywhere in its tile's) */
    int32_t sort_interval;     /* steps between checks for a full counting sort that repacks
                                  spilled particles (particles whose cell's slots were full,
                                  held in a list of a quarter of the species' capacity; the sort
                                  runs when a list has grown by > 1/16 of its size since the last
                                  sort);
                                  0 = default (8) */
    int32_t diag_interval;     /* steps between diagnostic records; 0 = no diagnostics */
    int32_t diag_capacity;     /* records kept in the device history ring (>= 1 if diag) */
    int32_t track_ids;         /* 1: carry an int32 id per particle (its load index) */
    int32_t flags;             /* PIC_FLAG_* */
    int32_t tile_x, tile_y, tile_z; /* cells per tile of the particle kernels: 2D 16 x 16,
                                       32 x 8 or 8 x 32 (tile_z ignored); 3D 8 x 8 x 4; other
                                       values are rejected; 0 = default (16 x 16 in 2D) */
    int32_t j_filter;          /* 1: smooth the step's current with one binomial 1-2-1 pass per
                                  axis (periodic) before the E update, against numerical
                                  Cherenkov radiation of the relativistic beam on the Yee grid
                                  (not in the paper); the sum is exact in int64 and scaled by
                                  4^-ndim; pic_get_fields returns the unfiltered J; 0 = off */
    int32_t ctas_per_sm;       /* 2D particle kernel: CTAs per SM its registers are budgeted
                                  for (2, 3 or 4); 0 = default (3); ignored in 3D */
} pic_config;

typedef struct pic_species {
    double q;      /* charge in units of e (electrons: -1) */
    double m;      /* mass in units of m_e (electrons: 1) */
    double w;      /* density carried by one macro-particle, units n0 (n_s / ppc) */
    double nu;     /* Krook rate on this species' cell-mean momentum (Eq. (3) friction); 0 = none */
} pic_species;

typedef struct pic_diag_rec {
    int64_t step;                    /* n */
    double t;                        /* n dt */
    double WE[3], WB[3];             /* sum over cells of F_i^2 dx dy (dz) at time n */
    double Ekin[PIC_MAX_SPECIES];    /* sum w (gamma(u^n) - 1) dx dy (dz), u^n = (u^{n-1/2}+u^{n+1/2})/2 */
    double P[3];                     /* sum over all species of w u^n dx dy (dz) */
    int32_t flags;                   /* device error flags seen by this step */
    int32_t reserved;
} pic_diag_rec;

typedef struct pic_kernel_time {
    char name[32];
    int64_t launches;
    double total_ms;                 /* sum of CUDA-event intervals on the context stream */
} pic_kernel_time;

/* Bytes of device arena needed for cfg.  Host-only; no CUDA call. */
int pic_required_bytes(const pic_config* cfg, size_t* bytes_out);

/* Create a context on the current CUDA device.  device_arena: caller-owned device memory of
 * arena_bytes >= pic_required_bytes(cfg), aligned to 256 bytes; cuda_stream: a cudaStream_t
 * (not the legacy default stream if graphs are used).  Fields start at E = B = 0. */
int pic_init(const pic_config* cfg, void* device_arena, size_t arena_bytes, void* cuda_stream,
             pic_ctx** out);

/* Batched scan: one context holding nruns independent 2D runs of different sizes that step
 * together (one set of launches, one CUDA graph, for all runs).  run_dims[3*r .. 3*r+2] = nx, ny,
 * nz of run r (nz ignored in 2D); run_capacity[PIC_MAX_SPECIES*r + s] = particle capacity of
 * species s in run r.  cfg supplies everything else (ndim, dx, dy, dz, dt, nspecies,
 * cell_capacity, sort_interval, diag_*, track_ids, flags, tiles); cfg->nx/ny/nz/capacity are
 * not used.  Each run keeps its own fields, species parameters (q must agree across runs) and
 * diagnostic history.  Same ownership and error rules as pic_required_bytes / pic_init. */
int pic_required_bytes_batch(const pic_config* cfg, int nruns, const int32_t* run_dims,
                             const int64_t* run_capacity, size_t* bytes_out);
int pic_init_batch(const pic_config* cfg, int nruns, const int32_t* run_dims,
                   const int64_t* run_capacity, void* device_arena, size_t arena_bytes,
                   void* cuda_stream, pic_ctx** out);
int pic_num_runs(const pic_ctx* ctx);

/* Load n particles of species index s (0-based) from HOST arrays: cell[n] (linear index,
 * x fastest), offset[ndim*n] (component-major: all x offsets, then y, then z; each in [0,1)),
 * u[3*n] (component-major u_x, u_y, u_z).  Copies, validates (PIC_EBADPART on a bad value),
 * bins the particles by cell (counting sort) and computes the cell-mean momentum used by the
 * drag.  When all three arrays are memory the device can address (pinned or registered host
 * memory, or device memory) the binning kernel reads them in place; other host arrays are
 * copied to the device first.  The arrays are not used after the call returns.  The initial u
 * is u^{-1/2}; particle i gets id i.  Each species is loaded once, before the first step.
 * Synchronises the stream. */
int pic_load_species(pic_ctx* ctx, int s, const pic_species* sp, int64_t n, const int32_t* cell,
                     const float* offset, const float* u);
/* The same for run `run` of a batch (cell indices local to the run); pic_load_species = run 0. */
int pic_load_species_run(pic_ctx* ctx, int run, int s, const pic_species* sp, int64_t n,
                         const int32_t* cell, const float* offset, const float* u);

/* Advance nsteps steps: gather + Boris + drag + move + Esirkepov deposit + re-binning of every
 * particle into its new cell, Yee update, a full counting sort every sort_interval steps when
 * the spill lists have grown (see sort_interval), diagnostics every diag_interval steps.
 * Asynchronous. */
int pic_step(pic_ctx* ctx, int nsteps);

/* Wait for the stream; report sticky device errors. */
int pic_sync(pic_ctx* ctx);

/* Wait for the stream, write the sticky device error bits to *flags_out (may be NULL; bit 1:
 * a non-finite or out-of-range particle, which the step kept unmoved and left out of the
 * current; 2: fixed-point headroom; 4: a bounded wait gave up; 8: a spill list was full; 16: an
 * index out of range in the bounds-checked debug build) and
 * clear them, so that a caller can read back the state that produced the error.  The state
 * after an error is the step's result for every particle that did not raise it.  PIC_OK. */
int pic_clear_flags(pic_ctx* ctx, int32_t* flags_out);

/* Copy up to max_recs diagnostic records (oldest first) to out.  Synchronises. */
int pic_diag(pic_ctx* ctx, pic_diag_rec* out, int max_recs, int* n_out);
int pic_diag_run(pic_ctx* ctx, int run, pic_diag_rec* out, int max_recs, int* n_out);

/* Copy species s to HOST arrays (any may be NULL): cell[n], offset[ndim*n], u[3*n], id[n]
 * (id requires track_ids).  Particles come in cell order (the order within a cell is not
 * fixed), then the spill list; n must equal the loaded count.  Synchronises. */
int pic_get_particles(pic_ctx* ctx, int s, int32_t* cell, float* offset, float* u, int32_t* id,
                      int64_t n);
int pic_get_particles_run(pic_ctx* ctx, int run, int s, int32_t* cell, float* offset, float* u,
                          int32_t* id, int64_t n);

/* Copy fields to HOST arrays (any may be NULL): E[3*ncell], B[3*ncell] component-major FP32;
 * J[3*ncell] int64 fixed point of the last step's current (J = value * 2^-shift, shift from
 * pic_fixed_point_shift); J needs PIC_FLAG_KEEP_J (PIC_ESTATE otherwise).  Synchronises. */
int pic_get_fields(pic_ctx* ctx, float* E, float* B, int64_t* J);
int pic_get_fields_run(pic_ctx* ctx, int run, float* E, float* B, int64_t* J);

/* Overwrite E and B from HOST arrays (component-major FP32, 3*ncell each).  Test and restart
 * use.  Synchronises. */
int pic_set_fields(pic_ctx* ctx, const float* E, const float* B);

/* Fixed-point shift S of the current accumulator (J_int = round(J * 2^S)). */
int pic_fixed_point_shift(const pic_ctx* ctx, int* shift_out);

/* Growth rate of W_B_perp = WB[0] + WB[1] from the device history (FP64 fit on the GPU):
 * noise level W0 = mean over t <= t_noise; windows of `width` records with all
 * W > start_factor * W0 and W < end_factor * max(W) (end_factor <= 0: no upper bound);
 * least-squares slope of ln W, largest over windows; Gamma = slope / 2.  gamma_out is NaN if
 * no window qualifies.  Synchronises. */
int pic_fit_growth(pic_ctx* ctx, int width, double t_noise, double start_factor,
                   double end_factor, double* gamma_out, double* t0_out, double* t1_out);
int pic_fit_growth_run(pic_ctx* ctx, int run, int width, double t_noise, double start_factor,
                       double end_factor, double* gamma_out, double* t0_out, double* t1_out);

/* Per-phase CUDA-event timings (PIC_FLAG_PROFILE).  Synchronises. */
int pic_kernel_times(pic_ctx* ctx, pic_kernel_time* out, int max, int* n_out);

typedef struct pic_stats {
    int64_t particles[PIC_MAX_SPECIES];   /* particles held (slots + spill list) */
    int32_t max_cell[PIC_MAX_SPECIES];    /* largest count of one binning unit (2D: a cell; 3D: a
                                             tile of the 3D particle kernel); may exceed the
                                             capacity */
    int32_t spilled[PIC_MAX_SPECIES];     /* particles in the spill list */
    int32_t cell_capacity[PIC_MAX_SPECIES];  /* slots per unit (2D: per cell; 3D: per tile, the
                                                tile's cells' cell_capacity together) */
    int32_t flags;                        /* sticky device error flags */
    int32_t reserved;
} pic_stats;

/* Occupancy of the particle bins of the current buffer.  Synchronises. */
int pic_get_stats(pic_ctx* ctx, pic_stats* out);

/* Closure-driven drag: replace the Krook rate of species s in run `run` by per-coarse-cell rates
 * nu (device float[(nx / bx) (ny / by)], the layout of pic_record_moments and pic_mlp_forward's
 * output; a coarse cell spans the whole z extent in 3D).  Each cell's factor 1 - exp(-nu dt) is
 * taken once at this call (negative or NaN rates act as 0); the drag then uses the factor of the
 * particle's cell.  Enables the drag for a species loaded with nu = 0.  nu == NULL restores the
 * species' scalar rate.  At most one species per run carries the drag (PIC_EINVAL otherwise).
 * Synchronises the context's stream; nu may be freed on return. */
int pic_set_drag_map(pic_ctx* ctx, int run, int s, const float* nu, int32_t bx, int32_t by);

/* Checkpoint and resume.  pic_checkpoint synchronises the context's stream and writes its whole
 * state to the file `path`: the device arena (particles in both buffers, spill lists, fields, J,
 * drag moments and maps, diagnostic history, control block with the step counter) and the host
 * state (species parameters, particle counts, Krook and collision settings, step count).  It
 * writes `path`.tmp first and renames it, so an existing checkpoint is replaced only by a
 * complete one.  A context with a sticky device error is not written (that error is returned).
 * pic_restore loads such a file into a context created by pic_init / pic_init_batch with the
 * same configuration (grids, capacities, species count, cell_capacity, dx..dt, sort_interval,
 * diag_interval / diag_capacity, track_ids, j_filter, PIC_FLAG_KEEP_J; PIC_FLAG_PROFILE and
 * PIC_FLAG_NO_GRAPH may differ), with or without species loaded; it replaces the context's whole
 * state and the run continues bit for bit as if it had not been interrupted (integer current
 * deposits, counter-based collision draws keyed by particle id and step).  A file of another
 * configuration, another library version, or of the wrong size returns PIC_EINVAL and leaves
 * the context unchanged (every check precedes the first copy; a read or CUDA error during the
 * copy leaves a partial state).  Launch counters and profiling timers are not part of the state.
 * Both synchronise; the file is read/written through a 64 MB host buffer. */
int pic_checkpoint(pic_ctx* ctx, const char* path);
int pic_restore(pic_ctx* ctx, const char* path);

/* Particles of species s loaded in run `run` (after a restore: those of the checkpoint); -1 on a
 * bad argument. */
int64_t pic_loaded_count(const pic_ctx* ctx, int run, int s);

/* Binary electron-ion collisions of species s in run `run` (the paper's collision model; its
 * scheme is not given there): every step, after the Boris push and any Krook drag, each particle's
 * momentum turns by a scattering angle theta with tan(theta / 2) ~ N(0, nu dt / 2) about a
 * uniform azimuth (Takizuka & Abe, J. Comput. Phys. 25, 205 (1977), with an immobile ion as the
 * partner), which keeps |u| and relaxes the mean momentum at the rate nu to first order in
 * nu dt.  The draws of particle p at step n are Philox4x32-10 (Salmon et al., SC'11) of the
 * counter (id_p, n, s) under the 64-bit key `seed`, so the context must carry particle ids
 * (track_ids); PIC_EINVAL otherwise.  nu = 0 switches the collisions off.  Synchronises. */
int pic_set_collisions(pic_ctx* ctx, int run, int s, double nu, uint64_t seed);

/* Growth rates of the collisional filamentation of a warm beam, Eq. (12) of the paper,
 *   w^2 = c_s^2 k^2 - w_b^2 beta0^2 k^2 / (k^2 + k_pe^2 / (1 + i nu / w)),
 * in units k_pe = c / w_p = 1, w_b^2 = n_b (the theory line for the temperature / collision-rate
 * scan).  params: device double[nsets][4] = (c_s^2, beta0, n_b, nu) per set; k scans nk
 * uniform points of [kmin, kmax].  gamma_out, kstar_out: device double[nsets], the largest
 * imaginary part of w over the k grid and the k where it occurs (the lowest such k).  The
 * relation is non-relativistic (the paper's), so a comparison with the relativistic runs is
 * qualitative.  Asynchronous on `stream`. */
int pic_dispersion_growth(const double* params, int32_t nsets, double kmin, double kmax, int32_t nk,
                          double* gamma_out, double* kstar_out, void* stream);

/* ---------------------------------------------------------------- hybrid model
 * The paper's quasi-neutral model (Eqs. 1-6) as a simulation of its own: a kinetic electron beam
 * in the transverse plane, the plasma return current as a fluid and the axial vector potential
 * from Ampere's law without the displacement current.  Units as above, a = e A_z / (m c^2):
 *   lap a = n_b beta_bz + n_p beta_p,  n_p = n0 - n_b   (Eq. 2; quasi-neutral plasma density)
 *   d beta_p / dt + nu beta_p = d a / dt                (Eq. 3)
 *   d u_perp / dt = -(beta_z - beta_p) grad a            (Eq. 4)
 *   u_z = P + a, P conserved per particle               (Eq. 6)
 * Without collisions the energy of Eq. 7 (beam, magnetic, plasma kinetic with the local n_p) is
 * an invariant; pic_hybrid_energies returns its three parts.
 * Periodic nx x ny grid (powers of two in [8, 2048]), a and beta_p at nodes (FP64), 5-point
 * Laplacian, CIC interpolation and deposit, particles FP32 (cell + offset).  A step pushes the
 * beam in the old fields, deposits its density and current at the new positions, solves
 * (lap - n_p) a^{n+1} = n_b beta_b + n_p (beta_p^n - a^n - nu dt beta_p^n) with
 * n_p = max(n0 - n_b, 0) per node (FP64 residual, FP32 conjugate-gradient correction
 * preconditioned by the constant-density spectral solve, stopped at a relative residual of tol or
 * after max_iter iterations) and updates beta_p^{n+1} = beta_p^n + a^{n+1} - a^n - nu dt beta_p^n.
 * The beam is kept in cell order by a counting sort every sort_interval steps; deposits are exact
 * integer sums, so results do not depend on the order.  Particle read-back is in the load order.
 * Steps replay a CUDA graph of one step unless a flag asks otherwise.  Host arrays are copied
 * during the calls; the arena (pic_hybrid_required_bytes, 256-byte aligned) and the stream belong
 * to the caller.  Deterministic: results do not depend on particle order or scheduling. */
typedef struct pic_hybrid pic_hybrid;
typedef struct pic_hybrid_config {
    int32_t nx, ny;             /* nodes per axis, powers of two in [8, 2048] */
    double dx, dy, dt;          /* c/w_p, 1/w_p; dt < dx and dt < dy */
    double n0;                  /* total electron density (1 in these units), > 0 */
    double nu;                  /* collision rate of the plasma flow, >= 0 */
    double w;                   /* beam density per macro-particle and cell, >= 0 */
    int64_t capacity;           /* beam particles, <= 2^31 */
    double tol;                 /* relative residual of the solve; 0 = 1e-5 */
    int32_t max_iter;           /* conjugate-gradient iterations per step; 0 = 16, <= 1000 */
    int32_t flags;              /* PIC_FLAG_PROFILE (phase timing, no graph), PIC_FLAG_NO_GRAPH */
    int32_t sort_interval;      /* steps between counting sorts of the beam by cell (keeps the
                                   deposit's lanes on shared cells); 0 = 16 */
} pic_hybrid_config;
int pic_hybrid_required_bytes(const pic_hybrid_config* cfg, size_t* bytes_out);
int pic_hybrid_init(const pic_hybrid_config* cfg, void* device_arena, size_t arena_bytes,
                    void* cuda_stream, pic_hybrid** out);
/* Beam particles (host: X, Y in cell units within the grid, momenta u = gamma beta) and the
 * plasma velocity beta_p at the nodes (host, ny x nx); a starts at 0, so P = u_z.
 * PIC_EBADPART for particles outside the grid or non-finite values.  Synchronous. */
int pic_hybrid_load(pic_hybrid* h, int64_t n, const double* X, const double* Y, const double* ux,
                    const double* uy, const double* uz, const double* beta_p);
int pic_hybrid_step(pic_hybrid* h, int nsteps);          /* asynchronous on the stream */
/* Read back (host arrays, any may be NULL): a and beta_p (ny x nx), particle X, Y, ux, uy in the
 * load order.  Synchronises. */
int pic_hybrid_get(pic_hybrid* h, double* a, double* beta_p, double* X, double* Y, double* ux,
                   double* uy);
/* Magnetic energy sum |D+ a|^2 / 2 dx dy, beam kinetic energy sum w (gamma - 1) dx dy and plasma
 * kinetic energy sum n_p beta_p^2 / 2 dx dy; deterministic.  Synchronises. */
int pic_hybrid_energies(pic_hybrid* h, double out3[3]);
/* {steps, conjugate-gradient iterations in total, steps that stopped at max_iter above tol,
 * iterations of the last step}.  Synchronises. */
int pic_hybrid_stats(pic_hybrid* h, int64_t out4[4]);
/* With PIC_FLAG_PROFILE: CUDA-event time on the stream per phase ("push_deposit", "field_solve",
 * "update", "sort"), accumulated over the steps so far; same record as pic_kernel_times.
 * Synchronises. */
int pic_hybrid_kernel_times(pic_hybrid* h, pic_kernel_time* out, int max, int* n_out);
/* Kernels launched by pic_hybrid_step so far: per step the push, the solve set-up and the update,
 * per conjugate-gradient iteration 4 kernels (5 in a graph, whose while node runs only the
 * iterations needed; direct launches run max_iter, returning at once after convergence), and 8
 * per sort.  Synchronises; -1 on error. */
int64_t pic_hybrid_launch_count(pic_hybrid* h);
int64_t pic_hybrid_step_count(const pic_hybrid* h);
void pic_hybrid_free(pic_hybrid* h);

/* ---------------------------------------------------------------- moment recorder
 * Coarse-grained state of run `run` at the current step: the inputs and the label parts of a
 * learned collision closure.  The paper's conclusion conjectures that the collisional friction on
 * the return current could be written through the local plasma state; the closure's inputs and
 * label are not given there, so these rows are this library's reading of it.
 *
 * Coarse cell = bx x by transverse cells x the whole z extent (3D) or bx x by cells (2D); bx, by
 * must divide nx, ny.  ncoarse = (nx / bx) (ny / by), numbered x fastest.  Particles count in the
 * coarse cell of the cell that holds them; species 0 is the beam (b), species 1 the background
 * (p), weights w as loaded.  out[row * ncoarse + c], float, rows:
 *   0 n_b, 1 n_p        sum w / cells of the coarse cell (density, units n0)
 *   2 uz_b, 3 uz_p      w-weighted mean u_z
 *   4 Tperp_b, 5 Tpar_b (Var u_x + Var u_y) / 2 and Var u_z of the beam (w-weighted variances of
 *   6 Tperp_p, 7 Tpar_p  the momentum u = gamma v / c), the same for the background
 *   8 W_ES              mean over the coarse cell's cells of sum_c (E_c - <E_c>_z)^2 with <E_c>_z
 *                       the mean of the stored E_c over the z column (0 in 2D)
 *   9 Fz_p              w-weighted mean of q (E + v x B)_z over the background particles, E and B
 *                       interpolated to each particle (CIC on the Yee lattice), v = u / gamma
 *   10 Fz_mean          q (Ebar_z + vbar_x Bbar_y - vbar_y Bbar_x): Ebar, Bbar means of the stored
 *                       fields over the coarse cell, vbar the background's mean velocity
 *   11 nu_eff           nu_p + (Fz_mean - Fz_p) / uz_p (0 where uz_p = 0), nu_p the background's
 *                       Krook rate; a single snapshot (a time average over 1/w_p averages rows
 *                       3, 9, 10 over snapshots first)
 * out: device memory of >= PIC_MOM_ROWS * ncoarse floats (out_cap floats).  scratch: device
 * memory of >= pic_record_moments_scratch_bytes() bytes, 8-byte aligned; both owned by the caller
 * and in use until the context's stream passes the call.  Particle sums are int64 fixed point, so
 * the record is bitwise reproducible.  Asynchronous on the context's stream; *ncoarse_out (may be
 * NULL) = ncoarse.  PIC_EINVAL on bad blocks, sizes, alignment or fewer than 2 species. */
#define PIC_MOM_ROWS 12
int pic_record_moments_scratch_bytes(pic_ctx* ctx, int run, int bx, int by, size_t* bytes_out);
int pic_record_moments(pic_ctx* ctx, int run, int bx, int by, float* out, int64_t out_cap,
                       void* scratch, size_t scratch_bytes, int64_t* ncoarse_out);

/* ---------------------------------------------------------------- closure network
 * The network that maps the coarse moments (rows 0..8 of pic_record_moments, or the first 8
 * without W_ES) to the friction rate nu_eff -- this library's reading of the closure the paper's
 * conclusion conjectures:
 *   xn = (x - mu) / sigma (features >= nin are 0),  h1 = silu(W1 xn + b1),  h2 = silu(W2 h1 + b2),
 *   y = w3 . h2 + b3,  silu(z) = z / (1 + exp(-z)),
 * W1 64 x 9, W2 64 x 64.  The two hidden layers run on the tensor cores with bfloat16 weights and
 * inputs and FP32 accumulation; the rest is FP32.
 * params: device float[PIC_MLP_NPARAM] in the order W1[64][9], b1[64], W2[64][64], b2[64],
 * w3[64], b3.  x: device float, feature-major, x[j * ldx + i] for feature j of sample i (the
 * moment recorder's output with ldx = ncoarse).  All device buffers are owned by the caller. */
#define PIC_MLP_IN 9
#define PIC_MLP_HIDDEN 64
#define PIC_MLP_NPARAM 4865
typedef struct pic_mlp_norm {
    float mu[PIC_MLP_IN];      /* per-feature offset */
    float sigma[PIC_MLP_IN];   /* per-feature scale (> 0) */
    int32_t nin;               /* inputs used: 9, or 8 for the variant without W_ES */
} pic_mlp_norm;

/* y[i] (device float[n]) = network(x[:, i]).  Asynchronous on `stream` (a cudaStream_t). */
int pic_mlp_forward(const float* params, const pic_mlp_norm* norm, const float* x, int64_t ldx,
                    int64_t n, float* y, void* stream);
/* One full-batch Adam step (beta1 0.9, beta2 0.999, eps 1e-8; t >= 1 the step number, adam_m and
 * adam_v device float[PIC_MLP_NPARAM] moment estimates, zero before t = 1) on the mean squared
 * error of y against target[n] (device); params updated in place; *loss (device float, may be
 * NULL) = the loss before the update.  scratch: device memory of >= pic_mlp_train_scratch_bytes()
 * bytes, 4-byte aligned, in use until the stream passes the call.  Deterministic: the gradient is
 * summed in a fixed order.  Asynchronous on `stream`. */
int pic_mlp_train_scratch_bytes(size_t* bytes_out);
int pic_mlp_train_step(float* params, float* adam_m, float* adam_v, int32_t t, float lr,
                       const pic_mlp_norm* norm, const float* x, int64_t ldx, const float* target,
                       int64_t n, float* loss, void* scratch, size_t scratch_bytes, void* stream);
/* Input normalisation of the network from its training set: per feature j < nin the mean and
 * the population standard deviation (FP64 sums in a fixed order) of x[j * ldx + i], i < n,
 * written to mu_sigma (device float[2 * PIC_MLP_IN]: the 9 means, then the 9 deviations;
 * features >= nin get 0 and 1, a constant feature a deviation of 1).  Asynchronous on `stream`. */
int pic_mlp_fit_norm(const float* x, int64_t ldx, int64_t n, int32_t nin, float* mu_sigma, void* stream);

/* Training samples of the closure from a series of moment snapshots -- this library's reading
 * of the conclusion's conjecture that the two-stream turbulence of a 3D run acts on the return
 * current like a collision rate, averaged over a time of order 1/w_p.  rows: device
 * float[nsnap][PIC_MOM_ROWS][nc], consecutive pic_record_moments outputs of one run.  Windows of
 * `window` consecutive snapshots (nsnap / window of them; a remainder is ignored) are averaged;
 * for window w and coarse cell c the sample's features are the window means of rows 0..8 and its
 * label is nu_p + (<Fz_mean> - <Fz_p>) / <uz_p> (nu_p: the background's Krook rate of the run).
 * A sample is kept where |<uz_p>| >= uz_min (below it the return current has stopped and the
 * ratio is ill-conditioned) and the label is finite.  Kept samples are written in (window, cell)
 * order: feat (device float, feature-major, feat[j * cap + i], j < 9), label (device float[cap]);
 * *n_out (device int64) = the number kept (only the first cap are written).  scratch: device
 * memory of >= pic_closure_samples_scratch_bytes(nsnap / window * nc) bytes, 16-byte aligned.
 * PIC_EINVAL on bad sizes or null pointers.  Asynchronous on `stream`. */
int pic_closure_samples_scratch_bytes(int64_t nsamples, size_t* bytes_out);
int pic_closure_samples(const float* rows, int32_t nsnap, int64_t nc, int32_t window, float nu_p, float uz_min,
                        float* feat, float* label, int64_t cap, int64_t* n_out, void* scratch,
                        size_t scratch_bytes, void* stream);

/* PIC_OK, or PIC_ETIMEOUT if a tensor-core completion wait of the network kernels gave up
 * (sticky until read with clear != 0).  The outputs of a call during which a wait gave up are
 * undefined: a kernel that times out waits once more (also bounded) for the tensor cores before
 * it frees its tensor memory and returns, and the network's results of that call are not
 * written in full.  Synchronous. */
int pic_mlp_status(int clear);

/* Test hook of the bounded wait above: one CTA on `stream` waits on a completion barrier that
 * nothing arrives on, with no tensor-core work issued, giving up after `polls` polls
 * (1 <= polls <= 2^20); the give-up sets the flag pic_mlp_status reports.  Asynchronous. */
int pic_mlp_wait_test(int64_t polls, void* stream);

/* Counting sort by cell, the binning primitive of the re-binning step, on caller device memory:
 * cell[n] (device) holds each particle's cell in [0, ncell); writes start[ncell + 1] (device;
 * start[c] = number of particles in cells below c) and order[n] (device; order[start[c] ..
 * start[c+1]) are the indices of the particles of cell c, in no fixed order within a cell).
 * Particles whose cell lies outside [0, ncell) are left out (start[ncell] counts the others).
 * scratch: caller device memory of at least pic_bin_cells_scratch_bytes(ncell) bytes, 256-byte
 * aligned, owned by the caller, not needed after the stream reaches the end of the call.
 * Asynchronous on `stream` (a cudaStream_t); PIC_EINVAL on bad sizes or null pointers. */
int pic_bin_cells_scratch_bytes(int32_t ncell, size_t* bytes_out);
int pic_bin_cells(const int32_t* cell, int64_t n, int32_t ncell, int32_t* start, int32_t* order,
                  void* scratch, size_t scratch_bytes, void* stream);

/* Allocation-free variant of pic_bin_cells, for callers that cannot allocate device memory
 * themselves: for example code embedded in a host application whose GPU memory belongs to
 * another allocator it cannot reach, or a timing-critical loop where a cudaMalloc (which can
 * synchronise the device) is not allowed.  The paper has no counterpart; this is a library
 * convenience.  Inputs and outputs are the caller's, exactly as for pic_bin_cells; the scratch
 * is a fixed array compiled into the library (PIC_BIN_NOALLOC_MAX_CELLS cells, about 4.2 MB),
 * which every GPU that loads the library holds until the process exits.  ncell above the
 * maximum returns PIC_EINVAL.  The first call on a device looks up that device's copy of the
 * array (make it before any stream capture); later calls reuse it.  All calls share the one
 * array: calls that may run at the same time on the GPU (different streams) race and must be
 * ordered by the caller.  Each call clears the part of the array that must start at zero.
 * Calls no cudaMalloc, cudaFree or other allocating routine.  Asynchronous on `stream`. */
#define PIC_BIN_NOALLOC_MAX_CELLS (1 << 20)
int pic_bin_cells_noalloc(const int32_t* cell, int64_t n, int32_t ncell, int32_t* start,
                          int32_t* order, void* stream);

/* Autotuner of the 2D particle kernel's compiled variants (tile shape 16 x 16, 32 x 8 or 8 x 32
 * cells; 2, 3 or 4 CTAs per SM; every one computes the same bits).  The next steps of the run
 * are taken with each variant whose tile divides every run's grid in turn: sort_interval steps to
 * warm up (graph capture), then steps_per_variant (rounded up to a multiple of sort_interval)
 * timed with CUDA events on the context's stream; the run stays exactly what it would have been
 * with any one variant.  The fastest variant is kept for the rest of the run and recorded in the
 * tuning cache under the key (dimension, grids, particles per run, GPU name): in memory and, if
 * a cache file is set (pic_tune_cache_set, or the environment variable PIC_TUNE_CACHE), in that
 * file (one JSON object per line, rewritten through path.tmp and a rename).  A context
 * created with tile_x = tile_y = ctas_per_sm = 0 whose key is cached starts with the cached
 * variant.  out (host, may be NULL when max_entries is 0) receives one entry per variant timed
 * (up to max_entries; *n_out the number written).  In 3D (one kernel) the step is timed and
 * nothing is chosen.  Synchronises. */
typedef struct pic_tune_entry {
    int32_t tile_x, tile_y, ctas_per_sm;   /* ctas_per_sm: tile_z in 3D */
    float ms_per_step;
} pic_tune_entry;
int pic_autotune(pic_ctx* ctx, int steps_per_variant, pic_tune_entry* out, int max_entries, int* n_out);
/* Set the tuning-cache file (NULL: memory only) and load its entries; replaces the in-memory
 * cache.  PIC_OK. */
int pic_tune_cache_set(const char* path);
/* The particle kernel's configuration: out3 = {tile_x, tile_y, ctas_per_sm} in 2D,
 * {tile_x, tile_y, tile_z} in 3D. */
int pic_tile_config(const pic_ctx* ctx, int32_t* out3);

/* Kernel launches issued so far by this context (graph replays count their kernel nodes). */
int64_t pic_launch_count(const pic_ctx* ctx);

/* Steps taken so far. */
int64_t pic_step_count(const pic_ctx* ctx);

/* Last error message of ctx (or of the last failed pic_init when ctx is NULL). */
const char* pic_last_error(const pic_ctx* ctx);

/* Destroy the context (does not free the caller's arena or stream). */
void pic_free(pic_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* PIC_H */
