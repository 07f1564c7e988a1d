// capi.cu -- the C ABI of libpic (include/pic.h): context, arena carving, particle loading,
// step scheduling (a CUDA graph of sort_interval steps), diagnostics, growth fit, profiling.
//
// A context holds one or more independent runs (a batch): each run has its own grid, fields,
// species parameters and diagnostic history; particles of all runs share the binned slot
// arrays (global cell index = run cell offset + local cell), and every kernel covers all runs
// through the (run, tile) work list, so a batch steps with the same launches as a single run.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <cstdlib>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pic.h"
#include "pic_internal.cuh"

using namespace pic;

static_assert(sizeof(pic_diag_rec) == sizeof(DiagRec), "diag record layout");
static_assert(PIC_MAX_SPECIES == PIC_NS, "species slots");

namespace {

thread_local std::string g_init_error;

enum Phase { PH_PUSH = 0, PH_YEE, PH_FINAL, PH_SORT, PH_N };
const char* kPhaseName[PH_N] = {"push_deposit", "yee", "finalize", "sort"};

struct RunGeo {
    int nx, ny, nz;
    int ntx, nty, ntz;
    long long ncell, ntiles;
    long long cell_off, work_off;
    long long capacity[PIC_NS];
};

struct Geometry {
    int tx, ty, tz;
    int push_variant;         // compiled variant of the 2D particle kernel (tile shape, CTAs/SM)
    long long ncell, nwork;
    long long nunit;          // particle units: cells (2D) or tiles (3D)
    int cap[PIC_NS];          // slots per unit per species
    int cap_stay[PIC_NS];     // of which the stay area
    int spill_cap[PIC_NS];
    long long capacity[PIC_NS];   // particles per species, all runs
    std::vector<RunGeo> runs;
};

struct Layout {
    size_t total = 0;
    size_t ctl, runs, work, work_off, kin;
    size_t so[PIC_NS][2][3], su[PIC_NS][2][3], sid[PIC_NS][2], slc[PIC_NS][2], scount[PIC_NS][2], sicount[PIC_NS][2];
    size_t sp_cell[PIC_NS][2], sp_o[PIC_NS][2][3], sp_u[PIC_NS][2][3], sp_id[PIC_NS][2], sp_n[PIC_NS][2];
    size_t slot_region[PIC_NS][2];   // start of the contiguous slot arrays (staging view)
    std::vector<size_t> E[3], B[3], J[3], Jlast[3], Jf[3], msum[3], mcnt, ubar[3];   // per run
    std::vector<size_t> dragmap[PIC_NS];                                     // per run
    size_t start, scan_tmp, gate;
    size_t xq, xo, xo_n;             // 2D crosser queues and their overflow list
    int xq_cap = 0, xo_cap = 0;
    size_t partials, hist, fit;
};

size_t take(size_t& off, size_t bytes) {
    off = (off + 255) & ~size_t(255);
    size_t at = off;
    off += bytes;
    return at;
}

int geometry(const pic_config* c, int nruns, const int32_t* dims, const int64_t* caps, Geometry* g,
             std::string* err) {
    if (c->ndim != 2 && c->ndim != 3) { *err = "ndim must be 2 or 3"; return PIC_EINVAL; }
    if (c->ndim == 3 && !pic::has_push3d()) { *err = "3D push not available in this build"; return PIC_EINVAL; }
    if (nruns < 1 || nruns > 65536) { *err = "nruns must be in [1, 65536]"; return PIC_EINVAL; }
    int t3[3];
    pic::push3d_tile(t3);
    const int dtx = c->ndim == 3 ? t3[0] : 16, dty = c->ndim == 3 ? t3[1] : 16, dtz = c->ndim == 3 ? t3[2] : 1;
    g->tx = c->tile_x > 0 ? c->tile_x : dtx;
    g->ty = c->tile_y > 0 ? c->tile_y : dty;
    g->tz = c->ndim == 3 ? (c->tile_z > 0 ? c->tile_z : dtz) : 1;
    g->push_variant = 0;
    if (c->ndim == 2) {
        if (c->ctas_per_sm < 0 || c->ctas_per_sm == 1 || c->ctas_per_sm > 4) { *err = "ctas_per_sm must be 0, 2, 3 or 4"; return PIC_EINVAL; }
        g->push_variant = pic::push2d_variant(g->tx, g->ty, c->ctas_per_sm);
        if (g->push_variant < 0) { *err = "2D tiles are 16 x 16, 32 x 8 or 8 x 32"; return PIC_EINVAL; }
    }
    if (c->ndim == 3 && (g->tx != t3[0] || g->ty != t3[1] || g->tz != t3[2])) {
        *err = "3D tiles must have the shape of the 3D particle kernel (pic_tile_config)";
        return PIC_EINVAL;
    }
    if (!(c->dx > 0 && c->dy > 0 && c->dt > 0) || (c->ndim == 3 && !(c->dz > 0))) { *err = "dx, dy, dz, dt must be > 0"; return PIC_EINVAL; }
    const double inv2 = 1.0 / (c->dx * c->dx) + 1.0 / (c->dy * c->dy) + (c->ndim == 3 ? 1.0 / (c->dz * c->dz) : 0.0);
    if (c->dt * std::sqrt(inv2) >= 1.0) { *err = "dt violates the Yee Courant condition"; return PIC_EINVAL; }
    if (c->nspecies < 1 || c->nspecies > PIC_NS) { *err = "nspecies must be 1..2"; return PIC_EINVAL; }
    if (c->diag_interval < 0 || (c->diag_interval > 0 && c->diag_capacity < 1)) { *err = "diag_capacity must be >= 1"; return PIC_EINVAL; }
    if (c->sort_interval < 0) { *err = "sort_interval must be >= 0"; return PIC_EINVAL; }
    if (c->j_filter != 0 && c->j_filter != 1) { *err = "j_filter must be 0 or 1"; return PIC_EINVAL; }
    g->runs.assign(nruns, RunGeo{});
    g->ncell = 0;
    g->nwork = 0;
    for (int s = 0; s < PIC_NS; ++s) g->capacity[s] = 0;
    for (int r = 0; r < nruns; ++r) {
        RunGeo& R = g->runs[r];
        R.nx = dims[3 * r];
        R.ny = dims[3 * r + 1];
        R.nz = c->ndim == 3 ? dims[3 * r + 2] : 1;
        if (R.nx <= 0 || R.ny <= 0 || R.nz <= 0) { *err = "grid sizes must be positive"; return PIC_EINVAL; }
        if (R.nx % g->tx || R.ny % g->ty || R.nz % g->tz) { *err = "grid sizes must be multiples of the tile"; return PIC_EINVAL; }
        R.ntx = R.nx / g->tx; R.nty = R.ny / g->ty; R.ntz = R.nz / g->tz;
        R.ncell = (long long)R.nx * R.ny * R.nz;
        R.ntiles = (long long)R.ntx * R.nty * R.ntz;
        R.cell_off = g->ncell;
        R.work_off = g->nwork;
        g->ncell += R.ncell;
        g->nwork += R.ntiles;
        for (int s = 0; s < PIC_NS; ++s) {
            R.capacity[s] = s < c->nspecies ? caps[PIC_NS * r + s] : 0;
            if (R.capacity[s] < 0) { *err = "capacity must be >= 0"; return PIC_EINVAL; }
            g->capacity[s] += R.capacity[s];
        }
    }
    if (g->ncell >= (1ll << 31) - 1) { *err = "too many cells for int32 cell indices"; return PIC_EINVAL; }
    g->nunit = c->ndim == 3 ? g->nwork : g->ncell;
    const long long ucells = c->ndim == 3 ? (long long)g->tx * g->ty * g->tz : 1;   // cells per unit
    for (int s = 0; s < PIC_NS; ++s) {
        g->cap[s] = 0;
        g->cap_stay[s] = 0;
        g->spill_cap[s] = 0;
        if (s >= c->nspecies) continue;
        if (g->capacity[s] >= (1ll << 31)) { *err = "capacity must be < 2^31 per species"; return PIC_EINVAL; }
        const long long mean = (g->capacity[s] + g->ncell - 1) / g->ncell;
        // default slots per cell: 2D 8x the mean in warp multiples (a warp owns a cell; the
        // beam pinches to ~9x its mean density in the nonlinear filamentation stage), 3D 3x the
        // mean in multiples of 8 (a tile holds its cells' slots together, so a filament that
        // compresses particles inside a tile does not spill; the spill list takes the rest)
        long long cap = c->cell_capacity[s];
        if (cap <= 0) {
            cap = c->ndim == 2 ? ((8 * mean + 31) / 32) * 32 : ((3 * mean + 7) / 8) * 8;
            cap = std::max(cap, c->ndim == 2 ? 32ll : 16ll);
        }
        if (cap < 2 || cap > 65535) { *err = "cell_capacity must be in [2, 65535]"; return PIC_EINVAL; }
        if (cap * g->ncell < 2 * g->capacity[s]) { *err = "cell_capacity must be >= 2 x capacity / cells"; return PIC_EINVAL; }
        if (cap * g->ncell >= (1ll << 31)) { *err = "cells x cell_capacity must be < 2^31"; return PIC_EINVAL; }
        // 3D: one slot range per tile, the tile's cells' capacities together, in blocks of 32
        const long long ucap = c->ndim == 3 ? ((cap * ucells + PIC_BLK - 1) / PIC_BLK) * PIC_BLK : cap;
        if (ucap * g->nunit >= (1ll << 31)) { *err = "cells x cell_capacity must be < 2^31"; return PIC_EINVAL; }
        g->cap[s] = (int)ucap;
        // immigrant area (>= 1 slot): 2D a quarter of the slots (only particles crossing a tile
        // edge arrive there); 3D a quarter of the tile's slots in whole blocks (particles
        // leaving a tile are ~7% of them per step in the hot beam: the beam's z flux through a
        // 4-cell-deep tile's bottom layer), so that both areas start on a block.  The rest keeps
        // the unit's stayers (in 2D also the particles arriving from the same tile).
        long long ci = c->ndim == 2 ? (ucap + 3) / 4 : ((ucap / 4 + PIC_BLK - 1) / PIC_BLK) * PIC_BLK;
        cap = ucap;
        if (ci < 1) ci = 1;
        if (ci >= cap) ci = cap > 1 ? cap - 1 : 0;
        g->cap_stay[s] = (int)(cap - ci);
        long long sc = g->capacity[s] / 4;   // room for the excess of dense filaments
        if (sc < 65536) sc = 65536;
        if (sc > g->capacity[s] + 1) sc = g->capacity[s] + 1;
        g->spill_cap[s] = (int)sc;
    }
    return PIC_OK;
}

// Arrays per particle slot: offsets, momenta, the optional id and, in 3D, the cell within the tile.
int slot_arrays(const pic_config* c) { return c->ndim + 3 + (c->track_ids ? 1 : 0) + (c->ndim == 3 ? 1 : 0); }

Layout make_layout(const pic_config* c, const Geometry& g) {
    Layout L{};
    size_t off = 0;
    const int nruns = (int)g.runs.size();
    const long long nc = g.ncell;
    const long long nu = g.nunit;
    L.ctl = take(off, sizeof(Ctl));
    L.runs = take(off, sizeof(RunDev) * nruns);
    L.work = take(off, sizeof(int2) * g.nwork);
    L.work_off = take(off, sizeof(int) * (nruns + 1));
    L.kin = take(off, sizeof(long long) * nruns * PIC_NS * 4);
    for (int s = 0; s < c->nspecies; ++s)
        for (int b = 0; b < 2; ++b) {
            // slot arrays in blocks of PIC_BLK slots (see Slots): array d of block k at
            // region + (k * na + d) * PIC_BLK floats
            const long long nblk = (nu * g.cap[s] + PIC_BLK - 1) / PIC_BLK;
            const int na = slot_arrays(c);
            const size_t r0 = take(off, (size_t)4 * nblk * na * PIC_BLK);
            L.slot_region[s][b] = r0;
            for (int d = 0; d < 3; ++d) L.so[s][b][d] = d < c->ndim ? r0 + (size_t)4 * PIC_BLK * d : 0;
            for (int d = 0; d < 3; ++d) L.su[s][b][d] = r0 + (size_t)4 * PIC_BLK * (c->ndim + d);
            L.sid[s][b] = c->track_ids ? r0 + (size_t)4 * PIC_BLK * (c->ndim + 3) : 0;
            L.slc[s][b] = c->ndim == 3 ? r0 + (size_t)4 * PIC_BLK * (c->ndim + 3 + (c->track_ids ? 1 : 0)) : 0;
            L.scount[s][b] = take(off, 4 * nu);
            L.sicount[s][b] = take(off, 4 * nu);
            const long long sp = g.spill_cap[s];
            L.sp_cell[s][b] = take(off, 4 * sp);
            for (int d = 0; d < 3; ++d) L.sp_o[s][b][d] = d < c->ndim ? take(off, 4 * sp) : 0;
            for (int d = 0; d < 3; ++d) L.sp_u[s][b][d] = take(off, 4 * sp);
            L.sp_id[s][b] = c->track_ids ? take(off, 4 * sp) : 0;
            L.sp_n[s][b] = take(off, 4);
        }
    for (int d = 0; d < 3; ++d) {
        L.E[d].resize(nruns); L.B[d].resize(nruns); L.J[d].resize(nruns); L.Jlast[d].resize(nruns);
        L.Jf[d].resize(nruns);
        L.msum[d].resize(nruns); L.ubar[d].resize(nruns);
    }
    L.mcnt.resize(nruns);
    for (int sp = 0; sp < PIC_NS; ++sp) L.dragmap[sp].assign(nruns, 0);
    for (int r = 0; r < nruns; ++r) {
        const long long n = g.runs[r].ncell;
        for (int d = 0; d < 3; ++d) L.E[d][r] = take(off, 4 * n);
        for (int d = 0; d < 3; ++d) L.B[d][r] = take(off, 4 * n);
        for (int d = 0; d < 3; ++d) L.J[d][r] = take(off, 8 * n);
        for (int d = 0; d < 3; ++d) L.Jlast[d][r] = (c->flags & PIC_FLAG_KEEP_J) ? take(off, 8 * n) : 0;
        for (int d = 0; d < 3; ++d) L.Jf[d][r] = c->j_filter ? take(off, 8 * n) : 0;
        for (int d = 0; d < 3; ++d) L.msum[d][r] = take(off, 8 * n);
        L.mcnt[r] = take(off, 4 * n);
        for (int d = 0; d < 3; ++d) L.ubar[d][r] = take(off, 4 * n);
        for (int sp = 0; sp < c->nspecies; ++sp) L.dragmap[sp][r] = take(off, 4 * n);
    }
    L.start = take(off, 4 * (nc + 1));
    L.scan_tmp = take(off, 4 * (nc / 2048 + 2));
    L.gate = take(off, 4);
    if (c->ndim == 2) {
        // crosser queue per tile: an eighth of the densest run's mean particles per tile (a step
        // moves at most half a cell, so only a fraction of a tile's particles cross an edge);
        // the excess of denser tiles goes to the overflow list
        long long per_tile = 0;
        for (const RunGeo& R : g.runs) {
            long long np = 0;
            for (int s = 0; s < PIC_NS; ++s) np += R.capacity[s];
            if (R.ntiles > 0) per_tile = std::max(per_tile, (np + R.ntiles - 1) / R.ntiles);
        }
        L.xq_cap = (int)std::max(256ll, ((per_tile / 8 + 31) / 32) * 32);
        L.xq = take(off, sizeof(Crosser) * (size_t)L.xq_cap * (size_t)g.nwork);
        long long tot = 0;
        for (int s = 0; s < PIC_NS; ++s) tot += g.capacity[s];
        L.xo_cap = (int)std::min<long long>(std::max(65536ll, tot / 16), (1ll << 31) - 1);
        L.xo = take(off, sizeof(CrosserX) * (size_t)L.xo_cap);
        L.xo_n = take(off, 4);
    }
    L.partials = take(off, sizeof(double) * 8 * g.nwork);
    L.hist = take(off, sizeof(DiagRec) * nruns * (c->diag_interval > 0 ? c->diag_capacity : 1));
    L.fit = take(off, sizeof(double) * 4);
    L.total = (off + 255) & ~size_t(255);
    return L;
}

}  // namespace

struct pic_ctx {
    pic_config cfg{};
    Geometry geo{};
    Layout lay{};
    cudaStream_t stream = nullptr;
    char* arena = nullptr;
    int nruns = 1;
    int sort_interval = 8;
    std::vector<RunDev> runs;
    Args args{};
    std::vector<long long> loaded;      // [nruns][PIC_NS]
    std::vector<double> nu;             // [nruns][PIC_NS] Krook rates as loaded
    double q[PIC_NS] = {0, 0};
    bool q_set[PIC_NS] = {false, false};
    long long host_step = 0;
    long long launches = 0;
    std::string err;
    // graph of one sort period
    cudaGraphExec_t graph = nullptr;
    long long graph_launches = 0;
    bool graph_dirty = true;
    // profiling
    struct Ev { int phase; cudaEvent_t a, b; };
    std::vector<Ev> pending;
    std::vector<cudaEvent_t> pool;
    double phase_ms[PH_N] = {0, 0, 0, 0};
    long long phase_n[PH_N] = {0, 0, 0, 0};
    std::string tune_key;               // workload and GPU key of the tuning cache
};

namespace {
std::string tune_key(const pic_config& c, int nruns, const int32_t* dims, const int64_t* caps);
}
int switch_variant(pic_ctx* ctx, int v);
void apply_cached_variant(pic_ctx* ctx);

namespace {

int fail(pic_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf; else g_init_error = buf;
    return code;
}

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(ctx, PIC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));        \
    } while (0)

template <class T> T* at(pic_ctx* c, size_t off) { return reinterpret_cast<T*>(c->arena + off); }

int upload_runs(pic_ctx* ctx) {
    ctx->args.anydrag = 0;
    for (int r = 0; r < ctx->nruns; ++r) ctx->args.anydrag |= ctx->runs[r].msum[0] != nullptr;
    CK(cudaMemcpyAsync(at<RunDev>(ctx, ctx->lay.runs), ctx->runs.data(), sizeof(RunDev) * ctx->nruns,
                       cudaMemcpyHostToDevice, ctx->stream));
    ctx->graph_dirty = true;
    return PIC_OK;
}

cudaEvent_t get_event(pic_ctx* c) {
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// One phase of a step: CUDA events around it (PIC_FLAG_PROFILE) and an NVTX range (PIC_FLAG_NVTX).
struct PhaseScope {
    pic_ctx* c;
    pic_ctx::Ev ev{};
    bool on, nvtx;
    PhaseScope(pic_ctx* c_, int ph)
        : c(c_), on((c_->cfg.flags & PIC_FLAG_PROFILE) != 0), nvtx((c_->cfg.flags & PIC_FLAG_NVTX) != 0) {
        if (nvtx) nvtxRangePushA(kPhaseName[ph]);
        if (!on) return;
        ev.phase = ph;
        ev.a = get_event(c);
        ev.b = get_event(c);
        cudaEventRecord(ev.a, c->stream);
    }
    ~PhaseScope() {
        if (on) {
            cudaEventRecord(ev.b, c->stream);
            c->pending.push_back(ev);
        }
        if (nvtx) nvtxRangePop();
    }
};

// An NVTX range around a C-ABI call (PIC_FLAG_NVTX).
struct NvtxCall {
    bool on;
    NvtxCall(const pic_ctx* c, const char* name) : on(c && (c->cfg.flags & PIC_FLAG_NVTX) != 0) {
        if (on) nvtxRangePushA(name);
    }
    ~NvtxCall() {
        if (on) nvtxRangePop();
    }
};

int launch_one_step(pic_ctx* ctx, long long step_index) {
    const Args& a = ctx->args;
    {
        PhaseScope ps(ctx, PH_PUSH);
        CK(launch_clear_next(a, ctx->stream));
        CK(ctx->cfg.ndim == 2 ? launch_push2d(a, ctx->stream) : launch_push3d(a, ctx->stream));
        CK(ctx->cfg.ndim == 2 ? launch_spill2d(a, ctx->stream) : launch_spill3d(a, ctx->stream));
        ctx->launches += 3;
    }
    {
        PhaseScope ps(ctx, PH_YEE);
        CK(ctx->cfg.ndim == 2 ? launch_yee2d(a, ctx->runs.data(), ctx->nruns, ctx->stream)
                              : launch_yee3d(a, ctx->runs.data(), ctx->nruns, ctx->stream));
        ctx->launches += (ctx->cfg.ndim == 2 ? 1 : ctx->nruns) * (ctx->cfg.j_filter ? 4 : 3);
    }
    {
        PhaseScope ps(ctx, PH_FINAL);
        CK(launch_finalize(a, ctx->stream));
        ctx->launches += 2;
    }
    if ((step_index + 1) % ctx->sort_interval == 0) {
        PhaseScope ps(ctx, PH_SORT);
        int l = 0;
        CK(launch_resort(a, ctx->stream, &l));
        ctx->launches += l;
    }
    return PIC_OK;
}

int build_graph(pic_ctx* ctx) {
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    const long long l0 = ctx->launches;
    int rc = PIC_OK;
    for (int i = 0; i < ctx->sort_interval && rc == PIC_OK; ++i) rc = launch_one_step(ctx, i);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    ctx->graph_launches = ctx->launches - l0;
    ctx->launches = l0;
    if (rc != PIC_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return fail(ctx, PIC_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ctx->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(ctx, PIC_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    ctx->graph_dirty = false;
    return PIC_OK;
}

int read_ctl(pic_ctx* ctx, Ctl* h) {
    CK(cudaMemcpyAsync(h, at<Ctl>(ctx, ctx->lay.ctl), sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PIC_OK;
}

int device_flags(pic_ctx* ctx) {
    Ctl h;
    int rc = read_ctl(ctx, &h);
    if (rc) return rc;
    if (h.err & ERR_BADPART) return fail(ctx, PIC_EBADPART, "device: non-finite or out-of-range particle");
    if (h.err & ERR_OVERFLOW) return fail(ctx, PIC_EOVERFLOW, "device: fixed-point headroom exceeded");
    if (h.err & ERR_TIMEOUT) return fail(ctx, PIC_ETIMEOUT, "device: bounded wait gave up");
    if (h.err & ERR_SPILL_FULL) return fail(ctx, PIC_ENOMEM, "device: spill list full (raise cell_capacity)");
    if (h.err & ERR_BOUNDS) return fail(ctx, PIC_EBOUNDS, "device: shared-tile or halo index out of range (debug build)");
    return PIC_OK;
}

// Fixed-point shift S of a run: every per-particle current term satisfies |term| * 2^S <= 2^21,
// so 32 warp lanes sum without int32 overflow and one FFMA rounds it exactly.  A term is bounded
// by |q| w max(dx/dt, dy/dt, dz/dt, 1) (|v| < c, CIC weights in [0, 1]).
int choose_shift(const pic_ctx* ctx, const RunDev& R) {
    const pic_config& c = ctx->cfg;
    double vmax = std::fmax(c.dx / c.dt, c.dy / c.dt);
    if (c.ndim == 3) vmax = std::fmax(vmax, c.dz / c.dt);
    vmax = std::fmax(vmax, 1.0);
    double bound = 0.0;
    for (int s = 0; s < c.nspecies; ++s)
        if (R.sp[s].active) bound = std::fmax(bound, std::fabs(ctx->q[s]) * R.sp[s].w * vmax);
    if (bound <= 0) return 30;
    int S = (int)std::floor(std::log2(2097152.0 / bound));
    if (S > 40) S = 40;
    if (S < 0) S = 0;
    return S;
}

void set_species_scales(pic_ctx* ctx, RunDev& R) {
    const pic_config& c = ctx->cfg;
    R.shift = choose_shift(ctx, R);
    const double two = std::ldexp(1.0, R.shift);
    for (int s = 0; s < c.nspecies; ++s) {
        SpeciesParams& P = R.sp[s];
        if (!P.active) continue;
        const double qw = ctx->q[s] * (double)P.w;
        P.jx = (float)(-qw * (c.dx / c.dt) * two);
        P.jy = (float)(-qw * (c.dy / c.dt) * two);
        P.jz = c.ndim == 2 ? (float)(qw * two) : (float)(-qw * (c.dz / c.dt) * two);
    }
    R.jscale = (float)std::ldexp(1.0, -R.shift);
    R.jfscale = (float)std::ldexp(1.0, -R.shift - 2 * c.ndim);
}

int check_run(pic_ctx* ctx, int run) {
    if (run < 0 || run >= ctx->nruns) return fail(ctx, PIC_EINVAL, "run %d out of range [0, %d)", run, ctx->nruns);
    return PIC_OK;
}

int init_common(const pic_config* cfg, int nruns, const int32_t* dims, const int64_t* caps,
                void* device_arena, size_t arena_bytes, void* cuda_stream, pic_ctx** out) {
    if (!cfg || !out || !dims || !caps) return fail(nullptr, PIC_EINVAL, "null argument");
    *out = nullptr;
    Geometry g;
    std::string err;
    int rc = geometry(cfg, nruns, dims, caps, &g, &err);
    if (rc != PIC_OK) return fail(nullptr, rc, "%s", err.c_str());
    Layout L = make_layout(cfg, g);
    if (!device_arena) return fail(nullptr, PIC_EINVAL, "null arena");
    if (arena_bytes < L.total) return fail(nullptr, PIC_ENOMEM, "arena has %zu bytes, needs %zu", arena_bytes, L.total);
    if (reinterpret_cast<uintptr_t>(device_arena) & 255) return fail(nullptr, PIC_EINVAL, "arena must be 256-byte aligned");
    pic_ctx* ctx = new (std::nothrow) pic_ctx;
    if (!ctx) return fail(nullptr, PIC_ENOMEM, "host allocation failed");
    ctx->cfg = *cfg;
    if (ctx->cfg.ndim == 2) ctx->cfg.dz = ctx->cfg.dx;
    ctx->geo = g;
    ctx->lay = L;
    ctx->nruns = nruns;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->arena = (char*)device_arena;
    ctx->sort_interval = cfg->sort_interval > 0 ? cfg->sort_interval : 8;
    ctx->loaded.assign((size_t)nruns * PIC_NS, 0);
    ctx->nu.assign((size_t)nruns * PIC_NS, 0.0);

    auto bail = [&](int code) { g_init_error = ctx->err; delete ctx; return code; };
#define CKI(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { fail(ctx, PIC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); return bail(PIC_ECUDA); } } while (0)
    CKI(preload_push2d());
    CKI(preload_push3d());
    CKI(preload_moments());
    CKI(preload_mlp());
    CKI(preload_bins());
    CKI(preload_fields());
    CKI(cudaMemsetAsync(ctx->arena, 0, L.total, ctx->stream));

    const pic_config& c = ctx->cfg;
    ctx->runs.assign(nruns, RunDev{});
    std::vector<int2> work(g.nwork);
    std::vector<int> work_off(nruns + 1);
    for (int r = 0; r < nruns; ++r) {
        const RunGeo& G = g.runs[r];
        RunDev& R = ctx->runs[r];
        R.nx = G.nx; R.ny = G.ny; R.nz = G.nz;
        R.ntx = G.ntx; R.nty = G.nty; R.ntz = G.ntz;
        R.work_off = (int)G.work_off;
        R.cell_off = (int)G.cell_off;
        R.dtdx = (float)(c.dt / c.dx); R.dtdy = (float)(c.dt / c.dy); R.dtdz = (float)(c.dt / c.dz);
        R.cx = R.dtdx; R.cy = R.dtdy; R.cz = R.dtdz;
        for (int d = 0; d < 3; ++d) {
            R.E[d] = at<float>(ctx, L.E[d][r]);
            R.B[d] = at<float>(ctx, L.B[d][r]);
            R.J[d] = at<long long>(ctx, L.J[d][r]);
            R.Jlast[d] = L.Jlast[d][r] ? at<long long>(ctx, L.Jlast[d][r]) : nullptr;
            R.Jf[d] = L.Jf[d][r] ? at<long long>(ctx, L.Jf[d][r]) : nullptr;
            R.msum[d] = nullptr;   // published when a drag species is loaded
            R.ubar[d] = nullptr;
        }
        R.mcnt = nullptr;
        for (int sp = 0; sp < PIC_NS; ++sp) R.dragmap[sp] = nullptr;
        R.shift = 30;
        R.jscale = (float)std::ldexp(1.0, -30);
        R.jfscale = (float)std::ldexp(1.0, -30 - 2 * c.ndim);
        for (long long t = 0; t < G.ntiles; ++t) work[G.work_off + t] = make_int2(r, (int)t);
        work_off[r] = (int)G.work_off;
    }
    work_off[nruns] = (int)g.nwork;
    CKI(cudaMemcpyAsync(at<int2>(ctx, L.work), work.data(), sizeof(int2) * g.nwork, cudaMemcpyHostToDevice, ctx->stream));
    CKI(cudaMemcpyAsync(at<int>(ctx, L.work_off), work_off.data(), sizeof(int) * (nruns + 1), cudaMemcpyHostToDevice, ctx->stream));

    Args& a = ctx->args;
    a.ctl = at<Ctl>(ctx, L.ctl);
    a.runs = at<RunDev>(ctx, L.runs);
    a.work = at<int2>(ctx, L.work);
    a.work_off = at<int>(ctx, L.work_off);
    a.kin = at<long long>(ctx, L.kin);
    a.nwork = (int)g.nwork;
    a.tx = g.tx; a.ty = g.ty; a.tz = g.tz;
    a.push_variant = g.push_variant;
    a.nspecies = c.nspecies;
    a.nruns = nruns;
    a.ndim = c.ndim;
    for (int s = 0; s < c.nspecies; ++s) {
        a.cap[s] = g.cap[s];
        a.cap_stay[s] = g.cap_stay[s];
        a.spill_cap[s] = g.spill_cap[s];
        a.stage_n[s] = g.capacity[s];
        for (int b = 0; b < 2; ++b) {
            Slots& S = a.slot[s][b];
            for (int d = 0; d < 3; ++d) {
                S.o[d] = L.so[s][b][d] ? at<float>(ctx, L.so[s][b][d]) : nullptr;
                S.u[d] = at<float>(ctx, L.su[s][b][d]);
                S.so[d] = L.sp_o[s][b][d] ? at<float>(ctx, L.sp_o[s][b][d]) : nullptr;
                S.su[d] = at<float>(ctx, L.sp_u[s][b][d]);
            }
            S.id = L.sid[s][b] ? at<int>(ctx, L.sid[s][b]) : nullptr;
            S.lc = L.slc[s][b] ? at<int>(ctx, L.slc[s][b]) : nullptr;
            S.bstride = (long long)slot_arrays(&c) * PIC_BLK;
            S.count = at<int>(ctx, L.scount[s][b]);
            S.icount = at<int>(ctx, L.sicount[s][b]);
            S.scell = at<int>(ctx, L.sp_cell[s][b]);
            S.sid = L.sp_id[s][b] ? at<int>(ctx, L.sp_id[s][b]) : nullptr;
            S.sn = at<int>(ctx, L.sp_n[s][b]);
            // staging when b is current = the slot memory of the other buffer
            a.stage[s][b ^ 1] = ctx->arena + L.slot_region[s][b];
        }
    }
    a.ncell = g.ncell;
    a.nunit = g.nunit;
    a.partials = at<double>(ctx, L.partials);
    a.hist = at<DiagRec>(ctx, L.hist);
    a.hist_cap = c.diag_interval > 0 ? c.diag_capacity : 1;
    a.diag_interval = c.diag_interval;
    a.dt = c.dt;
    a.dV = c.dx * c.dy * (c.ndim == 3 ? c.dz : 1.0);
    a.scan_tmp = at<int>(ctx, L.scan_tmp);
    a.start = at<int>(ctx, L.start);
    a.gate = at<int>(ctx, L.gate);
    a.xq = L.xq_cap ? at<Crosser>(ctx, L.xq) : nullptr;
    a.xq_cap = L.xq_cap;
    a.xo = L.xo_cap ? at<CrosserX>(ctx, L.xo) : nullptr;
    a.xo_n = L.xo_cap ? at<int>(ctx, L.xo_n) : nullptr;
    a.xo_cap = L.xo_cap;

    if (upload_runs(ctx) != PIC_OK) return bail(PIC_ECUDA);
    ctx->tune_key = tune_key(c, nruns, dims, caps);
    apply_cached_variant(ctx);
    CKI(cudaStreamSynchronize(ctx->stream));
#undef CKI
    *out = ctx;
    return PIC_OK;
}

// A run's particle units: its cells (2D) or its tiles (3D).
long long unit_off(const pic_ctx* ctx, const RunGeo& G) { return ctx->cfg.ndim == 3 ? G.work_off : G.cell_off; }
long long unit_n(const pic_ctx* ctx, const RunGeo& G) { return ctx->cfg.ndim == 3 ? G.ntiles : G.ncell; }

// Publish the drag moment arrays of run `run` and set the cell means <u> of species s from its
// loaded particles (the drag of the first step uses them).
int start_drag(pic_ctx* ctx, int run, int s) {
    RunDev& R = ctx->runs[run];
    const RunGeo& G = ctx->geo.runs[run];
    if (!R.msum[0]) {
        for (int d = 0; d < 3; ++d) {
            R.msum[d] = at<long long>(ctx, ctx->lay.msum[d][run]);
            R.ubar[d] = at<float>(ctx, ctx->lay.ubar[d][run]);
        }
        R.mcnt = at<int>(ctx, ctx->lay.mcnt[run]);
    }
    int rc = upload_runs(ctx);
    if (rc) return rc;
    CK(launch_moments_init(ctx->args, s, run, unit_off(ctx, G), unit_n(ctx, G), ctx->stream));
    CK(launch_moments_finalize(ctx->args, run, G.ncell, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return device_flags(ctx);
}

// Device address of host or device pointer p when the device can read it directly (device
// memory, or pinned / registered host memory mapped into the device's address space).
bool device_view(const void* p, void** dev) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if ((at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) &&
        at.devicePointer) {
        *dev = at.devicePointer;
        return true;
    }
    return false;
}

int load_run(pic_ctx* ctx, int run, int s, const pic_species* sp, int64_t n, const int32_t* cell,
             const float* offset, const float* u) {
    if (!ctx) return fail(nullptr, PIC_EINVAL, "null context");
    int rc = check_run(ctx, run);
    if (rc) return rc;
    const RunGeo& G = ctx->geo.runs[run];
    if (!sp || s < 0 || s >= ctx->cfg.nspecies) return fail(ctx, PIC_EINVAL, "bad species index");
    if (n < 0 || n > G.capacity[s]) return fail(ctx, PIC_ENOMEM, "n = %lld exceeds the run's capacity", (long long)n);
    if (n > 0 && (!cell || !offset || !u)) return fail(ctx, PIC_EINVAL, "null particle array");
    if (ctx->host_step != 0) return fail(ctx, PIC_ESTATE, "species are loaded before the first step");
    RunDev& R = ctx->runs[run];
    if (R.sp[s].active) return fail(ctx, PIC_ESTATE, "species %d of run %d is already loaded", s, run);
    if (!(std::isfinite(sp->q) && std::isfinite(sp->m) && sp->m > 0 && std::isfinite(sp->w) && sp->w >= 0 &&
          std::isfinite(sp->nu) && sp->nu >= 0 && std::fabs(sp->q) <= 1.0))
        return fail(ctx, PIC_EINVAL, "bad species parameters (|q| <= 1, m > 0, w >= 0, nu >= 0)");
    if (ctx->q_set[s] && ctx->q[s] != sp->q) return fail(ctx, PIC_EINVAL, "species %d has one charge in every run", s);
    if (sp->nu > 0)
        for (int o = 0; o < PIC_NS; ++o)
            if (o != s && R.sp[o].drag)
                return fail(ctx, PIC_EINVAL, "run %d: the Krook drag acts on one species per run", run);
    const pic_config& c = ctx->cfg;
    Ctl h;
    rc = read_ctl(ctx, &h);
    if (rc) return rc;
    // Arrays the device can address (pinned or registered host memory, device memory) are read
    // by the binning kernel directly; others go host -> staging (the other buffer's slot memory)
    // first.  Then a counting sort into the slots.
    Stage direct{};
    const bool zero_copy = n > 0 && device_view(cell, (void**)&direct.cell) && device_view(offset, (void**)&direct.o[0]) &&
                           device_view(u, (void**)&direct.u[0]);
    if (zero_copy) {
        for (int d = 1; d < 3; ++d) direct.o[d] = d < c.ndim ? direct.o[0] + (size_t)d * n : nullptr;
        for (int d = 1; d < 3; ++d) direct.u[d] = direct.u[0] + (size_t)d * n;
    } else if (n > 0) {
        const Stage T = stage_of(ctx->args, s, h.parity);
        CK(cudaMemcpyAsync(T.cell, cell, 4 * n, cudaMemcpyHostToDevice, ctx->stream));
        for (int d = 0; d < c.ndim; ++d)
            CK(cudaMemcpyAsync(T.o[d], offset + (size_t)d * n, 4 * n, cudaMemcpyHostToDevice, ctx->stream));
        for (int d = 0; d < 3; ++d)
            CK(cudaMemcpyAsync(T.u[d], u + (size_t)d * n, 4 * n, cudaMemcpyHostToDevice, ctx->stream));
    }
    CK(launch_bin(ctx->args, s, n, false, G.cell_off, G.ncell, nullptr, ctx->stream, zero_copy ? &direct : nullptr));
    rc = device_flags(ctx);
    if (rc) {
        // undo: empty the run's cells of this species and clear the flag
        const Slots& S = ctx->args.slot[s][h.parity];
        CK(cudaMemsetAsync(S.count + unit_off(ctx, G), 0, 4 * unit_n(ctx, G), ctx->stream));
        CK(cudaMemsetAsync(S.icount + unit_off(ctx, G), 0, 4 * unit_n(ctx, G), ctx->stream));
        Ctl z;
        int rc2 = read_ctl(ctx, &z);
        if (rc2) return rc2;
        z.err = 0;
        CK(cudaMemcpyAsync(at<Ctl>(ctx, ctx->lay.ctl), &z, sizeof(Ctl), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return rc;
    }
    ctx->loaded[(size_t)run * PIC_NS + s] = n;
    ctx->nu[(size_t)run * PIC_NS + s] = sp->nu;
    ctx->q[s] = sp->q;
    ctx->q_set[s] = true;

    SpeciesParams& P = R.sp[s];
    P.active = 1;
    P.qmdt2 = (float)(sp->q * c.dt / (2.0 * sp->m));
    P.w = (float)sp->w;
    P.dragf = (float)(-std::expm1(-sp->nu * c.dt));
    P.drag = sp->nu > 0 ? 1 : 0;
    set_species_scales(ctx, R);
    if (P.drag) return start_drag(ctx, run, s);
    rc = upload_runs(ctx);
    if (rc) return rc;
    CK(cudaStreamSynchronize(ctx->stream));
    return device_flags(ctx);
}

long long records_written(const pic_ctx* ctx) {
    const int M = ctx->cfg.diag_interval;
    if (M <= 0 || ctx->host_step <= 0) return 0;
    return (ctx->host_step - 1) / M + 1;
}

}  // namespace

// =============================================================================== C ABI

extern "C" int pic_required_bytes_batch(const pic_config* cfg, int nruns, const int32_t* run_dims,
                                        const int64_t* run_capacity, size_t* bytes_out) {
    if (!cfg || !bytes_out || !run_dims || !run_capacity) return fail(nullptr, PIC_EINVAL, "null argument");
    Geometry g;
    std::string err;
    int rc = geometry(cfg, nruns, run_dims, run_capacity, &g, &err);
    if (rc != PIC_OK) return fail(nullptr, rc, "%s", err.c_str());
    *bytes_out = make_layout(cfg, g).total;
    return PIC_OK;
}

extern "C" int pic_required_bytes(const pic_config* cfg, size_t* bytes_out) {
    if (!cfg || !bytes_out) return fail(nullptr, PIC_EINVAL, "null argument");
    const int32_t dims[3] = {cfg->nx, cfg->ny, cfg->nz};
    const int64_t caps[PIC_NS] = {cfg->capacity[0], cfg->capacity[1]};
    return pic_required_bytes_batch(cfg, 1, dims, caps, bytes_out);
}

extern "C" int pic_init(const pic_config* cfg, void* device_arena, size_t arena_bytes,
                        void* cuda_stream, pic_ctx** out) {
    if (!cfg) return fail(nullptr, PIC_EINVAL, "null argument");
    const int32_t dims[3] = {cfg->nx, cfg->ny, cfg->nz};
    const int64_t caps[PIC_NS] = {cfg->capacity[0], cfg->capacity[1]};
    return init_common(cfg, 1, dims, caps, device_arena, arena_bytes, cuda_stream, out);
}

extern "C" int pic_init_batch(const pic_config* cfg, int nruns, const int32_t* run_dims,
                              const int64_t* run_capacity, void* device_arena, size_t arena_bytes,
                              void* cuda_stream, pic_ctx** out) {
    return init_common(cfg, nruns, run_dims, run_capacity, device_arena, arena_bytes, cuda_stream, out);
}

extern "C" int pic_load_species(pic_ctx* ctx, int s, const pic_species* sp, int64_t n,
                                const int32_t* cell, const float* offset, const float* u) {
    return load_run(ctx, 0, s, sp, n, cell, offset, u);
}

extern "C" int pic_load_species_run(pic_ctx* ctx, int run, int s, const pic_species* sp, int64_t n,
                                    const int32_t* cell, const float* offset, const float* u) {
    return load_run(ctx, run, s, sp, n, cell, offset, u);
}

extern "C" int pic_step(pic_ctx* ctx, int nsteps) {
    if (!ctx) return fail(nullptr, PIC_EINVAL, "null context");
    if (nsteps < 0) return fail(ctx, PIC_EINVAL, "nsteps < 0");
    const NvtxCall range(ctx, "pic_step");
    const bool use_graph = !(ctx->cfg.flags & (PIC_FLAG_PROFILE | PIC_FLAG_NO_GRAPH | PIC_FLAG_NVTX));
    while (nsteps > 0) {
        const int K = ctx->sort_interval;
        if (use_graph && ctx->host_step % K == 0 && nsteps >= K) {
            if (ctx->graph_dirty || !ctx->graph) {
                int rc = build_graph(ctx);
                if (rc) return rc;
            }
            CK(cudaGraphLaunch(ctx->graph, ctx->stream));
            ctx->launches += ctx->graph_launches;
            ctx->host_step += K;
            nsteps -= K;
        } else {
            int rc = launch_one_step(ctx, ctx->host_step);
            if (rc) return rc;
            ctx->host_step += 1;
            nsteps -= 1;
        }
    }
    return PIC_OK;
}

extern "C" int pic_sync(pic_ctx* ctx) {
    if (!ctx) return fail(nullptr, PIC_EINVAL, "null context");
    CK(cudaStreamSynchronize(ctx->stream));
    return device_flags(ctx);
}

namespace pic {
// Kernels whose shared-memory limit is set, per device (the attribute is per device: a process
// that drives several GPUs sets it on each).
cudaError_t smem_attr_once(const void* fn, int bytes) {
    static std::mutex mu;
    static std::set<std::pair<int, const void*>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({dev, fn})) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.insert({dev, fn});
    return e;
}
}  // namespace pic

extern "C" int pic_clear_flags(pic_ctx* ctx, int32_t* flags_out) {
    if (!ctx) return fail(nullptr, PIC_EINVAL, "null context");
    CK(cudaStreamSynchronize(ctx->stream));
    Ctl h;
    int rc = read_ctl(ctx, &h);
    if (rc) return rc;
    if (flags_out) *flags_out = h.err;
    const int zero = 0;
    CK(cudaMemcpyAsync(reinterpret_cast<char*>(at<Ctl>(ctx, ctx->lay.ctl)) + offsetof(Ctl, err), &zero, sizeof zero,
                       cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return PIC_OK;
}

extern "C" int pic_diag_run(pic_ctx* ctx, int run, pic_diag_rec* out, int max_recs, int* n_out) {
    if (!ctx || !n_out || (max_recs > 0 && !out)) return fail(ctx, PIC_EINVAL, "null argument");
    int rc = check_run(ctx, run);
    if (rc) return rc;
    rc = pic_sync(ctx);
    if (rc) return rc;
    const long long nrec = records_written(ctx);
    const int cap = ctx->args.hist_cap;
    const long long first = nrec > cap ? nrec - cap : 0;
    long long n = nrec - first;
    if (n > max_recs) n = max_recs;
    const DiagRec* base = ctx->args.hist + (size_t)run * cap;
    for (long long r = 0; r < n; ++r) {
        const long long slot = (first + r) % cap;
        CK(cudaMemcpyAsync(out + r, base + slot, sizeof(DiagRec), cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    *n_out = (int)n;
    return PIC_OK;
}

extern "C" int pic_diag(pic_ctx* ctx, pic_diag_rec* out, int max_recs, int* n_out) {
    return pic_diag_run(ctx, 0, out, max_recs, n_out);
}

extern "C" int pic_get_particles_run(pic_ctx* ctx, int run, int s, int32_t* cell, float* offset,
                                     float* u, int32_t* id, int64_t n) {
    if (!ctx) return fail(nullptr, PIC_EINVAL, "null context");
    int rc = check_run(ctx, run);
    if (rc) return rc;
    if (s < 0 || s >= ctx->cfg.nspecies) return fail(ctx, PIC_EINVAL, "bad species index");
    const long long want = ctx->loaded[(size_t)run * PIC_NS + s];
    if (n != want) return fail(ctx, PIC_EINVAL, "n must equal the loaded count (%lld)", want);
    if (id && !ctx->cfg.track_ids) return fail(ctx, PIC_ESTATE, "ids need track_ids");
    rc = pic_sync(ctx);
    if (rc) return rc;
    const RunGeo& G = ctx->geo.runs[run];
    // compaction of the run's units into the staging area (unit order, then its spill entries)
    CK(launch_compact(ctx->args, s, unit_off(ctx, G), unit_n(ctx, G), G.cell_off, G.ncell, G.cell_off, nullptr,
                      ctx->stream));
    ctx->launches += 6;
    Ctl h;
    rc = read_ctl(ctx, &h);
    if (rc) return rc;
    if (h.staged[s] != n) return fail(ctx, PIC_ESTATE, "device holds %d particles of species %d in run %d, expected %lld",
                                      h.staged[s], s, run, (long long)n);
    const Stage T = stage_of(ctx->args, s, h.parity);
    if (n > 0) {
        if (cell) CK(cudaMemcpyAsync(cell, T.cell, 4 * n, cudaMemcpyDeviceToHost, ctx->stream));
        if (offset)
            for (int d = 0; d < ctx->cfg.ndim; ++d)
                CK(cudaMemcpyAsync(offset + (size_t)d * n, T.o[d], 4 * n, cudaMemcpyDeviceToHost, ctx->stream));
        if (u)
            for (int d = 0; d < 3; ++d)
                CK(cudaMemcpyAsync(u + (size_t)d * n, T.u[d], 4 * n, cudaMemcpyDeviceToHost, ctx->stream));
        if (id) CK(cudaMemcpyAsync(id, T.id, 4 * n, cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return PIC_OK;
}

extern "C" int pic_get_particles(pic_ctx* ctx, int s, int32_t* cell, float* offset, float* u,
                                 int32_t* id, int64_t n) {
    return pic_get_particles_run(ctx, 0, s, cell, offset, u, id, n);
}

extern "C" int pic_get_fields_run(pic_ctx* ctx, int run, float* E, float* B, int64_t* J) {
    if (!ctx) return fail(nullptr, PIC_EINVAL, "null context");
    int rc = check_run(ctx, run);
    if (rc) return rc;
    rc = pic_sync(ctx);
    if (rc) return rc;
    const RunDev& R = ctx->runs[run];
    const size_t nc = (size_t)ctx->geo.runs[run].ncell;
    for (int d = 0; d < 3; ++d) {
        if (E) CK(cudaMemcpyAsync(E + d * nc, R.E[d], 4 * nc, cudaMemcpyDeviceToHost, ctx->stream));
        if (B) CK(cudaMemcpyAsync(B + d * nc, R.B[d], 4 * nc, cudaMemcpyDeviceToHost, ctx->stream));
        if (J) {
            if (!R.Jlast[0]) return fail(ctx, PIC_ESTATE, "J needs PIC_FLAG_KEEP_J");
            CK(cudaMemcpyAsync(J + d * nc, R.Jlast[d], 8 * nc, cudaMemcpyDeviceToHost, ctx->stream));
        }
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return PIC_OK;
}

extern "C" int pic_get_fields(pic_ctx* ctx, float* E, float* B, int64_t* J) {
    return pic_get_fields_run(ctx, 0, E, B, J);
}

extern "C" int pic_set_fields(pic_ctx* ctx, const float* E, const float* B) {
    if (!ctx) return fail(nullptr, PIC_EINVAL, "null context");
    const RunDev& R = ctx->runs[0];
    const size_t nc = (size_t)ctx->geo.runs[0].ncell;
    for (int d = 0; d < 3; ++d) {
        if (E) CK(cudaMemcpyAsync(R.E[d], E + d * nc, 4 * nc, cudaMemcpyHostToDevice, ctx->stream));
        if (B) CK(cudaMemcpyAsync(R.B[d], B + d * nc, 4 * nc, cudaMemcpyHostToDevice, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return PIC_OK;
}

extern "C" int pic_fixed_point_shift(const pic_ctx* ctx, int* shift_out) {
    if (!ctx || !shift_out) return PIC_EINVAL;
    *shift_out = ctx->runs[0].shift;
    return PIC_OK;
}

extern "C" int pic_fit_growth_run(pic_ctx* ctx, int run, int width, double t_noise, double start_factor,
                                  double end_factor, double* gamma_out, double* t0_out, double* t1_out) {
    if (!ctx || !gamma_out) return fail(ctx, PIC_EINVAL, "null argument");
    int rc = check_run(ctx, run);
    if (rc) return rc;
    if (width < 2) return fail(ctx, PIC_EINVAL, "width must be >= 2");
    rc = pic_sync(ctx);
    if (rc) return rc;
    const long long nrec = records_written(ctx);
    const int cap = ctx->args.hist_cap;
    const long long first = nrec > cap ? nrec - cap : 0;
    const int n = (int)(nrec - first);
    double* d_out = at<double>(ctx, ctx->lay.fit);
    CK(launch_fit(ctx->args, run, first, n, width, t_noise, start_factor, end_factor, d_out, ctx->stream));
    ctx->launches += 1;
    double h[3];
    CK(cudaMemcpyAsync(h, d_out, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *gamma_out = h[0];
    if (t0_out) *t0_out = h[1];
    if (t1_out) *t1_out = h[2];
    return PIC_OK;
}

extern "C" int pic_fit_growth(pic_ctx* ctx, int width, double t_noise, double start_factor,
                              double end_factor, double* gamma_out, double* t0_out, double* t1_out) {
    return pic_fit_growth_run(ctx, 0, width, t_noise, start_factor, end_factor, gamma_out, t0_out, t1_out);
}

extern "C" int pic_kernel_times(pic_ctx* ctx, pic_kernel_time* out, int max, int* n_out) {
    if (!ctx || !n_out) return fail(ctx, PIC_EINVAL, "null argument");
    CK(cudaStreamSynchronize(ctx->stream));
    for (auto& ev : ctx->pending) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ev.a, ev.b));
        ctx->phase_ms[ev.phase] += ms;
        ctx->phase_n[ev.phase] += 1;
        ctx->pool.push_back(ev.a);
        ctx->pool.push_back(ev.b);
    }
    ctx->pending.clear();
    int n = 0;
    for (int p = 0; p < PH_N && n < max; ++p) {
        if (!out) break;
        std::snprintf(out[n].name, sizeof out[n].name, "%s", kPhaseName[p]);
        out[n].launches = ctx->phase_n[p];
        out[n].total_ms = ctx->phase_ms[p];
        ++n;
    }
    *n_out = n;
    return PIC_OK;
}

extern "C" int pic_get_stats(pic_ctx* ctx, pic_stats* out) {
    if (!ctx || !out) return fail(ctx, PIC_EINVAL, "null argument");
    CK(cudaStreamSynchronize(ctx->stream));
    Ctl h;
    int rc = read_ctl(ctx, &h);
    if (rc) return rc;
    std::memset(out, 0, sizeof(*out));
    std::vector<int> cnt((size_t)ctx->geo.nunit), icnt((size_t)ctx->geo.nunit);
    for (int s = 0; s < ctx->cfg.nspecies; ++s) {
        const Slots& S = ctx->args.slot[s][h.parity];
        CK(cudaMemcpyAsync(cnt.data(), S.count, 4 * cnt.size(), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(icnt.data(), S.icount, 4 * icnt.size(), cudaMemcpyDeviceToHost, ctx->stream));
        int sn = 0;
        CK(cudaMemcpyAsync(&sn, S.sn, 4, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        const int cs = ctx->geo.cap_stay[s], ci = ctx->geo.cap[s] - cs;
        long long tot = 0;
        int mx = 0;
        for (size_t c = 0; c < cnt.size(); ++c) {
            const int a = std::min(cnt[c], cs), b = std::min(icnt[c], ci);
            tot += a + b;
            mx = std::max(mx, cnt[c] + icnt[c]);
        }
        out->particles[s] = tot + std::min(sn, ctx->geo.spill_cap[s]);
        out->max_cell[s] = mx;
        out->spilled[s] = sn;
        out->cell_capacity[s] = ctx->geo.cap[s];
    }
    out->flags = h.err;
    return PIC_OK;
}

extern "C" int pic_bin_cells_scratch_bytes(int32_t ncell, size_t* bytes_out) {
    if (ncell <= 0 || !bytes_out) return fail(nullptr, PIC_EINVAL, "ncell must be > 0 and bytes_out non-null");
    *bytes_out = bin_cells_scratch_bytes(ncell);
    return PIC_OK;
}

extern "C" int pic_bin_cells(const int32_t* cell, int64_t n, int32_t ncell, int32_t* start, int32_t* order,
                             void* scratch, size_t scratch_bytes, void* stream) {
    if (n < 0 || n >= (1ll << 31) || ncell <= 0) return fail(nullptr, PIC_EINVAL, "bad n or ncell");
    if (!start || !scratch || (n > 0 && (!cell || !order))) return fail(nullptr, PIC_EINVAL, "null pointer");
    if (scratch_bytes < bin_cells_scratch_bytes(ncell)) return fail(nullptr, PIC_ENOMEM, "scratch too small");
    if (reinterpret_cast<uintptr_t>(scratch) & 255) return fail(nullptr, PIC_EINVAL, "scratch must be 256-byte aligned");
    const cudaError_t e = launch_bin_cells(cell, n, ncell, start, order, (int*)scratch, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(nullptr, PIC_ECUDA, "pic_bin_cells: %s", cudaGetErrorString(e));
    return PIC_OK;
}

extern "C" int pic_bin_cells_noalloc(const int32_t* cell, int64_t n, int32_t ncell, int32_t* start,
                                     int32_t* order, void* stream) {
    if (n < 0 || n >= (1ll << 31) || ncell <= 0) return fail(nullptr, PIC_EINVAL, "bad n or ncell");
    if (ncell > PIC_BIN_NOALLOC_MAX_CELLS)
        return fail(nullptr, PIC_EINVAL, "ncell = %d exceeds PIC_BIN_NOALLOC_MAX_CELLS = %d", (int)ncell,
                    (int)PIC_BIN_NOALLOC_MAX_CELLS);
    if (!start || (n > 0 && (!cell || !order))) return fail(nullptr, PIC_EINVAL, "null pointer");
    int* scratch = nullptr;
    cudaError_t e = noalloc_bin_scratch(&scratch);
    if (e != cudaSuccess) return fail(nullptr, PIC_ECUDA, "scratch lookup: %s", cudaGetErrorString(e));
    e = launch_bin_cells(cell, n, ncell, start, order, scratch, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(nullptr, PIC_ECUDA, "pic_bin_cells_noalloc: %s", cudaGetErrorString(e));
    return PIC_OK;
}

namespace {
int moment_geometry(pic_ctx* ctx, int run, int bx, int by, long long* nc, long long* ncol) {
    if (!ctx) return fail(nullptr, PIC_EINVAL, "null context");
    int rc = check_run(ctx, run);
    if (rc) return rc;
    const RunDev& R = ctx->runs[run];
    if (bx < 1 || by < 1 || R.nx % bx || R.ny % by)
        return fail(ctx, PIC_EINVAL, "coarse block %d x %d must divide the grid %d x %d", bx, by, R.nx, R.ny);
    *nc = (long long)(R.nx / bx) * (R.ny / by);
    *ncol = (long long)R.nx * R.ny;
    return PIC_OK;
}
}  // namespace

extern "C" int pic_record_moments_scratch_bytes(pic_ctx* ctx, int run, int bx, int by, size_t* bytes_out) {
    long long nc, ncol;
    int rc = moment_geometry(ctx, run, bx, by, &nc, &ncol);
    if (rc) return rc;
    if (!bytes_out) return fail(ctx, PIC_EINVAL, "null bytes_out");
    *bytes_out = moments_scratch_bytes(nc, ncol);
    return PIC_OK;
}

extern "C" int pic_record_moments(pic_ctx* ctx, int run, int bx, int by, float* out, int64_t out_cap,
                                  void* scratch, size_t scratch_bytes, int64_t* ncoarse_out) {
    long long nc, ncol;
    int rc = moment_geometry(ctx, run, bx, by, &nc, &ncol);
    if (rc) return rc;
    if (!out || !scratch) return fail(ctx, PIC_EINVAL, "null out or scratch");
    if (out_cap < (int64_t)PIC_MOM_ROWS * nc)
        return fail(ctx, PIC_EINVAL, "out holds %lld floats, needs %lld", (long long)out_cap, (long long)PIC_MOM_ROWS * nc);
    if (scratch_bytes < moments_scratch_bytes(nc, ncol))
        return fail(ctx, PIC_EINVAL, "scratch has %zu bytes, needs %zu", scratch_bytes, moments_scratch_bytes(nc, ncol));
    if (reinterpret_cast<uintptr_t>(scratch) & 7) return fail(ctx, PIC_EINVAL, "scratch must be 8-byte aligned");
    if (ctx->cfg.nspecies < 2) return fail(ctx, PIC_EINVAL, "the recorder needs beam and background species");
    const float q_bg = (float)ctx->q[1];
    const float nu_bg = (float)ctx->nu[(size_t)run * PIC_NS + 1];
    CK(launch_moments(ctx->args, ctx->runs[run], run, bx, by, q_bg, nu_bg, out, scratch, ctx->stream));
    if (ncoarse_out) *ncoarse_out = nc;
    return PIC_OK;
}

extern "C" int pic_set_drag_map(pic_ctx* ctx, int run, int s, const float* nu, int32_t bx, int32_t by) {
    if (!ctx) return fail(nullptr, PIC_EINVAL, "null context");
    int rc = check_run(ctx, run);
    if (rc) return rc;
    if (s < 0 || s >= ctx->cfg.nspecies) return fail(ctx, PIC_EINVAL, "species %d out of range", s);
    RunDev& R = ctx->runs[run];
    SpeciesParams& P = R.sp[s];
    if (!P.active) return fail(ctx, PIC_ESTATE, "species %d of run %d is not loaded", s, run);
    if (!nu) {
        R.dragmap[s] = nullptr;
        rc = upload_runs(ctx);
        if (rc) return rc;
        CK(cudaStreamSynchronize(ctx->stream));
        return PIC_OK;
    }
    if (bx < 1 || by < 1 || R.nx % bx || R.ny % by)
        return fail(ctx, PIC_EINVAL, "coarse block %d x %d must divide the grid %d x %d", bx, by, R.nx, R.ny);
    for (int o = 0; o < PIC_NS; ++o)
        if (o != s && R.sp[o].drag)
            return fail(ctx, PIC_EINVAL, "run %d: the Krook drag acts on one species per run", run);
    float* map = at<float>(ctx, ctx->lay.dragmap[s][run]);
    CK(launch_drag_map(R, map, nu, bx, by, ctx->cfg.dt, ctx->stream));
    R.dragmap[s] = map;
    if (!P.drag) {
        P.drag = 1;
        P.dragf = 0.f;
        return start_drag(ctx, run, s);
    }
    rc = upload_runs(ctx);
    if (rc) return rc;
    CK(cudaStreamSynchronize(ctx->stream));
    return device_flags(ctx);
}

extern "C" int pic_set_collisions(pic_ctx* ctx, int run, int s, double nu, uint64_t seed) {
    if (!ctx) return fail(nullptr, PIC_EINVAL, "null context");
    int rc = check_run(ctx, run);
    if (rc) return rc;
    if (s < 0 || s >= ctx->cfg.nspecies) return fail(ctx, PIC_EINVAL, "species %d out of range", s);
    if (!(std::isfinite(nu) && nu >= 0)) return fail(ctx, PIC_EINVAL, "collision rate must be finite and >= 0");
    if (nu > 0 && !ctx->cfg.track_ids)
        return fail(ctx, PIC_EINVAL, "binary collisions key their draws by particle id: set track_ids");
    SpeciesParams& P = ctx->runs[run].sp[s];
    if (!P.active) return fail(ctx, PIC_ESTATE, "species %d of run %d is not loaded", s, run);
    P.coll = nu > 0 ? 1 : 0;
    P.coll_sigma = (float)std::sqrt(0.5 * nu * ctx->cfg.dt);
    P.seed_lo = (unsigned)(seed & 0xffffffffu);
    P.seed_hi = (unsigned)(seed >> 32);
    rc = upload_runs(ctx);
    if (rc) return rc;
    CK(cudaStreamSynchronize(ctx->stream));
    return PIC_OK;
}

extern "C" int pic_dispersion_growth(const double* params, int32_t nsets, double kmin, double kmax, int32_t nk,
                                     double* gamma_out, double* kstar_out, void* stream) {
    if (nsets < 0 || nk < 1 || !(kmin >= 0) || !(kmax >= kmin) || !std::isfinite(kmax))
        return fail(nullptr, PIC_EINVAL, "need nsets >= 0, nk >= 1 and 0 <= kmin <= kmax");
    if (nsets == 0) return PIC_OK;
    if (!params || !gamma_out || !kstar_out) return fail(nullptr, PIC_EINVAL, "null pointer");
    cudaError_t e = launch_dispersion(params, nsets, kmin, kmax, nk, gamma_out, kstar_out, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(nullptr, PIC_ECUDA, "pic_dispersion_growth: %s", cudaGetErrorString(e));
    return PIC_OK;
}

// ---------------------------------------------------------------- closure network
namespace {
int mlp_norm(const pic_mlp_norm* in, MlpNorm* out) {
    if (!in) return fail(nullptr, PIC_EINVAL, "null norm");
    if (in->nin < 1 || in->nin > PIC_MLP_IN) return fail(nullptr, PIC_EINVAL, "nin must be in [1, %d]", PIC_MLP_IN);
    for (int j = 0; j < PIC_MLP_IN; ++j) {
        if (j < in->nin && !(std::isfinite(in->sigma[j]) && in->sigma[j] > 0 && std::isfinite(in->mu[j])))
            return fail(nullptr, PIC_EINVAL, "feature %d: sigma must be finite and > 0", j);
        out->mu[j] = j < in->nin ? in->mu[j] : 0.f;
        out->inv_sigma[j] = j < in->nin ? 1.0f / in->sigma[j] : 0.f;
    }
    out->nin = in->nin;
    return PIC_OK;
}
}  // namespace

extern "C" int pic_mlp_forward(const float* params, const pic_mlp_norm* norm, const float* x, int64_t ldx,
                               int64_t n, float* y, void* stream) {
    MlpNorm nm;
    int rc = mlp_norm(norm, &nm);
    if (rc) return rc;
    if (n < 0 || ldx < n) return fail(nullptr, PIC_EINVAL, "need n >= 0 and ldx >= n");
    if (n > 0 && (!params || !x || !y)) return fail(nullptr, PIC_EINVAL, "null pointer");
    cudaError_t e = launch_mlp_forward(params, nm, x, ldx, n, y, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(nullptr, PIC_ECUDA, "pic_mlp_forward: %s", cudaGetErrorString(e));
    return PIC_OK;
}

extern "C" int pic_mlp_train_scratch_bytes(size_t* bytes_out) {
    if (!bytes_out) return fail(nullptr, PIC_EINVAL, "null bytes_out");
    *bytes_out = mlp_train_scratch_bytes();
    return PIC_OK;
}

extern "C" int pic_mlp_train_step(float* params, float* adam_m, float* adam_v, int32_t t, float lr,
                                  const pic_mlp_norm* norm, const float* x, int64_t ldx, const float* target,
                                  int64_t n, float* loss, void* scratch, size_t scratch_bytes, void* stream) {
    MlpNorm nm;
    int rc = mlp_norm(norm, &nm);
    if (rc) return rc;
    if (n < 1 || ldx < n) return fail(nullptr, PIC_EINVAL, "need n >= 1 and ldx >= n");
    if (t < 1) return fail(nullptr, PIC_EINVAL, "Adam step t must be >= 1");
    if (!params || !adam_m || !adam_v || !x || !target || !scratch)
        return fail(nullptr, PIC_EINVAL, "null pointer");
    if (scratch_bytes < mlp_train_scratch_bytes())
        return fail(nullptr, PIC_EINVAL, "scratch has %zu bytes, needs %zu", scratch_bytes, mlp_train_scratch_bytes());
    cudaError_t e = launch_mlp_train(params, adam_m, adam_v, t, lr, nm, x, ldx, target, n, loss, scratch,
                                     (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(nullptr, PIC_ECUDA, "pic_mlp_train_step: %s", cudaGetErrorString(e));
    return PIC_OK;
}

extern "C" int pic_mlp_fit_norm(const float* x, int64_t ldx, int64_t n, int32_t nin, float* mu_sigma, void* stream) {
    if (!x || !mu_sigma) return fail(nullptr, PIC_EINVAL, "pic_mlp_fit_norm: null pointer");
    if (nin < 1 || nin > PIC_MLP_IN || n < 1 || ldx < n) return fail(nullptr, PIC_EINVAL, "pic_mlp_fit_norm: bad sizes");
    const cudaError_t e = launch_fit_norm(x, ldx, n, nin, mu_sigma, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(nullptr, PIC_ECUDA, "pic_mlp_fit_norm: %s", cudaGetErrorString(e));
    return PIC_OK;
}

extern "C" int pic_closure_samples_scratch_bytes(int64_t nsamples, size_t* bytes_out) {
    if (!bytes_out || nsamples < 0) return fail(nullptr, PIC_EINVAL, "pic_closure_samples_scratch_bytes: bad argument");
    *bytes_out = closure_samples_scratch_bytes(nsamples);
    return PIC_OK;
}

extern "C" int pic_closure_samples(const float* rows, int32_t nsnap, int64_t nc, int32_t window, float nu_p,
                                   float uz_min, float* feat, float* label, int64_t cap, int64_t* n_out,
                                   void* scratch, size_t scratch_bytes, void* stream) {
    if (!rows || !feat || !label || !n_out || !scratch) return fail(nullptr, PIC_EINVAL, "pic_closure_samples: null pointer");
    if (nsnap < 1 || nc < 1 || window < 1 || window > nsnap || cap < 0)
        return fail(nullptr, PIC_EINVAL, "pic_closure_samples: bad sizes");
    if (!(uz_min >= 0.f) || !std::isfinite(nu_p)) return fail(nullptr, PIC_EINVAL, "pic_closure_samples: bad uz_min or nu_p");
    const long long M = (long long)(nsnap / window) * nc;
    if (scratch_bytes < closure_samples_scratch_bytes(M) || (reinterpret_cast<uintptr_t>(scratch) & 15))
        return fail(nullptr, PIC_EINVAL, "pic_closure_samples: scratch too small or misaligned");
    const cudaError_t e = launch_closure_samples(rows, nsnap, nc, window, nu_p, uz_min, feat, label, cap,
                                                 reinterpret_cast<long long*>(n_out), scratch,
                                                 static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(nullptr, PIC_ECUDA, "pic_closure_samples: %s", cudaGetErrorString(e));
    return PIC_OK;
}

extern "C" int pic_mlp_wait_test(int64_t polls, void* stream) {
    if (polls < 1 || polls > (1 << 20)) return fail(nullptr, PIC_EINVAL, "polls must be in [1, 2^20]");
    const cudaError_t e = launch_mlp_wait_test(polls, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(nullptr, PIC_ECUDA, "pic_mlp_wait_test: %s", cudaGetErrorString(e));
    return PIC_OK;
}

extern "C" int pic_mlp_status(int clear) {
    int err = 0;
    cudaError_t e = mlp_status(&err, clear != 0);
    if (e != cudaSuccess) return fail(nullptr, PIC_ECUDA, "pic_mlp_status: %s", cudaGetErrorString(e));
    if (err) return fail(nullptr, PIC_ETIMEOUT, "a tensor-core completion wait of the closure network timed out");
    return PIC_OK;
}

// ============================================================== autotuner
//
// The compiled variants of the 2D particle kernel (tile shape 16 x 16, 32 x 8, 8 x 32; 2, 3 or
// 4 CTAs per SM) compute the same bits; which is fastest depends on the workload and the GPU.
// pic_autotune times each on the running context and keeps the fastest; picks are kept per key
// (dimension, grids, particles, GPU name) in memory and in a JSON file (PIC_TUNE_CACHE or
// pic_tune_cache_set), one object per line:
//   {"key": "...", "tile_x": 16, "tile_y": 16, "ctas_per_sm": 4, "ms_per_step": 2.70}
// A context created with tile_x = tile_y = ctas_per_sm = 0 starts with the cached pick.
namespace {

struct TunePick {
    int tx, ty, ctas;
    double ms;
};
std::mutex g_tune_mu;
std::map<std::string, TunePick> g_tune;
std::string g_tune_path;
bool g_tune_loaded = false;

std::string json_str_field(const std::string& line, const char* name) {
    const std::string k = std::string("\"") + name + "\"";
    size_t p = line.find(k);
    if (p == std::string::npos) return "";
    p = line.find('"', line.find(':', p + k.size()) + 1);
    if (p == std::string::npos) return "";
    const size_t q = line.find('"', p + 1);
    return q == std::string::npos ? "" : line.substr(p + 1, q - p - 1);
}
double json_num_field(const std::string& line, const char* name, bool* ok) {
    const std::string k = std::string("\"") + name + "\"";
    size_t p = line.find(k);
    if (p == std::string::npos) { *ok = false; return 0; }
    p = line.find(':', p + k.size());
    if (p == std::string::npos) { *ok = false; return 0; }
    char* end = nullptr;
    const double v = std::strtod(line.c_str() + p + 1, &end);
    if (end == line.c_str() + p + 1) *ok = false;
    return v;
}

// Caller holds g_tune_mu.
void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    if (g_tune_path.empty()) {
        const char* env = std::getenv("PIC_TUNE_CACHE");
        if (env) g_tune_path = env;
    }
    if (g_tune_path.empty()) return;
    std::FILE* f = std::fopen(g_tune_path.c_str(), "r");
    if (!f) return;
    char buf[1024];
    while (std::fgets(buf, sizeof buf, f)) {
        const std::string line(buf);
        const std::string key = json_str_field(line, "key");
        bool ok = true;
        TunePick t;
        t.tx = (int)json_num_field(line, "tile_x", &ok);
        t.ty = (int)json_num_field(line, "tile_y", &ok);
        t.ctas = (int)json_num_field(line, "ctas_per_sm", &ok);
        t.ms = json_num_field(line, "ms_per_step", &ok);
        if (ok && !key.empty() && pic::push2d_variant(t.tx, t.ty, t.ctas) >= 0) g_tune[key] = t;
    }
    std::fclose(f);
}

// Caller holds g_tune_mu.  Written to path.tmp and renamed.
int tune_save_locked() {
    if (g_tune_path.empty()) return PIC_OK;
    const std::string tmp = g_tune_path + ".tmp";
    std::FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return PIC_EINVAL;
    for (const auto& kv : g_tune)
        std::fprintf(f, "{\"key\": \"%s\", \"tile_x\": %d, \"tile_y\": %d, \"ctas_per_sm\": %d, \"ms_per_step\": %.6f}\n",
                     kv.first.c_str(), kv.second.tx, kv.second.ty, kv.second.ctas, kv.second.ms);
    const bool bad = std::fclose(f) != 0;
    if (bad || std::rename(tmp.c_str(), g_tune_path.c_str()) != 0) return PIC_EINVAL;
    return PIC_OK;
}

// Workload key: dimension, grids and particles per run (an FNV-1a hash of them for more than
// four runs), and the GPU's name.
std::string tune_key(const pic_config& c, int nruns, const int32_t* dims, const int64_t* caps) {
    int dev = 0;
    cudaDeviceProp prop;
    std::string gpu = "unknown";
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) gpu = prop.name;
    std::string k = "ndim=" + std::to_string(c.ndim) + ";runs=" + std::to_string(nruns) + ";";
    if (nruns <= 4) {
        for (int r = 0; r < nruns; ++r) {
            k += std::to_string(dims[3 * r]) + "x" + std::to_string(dims[3 * r + 1]);
            if (c.ndim == 3) k += "x" + std::to_string(dims[3 * r + 2]);
            k += ":";
            for (int s = 0; s < c.nspecies; ++s) k += std::to_string(caps[PIC_NS * r + s]) + (s + 1 < c.nspecies ? "+" : ";");
        }
    } else {
        unsigned long long h = 1469598103934665603ull;
        auto mix = [&](long long v) {
            for (int b = 0; b < 8; ++b) { h ^= (unsigned long long)((v >> (8 * b)) & 255); h *= 1099511628211ull; }
        };
        for (int r = 0; r < nruns; ++r) {
            for (int d = 0; d < 3; ++d) mix(dims[3 * r + d]);
            for (int s = 0; s < c.nspecies; ++s) mix(caps[PIC_NS * r + s]);
        }
        char hb[32];
        std::snprintf(hb, sizeof hb, "%016llx", h);
        k += std::string("batch=") + hb + ";";
    }
    for (char& ch : gpu) if (ch == '"' || ch == '\\') ch = '_';
    return k + "gpu=" + gpu;
}

}  // namespace

// Switch the 2D particle kernel (and the tiled field kernels) to variant v; the tile count per
// run is the same for every shape (256 cells per tile), so only the tile grid changes.
int switch_variant(pic_ctx* ctx, int v) {
    int tx, ty, mb;
    push2d_variant_info(v, &tx, &ty, &mb);
    for (const RunGeo& G : ctx->geo.runs)
        if (G.nx % tx || G.ny % ty) return fail(ctx, PIC_EINVAL, "tile %d x %d does not divide a %d x %d grid", tx, ty, G.nx, G.ny);
    ctx->geo.tx = tx;
    ctx->geo.ty = ty;
    ctx->geo.push_variant = v;
    for (int r = 0; r < ctx->nruns; ++r) {
        RunGeo& G = ctx->geo.runs[r];
        G.ntx = G.nx / tx;
        G.nty = G.ny / ty;
        ctx->runs[r].ntx = G.ntx;
        ctx->runs[r].nty = G.nty;
    }
    ctx->args.tx = tx;
    ctx->args.ty = ty;
    ctx->args.push_variant = v;
    return upload_runs(ctx);
}

// The cached pick for a new context configured with default tiles (2D), if any.
void apply_cached_variant(pic_ctx* ctx) {
    const pic_config& c = ctx->cfg;
    if (c.ndim != 2 || c.tile_x || c.tile_y || c.ctas_per_sm) return;
    TunePick t{};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load_locked();
        auto it = g_tune.find(ctx->tune_key);
        if (it == g_tune.end()) return;
        t = it->second;
    }
    const int v = push2d_variant(t.tx, t.ty, t.ctas);
    if (v >= 0 && v != ctx->geo.push_variant) switch_variant(ctx, v);
}

extern "C" int pic_tune_cache_set(const char* path) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
    g_tune_loaded = false;
    g_tune_path = path ? path : "";
    tune_load_locked();
    return PIC_OK;
}

extern "C" int pic_tile_config(const pic_ctx* ctx, int32_t* out3) {
    if (!ctx || !out3) return fail(nullptr, PIC_EINVAL, "null argument");
    int tx, ty, mb;
    if (ctx->cfg.ndim == 2) {
        push2d_variant_info(ctx->geo.push_variant, &tx, &ty, &mb);
    } else {
        tx = ctx->geo.tx; ty = ctx->geo.ty; mb = 0;
    }
    out3[0] = tx; out3[1] = ty; out3[2] = ctx->cfg.ndim == 2 ? mb : ctx->geo.tz;
    return PIC_OK;
}

extern "C" int pic_autotune(pic_ctx* ctx, int steps_per_variant, pic_tune_entry* out, int max_entries, int* n_out) {
    if (!ctx) return fail(nullptr, PIC_EINVAL, "null context");
    if (steps_per_variant < 1) return fail(ctx, PIC_EINVAL, "steps_per_variant must be >= 1");
    if (max_entries > 0 && !out) return fail(ctx, PIC_EINVAL, "null output");
    int rc = pic_sync(ctx);
    if (rc) return rc;
    const int K = ctx->sort_interval;
    const int steps = ((steps_per_variant + K - 1) / K) * K;
    std::vector<int> cand;
    if (ctx->cfg.ndim == 2) {
        for (int v = 0; v < push2d_num_variants(); ++v) {
            int tx, ty, mb;
            push2d_variant_info(v, &tx, &ty, &mb);
            bool fits = true;
            for (const RunGeo& G : ctx->geo.runs) fits = fits && G.nx % tx == 0 && G.ny % ty == 0;
            if (fits) cand.push_back(v);
        }
    } else {
        cand.push_back(-1);      // one 3D kernel: timed, nothing to choose
    }
    cudaEvent_t e0 = get_event(ctx), e1 = get_event(ctx);
    int best = -1, n = 0;
    double best_ms = 0;
    for (int v : cand) {
        if (v >= 0) {
            rc = switch_variant(ctx, v);
            if (rc) break;
        }
        rc = pic_step(ctx, K);            // warm-up: graph capture of the new variant
        if (rc) break;
        CK(cudaEventRecord(e0, ctx->stream));
        rc = pic_step(ctx, steps);
        if (rc) break;
        CK(cudaEventRecord(e1, ctx->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        const double per = ms / steps;
        int32_t cfg3[3];
        pic_tile_config(ctx, cfg3);
        if (n < max_entries) {
            out[n].tile_x = cfg3[0];
            out[n].tile_y = cfg3[1];
            out[n].ctas_per_sm = cfg3[2];
            out[n].ms_per_step = (float)per;
        }
        ++n;
        if (best < 0 || per < best_ms) { best = v; best_ms = per; }
    }
    ctx->pool.push_back(e0);
    ctx->pool.push_back(e1);
    if (rc) return rc;
    if (n_out) *n_out = std::min(n, std::max(max_entries, 0));
    if (best >= 0) {
        rc = switch_variant(ctx, best);
        if (rc) return rc;
        int tx, ty, mb;
        push2d_variant_info(best, &tx, &ty, &mb);
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load_locked();
        g_tune[ctx->tune_key] = TunePick{tx, ty, mb, best_ms};
        if (tune_save_locked() != PIC_OK) return fail(ctx, PIC_EINVAL, "cannot write the tuning cache %s", g_tune_path.c_str());
    }
    return pic_sync(ctx);
}

// ============================================================== checkpoint / restore
//
// File layout (little-endian, this library's struct layouts, checked by size fields):
//   CkptHeader; per run a CkptRunGeo (checked against the restoring context) and a CkptRunState
//   (host-side run state); then the context's arena bytes [0, layout total).
// Device pointers are never read back from a file: a restore rebuilds every pointer of the run
// table from the restoring context's own layout, so a file can only change values, not addresses.
namespace {

constexpr char kCkptMagic[8] = {'P', 'I', 'C', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kCkptVersion = 2;   // 2: 3D particles binned by tile
constexpr size_t kCkptChunk = size_t(64) << 20;

struct CkptHeader {
    char magic[8];
    uint32_t version, header_bytes, rungeo_bytes, runstate_bytes, species_bytes, ctl_bytes;
    int32_t ndim, nspecies, nruns, track_ids, keep_j, j_filter;
    int32_t diag_interval, diag_capacity, sort_interval, reserved;
    int32_t cap[PIC_NS], cap_stay[PIC_NS], spill_cap[PIC_NS];
    double dx, dy, dz, dt;
    uint64_t layout_total;
    int64_t host_step;
    double q[PIC_NS];
    int32_t q_set[PIC_NS];
};

struct CkptRunGeo {
    int64_t nx, ny, nz;
    int64_t capacity[PIC_NS];
};

struct CkptRunState {
    SpeciesParams sp[PIC_NS];
    int32_t shift;
    float jscale, jfscale;
    int32_t drag_moments;          // msum / mcnt / ubar published (a Krook species was loaded)
    int32_t dragmap[PIC_NS];       // per-cell drag map set for species s
    int32_t reserved;
    int64_t loaded[PIC_NS];
    double nu[PIC_NS];
};

CkptHeader ckpt_header(const pic_ctx* ctx) {
    CkptHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, kCkptMagic, sizeof h.magic);
    h.version = kCkptVersion;
    h.header_bytes = sizeof(CkptHeader);
    h.rungeo_bytes = sizeof(CkptRunGeo);
    h.runstate_bytes = sizeof(CkptRunState);
    h.species_bytes = sizeof(SpeciesParams);
    h.ctl_bytes = sizeof(Ctl);
    const pic_config& c = ctx->cfg;
    h.ndim = c.ndim;
    h.nspecies = c.nspecies;
    h.nruns = ctx->nruns;
    h.track_ids = c.track_ids ? 1 : 0;
    h.keep_j = (c.flags & PIC_FLAG_KEEP_J) ? 1 : 0;
    h.j_filter = c.j_filter;
    h.diag_interval = c.diag_interval;
    h.diag_capacity = c.diag_interval > 0 ? c.diag_capacity : 0;
    h.sort_interval = ctx->sort_interval;
    for (int s = 0; s < PIC_NS; ++s) {
        h.cap[s] = ctx->geo.cap[s];
        h.cap_stay[s] = ctx->geo.cap_stay[s];
        h.spill_cap[s] = ctx->geo.spill_cap[s];
        h.q[s] = ctx->q[s];
        h.q_set[s] = ctx->q_set[s] ? 1 : 0;
    }
    h.dx = c.dx; h.dy = c.dy; h.dz = c.dz; h.dt = c.dt;
    h.layout_total = ctx->lay.total;
    h.host_step = ctx->host_step;
    return h;
}

CkptRunGeo ckpt_rungeo(const pic_ctx* ctx, int r) {
    CkptRunGeo g;
    std::memset(&g, 0, sizeof g);
    const RunGeo& G = ctx->geo.runs[r];
    g.nx = G.nx; g.ny = G.ny; g.nz = G.nz;
    for (int s = 0; s < PIC_NS; ++s) g.capacity[s] = G.capacity[s];
    return g;
}

// Everything of the header that fixes the arena layout or the step schedule; host_step, q and
// q_set are state, not geometry.
bool ckpt_same_geometry(const CkptHeader& a, const CkptHeader& b) {
    CkptHeader x = a, y = b;
    x.host_step = y.host_step = 0;
    for (int s = 0; s < PIC_NS; ++s) { x.q[s] = y.q[s] = 0; x.q_set[s] = y.q_set[s] = 0; }
    return std::memcmp(&x, &y, sizeof x) == 0;
}

struct File {
    FILE* f = nullptr;
    ~File() { if (f) std::fclose(f); }
};

}  // namespace

extern "C" int pic_checkpoint(pic_ctx* ctx, const char* path) {
    if (!ctx) return fail(nullptr, PIC_EINVAL, "null context");
    if (!path || !*path) return fail(ctx, PIC_EINVAL, "null or empty path");
    int rc = pic_sync(ctx);              // the state of the last queued step, and its sticky flags
    if (rc) return rc;
    const std::string tmp = std::string(path) + ".tmp";
    {
        File out;
        out.f = std::fopen(tmp.c_str(), "wb");
        if (!out.f) return fail(ctx, PIC_EINVAL, "cannot open %s for writing", tmp.c_str());
        const CkptHeader h = ckpt_header(ctx);
        bool ok = std::fwrite(&h, sizeof h, 1, out.f) == 1;
        for (int r = 0; ok && r < ctx->nruns; ++r) {
            const CkptRunGeo g = ckpt_rungeo(ctx, r);
            const RunDev& R = ctx->runs[r];
            CkptRunState st;
            std::memset(&st, 0, sizeof st);
            for (int s = 0; s < PIC_NS; ++s) {
                st.sp[s] = R.sp[s];
                st.dragmap[s] = R.dragmap[s] ? 1 : 0;
                st.loaded[s] = ctx->loaded[(size_t)r * PIC_NS + s];
                st.nu[s] = ctx->nu[(size_t)r * PIC_NS + s];
            }
            st.shift = R.shift;
            st.jscale = R.jscale;
            st.jfscale = R.jfscale;
            st.drag_moments = R.msum[0] ? 1 : 0;
            ok = std::fwrite(&g, sizeof g, 1, out.f) == 1 && std::fwrite(&st, sizeof st, 1, out.f) == 1;
        }
        std::vector<char> buf(std::min(kCkptChunk, ctx->lay.total));
        cudaError_t ce = cudaSuccess;
        for (size_t off = 0; ok && off < ctx->lay.total; off += buf.size()) {
            const size_t n = std::min(buf.size(), ctx->lay.total - off);
            ce = cudaMemcpyAsync(buf.data(), ctx->arena + off, n, cudaMemcpyDeviceToHost, ctx->stream);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
            ok = ce == cudaSuccess && std::fwrite(buf.data(), 1, n, out.f) == n;
        }
        ok = ok && std::fflush(out.f) == 0;
        const int cl = std::fclose(out.f);
        out.f = nullptr;
        if (!ok || cl != 0) {
            std::remove(tmp.c_str());
            if (ce != cudaSuccess) return fail(ctx, PIC_ECUDA, "pic_checkpoint: %s", cudaGetErrorString(ce));
            return fail(ctx, PIC_EINVAL, "writing %s failed", tmp.c_str());
        }
    }
    if (std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return fail(ctx, PIC_EINVAL, "cannot rename %s to %s", tmp.c_str(), path);
    }
    return PIC_OK;
}

extern "C" int pic_restore(pic_ctx* ctx, const char* path) {
    if (!ctx) return fail(nullptr, PIC_EINVAL, "null context");
    if (!path || !*path) return fail(ctx, PIC_EINVAL, "null or empty path");
    File in;
    in.f = std::fopen(path, "rb");
    if (!in.f) return fail(ctx, PIC_EINVAL, "cannot open %s", path);
    CkptHeader h;
    if (std::fread(&h, sizeof h, 1, in.f) != 1) return fail(ctx, PIC_EINVAL, "%s: short header", path);
    if (std::memcmp(h.magic, kCkptMagic, sizeof h.magic) != 0) return fail(ctx, PIC_EINVAL, "%s: not a checkpoint", path);
    if (h.version != kCkptVersion || h.header_bytes != sizeof(CkptHeader) || h.rungeo_bytes != sizeof(CkptRunGeo) ||
        h.runstate_bytes != sizeof(CkptRunState) || h.species_bytes != sizeof(SpeciesParams) || h.ctl_bytes != sizeof(Ctl))
        return fail(ctx, PIC_EINVAL, "%s: written by an incompatible library version", path);
    if (!ckpt_same_geometry(h, ckpt_header(ctx)))
        return fail(ctx, PIC_EINVAL, "%s: configuration differs from this context's (grid, species, slots, "
                                     "dx, dt, intervals, ids, filter or KEEP_J)", path);
    if (h.host_step < 0) return fail(ctx, PIC_EINVAL, "%s: bad step count", path);
    std::vector<CkptRunState> st(ctx->nruns);
    for (int r = 0; r < ctx->nruns; ++r) {
        CkptRunGeo g;
        if (std::fread(&g, sizeof g, 1, in.f) != 1 || std::fread(&st[r], sizeof st[r], 1, in.f) != 1)
            return fail(ctx, PIC_EINVAL, "%s: short run table", path);
        const CkptRunGeo mine = ckpt_rungeo(ctx, r);
        if (std::memcmp(&g, &mine, sizeof g) != 0)
            return fail(ctx, PIC_EINVAL, "%s: run %d has another grid or capacity than this context's", path, r);
        for (int s = 0; s < PIC_NS; ++s)
            if (st[r].loaded[s] < 0 || st[r].loaded[s] > mine.capacity[s] || !(st[r].nu[s] >= 0))
                return fail(ctx, PIC_EINVAL, "%s: run %d: bad species state", path, r);
    }
    // the arena image must be exactly what is left of the file
    const long here = std::ftell(in.f);
    if (here < 0 || std::fseek(in.f, 0, SEEK_END) != 0) return fail(ctx, PIC_EINVAL, "%s: cannot seek", path);
    const long end = std::ftell(in.f);
    if (end < here || (unsigned long long)(end - here) != (unsigned long long)ctx->lay.total)
        return fail(ctx, PIC_EINVAL, "%s: arena image has %lld bytes, this context needs %zu", path,
                    (long long)(end - here), ctx->lay.total);
    if (std::fseek(in.f, here, SEEK_SET) != 0) return fail(ctx, PIC_EINVAL, "%s: cannot seek", path);

    CK(cudaStreamSynchronize(ctx->stream));
    std::vector<char> buf(std::min(kCkptChunk, ctx->lay.total));
    for (size_t off = 0; off < ctx->lay.total; off += buf.size()) {
        const size_t n = std::min(buf.size(), ctx->lay.total - off);
        if (std::fread(buf.data(), 1, n, in.f) != n) return fail(ctx, PIC_EINVAL, "%s: short arena image", path);
        CK(cudaMemcpyAsync(ctx->arena + off, buf.data(), n, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    // host state; pointers from this context's layout
    const Layout& L = ctx->lay;
    for (int r = 0; r < ctx->nruns; ++r) {
        RunDev& R = ctx->runs[r];
        for (int s = 0; s < PIC_NS; ++s) {
            R.sp[s] = st[r].sp[s];
            R.dragmap[s] = (st[r].dragmap[s] && s < ctx->cfg.nspecies) ? at<float>(ctx, L.dragmap[s][r]) : nullptr;
            ctx->loaded[(size_t)r * PIC_NS + s] = st[r].loaded[s];
            ctx->nu[(size_t)r * PIC_NS + s] = st[r].nu[s];
        }
        R.shift = st[r].shift;
        R.jscale = st[r].jscale;
        R.jfscale = st[r].jfscale;
        for (int d = 0; d < 3; ++d) {
            R.msum[d] = st[r].drag_moments ? at<long long>(ctx, L.msum[d][r]) : nullptr;
            R.ubar[d] = st[r].drag_moments ? at<float>(ctx, L.ubar[d][r]) : nullptr;
        }
        R.mcnt = st[r].drag_moments ? at<int>(ctx, L.mcnt[r]) : nullptr;
    }
    for (int s = 0; s < PIC_NS; ++s) {
        ctx->q[s] = h.q[s];
        ctx->q_set[s] = h.q_set[s] != 0;
    }
    ctx->host_step = h.host_step;
    int rc = upload_runs(ctx);           // overwrites the run table of the image
    if (rc) return rc;
    return pic_sync(ctx);
}

extern "C" int64_t pic_loaded_count(const pic_ctx* ctx, int run, int s) {
    if (!ctx || run < 0 || run >= ctx->nruns || s < 0 || s >= PIC_NS) return -1;
    return ctx->loaded[(size_t)run * PIC_NS + s];
}

extern "C" int64_t pic_launch_count(const pic_ctx* ctx) { return ctx ? ctx->launches : -1; }

extern "C" int64_t pic_step_count(const pic_ctx* ctx) { return ctx ? ctx->host_step : -1; }

extern "C" int pic_num_runs(const pic_ctx* ctx) { return ctx ? ctx->nruns : -1; }

namespace pic {
// Error text of a failed call that has no context (read back with pic_last_error(NULL)).
void set_call_error(const char* msg) { g_init_error = msg; }
}  // namespace pic

extern "C" const char* pic_last_error(const pic_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

extern "C" void pic_free(pic_ctx* ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    for (auto& ev : ctx->pending) { cudaEventDestroy(ev.a); cudaEventDestroy(ev.b); }
    for (auto e : ctx->pool) cudaEventDestroy(e);
    delete ctx;
}
