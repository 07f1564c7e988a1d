// push3d.cu -- fused 3D3V particle step: CIC field gather on the Yee lattice, relativistic Boris
// push, Krook drag, move with cell carry, charge-conserving Esirkepov current deposition (CIC,
// int64 fixed point) and rebinning of every particle into its new tile's slots of the other
// buffer.
//
// One CTA of 256 threads per (run, tile) of 8 x 8 x 4 cells.  Particles are binned by tile: a
// tile's slot range holds its particles in any order, each with its cell within the tile, so
// that a CTA reads and writes whole sectors (a cell's ~8 particles per species filled less than
// a sector of each array, and partly written sectors are read back from DRAM).  The CTA walks
// its list in batches of 512, one particle per thread per half batch.  Each particle is pushed
// and rebinned, and its move recorded in shared memory: moves inside one cell from the front,
// the others from the back.  In three dimensions a large share of the beam crosses a cell edge
// every step (v_z dt / dz ~ 0.47), so there is no per-cell register path; the batch's deposit
// then runs over the records, warps of in-cell moves adding the 12 terms of a move without
// crossings and warps of the other moves up to 3 x 18 terms, with predicated 32-bit shared
// reductions.  A batch adds at most 512 terms of magnitude <= 2^21 to any node, so the int32
// accumulators cannot overflow; after each batch they are folded into an int64 shared bank
// (each thread owns fixed nodes, no atomics) while the next batch is pushed.  Particles that
// stay inside the tile take the next places of the tile's stay area through a shared counter
// (one claim per warp and species); those leaving the tile claim places in the destination
// tile's immigrant area with one global atomic per destination among a warp's leavers.
#include "particle_math.cuh"
#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int TX = 8, TY = 8, TZ = 4;
constexpr int RX = TX + 3, RY = TY + 3, RZ = TZ + 3;   // tile + CIC/Esirkepov stencil halo
constexpr int RXY = RX * RY, RN = RXY * RZ;
constexpr int CELLS = TX * TY * TZ;
constexpr int NT = 256, NW = NT / 32;
constexpr int PER_THREAD = 2;
constexpr int BATCH = NT * PER_THREAD;   // particles per int32 accumulation round
constexpr unsigned FULL = 0xffffffffu;

static_assert(CELLS == NT, "one thread per tile cell in the setup loops");
static_assert(RN <= 1024, "region nodes fit the 10-bit field of a deposit record");
static_assert((CELLS & (CELLS - 1)) == 0, "in-tile cell indices are masked with CELLS - 1");

struct Smem {
    float F[6][RN];                  // Ex Ey Ez Bx By Bz of the region (origin: tile - 1 cell)
    int J32[3][RN];                  // current of the running batch
    long long J64[3][RN];            // current of the finished batches
    // deposit records of the batch: moves inside a cell from the front, the rest from the back;
    // old and new offsets and a meta word (region node of the old cell bits 0-9, species bit 10,
    // cell steps + 1 bits 11-16)
    float ro[3][BATCH];
    float rn[3][BATCH];
    int rm[BATCH];
    int nrs[2], nrm[2];              // records from the front and from the back (by batch parity)
    double red[NW][6];
    unsigned long long kin[5];
    int ln[PIC_NS];                  // particles of the tile's list per species (current buffer)
    int lns[PIC_NS];                 // of which in its stay area
    int sfill[PIC_NS];               // stay-area fill of the tile in the next buffer
    SpeciesParams sp[PIC_NS];
    // drag arrays last: a launch without drag allocates the shared memory up to `ub` only
    float ub[3][RN];                 // previous cell-mean momentum (drag)
    unsigned Mlo[3][RN];             // drag moments (fixed point 2^20), value = Mhi * 4096 + Mlo
    int Mhi[3][RN];
    int MC[RN];                      // drag counts
};

// Shared memory per SM (228 KB, 1 KB reserved per CTA) holds 3 CTAs without drag, 2 with.
static_assert(3 * (offsetof(Smem, ub) + 1024) <= 228 * 1024, "3 CTAs per SM without drag");
static_assert(2 * (sizeof(Smem) + 1024) <= 228 * 1024, "2 CTAs per SM with drag");

// ------------------------------------------------------------------ gather
// Per axis: node-lattice weights (points c, c+1) and half-lattice weights with their first point
// (c-1 for o < 1/2, else c), for an offset o in [0,1).
struct AxisW {
    float n0, n1;
    float h0, h1;
    int hb;
};
__device__ __forceinline__ AxisW axis_weights(float o) {
    AxisW w;
    w.n0 = __fsub_rn(1.f, o);
    w.n1 = o;
    const float d = __fsub_rn(o, 0.5f);
    if (d < 0.f) {
        w.hb = -1;
        w.h0 = -d;
        w.h1 = __fsub_rn(1.f, -d);
    } else {
        w.hb = 0;
        w.h0 = __fsub_rn(1.f, d);
        w.h1 = d;
    }
    return w;
}

// Trilinear interpolation of component c from accessor F(c, i, j, k) (offsets relative to the
// particle's cell node), half-shifted along the axes flagged in (hx, hy, hz).
template <class A>
__device__ __forceinline__ float interp(const A& F, int c, bool hx, bool hy, bool hz, const AxisW& wx,
                                        const AxisW& wy, const AxisW& wz) {
    const int i0 = hx ? wx.hb : 0, j0 = hy ? wy.hb : 0, k0 = hz ? wz.hb : 0;
    const float ax0 = hx ? wx.h0 : wx.n0, ax1 = hx ? wx.h1 : wx.n1;
    const float ay0 = hy ? wy.h0 : wy.n0, ay1 = hy ? wy.h1 : wy.n1;
    const float az0 = hz ? wz.h0 : wz.n0, az1 = hz ? wz.h1 : wz.n1;
    float fz[2];
#pragma unroll
    for (int dk = 0; dk < 2; ++dk) {
        float fy[2];
#pragma unroll
        for (int dj = 0; dj < 2; ++dj)
            fy[dj] = __fmaf_rn(ax1, F(c, i0 + 1, j0 + dj, k0 + dk), __fmul_rn(ax0, F(c, i0, j0 + dj, k0 + dk)));
        fz[dk] = __fmaf_rn(ay1, fy[1], __fmul_rn(ay0, fy[0]));
    }
    return __fmaf_rn(az1, fz[1], __fmul_rn(az0, fz[0]));
}

// Yee staggering: Ex (1/2,0,0) Ey (0,1/2,0) Ez (0,0,1/2) Bx (0,1/2,1/2) By (1/2,0,1/2) Bz (1/2,1/2,0).
template <class A>
__device__ __forceinline__ void gather3(const A& F, const AxisW& wx, const AxisW& wy, const AxisW& wz, float EB[6]) {
    EB[0] = interp(F, 0, true, false, false, wx, wy, wz);
    EB[1] = interp(F, 1, false, true, false, wx, wy, wz);
    EB[2] = interp(F, 2, false, false, true, wx, wy, wz);
    EB[3] = interp(F, 3, false, true, true, wx, wy, wz);
    EB[4] = interp(F, 4, true, false, true, wx, wy, wz);
    EB[5] = interp(F, 5, true, true, false, wx, wy, wz);
}

struct SharedFields3 {
    const Smem* s;
    int n0;   // region index of the particle's cell node
    int* err; // sticky flags (index checks of the bounds-checked build)
    __device__ __forceinline__ float operator()(int c, int i, int j, int k) const {
        const int n = n0 + k * RXY + j * RX + i;
        return dbg_in(n, RN, err) ? s->F[c][n] : 0.f;
    }
};
struct GlobalFields3 {
    const RunDev* R;
    int cx, cy, cz;
    __device__ __forceinline__ float operator()(int c, int i, int j, int k) const {
        const int gi = wrapi(cx + i, R->nx), gj = wrapi(cy + j, R->ny), gk = wrapi(cz + k, R->nz);
        const float* p = c < 3 ? R->E[c] : R->B[c - 3];
        return __ldg(p + ((size_t)gk * R->ny + gj) * R->nx + gi);
    }
};

// ------------------------------------------------------------------ one particle
struct Pushed3 {
    float ux, uy, uz;    // u^{n+1/2}
    float no[3];         // new offsets
    int st[3];           // cell steps
    bool bad;
};

template <bool DRAG, class A>
__device__ __forceinline__ Pushed3 push3_one(const A& F, const SpeciesParams& P, const RunConst& K,
                                             const float o[3], float ux, float uy, float uz,
                                             float b0, float b1, float b2, float df, int s, unsigned id,
                                             long long step) {
    Pushed3 r;
    const AxisW wx = axis_weights(o[0]), wy = axis_weights(o[1]), wz = axis_weights(o[2]);
    float EB[6];
    gather3(F, wx, wy, wz, EB);
    boris(P.qmdt2, EB, ux, uy, uz);
    if (DRAG && P.drag) {
        ux = __fmaf_rn(-df, b0, ux);
        uy = __fmaf_rn(-df, b1, uy);
        uz = __fmaf_rn(-df, b2, uz);
    }
    if (P.coll) collide_ion(ux, uy, uz, P, s, id, step);
    const float ig = rsqrtf(__fmaf_rn(uz, uz, __fmaf_rn(uy, uy, __fmaf_rn(ux, ux, 1.f))));
    const float rx = __fmaf_rn(__fmul_rn(ux, ig), K.dtdx, o[0]);
    const float ry = __fmaf_rn(__fmul_rn(uy, ig), K.dtdy, o[1]);
    const float rz = __fmaf_rn(__fmul_rn(uz, ig), K.dtdz, o[2]);
    r.bad = !(rx > -1.f && rx < 2.f && ry > -1.f && ry < 2.f && rz > -1.f && rz < 2.f);
    carry(rx, r.no[0], r.st[0]);
    carry(ry, r.no[1], r.st[1]);
    carry(rz, r.no[2], r.st[2]);
    r.ux = ux; r.uy = uy; r.uz = uz;
    return r;
}

// The current terms of one move (Esirkepov, CIC): for the axis a with the transverse axes b, c,
// J_a on the two edges k of the window = round(j_a C_a[k] F_bc), F_bc = S0_b p_c + S1_b q_c the
// path-averaged transverse shape (p = S0/3 + S1/6, q = S0/6 + S1/3).  add(comp, i, j, k, v)
// receives node offsets relative to the window base (b_x, b_y, b_z).  A particle that does not
// cross a cell edge along an axis has a zero third node (S0 = S1 = 0) and a zero second edge
// (C[1] = 0) on that axis: xa, ya, za (warp-uniform: "some lane of the warp crosses along x, y,
// z") skip those terms for the whole warp; the remaining terms are unchanged.
template <class Add>
__device__ __forceinline__ void deposit3(const Add& add, const SpeciesParams& P, const Win& wx, const Win& wy,
                                         const Win& wz, bool xa, bool ya, bool za) {
    float px[3], qx[3], py[3], qy[3], pz[3], qz[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        px[i] = zp(wx.S0[i], wx.S1[i]); qx[i] = zq(wx.S0[i], wx.S1[i]);
        py[i] = zp(wy.S0[i], wy.S1[i]); qy[i] = zq(wy.S0[i], wy.S1[i]);
        pz[i] = zp(wz.S0[i], wz.S1[i]); qz[i] = zq(wz.S0[i], wz.S1[i]);
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        if (m == 2 && !za) continue;
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            if (l == 2 && !ya) continue;
            const float f = zw(wy.S0[l], wy.S1[l], pz[m], qz[m]);
            add(0, 0, l, m, round_small(__fmul_rn(P.jx, wx.C[0]), f));
            if (xa) add(0, 1, l, m, round_small(__fmul_rn(P.jx, wx.C[1]), f));
        }
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        if (m == 2 && !za) continue;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (k == 2 && !xa) continue;
            const float f = zw(wz.S0[m], wz.S1[m], px[k], qx[k]);
            add(1, k, 0, m, round_small(__fmul_rn(P.jy, wy.C[0]), f));
            if (ya) add(1, k, 1, m, round_small(__fmul_rn(P.jy, wy.C[1]), f));
        }
    }
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        if (l == 2 && !ya) continue;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (k == 2 && !xa) continue;
            const float f = zw(wx.S0[k], wx.S1[k], py[l], qy[l]);
            add(2, k, l, 0, round_small(__fmul_rn(P.jz, wz.C[0]), f));
            if (za) add(2, k, l, 1, round_small(__fmul_rn(P.jz, wz.C[1]), f));
        }
    }
}

// Shared-memory reduction without a branch: `red` only when v != 0 (predicated).
__device__ __forceinline__ void red_shared_nz(int* p, int v) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.s32 q, %1, 0;\n\t@q red.shared.add.s32 [%0], %1;\n\t}\n"
                 ::"r"(a), "r"(v) : "memory");
}

// ------------------------------------------------------------------ rebinning
// Slot `slot` of buffer D (a tile's slot range; lc = the particle's cell within the tile).
__device__ __forceinline__ void store3(const Slots& D, long long slot, const float o[3], float ux, float uy,
                                       float uz, int id, int lc) {
    const size_t q = slot_elt(D, slot);
    D.o[0][q] = o[0]; D.o[1][q] = o[1]; D.o[2][q] = o[2];
    D.u[0][q] = ux; D.u[1][q] = uy; D.u[2][q] = uz;
    if (D.id) D.id[q] = id;
    D.lc[q] = lc;
}

// Spill-list entry of buffer D (global cell g).
__device__ __forceinline__ void spill3(const Slots& D, int spill_cap, long long g, const float o[3], float ux,
                                       float uy, float uz, int id, int* err) {
    const int sp = atomicAdd(D.sn, 1);
    if (sp < spill_cap) {
        D.scell[sp] = (int)g;
        D.so[0][sp] = o[0]; D.so[1][sp] = o[1]; D.so[2][sp] = o[2];
        D.su[0][sp] = ux; D.su[1][sp] = uy; D.su[2][sp] = uz;
        if (D.sid) D.sid[sp] = id;
    } else {
        atomicOr(err, ERR_SPILL_FULL);
    }
}

// Particle arriving in tile (unit) T of buffer D from elsewhere, claim pi of its immigrant area
// already taken: store it, or spill it when the area is full.
__device__ __forceinline__ void put_claimed3(const Slots& D, int cap, int cap_stay, int spill_cap, long long T,
                                             int pi, int lc, long long g, const float o[3], float ux, float uy,
                                             float uz, int id, int* err) {
    if (pi < cap - cap_stay) store3(D, T * cap + cap_stay + pi, o, ux, uy, uz, id, lc);
    else spill3(D, spill_cap, g, o, ux, uy, uz, id, err);
}
// The same with its own claim.
__device__ __forceinline__ void put_imm3(const Slots& D, int cap, int cap_stay, int spill_cap, long long T, int lc,
                                         long long g, const float o[3], float ux, float uy, float uz, int id,
                                         int* err) {
    put_claimed3(D, cap, cap_stay, spill_cap, T, atomicAdd(&D.icount[T], 1), lc, g, o, ux, uy, uz, id, err);
}

__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Deposit the batch's records: warps take records [0, nrs) (moves inside one cell: the 12 terms
// of deposit3 without crossings) and then [BATCH - nrm, BATCH) (the others: per warp, the terms
// of an axis are left out when no lane of the warp crosses along it).
__device__ __forceinline__ void deposit_records(Smem& sm, int cp, int lane, int warp, int* err) {
    const int nrs = sm.nrs[cp], nrm = sm.nrm[cp];
    const int nch = (nrs + 31) / 32 + (nrm + 31) / 32;   // warp chunks: stay records, then the rest
    for (int c = warp; c < nch; c += NW) {
        const int cs = (nrs + 31) / 32;
        const bool front = c < cs;
        const int i = front ? c * 32 + lane : BATCH - nrm + (c - cs) * 32 + lane;
        const bool valid = front ? i < nrs : i < BATCH;
        float o[3] = {0.f, 0.f, 0.f}, no[3] = {0.f, 0.f, 0.f};
        int meta = (1 << 11) | (1 << 13) | (1 << 15);
        if (valid && dbg_in(i, BATCH, err)) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                o[d] = sm.ro[d][i];
                no[d] = sm.rn[d][i];
            }
            meta = sm.rm[i];
        }
        const int n0 = meta & 1023, s = (meta >> 10) & 1;
        if (front) {
            // a move inside one cell: the windows and terms with no carry, known at compile time
            // (the same operations, so the same bits, as the general form below with zero carries)
            if (valid) {
                const SpeciesParams& P = sm.sp[s];
                const Win wx = window(o[0], 0, no[0]), wy = window(o[1], 0, no[1]), wz = window(o[2], 0, no[2]);
                auto add = [&](int cc, int ii, int jj, int kk, int v) {
                    if (dbg_in(n0 + kk * RXY + jj * RX + ii, RN, err)) red_shared_nz(&sm.J32[cc][n0 + kk * RXY + jj * RX + ii], v);
                };
                deposit3(add, P, wx, wy, wz, false, false, false);
            }
            continue;
        }
        const int stx = ((meta >> 11) & 3) - 1, sty = ((meta >> 13) & 3) - 1, stz = ((meta >> 15) & 3) - 1;
        const bool xa = __any_sync(FULL, stx != 0), ya = __any_sync(FULL, sty != 0), za = __any_sync(FULL, stz != 0);
        if (valid) {
            const SpeciesParams& P = sm.sp[s];
            const Win wx = window(o[0], stx, no[0]), wy = window(o[1], sty, no[1]), wz = window(o[2], stz, no[2]);
            const int nb = n0 + wz.off * RXY + wy.off * RX + wx.off;
            auto add = [&](int cc, int ii, int jj, int kk, int v) {
                if (dbg_in(nb + kk * RXY + jj * RX + ii, RN, err)) red_shared_nz(&sm.J32[cc][nb + kk * RXY + jj * RX + ii], v);
            };
            deposit3(add, P, wx, wy, wz, xa, ya, za);
        }
    }
}

// ------------------------------------------------------------------ tile kernel
// One CTA per tile (unit blockIdx.x).  The tile's particles are its list in the current buffer:
// species 0, then species 1, each the stay area's filled part then the immigrant area's.
template <bool DRAG>
__global__ void __launch_bounds__(NT, DRAG ? 2 : 3) push3d_kernel(const Args a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const int2 wk = a.work[blockIdx.x];
    const long long unit = blockIdx.x;
    const RunDev* Rp = &a.runs[wk.x];
    const RunConst K = run_const(Rp);
    const int nx = K.nx, ny = K.ny, nz = K.nz;
    const int tile = wk.y;
    const int tx = tile % Rp->ntx, tyz = tile / Rp->ntx;
    const int ttx = tx, tty = tyz % Rp->nty, ttz = tyz / Rp->nty;
    const int x0 = ttx * TX, y0 = tty * TY, z0 = ttz * TZ;
    const int gx0 = x0 - 1, gy0 = y0 - 1, gz0 = z0 - 1;
    const long long step = a.ctl->step;
    const int par = a.ctl->parity;
    const bool diag = a.diag_interval > 0 && (step % a.diag_interval) == 0;
    const bool anydrag = DRAG && Rp->msum[0] != nullptr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long cbase = K.cell_off;
    const unsigned lt = (1u << lane) - 1u;

    for (int i = tid; i < RN; i += NT) {
        const int rz = i / RXY, rr = i - rz * RXY, ry = rr / RX, rx = rr - ry * RX;
        const size_t g = ((size_t)wrapi(gz0 + rz, nz) * ny + wrapi(gy0 + ry, ny)) * nx + wrapi(gx0 + rx, nx);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sm.F[c][i] = Rp->E[c][g];
            sm.F[3 + c][i] = Rp->B[c][g];
            sm.J32[c][i] = 0;
            sm.J64[c][i] = 0;
        }
        if (anydrag) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                sm.ub[c][i] = Rp->ubar[c][g];
                sm.Mlo[c][i] = 0u;
                sm.Mhi[c][i] = 0;
            }
            sm.MC[i] = 0;
        }
    }
    if (tid < 5) sm.kin[tid] = 0ull;
    if (tid < 2) sm.nrs[tid] = sm.nrm[tid] = 0;
    if (tid < PIC_NS) {
        sm.sp[tid] = Rp->sp[tid];
        CellRange cr{0, 0};
        if (tid < a.nspecies && Rp->sp[tid].active) cr = cell_range(a.slot[tid][par], a.cap[tid], a.cap_stay[tid], unit);
        sm.ln[tid] = cr.n;
        sm.lns[tid] = cr.ns;
        sm.sfill[tid] = 0;
    }
    __syncthreads();

    if (diag) {
        // field energy of the tile's own cells (each cell counted by exactly one CTA)
        const int lx = tid % TX, ly = (tid / TX) % TY, lz = tid / (TX * TY);
        const int n = ((lz + 1) * RY + (ly + 1)) * RX + (lx + 1);
        double e[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const double f = sm.F[c][n];
            e[c] = f * f;
        }
#pragma unroll
        for (int c = 0; c < 6; ++c)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) e[c] += __shfl_down_sync(FULL, e[c], o);
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < 6; ++c) sm.red[warp][c] = e[c];
        __syncthreads();
        if (tid < 6) {
            double s = 0.0;
            for (int w = 0; w < NW; ++w) s += sm.red[w][tid];
            a.partials[(size_t)blockIdx.x * 8 + tid] = s;
        }
    }

    long long kacc[5] = {0, 0, 0, 0, 0};
    const int n0s = sm.ln[0], ptot = n0s + sm.ln[1];
    // Per batch: push, rebin and record (while other warps may still fold the previous batch's
    // current), barrier, deposit, barrier, fold into the int64 bank.
    for (int b0 = 0, cp = 0; b0 < ptot; b0 += BATCH, cp ^= 1) {
        // load the thread's particles of the batch (consecutive lanes: consecutive slots)
        float po[PER_THREAD][3], pu[PER_THREAD][3];
        int pid[PER_THREAD], plc[PER_THREAD], psp[PER_THREAD];
        bool pact[PER_THREAD];
#pragma unroll
        for (int r = 0; r < PER_THREAD; ++r) {
            const int p = b0 + r * NT + tid;
            pact[r] = p < ptot;
            pid[r] = 0;
            plc[r] = 0;
            psp[r] = 0;
            po[r][0] = po[r][1] = po[r][2] = 0.f;
            pu[r][0] = pu[r][1] = pu[r][2] = 0.f;
            if (pact[r]) {
                const int s = p >= n0s ? 1 : 0;
                const int e = s ? p - n0s : p;
                const int ns = sm.lns[s];
                const Slots& S = a.slot[s][par];
                const long long slot = unit * a.cap[s] + (e < ns ? e : a.cap_stay[s] + (e - ns));
                const size_t q = slot_elt(S, slot);
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    po[r][d] = S.o[d][q];
                    pu[r][d] = S.u[d][q];
                }
                if (S.id) pid[r] = S.id[q];
                plc[r] = S.lc[q];
                psp[r] = s;
            }
        }
#pragma unroll
        for (int r = 0; r < PER_THREAD; ++r) {
            const unsigned am = __ballot_sync(FULL, pact[r]);
            if (!pact[r]) continue;
            const int s = psp[r], lc = plc[r] & (CELLS - 1);
            const int lx = lc % TX, ly = (lc / TX) % TY, lz = lc / (TX * TY);
            const int ix = lx + 1, iy = ly + 1, iz = lz + 1;
            const int n0 = (iz * RY + iy) * RX + ix;
            const SpeciesParams& P = sm.sp[s];
            const int cap = a.cap[s], cst = a.cap_stay[s];
            const Slots& D = a.slot[s][par ^ 1];
            float b0v = 0.f, b1v = 0.f, b2v = 0.f;
            if (DRAG && P.drag && dbg_in(n0, RN, &a.ctl->err)) { b0v = sm.ub[0][n0]; b1v = sm.ub[1][n0]; b2v = sm.ub[2][n0]; }
            const long long g = cbase + ((long long)(z0 + lz) * ny + (y0 + ly)) * nx + (x0 + lx);
            const float df = DRAG && P.drag ? drag_of(K, P, s, g - cbase) : 0.f;
            const Pushed3 res = push3_one<DRAG>(SharedFields3{&sm, n0, &a.ctl->err}, P, K, po[r], pu[r][0], pu[r][1],
                                                pu[r][2], b0v, b1v, b2v, df, s, (unsigned)pid[r], step);
            const bool bad = res.bad;
            // destination: a bad particle stays where it was, unmoved (the sticky flag fails the run)
            const int mx = bad ? lx : lx + res.st[0], my = bad ? ly : ly + res.st[1], mz = bad ? lz : lz + res.st[2];
            const bool inside = mx >= 0 && mx < TX && my >= 0 && my < TY && mz >= 0 && mz < TZ;
            const float no[3] = {bad ? po[r][0] : res.no[0], bad ? po[r][1] : res.no[1], bad ? po[r][2] : res.no[2]};
            const float nux = bad ? pu[r][0] : res.ux, nuy = bad ? pu[r][1] : res.uy, nuz = bad ? pu[r][2] : res.uz;
            if (bad) atomicOr(&a.ctl->err, ERR_BADPART);
            // the move's deposit record: moves inside one cell from the front, the rest from the back
            const bool still = !bad && (res.st[0] | res.st[1] | res.st[2]) == 0;
            const unsigned mst = __ballot_sync(am, still), mmv = __ballot_sync(am, !bad && !still);
            int rb = 0;
            const int rl = __ffs(am) - 1;
            if (lane == rl) {
                if (mst) rb = atomicAdd(&sm.nrs[cp], __popc(mst));
                if (mmv) rb |= atomicAdd(&sm.nrm[cp], __popc(mmv)) << 16;
            }
            rb = __shfl_sync(am, rb, rl);
            if (!bad) {
                const int ri = still ? (rb & 0xffff) + __popc(mst & lt) : BATCH - 1 - ((rb >> 16) + __popc(mmv & lt));
                if (dbg_in(ri, BATCH, &a.ctl->err)) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        sm.ro[d][ri] = po[r][d];
                        sm.rn[d][ri] = res.no[d];
                    }
                    sm.rm[ri] = n0 | (s << 10) | ((res.st[0] + 1) << 11) | ((res.st[1] + 1) << 13) | ((res.st[2] + 1) << 15);
                }
                if (diag) kin_add(kacc, s, P.w, pu[r][0], pu[r][1], pu[r][2], res.ux, res.uy, res.uz);
                const int n1 = n0 + res.st[2] * RXY + res.st[1] * RX + res.st[0];
                if (DRAG && P.drag && dbg_in(n1, RN, &a.ctl->err)) {
                    add_split(&sm.Mlo[0][n1], &sm.Mhi[0][n1], f2ll_rn(res.ux * MOM_SCALE));
                    add_split(&sm.Mlo[1][n1], &sm.Mhi[1][n1], f2ll_rn(res.uy * MOM_SCALE));
                    add_split(&sm.Mlo[2][n1], &sm.Mhi[2][n1], f2ll_rn(res.uz * MOM_SCALE));
                    atomicAdd(&sm.MC[n1], 1);
                }
            }
            // particles staying in the tile: the next places of the tile's stay area (one shared
            // claim per species of the warp)
            const unsigned m0 = __ballot_sync(am, inside && s == 0), m1 = __ballot_sync(am, inside && s == 1);
            int base = 0;
            if (m0 && lane == __ffs(m0) - 1) base = atomicAdd(&sm.sfill[0], __popc(m0));
            if (m1 && lane == __ffs(m1) - 1) base = atomicAdd(&sm.sfill[1], __popc(m1));
            const int base0 = m0 ? __shfl_sync(am, base, __ffs(m0) - 1) : 0;
            const int base1 = m1 ? __shfl_sync(am, base, __ffs(m1) - 1) : 0;
            const int mlc = (mz * TY + my) * TX + mx;
            if (inside) {
                const int pos = (s ? base1 : base0) + __popc((s ? m1 : m0) & lt);
                if (pos < cst) store3(D, unit * cap + pos, no, nux, nuy, nuz, pid[r], mlc);
                else put_imm3(D, cap, cst, a.spill_cap[s], unit, mlc, g + ((long long)(mz - lz) * ny + (my - ly)) * nx + (mx - lx),
                              no, nux, nuy, nuz, pid[r], &a.ctl->err);
            } else {
                // leaving the tile: the destination tile's immigrant area (one claim per
                // destination and species among the warp's leavers)
                const int gx = wrap1(x0 + mx, nx), gy = wrap1(y0 + my, ny), gz = wrap1(z0 + mz, nz);
                const int dtx = gx / TX, dty = gy / TY, dtz = gz / TZ;
                const long long T1 = Rp->work_off + ((long long)dtz * Rp->nty + dty) * Rp->ntx + dtx;
                const int lc1 = ((gz - dtz * TZ) * TY + (gy - dty * TY)) * TX + (gx - dtx * TX);
                const long long g1 = cbase + ((long long)gz * ny + gy) * nx + gx;
                const unsigned lm = am & ~(m0 | m1);   // the warp's leavers
                const unsigned grp = __match_any_sync(lm, (long long)T1 * 2 + s);
                const int lead = __ffs(grp) - 1;
                int pi = 0;
                if (lane == lead) pi = atomicAdd(&D.icount[T1], __popc(grp));
                pi = __shfl_sync(grp, pi, lead) + __popc(grp & lt);
                put_claimed3(D, cap, cst, a.spill_cap[s], T1, pi, lc1, g1, no, nux, nuy, nuz, pid[r], &a.ctl->err);
            }
        }
        __syncthreads();
        // the other parity's counters were last read by the previous batch's deposit
        if (tid == 0) sm.nrs[cp ^ 1] = sm.nrm[cp ^ 1] = 0;
        deposit_records(sm, cp, lane, warp, &a.ctl->err);
        __syncthreads();
        // batch current -> int64 bank (the next batch's deposit starts after its first barrier)
        for (int i = tid; i < 3 * RN; i += NT) {
            int* p32 = &sm.J32[0][0] + i;
            const int v = *p32;
            if (v) {
                (&sm.J64[0][0])[i] += v;
                *p32 = 0;
            }
        }
    }
    __syncthreads();

    // stay-area fill of the tile in the next buffer
    if (tid < a.nspecies && sm.sp[tid].active) a.slot[tid][par ^ 1].count[unit] = sm.sfill[tid];

    if (diag) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            long long v = kacc[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
            if (lane == 0 && v != 0) atomicAdd(&sm.kin[k], (unsigned long long)v);
        }
        __syncthreads();
        if (tid < 5 && sm.kin[tid] != 0ull) {
            long long* Kk = a.kin + (size_t)wk.x * PIC_NS * 4;
            if (tid < 2) atomicAdd((unsigned long long*)&Kk[tid * 4], sm.kin[tid]);
            else atomicAdd((unsigned long long*)&Kk[tid - 1], sm.kin[tid]);
        }
    }

    // flush the region to global memory (halo nodes overlap neighbouring tiles: atomics)
    for (int i = tid; i < RN; i += NT) {
        const int rz = i / RXY, rr = i - rz * RXY, ry = rr / RX, rx = rr - ry * RX;
        const size_t g = ((size_t)wrapi(gz0 + rz, nz) * ny + wrapi(gy0 + ry, ny)) * nx + wrapi(gx0 + rx, nx);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long v = sm.J64[c][i];
            if (v) atomicAdd((unsigned long long*)&Rp->J[c][g], (unsigned long long)v);
        }
        if (anydrag) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const long long v = (long long)sm.Mhi[c][i] * 4096 + (long long)sm.Mlo[c][i];
                if (v) atomicAdd((unsigned long long*)&Rp->msum[c][g], (unsigned long long)v);
            }
            if (sm.MC[i]) atomicAdd(&Rp->mcnt[g], sm.MC[i]);
        }
    }
}

// Kinetic and momentum sums of spilled particles, kept per thread for its current run and
// added to the run's totals when the run changes and once at the end: per-particle atomics on
// the same five words serialised completely when filaments overflowed their cells and tens of
// millions of particles took this path.  At the end a warp whose lanes all hold the same run
// reduces in registers and adds once.
struct KinCache {
    long long v[5] = {0, 0, 0, 0, 0};
    int run = -1;
    __device__ void flush(const Args& a) {
        if (run < 0) return;
        long long* K = a.kin + (size_t)run * PIC_NS * 4;
        if (v[0]) atomicAdd((unsigned long long*)&K[0], (unsigned long long)v[0]);
        if (v[1]) atomicAdd((unsigned long long*)&K[4], (unsigned long long)v[1]);
        for (int c = 0; c < 3; ++c)
            if (v[2 + c]) atomicAdd((unsigned long long*)&K[1 + c], (unsigned long long)v[2 + c]);
        for (int c = 0; c < 5; ++c) v[c] = 0;
    }
    __device__ void use(const Args& a, int r) {
        if (r != run) { flush(a); run = r; }
    }
    // all threads of the warp call this once, after their loops
    __device__ void finish(const Args& a) {
        const int m = __reduce_max_sync(0xffffffffu, run);
        if (__all_sync(0xffffffffu, run < 0 || run == m) && m >= 0) {
            for (int c = 0; c < 5; ++c)
                for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
            run = (threadIdx.x & 31) == 0 ? m : -1;
        }
        flush(a);
    }
};

// ------------------------------------------------------------------ spilled particles
// Particles that found their cell full: one thread each, global-memory gather and atomics (the
// same formulas as the tile kernel), rebinned into the other buffer.
__global__ void __launch_bounds__(NT) spill3d_kernel(const Args a) {
    const int par = a.ctl->parity;
    const long long step = a.ctl->step;
    const bool diag = a.diag_interval > 0 && (step % a.diag_interval) == 0;
    KinCache kc;
    for (int s = 0; s < a.nspecies; ++s) {
        const Slots S = a.slot[s][par], D = a.slot[s][par ^ 1];
        const int ns = min(*S.sn, a.spill_cap[s]);
        const int cap = a.cap[s], cst = a.cap_stay[s];
        for (int k = blockIdx.x * NT + threadIdx.x; k < ns; k += gridDim.x * NT) {
            const int g = S.scell[k];
            const int run = run_of_cell(a, g);
            const RunDev* Rp = &a.runs[run];
            const int nx = Rp->nx, ny = Rp->ny, nz = Rp->nz;
            const SpeciesParams P = Rp->sp[s];
            const long long lc = g - Rp->cell_off;
            const int cz = (int)(lc / ((long long)nx * ny));
            const int rem = (int)(lc - (long long)cz * nx * ny);
            const int cy = rem / nx, cx = rem - cy * nx;
            const float o[3] = {S.so[0][k], S.so[1][k], S.so[2][k]};
            const float u0x = S.su[0][k], u0y = S.su[1][k], u0z = S.su[2][k];
            const int id = S.sid ? S.sid[k] : 0;
            float b0 = 0.f, b1 = 0.f, b2 = 0.f;
            if (P.drag) { b0 = Rp->ubar[0][lc]; b1 = Rp->ubar[1][lc]; b2 = Rp->ubar[2][lc]; }
            const RunConst K = run_const(Rp);
            const float df = P.drag ? drag_of(K, P, s, lc) : 0.f;
            const Pushed3 r = push3_one<true>(GlobalFields3{Rp, cx, cy, cz}, P, K, o, u0x, u0y, u0z, b0, b1, b2, df, s,
                                        (unsigned)id, step);
            if (r.bad) {
                atomicOr(&a.ctl->err, ERR_BADPART);
                int lcb;
                const long long Tb = unit_of_cell(a, g, &lcb);
                put_imm3(D, cap, cst, a.spill_cap[s], Tb, lcb, g, o, u0x, u0y, u0z, id, &a.ctl->err);
                continue;
            }
            if (diag) {
                kc.use(a, run);
                kin_add(kc.v, s, P.w, u0x, u0y, u0z, r.ux, r.uy, r.uz);
            }
            const Win wx = window(o[0], r.st[0], r.no[0]);
            const Win wy = window(o[1], r.st[1], r.no[1]);
            const Win wz = window(o[2], r.st[2], r.no[2]);
            const int bx = cx + wx.off, by = cy + wy.off, bz = cz + wz.off;
            auto add = [&](int c, int i, int j, int kk, int v) {
                if (v != 0) {
                    const size_t gi = ((size_t)wrapi(bz + kk, nz) * ny + wrapi(by + j, ny)) * nx + wrapi(bx + i, nx);
                    atomicAdd((unsigned long long*)&Rp->J[c][gi], (unsigned long long)(long long)v);
                }
            };
            deposit3(add, P, wx, wy, wz, true, true, true);
            const int ncx = wrap1(cx + r.st[0], nx), ncy = wrap1(cy + r.st[1], ny), ncz = wrap1(cz + r.st[2], nz);
            const long long l1 = ((long long)ncz * ny + ncy) * nx + ncx;
            if (P.drag) {
                atomicAdd((unsigned long long*)&Rp->msum[0][l1], (unsigned long long)f2ll_rn(r.ux * MOM_SCALE));
                atomicAdd((unsigned long long*)&Rp->msum[1][l1], (unsigned long long)f2ll_rn(r.uy * MOM_SCALE));
                atomicAdd((unsigned long long*)&Rp->msum[2][l1], (unsigned long long)f2ll_rn(r.uz * MOM_SCALE));
                atomicAdd(&Rp->mcnt[l1], 1);
            }
            int lc1;
            const long long T1 = unit_of_cell(a, Rp->cell_off + l1, &lc1);
            put_imm3(D, cap, cst, a.spill_cap[s], T1, lc1, Rp->cell_off + l1, r.no, r.ux, r.uy, r.uz, id, &a.ctl->err);
        }
    }
    kc.finish(a);
}

}  // namespace

bool has_push3d() { return true; }
void push3d_tile(int t[3]) { t[0] = TX; t[1] = TY; t[2] = TZ; }

cudaError_t launch_push3d(const Args& a, cudaStream_t s) {
    if (a.nwork == 0) return cudaSuccess;
    cudaError_t e = smem_attr_once((const void*)push3d_kernel<true>, (int)sizeof(Smem));
    if (e == cudaSuccess) e = smem_attr_once((const void*)push3d_kernel<false>, (int)offsetof(Smem, ub));
    if (e != cudaSuccess) return e;
    if (a.anydrag) push3d_kernel<true><<<a.nwork, NT, sizeof(Smem), s>>>(a);
    else push3d_kernel<false><<<a.nwork, NT, offsetof(Smem, ub), s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_spill3d(const Args& a, cudaStream_t s) {
    spill3d_kernel<<<152 * 8, NT, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t preload_push3d() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, push3d_kernel<true>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, push3d_kernel<false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, spill3d_kernel);
    return e;
}

}  // namespace pic
