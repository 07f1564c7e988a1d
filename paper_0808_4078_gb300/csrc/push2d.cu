// push2d.cu -- fused 2D3V particle step: CIC field gather, relativistic Boris push, Krook drag
// of the return-current electrons (Eq. (3) friction, per-cell mean-momentum relaxation), move
// with cell carry, charge-conserving Esirkepov current deposition (CIC) accumulated in int64
// fixed point, and rebinning of every particle into its new cell's slots of the other buffer.
//
// One CTA per (run, tile) of TX x TY = 256 cells (16 x 16, 32 x 8 or 8 x 32), 8 warps, 2, 3 or
// 4 CTAs per SM (the autotuner picks the variant); a warp walks its cells one at a time, each cell's species in order, 32
// particles per chunk, with the next chunk's particles loaded into registers while the current
// one is pushed.
//
// Gather: on entering a cell the warp writes a 14-entry table to shared memory: for each of the
// 13 (component, quadrant) combinations of the staggered CIC stencils, the bilinear form
// f = c0 + c1 t + c2 s + c3 t s of the component over the 2 x 2 points that bracket the quadrant
// (t, s the particle's coordinates relative to the patch), and the cell's drag mean.  A particle
// then reads 6 float4 (broadcast: the whole warp is in one cell) and evaluates each component
// with 3 FMAs instead of weighting 37 shared values.  Every path (this one, the queued crossers,
// the spill list) builds the same patches with the same roundings, so results do not depend on
// which path a particle took.
//
// Particles that stay in their cell (the large majority) add their 8 current terms and 4 drag
// moments to int32 registers (warp sums per cell put them in the shared tile) and claim slots of
// the cell's stay area in the other buffer with one shared-memory atomic per chunk.  Particles
// that cross a cell edge are queued with their pushed state in the CTA's crosser queue in global
// memory (L2-resident while the CTA runs); when the main loop is done, all threads deposit them
// with per-lane shared reductions over their 3 x 3 node window (keeping the deposit out of the
// main loop keeps its registers within the budget of 3 CTAs per SM); a crosser that stays inside
// the tile claims a slot in its new cell's stay area through the same shared counter, and only
// particles leaving the tile (or finding the stay area full) take the destination cell's
// immigrant area through a global atomic.  Crossers past the queue's capacity go to an overflow
// list that the spill kernel deposits.  The CTA writes its cells' stay counts when all this is
// done.  Every current term is an integer before it is summed, so results do not depend on
// particle order.
//
// Shared accumulators are pairs of 32-bit words (value = hi * 4096 + lo) so that all shared
// atomics are native 32-bit adds; 64-bit shared atomics are several times slower on this GPU.
// The tile is added to global int64 J with atomics at the end (halos overlap neighbours).
#include "pic_internal.cuh"
#include "particle_math.cuh"

namespace pic {
namespace {

constexpr int NT = 256, NW = NT / 32;
constexpr int FLUSH_CHUNKS = 8;          // register sums stay below 2^31 (8 x 32 particles)
constexpr int NTAB = 14;                 // 13 field patches + the drag mean of the warp's cell
constexpr unsigned FULL = 0xffffffffu;
static_assert(PIC_BLK == 32, "a chunk of 32 slots is one block of the slot arrays");

template <int TX, int TY>
struct Geo {
    static constexpr int RX = TX + 3, RY = TY + 3, RN = RX * RY, CELLS = TX * TY;
    static_assert(CELLS == 256, "a tile holds 256 cells (32 per warp)");
};

template <int TX, int TY>
struct Smem {
    static constexpr int RN = Geo<TX, TY>::RN, CELLS = Geo<TX, TY>::CELLS;
    float4 T[NW][NTAB];              // per-warp table of the cell being pushed
    double red[NW][6];
    unsigned long long kin[5];
    long long kl[5][NT];             // per-thread kinetic/momentum sums of a diagnostic step
    float* src[PIC_NS];              // block 0 of the slot arrays of the current buffer
    float* dst[PIC_NS];              // and of the other buffer
    float F[6][RN];                  // Ex Ey Ez Bx By Bz of the region (origin: tile - 1 cell)
    unsigned Jlo[3][RN];             // current accumulator, value = Jhi * 4096 + Jlo
    int Jhi[3][RN];
    unsigned Mlo[3][RN];             // drag moments (fixed point 2^20), same split
    int Mhi[3][RN];
    int MC[RN];                      // drag counts
    float ub[3][CELLS];              // previous cell-mean momentum of the tile's cells (drag)
    float df[PIC_NS][CELLS];         // drag factor 1 - exp(-nu dt) per species and cell
    int ns[PIC_NS][CELLS];           // stay part of the tile's cells (current buffer)
    int nn[PIC_NS][CELLS];           // all particles of the tile's cells (current buffer)
    int oc[PIC_NS][CELLS];           // stay-area claims in the other buffer
    int toff[16];                    // region offset of each table patch's first point
    int nq;                          // crossers queued by this CTA
    SpeciesParams sp[PIC_NS];
    Slots dslot[PIC_NS];             // slot descriptors of the other buffer
    int cap[PIC_NS], cst[PIC_NS], spc[PIC_NS];   // slots per cell, stay area, spill capacity
};


// ------------------------------------------------------------------ gather
// Bilinear patch of a component over the points (0,0), (1,0), (0,1), (1,1) of its own lattice:
// f(t, s) = c0 + c1 t + c2 s + c3 t s (x, y, z, w = c0, c1, c2, c3).
__device__ __forceinline__ float4 patch(float f00, float f10, float f01, float f11) {
    const float c1 = __fsub_rn(f10, f00), c2 = __fsub_rn(f01, f00);
    return make_float4(f00, c1, c2, __fsub_rn(__fsub_rn(f11, f10), c2));
}
__device__ __forceinline__ float peval(const float4 c, float t, float s) {
    return __fmaf_rn(t, __fmaf_rn(c.w, s, c.y), __fmaf_rn(c.z, s, c.x));
}

// Table entry e (0..12): component and the origin of its patch relative to the cell's node.
// Staggering: Ex, By at (1/2, 0); Ey, Bx at (0, 1/2); Ez at (0, 0); Bz at (1/2, 1/2).  A half-
// shifted axis has two patches, for offsets below and above 1/2 (origin -1 and 0 on that
// lattice, coordinate o + 1/2 and o - 1/2); a node axis one (origin 0, coordinate o).
//   0, 1 Ex (x half)    2, 3 By (x half)    4, 5 Ey (y half)    6, 7 Bx (y half)    8 Ez
//   9..12 Bz: 9 + [ox >= 1/2] + 2 [oy >= 1/2]
__device__ __forceinline__ void patch_origin(int e, int& c, int& dx, int& dy) {
    if (e < 4) {
        c = e < 2 ? 0 : 4; dx = (e & 1) - 1; dy = 0;
    } else if (e < 8) {
        c = e < 6 ? 1 : 3; dx = 0; dy = (e & 1) - 1;
    } else if (e == 8) {
        c = 2; dx = 0; dy = 0;
    } else {
        c = 5; dx = ((e - 9) & 1) - 1; dy = ((e - 9) >> 1) - 1;
    }
}
template <class A>
__device__ __forceinline__ float4 patch_at(const A& F, int e) {
    int c, dx, dy;
    patch_origin(e, c, dx, dy);
    return patch(F(c, dx, dy), F(c, dx + 1, dy), F(c, dx, dy + 1), F(c, dx + 1, dy + 1));
}

struct Quad {
    int qx, qy;
    float hx, hy;    // coordinates on the half-shifted lattices
};
__device__ __forceinline__ Quad quad(float ox, float oy) {
    Quad q;
    q.qx = ox >= 0.5f;
    q.qy = oy >= 0.5f;
    q.hx = __fadd_rn(ox, q.qx ? -0.5f : 0.5f);
    q.hy = __fadd_rn(oy, q.qy ? -0.5f : 0.5f);
    return q;
}
// E and B at the particle from the cell's table.
__device__ __forceinline__ void gather_tab(const float4* T, float ox, float oy, float EB[6]) {
    const Quad q = quad(ox, oy);
    const float4* ta = T + q.qx;
    const float4* tb = T + q.qy;
    EB[0] = peval(ta[0], q.hx, oy);
    EB[4] = peval(ta[2], q.hx, oy);
    EB[1] = peval(tb[4], ox, q.hy);
    EB[3] = peval(tb[6], ox, q.hy);
    EB[2] = peval(T[8], ox, oy);
    EB[5] = peval(ta[9 + 2 * q.qy], q.hx, q.hy);
}
// The same from a field accessor F(c, dx, dy) (component c at node offset (dx, dy)).
template <class A>
__device__ __forceinline__ void gather_fetch(const A& F, float ox, float oy, float EB[6]) {
    const Quad q = quad(ox, oy);
    EB[0] = peval(patch_at(F, q.qx), q.hx, oy);
    EB[4] = peval(patch_at(F, 2 + q.qx), q.hx, oy);
    EB[1] = peval(patch_at(F, 4 + q.qy), ox, q.hy);
    EB[3] = peval(patch_at(F, 6 + q.qy), ox, q.hy);
    EB[2] = peval(patch_at(F, 8), ox, oy);
    EB[5] = peval(patch_at(F, 9 + q.qx + 2 * q.qy), q.hx, q.hy);
}

template <int RX>
struct SharedFields {
    const float* F;   // region fields, component stride rn
    int rn;
    int n0;           // region index of the cell's node
    __device__ __forceinline__ float operator()(int c, int dx, int dy) const { return F[c * rn + n0 + dy * RX + dx]; }
};
struct GlobalFields {
    const RunDev* R;
    int cx, cy;
    __device__ __forceinline__ float operator()(int c, int dx, int dy) const {
        const int gi = wrapi(cx + dx, R->nx), gj = wrapi(cy + dy, R->ny);
        const float* p = c < 3 ? R->E[c] : R->B[c - 3];
        return __ldg(p + (size_t)gj * R->nx + gi);
    }
};

// Boris push, drag, collisions and move of one particle (shared by all paths).
struct Pushed {
    float ux, uy, uz;     // u^{n+1/2}
    float nox, noy;       // new offsets
    int sx, sy;           // cell steps
    float vz;
    bool bad;
};
__device__ __forceinline__ Pushed push_rest(const float EB[6], const SpeciesParams& P, const RunConst& K,
                                            float ox, float oy, float ux, float uy, float uz,
                                            float b0, float b1, float b2, float df,
                                            int s, unsigned id, long long step) {
    Pushed r;
    boris(P.qmdt2, EB, ux, uy, uz);
    if (P.drag) {
        ux = __fmaf_rn(-df, b0, ux);
        uy = __fmaf_rn(-df, b1, uy);
        uz = __fmaf_rn(-df, b2, uz);
    }
    if (P.coll) collide_ion(ux, uy, uz, P, s, id, step);
    const float ig = rsqrtf(__fmaf_rn(uz, uz, __fmaf_rn(uy, uy, __fmaf_rn(ux, ux, 1.f))));
    const float rx = __fmaf_rn(__fmul_rn(ux, ig), K.dtdx, ox);
    const float ry = __fmaf_rn(__fmul_rn(uy, ig), K.dtdy, oy);
    r.bad = !(rx > -1.f && rx < 2.f && ry > -1.f && ry < 2.f);
    carry(rx, r.nox, r.sx);
    carry(ry, r.noy, r.sy);
    r.ux = ux; r.uy = uy; r.uz = uz;
    r.vz = __fmul_rn(uz, ig);
    return r;
}

// The up-to-21 current terms of one particle, applied with `add(comp, i, j, value)`.
template <class Add>
__device__ __forceinline__ void deposit_terms(const Add& add, const SpeciesParams& P, int bi, int bj,
                                              const Win& wx, const Win& wy, float zf) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float a = __fmul_rn(P.jx, wx.C[k]);
#pragma unroll
        for (int l = 0; l < 3; ++l) add(0, bi + k, bj + l, round_small(a, wy.A[l]));
    }
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        const float a = __fmul_rn(P.jy, wy.C[l]);
#pragma unroll
        for (int k = 0; k < 3; ++k) add(1, bi + k, bj + l, round_small(a, wx.A[k]));
    }
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        const float p = zp(wy.S0[l], wy.S1[l]), q = zq(wy.S0[l], wy.S1[l]);
#pragma unroll
        for (int k = 0; k < 3; ++k) add(2, bi + k, bj + l, round_small(zf, zw(wx.S0[k], wx.S1[k], p, q)));
    }
}

// ------------------------------------------------------------------ rebinning
// Float offset of slot q >= 0 from block 0 (blocks of PIC_BLK = 32 slots, bstride floats apart):
// a 32 x 32 -> 64-bit product.
__device__ __forceinline__ size_t blk_off(int q, int bstride) {
    return (size_t)((unsigned)q >> 5) * (unsigned)bstride + ((unsigned)q & 31u);
}
// Slot q of the 2D slot arrays starting at block 0 = base: o_x, o_y, u_x, u_y, u_z[, id] are
// PIC_BLK floats apart within a block.  Stored with the evict-first policy: the next step reads
// them after gigabytes of other traffic, while the CTA's crosser queue is read back from L2
// (0.9% shorter launches at 1024^2 x 128 ppc than with default stores).
__device__ __forceinline__ void store2(float* base, int bstride, bool ids, int q, float ox, float oy,
                                       float ux, float uy, float uz, int id) {
    float* p = base + blk_off(q, bstride);
    __stcs(p, ox);
    __stcs(p + PIC_BLK, oy);
    __stcs(p + 2 * PIC_BLK, ux);
    __stcs(p + 3 * PIC_BLK, uy);
    __stcs(p + 4 * PIC_BLK, uz);
    if (ids) __stcs(reinterpret_cast<int*>(p) + 5 * PIC_BLK, id);
}
__device__ __forceinline__ void store_slot(const Slots& D, int q, float ox, float oy, float ux,
                                           float uy, float uz, int id) {
    store2(D.o[0], (int)D.bstride, D.id != nullptr, q, ox, oy, ux, uy, uz, id);
}

// Particle arriving in cell g of buffer D from another tile (or finding the stay area full):
// claim an immigrant slot, else spill.
__device__ __forceinline__ void put_imm(const Slots& D, int cap, int cap_stay, int spill_cap, int g,
                                        float ox, float oy, float ux, float uy, float uz, int id, int* err) {
    const int pi = atomicAdd(&D.icount[g], 1);
    if (pi < cap - cap_stay) {
        store_slot(D, g * cap + cap_stay + pi, ox, oy, ux, uy, uz, id);
    } else {
        const int sp = atomicAdd(D.sn, 1);
        if (sp < spill_cap) {
            D.scell[sp] = g;
            D.so[0][sp] = ox; D.so[1][sp] = oy;
            D.su[0][sp] = ux; D.su[1][sp] = uy; D.su[2][sp] = uz;
            if (D.sid) D.sid[sp] = id;
        } else {
            atomicOr(err, ERR_SPILL_FULL);
        }
    }
}

// ------------------------------------------------------------------ crossing particles
// Queue entry meta word: species (bit 0), tile cell (bits 1-10), x and y cell steps + 1 (bits
// 11-12, 13-14), bad (bit 15).  A bad particle is queued with its old state.
__device__ __forceinline__ int qmeta(int s, int ci, int sx, int sy, bool bad) {
    return s | (ci << 1) | ((sx + 1) << 11) | ((sy + 1) << 13) | ((int)bad << 15);
}

// Deposit and rebin one queued crosser of the tile (the CTA's closing phase; one per thread).
template <int TX, int TY>
__device__ __forceinline__ void cross_one(Smem<TX, TY>& sm, const Args& a, const RunConst& K, const Crosser& e,
                                          int x0, int y0) {
    constexpr int RX = Geo<TX, TY>::RX, RN = Geo<TX, TY>::RN;
    const float ox = e.o.x, oy = e.o.y, nox = e.o.z, noy = e.o.w;
    const float ux = e.u.x, uy = e.u.y, uz = e.u.z, vz = e.u.w;
    const int m = e.m.x, id = e.m.y;
    const int s = m & 1, ci = (m >> 1) & 1023, sx = ((m >> 11) & 3) - 1, sy = ((m >> 13) & 3) - 1;
    const SpeciesParams& P = sm.sp[s];
    const int lx = ci % TX, ly = ci / TX;
    const int cx = x0 + lx, cy = y0 + ly;
    const int nx = K.nx, ny = K.ny;
    const int g = K.cell_off + cy * nx + cx;
    const int cap = sm.cap[s], cst = sm.cst[s], spc = sm.spc[s];
    const Slots& D = sm.dslot[s];
    if (m & (1 << 15)) {
        // keep the particle where it was, unmoved; the sticky flag fails the run
        atomicOr(&a.ctl->err, ERR_BADPART);
        put_imm(D, cap, cst, spc, g, nox, noy, ux, uy, uz, id, &a.ctl->err);
        return;
    }
    const int ix = lx + 1, iy = ly + 1;
    const Win wx = window(ox, sx, nox), wy = window(oy, sy, noy);
    const float zf = __fmul_rn(P.jz, vz);
    auto add = [&](int c, int ii, int jj, int v) {
        if (dbg_in(jj * RX + ii, RN, &a.ctl->err))
            add_split_pred(&sm.Jlo[c][jj * RX + ii], &sm.Jhi[c][jj * RX + ii], v);
    };
    deposit_terms(add, P, ix + wx.off, iy + wy.off, wx, wy, zf);
    const int n1 = (iy + sy) * RX + (ix + sx);
    if (P.drag && dbg_in(n1, RN, &a.ctl->err)) {
        add_split_pred(&sm.Mlo[0][n1], &sm.Mhi[0][n1], f2ll_rn(ux * MOM_SCALE));
        add_split_pred(&sm.Mlo[1][n1], &sm.Mhi[1][n1], f2ll_rn(uy * MOM_SCALE));
        add_split_pred(&sm.Mlo[2][n1], &sm.Mhi[2][n1], f2ll_rn(uz * MOM_SCALE));
        atomicAdd(&sm.MC[n1], 1);
    }
    const int dlx = lx + sx, dly = ly + sy;
    if (dlx >= 0 && dlx < TX && dly >= 0 && dly < TY) {
        const int g1 = g + sy * nx + sx;
        const int pos = atomicAdd(&sm.oc[s][dly * TX + dlx], 1);
        if (pos < cst) store_slot(D, g1 * cap + pos, nox, noy, ux, uy, uz, id);
        else put_imm(D, cap, cst, spc, g1, nox, noy, ux, uy, uz, id, &a.ctl->err);
    } else {
        int ncx = cx + sx, ncy = cy + sy;
        ncx = ncx < 0 ? ncx + nx : (ncx >= nx ? ncx - nx : ncx);
        ncy = ncy < 0 ? ncy + ny : (ncy >= ny ? ncy - ny : ncy);
        put_imm(D, cap, cst, spc, K.cell_off + ncy * nx + ncx, nox, noy, ux, uy, uz, id, &a.ctl->err);
    }
}

// Register sums of "stay" particles of the cell at region node n0 -> shared tile: warp sums
// of the 12 accumulators (8 current terms, 4 drag moments when the cell has a drag species);
// lane i adds sum i.  At most 8 chunks are summed between flushes, so a warp sum of terms of at
// most 2^21 stays below 2^29.
template <int TX, int TY>
__device__ __forceinline__ void flush_acc(Smem<TX, TY>& sm, int acc[12], int n0, int lane, bool moments,
                                          int* err) {
    constexpr int RX = Geo<TX, TY>::RX, RN = Geo<TX, TY>::RN;
    int tot = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int t = __reduce_add_sync(FULL, acc[i]);
        tot = lane == i ? t : tot;
        acc[i] = 0;
    }
    if (moments) {
#pragma unroll
        for (int i = 8; i < 12; ++i) {
            const int t = __reduce_add_sync(FULL, acc[i]);
            tot = lane == i ? t : tot;
            acc[i] = 0;
        }
    }
    if (!dbg_in(n0, RN - RX - 1, err)) return;
    if (lane < 11) {
        // node offsets: Jx (0,0),(0,1); Jy (0,0),(1,0); Jz (0,0),(1,0),(0,1),(1,1); moments (0,0)
        const int off = (lane == 1 || lane == 6) ? RX : (lane == 3 || lane == 5) ? 1 : (lane == 7) ? RX + 1 : 0;
        const int c = lane < 2 ? 0 : (lane < 4 ? 1 : 2);
        unsigned* lo = lane < 8 ? &sm.Jlo[c][n0 + off] : &sm.Mlo[lane - 8][n0];
        int* hi = lane < 8 ? &sm.Jhi[c][n0 + off] : &sm.Mhi[lane - 8][n0];
        add_split_pred(lo, hi, tot);
    } else if (lane == 11) {
        red_nz(&sm.MC[n0], tot);
    }
}

// A warp's work is a sequence of segments, one per cell with particles: cells ci = warp,
// warp + NW, ...  A segment's particles are elements k = 0 .. n-1, species 0 first (k < n0), then
// species 1; element kk of species s lives in slot q0_s + kk for kk < ns_s (stay area), qi_s + kk
// beyond (immigrant area).  A chunk of 32 elements may hold both species of its cell.
struct Seg {
    int ci, n0, n;
    int ns0, ns1, q00, q01, qi0, qi1;
};
template <int TX, int TY>
__device__ __forceinline__ Seg seg_find(const Smem<TX, TY>& sm, int ci, int cell_off, int nx, int x0, int y0) {
    constexpr int CELLS = Geo<TX, TY>::CELLS;
    while (ci < CELLS && sm.nn[0][ci] + sm.nn[1][ci] == 0) ci += NW;
    Seg r;
    r.ci = ci;
    r.n0 = r.n = r.ns0 = r.ns1 = r.q00 = r.q01 = r.qi0 = r.qi1 = 0;
    if (ci < CELLS) {
        r.n0 = sm.nn[0][ci];
        r.n = r.n0 + sm.nn[1][ci];
        r.ns0 = sm.ns[0][ci];
        r.ns1 = sm.ns[1][ci];
        const int g = cell_off + (y0 + ci / TX) * nx + (x0 + ci % TX);
        r.q00 = g * sm.cap[0];
        r.q01 = g * sm.cap[1];
        r.qi0 = r.q00 + sm.cst[0] - r.ns0;
        r.qi1 = r.q01 + sm.cst[1] - r.ns1;
    }
    return r;
}

struct Part {
    float ox, oy, ux, uy, uz;
    int id;
    int s;      // species, -1 past the segment's end
    int q0;     // first slot of the cell for the particle's species
};
// The lane's particle of the chunk starting at element j of segment L (zeros past its end).
__device__ __forceinline__ Part load_part(const Seg& L, int j, int lane, float* const src[PIC_NS],
                                          int bstride, bool ids) {
    Part p;
    p.ox = p.oy = p.ux = p.uy = p.uz = 0.f;
    p.id = 0;
    p.s = -1;
    p.q0 = 0;
    const int k = j + lane;
    if (k < L.n) {
        const bool s1 = k >= L.n0;
        const int kk = s1 ? k - L.n0 : k;
        p.s = s1 ? 1 : 0;
        p.q0 = s1 ? L.q01 : L.q00;
        const int q = (kk < (s1 ? L.ns1 : L.ns0) ? p.q0 : (s1 ? L.qi1 : L.qi0)) + kk;
        const float* b = src[p.s] + blk_off(q, bstride);
        p.ox = __ldg(b);
        p.oy = __ldg(b + PIC_BLK);
        p.ux = __ldg(b + 2 * PIC_BLK);
        p.uy = __ldg(b + 3 * PIC_BLK);
        p.uz = __ldg(b + 4 * PIC_BLK);
        if (ids) p.id = __ldg(reinterpret_cast<const int*>(b) + 5 * PIC_BLK);
    }
    return p;
}

template <int TX, int TY, int MINB>
__global__ void __launch_bounds__(NT, MINB) push2d_kernel(const Args a) {
    using G = Geo<TX, TY>;
    constexpr int RX = G::RX, RN = G::RN, CELLS = G::CELLS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<TX, TY>& sm = *reinterpret_cast<Smem<TX, TY>*>(smem_raw);
    const int2 wk = a.work[blockIdx.x];
    const RunDev* Rp = &a.runs[wk.x];
    const RunConst K = run_const(Rp);
    const int nx = K.nx, ny = K.ny;
    const int tile = wk.y;
    const int ntx = Rp->ntx;
    const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
    const int gx0 = x0 - 1, gy0 = y0 - 1;
    const long long step = a.ctl->step;
    const int par = a.ctl->parity;
    const bool diag = a.diag_interval > 0 && (step % a.diag_interval) == 0;
    const bool anydrag = Rp->msum[0] != nullptr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nsp = a.nspecies;
    const int bstride = (int)a.slot[0][0].bstride;   // PIC_BLK x at most 7 arrays
    const bool ids = a.slot[0][0].id != nullptr;

    for (int i = tid; i < RN; i += NT) {
        const int ry = i / RX, rx = i - ry * RX;
        const size_t g = (size_t)wrapi(gy0 + ry, ny) * nx + wrapi(gx0 + rx, nx);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sm.F[c][i] = Rp->E[c][g];
            sm.F[3 + c][i] = Rp->B[c][g];
            sm.Jlo[c][i] = 0u;
            sm.Jhi[c][i] = 0;
        }
        if (anydrag) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                sm.Mlo[c][i] = 0u;
                sm.Mhi[c][i] = 0;
            }
            sm.MC[i] = 0;
        }
    }
    if (tid < 5) sm.kin[tid] = 0ull;
    if (tid == 0) sm.nq = 0;
    if (diag)
#pragma unroll
        for (int k = 0; k < 5; ++k) sm.kl[k][tid] = 0;
    if (tid < PIC_NS) {
        sm.sp[tid] = Rp->sp[tid];
        sm.src[tid] = a.slot[tid][par].o[0];
        sm.dst[tid] = a.slot[tid][par ^ 1].o[0];
        sm.dslot[tid] = a.slot[tid][par ^ 1];
        sm.cap[tid] = a.cap[tid];
        sm.cst[tid] = a.cap_stay[tid];
        sm.spc[tid] = a.spill_cap[tid];
    }
    if (tid >= 32 && tid < 32 + 13) {
        int c, dx, dy;
        patch_origin(tid - 32, c, dx, dy);
        sm.toff[tid - 32] = c * RN + dy * RX + dx;
    }
    for (int ci = tid; ci < CELLS; ci += NT) {
        const int lc = (y0 + ci / TX) * nx + (x0 + ci % TX);
        const int g = K.cell_off + lc;
#pragma unroll
        for (int s = 0; s < PIC_NS; ++s) {
            CellRange cr{0, 0};
            if (s < nsp && Rp->sp[s].active) cr = cell_range(a.slot[s][par], a.cap[s], a.cap_stay[s], g);
            sm.nn[s][ci] = cr.n;
            sm.ns[s][ci] = cr.ns;
            sm.oc[s][ci] = 0;
            float f = 0.f;
            if (Rp->sp[s].drag) {
                const float* m = s ? K.dmap1 : K.dmap0;
                f = m ? m[lc] : Rp->sp[s].dragf;
            }
            sm.df[s][ci] = f;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) sm.ub[c][ci] = anydrag ? Rp->ubar[c][lc] : 0.f;
    }
    __syncthreads();

    if (diag) {
        // field energy of the tile's own cells (each cell counted by exactly one CTA)
        const int i = (tid % TX) + 1, j = (tid / TX) + 1;
        double e[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const double f = sm.F[c][j * RX + i];
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

    // L: the segment the next chunk is loaded from (lj its first element); the chunk in
    // registers (nxt) is pushed in the following iteration.
    Seg L = seg_find(sm, warp, K.cell_off, nx, x0, y0);
    int lj = 0;
    Part nxt = load_part(L, 0, lane, sm.src, bstride, ids);
    int cur_ci = -1, n0 = 0, nchunk = 0;
    const bool cell_drag = anydrag;   // the tile's cells carry drag moments
    int acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = 0;
    const float4* Tw = sm.T[warp];
    const unsigned lt = (1u << lane) - 1u;
    while (L.ci < CELLS) {
        const int ci = L.ci;
        const Part p = nxt;
        lj += 32;
        if (lj >= L.n) {
            L = seg_find(sm, ci + NW, K.cell_off, nx, x0, y0);
            lj = 0;
        }
        if (L.ci < CELLS) nxt = load_part(L, lj, lane, sm.src, bstride, ids);
        if (ci != cur_ci) {
            if (nchunk) { flush_acc(sm, acc, n0, lane, cell_drag, &a.ctl->err); nchunk = 0; }
            cur_ci = ci;
            n0 = (ci / TX + 1) * RX + (ci % TX + 1);
            __syncwarp();
            if (lane < 13 && dbg_in(n0 + sm.toff[lane], 6 * RN - RX - 1, &a.ctl->err)) {
                const float* f = &sm.F[0][0] + n0 + sm.toff[lane];
                sm.T[warp][lane] = patch(f[0], f[1], f[RX], f[RX + 1]);
            } else if (lane == 13 && dbg_in(ci, CELLS, &a.ctl->err)) {
                sm.T[warp][13] = make_float4(sm.ub[0][ci], sm.ub[1][ci], sm.ub[2][ci], 0.f);
            }
            __syncwarp();
        }
        const bool act = p.s >= 0;
        const int s = act ? p.s : 0;
        const SpeciesParams& P = sm.sp[s];
        float EB[6];
        gather_tab(Tw, p.ox, p.oy, EB);
        const bool drag = P.drag;
        float b0 = 0.f, b1 = 0.f, b2 = 0.f, df = 0.f;
        if (drag) {
            const float4 d = Tw[13];
            b0 = d.x; b1 = d.y; b2 = d.z;
            df = sm.df[s][ci];
        }
        const Pushed r = push_rest(EB, P, K, p.ox, p.oy, p.ux, p.uy, p.uz, b0, b1, b2, df, s, (unsigned)p.id, step);
        if (diag && act && !r.bad) {
            long long kv[5] = {0, 0, 0, 0, 0};
            kin_add(kv, s, P.w, p.ux, p.uy, p.uz, r.ux, r.uy, r.uz);
#pragma unroll
            for (int k = 0; k < 5; ++k) sm.kl[k][tid] += kv[k];
        }
        const bool small_u = !drag || fmaxf(fabsf(r.ux), fmaxf(fabsf(r.uy), fabsf(r.uz))) < 4.f;
        const bool stay = act && !r.bad && r.sx == 0 && r.sy == 0 && small_u;
        if (stay) {
            const Win wx = window(p.ox, 0, r.nox), wy = window(p.oy, 0, r.noy);
            const float zf = __fmul_rn(P.jz, r.vz);
            const float jxa = __fmul_rn(P.jx, wx.C[0]), jya = __fmul_rn(P.jy, wy.C[0]);
            const float zp0 = zp(wy.S0[0], wy.S1[0]), zq0 = zq(wy.S0[0], wy.S1[0]);
            const float zp1 = zp(wy.S0[1], wy.S1[1]), zq1 = zq(wy.S0[1], wy.S1[1]);
            acc[0] += round_small(jxa, wy.A[0]);                          // Jx (c+1/2, c)
            acc[1] += round_small(jxa, wy.A[1]);                          // Jx (c+1/2, c+1)
            acc[2] += round_small(jya, wx.A[0]);                          // Jy (c, c+1/2)
            acc[3] += round_small(jya, wx.A[1]);                          // Jy (c+1, c+1/2)
            acc[4] += round_small(zf, zw(wx.S0[0], wx.S1[0], zp0, zq0));  // Jz (c, c)
            acc[5] += round_small(zf, zw(wx.S0[1], wx.S1[1], zp0, zq0));  // Jz (c+1, c)
            acc[6] += round_small(zf, zw(wx.S0[0], wx.S1[0], zp1, zq1));  // Jz (c, c+1)
            acc[7] += round_small(zf, zw(wx.S0[1], wx.S1[1], zp1, zq1));  // Jz (c+1, c+1)
            if (drag) {
                // |u| < 4: round_small gives rint(u 2^20), the value f2ll_rn gives on the other paths
                acc[8] += round_small(r.ux, MOM_SCALE);
                acc[9] += round_small(r.uy, MOM_SCALE);
                acc[10] += round_small(r.uz, MOM_SCALE);
                acc[11] += 1;
            }
        }
        // stayers take the next places of their cell's stay area in the other buffer (one claim
        // per species of the chunk)
        const unsigned smask0 = __ballot_sync(FULL, stay && s == 0), smask1 = __ballot_sync(FULL, stay && s == 1);
        if (smask0 | smask1) {
            int base = 0;
            if (lane == 0 && smask0) base = atomicAdd(&sm.oc[0][ci], __popc(smask0));
            if (lane == 1 && smask1) base = atomicAdd(&sm.oc[1][ci], __popc(smask1));
            const int base0 = __shfl_sync(FULL, base, 0), base1 = __shfl_sync(FULL, base, 1);
            if (stay) {
                const int pos = (s ? base1 : base0) + __popc((s ? smask1 : smask0) & lt);
                if (pos < sm.cst[s]) store2(sm.dst[s], bstride, ids, p.q0 + pos, r.nox, r.noy, r.ux, r.uy, r.uz, p.id);
                else put_imm(sm.dslot[s], sm.cap[s], sm.cst[s], sm.spc[s], p.q0 / sm.cap[s], r.nox, r.noy, r.ux,
                             r.uy, r.uz, p.id, &a.ctl->err);
            }
        }
        // the others are queued with their pushed state (bad ones with their old state) in the
        // CTA's crosser queue in global memory, deposited after the loop
        const bool defer = act && !stay;
        const unsigned dm = __ballot_sync(FULL, defer);
        if (dm) {
            int qb = 0;
            if (lane == 0) qb = atomicAdd(&sm.nq, __popc(dm));
            qb = __shfl_sync(FULL, qb, 0);
            if (defer) {
                Crosser e;
                e.o = make_float4(p.ox, p.oy, r.nox, r.noy);
                e.u = make_float4(r.ux, r.uy, r.uz, r.vz);
                e.m = make_int2(qmeta(s, ci, r.sx, r.sy, false), p.id);
                e.pad = make_int2(0, 0);
                if (r.bad) {
                    // rare: kept unmoved with its old state
                    e.o = make_float4(p.ox, p.oy, p.ox, p.oy);
                    e.u = make_float4(p.ux, p.uy, p.uz, r.vz);
                    e.m = make_int2(qmeta(s, ci, 0, 0, true), p.id);
                }
                const int k = qb + __popc(dm & lt);
                if (k < a.xq_cap) {
                    a.xq[(size_t)blockIdx.x * a.xq_cap + k] = e;
                } else {
                    // rare: past the CTA's queue, to the overflow list deposited by the spill kernel
                    const int o = atomicAdd(a.xo_n, 1);
                    if (o < a.xo_cap) {
                        a.xo[o].c = e;
                        a.xo[o].cell = p.q0 / sm.cap[s];
                    } else {
                        atomicOr(&a.ctl->err, ERR_SPILL_FULL);
                    }
                }
            }
        }
        if (++nchunk == FLUSH_CHUNKS) {
            flush_acc(sm, acc, n0, lane, cell_drag, &a.ctl->err);
            nchunk = 0;
        }
    }
    if (nchunk) flush_acc(sm, acc, n0, lane, cell_drag, &a.ctl->err);
    // the tile's crossers, one per thread
    __syncthreads();
    {
        const int nq = min(sm.nq, a.xq_cap);
        const Crosser* q = a.xq + (size_t)blockIdx.x * a.xq_cap;
        for (int i = tid; i < nq; i += NT) cross_one(sm, a, K, q[i], x0, y0);
    }

    if (diag) {
        // the threads' kinetic and momentum sums: warp sums, then the CTA's
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            long long v = sm.kl[k][tid];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
            if (lane == 0 && v != 0) atomicAdd(&sm.kin[k], (unsigned long long)v);
        }
        __syncthreads();
        if (tid < 5 && sm.kin[tid] != 0ull) {
            // Ekin per species, momentum summed into species 0's slots
            long long* Kk = a.kin + (size_t)wk.x * PIC_NS * 4;
            if (tid < 2) atomicAdd((unsigned long long*)&Kk[tid * 4], sm.kin[tid]);
            else atomicAdd((unsigned long long*)&Kk[tid - 1], sm.kin[tid]);
        }
    }
    __syncthreads();

    // stay counts of the tile's cells in the other buffer (readers clamp them to the stay area)
    for (int i = tid; i < PIC_NS * CELLS; i += NT) {
        const int s = i / CELLS, ci = i - s * CELLS;
        if (s < nsp && Rp->sp[s].active) {
            const int gg = K.cell_off + (y0 + ci / TX) * nx + (x0 + ci % TX);
            sm.dslot[s].count[gg] = sm.oc[s][ci];
        }
    }
    // flush the region to global memory (halo nodes overlap neighbouring tiles: atomics)
    for (int i = tid; i < RN; i += NT) {
        const int ry = i / RX, rx = i - ry * RX;
        const size_t gi = (size_t)wrapi(gy0 + ry, ny) * nx + wrapi(gx0 + rx, nx);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long v = (long long)sm.Jhi[c][i] * 4096 + (long long)sm.Jlo[c][i];
            if (v) atomicAdd((unsigned long long*)&Rp->J[c][gi], (unsigned long long)v);
        }
        if (anydrag) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const long long v = (long long)sm.Mhi[c][i] * 4096 + (long long)sm.Mlo[c][i];
                if (v) atomicAdd((unsigned long long*)&Rp->msum[c][gi], (unsigned long long)v);
            }
            if (sm.MC[i]) atomicAdd(&Rp->mcnt[gi], sm.MC[i]);
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
        long long* Kk = a.kin + (size_t)run * PIC_NS * 4;
        if (v[0]) atomicAdd((unsigned long long*)&Kk[0], (unsigned long long)v[0]);
        if (v[1]) atomicAdd((unsigned long long*)&Kk[4], (unsigned long long)v[1]);
        for (int c = 0; c < 3; ++c)
            if (v[2 + c]) atomicAdd((unsigned long long*)&Kk[1 + c], (unsigned long long)v[2 + c]);
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
// same formulas as the tile paths), rebinned into the other buffer.
__device__ __forceinline__ int run_of_cell(const Args& a, int g) {
    int lo = 0, hi = a.nruns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.runs[mid].cell_off <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(NT) spill2d_kernel(const Args a) {
    const int par = a.ctl->parity;
    const long long step = a.ctl->step;
    const bool diag = a.diag_interval > 0 && (step % a.diag_interval) == 0;
    // crossers past their CTA's queue (pushed and counted in the diagnostics by the particle
    // kernel): deposit with global atomics, rebin into the destination's immigrant area
    const int nxo = a.xo_n ? min(*a.xo_n, a.xo_cap) : 0;
    for (int k = blockIdx.x * NT + threadIdx.x; k < nxo; k += gridDim.x * NT) {
        const CrosserX& x = a.xo[k];
        const int g = x.cell;
        const RunDev* Rp = &a.runs[run_of_cell(a, g)];
        const int nx = Rp->nx, ny = Rp->ny;
        const int m = x.c.m.x, id = x.c.m.y;
        const int s = m & 1, sx = ((m >> 11) & 3) - 1, sy = ((m >> 13) & 3) - 1;
        const SpeciesParams P = Rp->sp[s];
        const Slots D = a.slot[s][par ^ 1];
        const int cap = a.cap[s], cst = a.cap_stay[s];
        const float ox = x.c.o.x, oy = x.c.o.y, nox = x.c.o.z, noy = x.c.o.w;
        const float ux = x.c.u.x, uy = x.c.u.y, uz = x.c.u.z, vz = x.c.u.w;
        if (m & (1 << 15)) {
            atomicOr(&a.ctl->err, ERR_BADPART);
            put_imm(D, cap, cst, a.spill_cap[s], g, nox, noy, ux, uy, uz, id, &a.ctl->err);
            continue;
        }
        const int lc = g - Rp->cell_off;
        const int cy = lc / nx, cx = lc - cy * nx;
        const Win wx = window(ox, sx, nox), wy = window(oy, sy, noy);
        const float zf = __fmul_rn(P.jz, vz);
        auto add = [&](int c, int i, int j, int v) {
            if (v != 0)
                atomicAdd((unsigned long long*)&Rp->J[c][(size_t)wrapi(j, ny) * nx + wrapi(i, nx)],
                          (unsigned long long)(long long)v);
        };
        deposit_terms(add, P, cx + wx.off, cy + wy.off, wx, wy, zf);
        int ncx = cx + sx, ncy = cy + sy;
        ncx = ncx < 0 ? ncx + nx : (ncx >= nx ? ncx - nx : ncx);
        ncy = ncy < 0 ? ncy + ny : (ncy >= ny ? ncy - ny : ncy);
        const int l1 = ncy * nx + ncx;
        if (P.drag) {
            atomicAdd((unsigned long long*)&Rp->msum[0][l1], (unsigned long long)f2ll_rn(ux * MOM_SCALE));
            atomicAdd((unsigned long long*)&Rp->msum[1][l1], (unsigned long long)f2ll_rn(uy * MOM_SCALE));
            atomicAdd((unsigned long long*)&Rp->msum[2][l1], (unsigned long long)f2ll_rn(uz * MOM_SCALE));
            atomicAdd(&Rp->mcnt[l1], 1);
        }
        put_imm(D, cap, cst, a.spill_cap[s], Rp->cell_off + l1, nox, noy, ux, uy, uz, id, &a.ctl->err);
    }
    KinCache kc;
    for (int s = 0; s < a.nspecies; ++s) {
        const Slots S = a.slot[s][par], D = a.slot[s][par ^ 1];
        const int ns = min(*S.sn, a.spill_cap[s]);
        const int cap = a.cap[s], cst = a.cap_stay[s];
        for (int k = blockIdx.x * NT + threadIdx.x; k < ns; k += gridDim.x * NT) {
            const int g = S.scell[k];
            const int run = run_of_cell(a, g);
            const RunDev* Rp = &a.runs[run];
            const int nx = Rp->nx, ny = Rp->ny;
            const SpeciesParams P = Rp->sp[s];
            const int lc = g - Rp->cell_off;
            const int cy = lc / nx, cx = lc - cy * nx;
            const float ox = S.so[0][k], oy = S.so[1][k];
            const float u0x = S.su[0][k], u0y = S.su[1][k], u0z = S.su[2][k];
            const int id = S.sid ? S.sid[k] : 0;
            float b0 = 0.f, b1 = 0.f, b2 = 0.f;
            if (P.drag) { b0 = Rp->ubar[0][lc]; b1 = Rp->ubar[1][lc]; b2 = Rp->ubar[2][lc]; }
            const RunConst K = run_const(Rp);
            const float df = P.drag ? drag_of(K, P, s, lc) : 0.f;
            float EB[6];
            gather_fetch(GlobalFields{Rp, cx, cy}, ox, oy, EB);
            const Pushed r = push_rest(EB, P, K, ox, oy, u0x, u0y, u0z, b0, b1, b2, df, s, (unsigned)id, step);
            if (r.bad) {
                atomicOr(&a.ctl->err, ERR_BADPART);
                put_imm(D, cap, cst, a.spill_cap[s], g, ox, oy, u0x, u0y, u0z, id, &a.ctl->err);
                continue;
            }
            if (diag) {
                kc.use(a, run);
                kin_add(kc.v, s, P.w, u0x, u0y, u0z, r.ux, r.uy, r.uz);
            }
            const Win wx = window(ox, r.sx, r.nox), wy = window(oy, r.sy, r.noy);
            const float zf = __fmul_rn(P.jz, r.vz);
            auto add = [&](int c, int i, int j, int v) {
                if (v != 0)
                    atomicAdd((unsigned long long*)&Rp->J[c][(size_t)wrapi(j, ny) * nx + wrapi(i, nx)],
                              (unsigned long long)(long long)v);
            };
            deposit_terms(add, P, cx + wx.off, cy + wy.off, wx, wy, zf);
            int ncx = cx + r.sx, ncy = cy + r.sy;
            ncx = ncx < 0 ? ncx + nx : (ncx >= nx ? ncx - nx : ncx);
            ncy = ncy < 0 ? ncy + ny : (ncy >= ny ? ncy - ny : ncy);
            const int l1 = ncy * nx + ncx;
            if (P.drag) {
                atomicAdd((unsigned long long*)&Rp->msum[0][l1], (unsigned long long)f2ll_rn(r.ux * MOM_SCALE));
                atomicAdd((unsigned long long*)&Rp->msum[1][l1], (unsigned long long)f2ll_rn(r.uy * MOM_SCALE));
                atomicAdd((unsigned long long*)&Rp->msum[2][l1], (unsigned long long)f2ll_rn(r.uz * MOM_SCALE));
                atomicAdd(&Rp->mcnt[l1], 1);
            }
            const int g1 = Rp->cell_off + l1;
            put_imm(D, cap, cst, a.spill_cap[s], g1, r.nox, r.noy, r.ux, r.uy, r.uz, id, &a.ctl->err);
        }
    }
    kc.finish(a);
}

// ------------------------------------------------------------------ variants and launch
// Compiled variants of the particle kernel: tile shape and CTAs per SM (the register budget).
struct Variant {
    void (*fn)(Args);
    int tx, ty, minb;
    size_t smem;
};
template <int TX, int TY, int MINB>
constexpr Variant make_variant() {
    return Variant{push2d_kernel<TX, TY, MINB>, TX, TY, MINB, sizeof(Smem<TX, TY>)};
}
const Variant kVariants[] = {
    make_variant<16, 16, 3>(), make_variant<16, 16, 2>(), make_variant<16, 16, 4>(),
    make_variant<32, 8, 3>(),  make_variant<32, 8, 2>(),  make_variant<32, 8, 4>(),
    make_variant<8, 32, 3>(),  make_variant<8, 32, 2>(),  make_variant<8, 32, 4>(),
};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);


}  // namespace

// Index of the compiled variant for a tile shape and CTAs per SM (minb 0: the default, 3 CTAs
// per SM with 80 registers), or -1.
int push2d_variant(int tx, int ty, int minb) {
    for (int v = 0; v < kNumVariants; ++v)
        if (kVariants[v].tx == tx && kVariants[v].ty == ty && kVariants[v].minb == (minb == 0 ? 3 : minb))
            return v;
    return -1;
}
int push2d_num_variants() { return kNumVariants; }
void push2d_variant_info(int v, int* tx, int* ty, int* minb) {
    *tx = kVariants[v].tx;
    *ty = kVariants[v].ty;
    *minb = kVariants[v].minb;
}

cudaError_t launch_push2d(const Args& a, cudaStream_t s) {
    if (a.nwork == 0) return cudaSuccess;
    const int v = a.push_variant;
    if (v < 0 || v >= kNumVariants || kVariants[v].tx != a.tx || kVariants[v].ty != a.ty) return cudaErrorInvalidValue;
    cudaError_t e = smem_attr_once((const void*)kVariants[v].fn, (int)kVariants[v].smem);
    if (e != cudaSuccess) return e;
    kVariants[v].fn<<<a.nwork, NT, kVariants[v].smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t preload_push2d() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, spill2d_kernel);
    for (int v = 0; v < kNumVariants && e == cudaSuccess; ++v) e = cudaFuncGetAttributes(&fa, kVariants[v].fn);
    return e;
}

cudaError_t launch_spill2d(const Args& a, cudaStream_t s) {
    spill2d_kernel<<<152 * 8, NT, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pic
