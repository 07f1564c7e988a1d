// push2d.cu -- fused 2D3V particle step: CIC field gather, relativistic Boris push, Krook drag
// of the return-current electrons (Eq. (3) friction, per-cell mean-momentum relaxation), move
// with cell carry, charge-conserving Esirkepov current deposition (CIC) accumulated in int64
// fixed point, and rebinning of every particle into its new cell's slots of the other buffer.
//
// One CTA per (run, tile) of 16 x 16 cells, 8 warps, a warp per cell, 3 CTAs per SM (80
// registers: the fields are read from the shared tile, not cached in registers, which buys the
// third CTA).  Particles that stay in the cell this step (the large majority) add their 8
// current terms and 4 drag moments to int32 registers (one warp transpose-reduce per cell puts
// them in the shared tile) and are written to the cell's new stay slots at warp-local offsets
// (no atomics).  Particles that cross
// a cell edge go to a per-warp queue and are processed 32 at a time: per-lane atomics over their
// 3 x 3 node window, and an atomic slot claim in the destination cell.  All paths evaluate the
// same explicitly-rounded formulas and every current term is an integer before it is summed, so
// results do not depend on particle order.
//
// Shared accumulators are pairs of 32-bit words (value = hi * 4096 + lo) so that all shared
// atomics are native 32-bit adds; 64-bit shared atomics are several times slower on this GPU.
// The tile is added to global int64 J with atomics at the end (halos overlap neighbours).
#include "pic_internal.cuh"
#include "particle_math.cuh"

namespace pic {
namespace {

constexpr int TX = 16, TY = 16;
constexpr int RX = TX + 3, RY = TY + 3, RN = RX * RY;   // tile + CIC/Esirkepov stencil halo
constexpr int NT = 256, NW = NT / 32, QCAP = 64;
constexpr int CELLS = TX * TY;
constexpr int FLUSH_CHUNKS = 8;          // register sums stay below 2^31 (8 x 32 particles)
constexpr int STAGES = 4;                // per-warp cp.async pipeline depth (chunks in flight)
constexpr unsigned FULL = 0xffffffffu;

struct Smem {
    float F[6][RN];                  // Ex Ey Ez Bx By Bz of the region (origin: tile - 1 cell)
    float ub[3][RN];                 // previous cell-mean momentum (drag)
    unsigned Jlo[3][RN];             // current accumulator, value = Jhi * 4096 + Jlo
    int Jhi[3][RN];
    unsigned Mlo[3][RN];             // drag moments (fixed point 2^20), same split
    int Mhi[3][RN];
    int MC[RN];                      // drag counts
    unsigned q[NW][QCAP];            // per-warp queue: species << 24 | tile cell << 16 | slot
    float stg[NW][STAGES][6][32];    // per-warp staged chunks: o0 o1 u0 u1 u2 id (by lane)
    int cnt[PIC_NS][CELLS];          // particles of the tile's cells (current buffer)
    int cns[PIC_NS][CELLS];          // of which in the stay area
    double red[NW][6];
    unsigned long long kin[5];
    SpeciesParams sp[PIC_NS];
};

// ------------------------------------------------------------------ async staging
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Position in a warp's work list: its cells ci = warp, warp + NW, ...; per cell the species in
// order; per species chunks of 32 slots.
struct Cursor {
    int ci, s, j;
};
__device__ __forceinline__ void advance(Cursor& c, const int (*cnt)[CELLS], int nsp) {
    c.j += 32;
    while (c.ci < CELLS) {
        if (c.j < cnt[c.s][c.ci]) return;
        c.j = 0;
        if (++c.s >= nsp) { c.s = 0; c.ci += NW; }
    }
}

// Slot of element k of cell g (32-bit: the library keeps cells x cap below 2^31).
__device__ __forceinline__ int slot32(int g, int cap, int cap_stay, int ns, int k) {
    return g * cap + (k < ns ? k : cap_stay + (k - ns));
}

// ------------------------------------------------------------------ gather
// CIC weights of an axis for an offset o in [0,1): node lattice (nodes c, c+1) and the
// half-shifted lattice (points c-1/2, c+1/2, c+3/2, stored at c-1, c, c+1).
struct W3 {
    float n[2];
    float h[3];
};
__device__ __forceinline__ W3 weights(float o) {
    W3 w;
    const float d = __fsub_rn(o, 0.5f);
    w.n[0] = __fsub_rn(1.f, o);
    w.n[1] = o;
    w.h[0] = fmaxf(-d, 0.f);
    w.h[1] = __fsub_rn(1.f, fabsf(d));
    w.h[2] = fmaxf(d, 0.f);
    return w;
}

// F(c, dx, dy): component c at offset (dx, dy) from the particle's cell node.
template <class A>
__device__ __forceinline__ float row_h(const A& F, const W3& wx, int c, int dy) {
    return __fmaf_rn(wx.h[2], F(c, 1, dy), __fmaf_rn(wx.h[1], F(c, 0, dy), __fmul_rn(wx.h[0], F(c, -1, dy))));
}
template <class A>
__device__ __forceinline__ float row_n(const A& F, const W3& wx, int c, int dy) {
    return __fmaf_rn(wx.n[1], F(c, 1, dy), __fmul_rn(wx.n[0], F(c, 0, dy)));
}
// Staggering: Ex, By (1/2, 0); Ey, Bx (0, 1/2); Ez (0, 0); Bz (1/2, 1/2).
template <class A>
__device__ __forceinline__ void gather(const A& F, const W3& wx, const W3& wy, float EB[6]) {
    EB[0] = __fmaf_rn(wy.n[1], row_h(F, wx, 0, 1), __fmul_rn(wy.n[0], row_h(F, wx, 0, 0)));
    EB[4] = __fmaf_rn(wy.n[1], row_h(F, wx, 4, 1), __fmul_rn(wy.n[0], row_h(F, wx, 4, 0)));
    EB[1] = __fmaf_rn(wy.h[2], row_n(F, wx, 1, 1), __fmaf_rn(wy.h[1], row_n(F, wx, 1, 0), __fmul_rn(wy.h[0], row_n(F, wx, 1, -1))));
    EB[3] = __fmaf_rn(wy.h[2], row_n(F, wx, 3, 1), __fmaf_rn(wy.h[1], row_n(F, wx, 3, 0), __fmul_rn(wy.h[0], row_n(F, wx, 3, -1))));
    EB[2] = __fmaf_rn(wy.n[1], row_n(F, wx, 2, 1), __fmul_rn(wy.n[0], row_n(F, wx, 2, 0)));
    EB[5] = __fmaf_rn(wy.h[2], row_h(F, wx, 5, 1), __fmaf_rn(wy.h[1], row_h(F, wx, 5, 0), __fmul_rn(wy.h[0], row_h(F, wx, 5, -1))));
}

struct SharedFields {
    const Smem* s;
    int n0;   // region index of the particle's cell node
    __device__ __forceinline__ float operator()(int c, int dx, int dy) const {
        return s->F[c][n0 + dy * RX + dx];
    }
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

// Warp sum of 16 int values; lane l returns the total of value index l >> 1.
__device__ __forceinline__ int transpose_reduce16(int v[16], int lane) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const bool hi = lane & 16;
        const int send = hi ? v[i] : v[i + 8];
        const int keep = hi ? v[i + 8] : v[i];
        v[i] = keep + __shfl_xor_sync(FULL, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool hi = lane & 8;
        const int send = hi ? v[i] : v[i + 4];
        const int keep = hi ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(FULL, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool hi = lane & 4;
        const int send = hi ? v[i] : v[i + 2];
        const int keep = hi ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(FULL, send, 4);
    }
    {
        const bool hi = lane & 2;
        const int send = hi ? v[0] : v[1];
        const int keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(FULL, send, 2);
    }
    return v[0] + __shfl_xor_sync(FULL, v[0], 1);
}

struct Pushed {
    float ux, uy, uz;     // u^{n+1/2}
    float nox, noy;       // new offsets
    int sx, sy;           // cell steps
    float vz;
    bool bad;
};

template <class A>
__device__ __forceinline__ Pushed push_one(const A& F, const SpeciesParams& P, const RunConst& K,
                                           float ox, float oy, float ux, float uy, float uz,
                                           float b0, float b1, float b2, float df,
                                           int s, unsigned id, long long step) {
    Pushed r;
    const W3 wx = weights(ox), wy = weights(oy);
    float EB[6];
    gather(F, wx, wy, EB);
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
__device__ __forceinline__ void store_slot(const Slots& D, int q, float ox, float oy, float ux,
                                           float uy, float uz, int id) {
    D.o[0][q] = ox; D.o[1][q] = oy;
    D.u[0][q] = ux; D.u[1][q] = uy; D.u[2][q] = uz;
    if (D.id) D.id[q] = id;
}

// Particle arriving in cell g of buffer D from elsewhere: claim an immigrant slot, else spill.
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
// Full step of up to 32 queued particles (one per lane) of the tile: shared-memory gather and
// deposit, then rebinning into the destination cell of the other buffer.
__device__ __forceinline__ void drain(Smem& sm, const Args& a, const RunConst& K, int par, int k,
                                      int lane, int warp, int x0, int y0, bool diag, long long step,
                                      long long kacc[5]) {
    if (lane >= k) return;
    const int nx = K.nx, ny = K.ny;
    const unsigned e = sm.q[warp][lane];
    const int s = e >> 24, ci = (e >> 16) & 255, i = e & 65535;
    const SpeciesParams& P = sm.sp[s];
    const int lx = ci % TX, ly = ci / TX;
    const int cx = x0 + lx, cy = y0 + ly;
    const int g = K.cell_off + cy * nx + cx;
    const int cap = a.cap[s], cst = a.cap_stay[s];
    const Slots S = a.slot[s][par], D = a.slot[s][par ^ 1];
    const int p = slot32(g, cap, cst, sm.cns[s][ci], i);
    const float ox = S.o[0][p], oy = S.o[1][p];
    const float u0x = S.u[0][p], u0y = S.u[1][p], u0z = S.u[2][p];
    const int id = S.id ? S.id[p] : 0;
    const int ix = lx + 1, iy = ly + 1;
    const int n0 = iy * RX + ix;
    float b0 = 0.f, b1 = 0.f, b2 = 0.f;
    if (P.drag) { b0 = sm.ub[0][n0]; b1 = sm.ub[1][n0]; b2 = sm.ub[2][n0]; }
    const float df = P.drag ? drag_of(K, P, s, g - K.cell_off) : 0.f;
    const Pushed r = push_one(SharedFields{&sm, n0}, P, K, ox, oy, u0x, u0y, u0z, b0, b1, b2, df, s, id, step);
    if (r.bad) {
        // keep the particle where it was, unmoved; the sticky flag fails the run
        atomicOr(&a.ctl->err, ERR_BADPART);
        put_imm(D, cap, cst, a.spill_cap[s], g, ox, oy, u0x, u0y, u0z, id, &a.ctl->err);
        return;
    }
    if (diag) kin_add(kacc, s, P.w, u0x, u0y, u0z, r.ux, r.uy, r.uz);
    const Win wx = window(ox, r.sx, r.nox), wy = window(oy, r.sy, r.noy);
    const float zf = __fmul_rn(P.jz, r.vz);
    auto add = [&](int c, int ii, int jj, int v) {
        if (v != 0) add_split(&sm.Jlo[c][jj * RX + ii], &sm.Jhi[c][jj * RX + ii], v);
    };
    deposit_terms(add, P, ix + wx.off, iy + wy.off, wx, wy, zf);
    if (P.drag) {
        const int n1 = (iy + r.sy) * RX + (ix + r.sx);
        add_split(&sm.Mlo[0][n1], &sm.Mhi[0][n1], f2ll_rn(r.ux * MOM_SCALE));
        add_split(&sm.Mlo[1][n1], &sm.Mhi[1][n1], f2ll_rn(r.uy * MOM_SCALE));
        add_split(&sm.Mlo[2][n1], &sm.Mhi[2][n1], f2ll_rn(r.uz * MOM_SCALE));
        atomicAdd(&sm.MC[n1], 1);
    }
    int ncx = cx + r.sx, ncy = cy + r.sy;
    ncx = ncx < 0 ? ncx + nx : (ncx >= nx ? ncx - nx : ncx);
    ncy = ncy < 0 ? ncy + ny : (ncy >= ny ? ncy - ny : ncy);
    const int g1 = K.cell_off + ncy * nx + ncx;
    put_imm(D, cap, cst, a.spill_cap[s], g1, r.nox, r.noy, r.ux, r.uy, r.uz, id, &a.ctl->err);
}

// Register sums of "stay" particles of the cell at region node n0 -> shared tile.
__device__ __forceinline__ void flush_acc(Smem& sm, int acc[12], int n0, int lane) {
    int v[16];
#pragma unroll
    for (int i = 0; i < 12; ++i) { v[i] = acc[i]; acc[i] = 0; }
    v[12] = v[13] = v[14] = v[15] = 0;
    const int tot = transpose_reduce16(v, lane);
    const int idx = lane >> 1;
    if ((lane & 1) || tot == 0 || idx > 11) return;
    if (idx == 11) { atomicAdd(&sm.MC[n0], tot); return; }
    // node offsets: Jx (0,0),(0,1); Jy (0,0),(1,0); Jz (0,0),(1,0),(0,1),(1,1); moments (0,0)
    const int off = (idx == 1 || idx == 6) ? RX : (idx == 3 || idx == 5) ? 1 : (idx == 7) ? RX + 1 : 0;
    unsigned* lo;
    int* hi;
    if (idx < 8) {
        const int c = idx < 2 ? 0 : (idx < 4 ? 1 : 2);
        lo = &sm.Jlo[c][n0 + off];
        hi = &sm.Jhi[c][n0 + off];
    } else {
        lo = &sm.Mlo[idx - 8][n0];
        hi = &sm.Mhi[idx - 8][n0];
    }
    add_split(lo, hi, tot);
}

__global__ void __launch_bounds__(NT, 3) push2d_kernel(const Args a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const int2 wk = a.work[blockIdx.x];
    const RunDev* Rp = &a.runs[wk.x];
    const RunConst K = run_const(Rp);
    const int nx = K.nx, ny = K.ny;
    const int tile = wk.y;
    const int x0 = (tile % Rp->ntx) * TX, y0 = (tile / Rp->ntx) * TY;
    const int gx0 = x0 - 1, gy0 = y0 - 1;
    const long long step = a.ctl->step;
    const int par = a.ctl->parity;
    const bool diag = a.diag_interval > 0 && (step % a.diag_interval) == 0;
    const bool anydrag = Rp->msum[0] != nullptr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;

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
                sm.ub[c][i] = Rp->ubar[c][g];
                sm.Mlo[c][i] = 0u;
                sm.Mhi[c][i] = 0;
            }
            sm.MC[i] = 0;
        }
    }
    if (tid < 5) sm.kin[tid] = 0ull;
    if (tid < PIC_NS) sm.sp[tid] = Rp->sp[tid];
    for (int i = tid; i < PIC_NS * CELLS; i += NT) {
        const int s = i / CELLS, ci = i - s * CELLS;
        const int g = K.cell_off + (y0 + ci / TX) * nx + (x0 + ci % TX);
        CellRange cr{0, 0};
        if (s < a.nspecies && Rp->sp[s].active) cr = cell_range(a.slot[s][par], a.cap[s], a.cap_stay[s], g);
        sm.cnt[s][ci] = cr.n;
        sm.cns[s][ci] = cr.ns;
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

    long long kacc[5] = {0, 0, 0, 0, 0};
    int qn = 0;
    const int nsp = a.nspecies;
    // issue the asynchronous copies of one chunk into stage st
    auto issue = [&](const Cursor& c, int st) {
        if (c.ci < CELLS) {
            const int i = c.j + lane;
            if (i < sm.cnt[c.s][c.ci]) {
                const int lx = c.ci % TX, ly = c.ci / TX;
                const int g = K.cell_off + (y0 + ly) * nx + (x0 + lx);
                const Slots S = a.slot[c.s][par];
                const int q = slot32(g, a.cap[c.s], a.cap_stay[c.s], sm.cns[c.s][c.ci], i);
                cp_async4(&sm.stg[warp][st][0][lane], S.o[0] + q);
                cp_async4(&sm.stg[warp][st][1][lane], S.o[1] + q);
                cp_async4(&sm.stg[warp][st][2][lane], S.u[0] + q);
                cp_async4(&sm.stg[warp][st][3][lane], S.u[1] + q);
                cp_async4(&sm.stg[warp][st][4][lane], S.u[2] + q);
                if (S.id) cp_async4(&sm.stg[warp][st][5][lane], S.id + q);
            }
        }
        cp_async_commit();
    };
    Cursor fc{warp, 0, -32};
    advance(fc, sm.cnt, nsp);
    Cursor pc = fc;
#pragma unroll
    for (int k = 0; k < STAGES - 1; ++k) {
        issue(fc, k);
        advance(fc, sm.cnt, nsp);
    }
    int st = 0;
    int cur_ci = -1, n0 = 0, g = 0, nchunk = 0;
    int seg_s = -1, seg_g = 0, wpos = 0;     // stay-area fill of the current (cell, species)
    int acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = 0;
    float ub0 = 0.f, ub1 = 0.f, ub2 = 0.f;
    while (pc.ci < CELLS) {
        issue(fc, (st + STAGES - 1) % STAGES);
        advance(fc, sm.cnt, nsp);
        if (pc.ci != cur_ci) {
            if (nchunk) { flush_acc(sm, acc, n0, lane); nchunk = 0; }
            cur_ci = pc.ci;
            const int lx = cur_ci % TX, ly = cur_ci / TX;
            g = K.cell_off + (y0 + ly) * nx + (x0 + lx);
            n0 = (ly + 1) * RX + (lx + 1);
            if (anydrag) { ub0 = sm.ub[0][n0]; ub1 = sm.ub[1][n0]; ub2 = sm.ub[2][n0]; }
        }
        const int s = pc.s;
        const SpeciesParams& P = sm.sp[s];
        const int cap = a.cap[s], cst = a.cap_stay[s];
        const Slots D = a.slot[s][par ^ 1];
        if (pc.j == 0) {
            // new (cell, species): record the previous one's stay count
            if (seg_s >= 0 && lane == 0) a.slot[seg_s][par ^ 1].count[seg_g] = wpos;
            seg_s = s;
            seg_g = g;
            wpos = 0;
        }
        const int i = pc.j + lane;
        const bool act = i < sm.cnt[s][pc.ci];
        cp_async_wait<STAGES - 1>();
        float ox = 0.f, oy = 0.f, ux = 0.f, uy = 0.f, uz = 0.f;
        int id = 0;
        if (act) {
            ox = sm.stg[warp][st][0][lane]; oy = sm.stg[warp][st][1][lane];
            ux = sm.stg[warp][st][2][lane]; uy = sm.stg[warp][st][3][lane]; uz = sm.stg[warp][st][4][lane];
            id = __float_as_int(sm.stg[warp][st][5][lane]);
        }
        const float df = P.drag ? drag_of(K, P, s, g - K.cell_off) : 0.f;
        const Pushed r = push_one(SharedFields{&sm, n0}, P, K, ox, oy, ux, uy, uz, ub0, ub1, ub2, df, s, (unsigned)id, step);
        const bool small_u = !P.drag || (fabsf(r.ux) < 4.f && fabsf(r.uy) < 4.f && fabsf(r.uz) < 4.f);
        const bool stay = act && !r.bad && r.sx == 0 && r.sy == 0 && small_u;
        if (stay) {
            const Win wx = window(ox, 0, r.nox), wy = window(oy, 0, r.noy);
            const float zf = __fmul_rn(P.jz, r.vz);
            const float jxa = __fmul_rn(P.jx, wx.C[0]), jya = __fmul_rn(P.jy, wy.C[0]);
            const float p0 = zp(wy.S0[0], wy.S1[0]), q0 = zq(wy.S0[0], wy.S1[0]);
            const float p1 = zp(wy.S0[1], wy.S1[1]), q1 = zq(wy.S0[1], wy.S1[1]);
            acc[0] += round_small(jxa, wy.A[0]);                          // Jx (c+1/2, c)
            acc[1] += round_small(jxa, wy.A[1]);                          // Jx (c+1/2, c+1)
            acc[2] += round_small(jya, wx.A[0]);                          // Jy (c, c+1/2)
            acc[3] += round_small(jya, wx.A[1]);                          // Jy (c+1, c+1/2)
            acc[4] += round_small(zf, zw(wx.S0[0], wx.S1[0], p0, q0));    // Jz (c, c)
            acc[5] += round_small(zf, zw(wx.S0[1], wx.S1[1], p0, q0));    // Jz (c+1, c)
            acc[6] += round_small(zf, zw(wx.S0[0], wx.S1[0], p1, q1));    // Jz (c, c+1)
            acc[7] += round_small(zf, zw(wx.S0[1], wx.S1[1], p1, q1));    // Jz (c+1, c+1)
            if (P.drag) {
                acc[8] += __float2int_rn(r.ux * MOM_SCALE);
                acc[9] += __float2int_rn(r.uy * MOM_SCALE);
                acc[10] += __float2int_rn(r.uz * MOM_SCALE);
                acc[11] += 1;
            }
            if (diag) kin_add(kacc, s, P.w, ux, uy, uz, r.ux, r.uy, r.uz);
        }
        // stayers keep their cell: the next free places of its stay area in the other buffer
        const unsigned sm_ = __ballot_sync(FULL, stay);
        if (stay) {
            const int pos = wpos + __popc(sm_ & lt);
            if (pos < cst) store_slot(D, g * cap + pos, r.nox, r.noy, r.ux, r.uy, r.uz, id);
            else put_imm(D, cap, cst, a.spill_cap[s], g, r.nox, r.noy, r.ux, r.uy, r.uz, id, &a.ctl->err);
        }
        wpos += __popc(sm_);
        const bool defer = act && !stay;
        const unsigned dm = __ballot_sync(FULL, defer);
        if (defer) sm.q[warp][qn + __popc(dm & lt)] = ((unsigned)s << 24) | ((unsigned)pc.ci << 16) | (unsigned)i;
        qn += __popc(dm);
        __syncwarp();
        if (qn >= 32) {
            drain(sm, a, K, par, 32, lane, warp, x0, y0, diag, step, kacc);
            __syncwarp();
            const int rest = qn - 32;
            const unsigned moved = lane < rest ? sm.q[warp][32 + lane] : 0u;
            __syncwarp();
            if (lane < rest) sm.q[warp][lane] = moved;
            __syncwarp();
            qn = rest;
        }
        if (++nchunk == FLUSH_CHUNKS) {
            flush_acc(sm, acc, n0, lane);
            nchunk = 0;
        }
        advance(pc, sm.cnt, nsp);
        st = (st + 1) % STAGES;
    }
    if (nchunk) flush_acc(sm, acc, n0, lane);
    if (seg_s >= 0 && lane == 0) a.slot[seg_s][par ^ 1].count[seg_g] = wpos;
    cp_async_wait<0>();
    if (qn > 0) drain(sm, a, K, par, qn, lane, warp, x0, y0, diag, step, kacc);
    __syncwarp();

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
            // Ekin per species, momentum summed into species 0's slots
            long long* K = a.kin + (size_t)wk.x * PIC_NS * 4;
            if (tid < 2) atomicAdd((unsigned long long*)&K[tid * 4], sm.kin[tid]);
            else atomicAdd((unsigned long long*)&K[tid - 1], sm.kin[tid]);
        }
    }
    __syncthreads();

    // flush the region to global memory (halo nodes overlap neighbouring tiles: atomics)
    for (int i = tid; i < RN; i += NT) {
        const int ry = i / RX, rx = i - ry * RX;
        const size_t g = (size_t)wrapi(gy0 + ry, ny) * nx + wrapi(gx0 + rx, nx);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long v = (long long)sm.Jhi[c][i] * 4096 + (long long)sm.Jlo[c][i];
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
// same formulas as the tile paths), rebinned into the other buffer.
__global__ void __launch_bounds__(NT) spill2d_kernel(const Args a) {
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
            int lo = 0, hi = a.nruns - 1;       // run holding cell g
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.runs[mid].cell_off <= g) lo = mid; else hi = mid - 1;
            }
            const int run = lo;
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
            const Pushed r = push_one(GlobalFields{Rp, cx, cy}, P, K, ox, oy, u0x, u0y, u0z, b0, b1, b2, df, s,
                                      (unsigned)id, step);
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

}  // namespace

cudaError_t launch_push2d(const Args& a, cudaStream_t s) {
    if (a.nwork == 0) return cudaSuccess;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(push2d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(Smem));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    push2d_kernel<<<a.nwork, NT, sizeof(Smem), s>>>(a);
    return cudaGetLastError();
}

cudaError_t preload_push2d() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, push2d_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, spill2d_kernel);
    return e;
}

cudaError_t launch_spill2d(const Args& a, cudaStream_t s) {
    spill2d_kernel<<<152 * 8, NT, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pic
