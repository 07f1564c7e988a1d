// push2d.cu -- fused 2D3V particle step: CIC field gather, relativistic Boris push, Krook drag
// of the return-current electrons (Eq. (3) friction, per-cell mean-momentum relaxation), move
// with cell carry, and charge-conserving Esirkepov current deposition (CIC), accumulated in
// int64 fixed point through a shared-memory tile.
//
// One CTA per (run, tile) of TX x TY cells.  Particles were binned by tile at the last counting
// sort, so the CTA walks the contiguous range [start[key0], start[key0 + TX*TY]) of each
// species.  Since then particles may have drifted up to DR cells out of the tile; the shared
// tile covers the tile plus that drift plus the CIC stencil.  A particle farther out takes the
// same arithmetic against global memory (global atomics), so results never depend on the sort
// interval: every current term is rounded to an integer before it is summed, and integer sums
// are order-independent, so J is bit-reproducible whatever the particle order.
//
// Deposit per particle uses a 3-node window per axis starting at min(old cell, new cell)
// (a particle moves less than one cell per step).  Warp aggregation: lanes that stay in the
// warp's reference cell (the common case for cell-sorted particles) touch the same 8 current
// nodes (and the same drag-moment cell); their integer terms are summed across the warp with a
// transpose reduce-scatter (15 shuffles for 16 values) and applied with one shared atomic per
// value.  Other lanes apply their up-to-21 terms individually.
#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int TX = 16, TY = 16, DR = 2;
constexpr int RX = TX + 2 * DR + 3, RY = TY + 2 * DR + 3, RN = RX * RY;
constexpr int NT = 256;
constexpr unsigned FULL = 0xffffffffu;

struct __align__(16) Smem {
    float F[6][RN];                  // Ex Ey Ez Bx By Bz of the region
    unsigned long long J[3][RN];     // current accumulator (int64 two's complement)
    float ub[3][RN];                 // previous cell-mean momentum (drag)
    unsigned long long M[3][RN];     // new drag moments, fixed point 2^20
    int MC[RN];                      // new drag counts
    double red[NT / 32][6];
    unsigned long long kin[4];
};

// CIC weights of the 3-node window [b, b+1, b+2] with b = min(old cell, new cell), for the old
// offset o in [0,1) and the carry c in {-1,0,1} with new offset no in [0,1).
struct Win {
    float S0[3], S1[3];
    float C[2];      // running sum of S1 - S0 along the axis (edges b+1/2, b+3/2)
    float A[3];      // (S0 + S1) / 2
    int off;         // b - old cell (-1 or 0)
};

__device__ __forceinline__ Win window(float o, int c, float no) {
    Win w;
    const float mo = __fsub_rn(1.f, o), mno = __fsub_rn(1.f, no);
    if (c < 0) {
        w.S0[0] = 0.f; w.S0[1] = mo; w.S0[2] = o;
        w.S1[0] = mno; w.S1[1] = no; w.S1[2] = 0.f;
        w.C[0] = mno; w.C[1] = o;
        w.off = -1;
    } else if (c == 0) {
        w.S0[0] = mo; w.S0[1] = o; w.S0[2] = 0.f;
        w.S1[0] = mno; w.S1[1] = no; w.S1[2] = 0.f;
        w.C[0] = __fsub_rn(o, no); w.C[1] = 0.f;
        w.off = 0;
    } else {
        w.S0[0] = mo; w.S0[1] = o; w.S0[2] = 0.f;
        w.S1[0] = 0.f; w.S1[1] = mno; w.S1[2] = no;
        w.C[0] = __fsub_rn(o, 1.f); w.C[1] = -no;
        w.off = 0;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) w.A[k] = __fmul_rn(0.5f, __fadd_rn(w.S0[k], w.S1[k]));
    return w;
}

// Path-averaged shape product of the out-of-plane current,
// S0x (S0y/3 + S1y/6) + S1x (S0y/6 + S1y/3), with every rounding fixed so that all code
// paths produce bitwise identical terms.
__device__ __forceinline__ float zp(float s0, float s1) {
    return __fmaf_rn(s1, 1.f / 6.f, __fmul_rn(s0, 1.f / 3.f));
}
__device__ __forceinline__ float zq(float s0, float s1) {
    return __fmaf_rn(s1, 1.f / 3.f, __fmul_rn(s0, 1.f / 6.f));
}
__device__ __forceinline__ float zw(float s0x, float s1x, float p, float q) {
    return __fmaf_rn(s1x, q, __fmul_rn(s0x, p));
}

// Warp sum of 16 int values; lane l returns the total of value index l >> 1.
__device__ __forceinline__ int transpose_reduce16(int v[16], int lane) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        bool hi = lane & 16;
        int send = hi ? v[i] : v[i + 8];
        int keep = hi ? v[i + 8] : v[i];
        v[i] = keep + __shfl_xor_sync(FULL, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        bool hi = lane & 8;
        int send = hi ? v[i] : v[i + 4];
        int keep = hi ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(FULL, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        bool hi = lane & 4;
        int send = hi ? v[i] : v[i + 2];
        int keep = hi ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(FULL, send, 4);
    }
    {
        bool hi = lane & 2;
        int send = hi ? v[0] : v[1];
        int keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(FULL, send, 2);
    }
    return v[0] + __shfl_xor_sync(FULL, v[0], 1);
}

__device__ __forceinline__ void sadd(unsigned long long* p, long long v) {
    if (v != 0) atomicAdd(p, (unsigned long long)v);
}

// Field access: region (shared) coordinates or global (periodic) coordinates.
struct SharedFields {
    const Smem* s;
    __device__ float operator()(int c, int i, int j) const { return s->F[c][j * RX + i]; }
};
struct GlobalFields {
    const RunDev* R;
    __device__ float operator()(int c, int i, int j) const {
        int gi = wrapi(i, R->nx), gj = wrapi(j, R->ny);
        const float* p = c < 3 ? R->E[c] : R->B[c - 3];
        return __ldg(p + (size_t)gj * R->nx + gi);
    }
};

__device__ __forceinline__ float lerp2(float w0, float w1, float a, float b) {
    return __fmaf_rn(w1, b, __fmul_rn(w0, a));
}

// CIC gather of the six staggered components at node (i, j) + offsets (ox, oy).  Roundings
// are explicit so that the shared-memory and global-memory instances agree bitwise.
template <class Acc>
__device__ __forceinline__ void gather(const Acc& F, int i, int j, float ox, float oy, float EB[6]) {
    // half-shifted lattices: position - 1/2
    const float hx = __fsub_rn(ox, 0.5f), hy = __fsub_rn(oy, 0.5f);
    const int ih = hx < 0.f ? i - 1 : i;
    const int jh = hy < 0.f ? j - 1 : j;
    const float fx = hx < 0.f ? __fadd_rn(hx, 1.f) : hx;
    const float fy = hy < 0.f ? __fadd_rn(hy, 1.f) : hy;
    const float wx0 = __fsub_rn(1.f, ox), wx1 = ox, wy0 = __fsub_rn(1.f, oy), wy1 = oy;
    const float hx0 = __fsub_rn(1.f, fx), hx1 = fx, hy0 = __fsub_rn(1.f, fy), hy1 = fy;
    // Ex (1/2, 0), By (1/2, 0)
    EB[0] = lerp2(wy0, wy1, lerp2(hx0, hx1, F(0, ih, j), F(0, ih + 1, j)), lerp2(hx0, hx1, F(0, ih, j + 1), F(0, ih + 1, j + 1)));
    EB[4] = lerp2(wy0, wy1, lerp2(hx0, hx1, F(4, ih, j), F(4, ih + 1, j)), lerp2(hx0, hx1, F(4, ih, j + 1), F(4, ih + 1, j + 1)));
    // Ey (0, 1/2), Bx (0, 1/2)
    EB[1] = lerp2(hy0, hy1, lerp2(wx0, wx1, F(1, i, jh), F(1, i + 1, jh)), lerp2(wx0, wx1, F(1, i, jh + 1), F(1, i + 1, jh + 1)));
    EB[3] = lerp2(hy0, hy1, lerp2(wx0, wx1, F(3, i, jh), F(3, i + 1, jh)), lerp2(wx0, wx1, F(3, i, jh + 1), F(3, i + 1, jh + 1)));
    // Ez (0, 0)
    EB[2] = lerp2(wy0, wy1, lerp2(wx0, wx1, F(2, i, j), F(2, i + 1, j)), lerp2(wx0, wx1, F(2, i, j + 1), F(2, i + 1, j + 1)));
    // Bz (1/2, 1/2)
    EB[5] = lerp2(hy0, hy1, lerp2(hx0, hx1, F(5, ih, jh), F(5, ih + 1, jh)), lerp2(hx0, hx1, F(5, ih, jh + 1), F(5, ih + 1, jh + 1)));
}

// Relativistic Boris rotation u^{n-1/2} -> u^{n+1/2}; h = q dt / (2 m).  Explicit roundings
// keep every particle's update independent of which code path the compiler emits.
__device__ __forceinline__ void boris(float h, const float EB[6], float& ux, float& uy, float& uz) {
    const float umx = __fmaf_rn(h, EB[0], ux), umy = __fmaf_rn(h, EB[1], uy), umz = __fmaf_rn(h, EB[2], uz);
    const float g2 = __fmaf_rn(umz, umz, __fmaf_rn(umy, umy, __fmaf_rn(umx, umx, 1.f)));
    const float ig = rsqrtf(g2);
    const float hg = __fmul_rn(h, ig);
    const float tx = __fmul_rn(hg, EB[3]), ty = __fmul_rn(hg, EB[4]), tz = __fmul_rn(hg, EB[5]);
    const float t2 = __fmaf_rn(tz, tz, __fmaf_rn(ty, ty, __fmaf_rn(tx, tx, 1.f)));
    const float sf = __fdividef(2.f, t2);
    const float upx = __fadd_rn(umx, __fmaf_rn(umy, tz, -__fmul_rn(umz, ty)));
    const float upy = __fadd_rn(umy, __fmaf_rn(umz, tx, -__fmul_rn(umx, tz)));
    const float upz = __fadd_rn(umz, __fmaf_rn(umx, ty, -__fmul_rn(umy, tx)));
    const float sx = __fmul_rn(sf, tx), sy = __fmul_rn(sf, ty), sz = __fmul_rn(sf, tz);
    ux = __fmaf_rn(h, EB[0], __fadd_rn(umx, __fmaf_rn(upy, sz, -__fmul_rn(upz, sy))));
    uy = __fmaf_rn(h, EB[1], __fadd_rn(umy, __fmaf_rn(upz, sx, -__fmul_rn(upx, sz))));
    uz = __fmaf_rn(h, EB[2], __fadd_rn(umz, __fmaf_rn(upx, sy, -__fmul_rn(upy, sx))));
}

// Apply the up-to-21 current terms of one particle; `at(c, i, j)` returns the accumulator.
template <class At>
__device__ __forceinline__ void deposit_terms(const At& at, const SpeciesParams& P, int bi, int bj,
                                              const Win& wx, const Win& wy, float zf) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float a = __fmul_rn(P.jx, wx.C[k]);
#pragma unroll
        for (int l = 0; l < 3; ++l) sadd(at(0, bi + k, bj + l), round_small(a, wy.A[l]));
    }
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        const float a = __fmul_rn(P.jy, wy.C[l]);
#pragma unroll
        for (int k = 0; k < 3; ++k) sadd(at(1, bi + k, bj + l), round_small(a, wx.A[k]));
    }
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        const float p = zp(wy.S0[l], wy.S1[l]), q = zq(wy.S0[l], wy.S1[l]);
#pragma unroll
        for (int k = 0; k < 3; ++k) sadd(at(2, bi + k, bj + l), round_small(zf, zw(wx.S0[k], wx.S1[k], p, q)));
    }
}

__global__ void __launch_bounds__(NT) push2d_kernel(const Args a) {
    __shared__ Smem sm;
    const int2 wk = a.work[blockIdx.x];
    const RunDev* Rp = &a.runs[wk.x];
    const int nx = Rp->nx, ny = Rp->ny;
    const int tile = wk.y;
    const int x0 = (tile % Rp->ntx) * TX, y0 = (tile / Rp->ntx) * TY;
    const int gx0 = x0 - DR - 1, gy0 = y0 - DR - 1;
    const long long step = a.ctl->step;
    const bool diag = a.diag_interval > 0 && (step % a.diag_interval) == 0;
    const bool anydrag = Rp->msum[0] != nullptr;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int i = tid; i < RN; i += NT) {
        const int ry = i / RX, rx = i - ry * RX;
        const size_t g = (size_t)wrapi(gy0 + ry, ny) * nx + wrapi(gx0 + rx, nx);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sm.F[c][i] = Rp->E[c][g];
            sm.F[3 + c][i] = Rp->B[c][g];
            sm.J[c][i] = 0ull;
        }
        if (anydrag) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                sm.ub[c][i] = Rp->ubar[c][g];
                sm.M[c][i] = 0ull;
            }
            sm.MC[i] = 0;
        }
    }
    if (tid < 4) sm.kin[tid] = 0ull;
    __syncthreads();

    if (diag) {
        // field energy of the tile's own cells (each cell counted by exactly one CTA)
        const int i = (tid % TX) + DR + 1, j = (tid / TX) + DR + 1;
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
            for (int w = 0; w < NT / 32; ++w) s += sm.red[w][tid];
            a.partials[(size_t)blockIdx.x * 8 + tid] = s;
        }
    }

    const SharedFields SF{&sm};
    const GlobalFields GF{Rp};
    auto sh_at = [&](int c, int i, int j) { return &sm.J[c][j * RX + i]; };
    auto gl_at = [&](int c, int i, int j) {
        return (unsigned long long*)&Rp->J[c][(size_t)wrapi(j, ny) * nx + wrapi(i, nx)];
    };

    for (int s = 0; s < a.nspecies; ++s) {
        const SpeciesParams P = Rp->sp[s];
        if (!P.active) continue;
        const SpeciesBuf B = a.buf[s][a.ctl->parity[s]];
        const int key0 = Rp->cell_off + tile * (TX * TY);
        const int beg = a.start[s][key0], end = a.start[s][key0 + TX * TY];
        long long kacc[4] = {0, 0, 0, 0};

        for (int base = beg + warp * 32; base < end; base += NT) {
            const int p = base + lane;
            const bool act = p < end;
            int lc = 0;
            float ox = 0.f, oy = 0.f, ux = 0.f, uy = 0.f, uz = 0.f;
            if (act) {
                lc = B.cell[p] - Rp->cell_off;
                ox = B.o[0][p]; oy = B.o[1][p];
                ux = B.u[0][p]; uy = B.u[1][p]; uz = B.u[2][p];
            }
            const int cy = lc / nx, cx = lc - cy * nx;
            const int rxi = wrapi(cx - x0 + DR, nx) - DR;
            const int ryi = wrapi(cy - y0 + DR, ny) - DR;
            const bool inreg = rxi < TX + DR && ryi < TY + DR;
            const int ix = rxi + DR + 1, iy = ryi + DR + 1;   // shared node index of (cx, cy)

            float EB[6];
            if (inreg) gather(SF, ix, iy, ox, oy, EB);
            else gather(GF, cx, cy, ox, oy, EB);
            const float u0x = ux, u0y = uy, u0z = uz;
            boris(P.qmdt2, EB, ux, uy, uz);
            if (P.drag) {
                float b0, b1, b2;
                if (inreg) {
                    const int si = iy * RX + ix;
                    b0 = sm.ub[0][si]; b1 = sm.ub[1][si]; b2 = sm.ub[2][si];
                } else {
                    const size_t g = (size_t)cy * nx + cx;
                    b0 = Rp->ubar[0][g]; b1 = Rp->ubar[1][g]; b2 = Rp->ubar[2][g];
                }
                ux = __fmaf_rn(-P.dragf, b0, ux);
                uy = __fmaf_rn(-P.dragf, b1, uy);
                uz = __fmaf_rn(-P.dragf, b2, uz);
            }
            const float ig = rsqrtf(__fmaf_rn(uz, uz, __fmaf_rn(uy, uy, __fmaf_rn(ux, ux, 1.f))));
            const float rx = __fmaf_rn(__fmul_rn(ux, ig), Rp->dtdx, ox);
            const float ry = __fmaf_rn(__fmul_rn(uy, ig), Rp->dtdy, oy);
            const bool bad = act && !(rx > -1.f && rx < 2.f && ry > -1.f && ry < 2.f);
            if (bad) atomicOr(&a.ctl->err, ERR_BADPART);
            const bool live = act && !bad;

            int sx = 0, sy = 0;
            float nox = rx, noy = ry;
            if (rx < 0.f) { nox = rx + 1.f; sx = -1; if (nox >= 1.f) { nox = 0.f; sx = 0; } }
            else if (rx >= 1.f) { nox = rx - 1.f; sx = 1; }
            if (ry < 0.f) { noy = ry + 1.f; sy = -1; if (noy >= 1.f) { noy = 0.f; sy = 0; } }
            else if (ry >= 1.f) { noy = ry - 1.f; sy = 1; }
            const float vz = __fmul_rn(uz, ig);

            if (diag && live) {
                const float mx = 0.5f * (u0x + ux), my = 0.5f * (u0y + uy), mz = 0.5f * (u0z + uz);
                const float gmid = sqrtf(1.f + mx * mx + my * my + mz * mz);
                const float sc = 4294967296.0f;   // 2^32
                kacc[0] += __float2ll_rn(P.w * (gmid - 1.f) * sc);
                kacc[1] += __float2ll_rn(P.w * mx * sc);
                kacc[2] += __float2ll_rn(P.w * my * sc);
                kacc[3] += __float2ll_rn(P.w * mz * sc);
            }

            // ---- warp-aggregated deposit for lanes staying in the reference cell
            const bool small_u = !P.drag || (fabsf(ux) < 32.f && fabsf(uy) < 32.f && fabsf(uz) < 32.f);
            const unsigned am = __ballot_sync(FULL, act);
            const int leader = am ? __ffs(am) - 1 : 0;
            const int ref = __shfl_sync(FULL, lc, leader);
            bool fast = live && inreg && sx == 0 && sy == 0 && lc == ref && small_u;
            const unsigned fm = __ballot_sync(FULL, fast);
            const Win wx = window(ox, sx, nox), wy = window(oy, sy, noy);
            const float zf = __fmul_rn(P.jz, vz);
            if (fm) {
                int v[16];
                const float jxa = __fmul_rn(P.jx, wx.C[0]), jya = __fmul_rn(P.jy, wy.C[0]);
                const float p0 = zp(wy.S0[0], wy.S1[0]), q0 = zq(wy.S0[0], wy.S1[0]);
                const float p1 = zp(wy.S0[1], wy.S1[1]), q1 = zq(wy.S0[1], wy.S1[1]);
                v[0] = round_small(jxa, wy.A[0]);                                  // Jx (cx+1/2, cy)
                v[1] = round_small(jxa, wy.A[1]);                                  // Jx (cx+1/2, cy+1)
                v[2] = round_small(jya, wx.A[0]);                                  // Jy (cx, cy+1/2)
                v[3] = round_small(jya, wx.A[1]);                                  // Jy (cx+1, cy+1/2)
                v[4] = round_small(zf, zw(wx.S0[0], wx.S1[0], p0, q0));            // Jz (cx, cy)
                v[5] = round_small(zf, zw(wx.S0[1], wx.S1[1], p0, q0));            // Jz (cx+1, cy)
                v[6] = round_small(zf, zw(wx.S0[0], wx.S1[0], p1, q1));            // Jz (cx, cy+1)
                v[7] = round_small(zf, zw(wx.S0[1], wx.S1[1], p1, q1));            // Jz (cx+1, cy+1)
                const float ms = 1048576.0f;   // 2^20
                v[8] = P.drag ? __float2int_rn(ux * ms) : 0;
                v[9] = P.drag ? __float2int_rn(uy * ms) : 0;
                v[10] = P.drag ? __float2int_rn(uz * ms) : 0;
                v[11] = P.drag ? 1 : 0;
                v[12] = v[13] = v[14] = v[15] = 0;
                if (!fast) {
#pragma unroll
                    for (int k = 0; k < 12; ++k) v[k] = 0;
                }
                const int tot = transpose_reduce16(v, lane);
                const int fl = __ffs(fm) - 1;
                const int rix = __shfl_sync(FULL, ix, fl), riy = __shfl_sync(FULL, iy, fl);
                const int idx = lane >> 1;
                if (!(lane & 1) && tot != 0) {
                    const int n0 = riy * RX + rix;
                    switch (idx) {
                        case 0: atomicAdd(&sm.J[0][n0], (unsigned long long)(long long)tot); break;
                        case 1: atomicAdd(&sm.J[0][n0 + RX], (unsigned long long)(long long)tot); break;
                        case 2: atomicAdd(&sm.J[1][n0], (unsigned long long)(long long)tot); break;
                        case 3: atomicAdd(&sm.J[1][n0 + 1], (unsigned long long)(long long)tot); break;
                        case 4: atomicAdd(&sm.J[2][n0], (unsigned long long)(long long)tot); break;
                        case 5: atomicAdd(&sm.J[2][n0 + 1], (unsigned long long)(long long)tot); break;
                        case 6: atomicAdd(&sm.J[2][n0 + RX], (unsigned long long)(long long)tot); break;
                        case 7: atomicAdd(&sm.J[2][n0 + RX + 1], (unsigned long long)(long long)tot); break;
                        case 8: atomicAdd(&sm.M[0][n0], (unsigned long long)(long long)tot); break;
                        case 9: atomicAdd(&sm.M[1][n0], (unsigned long long)(long long)tot); break;
                        case 10: atomicAdd(&sm.M[2][n0], (unsigned long long)(long long)tot); break;
                        case 11: atomicAdd(&sm.MC[n0], tot); break;
                        default: break;
                    }
                }
            }

            if (live && !fast) {
                if (inreg) {
                    deposit_terms(sh_at, P, ix + wx.off, iy + wy.off, wx, wy, zf);
                    if (P.drag) {
                        const int n1 = (iy + sy) * RX + (ix + sx);
                        const float ms = 1048576.0f;
                        sadd(&sm.M[0][n1], __float2ll_rn(ux * ms));
                        sadd(&sm.M[1][n1], __float2ll_rn(uy * ms));
                        sadd(&sm.M[2][n1], __float2ll_rn(uz * ms));
                        atomicAdd(&sm.MC[n1], 1);
                    }
                } else {
                    deposit_terms(gl_at, P, cx + wx.off, cy + wy.off, wx, wy, zf);
                    if (P.drag) {
                        const size_t g1 = (size_t)wrapi(cy + sy, ny) * nx + wrapi(cx + sx, nx);
                        const float ms = 1048576.0f;
                        sadd((unsigned long long*)&Rp->msum[0][g1], __float2ll_rn(ux * ms));
                        sadd((unsigned long long*)&Rp->msum[1][g1], __float2ll_rn(uy * ms));
                        sadd((unsigned long long*)&Rp->msum[2][g1], __float2ll_rn(uz * ms));
                        atomicAdd(&Rp->mcnt[g1], 1);
                    }
                }
            }

            if (live) {
                int ncx = cx + sx, ncy = cy + sy;
                ncx = ncx < 0 ? ncx + nx : (ncx >= nx ? ncx - nx : ncx);
                ncy = ncy < 0 ? ncy + ny : (ncy >= ny ? ncy - ny : ncy);
                B.cell[p] = Rp->cell_off + ncy * nx + ncx;
                B.o[0][p] = nox; B.o[1][p] = noy;
                B.u[0][p] = ux; B.u[1][p] = uy; B.u[2][p] = uz;
            }
        }

        if (diag) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                long long v = kacc[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
                if (lane == 0 && v != 0) atomicAdd(&sm.kin[k], (unsigned long long)v);
            }
            __syncthreads();
            if (tid < 4 && sm.kin[tid] != 0ull) {
                atomicAdd((unsigned long long*)&a.ctl->kin[s][tid], sm.kin[tid]);
                sm.kin[tid] = 0ull;
            }
        }
    }
    __syncthreads();

    // flush the region to global memory (halo nodes overlap neighbouring tiles: atomics)
    for (int i = tid; i < RN; i += NT) {
        const int ry = i / RX, rx = i - ry * RX;
        const size_t g = (size_t)wrapi(gy0 + ry, ny) * nx + wrapi(gx0 + rx, nx);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const unsigned long long v = sm.J[c][i];
            if (v) atomicAdd((unsigned long long*)&Rp->J[c][g], v);
        }
        if (anydrag) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const unsigned long long v = sm.M[c][i];
                if (v) atomicAdd((unsigned long long*)&Rp->msum[c][g], v);
            }
            if (sm.MC[i]) atomicAdd(&Rp->mcnt[g], sm.MC[i]);
        }
    }
}

}  // namespace

cudaError_t launch_push2d(const Args& a, cudaStream_t s) {
    if (a.nwork == 0) return cudaSuccess;
    push2d_kernel<<<a.nwork, NT, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pic
