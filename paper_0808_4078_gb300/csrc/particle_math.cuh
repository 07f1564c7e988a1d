// particle_math.cuh -- per-particle arithmetic shared by the 2D and 3D particle kernels:
// relativistic Boris rotation, the cell carry of a move, the 3-node CIC/Esirkepov window of one
// axis, the path-averaged transverse shape factor, fixed-point helpers and the kinetic
// diagnostic.  Every rounding is explicit so that all code paths (tile fast path, queued
// crossers, spill list) produce the same bits for the same particle.
#pragma once
#include "pic_internal.cuh"

namespace pic {

constexpr float MOM_SCALE = 1048576.0f;  // 2^20, fixed point of the drag moments

// Per-run constants of the particle kernels, read from the run table once, before the first
// store: the kernels store particles through pointers the compiler cannot tell apart from the
// table, so fields read through it later would be reloaded from memory after every store.
struct RunConst {
    float dtdx, dtdy, dtdz;     // cells moved per unit velocity per step
    int nx, ny, nz;
    int cell_off;
    const float* dmap0;         // per-cell drag factors of species 0 and 1 (or null)
    const float* dmap1;
};
__device__ __forceinline__ RunConst run_const(const RunDev* R) {
    static_assert(PIC_NS == 2, "two species slots");
    RunConst k;
    k.dtdx = R->dtdx; k.dtdy = R->dtdy; k.dtdz = R->dtdz;
    k.nx = R->nx; k.ny = R->ny; k.nz = R->nz;
    k.cell_off = R->cell_off;
    k.dmap0 = R->dragmap[0];
    k.dmap1 = R->dragmap[1];
    return k;
}
// Drag factor of species s in local cell lc: the per-cell map if one is set, else the scalar.
__device__ __forceinline__ float drag_of(const RunConst& k, const SpeciesParams& P, int s, long long lc) {
    const float* m = s ? k.dmap1 : k.dmap0;
    return m ? m[lc] : P.dragf;
}

// ------------------------------------------------------------------ shared accumulators
__device__ __forceinline__ void add_split(unsigned* lo, int* hi, long long v) {
    if (v != 0) {
        atomicAdd(lo, (unsigned)(v & 4095));
        const int h = (int)(v >> 12);
        if (h != 0) atomicAdd(hi, h);
    }
}
// Shared-memory add of v unless it is 0, as a predicated reduction (no branch, so lanes with
// different values do not diverge).
__device__ __forceinline__ void red_nz(void* p, int v) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.s32 q, %1, 0;\n\t@q red.shared.add.s32 [%0], %1;\n\t}\n"
                 ::"r"(a), "r"(v) : "memory");
}
// add_split without branches: value = hi * 4096 + lo.
__device__ __forceinline__ void add_split_pred(unsigned* lo, int* hi, long long v) {
    red_nz(lo, (int)(v & 4095));
    red_nz(hi, (int)(v >> 12));
}

// ------------------------------------------------------------------ Boris
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

// ------------------------------------------------------------------ Esirkepov window
// CIC weights of the 3-node window [b, b+1, b+2] with b = min(old cell, new cell), for the old
// offset o in [0,1) and the carry c in {-1,0,1} with new offset no in [0,1).
struct Win {
    float S0[3], S1[3];
    float C[2];      // running sum of S1 - S0 along the axis (edges b+1/2, b+3/2)
    float A[3];      // (S0 + S1) / 2
    int off;         // b - old cell (-1 or 0)
};

// (Selects rather than branches: lanes of one warp with different carries do not diverge.)
//   c < 0:  S0 = (0, 1-o, o),  S1 = (1-no, no, 0),  C = (1-no, o)
//   c = 0:  S0 = (1-o, o, 0),  S1 = (1-no, no, 0),  C = (o-no, 0)
//   c > 0:  S0 = (1-o, o, 0),  S1 = (0, 1-no, no),  C = (o-1, -no)
__device__ __forceinline__ Win window(float o, int c, float no) {
    Win w;
    const float mo = __fsub_rn(1.f, o), mno = __fsub_rn(1.f, no);
    const bool neg = c < 0, pos = c > 0;
    w.S0[0] = neg ? 0.f : mo;
    w.S0[1] = neg ? mo : o;
    w.S0[2] = neg ? o : 0.f;
    w.S1[0] = pos ? 0.f : mno;
    w.S1[1] = pos ? mno : no;
    w.S1[2] = pos ? no : 0.f;
    w.C[0] = neg ? mno : (pos ? __fsub_rn(o, 1.f) : __fsub_rn(o, no));
    w.C[1] = neg ? o : (pos ? -no : 0.f);
    w.off = neg ? -1 : 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) w.A[k] = __fmul_rn(0.5f, __fadd_rn(w.S0[k], w.S1[k]));
    return w;
}

// Path-averaged shape product of the out-of-plane current,
// S0x (S0y/3 + S1y/6) + S1x (S0y/6 + S1y/3), with every rounding fixed.
__device__ __forceinline__ float zp(float s0, float s1) {
    return __fmaf_rn(s1, 1.f / 6.f, __fmul_rn(s0, 1.f / 3.f));
}
__device__ __forceinline__ float zq(float s0, float s1) {
    return __fmaf_rn(s1, 1.f / 3.f, __fmul_rn(s0, 1.f / 6.f));
}
__device__ __forceinline__ float zw(float s0x, float s1x, float p, float q) {
    return __fmaf_rn(s1x, q, __fmul_rn(s0x, p));
}

// Carry a new offset r (relative to the old cell, in (-1, 2)) into [0,1) and the cell step.
// A negative r whose r + 1 rounds to 1 stays in the cell at offset 0.  Written with selects so
// that divergent lanes take no branches.
__device__ __forceinline__ void carry(float r, float& no, int& c) {
    const float up = __fadd_rn(r, 1.f), down = __fsub_rn(r, 1.f);
    const bool neg = r < 0.f, tie = up >= 1.f, big = r >= 1.f;
    no = neg ? (tie ? 0.f : up) : (big ? down : r);
    c = neg ? (tie ? 0 : -1) : (big ? 1 : 0);
}

// Kinetic energy per species and total momentum at time n, int64 fixed point 2^32:
// kacc = {Ekin_0, Ekin_1, Px, Py, Pz}.
// x rounded to the nearest int64, ties to even (the value of __float2ll_rn), through 32-bit
// conversions only: the 64-bit conversion executes on the FP64 unit, which this part has little
// of.  With a = |x|, hi = floor(a 2^-32) and a - hi 2^32 are exact in FP32 (either hi = 0, or
// ulp(a) >= 2^9), so hi 2^32 + rint(a - hi 2^32) = rint(a); valid for |x| < 2^62.
__device__ __forceinline__ long long f2ll_rn(float x) {
    const float a = fabsf(x);
    const float hi = floorf(a * 2.3283064365386963e-10f);
    const unsigned lo = __float2uint_rn(a - hi * 4294967296.0f);
    const long long v = (long long)__float2uint_rz(hi) * 4294967296LL + (long long)lo;
    return x < 0.0f ? -v : v;
}

__device__ __forceinline__ void kin_add(long long kacc[5], int s, float w, float u0x, float u0y,
                                        float u0z, float ux, float uy, float uz) {
    const float mx = 0.5f * (u0x + ux), my = 0.5f * (u0y + uy), mz = 0.5f * (u0z + uz);
    const float gmid = sqrtf(1.f + mx * mx + my * my + mz * mz);
    const float sc = 4294967296.0f;   // 2^32
    const long long e = f2ll_rn(w * (gmid - 1.f) * sc);
    kacc[0] += s ? 0 : e;
    kacc[1] += s ? e : 0;
    kacc[2] += f2ll_rn(w * mx * sc);
    kacc[3] += f2ll_rn(w * my * sc);
    kacc[4] += f2ll_rn(w * mz * sc);
}

// ------------------------------------------------------------------ binary collisions
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of
// (hi0, lo0) = M0 c0, (hi1, lo1) = M1 c2, c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), the key
// raised by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, unsigned k0, unsigned k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// (x + 1/2) 2^-32 in FP32: a uniform draw in (0, 1].
__device__ __forceinline__ float unit_open(unsigned x) {
    return __fmaf_rn(__uint2float_rn(x), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
}

// One binary collision of an electron with an immobile ion over the step (Takizuka & Abe 1977
// with an infinitely heavy partner): u turns by theta, tan(theta / 2) = delta ~ N(0, sigma^2),
// about a uniform azimuth; |u| is kept.  The draws of particle `id` of species `s` at step
// `step` are Philox4x32-10 of counter (id, step lo, step hi, s) under the key (seed_lo,
// seed_hi): r0, r1 give delta (Box-Muller), r2 the azimuth.  Every rounding is explicit.
__device__ __forceinline__ void collide_ion(float& ux, float& uy, float& uz, const SpeciesParams& P, int s,
                                            unsigned id, long long step) {
    const uint4 r = philox4x32_10(make_uint4(id, (unsigned)((unsigned long long)step & 0xffffffffu),
                                             (unsigned)((unsigned long long)step >> 32), (unsigned)s),
                                  P.seed_lo, P.seed_hi);
    const float twopi = 6.283185307179586f;
    // ln U for U = (r + 1/2) 2^-32: for U >= 1/2 through log1p of the exact complement
    // (2^32 - r - 1/2) 2^-32, which FP32 holds without the 2^-24 quantisation of U near 1
    const float lnu = r.x < 0x80000000u ? logf(unit_open(r.x)) : log1pf(-unit_open(~r.x));
    const float rad = sqrtf(__fmul_rn(-2.f, lnu));
    // accurate sine and cosine (their large-argument path is never taken for angles in (0, 2 pi])
    const float delta = __fmul_rn(__fmul_rn(P.coll_sigma, rad), cosf(__fmul_rn(twopi, unit_open(r.y))));
    const float phi = __fmul_rn(twopi, unit_open(r.z));
    const float sp = sinf(phi), cp = cosf(phi);
    const float d2 = __fmul_rn(delta, delta);
    const float inv = __fdiv_rn(1.f, __fadd_rn(1.f, d2));
    const float sn = __fmul_rn(__fmul_rn(2.f, delta), inv);
    const float omc = __fmul_rn(__fmul_rn(2.f, d2), inv);
    const float up2 = __fmaf_rn(uy, uy, __fmul_rn(ux, ux));
    const float uperp = sqrtf(up2);
    const float umag = sqrtf(__fmaf_rn(uz, uz, up2));
    float dx, dy, dz;
    if (uperp > 0.f) {
        const float a = __fdiv_rn(__fmul_rn(sn, cp), uperp);      // sin theta cos phi / u_perp
        const float b = __fdiv_rn(__fmul_rn(sn, sp), uperp);      // sin theta sin phi / u_perp
        dx = __fsub_rn(__fsub_rn(__fmul_rn(__fmul_rn(ux, uz), a), __fmul_rn(__fmul_rn(uy, umag), b)), __fmul_rn(ux, omc));
        dy = __fsub_rn(__fadd_rn(__fmul_rn(__fmul_rn(uy, uz), a), __fmul_rn(__fmul_rn(ux, umag), b)), __fmul_rn(uy, omc));
        dz = __fsub_rn(__fmul_rn(-uperp, __fmul_rn(sn, cp)), __fmul_rn(uz, omc));
    } else {
        dx = __fmul_rn(umag, __fmul_rn(sn, cp));
        dy = __fmul_rn(umag, __fmul_rn(sn, sp));
        dz = __fmul_rn(-uz, omc);
    }
    ux = __fadd_rn(ux, dx);
    uy = __fadd_rn(uy, dy);
    uz = __fadd_rn(uz, dz);
}

}  // namespace pic
