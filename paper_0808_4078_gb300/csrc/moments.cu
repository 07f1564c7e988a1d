// moments.cu -- coarse-grained moment recorder: the inputs and label parts of the learned
// collision closure, per coarse cell (bx x by transverse cells x the whole z extent).
//
// The paper closes by conjecturing that the collisional drag on the return current could be
// written through the local plasma state; the quantities recorded here are the reading of that
// closure's inputs and label (rows in pic.h: densities, mean u_z, momentum variances of beam and
// background, electrostatic fluctuation energy W_ES, and the background's mean particle force
// against the force of the coarse-grained fields).
//
// Two passes over the particles: the first sums w and w u per coarse cell and species, the
// second the centred second moments w (u - <u>)^2 (variances of a cold beam are ~1e-6 of <u>^2,
// far below what <u^2> - <u>^2 resolves) and the background's force and velocity sums.  Sums are
// int64 fixed point (2^36 per unit; a coarse cell's sum of |w u| must stay below 2^27),
// accumulated per CTA and added with one atomic per quantity, so they do not depend on the order
// of the particles; the field column sums are FP64 in a fixed order.  The record is bitwise
// reproducible.
#include "pic_internal.cuh"

namespace pic {

// psum rows: pass 1 per species w, w ux, w uy, w uz (rows 4 s + 0..3); pass 2 per species
// w (ux - <ux>)^2, w (uy - <uy>)^2, w (uz - <uz>)^2 (rows 8 + 3 s + 0..2), then the background's
// w Fz, w vx, w vy, w vz (rows 14..17).
constexpr int MOM_PSUMS = 18;
constexpr int MOM_COLS = 4;                 // per column: W_ES mean, mean Ez, mean Bx, mean By
constexpr double MOM_FIX = 68719476736.0;   // 2^36

namespace {

constexpr int NT = 256;

struct MomArgs {
    Args a;
    int run;
    int bx, by;        // coarse block in cells
    int zc;            // z layers per CTA
    int ncx, ncy;      // coarse cells per axis
    float q_bg;        // background charge
    float nu_bg;       // background Krook rate
    long long* psum;   // [MOM_PSUMS][nc]
    float* meanbuf;    // [nc][12]: coarse means of pass 1 as FP32 pairs
    double* col;       // [MOM_COLS][nx * ny]
    float* out;        // [PIC_MOM_ROWS][nc]
};

__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Component c of E (c < 3) or B at the particle, CIC on its Yee lattice, global memory.
__device__ __forceinline__ float gather_comp(const RunDev& R, int ndim, int c, int cx, int cy, int cz, float ox, float oy, float oz) {
    // half-shifted axes of each component: Ex x, Ey y, Ez z (3D); Bx y,z; By x,z; Bz x,y
    // (2D: Ez and the z shifts are absent)
    // bit c set: component c is half-shifted along the axis (c = Ex Ey Ez Bx By Bz)
    const bool hx = (0x31 >> c) & 1, hy = (0x2A >> c) & 1, hz = ndim == 3 && ((0x1C >> c) & 1);
    const float* F = c < 3 ? R.E[c] : R.B[c - 3];
    const float xs = hx ? ox - 0.5f : ox, ys = hy ? oy - 0.5f : oy, zs = hz ? oz - 0.5f : oz;
    const int i0 = xs < 0.f ? -1 : 0, j0 = ys < 0.f ? -1 : 0, k0 = zs < 0.f ? -1 : 0;
    const float ax = xs - (float)i0, ay = ys - (float)j0, az = zs - (float)k0;
    const int nz = ndim == 3 ? R.nz : 1;
    float v = 0.f;
    for (int dk = 0; dk < (ndim == 3 ? 2 : 1); ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                // neighbours within one cell of the particle's: one conditional wrap
                const int gi = wrap1(cx + i0 + di, R.nx), gj = wrap1(cy + j0 + dj, R.ny);
                const int gk = ndim == 3 ? wrap1(cz + k0 + dk, nz) : 0;
                const float wgt = (di ? ax : 1.f - ax) * (dj ? ay : 1.f - ay) *
                                  (ndim == 3 ? (dk ? az : 1.f - az) : 1.f);
                v += wgt * F[((size_t)gk * R.ny + gj) * R.nx + gi];
            }
    return v;
}

// v 2^36 rounded to the nearest int64 (ties to even) through 32-bit conversions only: the 64-bit
// ones run on the FP64 unit, which this part has little of.  With a = |v| 2^36 (an exact
// scaling), hi = floor(a 2^-32) and a - hi 2^32 are exact in FP32 (either hi = 0 or
// ulp(a) >= 2^9), so hi 2^32 + rint(a - hi 2^32) = rint(a); valid for |v| 2^36 < 2^62.
__device__ __forceinline__ long long fx(float v) {
    const float a = fabsf(v) * 68719476736.0f;
    const float hi = floorf(a * 2.3283064365386963e-10f);
    const unsigned lo = __float2uint_rn(a - hi * 4294967296.0f);
    const long long r = (long long)__float2uint_rz(hi) * 4294967296LL + (long long)lo;
    return v < 0.0f ? -r : r;
}

// Mean of a coarse cell as an unevaluated FP32 sum hi + lo, so that u - mean keeps FP32
// relative accuracy for the small deviations of a cold beam: u - hi is exact when u is within a
// factor 2 of hi (Sterbenz), then lo is subtracted.
struct Mean2 { float hi[2][3], lo[2][3]; };

// Add one particle to the thread's sums (FP32 arithmetic, exact fixed-point sums): pass 1 first
// moments, pass 2 centred second moments about its coarse cell's mean and the background force
// and velocity.
// Rows of each pass: pass 1 rows [0, 8), pass 2 rows [8, 18); acc holds the pass's rows only.
template <int PASS> struct PassRows;
template <> struct PassRows<1> { static constexpr int base = 0, n = 8; };
template <> struct PassRows<2> { static constexpr int base = 8, n = 10; };

template <int PASS>
__device__ __forceinline__ void add_particle(const MomArgs& m, const RunDev& R, int s, float w,
                                             const Mean2& mean, int cx, int cy, int cz, float ox,
                                             float oy, float oz, float ux, float uy, float uz,
                                             long long* acc) {
    const float du[3] = {ux, uy, uz};
    if (PASS == 1) {
        acc[4 * s] += fx(w);
#pragma unroll
        for (int d = 0; d < 3; ++d) acc[4 * s + 1 + d] += fx(__fmul_rn(w, du[d]));
        return;
    }
    acc -= 8;   // pass-2 rows are numbered from 8
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float e = __fsub_rn(__fsub_rn(du[d], mean.hi[s][d]), mean.lo[s][d]);
        acc[8 + 3 * s + d] += fx(__fmul_rn(w, __fmul_rn(e, e)));
    }
    if (s == 1) {
        const float ig = 1.0f / sqrtf(1.0f + ux * ux + uy * uy + uz * uz);
        const float vx = ux * ig, vy = uy * ig, vz = uz * ig;
        const int nd = m.a.ndim;
        const float ez = gather_comp(R, nd, 2, cx, cy, cz, ox, oy, oz);
        const float bx = gather_comp(R, nd, 3, cx, cy, cz, ox, oy, oz);
        const float by = gather_comp(R, nd, 4, cx, cy, cz, ox, oy, oz);
        const float fz = m.q_bg * (ez + vx * by - vy * bx);
        acc[14] += fx(w * fz);
        acc[15] += fx(w * vx);
        acc[16] += fx(w * vy);
        acc[17] += fx(w * vz);
    }
}

// Means <u> per species of each coarse cell from the pass-1 sums, computed once (FP64 divisions
// are costly on this part) and stored as FP32 pairs for pass 2: meanbuf[cc] = hi[6], lo[6].
__global__ void __launch_bounds__(NT) mom_means(const MomArgs m) {
    const long long nc = (long long)m.ncx * m.ncy;
    for (long long cc = blockIdx.x * (long long)NT + threadIdx.x; cc < nc; cc += (long long)gridDim.x * NT) {
        float* o = m.meanbuf + (size_t)cc * 12;
        for (int s = 0; s < 2; ++s) {
            const double sw = (double)m.psum[(size_t)(4 * s) * nc + cc];
            for (int d = 0; d < 3; ++d) {
                const double mu = sw > 0 ? (double)m.psum[(size_t)(4 * s + 1 + d) * nc + cc] / sw : 0.0;
                const float hi = (float)mu;
                o[3 * s + d] = hi;
                o[6 + 3 * s + d] = (float)(mu - (double)hi);
            }
        }
    }
}

__device__ __forceinline__ void coarse_means(const MomArgs& m, long long cc, Mean2& mean) {
    const float* o = m.meanbuf + (size_t)cc * 12;
    for (int s = 0; s < 2; ++s)
        for (int d = 0; d < 3; ++d) {
            mean.hi[s][d] = o[3 * s + d];
            mean.lo[s][d] = o[6 + 3 * s + d];
        }
}

// 2D (particles binned by cell): one CTA per (coarse cell, z chunk): a thread per fine cell, all its particles; one kernel per
// pass, each holding only its own sums (pass 2 with its field gathers runs 2 CTAs per SM without
// spilling, measured faster than 3 with spills).
template <int PASS>
__global__ void __launch_bounds__(NT, PASS == 1 ? 3 : 2) mom_particles(const MomArgs m) {
    constexpr int B = PassRows<PASS>::base, NR = PassRows<PASS>::n;
    __shared__ long long red[NT / 32][NR];
    const Args& a = m.a;
    const RunDev& R = a.runs[m.run];
    const int cc = blockIdx.x;
    Mean2 mean{};
    if (PASS == 2) coarse_means(m, cc, mean);
    const int X0 = (cc % m.ncx) * m.bx, Y0 = (cc / m.ncx) * m.by;
    const int per = m.bx * m.by;
    long long acc[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) acc[k] = 0;
    const int par = a.ctl->parity;
    for (int t = threadIdx.x; t < per * m.zc; t += NT) {
        const int col = t % per, lz = t / per;
        const int cx = X0 + col % m.bx, cy = Y0 + col / m.bx;
        const int cz = blockIdx.y * m.zc + lz;
        if (cz >= R.nz) continue;
        const long long g = R.cell_off + ((long long)cz * R.ny + cy) * R.nx + cx;
        for (int s = 0; s < a.nspecies && s < 2; ++s) {
            if (!R.sp[s].active) continue;
            const Slots& S = a.slot[s][par];
            const CellRange cr = cell_range(S, a.cap[s], a.cap_stay[s], g);
            const float w = R.sp[s].w;
            for (int k = 0; k < cr.n; ++k) {
                const size_t q = slot_elt(S, (long long)slot_of(g, a.cap[s], a.cap_stay[s], cr.ns, k));
                add_particle<PASS>(m, R, s, w, mean, cx, cy, cz, S.o[0][q], S.o[1][q],
                                   a.ndim == 3 ? S.o[2][q] : 0.f, S.u[0][q], S.u[1][q], S.u[2][q], acc);
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        long long v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < NR) {
        long long v = 0;
        for (int w = 0; w < NT / 32; ++w) v += red[w][threadIdx.x];
        if (v) atomicAdd((unsigned long long*)&m.psum[(size_t)(B + threadIdx.x) * m.ncx * m.ncy + cc], (unsigned long long)v);
    }
}

// 3D (particles binned by tile): one CTA per tile of the run.  A tile covers at most 8 x 8
// coarse columns.  Per species, in rounds of up to RB particles of the tile's list, the CTA
// sorts the particles' indices by column in shared memory (a counting sort), then walks the
// columns: each thread adds its share of a column's particles to registers, and each warp adds
// its column sums (a shuffle reduction) to the tile's shared accumulators; the tile adds its
// nonzero sums to psum at the end.
constexpr int RB = 4096;
template <int PASS>
__global__ void __launch_bounds__(NT, PASS == 1 ? 3 : 2) mom_tiles(const MomArgs m) {
    constexpr int B = PassRows<PASS>::base, NR = PassRows<PASS>::n;
    constexpr int MAXC = 64;
    __shared__ unsigned long long sacc[MAXC][NR];
    __shared__ unsigned short idx[RB];
    __shared__ int cstart[MAXC + 1], cfill[MAXC];
    const Args& a = m.a;
    const RunDev& R = a.runs[m.run];
    const long long T = R.work_off + blockIdx.x;
    const int t = blockIdx.x;
    const int x0 = (t % R.ntx) * a.tx, y0 = ((t / R.ntx) % R.nty) * a.ty, z0 = (t / (R.ntx * R.nty)) * a.tz;
    const int cx0 = x0 / m.bx, cy0 = y0 / m.by;
    const int ncxl = (x0 + a.tx - 1) / m.bx - cx0 + 1, ncyl = (y0 + a.ty - 1) / m.by - cy0 + 1;
    const int ncl = ncxl * ncyl;   // <= 64: a tile is at most 8 cells wide
    for (int i = threadIdx.x; i < ncl * NR; i += NT) (&sacc[0][0])[i] = 0ull;
    const int par = a.ctl->parity;
    // tile sides are powers of two (the host checks): the in-tile cell decodes with shifts
    const int lgx = __ffs(a.tx) - 1, lgy = __ffs(a.ty) - 1;
    const int cmask = a.tx * a.ty * a.tz - 1;
    const int lane = threadIdx.x & 31;
    auto column = [&](int lc) {
        const int cx = x0 + (lc & (a.tx - 1)), cy = y0 + ((lc >> lgx) & (a.ty - 1));
        return (cy / m.by - cy0) * ncxl + (cx / m.bx - cx0);
    };
    for (int s = 0; s < a.nspecies && s < 2; ++s) {
        if (!R.sp[s].active) continue;
        const Slots& S = a.slot[s][par];
        const CellRange cr = cell_range(S, a.cap[s], a.cap_stay[s], T);
        const float w = R.sp[s].w;
        for (int r0 = 0; r0 < cr.n; r0 += RB) {
            const int nr = min(RB, cr.n - r0);
            __syncthreads();   // idx and the column counts of the previous round are free
            for (int i = threadIdx.x; i < ncl; i += NT) cfill[i] = 0;
            __syncthreads();
            for (int i = threadIdx.x; i < nr; i += NT) {
                const size_t q = slot_elt(S, (long long)slot_of(T, a.cap[s], a.cap_stay[s], cr.ns, r0 + i));
                atomicAdd(&cfill[column(S.lc[q] & cmask)], 1);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int run = 0;
                for (int c = 0; c < ncl; ++c) {
                    cstart[c] = run;
                    run += cfill[c];
                    cfill[c] = cstart[c];
                }
                cstart[ncl] = run;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < nr; i += NT) {
                const size_t q = slot_elt(S, (long long)slot_of(T, a.cap[s], a.cap_stay[s], cr.ns, r0 + i));
                idx[atomicAdd(&cfill[column(S.lc[q] & cmask)], 1)] = (unsigned short)i;
            }
            __syncthreads();
            for (int c = 0; c < ncl; ++c) {
                const int e0 = cstart[c], e1 = cstart[c + 1];
                if (e0 == e1) continue;   // uniform: the CTA reads the same counts
                long long acc[NR];
#pragma unroll
                for (int k = 0; k < NR; ++k) acc[k] = 0;
                Mean2 mean{};
                const int ccx = cx0 + c % ncxl, ccy = cy0 + c / ncxl;
                if (PASS == 2) coarse_means(m, (long long)ccy * m.ncx + ccx, mean);
                for (int e = e0 + threadIdx.x; e < e1; e += NT) {
                    const size_t q = slot_elt(S, (long long)slot_of(T, a.cap[s], a.cap_stay[s], cr.ns, r0 + idx[e]));
                    const int lc = S.lc[q] & cmask;
                    const int cx = x0 + (lc & (a.tx - 1)), cy = y0 + ((lc >> lgx) & (a.ty - 1));
                    const int cz = z0 + (lc >> (lgx + lgy));
                    add_particle<PASS>(m, R, s, w, mean, cx, cy, cz, S.o[0][q], S.o[1][q], S.o[2][q],
                                       S.u[0][q], S.u[1][q], S.u[2][q], acc);
                }
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    long long v = acc[k];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0 && v != 0) atomicAdd(&sacc[c][k], (unsigned long long)v);
                }
            }
        }
    }
    __syncthreads();
    const long long nc = (long long)m.ncx * m.ncy;
    for (int i = threadIdx.x; i < ncl * NR; i += NT) {
        const int cl = i / NR, k = i - cl * NR;
        const unsigned long long v = sacc[cl][k];
        if (v) {
            const long long cc = (long long)(cy0 + cl / ncxl) * m.ncx + (cx0 + cl % ncxl);
            atomicAdd((unsigned long long*)&m.psum[(size_t)(B + k) * nc + cc], v);
        }
    }
}

// Spilled particles of the run (thread each).
template <int PASS>
__global__ void __launch_bounds__(NT) mom_spill(const MomArgs m) {
    constexpr int B = PassRows<PASS>::base, NR = PassRows<PASS>::n;
    const Args& a = m.a;
    const RunDev& R = a.runs[m.run];
    const int par = a.ctl->parity;
    const long long nc = (long long)m.ncx * m.ncy;
    for (int s = 0; s < a.nspecies && s < 2; ++s) {
        const Slots& S = a.slot[s][par];
        const int ns = min(*S.sn, a.spill_cap[s]);
        for (int k = blockIdx.x * NT + threadIdx.x; k < ns; k += gridDim.x * NT) {
            const long long g = S.scell[k];
            const long long lc = g - R.cell_off;
            if (lc < 0 || lc >= (long long)R.nx * R.ny * R.nz) continue;
            const int cz = (int)(lc / ((long long)R.nx * R.ny));
            const int rem = (int)(lc - (long long)cz * R.nx * R.ny);
            const int cy = rem / R.nx, cx = rem - cy * R.nx;
            long long acc[NR];
            for (int i = 0; i < NR; ++i) acc[i] = 0;
            const long long cc = (long long)(cy / m.by) * m.ncx + cx / m.bx;
            Mean2 mean{};
            if (PASS == 2) coarse_means(m, cc, mean);
            add_particle<PASS>(m, R, s, R.sp[s].w, mean, cx, cy, cz, S.so[0][k], S.so[1][k],
                               a.ndim == 3 ? S.so[2][k] : 0.f, S.su[0][k], S.su[1][k], S.su[2][k], acc);
            for (int i = 0; i < NR; ++i)
                if (acc[i]) atomicAdd((unsigned long long*)&m.psum[(size_t)(B + i) * nc + cc], (unsigned long long)acc[i]);
        }
    }
}

// Per (x, y) column: mean over z of sum_c (E_c - <E_c>_z)^2, and the z means of Ez, Bx, By.
__global__ void __launch_bounds__(NT) mom_columns(const MomArgs m) {
    const RunDev& R = m.a.runs[m.run];
    const long long ncol = (long long)R.nx * R.ny;
    const int nz = m.a.ndim == 3 ? R.nz : 1;
    for (long long c = blockIdx.x * (long long)NT + threadIdx.x; c < ncol; c += (long long)gridDim.x * NT) {
        double mean[3] = {0, 0, 0}, bx = 0, by = 0;
        for (int k = 0; k < nz; ++k) {
            const size_t g = (size_t)k * ncol + c;
            for (int d = 0; d < 3; ++d) mean[d] += R.E[d][g];
            bx += R.B[0][g];
            by += R.B[1][g];
        }
        for (int d = 0; d < 3; ++d) mean[d] /= nz;
        double w = 0;
        for (int k = 0; k < nz; ++k) {
            const size_t g = (size_t)k * ncol + c;
            for (int d = 0; d < 3; ++d) {
                const double e = (double)R.E[d][g] - mean[d];
                w += e * e;
            }
        }
        m.col[c] = w / nz;
        m.col[ncol + c] = mean[2];
        m.col[2 * ncol + c] = bx / nz;
        m.col[3 * ncol + c] = by / nz;
    }
}

__global__ void __launch_bounds__(NT) mom_finalize(const MomArgs m) {
    const RunDev& R = m.a.runs[m.run];
    const long long nc = (long long)m.ncx * m.ncy;
    const long long ncol = (long long)R.nx * R.ny;
    const int nz = m.a.ndim == 3 ? R.nz : 1;
    const double cells = (double)m.bx * m.by * nz;
    for (long long cc = blockIdx.x * (long long)NT + threadIdx.x; cc < nc; cc += (long long)gridDim.x * NT) {
        double p[MOM_PSUMS];
        for (int i = 0; i < MOM_PSUMS; ++i) p[i] = (double)m.psum[(size_t)i * nc + cc] / MOM_FIX;
        float* o = m.out;
        for (int s = 0; s < 2; ++s) {
            const double sw = p[4 * s];
            double mu[3] = {0, 0, 0}, var[3] = {0, 0, 0};
            if (sw > 0)
                for (int d = 0; d < 3; ++d) {
                    mu[d] = p[4 * s + 1 + d] / sw;
                    var[d] = p[8 + 3 * s + d] / sw;
                }
            o[(size_t)s * nc + cc] = (float)(sw / cells);
            o[(size_t)(2 + s) * nc + cc] = (float)mu[2];
            o[(size_t)(4 + 2 * s) * nc + cc] = (float)(0.5 * (var[0] + var[1]));
            o[(size_t)(5 + 2 * s) * nc + cc] = (float)var[2];
        }
        // field blocks, fixed order
        const int X0 = (int)(cc % m.ncx) * m.bx, Y0 = (int)(cc / m.ncx) * m.by;
        double f[MOM_COLS] = {0, 0, 0, 0};
        for (int j = 0; j < m.by; ++j)
            for (int i = 0; i < m.bx; ++i) {
                const long long c = (long long)(Y0 + j) * R.nx + (X0 + i);
                for (int k = 0; k < MOM_COLS; ++k) f[k] += m.col[(size_t)k * ncol + c];
            }
        for (int k = 0; k < MOM_COLS; ++k) f[k] /= (double)(m.bx * m.by);
        o[(size_t)8 * nc + cc] = (float)f[0];
        const double sw = p[4];
        double fzp = 0, vx = 0, vy = 0, uz = 0;
        if (sw > 0) {
            fzp = p[14] / sw;
            vx = p[15] / sw;
            vy = p[16] / sw;
            uz = p[7] / sw;
        }
        const double fzm = (double)m.q_bg * (f[1] + vx * f[3] - vy * f[2]);
        o[(size_t)9 * nc + cc] = (float)fzp;
        o[(size_t)10 * nc + cc] = (float)fzm;
        o[(size_t)11 * nc + cc] = uz != 0 ? (float)((double)m.nu_bg + (fzm - fzp) / uz) : 0.f;
    }
}

int grid_of(long long n) {
    long long g = (n + NT - 1) / NT;
    if (g > 152 * 32) g = 152 * 32;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

size_t moments_scratch_bytes(long long nc, long long ncol) {
    return (size_t)nc * MOM_PSUMS * sizeof(long long) + (size_t)ncol * MOM_COLS * sizeof(double) +
           (size_t)nc * 12 * sizeof(float);
}

cudaError_t launch_moments(const Args& a, const RunDev& host_run, int run, int bx, int by, float q_bg,
                           float nu_bg, float* out, void* scratch, cudaStream_t s) {
    auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
    if (a.ndim == 3 && !(pow2(a.tx) && pow2(a.ty) && pow2(a.tz))) return cudaErrorInvalidValue;
    MomArgs m;
    m.a = a;
    m.run = run;
    m.bx = bx;
    m.by = by;
    m.ncx = host_run.nx / bx;
    m.ncy = host_run.ny / by;
    const int nz = a.ndim == 3 ? host_run.nz : 1;
    const int per = bx * by;
    m.zc = per >= NT ? 1 : (NT / per < nz ? NT / per : nz);
    m.q_bg = q_bg;
    m.nu_bg = nu_bg;
    const long long nc = (long long)m.ncx * m.ncy;
    m.psum = static_cast<long long*>(scratch);
    m.col = reinterpret_cast<double*>(m.psum + (size_t)nc * MOM_PSUMS);
    m.meanbuf = reinterpret_cast<float*>(m.col + (size_t)host_run.nx * host_run.ny * MOM_COLS);
    m.out = out;
    cudaError_t e = cudaMemsetAsync(m.psum, 0, (size_t)nc * MOM_PSUMS * sizeof(long long), s);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)nc, (unsigned)((nz + m.zc - 1) / m.zc));
    const unsigned tgrid = (unsigned)host_run.ntx * host_run.nty * host_run.ntz;
    if (a.ndim == 3) mom_tiles<1><<<tgrid, NT, 0, s>>>(m);
    else mom_particles<1><<<grid, NT, 0, s>>>(m);
    mom_spill<1><<<152, NT, 0, s>>>(m);
    mom_means<<<grid_of(nc), NT, 0, s>>>(m);
    if (a.ndim == 3) mom_tiles<2><<<tgrid, NT, 0, s>>>(m);
    else mom_particles<2><<<grid, NT, 0, s>>>(m);
    mom_spill<2><<<152, NT, 0, s>>>(m);
    mom_columns<<<grid_of((long long)host_run.nx * host_run.ny), NT, 0, s>>>(m);
    mom_finalize<<<grid_of(nc), NT, 0, s>>>(m);
    return cudaGetLastError();
}

cudaError_t preload_moments() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, mom_particles<1>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, mom_particles<2>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, mom_tiles<1>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, mom_tiles<2>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, mom_spill<1>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, mom_spill<2>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, mom_means);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, mom_columns);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, mom_finalize);
    return e;
}

}  // namespace pic
