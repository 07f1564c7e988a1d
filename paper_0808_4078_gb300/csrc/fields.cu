// fields.cu -- Yee FDTD update, drag-moment finalisation, diagnostics records, growth fit,
// particle validation.
//
// Yee step (periodic):  B^n -> B^{n+1/2}: B -= (dt/2) curl E;  E^{n+1} = E^n + dt (curl B - J);
// B^{n+1/2} -> B^{n+1}: B -= (dt/2) curl E.  J is the int64 fixed-point current of the step,
// converted with 2^-S and cleared after use.  The E kernel also turns the drag moments
// accumulated by the push (sum u, count per cell) into the cell-mean momentum <u> for the next
// step's Krook drag (Eq. (3) friction) and clears the accumulators.
#include <cfloat>
#include <cmath>

#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int NT = 256;

// ------------------------------------------------------------------ Yee cells
// E update of one cell (2D or 3D): curl B from the backward neighbours (offsets dxm, dym, dzm;
// dzm = 0 in 2D), the step's current (int64 fixed point, cleared after use, kept in Jlast on
// request) and the drag-moment finalisation.  Every pointer is read from the run table before
// the first store: otherwise each store could alias the table and force the pointers to be
// reloaded from memory in a dependent chain.
__device__ __forceinline__ void e_cell(const RunDev& R, long long c, long long dxm, long long dym, long long dzm,
                                       float dt) {
    float* __restrict__ Ex = R.E[0];
    float* __restrict__ Ey = R.E[1];
    float* __restrict__ Ez = R.E[2];
    const float* __restrict__ Bx = R.B[0];
    const float* __restrict__ By = R.B[1];
    const float* __restrict__ Bz = R.B[2];
    long long* __restrict__ J0 = R.J[0];
    long long* __restrict__ J1 = R.J[1];
    long long* __restrict__ J2 = R.J[2];
    long long* __restrict__ L0 = R.Jlast[0];
    long long* __restrict__ L1 = R.Jlast[1];
    long long* __restrict__ L2 = R.Jlast[2];
    long long* __restrict__ M0 = R.msum[0];
    long long* __restrict__ M1 = R.msum[1];
    long long* __restrict__ M2 = R.msum[2];
    int* __restrict__ MC = R.mcnt;
    float* __restrict__ U0 = R.ubar[0];
    float* __restrict__ U1 = R.ubar[1];
    float* __restrict__ U2 = R.ubar[2];
    const long long* __restrict__ F0 = R.Jf[0];
    const long long* __restrict__ F1 = R.Jf[1];
    const long long* __restrict__ F2 = R.Jf[2];
    const float cx = R.cx, cy = R.cy, cz = R.cz;
    const float js = (F0 ? R.jfscale : R.jscale) * dt;
    const long long j0 = J0[c], j1 = J1[c], j2 = J2[c];
    const long long u0 = F0 ? F0[c] : j0, u1 = F0 ? F1[c] : j1, u2 = F0 ? F2[c] : j2;
    const float bx = Bx[c], by = By[c], bz = Bz[c];
    const float bz_ym = Bz[c - dym], bz_xm = Bz[c - dxm], by_xm = By[c - dxm], bx_ym = Bx[c - dym];
    const float by_zm = dzm ? By[c - dzm] : by, bx_zm = dzm ? Bx[c - dzm] : bx;
    const float ex = Ex[c], ey = Ey[c], ez = Ez[c];
    // the drag moments are loaded with the rest, before the first store (one round trip)
    const int cnt = M0 ? MC[c] : 0;
    const long long m0 = M0 ? M0[c] : 0, m1 = M0 ? M1[c] : 0, m2 = M0 ? M2[c] : 0;
    const float jx = (float)u0 * js, jy = (float)u1 * js, jz = (float)u2 * js;
    J0[c] = 0; J1[c] = 0; J2[c] = 0;
    if (L0) { L0[c] = j0; L1[c] = j1; L2[c] = j2; }
    Ex[c] = ex + (cy * (bz - bz_ym) - cz * (by - by_zm) - jx);
    Ey[c] = ey + (cz * (bx - bx_zm) - cx * (bz - bz_xm) - jy);
    Ez[c] = ez + (cx * (by - by_xm) - cy * (bx - bx_ym) - jz);
    if (M0) {
        const float inv = cnt > 0 ? 1.0f / (float)cnt : 0.f;
        const float sc = inv * (1.0f / 1048576.0f);
        U0[c] = (float)m0 * sc;
        U1[c] = (float)m1 * sc;
        U2[c] = (float)m2 * sc;
        M0[c] = 0; M1[c] = 0; M2[c] = 0;
        MC[c] = 0;
    }
}

// B half step of one cell from the forward neighbours (dzp = 0 in 2D), pointers read first.
__device__ __forceinline__ void b_cell(const RunDev& R, long long c, long long dxp, long long dyp, long long dzp) {
    const float* __restrict__ Ex = R.E[0];
    const float* __restrict__ Ey = R.E[1];
    const float* __restrict__ Ez = R.E[2];
    float* __restrict__ Bx = R.B[0];
    float* __restrict__ By = R.B[1];
    float* __restrict__ Bz = R.B[2];
    const float hx = 0.5f * R.cx, hy = 0.5f * R.cy, hz = 0.5f * R.cz;
    const float ex = Ex[c], ey = Ey[c], ez = Ez[c];
    const float ez_yp = Ez[c + dyp], ez_xp = Ez[c + dxp], ey_xp = Ey[c + dxp], ex_yp = Ex[c + dyp];
    const float ey_zp = dzp ? Ey[c + dzp] : ey, ex_zp = dzp ? Ex[c + dzp] : ex;
    const float bx = Bx[c], by = By[c], bz = Bz[c];
    Bx[c] = bx - (hy * (ez_yp - ez) - hz * (ey_zp - ey));
    By[c] = by - (hz * (ex_zp - ex) - hx * (ez_xp - ez));
    Bz[c] = bz - (hx * (ey_xp - ey) - hy * (ex_yp - ex));
}

// Tile-batched 2D Yee over the (run, tile) work list: one CTA per tile of a.tx x a.ty = 256
// cells (the particle kernel's tile shape), a thread per cell, every run of a batch in one launch.

__global__ void __launch_bounds__(NT) yee_b_half_2d_tiles(Args a) {
    const int2 wk = a.work[blockIdx.x];
    const RunDev& R = a.runs[wk.x];
    const int nx = R.nx, ny = R.ny;
    const int i = (wk.y % R.ntx) * a.tx + threadIdx.x % a.tx;
    const int j = (wk.y / R.ntx) * a.ty + threadIdx.x / a.tx;
    const long long dxp = i + 1 == nx ? -(long long)(nx - 1) : 1;
    const long long dyp = j + 1 == ny ? -(long long)(ny - 1) * nx : nx;
    b_cell(R, (long long)j * nx + i, dxp, dyp, 0);
}

__global__ void __launch_bounds__(NT) yee_e_2d_tiles(Args a, float dt) {
    const int2 wk = a.work[blockIdx.x];
    const RunDev& R = a.runs[wk.x];
    const int nx = R.nx, ny = R.ny;
    const int i = (wk.y % R.ntx) * a.tx + threadIdx.x % a.tx;
    const int j = (wk.y / R.ntx) * a.ty + threadIdx.x / a.tx;
    const long long dxm = i == 0 ? -(long long)(nx - 1) : 1;
    const long long dym = j == 0 ? -(long long)(ny - 1) * nx : nx;
    e_cell(R, (long long)j * nx + i, dxm, dym, 0, dt);
}

// ------------------------------------------------------------------ current filter
// Binomial 1-2-1 pass per axis (periodic) of the three current components, as one 3^ndim
// stencil with integer weights (1, 2, 1) x (1, 2, 1) [x (1, 2, 1)]: exact in int64; the E update
// scales by 4^-ndim.  Reads J at the neighbours, so it runs as its own kernel before the E update
// (which clears J).
__device__ __forceinline__ long long row121(const long long* __restrict__ J, long long c, long long dxm, long long dxp) {
    return J[c - dxm] + 2 * J[c] + J[c + dxp];
}

__global__ void __launch_bounds__(NT) jfilter_2d_tiles(Args a) {
    const int2 wk = a.work[blockIdx.x];
    const RunDev& R = a.runs[wk.x];
    const int nx = R.nx, ny = R.ny;
    const int i = (wk.y % R.ntx) * a.tx + threadIdx.x % a.tx;
    const int j = (wk.y / R.ntx) * a.ty + threadIdx.x / a.tx;
    const long long c = (long long)j * nx + i;
    const long long dxm = i == 0 ? -(long long)(nx - 1) : 1;
    const long long dxp = i + 1 == nx ? -(long long)(nx - 1) : 1;
    const long long dym = j == 0 ? -(long long)(ny - 1) * nx : nx;
    const long long dyp = j + 1 == ny ? -(long long)(ny - 1) * nx : nx;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const long long* __restrict__ J = R.J[d];
        R.Jf[d][c] = row121(J, c - dym, dxm, dxp) + 2 * row121(J, c, dxm, dxp) + row121(J, c + dyp, dxm, dxp);
    }
}

// ------------------------------------------------------------------ 3D Yee
// Thread per cell on a 3D launch grid (32 x 8 threads per block along x, y; one z plane per
// block row), so no index division; neighbours come through L1/L2.
constexpr int Y3X = 32, Y3Y = 8;

__global__ void __launch_bounds__(Y3X * Y3Y) yee_b_half_3d(const RunDev* __restrict__ runs, int run) {
    const RunDev& R = runs[run];
    const int nx = R.nx, ny = R.ny, nz = R.nz;
    const int i = blockIdx.x * Y3X + threadIdx.x, j = blockIdx.y * Y3Y + threadIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const long long nxy = (long long)nx * ny;
    const long long dxp = (i + 1 == nx ? -(long long)(nx - 1) : 1);
    const long long dyp = (j + 1 == ny ? -(long long)(ny - 1) * nx : nx);
    const long long dzp = (k + 1 == nz ? -(long long)(nz - 1) * nxy : nxy);
    b_cell(R, k * nxy + (long long)j * nx + i, dxp, dyp, dzp);
}

__global__ void __launch_bounds__(Y3X * Y3Y) yee_e_3d(const RunDev* __restrict__ runs, int run, float dt) {
    const RunDev& R = runs[run];
    const int nx = R.nx, ny = R.ny, nz = R.nz;
    const int i = blockIdx.x * Y3X + threadIdx.x, j = blockIdx.y * Y3Y + threadIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const long long nxy = (long long)nx * ny;
    const long long dxm = (i == 0 ? -(long long)(nx - 1) : 1);
    const long long dym = (j == 0 ? -(long long)(ny - 1) * nx : nx);
    const long long dzm = (k == 0 ? -(long long)(nz - 1) * nxy : nxy);
    e_cell(R, k * nxy + (long long)j * nx + i, dxm, dym, dzm, dt);
}

__global__ void __launch_bounds__(Y3X * Y3Y) jfilter_3d(const RunDev* __restrict__ runs, int run) {
    const RunDev& R = runs[run];
    const int nx = R.nx, ny = R.ny, nz = R.nz;
    const int i = blockIdx.x * Y3X + threadIdx.x, j = blockIdx.y * Y3Y + threadIdx.y, k = blockIdx.z;
    if (i >= nx) return;
    const long long nxy = (long long)nx * ny;
    const long long c = k * nxy + (long long)j * nx + i;
    const long long dxm = i == 0 ? -(long long)(nx - 1) : 1;
    const long long dxp = i + 1 == nx ? -(long long)(nx - 1) : 1;
    const long long dym = j == 0 ? -(long long)(ny - 1) * nx : nx;
    const long long dyp = j + 1 == ny ? -(long long)(ny - 1) * nx : nx;
    const long long dzm = k == 0 ? -(long long)(nz - 1) * nxy : nxy;
    const long long dzp = k + 1 == nz ? -(long long)(nz - 1) * nxy : nxy;
    for (int d = 0; d < 3; ++d) {
        const long long* __restrict__ J = R.J[d];
        auto plane = [&](long long cc) {
            return row121(J, cc - dym, dxm, dxp) + 2 * row121(J, cc, dxm, dxp) + row121(J, cc + dyp, dxm, dxp);
        };
        R.Jf[d][c] = plane(c - dzm) + 2 * plane(c) + plane(c + dzp);
    }
}

// Moments -> <u> without a field update (after loading particles).
__global__ void moments_finalize_kernel(const RunDev* __restrict__ runs, int run) {
    const RunDev& R = runs[run];
    if (!R.msum[0]) return;
    const long long n = (long long)R.nx * R.ny * R.nz;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const int cnt = R.mcnt[c];
        const float inv = cnt > 0 ? 1.0f / (float)cnt : 0.f;
        const float sc = inv * (1.0f / 1048576.0f);
        for (int q = 0; q < 3; ++q) {
            R.ubar[q][c] = (float)R.msum[q][c] * sc;
            R.msum[q][c] = 0;
        }
        R.mcnt[c] = 0;
    }
}

// Drag moments of the loaded particles of species s in units [u0, u0 + nu) of run `run` (NGP
// cell = the particle's cell), current buffer, and the run's spill entries.
__global__ void moments_init_kernel(Args a, int s, int run, long long u0, long long nu) {
    const RunDev& R = a.runs[run];
    if (!R.sp[s].drag || !R.msum[0]) return;
    const Slots S = a.slot[s][a.ctl->parity];
    const int cap = a.cap[s], cs = a.cap_stay[s];
    const float ms = 1048576.0f;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nu;
         k += (long long)gridDim.x * blockDim.x) {
        const long long c = u0 + k;
        const CellRange cr = cell_range(S, cap, cs, c);
        if (S.lc) {
            // 3D: a tile; each particle adds to its own cell
            for (int i = 0; i < cr.n; ++i) {
                const size_t q = slot_elt(S, (long long)slot_of(c, cap, cs, cr.ns, i));
                const long long lc = cell_of_unit(a, R, c, S.lc[q]) - R.cell_off;
                for (int d = 0; d < 3; ++d)
                    atomicAdd((unsigned long long*)&R.msum[d][lc], (unsigned long long)__float2ll_rn(S.u[d][q] * ms));
                atomicAdd(&R.mcnt[lc], 1);
            }
            continue;
        }
        long long m[3] = {0, 0, 0};
        for (int i = 0; i < cr.n; ++i)
            for (int d = 0; d < 3; ++d) m[d] += __float2ll_rn(S.u[d][slot_elt(S, (long long)slot_of(c, cap, cs, cr.ns, i))] * ms);
        const long long lc = c - R.cell_off;
        for (int d = 0; d < 3; ++d) atomicAdd((unsigned long long*)&R.msum[d][lc], (unsigned long long)m[d]);
        atomicAdd(&R.mcnt[lc], cr.n);
    }
    const long long c0 = R.cell_off, nc = (long long)R.nx * R.ny * R.nz;
    const int ns = min(*S.sn, a.spill_cap[s]);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ns; k += gridDim.x * blockDim.x) {
        const long long c = S.scell[k];
        if (c < c0 || c >= c0 + nc) continue;
        const long long lc = c - R.cell_off;
        for (int d = 0; d < 3; ++d)
            atomicAdd((unsigned long long*)&R.msum[d][lc], (unsigned long long)__float2ll_rn(S.su[d][k] * ms));
        atomicAdd(&R.mcnt[lc], 1);
    }
}

// ------------------------------------------------------------------ step finalisation
// One block per run: on diagnostic steps reduce the run's per-CTA field-energy partials in a
// fixed order (deterministic FP64), convert its int64 kinetic/momentum sums and write one
// history record.  Then `advance_kernel` moves the step counter and flips the particle buffer.
__global__ void __launch_bounds__(NT) finalize_kernel(Args a) {
    __shared__ double red[NT][6];
    const int run = blockIdx.x;
    const long long step = a.ctl->step;
    const bool diag = a.diag_interval > 0 && (step % a.diag_interval) == 0;
    if (!diag) return;
    const int w0 = a.work_off[run], w1 = a.work_off[run + 1];
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int w = w0 + threadIdx.x; w < w1; w += NT)
        for (int c = 0; c < 6; ++c) s[c] += a.partials[(size_t)w * 8 + c];
    for (int c = 0; c < 6; ++c) red[threadIdx.x][c] = s[c];
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int c = 0; c < 6; ++c) red[threadIdx.x][c] += red[threadIdx.x + o][c];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long r = step / a.diag_interval;
        DiagRec& d = a.hist[(size_t)run * a.hist_cap + r % a.hist_cap];
        d.step = step;
        d.t = (double)step * a.dt;
        for (int c = 0; c < 3; ++c) {
            d.WE[c] = red[0][c] * a.dV;
            d.WB[c] = red[0][3 + c] * a.dV;
        }
        const double sc = a.dV / 4294967296.0;
        long long* K = a.kin + (size_t)run * PIC_NS * 4;
        double P[3] = {0, 0, 0};
        for (int sp = 0; sp < PIC_NS; ++sp) {
            d.Ekin[sp] = (double)K[sp * 4 + 0] * sc;
            for (int c = 0; c < 3; ++c) P[c] += (double)K[sp * 4 + 1 + c] * sc;
            for (int c = 0; c < 4; ++c) K[sp * 4 + c] = 0;
        }
        for (int c = 0; c < 3; ++c) d.P[c] = P[c];
        d.flags = a.ctl->err;
        d.reserved = 0;
    }
}

__global__ void advance_kernel(Ctl* ctl) {
    ctl->step += 1;
    ctl->parity ^= 1;          // the particles now live in the other buffer
}

// ------------------------------------------------------------------ growth fit (FP64)
// Records are in ring order starting at record index first.  Windows of `width` consecutive
// records with all W in (lo, hi); least-squares slope of ln W; the largest slope wins.
__global__ void __launch_bounds__(NT) fit_kernel(const DiagRec* __restrict__ hist, int cap,
                                                 long long first, int nrec, int width,
                                                 double t_noise, double start_factor,
                                                 double end_factor, double* out) {
    __shared__ double s_noise[NT], s_cnt[NT], s_max[NT];
    __shared__ double s_best[NT];
    __shared__ int s_bi[NT];
    auto W = [&](int r) {
        const DiagRec& d = hist[(first + r) % cap];
        return d.WB[0] + d.WB[1];
    };
    auto T = [&](int r) { return hist[(first + r) % cap].t; };
    double sn = 0, cn = 0, mx = -DBL_MAX;
    for (int r = threadIdx.x; r < nrec; r += NT) {
        const double w = W(r);
        if (T(r) <= t_noise) { sn += w; cn += 1; }
        mx = fmax(mx, w);
    }
    s_noise[threadIdx.x] = sn; s_cnt[threadIdx.x] = cn; s_max[threadIdx.x] = mx;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s_noise[threadIdx.x] += s_noise[threadIdx.x + o];
            s_cnt[threadIdx.x] += s_cnt[threadIdx.x + o];
            s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + o]);
        }
        __syncthreads();
    }
    const double lo = s_cnt[0] > 0 ? start_factor * s_noise[0] / s_cnt[0] : DBL_MAX;
    const double hi = end_factor > 0 ? end_factor * s_max[0] : DBL_MAX;
    double best = -DBL_MAX;
    int bi = -1;
    for (int a0 = threadIdx.x; a0 + width <= nrec; a0 += NT) {
        bool ok = s_cnt[0] > 0;
        double st = 0, sy = 0;
        for (int r = a0; r < a0 + width && ok; ++r) {
            const double w = W(r);
            ok = w > lo && w < hi;
            st += T(r);
            sy += log(w);
        }
        if (!ok) continue;
        const double tm = st / width, ym = sy / width;
        double num = 0, den = 0;
        for (int r = a0; r < a0 + width; ++r) {
            const double dt = T(r) - tm;
            num += dt * (log(W(r)) - ym);
            den += dt * dt;
        }
        const double slope = num / den;
        if (slope > best) { best = slope; bi = a0; }
    }
    s_best[threadIdx.x] = best; s_bi[threadIdx.x] = bi;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const double b2 = s_best[threadIdx.x + o];
            const int i2 = s_bi[threadIdx.x + o];
            // larger slope wins; ties go to the earlier window
            if (b2 > s_best[threadIdx.x] || (b2 == s_best[threadIdx.x] && i2 >= 0 &&
                                             (s_bi[threadIdx.x] < 0 || i2 < s_bi[threadIdx.x]))) {
                s_best[threadIdx.x] = b2;
                s_bi[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (s_bi[0] < 0) {
            out[0] = nan(""); out[1] = nan(""); out[2] = nan("");
        } else {
            out[0] = 0.5 * s_best[0];
            out[1] = T(s_bi[0]);
            out[2] = T(s_bi[0] + width - 1);
        }
    }
}

int grid_for(long long n) {
    long long g = (n + NT - 1) / NT;
    if (g > 152 * 32) g = 152 * 32;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t preload_fields() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, yee_b_half_2d_tiles);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, yee_b_half_3d);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, yee_e_3d);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, moments_finalize_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, moments_init_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, finalize_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fit_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, yee_b_half_2d_tiles);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, yee_e_2d_tiles);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, advance_kernel);
    return e;
}

cudaError_t launch_yee2d(const Args& a, const RunDev* host_runs, int, cudaStream_t s) {
    yee_b_half_2d_tiles<<<a.nwork, NT, 0, s>>>(a);
    if (host_runs[0].Jf[0]) jfilter_2d_tiles<<<a.nwork, NT, 0, s>>>(a);
    yee_e_2d_tiles<<<a.nwork, NT, 0, s>>>(a, (float)a.dt);
    yee_b_half_2d_tiles<<<a.nwork, NT, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_yee3d(const Args& a, const RunDev* host_runs, int nruns, cudaStream_t s) {
    for (int r = 0; r < nruns; ++r) {
        const RunDev& R = host_runs[r];
        const dim3 grid((R.nx + Y3X - 1) / Y3X, R.ny / Y3Y, R.nz), block(Y3X, Y3Y);
        yee_b_half_3d<<<grid, block, 0, s>>>(a.runs, r);
        if (R.Jf[0]) jfilter_3d<<<grid, block, 0, s>>>(a.runs, r);
        yee_e_3d<<<grid, block, 0, s>>>(a.runs, r, (float)a.dt);
        yee_b_half_3d<<<grid, block, 0, s>>>(a.runs, r);
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Args& a, cudaStream_t s) {
    finalize_kernel<<<a.nruns, NT, 0, s>>>(a);
    advance_kernel<<<1, 1, 0, s>>>(a.ctl);
    return cudaGetLastError();
}

cudaError_t launch_moments_init(const Args& a, int species, int run, long long u0, long long nu,
                                cudaStream_t s) {
    moments_init_kernel<<<grid_for(nu), NT, 0, s>>>(a, species, run, u0, nu);
    return cudaGetLastError();
}

cudaError_t launch_moments_finalize(const Args& a, int run, long long ncell, cudaStream_t s) {
    moments_finalize_kernel<<<grid_for(ncell), NT, 0, s>>>(a.runs, run);
    return cudaGetLastError();
}

namespace {
__global__ void drag_map_kernel(float* __restrict__ map, const float* __restrict__ nu, int nx, int ny,
                                long long n, int bx, int by, double dt) {
    const int ncx = nx / bx;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const long long col = c % ((long long)nx * ny);
        const int j = (int)(col / nx), i = (int)(col - (long long)j * nx);
        const float r = nu[(long long)(j / by) * ncx + i / bx];
        map[c] = r > 0.f ? (float)(-expm1(-(double)r * dt)) : 0.f;
    }
}
}  // namespace

cudaError_t launch_drag_map(const RunDev& R, float* map, const float* nu, int bx, int by, double dt, cudaStream_t s) {
    const long long n = (long long)R.nx * R.ny * R.nz;
    drag_map_kernel<<<grid_for(n), NT, 0, s>>>(map, nu, R.nx, R.ny, n, bx, by, dt);
    return cudaGetLastError();
}

cudaError_t launch_fit(const Args& a, int run, long long first, int nrec, int width, double t_noise,
                       double start_factor, double end_factor, double* out3, cudaStream_t s) {
    fit_kernel<<<1, NT, 0, s>>>(a.hist + (size_t)run * a.hist_cap, a.hist_cap, first, nrec, width,
                                t_noise, start_factor, end_factor, out3);
    return cudaGetLastError();
}

}  // namespace pic
