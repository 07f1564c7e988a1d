// hybrid.cu -- the paper's quasi-neutral hybrid model (Eqs. 1-6) on the GPU: a kinetic electron
// beam in the transverse plane, the plasma return current as a fluid, and the axial vector
// potential from Ampere's law without the displacement current.  Units: time 1/w_p, length c/w_p,
// velocity c, a = e A_z / (m c^2), densities n0.
//
//   Ampere (Eq. 2):        lap a = n_b beta_bz + n_p beta_p,   n_p = n0 - n_b (quasi-neutrality)
//   plasma (Eq. 3):        d beta_p / dt + nu beta_p = d a / dt
//   beam (Eq. 4):          d u_perp / dt = -(beta_z - beta_p) grad a
//   beam, axial (Eq. 6):   u_z = P + a, P conserved per particle
//
// One step (the discretisation is this library's reading; the paper gives none): push the beam at
// the old fields (CIC gather of a, of the gradient of its bilinear interpolant, and of beta_p),
// deposit its density and current at the new positions with the old a, then solve
//   (lap - n_p) a^{n+1} = n_b beta_b + n_p (beta_p^n - a^n - nu dt beta_p^n)
// with n_p = max(n0 - n_b, 0) per node, and update beta_p^{n+1} = beta_p^n + a^{n+1} - a^n -
// nu dt beta_p^n.
//
// Precision split for a part with little FP64 throughput: particles are FP32 (int32 cell plus
// FP32 offsets, as in the main engine), a and beta_p are FP64, and the variable-coefficient solve
// is mixed-precision refinement: the residual of a^n is formed in FP64, the correction
// d = a^{n+1} - a^n is solved in FP32 by conjugate gradients preconditioned with the exact inverse
// of the constant-density operator (lap - n_bar) -- a spectral solve by this file's own FP32
// radix-4 Stockham FFT in shared memory: forward transforms of the rows (fused into the kernels
// that produce the residual), a column pass on strips of 4 columns (forward, division, inverse),
// inverse transforms of the rows.  Beam density and current are exact integer sums, so they do
// not depend on particle order; every inner product is a fixed-order two-level sum (per-block
// partials, then the last block to finish adds them in block order), so a run is bitwise
// reproducible.  Every kernel of a CG iteration returns at once when the previous one found the
// residual below the tolerance; in a CUDA graph the iterations are the body of a while node that
// stops after convergence.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pic.h"
#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr double JFIX = 1099511627776.0;   // 2^40
constexpr int NT = 256;
constexpr int WIN = 256;                   // nodes per deposit window of the push
constexpr int RGRID = 8 * 152;             // blocks of the reducing node kernels (full occupancy)

// scalar slots of the solver state (device doubles)
enum { S_RR0 = 0, S_RZ, S_BETA, S_ALPHA, S_RR, S_DONE, S_ITER, S_ITERS_TOTAL, S_NOCONV, S_LAST_ITERS, S_LOOP, S_LOOPS_TOTAL, S_NSLOT };

struct HybDev {
    int nx, ny, lx;                 // lx = log2(nx)
    float dx, dy, dt, w;
    float idx, idy;                 // 1/dx, 1/dy (FP32)
    double dxd, dyd, dtd, n0, nu, tol2;
    double idx1, idy1, idx2, idy2;  // 1/dx, 1/dy, 1/dx^2, 1/dy^2 (FP64): no FP64 division on the device
    double keep;                    // 1 - nu dt
    long long n;
    // particles (and the second buffer the periodic sort permutes into)
    int* cell; float* ox; float* oy; float* ux; float* uy; float* P; int* id;
    int* cell2; float* ox2; float* oy2; float* ux2; float* uy2; float* P2; int* id2;
    int* order; int* start; int* bscratch;   // counting sort by cell
    float sfix;                     // 2^S32: per-particle deposit terms as int32 at this scale
    int sshift;                     // 40 - S32: int32 group sums shifted into the 2^40 grids
    long long* ebeam;               // fixed-point beam-energy partials
    // grid
    double* a; double* bp;          // [ny][nx]
    float2* f32;                    // (a, beta_p) in FP32 for the gather
    long long* J; long long* N;     // beam current and density, fixed point
    float* np;                      // plasma density of the current positions
    float* d; float* r; float* z; float* q; float* p0; float* p1;
    float2* ws0;                    // FFT work, [ny][nx]
    const float2* twx; const float2* twy;   // exp(-2 pi i m / N), m < N
    const float* lamx; const float* lamy;   // 5-point eigenvalues per axis
    float nbar;                     // preconditioner density
    double* S;                      // solver scalars
    double* part;                   // per-block partials
    unsigned* ticket;
};

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ---------------------------------------------------------------- FFT
// Stockham autosort passes over ncol columns held in shared memory (column c at b0 + c ld), all
// threads of the block taking part.  Radix-4 stages at span Ns: inputs j + r N/4 (r < 4) are
// twiddled by exp(sign 2 pi i r (j % Ns) / (4 Ns)) = tw[r (j % Ns) N / (4 Ns)] (conjugated for the
// inverse), combined by the 4-point DFT and written to (j / Ns) 4 Ns + (j % Ns) + r Ns; when
// log2 N is odd a last radix-2 stage (inputs j, j + N/2, outputs (j / Ns) 2 Ns + (j % Ns) + r Ns)
// completes the transform.  tw holds exp(-2 pi i m / N) for m < N.  Returns the buffer with the
// result.
__device__ __forceinline__ float2 twid(const float2* __restrict__ tw, int m, bool inverse) {
    const float2 t = tw[m];
    return inverse ? make_float2(t.x, -t.y) : t;
}
__device__ float2* fft_multi(float2* b0, float2* b1, int ncol, int ld, int N, int logn,
                             const float2* __restrict__ tw, bool inverse) {
    int Ns = 1, ls = 0;
    for (; ls + 2 <= logn; Ns <<= 2, ls += 2) {
        const int q = N >> 2, lq = logn - 2, sh = logn - 2 - ls;
        for (int t = threadIdx.x; t < ncol * q; t += blockDim.x) {
            const int c = t >> lq, j = t & (q - 1);
            const float2* x = b0 + c * ld;
            float2* y = b1 + c * ld;
            const int k = j & (Ns - 1);
            float2 v0 = x[j], v1 = x[j + q], v2 = x[j + 2 * q], v3 = x[j + 3 * q];
            if (k) {
                v1 = cmulf(v1, twid(tw, k << sh, inverse));
                v2 = cmulf(v2, twid(tw, (2 * k) << sh, inverse));
                v3 = cmulf(v3, twid(tw, (3 * k) << sh, inverse));
            }
            const float2 a0 = make_float2(v0.x + v2.x, v0.y + v2.y), a1 = make_float2(v0.x - v2.x, v0.y - v2.y);
            const float2 a2 = make_float2(v1.x + v3.x, v1.y + v3.y), a3 = make_float2(v1.x - v3.x, v1.y - v3.y);
            // -i a3 for the forward transform, +i a3 for the inverse
            const float2 ia3 = inverse ? make_float2(-a3.y, a3.x) : make_float2(a3.y, -a3.x);
            const int idx = ((j - k) << 2) + k;
            y[idx] = make_float2(a0.x + a2.x, a0.y + a2.y);
            y[idx + Ns] = make_float2(a1.x + ia3.x, a1.y + ia3.y);
            y[idx + 2 * Ns] = make_float2(a0.x - a2.x, a0.y - a2.y);
            y[idx + 3 * Ns] = make_float2(a1.x - ia3.x, a1.y - ia3.y);
        }
        __syncthreads();
        float2* t = b0; b0 = b1; b1 = t;
    }
    if (ls < logn) {
        const int half = N >> 1, lh = logn - 1;
        for (int t = threadIdx.x; t < ncol * half; t += blockDim.x) {
            const int c = t >> lh, j = t & (half - 1);
            const float2* x = b0 + c * ld;
            float2* y = b1 + c * ld;
            const int k = j & (Ns - 1);
            const float2 v0 = x[j];
            const float2 v1 = cmulf(x[j + half], twid(tw, k << (logn - 1 - ls), inverse));
            const int idx = ((j - k) << 1) + k;
            y[idx] = make_float2(v0.x + v1.x, v0.y + v1.y);
            y[idx + Ns] = make_float2(v0.x - v1.x, v0.y - v1.y);
        }
        __syncthreads();
        float2* t = b0; b0 = b1; b1 = t;
    }
    return b0;
}

// One row (N complex values) held in shared memory.
__device__ __forceinline__ float2* fft_smem(float2* b0, float2* b1, int N, int logn, const float2* __restrict__ tw,
                                            bool inverse) {
    return fft_multi(b0, b1, 1, N, N, logn, tw, inverse);
}

__device__ __forceinline__ bool solver_done(const HybDev& h) { return h.S[S_DONE] != 0.0; }

// Column pass of the spectral solve on a strip of CW columns of the row-major spectrum (ws0
// holds the rows' forward transforms): forward transforms along y, division by the eigenvalue of
// (lap - n_bar) with the 1/(nx ny) of the inverse, inverse transforms; in place.  A strip row of
// CW complex values is one 32-byte sector, so the strided access wastes no DRAM bandwidth and no
// transpose is needed.
constexpr int CW = 4;
constexpr int NTC = 512;   // threads of the column-strip kernel
__global__ void __launch_bounds__(NTC) fft_cols_strip_kernel(const HybDev h, int logny) {
    if (solver_done(h)) return;
    extern __shared__ float2 fsh[];
    const int N = h.ny, ld = N + 1, kx0 = blockIdx.x * CW;
    float2* b0 = fsh;
    float2* b1 = fsh + CW * ld;
    for (int e = threadIdx.x; e < CW * N; e += blockDim.x) {
        const int row = e / CW, c = e - row * CW;
        b0[c * ld + row] = h.ws0[((size_t)row << h.lx) + kx0 + c];
    }
    __syncthreads();
    float2* res = fft_multi(b0, b1, CW, ld, N, logny, h.twy, false);
    float2* oth = res == b0 ? b1 : b0;
    const float scale = 1.0f / ((float)h.nx * (float)h.ny);
    for (int e = threadIdx.x; e < CW * N; e += blockDim.x) {
        const int c = e >> logny, ky = e & (N - 1);
        const float inv = scale / (h.lamx[kx0 + c] + h.lamy[ky] - h.nbar);
        float2* v = res + c * ld + ky;
        *v = make_float2(v->x * inv, v->y * inv);
    }
    __syncthreads();
    const float2* out = fft_multi(res, oth, CW, ld, N, logny, h.twy, true);
    for (int e = threadIdx.x; e < CW * N; e += blockDim.x) {
        const int row = e / CW, c = e - row * CW;
        h.ws0[((size_t)row << h.lx) + kx0 + c] = out[c * ld + row];
    }
}

// ---------------------------------------------------------------- reductions
// Fixed-order sum of one double per thread over the grid: block partials in part[], the last
// block to arrive adds them in block order and calls fin(total) on thread 0.
template <class Fin>
__device__ __forceinline__ void grid_sum(const HybDev& h, double v, Fin fin) {
    __shared__ double red[NT];
    __shared__ bool last;
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        h.part[blockIdx.x] = red[0];
        __threadfence();
        last = atomicAdd(h.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += NT) s += ((volatile double*)h.part)[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *h.ticket = 0u;
        fin(red[0]);
    }
}

// The same for kernels with one CTA per grid row (blockDim up to 1024): block sums by 32
// strided partial sums then thread 0, row partials in part[], the last CTA adds them.
template <class Fin>
__device__ __forceinline__ void rows_sum(const HybDev& h, double v, Fin fin) {
    __shared__ double rs[1024];
    __shared__ double r32[32];
    __shared__ bool last;
    const int nw = blockDim.x < 32 ? (int)blockDim.x : 32;
    rs[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = 0.0;
        for (int t = threadIdx.x; t < (int)blockDim.x; t += 32) s += rs[t];
        r32[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int t = 0; t < nw; ++t) s += r32[t];
        h.part[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(h.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += ((volatile double*)h.part)[b];
    rs[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t2 = 0.0;
        for (int t = threadIdx.x; t < (int)blockDim.x; t += 32) t2 += rs[t];
        r32[threadIdx.x] = t2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int t = 0; t < nw; ++t) tot += r32[t];
        *h.ticket = 0u;
        fin(tot);
    }
}

// Forward transform of a row held in shared memory (nx complex values), stored to its ws0 row.
__device__ __forceinline__ void row_fft_store(const HybDev& h, float2* fsh, int j) {
    __syncthreads();
    const int N = h.nx;
    const float2* out = fft_smem(fsh, fsh + N, N, h.lx, h.twx, false);
    float2* row = h.ws0 + ((size_t)j << h.lx);
    for (int i = threadIdx.x; i < N; i += blockDim.x) row[i] = out[i];
}

// ---------------------------------------------------------------- particles
struct Node4 {
    int c00, c10, c01, c11;
    float fx, fy;
};
__device__ __forceinline__ Node4 nodes(const HybDev& h, int cell, float ox, float oy) {
    Node4 n;
    const int i = cell & (h.nx - 1), j = cell >> h.lx;
    const int i1 = (i + 1) & (h.nx - 1), j1 = j + 1 == h.ny ? 0 : j + 1;
    n.c00 = cell; n.c10 = (j << h.lx) + i1; n.c01 = (j1 << h.lx) + i; n.c11 = (j1 << h.lx) + i1;
    n.fx = ox; n.fy = oy;
    return n;
}

__device__ __forceinline__ void red_add(long long* p, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
}

// Push (move = 1) or only deposit (move = 0): gather, Eq. 4 and Eq. 6, move, and the CIC deposit
// of density w and current w beta_z at the new position with the old a.  The particles are kept
// in cell order by a periodic counting sort (they cross a cell in tens of steps), so a CTA's chunk
// of NT particles covers a few dozen neighbouring cells: its integer terms are summed with shared
// atomics in two windows of nodes (from the chunk's lowest cell, and one row up) whose nonzero
// entries are then added to the int64 grids; nodes outside the windows go straight to the grids.
__global__ void __launch_bounds__(NT) push_kernel(const HybDev h, int move) {
    // two node windows x (current, density), int32 at 2^S32
    __shared__ int win[4][WIN];
    __shared__ int wmins[NT / 32];
    for (int e = threadIdx.x; e < 4 * WIN; e += NT) (&win[0][0])[e] = 0;
    const long long stride = (long long)gridDim.x * NT;
    const int lane = threadIdx.x & 31;
    // block-uniform chunks of NT particles (the window passes below synchronise the block)
    for (long long base = blockIdx.x * (long long)NT; base < h.n; base += stride) {
        const long long p = base + threadIdx.x;
        const bool act = p < h.n;
        int cell = 0;
        float ox = 0.f, oy = 0.f, ux = 0.f, uy = 0.f, P = 0.f;
        if (act) {
            cell = h.cell[p];
            ox = h.ox[p]; oy = h.oy[p]; ux = h.ux[p]; uy = h.uy[p];
            P = h.P[p];
        }
        if (act && move) {
            const Node4 c = nodes(h, cell, ox, oy);
            const float2 f00 = h.f32[c.c00], f10 = h.f32[c.c10], f01 = h.f32[c.c01], f11 = h.f32[c.c11];
            const float gx0 = 1.0f - c.fx, gy0 = 1.0f - c.fy;
            const float av = gy0 * (gx0 * f00.x + c.fx * f10.x) + c.fy * (gx0 * f01.x + c.fx * f11.x);
            const float bpp = gy0 * (gx0 * f00.y + c.fx * f10.y) + c.fy * (gx0 * f01.y + c.fx * f11.y);
            const float gax = (gy0 * (f10.x - f00.x) + c.fy * (f11.x - f01.x)) * h.idx;
            const float gay = (gx0 * (f01.x - f00.x) + c.fx * (f11.x - f10.x)) * h.idy;
            const float uz = P + av;
            const float f = uz / sqrtf(1.0f + ux * ux + uy * uy + uz * uz) - bpp;
            ux = ux - h.dt * f * gax;
            uy = uy - h.dt * f * gay;
            const float ig2 = 1.0f / sqrtf(1.0f + ux * ux + uy * uy + uz * uz);
            ox = ox + h.dt * ux * ig2 * h.idx;
            oy = oy + h.dt * uy * ig2 * h.idy;
            int di = (int)floorf(ox), dj = (int)floorf(oy);
            ox -= (float)di; oy -= (float)dj;
            if (ox >= 1.0f) { ox -= 1.0f; ++di; }
            if (oy >= 1.0f) { oy -= 1.0f; ++dj; }
            di = max(-1, min(1, di));   // |beta| dt < dx: at most one cell; keeps indices in range
            dj = max(-1, min(1, dj));
            int i = (cell & (h.nx - 1)) + di, j = (cell >> h.lx) + dj;
            i &= h.nx - 1;
            j = j < 0 ? j + h.ny : (j >= h.ny ? j - h.ny : j);
            cell = (j << h.lx) + i;
            h.cell[p] = cell; h.ox[p] = ox; h.oy[p] = oy; h.ux[p] = ux; h.uy[p] = uy;
        }
        const Node4 c = nodes(h, cell, ox, oy);
        const float gx0 = 1.0f - c.fx, gy0 = 1.0f - c.fy;
        // per-particle terms as int32 at 2^S32 (exact integer sums from here on, so the grids do
        // not depend on particle order): density w S and current w beta_z S per node
        int v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (act) {
            const float av = gy0 * (gx0 * h.f32[c.c00].x + c.fx * h.f32[c.c10].x) +
                             c.fy * (gx0 * h.f32[c.c01].x + c.fx * h.f32[c.c11].x);
            const float uzs = P + av;
            const float q = uzs / sqrtf(1.0f + ux * ux + uy * uy + uzs * uzs);
            const float sw = h.w * h.sfix, sq = sw * q;
            const float w4[4] = {gx0 * gy0, c.fx * gy0, gx0 * c.fy, c.fx * c.fy};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                v[k] = __float2int_rn(sq * w4[k]);
                v[4 + k] = __float2int_rn(sw * w4[k]);
            }
        }
        // the chunk's lowest cell anchors two windows of nodes: [cmin, cmin + WIN) and the same
        // columns one row up; particles kept in cell order by the periodic sort land in them
        const int wmin = __reduce_min_sync(0xffffffffu, act ? cell : 0x7fffffff);
        if (lane == 0) wmins[threadIdx.x >> 5] = wmin;
        __syncthreads();
        int cmin = wmins[0];
#pragma unroll
        for (int wi = 1; wi < NT / 32; ++wi) cmin = min(cmin, wmins[wi]);
        if (act) {
            const int nd[4] = {c.c00, c.c10, c.c01, c.c11};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int o = nd[k] - cmin;
                int* slot = nullptr;
                if (o >= 0 && o < WIN) slot = &win[0][o];
                else if (o - h.nx >= 0 && o - h.nx < WIN) slot = &win[1][o - h.nx];
                if (slot) {
                    if (v[k]) atomicAdd(slot, v[k]);
                    if (v[4 + k]) atomicAdd(slot + 2 * WIN, v[4 + k]);
                } else {   // outside the windows: straight to the grids
                    if (v[k]) red_add(&h.J[nd[k]], (long long)v[k] << h.sshift);
                    if (v[4 + k]) red_add(&h.N[nd[k]], (long long)v[4 + k] << h.sshift);
                }
            }
        }
        __syncthreads();
        // flush the windows' nonzero entries and clear them for the next chunk
        for (int e = threadIdx.x; e < 2 * WIN; e += NT) {
            const int node = cmin + (e < WIN ? e : h.nx + e - WIN);
            int* wj = &win[0][0] + e;
            int* wn = wj + 2 * WIN;
            const int sj = *wj, sn = *wn;
            if (sj) { red_add(&h.J[node], (long long)sj << h.sshift); *wj = 0; }
            if (sn) { red_add(&h.N[node], (long long)sn << h.sshift); *wn = 0; }
        }
        __syncthreads();
    }
}

// Sort support: gather the particle arrays into the second buffer in cell order, then copy back.
__global__ void __launch_bounds__(NT) permute_kernel(const HybDev h) {
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < h.n; i += (long long)gridDim.x * NT) {
        const int q = h.order[i];
        h.cell2[i] = h.cell[q]; h.ox2[i] = h.ox[q]; h.oy2[i] = h.oy[q];
        h.ux2[i] = h.ux[q]; h.uy2[i] = h.uy[q]; h.P2[i] = h.P[q]; h.id2[i] = h.id[q];
    }
}
__global__ void __launch_bounds__(NT) copy_back_kernel(const HybDev h) {
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < h.n; i += (long long)gridDim.x * NT) {
        h.cell[i] = h.cell2[i]; h.ox[i] = h.ox2[i]; h.oy[i] = h.oy2[i];
        h.ux[i] = h.ux2[i]; h.uy[i] = h.uy2[i]; h.P[i] = h.P2[i]; h.id[i] = h.id2[i];
    }
}

// n_p from the deposited density (load only); clears J and N.
__global__ void __launch_bounds__(NT) density_kernel(const HybDev h) {
    const long long nc = (long long)h.nx * h.ny;
    for (long long c = blockIdx.x * (long long)NT + threadIdx.x; c < nc; c += (long long)gridDim.x * NT) {
        h.np[c] = (float)fmax(h.n0 - (double)h.N[c] / JFIX, 0.0);
        h.J[c] = 0; h.N[c] = 0;
    }
}

__device__ __forceinline__ double lap64(const HybDev& h, const double* F, int i, int j) {
    const int im = (i - 1) & (h.nx - 1), ip = (i + 1) & (h.nx - 1);
    const int jm = j == 0 ? h.ny - 1 : j - 1, jp = j + 1 == h.ny ? 0 : j + 1;
    const double f = F[(j << h.lx) + i];
    return (F[(j << h.lx) + ip] - 2.0 * f + F[(j << h.lx) + im]) * h.idx2 +
           (F[(jp << h.lx) + i] - 2.0 * f + F[(jm << h.lx) + i]) * h.idy2;
}

// n_p of the new positions; FP64 residual r0 = b - (lap - n_p) a^n of the initial guess; d = 0;
// <r0, r0> opens the solve; one CTA per row, which also applies the preconditioner's forward
// transform along x to its row of r0 (into ws0).
__global__ void rhs_rows_kernel(const HybDev h) {
    extern __shared__ float2 fsh[];
    const int j = blockIdx.x;
    float rr = 0.0f;   // a few nodes per thread in FP32, the rest of the sum in FP64
    for (int i = threadIdx.x; i < h.nx; i += blockDim.x) {
        const int c = (j << h.lx) + i;
        const double jb = (double)h.J[c] / JFIX, nb = (double)h.N[c] / JFIX;
        h.J[c] = 0; h.N[c] = 0;
        const float npf = (float)fmax(h.n0 - nb, 0.0);
        const double npd = (double)npf;
        h.np[c] = npf;
        // b - (lap - n_p) a^n with b = n_b beta_b + n_p (beta_p - a^n - nu dt beta_p): the n_p a^n
        // terms cancel
        const double r0 = jb + npd * (h.keep * h.bp[c]) - lap64(h, h.a, i, j);
        const float rf = (float)r0;
        h.r[c] = rf;
        h.d[c] = 0.0f;
        fsh[i] = make_float2(rf, 0.0f);
        rr = fmaf(rf, rf, rr);
    }
    row_fft_store(h, fsh, j);
    rows_sum(h, (double)rr, [&](double t) {
        h.S[S_RR0] = t; h.S[S_RR] = t; h.S[S_ITER] = 0.0; h.S[S_RZ] = 0.0; h.S[S_BETA] = 0.0;
        h.S[S_LOOP] = 0.0;
        h.S[S_DONE] = t == 0.0 ? 1.0 : 0.0;
    });
}

// last preconditioner stage: inverse row transforms, z = real part, <r, z>, beta
__global__ void fft_rows_inv_z_kernel(const HybDev h) {
    if (solver_done(h)) return;
    extern __shared__ float2 fsh[];
    const int N = h.nx;
    const float2* row = h.ws0 + (size_t)blockIdx.x * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) fsh[i] = row[i];
    __syncthreads();
    const float2* out = fft_smem(fsh, fsh + N, N, h.lx, h.twx, true);
    float rz = 0.0f;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int c = blockIdx.x * N + i;
        const float zv = out[i].x;
        h.z[c] = zv;
        rz = fmaf(h.r[c], zv, rz);
    }
    rows_sum(h, (double)rz, [&](double tot) {
        const double it = h.S[S_ITER];
        h.S[S_BETA] = it == 0.0 ? 0.0 : tot / h.S[S_RZ];
        h.S[S_RZ] = tot;
    });
}

// p_new = z + beta p_old; q = (lap - n_p) p_new in FP32; <p_new, q>; alpha.  The two direction
// buffers alternate with the iteration count, so the same launches serve every iteration.
__global__ void __launch_bounds__(NT) apply_kernel(const HybDev h) {
    if (solver_done(h)) return;
    const int nc = h.nx * h.ny;
    const float beta = (float)h.S[S_BETA];
    const int iter = (int)h.S[S_ITER];
    const bool first = iter == 0;
    const float* __restrict__ pold = (iter & 1) ? h.p1 : h.p0;
    float* __restrict__ pnew = (iter & 1) ? h.p0 : h.p1;
    const float ix2 = 1.0f / (h.dx * h.dx), iy2 = 1.0f / (h.dy * h.dy);
    float pq = 0.0f;
    for (int c = blockIdx.x * NT + threadIdx.x; c < nc; c += gridDim.x * NT) {
        const int i = c & (h.nx - 1), j = c >> h.lx;
        const int im = (i - 1) & (h.nx - 1), ip = (i + 1) & (h.nx - 1);
        const int jm = j == 0 ? h.ny - 1 : j - 1, jp = j + 1 == h.ny ? 0 : j + 1;
        auto pv = [&](int k) { return first ? h.z[k] : fmaf(beta, pold[k], h.z[k]); };
        const float pc = pv(c);
        const float pe = pv((j << h.lx) + ip), pw = pv((j << h.lx) + im);
        const float pn = pv((jp << h.lx) + i), ps = pv((jm << h.lx) + i);
        const float qv = (pe - 2.0f * pc + pw) * ix2 + (pn - 2.0f * pc + ps) * iy2 - h.np[c] * pc;
        pnew[c] = pc;
        h.q[c] = qv;
        pq = fmaf(pc, qv, pq);
    }
    grid_sum(h, (double)pq, [&](double t) { h.S[S_ALPHA] = h.S[S_RZ] / t; });
}

// d += alpha p; r -= alpha q; <r, r>; stop test; one CTA per row, which also applies the next
// iteration's forward transform along x to its row of r (into ws0).
__global__ void axpy_rows_kernel(const HybDev h) {
    if (solver_done(h)) return;
    extern __shared__ float2 fsh[];
    const int j = blockIdx.x;
    const float* __restrict__ p = ((int)h.S[S_ITER] & 1) ? h.p0 : h.p1;
    const float alpha = (float)h.S[S_ALPHA];
    float rr = 0.0f;
    for (int i = threadIdx.x; i < h.nx; i += blockDim.x) {
        const int c = (j << h.lx) + i;
        h.d[c] = fmaf(alpha, p[c], h.d[c]);
        const float rv = fmaf(-alpha, h.q[c], h.r[c]);
        h.r[c] = rv;
        fsh[i] = make_float2(rv, 0.0f);
        rr = fmaf(rv, rv, rr);
    }
    row_fft_store(h, fsh, j);
    rows_sum(h, (double)rr, [&](double t) {
        h.S[S_RR] = t;
        h.S[S_ITER] += 1.0;
        h.S[S_ITERS_TOTAL] += 1.0;
        if (t <= h.tol2 * h.S[S_RR0]) h.S[S_DONE] = 1.0;
    });
}

// Loop control of the graph's while node (one thread, never skipped): counts the iterations and
// stops the loop once the residual test passed or max_iter iterations ran, so it always ends.
__global__ void loop_ctl_kernel(const HybDev h, cudaGraphConditionalHandle cond, int max_iter) {
    const double l = h.S[S_LOOP] + 1.0;
    h.S[S_LOOP] = l;
    h.S[S_LOOPS_TOTAL] += 1.0;
    cudaGraphSetConditional(cond, (h.S[S_DONE] != 0.0 || l >= (double)max_iter) ? 0u : 1u);
}

// a^{n+1} = a^n + d, beta_p update, FP32 copies for the gather; solver bookkeeping.
__global__ void __launch_bounds__(NT) update_kernel(const HybDev h) {
    const int nc = h.nx * h.ny;
    for (int c = blockIdx.x * NT + threadIdx.x; c < nc; c += gridDim.x * NT) {
        const double dd = (double)h.d[c];
        const double an = h.a[c] + dd, bp = h.bp[c];
        const double bn = bp + dd - h.nu * h.dtd * bp;
        h.a[c] = an;
        h.bp[c] = bn;
        h.f32[c] = make_float2((float)an, (float)bn);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (h.S[S_DONE] == 0.0) h.S[S_NOCONV] += 1.0;
        h.S[S_LAST_ITERS] = h.S[S_ITER];
    }
}

// Energy partials per block: magnetic (forward differences), beam kinetic, plasma kinetic.
__global__ void __launch_bounds__(NT) energy_kernel(const HybDev h) {
    __shared__ double red[NT][3];
    double e[3] = {0, 0, 0};
    const int nc = h.nx * h.ny;
    for (int c = blockIdx.x * NT + threadIdx.x; c < nc; c += gridDim.x * NT) {
        const int i = c & (h.nx - 1), j = c >> h.lx;
        const double a0 = h.a[c];
        const double ax = (h.a[(j << h.lx) + ((i + 1) & (h.nx - 1))] - a0) * h.idx1;
        const double ay = (h.a[((j + 1 == h.ny ? 0 : j + 1) << h.lx) + i] - a0) * h.idy1;
        e[0] += 0.5 * (ax * ax + ay * ay);
        e[2] += 0.5 * (double)h.np[c] * h.bp[c] * h.bp[c];
    }
    // beam: gamma - 1 in FP32 per particle (the FP64 unit is scarce), summed exactly in fixed
    // point (integer part and 30 fraction bits), so the sum does not depend on particle order
    long long eb = 0;
    for (long long p = blockIdx.x * (long long)NT + threadIdx.x; p < h.n; p += (long long)gridDim.x * NT) {
        const Node4 c = nodes(h, h.cell[p], h.ox[p], h.oy[p]);
        const float gx0 = 1.0f - c.fx, gy0 = 1.0f - c.fy;
        const float av = gy0 * (gx0 * h.f32[c.c00].x + c.fx * h.f32[c.c10].x) +
                         c.fy * (gx0 * h.f32[c.c01].x + c.fx * h.f32[c.c11].x);
        const float uz = h.P[p] + av, ux = h.ux[p], uy = h.uy[p];
        const float u2 = ux * ux + uy * uy + uz * uz;
        const float gm1 = u2 / (1.0f + sqrtf(1.0f + u2));   // gamma - 1 without cancellation
        const float ip = floorf(gm1);
        eb += (long long)(int)ip * 1073741824LL + (long long)__float2int_rn((gm1 - ip) * 1073741824.0f);
    }
    __shared__ long long redb[NT];
    redb[threadIdx.x] = eb;
    for (int k = 0; k < 3; ++k) red[threadIdx.x][k] = e[k];
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            for (int k = 0; k < 3; ++k) red[threadIdx.x][k] += red[threadIdx.x + o][k];
            redb[threadIdx.x] += redb[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x < 3) h.part[blockIdx.x * 3 + threadIdx.x] = red[0][threadIdx.x];
    if (threadIdx.x == 0) h.ebeam[blockIdx.x] = redb[0];
}

int gridn(long long n) {
    long long g = (n + NT - 1) / NT;
    if (g > 152 * 8) g = 152 * 8;
    return (int)(g < 1 ? 1 : g);
}
int gridr(long long n) {
    long long g = (n + NT - 1) / NT;
    return (int)(g < 1 ? 1 : (g > RGRID ? RGRID : g));
}

int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

}  // namespace
}  // namespace pic

using namespace pic;

struct pic_hybrid {
    pic_hybrid_config cfg{};
    HybDev d{};
    cudaStream_t stream = nullptr;
    long long steps = 0;
    long long direct_launches = 0;   // kernels of directly launched steps
    long long graph_steps = 0;       // steps replayed as a graph (their CG loops vary in length)
    long long sorts = 0;
    int max_iter = 0;
    int sort_interval = 16;          // steps between counting sorts of the particles by cell
    // one step captured as a CUDA graph, plain and with the sort in front (rebuilt after a load
    // changes the kernel arguments)
    cudaGraph_t graph = nullptr, graph_s = nullptr;
    cudaGraphExec_t graph_exec = nullptr, graph_exec_s = nullptr;
    bool graph_dirty = true;
    // phase timing (flag PIC_FLAG_PROFILE): event pairs resolved by pic_hybrid_kernel_times
    struct Ev { int phase; cudaEvent_t a, b; };
    std::vector<Ev> pending;
    std::vector<cudaEvent_t> pool;
    double phase_ms[4] = {0, 0, 0, 0};
    long long phase_n[4] = {0, 0, 0, 0};
};

namespace {

bool pow2(int n) { return n >= 8 && n <= 2048 && (n & (n - 1)) == 0; }

int hfail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    pic::set_call_error(buf);
    return code;
}

#define HCK(call)                                                                                \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return hfail(PIC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct HLayout {
    size_t cell, ox, oy, ux, uy, P, id, cell2, ox2, oy2, ux2, uy2, P2, id2, order, start, bscratch, ebeam;
    size_t a, bp, f32, J, N, np, d, r, z, q, p0, p1, ws0, twx, twy, lamx, lamy, S, part, ticket, total;
};
HLayout hlayout(const pic_hybrid_config* c) {
    HLayout L{};
    size_t off = 0;
    const size_t nc = (size_t)c->nx * c->ny, np = (size_t)c->capacity;
    auto take = [&](size_t bytes) { off = align256(off); size_t at = off; off += bytes; return at; };
    L.cell = take(4 * np); L.ox = take(4 * np); L.oy = take(4 * np);
    L.ux = take(4 * np); L.uy = take(4 * np); L.P = take(4 * np); L.id = take(4 * np);
    L.cell2 = take(4 * np); L.ox2 = take(4 * np); L.oy2 = take(4 * np);
    L.ux2 = take(4 * np); L.uy2 = take(4 * np); L.P2 = take(4 * np); L.id2 = take(4 * np);
    L.order = take(4 * np); L.start = take(4 * (nc + 1)); L.bscratch = take(pic::bin_cells_scratch_bytes((long long)nc));
    L.ebeam = take(8 * (size_t)RGRID);
    L.a = take(8 * nc); L.bp = take(8 * nc); L.f32 = take(8 * nc); L.J = take(8 * nc); L.N = take(8 * nc);
    L.np = take(4 * nc); L.d = take(4 * nc); L.r = take(4 * nc); L.z = take(4 * nc); L.q = take(4 * nc);
    L.p0 = take(4 * nc); L.p1 = take(4 * nc); L.ws0 = take(8 * nc);
    L.twx = take(8 * (size_t)c->nx); L.twy = take(8 * (size_t)c->ny);
    L.lamx = take(4 * (size_t)c->nx); L.lamy = take(4 * (size_t)c->ny);
    L.S = take(8 * S_NSLOT); L.part = take(8 * 3 * (size_t)(RGRID > 2048 ? RGRID : 2048)); L.ticket = take(4);
    L.total = align256(off);
    return L;
}

int check_cfg(const pic_hybrid_config* c) {
    if (!c) return hfail(PIC_EINVAL, "null config");
    if (!pow2(c->nx) || !pow2(c->ny)) return hfail(PIC_EINVAL, "nx, ny must be powers of two in [8, 2048]");
    if (!(c->dx > 0 && c->dy > 0 && c->dt > 0)) return hfail(PIC_EINVAL, "dx, dy, dt must be > 0");
    if (!(c->dt < c->dx && c->dt < c->dy)) return hfail(PIC_EINVAL, "dt must be below dx and dy (a particle crosses at most one cell per step)");
    if (!(c->n0 > 0) || !(c->nu >= 0) || !(c->w >= 0)) return hfail(PIC_EINVAL, "need n0 > 0, nu >= 0, w >= 0");
    if (c->capacity < 0 || c->capacity > (int64_t)1 << 31) return hfail(PIC_EINVAL, "capacity must be in [0, 2^31]");
    if (c->tol < 0 || c->max_iter < 0 || c->max_iter > 1000) return hfail(PIC_EINVAL, "need tol >= 0, max_iter in [0, 1000]");
    if (c->flags & ~(PIC_FLAG_PROFILE | PIC_FLAG_NO_GRAPH)) return hfail(PIC_EINVAL, "unknown flags");
    if (c->sort_interval < 0) return hfail(PIC_EINVAL, "sort_interval must be >= 0");
    if (!(c->w <= 1e6)) return hfail(PIC_EINVAL, "w must be <= 1e6");
    return PIC_OK;
}

const char* const kHybPhase[4] = {"push_deposit", "field_solve", "update", "sort"};

cudaEvent_t get_event(pic_hybrid* h) {
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct HPhase {
    pic_hybrid* h;
    pic_hybrid::Ev ev{};
    bool on;
    HPhase(pic_hybrid* h_, int ph) : h(h_), on((h_->cfg.flags & PIC_FLAG_PROFILE) != 0) {
        if (!on) return;
        ev.phase = ph;
        ev.a = get_event(h);
        ev.b = get_event(h);
        cudaEventRecord(ev.a, h->stream);
    }
    ~HPhase() {
        if (!on) return;
        cudaEventRecord(ev.b, h->stream);
        h->pending.push_back(ev);
    }
};

// launches of one step: push, solve set-up, 7 per CG iteration run (+1 loop control in a graph),
// update; counted from the iterations the solver reports when the step is a graph
int step_launches(const pic_hybrid* h, int iters, bool graph) {
    return (h->d.n > 0 ? 1 : 0) + 2 + (graph ? 5 : 4) * iters;
}

void launch_pre(pic_hybrid* h) {
    HybDev& d = h->d;
    if (d.n > 0) push_kernel<<<gridn(d.n), NT, 0, h->stream>>>(d, 1);
}

// Counting sort of the particles by cell (the library's binning: histogram, scan, scatter of
// indices), then a gather into the second buffer and a copy back: 6 launches.
void launch_sort(pic_hybrid* h) {
    HybDev& d = h->d;
    if (d.n == 0) return;
    pic::launch_bin_cells(d.cell, d.n, d.nx * d.ny, d.start, d.order, d.bscratch, h->stream);
    permute_kernel<<<gridn(d.n), NT, 0, h->stream>>>(d);
    copy_back_kernel<<<gridn(d.n), NT, 0, h->stream>>>(d);
}
constexpr int SORT_LAUNCHES = 8;   // 6 of the binning (zero, histogram, 3 scan passes, scatter) + 2

int row_threads(int n) { return n / 4 < 1024 ? n / 4 : 1024; }   // one radix-4 butterfly per thread

void launch_rhs(pic_hybrid* h) {
    HybDev& d = h->d;
    rhs_rows_kernel<<<d.ny, row_threads(d.nx), 2 * (size_t)d.nx * sizeof(float2), h->stream>>>(d);
}

// one preconditioned CG iteration (every kernel returns at once after convergence): the column
// pass and the inverse row transforms of the preconditioner, the direction update, the residual
// update with the next forward row transforms
void launch_iteration(pic_hybrid* h) {
    HybDev& d = h->d;
    const int nx = d.nx, ny = d.ny, nc = nx * ny;
    const size_t shx = 2 * (size_t)nx * sizeof(float2), shc = 2 * (size_t)CW * (ny + 1) * sizeof(float2);
    fft_cols_strip_kernel<<<nx / CW, NTC, shc, h->stream>>>(d, ilog2(ny));
    fft_rows_inv_z_kernel<<<ny, row_threads(nx), shx, h->stream>>>(d);
    apply_kernel<<<gridr(nc), NT, 0, h->stream>>>(d);
    axpy_rows_kernel<<<ny, row_threads(nx), shx, h->stream>>>(d);
}

void launch_post(pic_hybrid* h) {
    HybDev& d = h->d;
    update_kernel<<<gridr((long long)d.nx * d.ny), NT, 0, h->stream>>>(d);
}

// (Sort,) push and deposit, the solve (max_iter CG iterations, early-exiting kernels), the update.
int launch_step(pic_hybrid* h, bool sort) {
    if (sort) {
        HPhase ps(h, 3);
        launch_sort(h);
    }
    {
        HPhase ph(h, 0);
        launch_pre(h);
    }
    {
        HPhase ph(h, 1);
        launch_rhs(h);
        for (int it = 0; it < h->max_iter; ++it) launch_iteration(h);
    }
    {
        HPhase pu(h, 2);
        launch_post(h);
    }
    HCK(cudaGetLastError());
    return PIC_OK;
}

void drop_graph(pic_hybrid* h) {
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->graph_exec_s) cudaGraphExecDestroy(h->graph_exec_s);
    if (h->graph_s) cudaGraphDestroy(h->graph_s);
    h->graph_exec = h->graph_exec_s = nullptr;
    h->graph = h->graph_s = nullptr;
    h->graph_dirty = true;
}

// One step as a graph: push and solve set-up, a while node whose body is one CG iteration plus
// the loop control (the loop runs only the iterations the solve needs, at most max_iter), then
// the update.  Each part is captured from the stream into the graph.
int build_one_graph(pic_hybrid* h, bool sort, cudaGraph_t* gout, cudaGraphExec_t* xout) {
    cudaGraph_t g = nullptr;
    HCK(cudaGraphCreate(&g, 0));
    *gout = g;
    cudaGraphConditionalHandle cond{};
    HCK(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
    const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
    auto capture = [&](cudaGraph_t into, const cudaGraphNode_t* deps, size_t ndeps, auto&& body,
                       std::vector<cudaGraphNode_t>* leaves) -> cudaError_t {
        cudaError_t e = cudaStreamBeginCaptureToGraph(h->stream, into, deps, nullptr, ndeps, mode);
        if (e != cudaSuccess) return e;
        body();
        if (leaves) {
            cudaStreamCaptureStatus st;
            const cudaGraphNode_t* dn = nullptr;
            size_t nd = 0;
            e = cudaStreamGetCaptureInfo(h->stream, &st, nullptr, nullptr, &dn, nullptr, &nd);
            if (e == cudaSuccess) leaves->assign(dn, dn + nd);
        }
        cudaGraph_t out = into;
        const cudaError_t e2 = cudaStreamEndCapture(h->stream, &out);
        if (e != cudaSuccess) return e;
        if (e2 != cudaSuccess) return e2;
        return cudaGetLastError();
    };
    std::vector<cudaGraphNode_t> pre;
    cudaError_t e = capture(g, nullptr, 0, [&] {
        if (sort) launch_sort(h);
        launch_pre(h);
        launch_rhs(h);
    }, &pre);
    if (e != cudaSuccess) { drop_graph(h); return hfail(PIC_ECUDA, "graph capture (push): %s", cudaGetErrorString(e)); }
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop = nullptr;
    e = cudaGraphAddNode(&loop, g, pre.data(), nullptr, pre.size(), &cp);
    if (e != cudaSuccess) { drop_graph(h); return hfail(PIC_ECUDA, "conditional node: %s", cudaGetErrorString(e)); }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    const int max_iter = h->max_iter;
    e = capture(body, nullptr, 0, [&] {
        launch_iteration(h);
        loop_ctl_kernel<<<1, 1, 0, h->stream>>>(h->d, cond, max_iter);
    }, nullptr);
    if (e != cudaSuccess) { drop_graph(h); return hfail(PIC_ECUDA, "graph capture (solve): %s", cudaGetErrorString(e)); }
    e = capture(g, &loop, 1, [&] { launch_post(h); }, nullptr);
    if (e != cudaSuccess) { drop_graph(h); return hfail(PIC_ECUDA, "graph capture (update): %s", cudaGetErrorString(e)); }
    e = cudaGraphInstantiate(xout, g, 0);
    if (e != cudaSuccess) { drop_graph(h); return hfail(PIC_ECUDA, "graph instantiate: %s", cudaGetErrorString(e)); }
    return PIC_OK;
}

int build_graph(pic_hybrid* h) {
    drop_graph(h);
    int rc = build_one_graph(h, false, &h->graph, &h->graph_exec);
    if (rc == PIC_OK) rc = build_one_graph(h, true, &h->graph_s, &h->graph_exec_s);
    if (rc == PIC_OK) h->graph_dirty = false;
    return rc;
}

}  // namespace

extern "C" int pic_hybrid_required_bytes(const pic_hybrid_config* cfg, size_t* bytes_out) {
    int rc = check_cfg(cfg);
    if (rc) return rc;
    if (!bytes_out) return hfail(PIC_EINVAL, "null bytes_out");
    *bytes_out = hlayout(cfg).total;
    return PIC_OK;
}

extern "C" int pic_hybrid_init(const pic_hybrid_config* cfg, void* arena, size_t arena_bytes, void* stream,
                               pic_hybrid** out) {
    int rc = check_cfg(cfg);
    if (rc) return rc;
    if (!out || !arena) return hfail(PIC_EINVAL, "null argument");
    const HLayout L = hlayout(cfg);
    if (arena_bytes < L.total) return hfail(PIC_ENOMEM, "arena has %zu bytes, needs %zu", arena_bytes, L.total);
    if (reinterpret_cast<uintptr_t>(arena) & 255) return hfail(PIC_EINVAL, "arena must be 256-byte aligned");
    const int shmax = 2 * 2048 * (int)sizeof(float2);
    const int shcol = 2 * CW * (2048 + 1) * (int)sizeof(float2);
    HCK(cudaFuncSetAttribute(rhs_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, shmax));
    HCK(cudaFuncSetAttribute(axpy_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, shmax));
    HCK(cudaFuncSetAttribute(fft_cols_strip_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, shcol));
    HCK(cudaFuncSetAttribute(fft_rows_inv_z_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, shmax));
    pic_hybrid* h = new pic_hybrid;
    h->cfg = *cfg;
    h->stream = (cudaStream_t)stream;
    h->max_iter = cfg->max_iter > 0 ? cfg->max_iter : 16;
    char* base = static_cast<char*>(arena);
    HybDev& d = h->d;
    d.nx = cfg->nx; d.ny = cfg->ny; d.lx = ilog2(cfg->nx);
    d.dx = (float)cfg->dx; d.dy = (float)cfg->dy; d.dt = (float)cfg->dt; d.w = (float)cfg->w;
    d.dxd = cfg->dx; d.dyd = cfg->dy; d.dtd = cfg->dt; d.n0 = cfg->n0; d.nu = cfg->nu;
    d.idx = (float)(1.0 / cfg->dx); d.idy = (float)(1.0 / cfg->dy);
    d.idx1 = 1.0 / cfg->dx; d.idy1 = 1.0 / cfg->dy;
    d.idx2 = 1.0 / (cfg->dx * cfg->dx); d.idy2 = 1.0 / (cfg->dy * cfg->dy);
    d.keep = 1.0 - cfg->nu * cfg->dt;
    const double tol = cfg->tol > 0 ? cfg->tol : 1e-5;
    d.tol2 = tol * tol;
    d.n = 0;
    auto F = [&](size_t o) { return reinterpret_cast<float*>(base + o); };
    d.cell = reinterpret_cast<int*>(base + L.cell);
    d.ox = F(L.ox); d.oy = F(L.oy); d.ux = F(L.ux); d.uy = F(L.uy); d.P = F(L.P);
    d.id = reinterpret_cast<int*>(base + L.id);
    d.cell2 = reinterpret_cast<int*>(base + L.cell2);
    d.ox2 = F(L.ox2); d.oy2 = F(L.oy2); d.ux2 = F(L.ux2); d.uy2 = F(L.uy2); d.P2 = F(L.P2);
    d.id2 = reinterpret_cast<int*>(base + L.id2);
    d.order = reinterpret_cast<int*>(base + L.order);
    d.start = reinterpret_cast<int*>(base + L.start);
    d.bscratch = reinterpret_cast<int*>(base + L.bscratch);
    d.ebeam = reinterpret_cast<long long*>(base + L.ebeam);
    h->sort_interval = cfg->sort_interval > 0 ? cfg->sort_interval : 16;
    // deposit terms: |term| <= w, and a window entry sums at most NT of them below 2^31:
    // 2^S32 <= 2^31 / (NT w); S32 <= 40 (the grids' scale) so the sums enter the grids by a shift
    {
        int s32 = 40;
        const double lim = 2147483647.0 / (double)NT;
        while (s32 > 0 && cfg->w * std::ldexp(1.0, s32) >= lim) --s32;
        d.sfix = (float)std::ldexp(1.0, s32);
        d.sshift = 40 - s32;
    }
    d.a = reinterpret_cast<double*>(base + L.a);
    d.bp = reinterpret_cast<double*>(base + L.bp);
    d.f32 = reinterpret_cast<float2*>(base + L.f32);
    d.J = reinterpret_cast<long long*>(base + L.J);
    d.N = reinterpret_cast<long long*>(base + L.N);
    d.np = F(L.np); d.d = F(L.d); d.r = F(L.r); d.z = F(L.z); d.q = F(L.q); d.p0 = F(L.p0); d.p1 = F(L.p1);
    d.ws0 = reinterpret_cast<float2*>(base + L.ws0);
    d.twx = reinterpret_cast<const float2*>(base + L.twx);
    d.twy = reinterpret_cast<const float2*>(base + L.twy);
    d.lamx = reinterpret_cast<const float*>(base + L.lamx);
    d.lamy = reinterpret_cast<const float*>(base + L.lamy);
    d.S = reinterpret_cast<double*>(base + L.S);
    d.part = reinterpret_cast<double*>(base + L.part);
    d.ticket = reinterpret_cast<unsigned*>(base + L.ticket);
    d.nbar = (float)cfg->n0;   // until a load fixes the mean beam density
    // twiddles and eigenvalues from the host's double-precision sin/cos
    std::vector<float2> twx(cfg->nx), twy(cfg->ny);
    std::vector<float> lamx(cfg->nx), lamy(cfg->ny);
    const double pi = 3.14159265358979323846;
    for (int m = 0; m < cfg->nx; ++m) twx[m] = make_float2((float)std::cos(2 * pi * m / cfg->nx), (float)-std::sin(2 * pi * m / cfg->nx));
    for (int m = 0; m < cfg->ny; ++m) twy[m] = make_float2((float)std::cos(2 * pi * m / cfg->ny), (float)-std::sin(2 * pi * m / cfg->ny));
    for (int m = 0; m < cfg->nx; ++m) { const double s = std::sin(pi * m / cfg->nx); lamx[m] = (float)(-4.0 / (cfg->dx * cfg->dx) * s * s); }
    for (int m = 0; m < cfg->ny; ++m) { const double s = std::sin(pi * m / cfg->ny); lamy[m] = (float)(-4.0 / (cfg->dy * cfg->dy) * s * s); }
    const size_t nc = (size_t)cfg->nx * cfg->ny;
    cudaError_t e = cudaMemsetAsync(base, 0, L.total, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void*)d.twx, twx.data(), 8 * twx.size(), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void*)d.twy, twy.data(), 8 * twy.size(), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void*)d.lamx, lamx.data(), 4 * lamx.size(), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void*)d.lamy, lamy.data(), 4 * lamy.size(), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    (void)nc;
    if (e != cudaSuccess) {
        delete h;
        return hfail(PIC_ECUDA, "pic_hybrid_init: %s", cudaGetErrorString(e));
    }
    *out = h;
    return PIC_OK;
}

extern "C" int pic_hybrid_load(pic_hybrid* h, int64_t n, const double* X, const double* Y, const double* ux,
                               const double* uy, const double* uz, const double* beta_p) {
    if (!h) return hfail(PIC_EINVAL, "null context");
    if (n < 0 || n > h->cfg.capacity) return hfail(PIC_EINVAL, "n must be in [0, capacity]");
    if (n > 0 && (!X || !Y || !ux || !uy || !uz)) return hfail(PIC_EINVAL, "null particle array");
    if (!beta_p) return hfail(PIC_EINVAL, "null beta_p");
    const int nx = h->cfg.nx, ny = h->cfg.ny;
    std::vector<int> cell(n);
    std::vector<float> ox(n), oy(n), fux(n), fuy(n), fP(n);
    for (int64_t p = 0; p < n; ++p) {
        if (!(X[p] >= 0 && X[p] < nx && Y[p] >= 0 && Y[p] < ny && std::isfinite(ux[p]) && std::isfinite(uy[p]) &&
              std::isfinite(uz[p])))
            return hfail(PIC_EBADPART, "particle %lld out of the grid or not finite", (long long)p);
        int i = (int)std::floor(X[p]), j = (int)std::floor(Y[p]);
        float fx = (float)(X[p] - i), fy = (float)(Y[p] - j);
        if (fx >= 1.0f) { fx = 0.0f; i = (i + 1) % nx; }
        if (fy >= 1.0f) { fy = 0.0f; j = (j + 1) % ny; }
        cell[p] = j * nx + i; ox[p] = fx; oy[p] = fy;
        fux[p] = (float)ux[p]; fuy[p] = (float)uy[p]; fP[p] = (float)uz[p];   // a = 0 at load: P = u_z
    }
    const size_t nc = (size_t)nx * ny;
    std::vector<float2> f32(nc);
    for (size_t c = 0; c < nc; ++c) {
        if (!std::isfinite(beta_p[c])) return hfail(PIC_EBADPART, "beta_p[%zu] not finite", c);
        f32[c] = make_float2(0.0f, (float)beta_p[c]);
    }
    HybDev& d = h->d;
    d.n = n;
    // preconditioner density: n0 minus the mean beam density (any positive value is valid)
    const double nbar = h->cfg.n0 - (double)n * h->cfg.w / (double)nc;
    d.nbar = (float)(nbar > 0.05 * h->cfg.n0 ? nbar : 0.05 * h->cfg.n0);
    HCK(cudaMemcpyAsync(d.cell, cell.data(), 4 * n, cudaMemcpyHostToDevice, h->stream));
    HCK(cudaMemcpyAsync(d.ox, ox.data(), 4 * n, cudaMemcpyHostToDevice, h->stream));
    HCK(cudaMemcpyAsync(d.oy, oy.data(), 4 * n, cudaMemcpyHostToDevice, h->stream));
    HCK(cudaMemcpyAsync(d.ux, fux.data(), 4 * n, cudaMemcpyHostToDevice, h->stream));
    HCK(cudaMemcpyAsync(d.uy, fuy.data(), 4 * n, cudaMemcpyHostToDevice, h->stream));
    HCK(cudaMemcpyAsync(d.P, fP.data(), 4 * n, cudaMemcpyHostToDevice, h->stream));
    std::vector<int> ids(n);
    for (int64_t p = 0; p < n; ++p) ids[p] = (int)p;
    HCK(cudaMemcpyAsync(d.id, ids.data(), 4 * n, cudaMemcpyHostToDevice, h->stream));
    HCK(cudaMemcpyAsync(d.bp, beta_p, 8 * nc, cudaMemcpyHostToDevice, h->stream));
    HCK(cudaMemcpyAsync(d.f32, f32.data(), 8 * nc, cudaMemcpyHostToDevice, h->stream));
    HCK(cudaMemsetAsync(d.a, 0, 8 * nc, h->stream));
    HCK(cudaMemsetAsync(d.J, 0, 8 * nc, h->stream));
    HCK(cudaMemsetAsync(d.N, 0, 8 * nc, h->stream));
    HCK(cudaMemsetAsync(d.S, 0, 8 * S_NSLOT, h->stream));
    launch_sort(h);   // cell order from the start, whatever the caller's order
    HCK(cudaGetLastError());
    if (n > 0) push_kernel<<<gridn(n), NT, 0, h->stream>>>(d, 0);
    density_kernel<<<gridn((long long)nc), NT, 0, h->stream>>>(d);
    HCK(cudaGetLastError());
    HCK(cudaStreamSynchronize(h->stream));
    h->steps = 0;
    drop_graph(h);
    return PIC_OK;
}

extern "C" int pic_hybrid_step(pic_hybrid* h, int nsteps) {
    if (!h) return hfail(PIC_EINVAL, "null context");
    if (nsteps < 0) return hfail(PIC_EINVAL, "nsteps must be >= 0");
    const bool use_graph = !(h->cfg.flags & (PIC_FLAG_PROFILE | PIC_FLAG_NO_GRAPH));
    for (int s = 0; s < nsteps; ++s) {
        const bool sort = h->sort_interval > 0 && h->d.n > 0 && h->steps > 0 && h->steps % h->sort_interval == 0;
        if (use_graph) {
            if (h->graph_dirty) {
                int rc = build_graph(h);
                if (rc) return rc;
            }
            HCK(cudaGraphLaunch(sort ? h->graph_exec_s : h->graph_exec, h->stream));
            ++h->graph_steps;
        } else {
            int rc = launch_step(h, sort);
            if (rc) return rc;
            h->direct_launches += step_launches(h, h->max_iter, false);
        }
        if (sort) { h->direct_launches += SORT_LAUNCHES; ++h->sorts; }
        ++h->steps;
    }
    return PIC_OK;
}

extern "C" int pic_hybrid_kernel_times(pic_hybrid* h, pic_kernel_time* out, int max, int* n_out) {
    if (!h || !n_out) return hfail(PIC_EINVAL, "null argument");
    HCK(cudaStreamSynchronize(h->stream));
    for (auto& ev : h->pending) {
        float ms = 0.f;
        HCK(cudaEventElapsedTime(&ms, ev.a, ev.b));
        h->phase_ms[ev.phase] += ms;
        h->phase_n[ev.phase] += 1;
        h->pool.push_back(ev.a);
        h->pool.push_back(ev.b);
    }
    h->pending.clear();
    int n = 0;
    for (int p = 0; p < 4 && n < max && out; ++p, ++n) {
        std::snprintf(out[n].name, sizeof out[n].name, "%s", kHybPhase[p]);
        out[n].launches = h->phase_n[p];
        out[n].total_ms = h->phase_ms[p];
    }
    *n_out = n;
    return PIC_OK;
}

extern "C" int64_t pic_hybrid_launch_count(pic_hybrid* h) {
    if (!h) return -1;
    // graph steps: push, set-up and update per step and 5 kernels per run of the loop body (the
    // loop control counts the runs on the device)
    double S[S_NSLOT];
    if (cudaMemcpyAsync(S, h->d.S, sizeof S, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return -1;
    return h->direct_launches + h->graph_steps * ((h->d.n > 0 ? 1 : 0) + 2) + 5 * (long long)S[S_LOOPS_TOTAL];
}

extern "C" int pic_hybrid_get(pic_hybrid* h, double* a, double* beta_p, double* X, double* Y, double* ux,
                              double* uy) {
    if (!h) return hfail(PIC_EINVAL, "null context");
    const HybDev& d = h->d;
    const size_t nc = (size_t)d.nx * d.ny;
    const long long n = d.n;
    if (a) HCK(cudaMemcpyAsync(a, d.a, 8 * nc, cudaMemcpyDeviceToHost, h->stream));
    if (beta_p) HCK(cudaMemcpyAsync(beta_p, d.bp, 8 * nc, cudaMemcpyDeviceToHost, h->stream));
    std::vector<int> cell(X || Y ? n : 0), ids(n);
    std::vector<float> ox(X ? n : 0), oy(Y ? n : 0), fux(ux ? n : 0), fuy(uy ? n : 0);
    HCK(cudaMemcpyAsync(ids.data(), d.id, 4 * n, cudaMemcpyDeviceToHost, h->stream));
    if (X || Y) HCK(cudaMemcpyAsync(cell.data(), d.cell, 4 * n, cudaMemcpyDeviceToHost, h->stream));
    if (X) HCK(cudaMemcpyAsync(ox.data(), d.ox, 4 * n, cudaMemcpyDeviceToHost, h->stream));
    if (Y) HCK(cudaMemcpyAsync(oy.data(), d.oy, 4 * n, cudaMemcpyDeviceToHost, h->stream));
    if (ux) HCK(cudaMemcpyAsync(fux.data(), d.ux, 4 * n, cudaMemcpyDeviceToHost, h->stream));
    if (uy) HCK(cudaMemcpyAsync(fuy.data(), d.uy, 4 * n, cudaMemcpyDeviceToHost, h->stream));
    HCK(cudaStreamSynchronize(h->stream));
    for (long long p = 0; p < n; ++p) {   // back to the load order
        const int q = ids[p];
        if (q < 0 || q >= n) return hfail(PIC_ESTATE, "particle ids corrupted");
        if (X) X[q] = (double)(cell[p] & (d.nx - 1)) + (double)ox[p];
        if (Y) Y[q] = (double)(cell[p] >> d.lx) + (double)oy[p];
        if (ux) ux[q] = fux[p];
        if (uy) uy[q] = fuy[p];
    }
    return PIC_OK;
}

extern "C" int pic_hybrid_energies(pic_hybrid* h, double out3[3]) {
    if (!h || !out3) return hfail(PIC_EINVAL, "null argument");
    const HybDev& d = h->d;
    energy_kernel<<<RGRID, NT, 0, h->stream>>>(d);
    HCK(cudaGetLastError());
    std::vector<double> part(3 * RGRID);
    std::vector<long long> eb(RGRID);
    HCK(cudaMemcpyAsync(part.data(), d.part, 8 * part.size(), cudaMemcpyDeviceToHost, h->stream));
    HCK(cudaMemcpyAsync(eb.data(), d.ebeam, 8 * eb.size(), cudaMemcpyDeviceToHost, h->stream));
    HCK(cudaStreamSynchronize(h->stream));
    const double dA = d.dxd * d.dyd;
    for (int k = 0; k < 3; k += 2) {
        double s = 0.0;
        for (int b = 0; b < RGRID; ++b) s += part[3 * b + k];
        out3[k] = s * dA;
    }
    long long sb = 0;
    for (int b = 0; b < RGRID; ++b) sb += eb[b];
    out3[1] = (double)sb * 0x1p-30 * h->cfg.w * dA;
    return PIC_OK;
}

extern "C" int pic_hybrid_stats(pic_hybrid* h, int64_t out4[4]) {
    if (!h || !out4) return hfail(PIC_EINVAL, "null argument");
    double S[S_NSLOT];
    HCK(cudaMemcpyAsync(S, h->d.S, sizeof S, cudaMemcpyDeviceToHost, h->stream));
    HCK(cudaStreamSynchronize(h->stream));
    out4[0] = h->steps;
    out4[1] = (int64_t)S[S_ITERS_TOTAL];
    out4[2] = (int64_t)S[S_NOCONV];
    out4[3] = (int64_t)S[S_LAST_ITERS];
    return PIC_OK;
}

extern "C" int64_t pic_hybrid_step_count(const pic_hybrid* h) { return h ? h->steps : -1; }

extern "C" void pic_hybrid_free(pic_hybrid* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    drop_graph(h);
    for (auto& ev : h->pending) { cudaEventDestroy(ev.a); cudaEventDestroy(ev.b); }
    for (auto e : h->pool) cudaEventDestroy(e);
    delete h;
}
