// closure.cu -- training samples of the learned collision closure and the network's input
// normalisation, on the device.
//
// Samples: the paper's conclusion conjectures that the two-stream turbulence of a 3D run acts on
// the return current like collisions.  This library reads that as a friction rate nu_eff per
// coarse cell, averaged over a time of order 1/w_p: the moment recorder's snapshots (rows n_b,
// n_p, uz_b, uz_p, Tperp_b, Tpar_b, Tperp_p, Tpar_p, W_ES, Fz_p, Fz_mean, nu_eff) are averaged
// over windows of consecutive snapshots, and per window and coarse cell
//     features = the window means of rows 0..8,
//     label    = nu_p + (<Fz_mean> - <Fz_p>) / <uz_p>,
// kept where |<uz_p>| >= uz_min (where the return current has stopped the ratio says nothing).
// One kernel forms every (window, cell) sample and its keep flag; a second, one CTA, scans the
// flags in (window, cell) order and writes the kept samples contiguously, so the training set
// and everything trained on it are the same on every run.
//
// Normalisation: per-feature mean and population standard deviation in FP64, summed in a fixed
// order by one CTA per feature.
#include <cmath>

#include "../../include/pic.h"
#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int NT = 256;
constexpr int NROW = PIC_MOM_ROWS;
constexpr int NFEAT = PIC_MLP_IN;

// Sample m = w * nc + c: window means, label, keep flag.
__global__ void __launch_bounds__(NT) samples_kernel(const float* __restrict__ rows, long long nc, int nw,
                                                     int window, float nu_p, float uz_min,
                                                     float* __restrict__ feat, float* __restrict__ label,
                                                     int* __restrict__ keep) {
    const long long M = (long long)nw * nc;
    for (long long m = blockIdx.x * (long long)NT + threadIdx.x; m < M; m += (long long)gridDim.x * NT) {
        const long long w = m / nc, c = m - w * nc;
        double mean[NROW];
#pragma unroll
        for (int r = 0; r < NROW; ++r) mean[r] = 0.0;
        for (int k = 0; k < window; ++k) {
            const float* snap = rows + (w * window + k) * (long long)NROW * nc;
#pragma unroll
            for (int r = 0; r < NROW; ++r) mean[r] += (double)snap[(long long)r * nc + c];
        }
        const double inv = 1.0 / (double)window;
#pragma unroll
        for (int r = 0; r < NFEAT; ++r) feat[(long long)r * M + m] = (float)(mean[r] * inv);
        const double uz = mean[3] * inv, fzp = mean[9] * inv, fzm = mean[10] * inv;
        const double lab = (double)nu_p + (fzm - fzp) / uz;
        const bool ok = fabs(uz) >= (double)uz_min && isfinite(lab);
        label[m] = ok ? (float)lab : 0.f;
        keep[m] = ok ? 1 : 0;
    }
}

// One CTA: exclusive scan of keep[] in order, kept samples to out (feature-major, ldo = cap).
__global__ void __launch_bounds__(1024) compact_samples_kernel(const float* __restrict__ feat,
                                                               const float* __restrict__ label,
                                                               const int* __restrict__ keep, long long M,
                                                               float* __restrict__ ofeat,
                                                               float* __restrict__ olabel, long long cap,
                                                               long long* __restrict__ n_out) {
    __shared__ int warp_sum[32];
    __shared__ long long base;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) base = 0;
    __syncthreads();
    for (long long c0 = 0; c0 < M; c0 += 1024) {
        const long long m = c0 + tid;
        const int f = m < M ? keep[m] : 0;
        int incl = f;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) warp_sum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int s = warp_sum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += v;
            }
            warp_sum[lane] = s;            // inclusive over warps
        }
        __syncthreads();
        const long long pos = base + (wid ? warp_sum[wid - 1] : 0) + incl - f;
        if (f && pos < cap) {
            for (int r = 0; r < NFEAT; ++r) ofeat[(long long)r * cap + pos] = feat[(long long)r * M + m];
            olabel[pos] = label[m];
        }
        __syncthreads();
        if (tid == 0) base += warp_sum[31];
        __syncthreads();
    }
    if (tid == 0) *n_out = base;
}

// One CTA per feature: FP64 mean and population standard deviation in a fixed order.
__global__ void __launch_bounds__(NT) fit_norm_kernel(const float* __restrict__ x, long long ldx, long long n,
                                                      int nin, float* __restrict__ mu_sigma) {
    __shared__ double s1[NT], s2[NT];
    const int j = blockIdx.x;
    double a = 0.0, b = 0.0;
    if (j < nin)
        for (long long i = threadIdx.x; i < n; i += NT) {
            const double v = (double)x[(long long)j * ldx + i];
            a += v;
            b += v * v;
        }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        float mu = 0.f, sd = 1.f;
        if (j < nin && n > 0) {
            const double m = s1[0] / (double)n;
            const double var = fmax(s2[0] / (double)n - m * m, 0.0);
            mu = (float)m;
            sd = var > 0.0 ? (float)sqrt(var) : 1.f;
        }
        mu_sigma[j] = mu;
        mu_sigma[NFEAT + j] = sd;
    }
}

}  // namespace

size_t closure_samples_scratch_bytes(long long m) {
    return (size_t)m * (NFEAT + 1) * sizeof(float) + (size_t)m * sizeof(int) + 256;
}

cudaError_t launch_closure_samples(const float* rows, int nsnap, long long nc, int window, float nu_p, float uz_min,
                                   float* feat, float* label, long long cap, long long* n_out, void* scratch,
                                   cudaStream_t s) {
    const int nw = nsnap / window;
    const long long M = (long long)nw * nc;
    float* tf = static_cast<float*>(scratch);
    float* tl = tf + (size_t)M * NFEAT;
    int* keep = reinterpret_cast<int*>(tl + M);
    if (M > 0) {
        long long g = (M + NT - 1) / NT;
        if (g > 152 * 8) g = 152 * 8;
        samples_kernel<<<(int)g, NT, 0, s>>>(rows, nc, nw, window, nu_p, uz_min, tf, tl, keep);
    }
    compact_samples_kernel<<<1, 1024, 0, s>>>(tf, tl, keep, M, feat, label, cap, n_out);
    return cudaGetLastError();
}

cudaError_t launch_fit_norm(const float* x, long long ldx, long long n, int nin, float* mu_sigma, cudaStream_t s) {
    fit_norm_kernel<<<NFEAT, NT, 0, s>>>(x, ldx, n, nin, mu_sigma);
    return cudaGetLastError();
}

}  // namespace pic
