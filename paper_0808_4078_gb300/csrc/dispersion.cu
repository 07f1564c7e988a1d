// dispersion.cu -- growth rates of the collisional (resistive) filamentation dispersion relation,
// Eq. (12): w^2 = c_s^2 k^2 - w_b^2 beta0^2 k^2 / (k^2 + k_pe^2 / (1 + i nu / w)), in units with
// k_pe = c / w_p = 1 and w_b^2 = n_b.  Multiplied out it is the cubic in w
//   (k^2 + 1) w^3 + i nu k^2 w^2 + (b - a (k^2 + 1)) w + i nu (b - a k^2) = 0,
//   a = c_s^2 k^2,  b = n_b beta0^2 k^2,
// whose root of largest imaginary part gives the growth rate at k.  One CTA per parameter set
// scans a uniform k grid (a thread per k), solves each cubic in FP64 by Durand-Kerner iteration
// followed by Newton polishing, and reduces max Im w with the k where it occurs (lowest k on
// ties, so the result is deterministic).
#include <cfloat>

#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int NT = 128;

struct cplx {
    double re, im;
};
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
    const double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
__device__ __forceinline__ double cabs2(cplx a) { return a.re * a.re + a.im * a.im; }

// Monic cubic w^3 + c2 w^2 + c1 w + c0 and its derivative at w.
__device__ __forceinline__ cplx horner(cplx c2, cplx c1, cplx c0, cplx w) {
    return cadd(cmul(cadd(cmul(cadd(w, c2), w), c1), w), c0);
}
__device__ __forceinline__ cplx dhorner(cplx c2, cplx c1, cplx w) {
    const cplx three_w = {3.0 * w.re, 3.0 * w.im}, two_c2 = {2.0 * c2.re, 2.0 * c2.im};
    return cadd(cmul(cadd(three_w, two_c2), w), c1);
}

// Largest imaginary part among the three roots of the monic cubic.
__device__ double max_imag_root(cplx c2, cplx c1, cplx c0) {
    // Cauchy bound on the root moduli; start points spread on a circle of that radius
    const double R = 1.0 + fmax(sqrt(cabs2(c2)), fmax(sqrt(cabs2(c1)), sqrt(cabs2(c0))));
    cplx z[3];
    for (int k = 0; k < 3; ++k) {
        double s, c;
        sincos(0.4 + 2.0943951023931957 * k, &s, &c);
        z[k] = {R * c, R * s};
    }
    for (int it = 0; it < 200; ++it) {
        double change = 0.0;
        for (int k = 0; k < 3; ++k) {
            cplx den = {1.0, 0.0};
            for (int j = 0; j < 3; ++j)
                if (j != k) den = cmul(den, csub(z[k], z[j]));
            if (cabs2(den) == 0.0) den = {DBL_MIN, 0.0};
            const cplx step = cdiv(horner(c2, c1, c0, z[k]), den);
            z[k] = csub(z[k], step);
            change = fmax(change, cabs2(step) / fmax(cabs2(z[k]), 1e-300));
        }
        if (change < 1e-30) break;
    }
    double best = -DBL_MAX;
    for (int k = 0; k < 3; ++k) {
        for (int it = 0; it < 2; ++it) {
            const cplx d = dhorner(c2, c1, z[k]);
            if (cabs2(d) > 0.0) z[k] = csub(z[k], cdiv(horner(c2, c1, c0, z[k]), d));
        }
        best = fmax(best, z[k].im);
    }
    return best;
}

__global__ void __launch_bounds__(NT) dispersion_kernel(const double* __restrict__ params, double kmin, double dk,
                                                        int nk, double* __restrict__ gamma, double* __restrict__ kstar) {
    __shared__ double sg[NT];
    __shared__ int si[NT];
    const double cs2 = params[4 * blockIdx.x], beta0 = params[4 * blockIdx.x + 1];
    const double nb = params[4 * blockIdx.x + 2], nu = params[4 * blockIdx.x + 3];
    double best = -DBL_MAX;
    int bi = 0;
    for (int i = threadIdx.x; i < nk; i += NT) {
        const double k = kmin + dk * i, k2 = k * k;
        const double a = cs2 * k2, b = nb * beta0 * beta0 * k2;
        const double lead = k2 + 1.0;
        const cplx c2 = {0.0, nu * k2 / lead};
        const cplx c1 = {(b - a * lead) / lead, 0.0};
        const cplx c0 = {0.0, nu * (b - a * k2) / lead};
        const double g = max_imag_root(c2, c1, c0);
        if (g > best) { best = g; bi = i; }
    }
    sg[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const double g2 = sg[threadIdx.x + o];
            const int i2 = si[threadIdx.x + o];
            if (g2 > sg[threadIdx.x] || (g2 == sg[threadIdx.x] && i2 < si[threadIdx.x])) {
                sg[threadIdx.x] = g2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        gamma[blockIdx.x] = sg[0];
        kstar[blockIdx.x] = kmin + dk * si[0];
    }
}

}  // namespace

cudaError_t launch_dispersion(const double* params, int nsets, double kmin, double kmax, int nk, double* gamma,
                              double* kstar, cudaStream_t s) {
    const double dk = nk > 1 ? (kmax - kmin) / (nk - 1) : 0.0;
    dispersion_kernel<<<nsets, NT, 0, s>>>(params, kmin, dk, nk, gamma, kstar);
    return cudaGetLastError();
}

}  // namespace pic
