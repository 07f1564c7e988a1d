// mlp.cu -- the closure network on the tensor cores: 9 (or 8) inputs -> 64 -> 64 -> 1, SiLU,
// bfloat16 weights and matrix inputs, FP32 accumulation.  Forward (inference) and one Adam
// training step over a batch (mean squared error).
//
// The paper's conclusion conjectures that the collisional friction on the return current can be
// expressed through the local plasma state; this network is the library's reading of that
// closure (inputs: the coarse moments of pic_record_moments rows 0..8; output: nu_eff).
//
// A CTA of 128 threads owns tiles of 128 samples, one sample (row) per thread.  The two hidden
// layers are tcgen05 matrix products with M = 128 rows, N = 64, K = 16 (layer 1, inputs zero
// padded) and K = 64 (layer 2): the operands are staged in shared memory as bfloat16 in the
// no-swizzle K-major layout (8-row x 16-byte core matrices; LBO = stride between core matrices
// along K, SBO = stride between 8-row groups), one thread issues the MMAs, the accumulator lives
// in 64 TMEM columns and each warp reads its 32 rows back with tcgen05.ld.  Bias, SiLU and the
// 64 -> 1 output layer run on the CUDA cores.  Training adds the backward product
// delta1 = (delta2 W2) * silu'(z1) on the tensor cores (W2 transposed in shared memory) and
// accumulates the weight gradients per CTA on the CUDA cores; a second kernel sums the CTA
// partials in a fixed order and applies Adam, so a training step is deterministic.
//
// Every wait on the MMA completion barrier is bounded: on timeout the kernel records an error
// flag (read by pic_mlp_status), waits once more (bounded) so that a late MMA does not write into
// TMEM that has been freed, frees its TMEM and returns; that call's outputs are undefined.
#include <cuda_bf16.h>

#include "pic_internal.cuh"

namespace pic {

constexpr int MLP_IN = 9, MLP_H = 64, MLP_KIN = 16;
constexpr int MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;   // 4865
constexpr int OFF_W1 = 0, OFF_B1 = MLP_H * MLP_IN, OFF_W2 = OFF_B1 + MLP_H, OFF_B2 = OFF_W2 + MLP_H * MLP_H,
              OFF_W3 = OFF_B2 + MLP_H, OFF_B3 = OFF_W3 + MLP_H;
static_assert(OFF_B3 + 1 == MLP_NPARAM, "parameter layout");

__device__ int g_mlp_err;     // sticky: 1 = an MMA completion wait timed out

namespace {

constexpr int NT = 128, ROWS = 128;
constexpr long long WAIT_LIMIT = 1ll << 26;   // polls of the completion barrier (~seconds)

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle, K-major: start address, LBO (next core matrix
// along K), SBO (next 8-row group), descriptor version 1.
__device__ __forceinline__ unsigned long long mdesc(const void* p, unsigned lbo, unsigned sbo) {
    const unsigned long long a = smem_u32(p);
    return ((a >> 4) & 0x3FFFull) | ((unsigned long long)((lbo >> 4) & 0x3FFF) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D F32, A and B BF16, both K-major, N = 64, M = 128.
constexpr unsigned IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_bf16(unsigned tmem, unsigned long long a, unsigned long long b, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(tmem), "l"(a), "l"(b), "r"(IDESC), "r"(acc) : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                 ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool bar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// Bounded wait for the phase `parity` of the barrier; false after `limit` polls.
__device__ __forceinline__ bool bar_wait(unsigned long long* bar, unsigned parity, long long limit = WAIT_LIMIT) {
    for (long long i = 0; i < limit; ++i)
        if (bar_try_wait(bar, parity)) return true;
    return false;
}
// After a wait gave up: flag it, then wait once more (bounded) so that no committed MMA is
// still writing when the kernel frees its TMEM; if that wait gives up too the flag says so (2).
__device__ __forceinline__ void timed_out(unsigned long long* bar, unsigned parity) {
    const bool late = bar_wait(bar, parity);
    atomicMax(&g_mlp_err, late ? 1 : 2);
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// 16 consecutive FP32 accumulator columns of this thread's row (TMEM lane = row).
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float* v) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr) : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// Byte offset of element (row, k) of a K-major tile with KB core matrices per 8-row group.
template <int KB>
__device__ __forceinline__ int kmaj(int row, int k) {
    return (((row >> 3) * KB + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}
template <int KB>
__device__ __forceinline__ void put_bf16(unsigned char* tile, int row, int k, float v) {
    *reinterpret_cast<__nv_bfloat16*>(tile + kmaj<KB>(row, k)) = __float2bfloat16_rn(v);
}
template <int KB>
__device__ __forceinline__ float get_bf16(const unsigned char* tile, int row, int k) {
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(tile + kmaj<KB>(row, k)));
}

// Logistic sigmoid through sigma(z) = (1 + tanh(z / 2)) / 2: one special-function operation
// (tanh.approx, relative error ~2^-11, below the bfloat16 rounding of the hidden activations)
// instead of an exponential and a reciprocal.  SiLU and its derivative use it in both the
// forward and the training kernels, so training optimises the function inference evaluates.
__device__ __forceinline__ float tanh_approx(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sigmoid(float z) { return fmaf(0.5f, tanh_approx(0.5f * z), 0.5f); }
__device__ __forceinline__ float silu(float z) { return z * sigmoid(z); }
__device__ __forceinline__ float dsilu(float z) {
    const float s = sigmoid(z);
    return s * (1.f + z * (1.f - s));
}

// Eight consecutive values of one row into a K-major tile as one 16-byte store (k0 % 8 == 0).
template <int KB>
__device__ __forceinline__ void put8_bf16(unsigned char* tile, int row, int k0, const float* v) {
    uint4 q;
    unsigned* w = reinterpret_cast<unsigned*>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        w[i] = *reinterpret_cast<const unsigned*>(&b);
    }
    *reinterpret_cast<uint4*>(tile + kmaj<KB>(row, k0)) = q;
}

struct MlpArgs {
    const float* params;   // [MLP_NPARAM] FP32 master parameters
    MlpNorm norm;
    const float* x;        // feature-major: x[j * ldx + i]
    long long ldx;
    long long n;
    const float* target;   // training: [n]
    float* y;              // inference: [n]
    float* part;           // training: [gridDim.x][MLP_NPARAM + 1] gradient and loss partials
};

struct __align__(1024) MlpSmem {
    unsigned char X[ROWS * MLP_KIN * 2];      // layer-1 A: normalised inputs (K = 16)
    unsigned char H[ROWS * MLP_H * 2];        // layer-2 A: h1
    unsigned char W1[MLP_H * MLP_KIN * 2];    // layer-1 B: W1[n][k]
    unsigned char W2[MLP_H * MLP_H * 2];      // layer-2 B: W2[n][k]
    float b1[MLP_H], b2[MLP_H], w3[MLP_H];
    float b3;
    unsigned long long bar;
    unsigned tmem;
};

struct __align__(1024) MlpTrainSmem {
    MlpSmem f;
    unsigned char D[ROWS * MLP_H * 2];        // backward A: delta2 (bf16)
    unsigned char W2T[MLP_H * MLP_H * 2];     // backward B: W2 transposed, W2T[k][n] = W2[n][k]
    float buf[ROWS][MLP_H + 1];               // FP32 row-by-unit products for the column sums
    float g[MLP_NPARAM + 1];                  // this CTA's gradient and loss partials
};

// Parameters -> shared memory (bfloat16 operand tiles and FP32 vectors); zero the padding.
template <class S>
__device__ void load_params(S& s, const float* p, unsigned char* w2t) {
    const int NT = blockDim.x;
    for (int i = threadIdx.x; i < MLP_H * MLP_KIN; i += NT) {
        const int n = i / MLP_KIN, k = i % MLP_KIN;
        put_bf16<2>(s.W1, n, k, k < MLP_IN ? p[OFF_W1 + n * MLP_IN + k] : 0.f);
    }
    for (int i = threadIdx.x; i < MLP_H * MLP_H; i += NT) {
        const int n = i / MLP_H, k = i % MLP_H;
        const float w = p[OFF_W2 + i];
        put_bf16<8>(s.W2, n, k, w);
        if (w2t) put_bf16<8>(w2t, k, n, w);
    }
    for (int i = threadIdx.x; i < MLP_H; i += NT) {
        s.b1[i] = p[OFF_B1 + i];
        s.b2[i] = p[OFF_B2 + i];
        s.w3[i] = p[OFF_W3 + i];
    }
    if (threadIdx.x == 0) s.b3 = p[OFF_B3];
}

// TMEM (NCOL columns) and the completion barrier; every thread gets the TMEM address.
template <int NCOL = 64, class S>
__device__ void setup(S& s) {
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(smem_u32(&s.tmem)), "r"(NCOL) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&s.bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
}

template <int NCOL = 64, class S>
__device__ void teardown(S& s) {
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(s.tmem), "r"(NCOL) : "memory");
}

// One product into the accumulator: `ksteps` MMAs of K = 16 over the A and B tiles (KB core
// matrices per 8-row group), issued by thread 0 after the operand writes are visible to the
// tensor cores; returns false (all threads) if the completion did not arrive in time.
template <int KB>
__device__ bool product(MlpSmem& s, const unsigned char* A, const unsigned char* B, unsigned& phase) {
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x == 0) {
        constexpr unsigned LBO = 128, SBO = 128 * KB;
#pragma unroll
        for (int ks = 0; ks < KB / 2; ++ks)
            mma_bf16(s.tmem, mdesc(A + ks * 256, LBO, SBO), mdesc(B + ks * 256, LBO, SBO), ks > 0);
        mma_commit(&s.bar);
    }
    const bool ok = bar_wait(&s.bar, phase);
    if (!ok) timed_out(&s.bar, phase);
    phase ^= 1u;
    fence_after();
    return __syncthreads_and(ok);
}

// This thread's row of the accumulator (64 FP32).
__device__ __forceinline__ void read_row(const MlpSmem& s, float* v) {
    const unsigned taddr = s.tmem + ((unsigned)(threadIdx.x & ~31) << 16);
#pragma unroll
    for (int c = 0; c < MLP_H; c += 16) tmem_ld16(taddr + c, v + c);
    tmem_ld_wait();
}

// Normalised inputs of sample i into row r of the X tile (zeros past nin and past n).
__device__ __forceinline__ void stage_inputs(MlpSmem& s, const MlpArgs& m, long long i, int r, float xn[MLP_IN]) {
#pragma unroll
    for (int j = 0; j < MLP_IN; ++j) {
        float v = 0.f;
        if (i < m.n && j < m.norm.nin) v = (m.x[j * m.ldx + i] - m.norm.mu[j]) * m.norm.inv_sigma[j];
        xn[j] = __bfloat162float(__float2bfloat16_rn(v));
        put_bf16<2>(s.X, r, j, v);
    }
#pragma unroll
    for (int j = MLP_IN; j < MLP_KIN; ++j) put_bf16<2>(s.X, r, j, 0.f);
}

// ------------------------------------------------------------------ inference
// 256 threads: two sub-tiles of 128 rows (thread = sample row; warps 0-3 sub-tile 0, warps 4-7
// sub-tile 1), so each MMA round trip serves 256 samples.  Sub-tile h accumulates in TMEM
// columns 64 h .. 64 h + 63 (128 columns allocated).  The next tile's inputs are loaded while
// the tensor cores work.
constexpr int FWD_NT = 256, FWD_SUB = 2, FWD_ROWS = FWD_SUB * ROWS;

struct __align__(1024) MlpFwdSmem {
    unsigned char X[FWD_SUB][ROWS * MLP_KIN * 2];     // stride ROWS * 2 * 16 bytes (KB = 2)
    unsigned char H[FWD_SUB][ROWS * MLP_H * 2];       // stride ROWS * 8 * 16 bytes (KB = 8)
    unsigned char W1[MLP_H * MLP_KIN * 2];
    unsigned char W2[MLP_H * MLP_H * 2];
    float b1[MLP_H], b2[MLP_H], w3[MLP_H];
    float b3;
    unsigned long long bar;
    unsigned tmem;
};
static_assert(sizeof(((MlpFwdSmem*)0)->X[0]) == ROWS * 2 * 16 && sizeof(((MlpFwdSmem*)0)->H[0]) == ROWS * 8 * 16,
              "sub-tile strides");

// Both sub-tiles' products (KB core matrices per row group; sub-tile h's A tile at
// A0 + h * ROWS * KB * 16 bytes), one commit; false on timeout.
template <int KB>
__device__ bool product2(MlpFwdSmem& s, const unsigned char* A0, const unsigned char* B, unsigned& phase) {
    constexpr int ASTRIDE = ROWS * KB * 16;
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x == 0) {
        constexpr unsigned LBO = 128, SBO = 128 * KB;
#pragma unroll
        for (int h = 0; h < FWD_SUB; ++h)
#pragma unroll
            for (int ks = 0; ks < KB / 2; ++ks)
                mma_bf16(s.tmem + MLP_H * h, mdesc(A0 + h * ASTRIDE + ks * 256, LBO, SBO),
                         mdesc(B + ks * 256, LBO, SBO), ks > 0);
        mma_commit(&s.bar);
    }
    const bool ok = bar_wait(&s.bar, phase);
    if (!ok) timed_out(&s.bar, phase);
    phase ^= 1u;
    fence_after();
    return __syncthreads_and(ok);
}

__device__ __forceinline__ void load_x(const MlpArgs& m, long long i, float x[MLP_IN]) {
#pragma unroll
    for (int j = 0; j < MLP_IN; ++j) x[j] = (i < m.n && j < m.norm.nin) ? __ldg(m.x + j * m.ldx + i) : 0.f;
}

__global__ void __launch_bounds__(FWD_NT) mlp_forward_kernel(const MlpArgs m) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    MlpFwdSmem& s = *reinterpret_cast<MlpFwdSmem*>(smem_raw);
    load_params(s, m.params, nullptr);
    setup<FWD_SUB * MLP_H>(s);
    const int h = threadIdx.x >> 7, r = threadIdx.x & (ROWS - 1);
    const unsigned taddr = s.tmem + ((unsigned)(r & ~31) << 16) + MLP_H * h;
    unsigned phase = 0;
    const long long ntiles = (m.n + FWD_ROWS - 1) / FWD_ROWS;
    float xr[MLP_IN];
    load_x(m, (long long)blockIdx.x * FWD_ROWS + threadIdx.x, xr);
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long i = t * FWD_ROWS + threadIdx.x;
        float xs[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
            xs[j] = j < MLP_IN && j < m.norm.nin ? (xr[j] - m.norm.mu[j]) * m.norm.inv_sigma[j] : 0.f;
        put8_bf16<2>(s.X[h], r, 0, xs);
        put8_bf16<2>(s.X[h], r, 8, xs + 8);
        load_x(m, i + (long long)gridDim.x * FWD_ROWS, xr);      // next tile, in flight meanwhile
        if (!product2<2>(s, s.X[0], s.W1, phase)) break;
        float z[MLP_H];
#pragma unroll
        for (int c = 0; c < MLP_H; c += 16) tmem_ld16(taddr + c, z + c);
        tmem_ld_wait();
#pragma unroll
        for (int c = 0; c < MLP_H; c += 8) {
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = silu(z[c + q] + s.b1[c + q]);
            put8_bf16<8>(s.H[h], r, c, v);
        }
        if (!product2<8>(s, s.H[0], s.W2, phase)) break;
#pragma unroll
        for (int c = 0; c < MLP_H; c += 16) tmem_ld16(taddr + c, z + c);
        tmem_ld_wait();
        float y = s.b3;
#pragma unroll
        for (int k = 0; k < MLP_H; ++k) y = fmaf(s.w3[k], silu(z[k] + s.b2[k]), y);
        if (i < m.n) m.y[i] = y;
    }
    teardown<FWD_SUB * MLP_H>(s);
}

// ------------------------------------------------------------------ training
// Column sums over the 128 rows of buf into g[off + n] (thread n < 64 per column) -- fixed order.
__device__ __forceinline__ void column_sums(MlpTrainSmem& s, int off, int ncols) {
    __syncthreads();
    for (int c = threadIdx.x; c < ncols; c += NT) {
        float a = 0.f;
        for (int r = 0; r < ROWS; ++r) a += s.buf[r][c];
        s.g[off + c] += a;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(NT) mlp_train_kernel(const MlpArgs m) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    MlpTrainSmem& S = *reinterpret_cast<MlpTrainSmem*>(smem_raw);
    MlpSmem& s = S.f;
    load_params(s, m.params, S.W2T);
    for (int i = threadIdx.x; i <= MLP_NPARAM; i += NT) S.g[i] = 0.f;
    setup(s);
    unsigned phase = 0;
    const int r = threadIdx.x;
    const long long ntiles = (m.n + ROWS - 1) / ROWS;
    const float inv_n = 1.f / (float)m.n;
    bool ok = true;
    for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const long long i = t * ROWS + r;
        const bool live = i < m.n;
        float xn[MLP_IN];
        stage_inputs(s, m, i, r, xn);
        if (!(ok = product<2>(s, s.X, s.W1, phase))) break;
        float z1[MLP_H];
        read_row(s, z1);
#pragma unroll
        for (int k = 0; k < MLP_H; ++k) {
            z1[k] += s.b1[k];
            put_bf16<8>(s.H, r, k, silu(z1[k]));
        }
        if (!(ok = product<8>(s, s.H, s.W2, phase))) break;
        float z2[MLP_H];
        read_row(s, z2);
        float y = s.b3;
#pragma unroll
        for (int k = 0; k < MLP_H; ++k) {
            z2[k] += s.b2[k];
            y = fmaf(s.w3[k], silu(z2[k]), y);
        }
        const float res = live ? y - m.target[i] : 0.f;
        const float dy = 2.f * res * inv_n;
        // w3 and b3: dy * h2
#pragma unroll
        for (int k = 0; k < MLP_H; ++k) S.buf[r][k] = dy * silu(z2[k]);
        S.buf[r][MLP_H] = dy;
        column_sums(S, OFF_W3, MLP_H + 1);      // columns 0..63 -> w3, column 64 -> b3
        // delta2 = dy w3 * silu'(z2): b2 from the column sums, W2 = delta2^T h1, and the bf16
        // copy of delta2 for the backward product
#pragma unroll
        for (int k = 0; k < MLP_H; ++k) {
            const float d2 = dy * s.w3[k] * dsilu(z2[k]);
            S.buf[r][k] = d2;
            put_bf16<8>(S.D, r, k, d2);
        }
        S.buf[r][MLP_H] = res * res;
        column_sums(S, OFF_B2, MLP_H);
        if (threadIdx.x == 0) {
            float a = 0.f;
            for (int q = 0; q < ROWS; ++q) a += S.buf[q][MLP_H];
            S.g[MLP_NPARAM] += a;
        }
        // W2[n][k] += sum_r delta2[r][n] h1[r][k]: thread pairs (n, k0..k0+31)
        for (int o = threadIdx.x; o < MLP_H * 2; o += NT) {
            const int n = o >> 1, k0 = (o & 1) * 32;
            float acc[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) acc[q] = 0.f;
            for (int q = 0; q < ROWS; ++q) {
                const float d = S.buf[q][n];
#pragma unroll
                for (int kk = 0; kk < 32; ++kk) acc[kk] = fmaf(d, get_bf16<8>(s.H, q, k0 + kk), acc[kk]);
            }
#pragma unroll
            for (int kk = 0; kk < 32; ++kk) S.g[OFF_W2 + n * MLP_H + k0 + kk] += acc[kk];
        }
        // delta1 = (delta2 W2) * silu'(z1) on the tensor cores
        if (!(ok = product<8>(s, S.D, S.W2T, phase))) break;
        float d1[MLP_H];
        read_row(s, d1);
        __syncthreads();                        // buf reads of the W2 sums are done
#pragma unroll
        for (int k = 0; k < MLP_H; ++k) S.buf[r][k] = d1[k] * dsilu(z1[k]);
        column_sums(S, OFF_B1, MLP_H);
        // W1[n][j] += sum_r delta1[r][n] xn[r][j]
        for (int o = threadIdx.x; o < MLP_H * MLP_IN; o += NT) {
            const int n = o / MLP_IN, j = o % MLP_IN;
            float a = 0.f;
            for (int q = 0; q < ROWS; ++q) a = fmaf(S.buf[q][n], get_bf16<2>(s.X, q, j), a);
            S.g[OFF_W1 + n * MLP_IN + j] += a;
        }
        __syncthreads();
    }
    teardown(s);
    float* out = m.part + (size_t)blockIdx.x * (MLP_NPARAM + 1);
    for (int i = threadIdx.x; i <= MLP_NPARAM; i += NT) out[i] = S.g[i];
}

// Sum the CTA partials in order and take one Adam step (Kingma & Ba 2015, Algorithm 1).
__global__ void mlp_adam_kernel(float* params, float* am, float* av, const float* part, int nparts, int t,
                                float lr, float beta1, float beta2, float eps, long long n, float* loss) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= MLP_NPARAM; i += gridDim.x * blockDim.x) {
        float g = 0.f;
        for (int c = 0; c < nparts; ++c) g += part[(size_t)c * (MLP_NPARAM + 1) + i];
        if (i == MLP_NPARAM) {
            if (loss) *loss = g / (float)n;
            continue;
        }
        const float mi = beta1 * am[i] + (1.f - beta1) * g;
        const float vi = beta2 * av[i] + (1.f - beta2) * g * g;
        am[i] = mi;
        av[i] = vi;
        const float mh = mi / (1.f - powf(beta1, (float)t));
        const float vh = vi / (1.f - powf(beta2, (float)t));
        params[i] -= lr * mh / (sqrtf(vh) + eps);
    }
}


}  // namespace

constexpr int MLP_TRAIN_GRID = 152;

size_t mlp_train_scratch_bytes() { return (size_t)MLP_TRAIN_GRID * (MLP_NPARAM + 1) * sizeof(float); }

cudaError_t launch_mlp_forward(const float* params, const MlpNorm& norm, const float* x, long long ldx, long long n,
                               float* y, cudaStream_t s) {
    cudaError_t e = smem_attr_once((const void*)mlp_forward_kernel, (int)sizeof(MlpFwdSmem));
    if (e != cudaSuccess) return e;
    if (n <= 0) return cudaSuccess;
    MlpArgs m{params, norm, x, ldx, n, nullptr, y, nullptr};
    const long long tiles = (n + FWD_ROWS - 1) / FWD_ROWS;
    const int grid = (int)(tiles < 152LL * 4 ? tiles : 152LL * 4);
    mlp_forward_kernel<<<grid, FWD_NT, sizeof(MlpFwdSmem), s>>>(m);
    return cudaGetLastError();
}

cudaError_t launch_mlp_train(float* params, float* am, float* av, int t, float lr, const MlpNorm& norm,
                             const float* x, long long ldx, const float* target, long long n, float* loss,
                             void* scratch, cudaStream_t s) {
    cudaError_t e = smem_attr_once((const void*)mlp_train_kernel, (int)sizeof(MlpTrainSmem));
    if (e != cudaSuccess) return e;
    float* part = static_cast<float*>(scratch);
    MlpArgs m{params, norm, x, ldx, n, target, nullptr, part};
    // a fixed grid: CTA c takes tiles c, c + grid, ... so the partials and their sum are fixed
    mlp_train_kernel<<<MLP_TRAIN_GRID, NT, sizeof(MlpTrainSmem), s>>>(m);
    mlp_adam_kernel<<<20, 256, 0, s>>>(params, am, av, part, MLP_TRAIN_GRID, t, lr, 0.9f, 0.999f, 1e-8f, n, loss);
    return cudaGetLastError();
}

// Test hook: one CTA waits on a barrier that nothing arrives on (no MMA is issued), gives up
// after `polls` polls and sets the flag as a timed-out network kernel does.
__global__ void mlp_wait_test_kernel(long long polls) {
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !bar_wait(&bar, 0, polls)) atomicMax(&g_mlp_err, 1);
}

cudaError_t launch_mlp_wait_test(long long polls, cudaStream_t s) {
    mlp_wait_test_kernel<<<1, 32, 0, s>>>(polls);
    return cudaGetLastError();
}

cudaError_t mlp_status(int* err, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(err, g_mlp_err, sizeof(int));
    if (e == cudaSuccess && clear && *err) {
        const int z = 0;
        e = cudaMemcpyToSymbol(g_mlp_err, &z, sizeof(int));
    }
    return e;
}

cudaError_t preload_mlp() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, mlp_forward_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, mlp_train_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, mlp_adam_kernel);
    return e;
}

}  // namespace pic
