// sort.cu -- periodic counting-sort re-binning of particles by tile-major cell key.
//
// key(cell) = cell_off + tile_index * (TX*TY*TZ) + local index within the tile, so after a
// sort each tile's particles are one contiguous range [start[key0], start[key0 + TX*TY*TZ]).
// Three passes per species: histogram (warp-aggregated atomics), exclusive scan of the counts
// (block scans + a scan of block sums), scatter into the other buffer (warp-aggregated cursor
// atomics); then the buffer parity flips on the device.  The order of particles within a cell
// is not fixed; nothing downstream depends on it (the deposit is integer).
#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int NT = 256;
constexpr int ITEMS = 8;                 // scan items per thread
constexpr int CHUNK = NT * ITEMS;        // keys per scan block
constexpr unsigned FULL = 0xffffffffu;

struct TileShape { int tx, ty, tz; };

__device__ __forceinline__ int find_run(const RunDev* runs, int nruns, int cell) {
    int lo = 0, hi = nruns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (runs[mid].cell_off <= cell) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int tile_key(const RunDev& R, int cell, TileShape T) {
    const int lc = cell - R.cell_off;
    const int nxy = R.nx * R.ny;
    const int cz = lc / nxy;
    const int r = lc - cz * nxy;
    const int cy = r / R.nx, cx = r - cy * R.nx;
    const int tx = cx / T.tx, ty = cy / T.ty, tz = cz / T.tz;
    const int lx = cx - tx * T.tx, ly = cy - ty * T.ty, lz = cz - tz * T.tz;
    const int tile = (tz * R.nty + ty) * R.ntx + tx;
    return R.cell_off + tile * (T.tx * T.ty * T.tz) + (lz * T.ty + ly) * T.tx + lx;
}

__global__ void __launch_bounds__(NT) count_kernel(Args a, int s, int nruns, TileShape T) {
    const SpeciesBuf B = a.buf[s][a.ctl->parity[s]];
    const long long n = a.npart[s];
    const int lane = threadIdx.x & 31;
    int* __restrict__ count = a.count[s];
    for (long long base = (blockIdx.x * (long long)NT + (threadIdx.x & ~31)); base < n;
         base += (long long)gridDim.x * NT) {
        const long long p = base + lane;
        int key = -1 - lane;
        if (p < n) {
            const int cell = B.cell[p];
            key = tile_key(a.runs[find_run(a.runs, nruns, cell)], cell, T);
        }
        const unsigned peers = __match_any_sync(FULL, key);
        if (p < n && lane == __ffs(peers) - 1) atomicAdd(&count[key], __popc(peers));
    }
}

// Exclusive scan of count[0..n) into start[0..n), block sums into tmp.
__global__ void __launch_bounds__(NT) scan_blocks(const int* __restrict__ count, int* __restrict__ start,
                                                  int* __restrict__ tmp, long long n) {
    __shared__ int warp_sums[NT / 32];
    const long long off = (long long)blockIdx.x * CHUNK + (long long)threadIdx.x * ITEMS;
    int v[ITEMS];
    int sum = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        v[i] = off + i < n ? count[off + i] : 0;
        sum += v[i];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < NT / 32 ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += t;
        }
        if (lane < NT / 32) warp_sums[lane] = w;   // inclusive
    }
    __syncthreads();
    int run = incl - sum + (warp > 0 ? warp_sums[warp - 1] : 0);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (off + i < n) start[off + i] = run;
        run += v[i];
    }
    if (threadIdx.x == NT - 1) tmp[blockIdx.x] = warp_sums[NT / 32 - 1];
}

// In-place exclusive scan of tmp[0..m) by one block, chunk by chunk with a running carry.
__global__ void __launch_bounds__(NT) scan_tmp(int* __restrict__ tmp, int m, int* __restrict__ total) {
    __shared__ int warp_sums[NT / 32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < m; base += NT) {
        const int i = base + threadIdx.x;
        const int x = i < m ? tmp[i] : 0;
        int incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int w = lane < NT / 32 ? warp_sums[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(FULL, w, o);
                if (lane >= o) w += t;
            }
            if (lane < NT / 32) warp_sums[lane] = w;
        }
        __syncthreads();
        const int excl = carry + incl - x + (warp > 0 ? warp_sums[warp - 1] : 0);
        if (i < m) tmp[i] = excl;
        __syncthreads();
        if (threadIdx.x == NT - 1) carry = excl + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(NT) scan_add(int* __restrict__ start, int* __restrict__ cursor,
                                               const int* __restrict__ tmp, long long n) {
    const long long off = (long long)blockIdx.x * CHUNK;
    const int add = tmp[blockIdx.x];
    for (int i = threadIdx.x; i < CHUNK; i += NT) {
        const long long k = off + i;
        if (k < n) {
            const int v = start[k] + add;
            start[k] = v;
            cursor[k] = v;
        }
    }
}

__global__ void __launch_bounds__(NT) scatter_kernel(Args a, int s, int nruns, TileShape T) {
    const int par = a.ctl->parity[s];
    const SpeciesBuf S = a.buf[s][par];
    const SpeciesBuf D = a.buf[s][par ^ 1];
    const long long n = a.npart[s];
    const int lane = threadIdx.x & 31;
    int* __restrict__ cursor = a.cursor[s];
    for (long long base = (blockIdx.x * (long long)NT + (threadIdx.x & ~31)); base < n;
         base += (long long)gridDim.x * NT) {
        const long long p = base + lane;
        int key = -1 - lane, cell = 0;
        if (p < n) {
            cell = S.cell[p];
            key = tile_key(a.runs[find_run(a.runs, nruns, cell)], cell, T);
        }
        const unsigned peers = __match_any_sync(FULL, key);
        const int leader = __ffs(peers) - 1;
        int pos = 0;
        if (p < n && lane == leader) pos = atomicAdd(&cursor[key], __popc(peers));
        pos = __shfl_sync(FULL, pos, leader) + __popc(peers & ((1u << lane) - 1u));
        if (p < n) {
            D.cell[pos] = cell;
            for (int d = 0; d < a.ndim; ++d) D.o[d][pos] = S.o[d][p];
#pragma unroll
            for (int d = 0; d < 3; ++d) D.u[d][pos] = S.u[d][p];
            if (S.id) D.id[pos] = S.id[p];
        }
    }
}

__global__ void flip_kernel(Ctl* ctl, int s) { ctl->parity[s] ^= 1; }

int grid_for(long long n) {
    long long g = (n + NT - 1) / NT;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_sort(const Args& a, int s, int tile_x, int tile_y, int tile_z, cudaStream_t st) {
    const long long n = a.npart[s];
    const long long nk = a.nkeys;
    const TileShape T{tile_x, tile_y, tile_z};
    cudaError_t e = cudaMemsetAsync(a.count[s], 0, sizeof(int) * nk, st);
    if (e != cudaSuccess) return e;
    if (n > 0) count_kernel<<<grid_for(n), NT, 0, st>>>(a, s, a.nruns, T);
    const int nb = (int)((nk + CHUNK - 1) / CHUNK);
    scan_blocks<<<nb, NT, 0, st>>>(a.count[s], a.start[s], a.scan_tmp, nk);
    scan_tmp<<<1, NT, 0, st>>>(a.scan_tmp, nb, a.start[s] + nk);
    scan_add<<<nb, NT, 0, st>>>(a.start[s], a.cursor[s], a.scan_tmp, nk);
    if (n > 0) scatter_kernel<<<grid_for(n), NT, 0, st>>>(a, s, a.nruns, T);
    flip_kernel<<<1, 1, 0, st>>>(a.ctl, s);
    return cudaGetLastError();
}

int sort_launches(long long n) { return n > 0 ? 6 : 4; }

}  // namespace pic
