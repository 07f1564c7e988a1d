// bins.cu -- counting-sort binning of particles into per-unit slots (a unit is a cell in 2D and
// a tile of the 3D particle kernel in 3D), and the inverse compaction.
//
// Binning (load): each particle takes the next free slot of its unit with an atomic per-unit
// counter (a counting sort into fixed-capacity bins; in 3D the particle's cell within the tile
// is stored beside it); a particle whose unit is full goes to the species' spill list.  Counters
// may exceed the capacity; readers clamp them.  The step kernels rebin every particle into the
// other buffer the same way, fused into the push.
// Compaction (read-back): exclusive scan of the clamped counts, then each unit's particles are
// copied to a dense array in unit order (2D: cell order), followed by the spill list.
#include <mutex>

#include "../../include/pic.h"
#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int NT = 256;
constexpr int ITEMS = 8;                 // scan items per thread
constexpr int CHUNK = NT * ITEMS;        // keys per scan block
constexpr unsigned FULL = 0xffffffffu;

int grid_for(long long n) {
    long long g = (n + NT - 1) / NT;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g < 1 ? 1 : g);
}

// src.cell non-null: read the particles from src (arrays the device can address, e.g. the
// caller's pinned host arrays) instead of the staging area.
__global__ void __launch_bounds__(NT) bin_kernel(Args a, int s, long long n, bool with_ids, long long cell_base,
                                                 long long ncell_lim, const int* gate, Stage src) {
    if (gate && *gate == 0) return;
    const int par = a.ctl->parity;
    const Slots S = a.slot[s][par];
    const Stage T = src.cell ? src : stage_of(a, s, par);
    const int cap = a.cap[s];
    if (n < 0) n = a.ctl->staged[s];   // after a compaction
    const int lane = threadIdx.x & 31;
    const int cs = a.cap_stay[s];
    // whole warps per iteration: the lanes claiming slots of one unit take them with one atomic
    // (input in cell order sends a warp's particles to one or a few units)
    for (long long p0 = blockIdx.x * (long long)NT + (threadIdx.x & ~31); p0 < n; p0 += (long long)gridDim.x * NT) {
        const long long p = p0 + lane;
        bool ok = p < n;
        int cl = 0;
        float ov[3] = {0.f, 0.f, 0.f}, uv[3] = {0.f, 0.f, 0.f};
        if (ok) {
            cl = T.cell[p];
            ok = cl >= 0 && cl < ncell_lim;
            for (int d = 0; d < a.ndim; ++d) {
                ov[d] = T.o[d][p];
                ok = ok && ov[d] >= 0.f && ov[d] < 1.f;
            }
            for (int d = 0; d < 3; ++d) {
                uv[d] = T.u[d][p];
                ok = ok && isfinite(uv[d]) && fabsf(uv[d]) < 1e6f;
            }
            if (!ok) atomicOr(&a.ctl->err, ERR_BADPART);
        }
        const unsigned okm = __ballot_sync(0xffffffffu, ok);
        if (!ok) continue;
        const long long c = cell_base + cl;
        const int id = with_ids ? T.id[p] : (int)p;
        int lc;
        const long long unit = unit_of_cell(a, c, &lc);
        const unsigned grp = __match_any_sync(okm, unit);
        const int lead = __ffs(grp) - 1;
        int base = 0;
        if (lane == lead) base = atomicAdd(&S.count[unit], __popc(grp));
        int pos = __shfl_sync(grp, base, lead) + __popc(grp & ((1u << lane) - 1u));
        if (pos >= cs) {
            const int pi = atomicAdd(&S.icount[unit], 1);
            pos = pi < cap - cs ? cs + pi : cap;
        }
        if (pos < cap) {
            const size_t q = slot_elt(S, unit * cap + pos);
            for (int d = 0; d < a.ndim; ++d) S.o[d][q] = ov[d];
            for (int d = 0; d < 3; ++d) S.u[d][q] = uv[d];
            if (S.id) S.id[q] = id;
            if (S.lc) S.lc[q] = lc;
        } else {
            const int sp = atomicAdd(S.sn, 1);
            if (sp < a.spill_cap[s]) {
                S.scell[sp] = (int)c;
                for (int d = 0; d < a.ndim; ++d) S.so[d][sp] = ov[d];
                for (int d = 0; d < 3; ++d) S.su[d][sp] = uv[d];
                if (S.sid) S.sid[sp] = id;
            } else {
                atomicOr(&a.ctl->err, ERR_SPILL_FULL);
            }
        }
    }
}

// Exclusive scan of the particles per unit (both slot areas) into start, block sums into tmp.
__global__ void __launch_bounds__(NT) scan_blocks(Args a, int s, long long c0, int* __restrict__ start,
                                                  int* __restrict__ tmp, long long n, const int* gate) {
    if (gate && *gate == 0) return;
    const Slots S = a.slot[s][a.ctl->parity];
    const int cap = a.cap[s], cs = a.cap_stay[s];
    __shared__ int warp_sums[NT / 32];
    const long long off = (long long)blockIdx.x * CHUNK + (long long)threadIdx.x * ITEMS;
    int v[ITEMS];
    int sum = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        v[i] = off + i < n ? cell_range(S, cap, cs, c0 + off + i).n : 0;
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
__global__ void __launch_bounds__(NT) scan_tmp(int* __restrict__ tmp, int m, int* __restrict__ total,
                                               const int* gate) {
    if (gate && *gate == 0) return;
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

__global__ void __launch_bounds__(NT) scan_add(int* __restrict__ start, const int* __restrict__ tmp, long long n,
                                               const int* gate) {
    if (gate && *gate == 0) return;
    const long long off = (long long)blockIdx.x * CHUNK;
    const int add = tmp[blockIdx.x];
    for (int i = threadIdx.x; i < CHUNK; i += NT) {
        const long long k = off + i;
        if (k < n) start[k] += add;
    }
}

// One thread per unit of [c0, c0 + nc): copy its slots to the staging arrays at start[c - c0] ...
// in unit order, with the cell index minus cell_base; the spill entries of the cells
// [cell_lo, cell_lo + ncells) follow at start[nc] (their order is not fixed).
__global__ void __launch_bounds__(NT) compact_kernel(Args a, int s, long long c0, long long nc, long long cell_lo,
                                                     long long ncells, long long cell_base, const int* gate) {
    if (gate && *gate == 0) return;
    const int par = a.ctl->parity;
    const Slots S = a.slot[s][par];
    const Stage T = stage_of(a, s, par);
    const int cap = a.cap[s];
    const int* __restrict__ start = a.start;
    const int cs = a.cap_stay[s];
    for (long long k = blockIdx.x * (long long)NT + threadIdx.x; k < nc; k += (long long)gridDim.x * NT) {
        const long long c = c0 + k;
        const CellRange cr = cell_range(S, cap, cs, c);
        const int b = start[k];
        const RunDev* R = S.lc ? &a.runs[run_of_unit(a, c)] : nullptr;
        for (int i = 0; i < cr.n; ++i) {
            const size_t q = slot_elt(S, (long long)slot_of(c, cap, cs, cr.ns, i));
            T.cell[b + i] = (int)((S.lc ? cell_of_unit(a, *R, c, S.lc[q]) : c) - cell_base);
            for (int d = 0; d < a.ndim; ++d) T.o[d][b + i] = S.o[d][q];
            for (int d = 0; d < 3; ++d) T.u[d][b + i] = S.u[d][q];
            T.id[b + i] = S.id ? S.id[q] : 0;
        }
    }
    const int ns = min(*S.sn, a.spill_cap[s]);
    for (int k = blockIdx.x * NT + threadIdx.x; k < ns; k += gridDim.x * NT) {
        const long long c = S.scell[k];
        if (c < cell_lo || c >= cell_lo + ncells) continue;
        const int b = start[nc] + atomicAdd(&a.ctl->staged[s], 1);
        T.cell[b] = (int)(c - cell_base);
        for (int d = 0; d < a.ndim; ++d) T.o[d][b] = S.so[d][k];
        for (int d = 0; d < 3; ++d) T.u[d][b] = S.su[d][k];
        T.id[b] = S.sid ? S.sid[k] : 0;
    }
}

// After a compaction: staged count = slot particles + the spill entries appended.
__global__ void staged_total_kernel(Args a, int s, long long nc, const int* gate) {
    if (gate && *gate == 0) return;
    a.ctl->staged[s] += a.start[nc];
}
__global__ void staged_zero_kernel(Args a, int s, const int* gate) {
    if (gate && *gate == 0) return;
    a.ctl->staged[s] = 0;
}

// Gate of the periodic re-sort.  The spill kernel processes spilled particles every step, so the
// list only needs repacking before it can fill: re-sort when any species' list has grown by more
// than 1/16 of its capacity since the last re-sort.  (Particles of cells denser than their slots,
// as in pinched filaments, stay in the list after a re-sort; counting from the last fill keeps
// them from triggering a full sort every interval.)
__global__ void spill_gate_kernel(Args a) {
    int any = 0;
    for (int s = 0; s < a.nspecies; ++s)
        any |= *a.slot[s][a.ctl->parity].sn > a.ctl->spill_base[s] + a.spill_cap[s] / 16;
    *a.gate = any;
}

// After a gated re-sort: the new fill of every spill list is the base of the next gate.
__global__ void spill_base_kernel(Args a) {
    if (*a.gate == 0) return;
    for (int s = 0; s < a.nspecies; ++s) a.ctl->spill_base[s] = min(*a.slot[s][a.ctl->parity].sn, a.spill_cap[s]);
}

// Zero the counts and spill counter of species s in the current buffer (before re-binning).
__global__ void clear_current_kernel(Args a, int s, const int* gate) {
    if (gate && *gate == 0) return;
    const Slots S = a.slot[s][a.ctl->parity];
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.nunit;
         c += (long long)gridDim.x * blockDim.x) {
        S.count[c] = 0;
        S.icount[c] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *S.sn = 0;
}

// Zero the per-unit counts and spill counters of the buffer the next step writes.
__global__ void clear_next_kernel(Args a) {
    const int nb = a.ctl->parity ^ 1;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.nunit;
         c += (long long)gridDim.x * blockDim.x)
        for (int s = 0; s < a.nspecies; ++s) {
            a.slot[s][nb].count[c] = 0;
            a.slot[s][nb].icount[c] = 0;
        }
    if (blockIdx.x == 0 && threadIdx.x < a.nspecies) *a.slot[threadIdx.x][nb].sn = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.xo_n) *a.xo_n = 0;
}

// ------------------------------------------------------------------ standalone counting sort
__global__ void __launch_bounds__(NT) zero_kernel(int* __restrict__ p, long long n) {
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) p[i] = 0;
}

// Histogram of cells with warp-aggregated atomics (lanes of equal cell add once).
__global__ void __launch_bounds__(NT) cell_hist_kernel(const int* __restrict__ cell, long long n, int ncell,
                                                       int* __restrict__ count) {
    const int lane = threadIdx.x & 31;
    for (long long base = blockIdx.x * (long long)NT + (threadIdx.x & ~31); base < n; base += (long long)gridDim.x * NT) {
        const long long p = base + lane;
        int key = -1 - lane;
        if (p < n) {
            const int c = cell[p];
            if (c >= 0 && c < ncell) key = c;
        }
        const unsigned peers = __match_any_sync(FULL, key);
        if (key >= 0 && lane == __ffs(peers) - 1) atomicAdd(&count[key], __popc(peers));
    }
}

// Plain exclusive scan of count[0..n) into start (block sums into tmp).
__global__ void __launch_bounds__(NT) plain_scan_blocks(const int* __restrict__ count, int* __restrict__ start,
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
        if (lane < NT / 32) warp_sums[lane] = w;
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

// start += block offsets; the cursors (count array reused) start at the cell starts.
__global__ void __launch_bounds__(NT) scan_add_cursor(int* __restrict__ start, int* __restrict__ cursor,
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

// Scatter particle indices to their cell's range (warp-aggregated cursor claims).
__global__ void __launch_bounds__(NT) cell_scatter_kernel(const int* __restrict__ cell, long long n, int ncell,
                                                          int* __restrict__ cursor, int* __restrict__ order) {
    const int lane = threadIdx.x & 31;
    for (long long base = blockIdx.x * (long long)NT + (threadIdx.x & ~31); base < n; base += (long long)gridDim.x * NT) {
        const long long p = base + lane;
        int key = -1 - lane;
        if (p < n) {
            const int c = cell[p];
            if (c >= 0 && c < ncell) key = c;
        }
        const unsigned peers = __match_any_sync(FULL, key);
        const int leader = __ffs(peers) - 1;
        int pos = 0;
        if (key >= 0 && lane == leader) pos = atomicAdd(&cursor[key], __popc(peers));
        pos = __shfl_sync(FULL, pos, leader) + __popc(peers & ((1u << lane) - 1u));
        if (key >= 0) order[pos] = (int)p;
    }
}

}  // namespace

// Scratch layout of the standalone counting sort: count/cursor [ncell] then block sums.
size_t bin_cells_scratch_bytes(long long ncell) {
    const long long nb = (ncell + CHUNK - 1) / CHUNK + 1;
    return (size_t)((4 * (ncell + nb) + 255) / 256 * 256);
}

cudaError_t launch_bin_cells(const int* cell, long long n, int ncell, int* start, int* order, int* scratch,
                             cudaStream_t st) {
    int* count = scratch;
    int* tmp = scratch + ncell;
    const int nb = (int)((ncell + CHUNK - 1) / CHUNK);
    zero_kernel<<<grid_for(ncell), NT, 0, st>>>(count, ncell);
    if (n > 0) cell_hist_kernel<<<grid_for(n), NT, 0, st>>>(cell, n, ncell, count);
    plain_scan_blocks<<<nb, NT, 0, st>>>(count, start, tmp, ncell);
    scan_tmp<<<1, NT, 0, st>>>(tmp, nb, start + ncell, nullptr);
    scan_add_cursor<<<nb, NT, 0, st>>>(start, count, tmp, ncell);
    if (n > 0) cell_scatter_kernel<<<grid_for(n), NT, 0, st>>>(cell, n, ncell, count, order);
    return cudaGetLastError();
}

// Scratch of the allocation-free counting sort: count/cursor for up to the maximum number of
// cells, then the scan's block sums.  Device code could name it directly; host code only holds a
// stand-in for it, so the entry point passes the device address found below.
static __device__ __align__(256) int g_bin_scratch[PIC_BIN_NOALLOC_MAX_CELLS + PIC_BIN_NOALLOC_MAX_CELLS / 2048 + 64];

// Device address of g_bin_scratch on the current device, looked up once per device.
cudaError_t noalloc_bin_scratch(int** out) {
    static std::mutex mu;
    static int* addr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bin_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = static_cast<int*>(p);
    }
    *out = addr[dev];
    return cudaSuccess;
}

cudaError_t launch_bin(const Args& a, int s, long long n, bool with_ids, long long cell_base,
                       long long ncell_lim, const int* gate, cudaStream_t st, const Stage* src) {
    if (n == 0) return cudaSuccess;
    const int g = n > 0 ? grid_for(n) : 152 * 16;
    Stage none{};
    bin_kernel<<<g, NT, 0, st>>>(a, s, n, with_ids, cell_base, ncell_lim, gate, src ? *src : none);
    return cudaGetLastError();
}

cudaError_t launch_compact(const Args& a, int s, long long c0, long long nc, long long cell_lo, long long ncells,
                           long long cell_base, const int* gate, cudaStream_t st) {
    const int nb = (int)((nc + CHUNK - 1) / CHUNK);
    scan_blocks<<<nb, NT, 0, st>>>(a, s, c0, a.start, a.scan_tmp, nc, gate);
    scan_tmp<<<1, NT, 0, st>>>(a.scan_tmp, nb, a.start + nc, gate);
    scan_add<<<nb, NT, 0, st>>>(a.start, a.scan_tmp, nc, gate);
    staged_zero_kernel<<<1, 1, 0, st>>>(a, s, gate);
    compact_kernel<<<grid_for(nc), NT, 0, st>>>(a, s, c0, nc, cell_lo, ncells, cell_base, gate);
    staged_total_kernel<<<1, 1, 0, st>>>(a, s, nc, gate);
    return cudaGetLastError();
}

cudaError_t launch_spill_gate(const Args& a, cudaStream_t st) {
    spill_gate_kernel<<<1, 1, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_clear_current(const Args& a, int s, const int* gate, cudaStream_t st) {
    clear_current_kernel<<<grid_for(a.nunit), NT, 0, st>>>(a, s, gate);
    return cudaGetLastError();
}

cudaError_t launch_clear_next(const Args& a, cudaStream_t st) {
    clear_next_kernel<<<grid_for(a.nunit), NT, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t preload_bins() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, bin_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, scan_blocks);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, scan_tmp);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, scan_add);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, compact_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, spill_gate_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, spill_base_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, clear_current_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, clear_next_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, staged_total_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, staged_zero_kernel);
    return e;
}

cudaError_t launch_resort(const Args& a, cudaStream_t st, int* launches) {
    spill_gate_kernel<<<1, 1, 0, st>>>(a);
    int l = 1;
    for (int s = 0; s < a.nspecies; ++s) {
        cudaError_t e = launch_compact(a, s, 0, a.nunit, 0, a.ncell, 0, a.gate, st);
        if (e != cudaSuccess) return e;
        clear_current_kernel<<<grid_for(a.nunit), NT, 0, st>>>(a, s, a.gate);
        // n < 0: the bin kernel takes the staged count recorded by the compaction
        bin_kernel<<<152 * 16, NT, 0, st>>>(a, s, -1, true, 0, a.ncell, a.gate, Stage{});
        l += 8;
    }
    spill_base_kernel<<<1, 1, 0, st>>>(a);
    *launches += l + 1;
    return cudaGetLastError();
}

}  // namespace pic
