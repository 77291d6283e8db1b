// k_batch.cu -- device side of the batch engine: many independent
// simulations advanced by the same launches.
//
// Per step: begin_step (one CTA: which members still step, their step
// counters, their field ping-pong parity), then one persistent particle
// launch over the (simulation, tile) items of every member and one field
// launch over the (simulation, block) items.  Finished members are skipped on
// the device, so a captured CUDA graph of many steps stays valid while members
// reach their own step counts.
//
// Every sort_interval steps the free and Dirac species of all members are
// re-sorted by tile in a handful of launches over a segment table (one
// segment per species of a member): counts, per-segment scans, a scatter into
// the species' scratch half, a copy back (the pointers in the parameter
// blocks never change) and the active-tile item lists.
#include "pic_internal.cuh"

namespace pic {

namespace {

__global__ void begin_step_kernel(int n, const int *member, int *active, int *fpar,
                                  long long *done, const long long *target,
                                  long long *const *counters) {
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        if (active[s]) {  // the previous step of this member ran
            done[s] += 1;
            fpar[s] ^= 1;
        }
        active[s] = member[s] && done[s] < target[s];
        if (active[s] && counters[s]) *counters[s] += 1;  // particle phase of this step
    }
}

__global__ void finalize_kernel(int n, int *active, int *fpar, long long *done) {
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        if (active[s]) {
            done[s] += 1;
            fpar[s] ^= 1;
        }
        active[s] = 0;
    }
}

__device__ inline int seg_of(const SortSeg *segs, int nseg, long long p) {
    int lo = 0, hi = nseg;  // largest s with poff <= p
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (segs[mid].poff <= p) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ inline int tile_of(const TileP &tp, uint32_t c) {
    int tx = cell_x(c) / tp.T[0], ty = cell_y(c) / tp.T[1], tz = cell_z(c) / tp.T[2];
    return (tz * tp.nt[1] + ty) * tp.nt[0] + tx;
}

__global__ void zero_counts_kernel(const SortSeg *segs) {
    const SortSeg &S = segs[blockIdx.x];
    for (int t = threadIdx.x; t <= S.tp.ntiles; t += blockDim.x) S.count[t] = 0;
}

__global__ void batch_hist_kernel(const SortSeg *segs, int nseg, long long total) {
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += stride) {
        const long long p = base + threadIdx.x;
        const bool valid = p < total;
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        if (!valid) continue;
        const int sg = seg_of(segs, nseg, p);
        const SortSeg &S = segs[sg];
        const long long q = p - S.poff;
        const int t = tile_of(S.tp, S.src.cell[q]);
        const unsigned key = ((unsigned)sg << 20) | (unsigned)t;
        const unsigned m = __match_any_sync(vm, key);
        const int leader = __ffs(m) - 1;
        int b = 0;
        if (lane == leader) b = atomicAdd(&S.count[t], __popc(m));
        b = __shfl_sync(m, b, leader);
        S.rank[q] = b + __popc(m & ((1u << lane) - 1u));
    }
}

// exclusive scan of count[0 .. ntiles) into tile_start[0 .. ntiles], one CTA
// (1024 threads) per segment, chunk by chunk with a running carry
__global__ void batch_scan_kernel(const SortSeg *segs) {
    __shared__ int warp_sums[32];
    __shared__ int carry;
    const SortSeg &S = segs[blockIdx.x];
    const int n = S.tp.ntiles;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < n ? S.count[i] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[w] = x;
        __syncthreads();
        if (w == 0) {
            int sv = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, sv, o);
                if (lane >= o) sv += y;
            }
            warp_sums[lane] = sv;
        }
        __syncthreads();
        const int before = (w > 0 ? warp_sums[w - 1] : 0) + x - v;
        if (i < n) S.tile_start[i] = carry + before;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_sums[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) S.tile_start[n] = carry;
}

template <class T>
__device__ inline void cp(T *dst, const T *src, long long d, long long s) {
    dst[d] = src[s];
}

__global__ void batch_scatter_kernel(const SortSeg *segs, int nseg, long long total) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const SortSeg &S = segs[seg_of(segs, nseg, p)];
        const long long q = p - S.poff;
        const uint32_t c = S.src.cell[q];
        const int t = tile_of(S.tp, c);
        const long long cnt = (long long)S.tile_start[t + 1] - S.tile_start[t];
        long long P = 7919;
        if (cnt % P == 0) P = 7907;
        if (cnt % P == 0) P = 7901;
        const long long d = (long long)S.tile_start[t] + ((long long)S.rank[q] * P) % cnt;
        S.tmp.cell[d] = c;
        S.pid_tmp[d] = S.pid_src[q];
        for (int a = 0; a < 3; ++a) {
            cp(S.tmp.v[a], S.src.v[a], d, q);
            cp(S.tmp.o[a], S.src.o[a], d, q);
        }
    }
}

__global__ void batch_copyback_kernel(const SortSeg *segs, int nseg, long long total) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const SortSeg &S = segs[seg_of(segs, nseg, p)];
        const long long q = p - S.poff;
        S.src.cell[q] = S.tmp.cell[q];
        const_cast<uint32_t *>(S.pid_src)[q] = S.pid_tmp[q];
        for (int a = 0; a < 3; ++a) {
            S.src.v[a][q] = S.tmp.v[a][q];
            S.src.o[a][q] = S.tmp.o[a][q];
        }
    }
}

// items[ioff .. ioff + ntiles) of one member: its active tiles, then padding
__global__ void batch_items_kernel(const SimTiles *sims, int2 *items) {
    __shared__ int warp_sums[32];
    __shared__ int carry;
    const SimTiles &M = sims[blockIdx.x];
    const int n = M.ntiles;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int t = base + threadIdx.x;
        int f = 0;
        if (t < n)
            for (int k = 0; k < M.nsp; ++k) f |= (M.starts[k][t + 1] - M.starts[k][t]) > 0;
        int x = f;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[w] = x;
        __syncthreads();
        if (w == 0) {
            int sv = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, sv, o);
                if (lane >= o) sv += y;
            }
            warp_sums[lane] = sv;
        }
        __syncthreads();
        const int pos = carry + (w > 0 ? warp_sums[w - 1] : 0) + x - f;
        if (f) items[M.ioff + pos] = make_int2(M.sim, t);
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_sums[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    for (int k = carry + threadIdx.x; k < n; k += blockDim.x) items[M.ioff + k] = make_int2(M.sim, -1);
}

int grid_for(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

}  // namespace

cudaError_t launch_begin_step(int n, const int *member, int *active, int *fpar, long long *done,
                              const long long *target, long long *const *counters, cudaStream_t s) {
    begin_step_kernel<<<1, 1024, 0, s>>>(n, member, active, fpar, done, target, counters);
    return cudaGetLastError();
}

cudaError_t launch_finalize(int n, int *active, int *fpar, long long *done, cudaStream_t s) {
    finalize_kernel<<<1, 1024, 0, s>>>(n, active, fpar, done);
    return cudaGetLastError();
}

cudaError_t launch_batch_sort(const SortSeg *segs, int nseg, long long total, cudaStream_t s,
                              int *nlaunch) {
    *nlaunch = 0;
    if (nseg <= 0) return cudaSuccess;
    zero_counts_kernel<<<nseg, 256, 0, s>>>(segs);
    if (total > 0) batch_hist_kernel<<<grid_for(total), 256, 0, s>>>(segs, nseg, total);
    batch_scan_kernel<<<nseg, 1024, 0, s>>>(segs);
    if (total > 0) {
        batch_scatter_kernel<<<grid_for(total), 256, 0, s>>>(segs, nseg, total);
        batch_copyback_kernel<<<grid_for(total), 256, 0, s>>>(segs, nseg, total);
    }
    *nlaunch = total > 0 ? 5 : 2;
    return cudaGetLastError();
}

cudaError_t launch_batch_items(const SimTiles *sims, int nsims, int2 *items, cudaStream_t s) {
    if (nsims <= 0) return cudaSuccess;
    batch_items_kernel<<<nsims, 1024, 0, s>>>(sims, items);
    return cudaGetLastError();
}

}  // namespace pic
