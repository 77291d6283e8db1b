// k_sort.cu -- counting sort of particles by tile, prefix sums, the active
// tile list and per-cell particle counts.
//
// The sort keeps each species' SoA arrays grouped by particle tile so that
// one CTA of the particle kernel finds the particles of its tile in one
// contiguous range (tile_start[t] .. tile_start[t+1]).  Order inside a tile
// is the order in which warps claimed slots (it carries no meaning).
#include <algorithm>

#include "pic_internal.cuh"

namespace pic {

namespace {

__device__ inline int tile_of(const TileP &tp, uint32_t c) {
    int tx = cell_x(c) / tp.T[0], ty = cell_y(c) / tp.T[1], tz = cell_z(c) / tp.T[2];
    return (tz * tp.nt[1] + ty) * tp.nt[0] + tx;
}

// count[t] += particles of tile t; rank[p] = slot of p inside its tile.
// Warp-aggregated: lanes with the same tile share one atomic.
__global__ void tile_hist_kernel(TileP tp, const uint32_t *cell, long long n, int *count,
                                 int *rank) {
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += stride) {
        long long p = base + threadIdx.x;
        bool valid = p < n;
        unsigned vm = __ballot_sync(0xffffffffu, valid);
        if (!valid) continue;
        int t = tile_of(tp, cell[p]);
        unsigned m = __match_any_sync(vm, t);
        int leader = __ffs(m) - 1;
        int b = 0;
        if (lane == leader) b = atomicAdd(&count[t], __popc(m));
        b = __shfl_sync(m, b, leader);
        rank[p] = b + __popc(m & ((1u << lane) - 1u));
    }
}

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ inline int block_excl_scan(int v, int *total) {
    __shared__ int warp_sums[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < (blockDim.x >> 5) ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    int before = w > 0 ? warp_sums[w - 1] : 0;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void scan_reduce_kernel(const int *in, long long n, int *sums) {
    long long base = (long long)blockIdx.x * kScanChunk;
    int s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        long long i = base + (long long)threadIdx.x * kScanItems + k;
        if (i < n) s += in[i];
    }
    int total;
    block_excl_scan(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// out[i] = offsets[block] + exclusive scan inside the block; out[n] = total
__global__ void scan_down_kernel(const int *in, long long n, const int *offsets, int *out) {
    long long base = (long long)blockIdx.x * kScanChunk;
    int v[kScanItems];
    int s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        long long i = base + (long long)threadIdx.x * kScanItems + k;
        v[k] = i < n ? in[i] : 0;
        s += v[k];
    }
    int total;
    int pre = block_excl_scan(s, &total) + (offsets ? offsets[blockIdx.x] : 0);
    for (int k = 0; k < kScanItems; ++k) {
        long long i = base + (long long)threadIdx.x * kScanItems + k;
        if (i < n) out[i] = pre;
        pre += v[k];
        if (i == n - 1) out[n] = pre;
    }
}

template <class T>
__device__ inline void mv(T *dst, const T *src, long long d, long long s) {
    dst[d] = src[s];
}

__global__ void tile_scatter_kernel(TileP tp, SpeciesP src, const uint32_t *pid_src, SpeciesP dst,
                                    uint32_t *pid_dst, const int *start, const int *rank,
                                    int spread) {
    const long long n = src.n;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        uint32_t c = src.cell[p];
        const int t = tile_of(tp, c);
        // Spread the slots of a tile with a multiplicative permutation so
        // that consecutive particles (one warp) land in different cells and
        // their shared-memory current atomics do not collide.
        const long long cnt = (long long)start[t + 1] - start[t];
        long long P = 7919;
        if (cnt % P == 0) P = 7907;
        if (cnt % P == 0) P = 7901;
        long long d = (long long)start[t] + (spread ? ((long long)rank[p] * P) % cnt : rank[p]);
        dst.cell[d] = c;
        pid_dst[d] = pid_src[p];
        for (int a = 0; a < 3; ++a) mv(dst.v[a], src.v[a], d, p);
        if (src.kind == PIC_BOUND) {
            for (int a = 0; a < 3; ++a) {
                mv(const_cast<double *>(dst.anchor[a]), src.anchor[a], d, p);
                mv(const_cast<float *>(dst.anchor32[a]), src.anchor32[a], d, p);
                mv(dst.disp[a], src.disp[a], d, p);
            }
        } else {
            for (int a = 0; a < 3; ++a) mv(dst.o[a], src.o[a], d, p);
        }
    }
}

// Cell-interleaved order inside a tile.  The tile's cells (x fastest) are
// cut into chunks of `chunk` consecutive cells -- the particle kernel's CTA
// width -- and each chunk's particles are arranged by their rank inside
// their cell first and by their cell second.  The lanes of a warp then sit
// in consecutive cells (the gather's shared loads spread over the banks),
// and a thread of the particle kernel, which takes every chunk-th particle,
// meets the particles of one cell in a row (its current can be summed in
// registers before it goes to the shared J tile).  Inside chunk h the
// particle of rank r in cell c goes to
//   (particles of the chunks before h) + sum_{r' < r} N_{h,r'}
//     + #{c' in h, c' < c : count(c') > r},
// N_{h,r'} the number of cells of h with more than r' particles.  One CTA
// per tile; src holds each tile's particles contiguously (from the tile
// scatter), dst receives them in the same range.  A tile whose fullest cell
// holds more than rmax particles is written in plain cell order (rank inside
// the cell last) instead.
__device__ inline int local_cell_index(const TileP &tp, int t, uint32_t c) {
    const int tx = t % tp.nt[0], ty = (t / tp.nt[0]) % tp.nt[1], tz = t / (tp.nt[0] * tp.nt[1]);
    const int lx = cell_x(c) - tx * tp.T[0], ly = cell_y(c) - ty * tp.T[1];
    const int lz = cell_z(c) - tz * tp.T[2];
    return (lz * tp.T[1] + ly) * tp.T[0] + lx;
}

// exclusive scan of the counts over the ncl cells, each thread owning a run
// of consecutive cells; out[ncl] = the total (scratch: 32 ints)
__device__ inline void block_scan_counts(const int *cnt, int ncl, int *out, int *wsum) {
    const int per = (ncl + blockDim.x - 1) / blockDim.x;
    const int c0 = min(threadIdx.x * per, ncl), c1 = min(c0 + per, ncl);
    int sum = 0;
    for (int c = c0; c < c1; ++c) sum += cnt[c];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int v = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    int run = (w > 0 ? wsum[w - 1] : 0) + x - sum;
    for (int c = c0; c < c1; ++c) {
        out[c] = run;
        run += cnt[c];
    }
    if (threadIdx.x == blockDim.x - 1) out[ncl] = wsum[(blockDim.x >> 5) - 1];
    __syncthreads();  // wsum is reused
}

// One CTA per tile (blockDim = chunk).  The chunks are reordered one after
// another: thread t stands for cell lo + t of the chunk, and for every rank
// r a warp ballot of (count > r) gives the cells before it within the warp;
// the warps' totals give the rest (two barriers per chunk, whatever the
// largest count).
__global__ void tile_interleave_kernel(TileP tp, SpeciesP src, const uint32_t *pid_src,
                                       SpeciesP dst, uint32_t *pid_dst, const int *start,
                                       int *rank, int rmax, int chunk) {
    extern __shared__ int sm[];
    __shared__ int wsum[32];
    __shared__ int s_R;
    const int t = blockIdx.x;
    const int a = start[t], b = start[t + 1];
    if (a == b) return;
    const int ncl = tp.T[0] * tp.T[1] * tp.T[2];
    const int nw = blockDim.x >> 5;
    int *cnt = sm;                      // [ncl]
    int *cs = cnt + ncl;                // [ncl + 1]: particles in the cells before c
    int *pre = cs + ncl + 1;            // [rmax + 1]: particles of the ranks below r (chunk)
    int *wt = pre + rmax + 1;           // [rmax][nw]: cells above rank r, per warp
    int *tab = wt + rmax * nw;          // [rmax][chunk]: cells before c above rank r (chunk)
    for (int c = threadIdx.x; c < ncl; c += blockDim.x) cnt[c] = 0;
    __syncthreads();
    for (int i = a + threadIdx.x; i < b; i += blockDim.x)
        rank[i] = atomicAdd(&cnt[local_cell_index(tp, t, src.cell[i])], 1);
    __syncthreads();
    block_scan_counts(cnt, ncl, cs, wsum);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    for (int lo = 0; lo < ncl; lo += chunk) {
        const int hi = min(lo + chunk, ncl);
        const int c = lo + threadIdx.x;
        const int k = c < hi ? cnt[c] : 0;
        if (threadIdx.x == 0) s_R = 0;
        __syncthreads();
        if (k > 0) atomicMax(&s_R, k);
        __syncthreads();
        const int R = s_R;
        const bool inter = R <= rmax;
        if (inter) {
            for (int r = 0; r < R; ++r) {
                const unsigned m = __ballot_sync(0xffffffffu, k > r);
                tab[r * chunk + threadIdx.x] = __popc(m & below);
                if (lane == 0) wt[r * nw + w] = __popc(m);
            }
        }
        __syncthreads();
        if (inter) {
            for (int r = 0; r < R; ++r) {
                int cross = 0;
                for (int q = 0; q < w; ++q) cross += wt[r * nw + q];
                tab[r * chunk + threadIdx.x] += cross;
            }
            if (threadIdx.x == 0) {
                int acc = 0;
                for (int r = 0; r < R; ++r) {
                    pre[r] = acc;
                    for (int q = 0; q < nw; ++q) acc += wt[r * nw + q];
                }
            }
        }
        __syncthreads();
        for (int i = a + threadIdx.x; i < b; i += blockDim.x) {
            const uint32_t cell = src.cell[i];
            const int lc = local_cell_index(tp, t, cell);
            if (lc < lo || lc >= hi) continue;
            const int r = rank[i];
            const long long pos =
                inter ? cs[lo] + pre[r] + tab[r * chunk + (lc - lo)] : cs[lc] + r;
            const long long d = a + pos;
            dst.cell[d] = cell;
            pid_dst[d] = pid_src[i];
            for (int q = 0; q < 3; ++q) mv(dst.v[q], src.v[q], d, (long long)i);
            if (src.kind == PIC_BOUND) {
                for (int q = 0; q < 3; ++q) {
                    mv(const_cast<double *>(dst.anchor[q]), src.anchor[q], d, (long long)i);
                    mv(const_cast<float *>(dst.anchor32[q]), src.anchor32[q], d, (long long)i);
                    mv(dst.disp[q], src.disp[q], d, (long long)i);
                }
            } else {
                for (int q = 0; q < 3; ++q) mv(dst.o[q], src.o[q], d, (long long)i);
            }
        }
        __syncthreads();  // the tables are rebuilt for the next chunk
    }
}

// The active-tile list goes to the particle kernel, whose persistent CTAs
// take tiles from it in order as they become free: listing the tiles by
// descending particle count (largest first) evens out the CTAs' loads.  The
// order is a counting sort over kWorkBuckets count buckets (counts above the
// last bucket share it).
constexpr int kWorkBuckets = 8192;

__device__ inline int tile_count(const int *const *starts, int nsp, int t) {
    int c = 0;
    for (int s = 0; s < nsp; ++s) c += starts[s][t + 1] - starts[s][t];
    return c;
}

__device__ inline int work_key(int count) {  // bucket of a count, largest first
    return kWorkBuckets - 1 - min(count, kWorkBuckets - 1);
}

__global__ void active_flags_kernel(TileP tp, const int *const *starts, int nsp, int *flags,
                                    int *hist) {
    const int n = max(tp.ntiles, kWorkBuckets + 1);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        if (t < tp.ntiles) flags[t] = tile_count(starts, nsp, t) > 0;
        if (t <= kWorkBuckets) hist[t] = 0;
    }
}

__global__ void active_scatter_kernel(int ntiles, const int *const *starts, int nsp,
                                      const int *flags, const int *pos, int *unsorted, int *rank,
                                      int *hist, int *nactive) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
        if (flags[t]) {
            const int i = pos[t];
            unsorted[i] = t;
            rank[i] = atomicAdd(&hist[work_key(tile_count(starts, nsp, t))], 1);
        }
        if (t == ntiles - 1) *nactive = pos[ntiles];
    }
}

__global__ void active_order_kernel(int ntiles, const int *const *starts, int nsp,
                                    const int *unsorted, const int *rank, const int *bstart,
                                    const int *nactive, int *active) {
    const int n = *nactive;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n && i < ntiles;
         i += gridDim.x * blockDim.x) {
        const int t = unsorted[i];
        active[bstart[work_key(tile_count(starts, nsp, t))] + rank[i]] = t;
    }
}

__global__ void cell_hist_kernel(GridP g, SpeciesP sp, int *counts) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < sp.n;
         p += (long long)gridDim.x * blockDim.x) {
        uint32_t c = sp.cell[p];
        int x[3] = {cell_x(c), cell_y(c), cell_z(c)};
        if (sp.kind == PIC_BOUND) {
            for (int a = 0; a < g.dims; ++a) {
                double X = sp.anchor[a][p] + (double)sp.disp[a][p] * (double)g.inv_d[a];
                x[a] += (int)floor(X);
                if (g.per[a]) x[a] = (x[a] % g.n[a] + g.n[a]) % g.n[a];
            }
        }
        bool in = true;
        for (int a = 0; a < 3; ++a) in = in && x[a] >= 0 && x[a] < g.n[a];
        if (in) atomicAdd(&counts[((long long)x[2] * g.n[1] + x[1]) * g.n[0] + x[0]], 1);
    }
}

int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

}  // namespace

cudaError_t launch_tile_histogram(const GridP &g, const TileP &tp, const uint32_t *cell,
                                  long long n, int *count, int *rank, cudaStream_t s) {
    (void)g;
    if (n <= 0) return cudaSuccess;
    tile_hist_kernel<<<grid_for(n, 256), 256, 0, s>>>(tp, cell, n, count, rank);
    return cudaGetLastError();
}

long long scan_tmp_len(long long n) {
    long long nb = (n + kScanChunk - 1) / kScanChunk;
    if (nb <= 1) return 1;
    return nb + (nb + 1) + scan_tmp_len(nb);
}

int scan_kernel_count(long long n) {
    if (n <= 0) return 0;
    long long nb = (n + kScanChunk - 1) / kScanChunk;
    return nb == 1 ? 1 : 2 + scan_kernel_count(nb);
}

// Exclusive scan of n ints: out[0..n] (out[n] = total).  tmp: scan_tmp_len(n).
cudaError_t launch_scan_int(const int *in, int *out_excl, long long n, int *tmp, long long tmp_len,
                            cudaStream_t s) {
    (void)tmp_len;
    if (n <= 0) {
        return cudaMemsetAsync(out_excl, 0, sizeof(int), s);
    }
    long long nb = (n + kScanChunk - 1) / kScanChunk;
    if (nb == 1) {
        scan_down_kernel<<<1, kScanThreads, 0, s>>>(in, n, nullptr, out_excl);
        return cudaGetLastError();
    }
    int *sums = tmp;
    int *sums_scan = tmp + nb;  // nb + 1 entries ... recursion uses the rest
    scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // scan of the block sums into sums_scan (needs its own tmp beyond it)
    e = launch_scan_int(sums, sums_scan, nb, sums_scan + nb + 1, 0, s);
    if (e != cudaSuccess) return e;
    scan_down_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums_scan, out_excl);
    return cudaGetLastError();
}

cudaError_t launch_tile_scatter(const GridP &g, const TileP &tp, const SpeciesP &src,
                                const uint32_t *pid_src, SpeciesP &dst, uint32_t *pid_dst,
                                const int *start, const int *rank, bool spread, cudaStream_t s) {
    (void)g;
    if (src.n <= 0) return cudaSuccess;
    tile_scatter_kernel<<<grid_for(src.n, 256), 256, 0, s>>>(tp, src, pid_src, dst, pid_dst, start,
                                                             rank, spread ? 1 : 0);
    return cudaGetLastError();
}

// Shared memory of the interleave kernel: cell counts, their scan, and one
// chunk's per-rank tables for cell counts up to rmax, within 48 KB.
static int interleave_rmax(int ncl, int chunk) {
    const long long budget = 48 * 1024 / 4;
    const long long nw = chunk / 32;
    const long long r = (budget - 2LL * ncl - 2) / (1 + nw + chunk);
    return (int)std::max<long long>(0, std::min<long long>(r, 255));
}

static size_t interleave_smem(int ncl, int chunk, int rmax) {
    const long long nw = chunk / 32;
    return (size_t)(2LL * ncl + 2 + (long long)rmax * (1 + nw + chunk)) * sizeof(int);
}

cudaError_t launch_tile_interleave(const TileP &tp, const SpeciesP &src, const uint32_t *pid_src,
                                   SpeciesP &dst, uint32_t *pid_dst, const int *start, int *rank,
                                   int chunk, cudaStream_t s) {
    if (src.n <= 0) return cudaSuccess;
    if (chunk % 32 != 0 || chunk > 1024) return cudaErrorInvalidValue;
    const int ncl = tp.T[0] * tp.T[1] * tp.T[2];
    const int rmax = interleave_rmax(ncl, chunk);
    const size_t smem = interleave_smem(ncl, chunk, rmax);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;  // tile too large to reorder
    cudaError_t e = allow_max_dynamic_smem(tile_interleave_kernel);
    if (e != cudaSuccess) return e;
    tile_interleave_kernel<<<tp.ntiles, chunk, smem, s>>>(tp, src, pid_src, dst, pid_dst, start,
                                                          rank, rmax, chunk);
    return cudaGetLastError();
}

long long active_tiles_work_len(long long ntiles) {
    return 4 * (ntiles + 1) + 2 * (kWorkBuckets + 1) +
           std::max(scan_tmp_len(ntiles), scan_tmp_len(kWorkBuckets));
}

int active_tiles_kernel_count(long long ntiles) {
    return 3 + scan_kernel_count(ntiles) + scan_kernel_count(kWorkBuckets);
}

// Scratch in `work` (active_tiles_work_len(ntiles) ints): tile flags, their
// exclusive scan, the unsorted list, ranks inside a count bucket, the bucket
// histogram and its scan, the scan's own scratch.
cudaError_t launch_active_tiles_work(const TileP &tp, const int *const *starts_dev, int nsp,
                                     int *active, int *nactive, int *work, cudaStream_t s) {
    const long long nt = tp.ntiles;
    int *flags = work;
    int *pos = flags + nt + 1;
    int *unsorted = pos + nt + 1;
    int *rank = unsorted + nt + 1;
    int *hist = rank + nt + 1;
    int *bstart = hist + kWorkBuckets + 1;
    int *tmp = bstart + kWorkBuckets + 1;
    const int nb = grid_for(std::max<long long>(nt, kWorkBuckets + 1), 256);
    active_flags_kernel<<<nb, 256, 0, s>>>(tp, starts_dev, nsp, flags, hist);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_scan_int(flags, pos, nt, tmp, 0, s);
    if (e != cudaSuccess) return e;
    active_scatter_kernel<<<grid_for(nt, 256), 256, 0, s>>>(tp.ntiles, starts_dev, nsp, flags, pos,
                                                           unsorted, rank, hist, nactive);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_scan_int(hist, bstart, kWorkBuckets, tmp, 0, s);
    if (e != cudaSuccess) return e;
    active_order_kernel<<<grid_for(nt, 256), 256, 0, s>>>(tp.ntiles, starts_dev, nsp, unsorted, rank,
                                                         bstart, nactive, active);
    return cudaGetLastError();
}

cudaError_t launch_cell_histogram(const GridP &g, const SpeciesP &sp, int *counts, cudaStream_t s) {
    if (sp.n <= 0) return cudaSuccess;
    cell_hist_kernel<<<grid_for(sp.n, 256), 256, 0, s>>>(g, sp, counts);
    return cudaGetLastError();
}

}  // namespace pic
