// k_boundary.cu -- setup of the particle boundary variants of Sec. 3: the
// work-function barrier as an external electrostatic field.
//
// Node potential phi = -(W / e) f, f the vacuum fraction of the cells that
// share the node (cells i-1..i, j-1..j, k-1..k; in 2D the four cells of the
// plane; cells beyond a non-periodic face do not count), and
// E_a(cell) = -(phi(node + e_a) - phi(node)) / d_a on the Yee stagger
// (node = the cell's own corner), E_z = 0 in 2D.  FP64 arithmetic, one
// rounding to FP32 per value.  Runs once per call, not in the step.
#include "pic_internal.cuh"

namespace pic {

namespace {

__device__ inline int wrap_or_out(int i, int n, int per) {
    if (i >= 0 && i < n) return i;
    if (!per) return -1;
    int r = i % n;
    return r < 0 ? r + n : r;
}

__device__ double node_vacuum(const GridP &g, const uint8_t *mask, int i, int j, int k) {
    if (!mask) return 0.0;
    int nin = 0, nvac = 0;
    const int kn = g.dims == 3 ? 2 : 1;
    for (int dk = 0; dk < kn; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                const int x = wrap_or_out(i - 1 + di, g.n[0], g.per[0]);
                const int y = wrap_or_out(j - 1 + dj, g.n[1], g.per[1]);
                const int z = g.dims == 3 ? wrap_or_out(k - 1 + dk, g.n[2], g.per[2]) : 0;
                if (x < 0 || y < 0 || z < 0) continue;
                ++nin;
                if (!mask[((long long)z * g.n[1] + y) * g.n[0] + x]) ++nvac;
            }
    return nin ? (double)nvac / nin : 0.0;
}

__global__ void work_function_kernel(GridP g, const uint8_t *mask, double W, float *ex, float *ey,
                                     float *ez) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.ncell) return;
    const int i = (int)(c % g.n[0]);
    const int j = (int)((c / g.n[0]) % g.n[1]);
    const int k = (int)(c / ((long long)g.n[0] * g.n[1]));
    const double f0 = node_vacuum(g, mask, i, j, k);
    // E_a = -(phi1 - phi0) / d_a with phi = -W f
    ex[c] = (float)(W * (node_vacuum(g, mask, i + 1, j, k) - f0) / (double)g.d[0]);
    ey[c] = (float)(W * (node_vacuum(g, mask, i, j + 1, k) - f0) / (double)g.d[1]);
    ez[c] = g.dims == 3
                ? (float)(W * (node_vacuum(g, mask, i, j, k + 1) - f0) / (double)g.d[2])
                : 0.f;
}

}  // namespace

cudaError_t launch_work_function(const GridP &g, const uint8_t *mask, double W_eV,
                                 float *const E[3], cudaStream_t s) {
    const int bs = 256;
    const long long nb = (g.ncell + bs - 1) / bs;
    work_function_kernel<<<(unsigned)nb, bs, 0, s>>>(g, mask, W_eV, E[0], E[1], E[2]);
    return cudaGetLastError();
}

}  // namespace pic
