// k_diag.cu -- FP64 diagnostic reductions (kinetic and field energy, the
// Gauss-law residual div E - rho/eps0 on the Yee nodes, the kinetic-energy
// histogram of the relaxation study of Sec. 2) and the copy helpers
// used by the ABI (un-sorting particles back to load order, layout and
// precision conversions).
#include <math.h>

#include "pic_internal.cuh"

namespace pic {

namespace {

int blocks_for(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 152 * 8 ? 152 * 8 : b));
}

__device__ inline double block_sum(double v) {
    __shared__ double ws[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) ws[w] = v;
    __syncthreads();
    double s = 0.0;
    if (w == 0) {
        s = lane < (blockDim.x >> 5) ? ws[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    return s;  // valid in thread 0
}

__device__ inline double block_max(double v) {
    __shared__ double wm[32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wm[w] = v;
    __syncthreads();
    double s = 0.0;
    if (w == 0) {
        s = lane < (blockDim.x >> 5) ? wm[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, o));
    }
    __syncthreads();
    return s;
}

__global__ void kinetic_kernel(SpeciesP sp, double mw_half, double *acc) {
    double s = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < sp.n;
         p += (long long)gridDim.x * blockDim.x) {
        double a = sp.v[0][p], b = sp.v[1][p], c = sp.v[2][p];
        s += a * a + b * b + c * c;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) atomicAdd(acc, s * mw_half);
}

// Kinetic-energy histogram (the relaxation study of Sec. 2): E in FP64 from
// the FP32 velocities as half_m ((vx vx + vy vy) + vz vz), bin floor(E / D),
// every operation rounded once (no contraction), so the counts are exact
// for given velocities.  Block-private counters in shared memory when
// `priv` (nbins + 1 of them fit), global atomics otherwise.
__global__ void energy_hist_kernel(SpeciesP sp, double half_m, double e_max, double D, int nbins,
                                   int priv, unsigned long long *out) {
    extern __shared__ unsigned int hist[];
    if (priv) {
        for (int b = threadIdx.x; b <= nbins; b += blockDim.x) hist[b] = 0;
        __syncthreads();
    }
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < sp.n;
         p += (long long)gridDim.x * blockDim.x) {
        const double a = sp.v[0][p], b = sp.v[1][p], c = sp.v[2][p];
        const double v2 = __dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c));
        const double E = __dmul_rn(half_m, v2);
        int bin;
        if (E >= e_max) bin = nbins;
        else {
            const double f = floor(__ddiv_rn(E, D));
            bin = f > (double)(nbins - 1) ? nbins - 1 : (int)f;
        }
        if (priv) atomicAdd(&hist[bin], 1u);
        else atomicAdd(&out[bin], 1ull);
    }
    if (priv) {
        __syncthreads();
        for (int b = threadIdx.x; b <= nbins; b += blockDim.x)
            if (hist[b]) atomicAdd(&out[b], (unsigned long long)hist[b]);
    }
}

__global__ void field_energy_kernel(long long n, const float *E0, const float *E1, const float *E2,
                                    const float *B0, const float *B1, const float *B2,
                                    DiagAcc *acc) {
    double e = 0.0, b = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double x = E0[i], y = E1[i], z = E2[i];
        e += x * x + y * y + z * z;
        x = B0[i]; y = B1[i]; z = B2[i];
        b += x * x + y * y + z * z;
    }
    e = block_sum(e);
    b = block_sum(b);
    if (threadIdx.x == 0) {
        atomicAdd(&acc->e2, e);
        atomicAdd(&acc->b2, b);
    }
}

__device__ inline int wrap_or_neg(int i, int n, int per) {
    if (i >= 0 && i < n) return i;
    if (!per) return -1;
    int r = i % n;
    return r < 0 ? r + n : r;
}

// TSC weight of a node at distance r (order 2, the quadratic B-spline).
__device__ inline double tsc_w(double r) {
    r = fabs(r);
    if (r < 0.5) return 0.75 - r * r;
    if (r < 1.5) return 0.5 * (1.5 - r) * (1.5 - r);
    return 0.0;
}

// Charge density on the integer nodes with the species' shape (CIC, or TSC
// for order 2: the three nodes around the nearest), FP64 atomics.
__global__ void rho_kernel(GridP g, SpeciesP sp, double qv, int order, double *rho) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < sp.n;
         p += (long long)gridDim.x * blockDim.x) {
        uint32_t c = sp.cell[p];
        int ci[3] = {cell_x(c), cell_y(c), cell_z(c)};
        double X[3];
        for (int a = 0; a < 3; ++a) {
            if (sp.kind == PIC_BOUND)
                X[a] = ci[a] + sp.anchor[a][p] + (double)sp.disp[a][p] * (double)g.inv_d[a];
            else
                X[a] = ci[a] + (double)sp.o[a][p];
        }
        if (order == 2) {
            int n0[3];
            for (int a = 0; a < 3; ++a) n0[a] = (int)floor(X[a] + 0.5) - 1;
            const int kn = g.dims == 3 ? 3 : 1;
            for (int k = 0; k < kn; ++k)
                for (int j = 0; j < 3; ++j)
                    for (int i = 0; i < 3; ++i) {
                        double w = tsc_w(X[0] - (n0[0] + i)) * tsc_w(X[1] - (n0[1] + j));
                        if (g.dims == 3) w *= tsc_w(X[2] - (n0[2] + k));
                        int gx = wrap_or_neg(n0[0] + i, g.n[0], g.per[0]);
                        int gy = wrap_or_neg(n0[1] + j, g.n[1], g.per[1]);
                        int gz = g.dims == 3 ? wrap_or_neg(n0[2] + k, g.n[2], g.per[2]) : 0;
                        if (gx < 0 || gy < 0 || gz < 0) continue;
                        atomicAdd(&rho[((long long)gz * g.n[1] + gy) * g.n[0] + gx], qv * w);
                    }
            continue;
        }
        int i0 = (int)floor(X[0]), j0 = (int)floor(X[1]), k0 = (int)floor(X[2]);
        double fx = X[0] - i0, fy = X[1] - j0, fz = X[2] - k0;
        int kn = g.dims == 3 ? 2 : 1;
        for (int k = 0; k < kn; ++k)
            for (int j = 0; j < 2; ++j)
                for (int i = 0; i < 2; ++i) {
                    double w = (i ? fx : 1.0 - fx) * (j ? fy : 1.0 - fy);
                    if (g.dims == 3) w *= (k ? fz : 1.0 - fz);
                    int gx = wrap_or_neg(i0 + i, g.n[0], g.per[0]);
                    int gy = wrap_or_neg(j0 + j, g.n[1], g.per[1]);
                    int gz = g.dims == 3 ? wrap_or_neg(k0 + k, g.n[2], g.per[2]) : 0;
                    if (gx < 0 || gy < 0 || gz < 0) continue;
                    atomicAdd(&rho[((long long)gz * g.n[1] + gy) * g.n[0] + gx], qv * w);
                }
    }
}

__device__ inline float eget(const GridP &g, const float *F, int i, int j, int k) {
    int gi = wrap_or_neg(i, g.n[0], g.per[0]);
    int gj = wrap_or_neg(j, g.n[1], g.per[1]);
    int gk = g.dims == 3 ? wrap_or_neg(k, g.n[2], g.per[2]) : 0;
    if (gi < 0 || gj < 0 || gk < 0) return 0.f;
    return F[((long long)gk * g.n[1] + gj) * g.n[0] + gi];
}

// eps_r E at the E node of cell (i, j, k) (D / eps0; E beyond a wall is 0)
__device__ inline double dget(const GridP &g, const float *F, const float *inv_eps, int i, int j,
                              int k) {
    int gi = wrap_or_neg(i, g.n[0], g.per[0]);
    int gj = wrap_or_neg(j, g.n[1], g.per[1]);
    int gk = g.dims == 3 ? wrap_or_neg(k, g.n[2], g.per[2]) : 0;
    if (gi < 0 || gj < 0 || gk < 0) return 0.0;
    const long long c = ((long long)gk * g.n[1] + gj) * g.n[0] + gi;
    return inv_eps ? (double)F[c] / (double)inv_eps[c] : (double)F[c];
}

// Gauss's law for D = eps0 eps_r E: div(eps_r E) - rho / eps0
__global__ void gauss_kernel(GridP g, const float *Ex, const float *Ey, const float *Ez,
                             const float *inv_eps, const double *rho, const double *rho_bg,
                             DiagAcc *acc) {
    double rmax = 0.0, rsum = 0.0, qmax = 0.0;
    const double inv_eps0 = 1.0 / kEps0;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < g.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        int i = (int)(c % g.n[0]), j = (int)((c / g.n[0]) % g.n[1]);
        int k = (int)(c / ((long long)g.n[0] * g.n[1]));
        double div = (dget(g, Ex, inv_eps, i, j, k) - dget(g, Ex, inv_eps, i - 1, j, k)) / g.d[0] +
                     (dget(g, Ey, inv_eps, i, j, k) - dget(g, Ey, inv_eps, i, j - 1, k)) / g.d[1];
        if (g.dims == 3)
            div += (dget(g, Ez, inv_eps, i, j, k) - dget(g, Ez, inv_eps, i, j, k - 1)) / g.d[2];
        double q = (rho[c] + (rho_bg ? rho_bg[c] : 0.0)) * inv_eps0;
        double r = div - q;
        rmax = fmax(rmax, fabs(r));
        rsum += r * r;
        qmax = fmax(qmax, fabs(q));
    }
    rsum = block_sum(rsum);
    rmax = block_max(rmax);
    qmax = block_max(qmax);
    if (threadIdx.x == 0) {
        atomicAdd(&acc->gauss_sum2, rsum);
        atomicMax(&acc->gauss_max_bits, (unsigned long long)__double_as_longlong(rmax));
        atomicMax(&acc->rho_max_bits, (unsigned long long)__double_as_longlong(qmax));
    }
}

__global__ void add_uniform_kernel(double *rho, long long n, double v) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        rho[i] += v;
}

__global__ void unsort_kernel(GridP g, SpeciesP sp, const uint32_t *pid, int32_t *cell_out,
                              float *off_out, float *v_out, double *anchor_out, float *disp_out) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < sp.n;
         p += (long long)gridDim.x * blockDim.x) {
        long long q = pid[p];
        uint32_t c = sp.cell[p];
        cell_out[q] = (int32_t)(((long long)cell_z(c) * g.n[1] + cell_y(c)) * g.n[0] + cell_x(c));
        for (int a = 0; a < 3; ++a) {
            v_out[3 * q + a] = sp.v[a][p];
            if (sp.kind == PIC_BOUND) {
                anchor_out[3 * q + a] = sp.anchor[a][p];
                disp_out[3 * q + a] = sp.disp[a][p];
            } else {
                off_out[3 * q + a] = sp.o[a][p];
            }
        }
    }
}

__global__ void pack_explicit_kernel(GridP g, long long n, const int32_t *lin, uint32_t *packed,
                                     uint32_t *pid) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        long long c = lin[p];
        int x = (int)(c % g.n[0]), y = (int)((c / g.n[0]) % g.n[1]);
        int z = (int)(c / ((long long)g.n[0] * g.n[1]));
        packed[p] = pack_cell(x, y, z);
        pid[p] = (uint32_t)p;
    }
}

__global__ void f32_to_f64_kernel(const float *in, double *out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = in[i];
}

__global__ void f64_to_f32_kernel(const double *in, float *out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

}  // namespace

cudaError_t launch_kinetic(const SpeciesP &sp, double mw_half, double *acc, cudaStream_t s) {
    if (sp.n <= 0) return cudaSuccess;
    kinetic_kernel<<<blocks_for(sp.n), 256, 0, s>>>(sp, mw_half, acc);
    return cudaGetLastError();
}

cudaError_t launch_energy_histogram(const SpeciesP &sp, double half_m, double e_max, int nbins,
                                    unsigned long long *out, cudaStream_t s) {
    if (sp.n <= 0) return cudaSuccess;
    const size_t smem = (size_t)(nbins + 1) * sizeof(unsigned int);
    const int priv = smem <= 32 * 1024;
    const double D = e_max / nbins;
    energy_hist_kernel<<<blocks_for(sp.n), 256, priv ? smem : 0, s>>>(sp, half_m, e_max, D, nbins,
                                                                      priv, out);
    return cudaGetLastError();
}

cudaError_t launch_field_energy(const GridP &g, const float *const *E, const float *const *B,
                                DiagAcc *acc, cudaStream_t s) {
    field_energy_kernel<<<blocks_for(g.ncell), 256, 0, s>>>(g.ncell, E[0], E[1], E[2], B[0], B[1],
                                                            B[2], acc);
    return cudaGetLastError();
}

cudaError_t launch_rho_deposit(const GridP &g, const SpeciesP &sp, double qw_over_V, int order,
                               double *rho, cudaStream_t s) {
    if (sp.n <= 0) return cudaSuccess;
    rho_kernel<<<blocks_for(sp.n), 256, 0, s>>>(g, sp, qw_over_V, order, rho);
    return cudaGetLastError();
}

cudaError_t launch_gauss(const GridP &g, const float *const *E, const float *inv_eps,
                         const double *rho, const double *rho_bg, DiagAcc *acc, cudaStream_t s) {
    gauss_kernel<<<blocks_for(g.ncell), 256, 0, s>>>(g, E[0], E[1], E[2], inv_eps, rho, rho_bg,
                                                     acc);
    return cudaGetLastError();
}

cudaError_t launch_add_uniform(double *rho, long long n, double v, cudaStream_t s) {
    add_uniform_kernel<<<blocks_for(n), 256, 0, s>>>(rho, n, v);
    return cudaGetLastError();
}

cudaError_t launch_unsort(const GridP &g, const SpeciesP &sp, const uint32_t *pid,
                          int32_t *cell_out, float *off_out, float *v_out, double *anchor_out,
                          float *disp_out, cudaStream_t s) {
    if (sp.n <= 0) return cudaSuccess;
    unsort_kernel<<<blocks_for(sp.n), 256, 0, s>>>(g, sp, pid, cell_out, off_out, v_out,
                                                   anchor_out, disp_out);
    return cudaGetLastError();
}

cudaError_t launch_pack_explicit(const GridP &g, long long n, const int32_t *cell_lin,
                                 uint32_t *cell_packed, uint32_t *pid, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    pack_explicit_kernel<<<blocks_for(n), 256, 0, s>>>(g, n, cell_lin, cell_packed, pid);
    return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(const float *in, double *out, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    f32_to_f64_kernel<<<blocks_for(n), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_f64_to_f32(const double *in, float *out, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    f64_to_f32_kernel<<<blocks_for(n), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

}  // namespace pic
