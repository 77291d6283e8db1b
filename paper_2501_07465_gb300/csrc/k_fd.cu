// k_fd.cu -- the Fermi-Dirac loader (Sec. 2 of the paper, Eq. fddist):
// macro-particles placed in every material cell with momenta drawn from
// f_FD = 1 / (1 + exp((E - mu) / kT)), mu = E_F.
//
// Random numbers: Philox-4x32-10 (Salmon et al., SC'11), key = seed, counter
// (id_lo, id_hi, call, stream), three calls per particle -> six uniforms
// u = (hi27 * 2^26 + lo26 + 1/2) / 2^53 from word pairs.  Particle id =
// material-cell rank * ppc + j.
//
// |p| is drawn by inverting the radial CDF F(p) = int_0^p g / int_0^pmax g,
// g = p^2 f(p^2/2m) (3D electrons) or p f(v_F p) (2D Dirac sheet), all in
// FP64: a 4096-panel table of the cumulative integral (8-point
// Gauss-Legendre per panel, block scan), binary search for the panel, then
// Newton steps on the partial-panel integral.  pmax: carrier energy
// mu + 40 kT.  At T = 0 the closed forms p_F u^(1/3) (3D) and p_F u^(1/2)
// (2D) are used.
#include <math.h>

#include "pic_internal.cuh"

namespace pic {

namespace {

__device__ inline double u53(uint32_t a, uint32_t b) {
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6) + 0.5) * (1.0 / 9007199254740992.0);
}

__device__ inline void uniforms(uint64_t seed, uint32_t stream, uint64_t id, double *u) {
    for (uint32_t call = 0; call < 3; ++call) {
        uint32_t x[4] = {(uint32_t)id, (uint32_t)(id >> 32), call, stream};
        philox4x32_10(x, (uint32_t)seed, (uint32_t)(seed >> 32));
        u[2 * call] = u53(x[0], x[1]);
        u[2 * call + 1] = u53(x[2], x[3]);
    }
}

// radial density of |p|
__device__ inline double fd_g(const FDRequest &r, double p) {
    const bool dirac = r.kind == PIC_DIRAC;
    double E = dirac ? r.vF * p : p * p / (2.0 * r.m);
    double f = 1.0 / (1.0 + exp((E - r.mu) / r.kT));
    return (dirac ? p : p * p) * f;
}

// 8-point Gauss-Legendre on [a, b]
__device__ inline double gl8(const FDRequest &r, double a, double b) {
    const double x[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267,
                         0.9602898564975363};
    const double w[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745,
                         0.1012285362903763};
    double c = 0.5 * (a + b), h = 0.5 * (b - a), s = 0.0;
    for (int i = 0; i < 4; ++i) s += w[i] * (fd_g(r, c - h * x[i]) + fd_g(r, c + h * x[i]));
    return s * h;
}

// table[0] = 0, table[k+1] = int_0^{(k+1) h} g (one block of 1024 threads)
__global__ void fd_table_kernel(FDRequest r, double *table, double pmax) {
    constexpr int per = kFDPanels / 1024;
    __shared__ double warp_sums[32];
    const double h = pmax / kFDPanels;
    double v[per];
    double s = 0.0;
    for (int q = 0; q < per; ++q) {
        int k = threadIdx.x * per + q;
        v[q] = gl8(r, k * h, (k + 1) * h);
        s += v[q];
    }
    // inclusive block scan of s
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double x = s;
    for (int o = 1; o < 32; o <<= 1) {
        double y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        double t = warp_sums[lane];
        for (int o = 1; o < 32; o <<= 1) {
            double y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_sums[lane] = t;
    }
    __syncthreads();
    double pre = (wid > 0 ? warp_sums[wid - 1] : 0.0) + x - s;
    if (threadIdx.x == 0) table[0] = 0.0;
    for (int q = 0; q < per; ++q) {
        pre += v[q];
        table[threadIdx.x * per + q + 1] = pre;
    }
}

__device__ inline double fd_invert(const FDRequest &r, const double *table, double pmax,
                                   double u) {
    if (r.kT <= 0.0) {
        double pF = r.kind == PIC_DIRAC ? r.mu / r.vF : sqrt(2.0 * r.m * r.mu);
        return r.kind == PIC_DIRAC ? pF * sqrt(u) : pF * cbrt(u);
    }
    const double h = pmax / kFDPanels;
    const double target = u * table[kFDPanels];
    int lo = 0, hi = kFDPanels;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (table[mid] <= target) lo = mid;
        else hi = mid;
    }
    const double a = lo * h, b = a + h;
    const double Fa = table[lo], dF = table[lo + 1] - table[lo];
    double p = dF > 0.0 ? a + h * (target - Fa) / dF : a;
    for (int it = 0; it < 8; ++it) {
        double G = Fa + gl8(r, a, p) - target;
        double gp = fd_g(r, p);
        if (!(gp > 0.0)) break;
        double dp = G / gp;
        double pn = fmin(fmax(p - dp, a), b);
        if (fabs(pn - p) <= 1e-15 * h) {
            p = pn;
            break;
        }
        p = pn;
    }
    return p;
}

__device__ inline float below_one(double u) {
    float f = (float)u;
    return f < 1.0f ? f : 0x1.fffffep-1f;
}

__global__ void fd_particles_kernel(GridP g, FDRequest r, const int *mat_cells, long long np,
                                    const double *table, double pmax, SpeciesP out,
                                    uint32_t *pid) {
    int lat = 1;
    if (r.quiet) {
        lat = (int)llround(pow((double)r.ppc, 1.0 / r.dims));
    }
    for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < np;
         id += (long long)gridDim.x * blockDim.x) {
        long long rank = id / r.ppc;
        int j = (int)(id - rank * r.ppc);
        long long c = mat_cells ? mat_cells[rank] : rank;
        int x = (int)(c % g.n[0]);
        int y = (int)((c / g.n[0]) % g.n[1]);
        int z = (int)(c / ((long long)g.n[0] * g.n[1]));
        double u[6];
        uniforms(r.seed, r.stream, (uint64_t)id, u);
        double off[3];
        if (r.quiet) {
            int a0 = j % lat, a1 = (j / lat) % lat, a2 = j / (lat * lat);
            off[0] = (a0 + 0.5) / lat;
            off[1] = (a1 + 0.5) / lat;
            off[2] = r.dims == 3 ? (a2 + 0.5) / lat : 0.5;
        } else {
            off[0] = u[0];
            off[1] = u[1];
            off[2] = u[2];
        }
        out.cell[id] = pack_cell(x, y, z);
        pid[id] = (uint32_t)id;
        if (r.kind == PIC_BOUND) {
            for (int a = 0; a < 3; ++a) {
                const_cast<double *>(out.anchor[a])[id] = off[a];
                const_cast<float *>(out.anchor32[a])[id] = below_one(off[a]);
                out.disp[a][id] = 0.f;
                out.v[a][id] = 0.f;
            }
            continue;
        }
        for (int a = 0; a < 3; ++a) out.o[a][id] = below_one(off[a]);
        if (r.kind == PIC_DIRAC) {
            double phi = 2.0 * kPi * u[5];
            out.v[0][id] = (float)(r.vF * cos(phi));
            out.v[1][id] = (float)(r.vF * sin(phi));
            out.v[2][id] = 0.f;
        } else {
            double p = fd_invert(r, table, pmax, u[3]);
            double ct = 2.0 * u[4] - 1.0;
            double st = sqrt(fmax(0.0, 1.0 - ct * ct));
            double phi = 2.0 * kPi * u[5];
            double sp = p / r.m;
            out.v[0][id] = (float)(sp * st * cos(phi));
            out.v[1][id] = (float)(sp * st * sin(phi));
            out.v[2][id] = (float)(sp * ct);
        }
    }
}

__global__ void mask_to_int_kernel(const uint8_t *mask, long long n, int *out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = mask[i] != 0;
}

__global__ void material_cells_kernel(long long n, const uint8_t *mask, const int *rank,
                                      int *mat_cells) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        if (mask[i]) mat_cells[rank[i]] = (int)i;
}

int blocks_for(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

}  // namespace

double fd_pmax(const FDRequest &r) {
    double Emax = r.mu + 40.0 * r.kT;
    return r.kind == PIC_DIRAC ? Emax / r.vF : sqrt(2.0 * r.m * Emax);
}

cudaError_t launch_fd_table(const FDRequest &r, double *table, double pmax, cudaStream_t s) {
    fd_table_kernel<<<1, 1024, 0, s>>>(r, table, pmax);
    return cudaGetLastError();
}

cudaError_t launch_fd_particles(const GridP &g, const FDRequest &r, const int *mat_cells,
                                long long np, const double *table, double pmax, SpeciesP out,
                                uint32_t *pid, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    fd_particles_kernel<<<blocks_for(np), 256, 0, s>>>(g, r, mat_cells, np, table, pmax, out, pid);
    return cudaGetLastError();
}

cudaError_t launch_mask_to_int(const uint8_t *mask, long long n, int *out, cudaStream_t s) {
    mask_to_int_kernel<<<blocks_for(n), 256, 0, s>>>(mask, n, out);
    return cudaGetLastError();
}

cudaError_t launch_material_cells(const GridP &g, const uint8_t *mask, const int *rank,
                                  int *mat_cells, cudaStream_t s) {
    material_cells_kernel<<<blocks_for(g.ncell), 256, 0, s>>>(g.ncell, mask, rank, mat_cells);
    return cudaGetLastError();
}

}  // namespace pic
