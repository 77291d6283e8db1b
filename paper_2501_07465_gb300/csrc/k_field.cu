// k_field.cu -- Yee FDTD update with CPML layers and a soft plane-wave
// current sheet, fused into one pass over the grid.
//
//   B^{n+1/2} = B^{n-1/2} - dt (curl E^n + psi_B)
//   E^{n+1}   = E^n + dt (c^2 (curl B^{n+1/2} + psi_E) - J^{n+1/2} / eps0)
//
// (Maxwell's curl equations on the Yee stagger, Sec. 4.1 of the paper; Eq.
// consteps with eps = eps0.)  CPML memory terms follow Roden & Gedney
// (kappa = 1, alpha = 0): psi <- b psi + a dF/dx inside the slabs.
//
// Layout: every component is an [nz][ny][nx] FP32 array.  E, B and psi are
// ping-ponged (read n, write n+1) so that a CTA may recompute the B values of
// its neighbours' edge cells without a grid-wide barrier.
//
// Each CTA owns a 32 x 8 column of cells and marches up a chunk of z planes
// (2.5D blocking): the E^n planes k and k+1 live in shared memory with a
// one-cell x/y halo, B^{n+1/2} of plane k is computed for the tile plus the
// low-x column and low-y row it needs, and the own-cell B_x, B_y of plane
// k-1 stay in registers.  Each own value is read from and written to HBM
// once; halo reads are L2 hits.
#include "pic_internal.cuh"

namespace pic {

namespace {

constexpr int BX = kFieldBX, BY = kFieldBY;
constexpr int SX = BX + 2, SY = BY + 2;  // E plane with halo [-1, BX] x [-1, BY]

struct Slab {
    // slab index of a cell along a PML axis, or -1 outside the slabs
    __device__ static inline int idx(int i, int n, int P) {
        if (i < P) return i;
        if (i >= n - P) return i - (n - 2 * P);
        return -1;
    }
};

__device__ inline int wrap_or_neg(int i, int n, int per) {
    if (i >= 0 && i < n) return i;
    if (!per) return -1;
    return i < 0 ? i + n : i - n;
}

template <int DIM>
__device__ inline void load_plane(float (*dst)[SY][SX], const GridP &g, const float *const *E,
                                  int i0, int j0, int k) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    int kk = k;
    if (DIM == 3) kk = wrap_or_neg(k, nz, g.per[2]);
    for (int e = threadIdx.x; e < SX * SY; e += blockDim.x) {
        int ly = e / SX - 1, lx = e % SX - 1;
        int gi = wrap_or_neg(i0 + lx, nx, g.per[0]);
        int gj = wrap_or_neg(j0 + ly, ny, g.per[1]);
        float a = 0.f, b = 0.f, c = 0.f;
        if (gi >= 0 && gj >= 0 && kk >= 0) {
            long long o = ((long long)kk * ny + gj) * nx + gi;
            a = __ldg(E[0] + o);
            b = __ldg(E[1] + o);
            c = __ldg(E[2] + o);
        }
        dst[0][ly + 1][lx + 1] = a;
        dst[1][ly + 1][lx + 1] = b;
        dst[2][ly + 1][lx + 1] = c;
    }
}

// psi index of (i,j,k) in the slab array of axis a, or -1
__device__ inline long long psi_index(const GridP &g, const FieldP &f, int a, int i, int j, int k) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], P = f.P;
    if (!f.pml[a]) return -1;
    if (a == 0) {
        int s = Slab::idx(i, nx, P);
        return s < 0 ? -1 : ((long long)k * ny + j) * (2 * P) + s;
    } else if (a == 1) {
        int s = Slab::idx(j, ny, P);
        return s < 0 ? -1 : ((long long)k * (2 * P) + s) * nx + i;
    } else {
        int s = Slab::idx(k, nz, P);
        return s < 0 ? -1 : ((long long)s * ny + j) * nx + i;
    }
}

// derivative plus CPML memory term; psi slot `slot` of axis `a`; position
// index `pos` into the axis coefficient arrays; half = B-type (h) profile.
__device__ inline float cpml_term(const FieldP &f, int a, int slot, long long pidx, int pos,
                                  bool half, float deriv, bool write) {
    if (pidx < 0) return deriv;
    float b = half ? __ldg(f.cb_h[a] + pos) : __ldg(f.cb_e[a] + pos);
    float c = half ? __ldg(f.ca_h[a] + pos) : __ldg(f.ca_e[a] + pos);
    float psi = b * __ldg(f.psi_in[a][slot] + pidx) + c * deriv;
    if (write) f.psi_out[a][slot][pidx] = psi;
    return deriv + psi;
}

// B^{n+1/2} components at local (lx, ly) of plane k (global gi, gj, k valid),
// from E^n planes k (cur) and k+1 (nxt).  mask selects components.
template <int DIM>
__device__ inline void compute_B(const GridP &g, const FieldP &f, float (*cur)[SY][SX],
                                 float (*nxt)[SY][SX], int lx, int ly, int gi, int gj, int k,
                                 int comps, bool write_psi, float *out) {
    const long long o = ((long long)k * g.n[1] + gj) * g.n[0] + gi;
    const float dt = g.dt;
    const long long px = psi_index(g, f, 0, gi, gj, k);
    const long long py = psi_index(g, f, 1, gi, gj, k);
    const long long pz = DIM == 3 ? psi_index(g, f, 2, gi, gj, k) : -1;
    const int X = lx + 1, Y = ly + 1;
    if (comps & 1) {  // B_x at (i, j+1/2, k+1/2)
        float dEz_dy = (cur[2][Y + 1][X] - cur[2][Y][X]) * g.inv_d[1];
        float t1 = cpml_term(f, 1, 2, py, gj, true, dEz_dy, write_psi);
        float t2 = 0.f;
        if (DIM == 3) {
            float dEy_dz = (nxt[1][Y][X] - cur[1][Y][X]) * g.inv_d[2];
            t2 = cpml_term(f, 2, 2, pz, k, true, dEy_dz, write_psi);
        }
        out[0] = __ldg(f.B[0] + o) - dt * (t1 - t2);
    }
    if (comps & 2) {  // B_y at (i+1/2, j, k+1/2)
        float t1 = 0.f;
        if (DIM == 3) {
            float dEx_dz = (nxt[0][Y][X] - cur[0][Y][X]) * g.inv_d[2];
            t1 = cpml_term(f, 2, 3, pz, k, true, dEx_dz, write_psi);
        }
        float dEz_dx = (cur[2][Y][X + 1] - cur[2][Y][X]) * g.inv_d[0];
        float t2 = cpml_term(f, 0, 2, px, gi, true, dEz_dx, write_psi);
        out[1] = __ldg(f.B[1] + o) - dt * (t1 - t2);
    }
    if (comps & 4) {  // B_z at (i+1/2, j+1/2, k)
        float dEy_dx = (cur[1][Y][X + 1] - cur[1][Y][X]) * g.inv_d[0];
        float dEx_dy = (cur[0][Y + 1][X] - cur[0][Y][X]) * g.inv_d[1];
        float t1 = cpml_term(f, 0, 3, px, gi, true, dEy_dx, write_psi);
        float t2 = cpml_term(f, 1, 3, py, gj, true, dEx_dy, write_psi);
        out[2] = __ldg(f.B[2] + o) - dt * (t1 - t2);
    }
}

// One 32 x 8 column block (block coordinates bx, by, chunk bz) of one
// simulation.  g and f must live in parameter or shared memory.
template <int DIM>
__device__ void field_block(const GridP &g, const FieldP &f, const int blk_x, const int blk_y,
                            const int blk_z) {
    __shared__ float sE[2][3][SY][SX];
    __shared__ float sB[3][BY + 1][BX + 1];  // local [-1, BY) x [-1, BX)
    __shared__ double s_src;

    const int tx = threadIdx.x % BX, ty = threadIdx.x / BX;
    const int i0 = blk_x * BX, j0 = blk_y * BY;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int i = i0 + tx, j = j0 + ty;
    const bool own = (i < nx) && (j < ny);
    const int kbeg = DIM == 3 ? blk_z * f.zchunk : 0;
    const int kend = DIM == 3 ? min(kbeg + f.zchunk, nz) : 1;

    const long long bflag = ((long long)blk_z * f.nby + blk_y) * f.nbx + blk_x;
    const bool jdirty = !f.splitJ && f.jdirty[bflag] != 0;
    __syncthreads();  // every thread has read the flag (cleared at the end)

    if (threadIdx.x == 0) {
        double v = 0.0;
        if (f.src_on) {
            // the particle phase of step n has run (fused step) or runs now (split)
            long long n = *f.step_counter - (f.splitJ ? 0 : 1);
            double t = ((double)n + 0.5) * f.dt64 - f.src_t0;
            v = f.src_amp * exp(-2.0 * 0.6931471805599453 * t * t / (f.src_tau * f.src_tau)) *
                sin(f.src_omega * t);
        }
        s_src = v;
    }

    // halo work items: column lx = -1 (ly in [0,BY)) needs B_z, B_y; row
    // ly = -1 (lx in [0,BX)) needs B_z, B_x.
    const int hid = threadIdx.x;
    const bool halo_col = hid < BY;
    const bool halo_row = hid >= BY && hid < BY + BX;
    int hlx = halo_col ? -1 : hid - BY, hly = halo_col ? hid : -1;
    int hgi = wrap_or_neg(i0 + hlx, nx, g.per[0]);
    int hgj = wrap_or_neg(j0 + hly, ny, g.per[1]);
    const bool halo_valid_xy = (halo_col && j0 + hly < ny && hgi >= 0) ||
                               (halo_row && i0 + hlx < nx && hgj >= 0);

    int cur = 0, nxt = 1;
    float Bx_prev = 0.f, By_prev = 0.f;

    if (DIM == 3) {
        // B^{n+1/2} of plane kbeg-1 at the own cell (x, y components only)
        int km1 = wrap_or_neg(kbeg - 1, nz, g.per[2]);
        load_plane<DIM>(sE[1], g, f.E, i0, j0, kbeg - 1);
        load_plane<DIM>(sE[0], g, f.E, i0, j0, kbeg);
        __syncthreads();
        if (own && km1 >= 0) {
            float b[3];
            compute_B<DIM>(g, f, sE[1], sE[0], tx, ty, i, j, km1, 3, false, b);
            Bx_prev = b[0];
            By_prev = b[1];
        }
        __syncthreads();
    } else {
        load_plane<DIM>(sE[0], g, f.E, i0, j0, 0);
    }

    for (int k = kbeg; k < kend; ++k) {
        if (DIM == 3) load_plane<DIM>(sE[nxt], g, f.E, i0, j0, k + 1);
        __syncthreads();
        const long long o = ((long long)k * ny + j) * nx + i;
        float bown[3] = {0.f, 0.f, 0.f};
        if (own) {
            compute_B<DIM>(g, f, sE[cur], sE[nxt], tx, ty, i, j, k, 7, true, bown);
            f.Bn[0][o] = bown[0];
            f.Bn[1][o] = bown[1];
            f.Bn[2][o] = bown[2];
        }
        sB[0][ty + 1][tx + 1] = bown[0];
        sB[1][ty + 1][tx + 1] = bown[1];
        sB[2][ty + 1][tx + 1] = bown[2];
        if (halo_col || halo_row) {
            float hb[3] = {0.f, 0.f, 0.f};
            if (halo_valid_xy) {
                int comps = halo_col ? (4 | 2) : (4 | 1);
                compute_B<DIM>(g, f, sE[cur], sE[nxt], hlx, hly, hgi, hgj, k, comps, false, hb);
            }
            sB[0][hly + 1][hlx + 1] = hb[0];
            sB[1][hly + 1][hlx + 1] = hb[1];
            sB[2][hly + 1][hlx + 1] = hb[2];
        }
        __syncthreads();
        if (own) {
            const int X = tx + 1, Y = ty + 1;
            float jx = 0.f, jy = 0.f, jz = 0.f;
            if (jdirty) {
                jx = f.J[0][o];
                jy = f.J[1][o];
                jz = f.J[2][o];
                if (!f.keepJ) {
                    f.J[0][o] = 0.f;
                    f.J[1][o] = 0.f;
                    f.J[2][o] = 0.f;
                }
            }
            if (f.src_on) {
                int pos = f.inc == 0 ? i : (f.inc == 1 ? j : k);
                if (pos == f.src_index) {
                    float sv = (float)s_src;
                    if (f.pol == 0) jx += sv;
                    else if (f.pol == 1) jy += sv;
                    else jz += sv;
                }
            }
            const long long px = psi_index(g, f, 0, i, j, k);
            const long long py = psi_index(g, f, 1, i, j, k);
            const long long pz = DIM == 3 ? psi_index(g, f, 2, i, j, k) : -1;
            const float bx = sB[0][Y][X], by = sB[1][Y][X], bz = sB[2][Y][X];
            // E_x at (i+1/2, j, k)
            float dBz_dy = (bz - sB[2][Y - 1][X]) * g.inv_d[1];
            float tExy = cpml_term(f, 1, 0, py, j, false, dBz_dy, true);
            float tExz = 0.f, tEyz = 0.f;
            if (DIM == 3) {
                float dBy_dz = (by - By_prev) * g.inv_d[2];
                tExz = cpml_term(f, 2, 0, pz, k, false, dBy_dz, true);
                float dBx_dz = (bx - Bx_prev) * g.inv_d[2];
                tEyz = cpml_term(f, 2, 1, pz, k, false, dBx_dz, true);
            }
            float dBz_dx = (bz - sB[2][Y][X - 1]) * g.inv_d[0];
            float tEyx = cpml_term(f, 0, 0, px, i, false, dBz_dx, true);
            float dBy_dx = (by - sB[1][Y][X - 1]) * g.inv_d[0];
            float tEzx = cpml_term(f, 0, 1, px, i, false, dBy_dx, true);
            float dBx_dy = (bx - sB[0][Y - 1][X]) * g.inv_d[1];
            float tEzy = cpml_term(f, 1, 1, py, j, false, dBx_dy, true);
            if (f.inv_eps) {  // eps dE/dt = curl H - J (Eq. consteps), uniform per CTA
                const float ie = __ldg(f.inv_eps + o);
                f.En[0][o] = sE[cur][0][Y][X] + ie * (f.c2dt * (tExy - tExz) - f.dt_eps0 * jx);
                f.En[1][o] = sE[cur][1][Y][X] + ie * (f.c2dt * (tEyz - tEyx) - f.dt_eps0 * jy);
                f.En[2][o] = sE[cur][2][Y][X] + ie * (f.c2dt * (tEzx - tEzy) - f.dt_eps0 * jz);
            } else {
                f.En[0][o] = sE[cur][0][Y][X] + f.c2dt * (tExy - tExz) - f.dt_eps0 * jx;
                f.En[1][o] = sE[cur][1][Y][X] + f.c2dt * (tEyz - tEyx) - f.dt_eps0 * jy;
                f.En[2][o] = sE[cur][2][Y][X] + f.c2dt * (tEzx - tEzy) - f.dt_eps0 * jz;
            }
            Bx_prev = bx;
            By_prev = by;
        }
        cur ^= 1;
        nxt ^= 1;
        __syncthreads();
    }
    if (threadIdx.x == 0 && jdirty) f.jdirty_clear[bflag] = 0;
}

template <int DIM>
__global__ void __launch_bounds__(BX * BY) field_kernel(GridP g, FieldP f) {
    field_block<DIM>(g, f, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Many simulations in one launch: one CTA per item (simulation, bx, by, bz);
// the simulation's parameter blocks (FieldP per field ping-pong parity) are
// copied to shared memory.
template <int DIM>
__global__ void __launch_bounds__(BX * BY)
    batch_field_kernel(const GridP *grids, const FieldP *fdescs, const int *fpar, const int *active,
                       const int4 *items) {
    __shared__ GridP sg;
    __shared__ FieldP sf;
    const int4 w = items[blockIdx.x];
    if (!active[w.x]) return;
    {
        const int *src = reinterpret_cast<const int *>(grids + w.x);
        int *dst = reinterpret_cast<int *>(&sg);
        for (int q = threadIdx.x; q < (int)(sizeof(GridP) / 4); q += blockDim.x) dst[q] = src[q];
        src = reinterpret_cast<const int *>(fdescs + 2 * w.x + fpar[w.x]);
        dst = reinterpret_cast<int *>(&sf);
        for (int q = threadIdx.x; q < (int)(sizeof(FieldP) / 4); q += blockDim.x) dst[q] = src[q];
    }
    __syncthreads();
    field_block<DIM>(sg, sf, w.y, w.z, w.w);
}

// The current pass of an overlapped step: the field update ran without J
// (concurrently with the particle phase), so E^{n+1} -= (dt/eps0) J^{n+1/2}
// here, over the field blocks the deposit flagged; J and the flags are then
// cleared and the step counter advances.  Same arithmetic as the fused update
// (E^n + c^2 dt curl B - (dt/eps0) J, one multiply-add per term).
template <int DIM>
__global__ void __launch_bounds__(BX * BY)
    japply_kernel(GridP g, FieldP f, const float *inv_eps, long long *counter) {
    const long long b = ((long long)blockIdx.z * f.nby + blockIdx.y) * f.nbx + blockIdx.x;
    if (counter && threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)
        *counter += 1;
    if (!f.jdirty[b]) return;  // uniform over the CTA
    const int i = blockIdx.x * BX + threadIdx.x % BX, j = blockIdx.y * BY + threadIdx.x / BX;
    const int k0 = DIM == 3 ? blockIdx.z * f.zchunk : 0;
    const int k1 = DIM == 3 ? min(k0 + f.zchunk, g.n[2]) : 1;
    if (i < g.n[0] && j < g.n[1]) {
        for (int k = k0; k < k1; ++k) {
            const long long o = ((long long)k * g.n[1] + j) * g.n[0] + i;
            // eps dE/dt = curl H - J (Eq. consteps): the current's share of
            // E^{n+1}, 1/eps_r of it where a permittivity is set
            const float dte = inv_eps ? f.dt_eps0 * __ldg(inv_eps + o) : f.dt_eps0;
            for (int c = 0; c < 3; ++c) {
                const float jc = f.J[c][o];
                f.En[c][o] = __fmaf_rn(-dte, jc, f.En[c][o]);
                if (!f.keepJ) f.J[c][o] = 0.f;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) f.jdirty_clear[b] = 0;
}

}  // namespace

cudaError_t launch_batch_field(int dims, const GridP *grids, const FieldP *fdescs, const int *fpar,
                               const int *active, const int4 *items, int nitems, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    if (dims == 3) batch_field_kernel<3><<<nitems, BX * BY, 0, s>>>(grids, fdescs, fpar, active, items);
    else batch_field_kernel<2><<<nitems, BX * BY, 0, s>>>(grids, fdescs, fpar, active, items);
    return cudaGetLastError();
}

cudaError_t launch_japply(const GridP &g, const FieldP &f, const float *inv_eps, long long *counter,
                          cudaStream_t s) {
    dim3 grid(f.nbx, f.nby, f.nbz);
    if (g.dims == 3) japply_kernel<3><<<grid, BX * BY, 0, s>>>(g, f, inv_eps, counter);
    else japply_kernel<2><<<grid, BX * BY, 0, s>>>(g, f, inv_eps, counter);
    return cudaGetLastError();
}

cudaError_t launch_field(const GridP &g, const FieldP &f, cudaStream_t s) {
    dim3 block(BX * BY);
    if (g.dims == 3) {
        dim3 grid((g.n[0] + BX - 1) / BX, (g.n[1] + BY - 1) / BY, (g.n[2] + f.zchunk - 1) / f.zchunk);
        field_kernel<3><<<grid, block, 0, s>>>(g, f);
    } else {
        dim3 grid((g.n[0] + BX - 1) / BX, (g.n[1] + BY - 1) / BY, 1);
        field_kernel<2><<<grid, block, 0, s>>>(g, f);
    }
    return cudaGetLastError();
}

}  // namespace pic
