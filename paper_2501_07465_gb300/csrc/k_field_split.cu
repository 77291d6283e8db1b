// k_field_split.cu -- the Yee + CPML + source update as two streaming passes.
//
//   pass B:  B^{n+1/2} = B^{n-1/2} - dt (curl E^n + psi_B)
//   pass E:  E^{n+1}   = E^n + c^2 dt (curl B^{n+1/2} + psi_E) - (dt/eps0) J^{n+1/2}
// (Maxwell's curl equations on the Yee stagger, Sec. 4.1; Eq. consteps with
// eps = eps0; CPML after Roden & Gedney with kappa = 1, alpha = 0.)
//
// The fused kernels (k_field.cu, k_field_tma.cu) move 48 B per cell but
// recompute the B halo of every tile and hold each plane behind two CTA
// barriers; on sm_103a they stay latency- and issue-bound near 45 % of copy
// bandwidth.  Here each pass is a plain stencil stream with no shared memory
// and no barrier: one thread per (i, j) column marches up a chunk of z planes,
// keeps the z neighbour of the previous plane in registers and reads the x / y
// neighbours through L1 (they are the neighbouring threads' own values).  The
// two passes move 36 B per cell each (+ the memory terms in the CPML slabs,
// + J where the deposit flagged a block).  Pass B does not need this step's
// current, so it may run beside the particle phase.
//
// The CTA grid is the field-block grid of the fused kernels (32 x 8 columns
// x field_zchunk planes), so the particle kernel's block flags index it
// unchanged.
#include "pic_internal.cuh"

namespace pic {

namespace {

constexpr int BX = kFieldBX, BY = kFieldBY;

__device__ inline int slab_of(int i, int n, int P) {
    if (i < P) return i;
    if (i >= n - P) return i - (n - 2 * P);
    return -1;
}

// offsets of a column's memory terms: x slab [nz][ny][2P], y slab
// [nz][2P][nx], z slab [2P][ny][nx] (32-bit: grids of < 2^31 cells)
struct ColSlab {
    int sx, sy;      // slab index along x / y or -1
    int ox, oy, oz;  // offset at plane 0 (x, y) or slab plane 0 (z)
    int stx, sty, stz;
};

__device__ inline ColSlab col_slab(const GridP &g, const FieldP &f, int i, int j) {
    ColSlab c;
    const int nx = g.n[0], ny = g.n[1], P = f.P;
    c.sx = f.pml[0] ? slab_of(i, nx, P) : -1;
    c.sy = f.pml[1] ? slab_of(j, ny, P) : -1;
    c.ox = j * 2 * P + c.sx;
    c.oy = c.sy * nx + i;
    c.oz = j * nx + i;
    c.stx = ny * 2 * P;
    c.sty = 2 * P * nx;
    c.stz = nx * ny;
    return c;
}

// CTA-uniform: does any column or plane of this field block lie in a CPML
// slab?  Blocks that do are updated by the <PML = true> instantiation, the
// others by the lean one (each launch skips the other kind's blocks), so the
// register budget of the lean kernel does not carry the memory terms.
template <int DIM>
__device__ inline bool block_has_pml(const GridP &g, const FieldP &f) {
    const int P = f.P;
    const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY;
    bool r = (f.pml[0] && (i0 < P || i0 + BX > g.n[0] - P)) ||
             (f.pml[1] && (j0 < P || j0 + BY > g.n[1] - P));
    if (DIM == 3 && f.pml[2]) {
        const int k0 = blockIdx.z * f.zchunk, k1 = min(k0 + f.zchunk, g.n[2]);
        r = r || k0 < P || k1 > g.n[2] - P;
    }
    return r;
}

// slab offsets of a column at plane k (-1 outside the slab)
template <int DIM>
__device__ inline void slab_offsets(const GridP &g, const FieldP &f, const ColSlab &cs, int k,
                                    int &qx, int &qy, int &qz) {
    qx = cs.sx >= 0 ? cs.ox + k * cs.stx : -1;
    qy = cs.sy >= 0 ? cs.oy + k * cs.sty : -1;
    const int zs = (DIM == 3 && f.pml[2]) ? slab_of(k, g.n[2], f.P) : -1;
    qz = zs >= 0 ? cs.oz + zs * cs.stz : -1;
}

// everything the B pass reads for one plane, issued one plane ahead: E^n of
// the cell and its +x / +y neighbours, B^{n-1/2}, E_x / E_y of the plane
// above, and in CPML blocks the two B memory terms per slab axis
struct BLoads {
    float ez, ez_y, ex_y, ez_x, ey_x, bx, by, bz, exk, eyk;
    float px[2], py[2], pz[2];
    int qx, qy, qz;
};

template <int DIM, bool PML>
__device__ inline void b_loads(const GridP &g, const FieldP &f, const ColSlab &cs, long long o,
                               int k, long long dyp, int dxp, bool hx, bool hy, BLoads &L) {
    const long long pl = (long long)g.n[0] * g.n[1];
    const int nz = g.n[2];
    L.exk = L.eyk = 0.f;
    if (DIM == 3 && (k + 1 < nz || g.per[2])) {
        const long long oz = k + 1 < nz ? o + pl : o - (long long)(nz - 1) * pl;
        L.exk = __ldg(f.E[0] + oz);
        L.eyk = __ldg(f.E[1] + oz);
    }
    L.ez = __ldg(f.E[2] + o);
    L.ez_y = hy ? __ldg(f.E[2] + o + dyp) : 0.f;
    L.ex_y = hy ? __ldg(f.E[0] + o + dyp) : 0.f;
    L.ez_x = hx ? __ldg(f.E[2] + o + dxp) : 0.f;
    L.ey_x = hx ? __ldg(f.E[1] + o + dxp) : 0.f;
    L.bx = __ldg(f.B[0] + o);
    L.by = __ldg(f.B[1] + o);
    L.bz = __ldg(f.B[2] + o);
    if (PML) {
        slab_offsets<DIM>(g, f, cs, k, L.qx, L.qy, L.qz);
        // x slab: B_y, B_z (slots 2, 3); y slab: B_x, B_z; z slab: B_x, B_y
        if (L.qx >= 0) {
            L.px[0] = __ldg(f.psi_in[0][2] + L.qx);
            L.px[1] = __ldg(f.psi_in[0][3] + L.qx);
        }
        if (L.qy >= 0) {
            L.py[0] = __ldg(f.psi_in[1][2] + L.qy);
            L.py[1] = __ldg(f.psi_in[1][3] + L.qy);
        }
        if (L.qz >= 0) {
            L.pz[0] = __ldg(f.psi_in[2][2] + L.qz);
            L.pz[1] = __ldg(f.psi_in[2][3] + L.qz);
        }
    }
}

// memory term from a preloaded old value: psi <- b psi + c deriv, stored;
// returns deriv + psi
__device__ inline float cpml_pre(float *psi_out, int q, float old, float b, float c, float deriv) {
    const float psi = b * old + c * deriv;
    psi_out[q] = psi;
    return deriv + psi;
}

template <int DIM, bool PML>
__global__ void __launch_bounds__(BX * BY, DIM == 3 ? (PML ? 4 : 5) : 8) field_b_kernel(GridP g, FieldP f) {
    int bx = blockIdx.x, by = blockIdx.y, bz = blockIdx.z;
    if (f.blk[0]) {
        field_list_block(f, PML ? 2 : (f.tma_b ? 1 : 3), bx, by, bz);
    } else {
        if (block_has_pml<DIM>(g, f) != PML) return;  // the other instantiation's block
        if (!PML && field_b_tma_block(g, f, bx, by, bz)) return;  // the TMA pass's block
    }
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int i = bx * BX + threadIdx.x % BX;
    const int j = by * BY + threadIdx.x / BX;
    if (i >= nx || j >= ny) return;
    const int k0 = DIM == 3 ? bz * f.zchunk : 0;
    const int k1 = DIM == 3 ? min(k0 + f.zchunk, nz) : 1;
    const long long pl = (long long)nx * ny;
    // neighbour offsets (+x, +y) with the periodic wrap; beyond a wall E = 0
    const int dxp = i + 1 < nx ? 1 : (g.per[0] ? 1 - nx : 0);
    const bool hx = i + 1 < nx || g.per[0];
    const long long dyp = j + 1 < ny ? nx : (g.per[1] ? (long long)(1 - ny) * nx : 0);
    const bool hy = j + 1 < ny || g.per[1];
    const float dt = g.dt, idx_ = g.inv_d[0], idy = g.inv_d[1], idz = g.inv_d[2];
    ColSlab cs{};
    float bhx = 0.f, ahx = 0.f, bhy = 0.f, ahy = 0.f;
    if (PML) {
        cs = col_slab(g, f, i, j);
        if (cs.sx >= 0) {
            bhx = __ldg(f.cb_h[0] + i);
            ahx = __ldg(f.ca_h[0] + i);
        }
        if (cs.sy >= 0) {
            bhy = __ldg(f.cb_h[1] + j);
            ahy = __ldg(f.ca_h[1] + j);
        }
    }
    long long o = ((long long)k0 * ny + j) * nx + i;
    float ex = __ldg(f.E[0] + o), ey = __ldg(f.E[1] + o);
    BLoads cur, nxt;
    b_loads<DIM, PML>(g, f, cs, o, k0, dyp, dxp, hx, hy, cur);
    for (int k = k0; k < k1; ++k, o += pl) {
        if (k + 1 < k1) b_loads<DIM, PML>(g, f, cs, o + pl, k + 1, dyp, dxp, hx, hy, nxt);
        float dEz_dy = (cur.ez_y - cur.ez) * idy;
        float dEx_dy = (cur.ex_y - ex) * idy;
        float dEz_dx = (cur.ez_x - cur.ez) * idx_;
        float dEy_dx = (cur.ey_x - ey) * idx_;
        float dEy_dz = 0.f, dEx_dz = 0.f;
        if (DIM == 3) {
            dEy_dz = (cur.eyk - ey) * idz;
            dEx_dz = (cur.exk - ex) * idz;
        }
        if (PML) {
            if (cur.qy >= 0) {
                dEz_dy = cpml_pre(f.psi_out[1][2], cur.qy, cur.py[0], bhy, ahy, dEz_dy);
                dEx_dy = cpml_pre(f.psi_out[1][3], cur.qy, cur.py[1], bhy, ahy, dEx_dy);
            }
            if (cur.qx >= 0) {
                dEz_dx = cpml_pre(f.psi_out[0][2], cur.qx, cur.px[0], bhx, ahx, dEz_dx);
                dEy_dx = cpml_pre(f.psi_out[0][3], cur.qx, cur.px[1], bhx, ahx, dEy_dx);
            }
            if (cur.qz >= 0) {
                const float bhz = __ldg(f.cb_h[2] + k), ahz = __ldg(f.ca_h[2] + k);
                dEy_dz = cpml_pre(f.psi_out[2][2], cur.qz, cur.pz[0], bhz, ahz, dEy_dz);
                dEx_dz = cpml_pre(f.psi_out[2][3], cur.qz, cur.pz[1], bhz, ahz, dEx_dz);
            }
        }
        f.Bn[0][o] = cur.bx - dt * (dEz_dy - dEy_dz);
        f.Bn[1][o] = cur.by - dt * (dEx_dz - dEz_dx);
        f.Bn[2][o] = cur.bz - dt * (dEy_dx - dEx_dy);
        ex = cur.exk;
        ey = cur.eyk;
        cur = nxt;
    }
}

// everything the E pass reads for one plane, issued one plane ahead:
// B^{n+1/2} of the cell and its -x / -y neighbours, E^n, J in flagged blocks,
// and in CPML blocks the two E memory terms per slab axis
struct ELoads {
    float bx, by, bz, bz_y, bx_y, bz_x, by_x, e0, e1, e2, jx, jy, jz;
    float ie;  // 1 / eps_r of the cell
    float px[2], py[2], pz[2];
    int qx, qy, qz;
};

template <int DIM, bool PML, bool EPS>
__device__ inline void e_loads(const GridP &g, const FieldP &f, const float *inv_eps,
                               const ColSlab &cs, long long o, int k, long long dym, int dxm,
                               bool hx, bool hy, bool jdirty, ELoads &L) {
    L.bx = __ldg(f.Bn[0] + o);
    L.by = __ldg(f.Bn[1] + o);
    L.bz = __ldg(f.Bn[2] + o);
    L.bz_y = hy ? __ldg(f.Bn[2] + o + dym) : 0.f;
    L.bx_y = hy ? __ldg(f.Bn[0] + o + dym) : 0.f;
    L.bz_x = hx ? __ldg(f.Bn[2] + o + dxm) : 0.f;
    L.by_x = hx ? __ldg(f.Bn[1] + o + dxm) : 0.f;
    L.e0 = __ldg(f.E[0] + o);
    L.e1 = __ldg(f.E[1] + o);
    L.e2 = __ldg(f.E[2] + o);
    L.ie = EPS ? __ldg(inv_eps + o) : 1.f;
    L.jx = L.jy = L.jz = 0.f;
    if (jdirty) {  // J is cleared by this thread one plane later
        L.jx = __ldcg(f.J[0] + o);
        L.jy = __ldcg(f.J[1] + o);
        L.jz = __ldcg(f.J[2] + o);
    }
    if (PML) {
        slab_offsets<DIM>(g, f, cs, k, L.qx, L.qy, L.qz);
        // x slab: E_y, E_z (slots 0, 1); y slab: E_x, E_z; z slab: E_x, E_y
        if (L.qx >= 0) {
            L.px[0] = __ldg(f.psi_in[0][0] + L.qx);
            L.px[1] = __ldg(f.psi_in[0][1] + L.qx);
        }
        if (L.qy >= 0) {
            L.py[0] = __ldg(f.psi_in[1][0] + L.qy);
            L.py[1] = __ldg(f.psi_in[1][1] + L.qy);
        }
        if (L.qz >= 0) {
            L.pz[0] = __ldg(f.psi_in[2][0] + L.qz);
            L.pz[1] = __ldg(f.psi_in[2][1] + L.qz);
        }
    }
}

// the soft source's current density at step n (t = (n + 1/2) dt)
__device__ inline float source_value(const FieldP &f) {
    if (!f.src_on) return 0.f;
    if (f.src_host) return f.src_val;
    const long long n = *f.step_counter - 1;  // the particle phase of step n ran
    const double t = ((double)n + 0.5) * f.dt64 - f.src_t0;
    return (float)(f.src_amp * exp(-2.0 * 0.6931471805599453 * t * t / (f.src_tau * f.src_tau)) *
                   sin(f.src_omega * t));
}

// EPS: a permittivity is set (its own instantiation: the vacuum kernel keeps
// its registers)
// Register budgets pinned (a change elsewhere in the kernel once moved the
// vacuum E pass from 64 to 80 registers and one CTA per SM, 0.166 -> 0.181 ms
// at 256^3): 4 CTAs of 256 threads per SM (64 registers) for the vacuum lean
// pass, 3 (80) with CPML memory terms or a permittivity; the B pass 5 (48)
// and 4 (64).  2D: the E pass 8 (32) and 6 (40) with CPML, the B pass 8.
template <int DIM, bool PML, bool EPS>
__global__ void __launch_bounds__(BX * BY, DIM == 3 ? ((PML || EPS) ? 3 : 4) : (PML ? 6 : 8))
    field_e_kernel(GridP g, FieldP f, const float *inv_eps) {
    int bx = blockIdx.x, by = blockIdx.y, bz = blockIdx.z;
    if (f.blk[0]) field_list_block(f, PML ? 2 : 3, bx, by, bz);
    else if (block_has_pml<DIM>(g, f) != PML) return;  // the other instantiation's block
    __shared__ float s_src;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long long bflag = ((long long)bz * f.nby + by) * f.nbx + bx;
    // splitJ: the pass runs beside the particle phase and leaves J (and the
    // block flags) to the current pass that follows it
    const bool jdirty = !f.splitJ && f.jdirty[bflag] != 0;
    float src;
    if (f.src_host || !f.src_on) {
        src = f.src_on ? f.src_val : 0.f;
    } else {
        if (threadIdx.x == 0) s_src = source_value(f);
        __syncthreads();
        src = s_src;
    }
    const int i = bx * BX + threadIdx.x % BX;
    const int j = by * BY + threadIdx.x / BX;
    const int k0 = DIM == 3 ? bz * f.zchunk : 0;
    const int k1 = DIM == 3 ? min(k0 + f.zchunk, nz) : 1;
    if (i < nx && j < ny) {
        const long long pl = (long long)nx * ny;
        const int dxm = i > 0 ? -1 : (g.per[0] ? nx - 1 : 0);
        const bool hx = i > 0 || g.per[0];
        const long long dym = j > 0 ? -(long long)nx : (g.per[1] ? (long long)(ny - 1) * nx : 0);
        const bool hy = j > 0 || g.per[1];
        const float c2dt = f.c2dt, dte = f.dt_eps0;
        const float idx_ = g.inv_d[0], idy = g.inv_d[1], idz = g.inv_d[2];
        ColSlab cs{};
        float bex = 0.f, aex = 0.f, bey = 0.f, aey = 0.f;
        if (PML) {
            cs = col_slab(g, f, i, j);
            if (cs.sx >= 0) {
                bex = __ldg(f.cb_e[0] + i);
                aex = __ldg(f.ca_e[0] + i);
            }
            if (cs.sy >= 0) {
                bey = __ldg(f.cb_e[1] + j);
                aey = __ldg(f.ca_e[1] + j);
            }
        }
        const int spos = f.inc == 0 ? i : (f.inc == 1 ? j : -1);
        const bool clearJ = jdirty && !f.keepJ;
        long long o = ((long long)k0 * ny + j) * nx + i;
        // B_x, B_y of plane k-1
        float bxm = 0.f, bym = 0.f;
        if (DIM == 3 && (k0 > 0 || g.per[2])) {
            const long long om = k0 > 0 ? o - pl : o + (long long)(nz - 1) * pl;
            bxm = __ldg(f.Bn[0] + om);
            bym = __ldg(f.Bn[1] + om);
        }
        ELoads cur, nxt;
        e_loads<DIM, PML, EPS>(g, f, inv_eps, cs, o, k0, dym, dxm, hx, hy, jdirty, cur);
        for (int k = k0; k < k1; ++k, o += pl) {
            if (k + 1 < k1)
                e_loads<DIM, PML, EPS>(g, f, inv_eps, cs, o + pl, k + 1, dym, dxm, hx, hy, jdirty,
                                       nxt);
            if (clearJ) {
                __stcg(f.J[0] + o, 0.f);
                __stcg(f.J[1] + o, 0.f);
                __stcg(f.J[2] + o, 0.f);
            }
            float jx = cur.jx, jy = cur.jy, jz = cur.jz;
            if (f.src_on && (f.inc == 2 ? k : spos) == f.src_index) {
                if (f.pol == 0) jx += src;
                else if (f.pol == 1) jy += src;
                else jz += src;
            }
            float tExy = (cur.bz - cur.bz_y) * idy;
            float tEzy = (cur.bx - cur.bx_y) * idy;
            float tEyx = (cur.bz - cur.bz_x) * idx_;
            float tEzx = (cur.by - cur.by_x) * idx_;
            float tExz = 0.f, tEyz = 0.f;
            if (DIM == 3) {
                tExz = (cur.by - bym) * idz;
                tEyz = (cur.bx - bxm) * idz;
            }
            if (PML) {
                if (cur.qy >= 0) {
                    tExy = cpml_pre(f.psi_out[1][0], cur.qy, cur.py[0], bey, aey, tExy);
                    tEzy = cpml_pre(f.psi_out[1][1], cur.qy, cur.py[1], bey, aey, tEzy);
                }
                if (cur.qx >= 0) {
                    tEyx = cpml_pre(f.psi_out[0][0], cur.qx, cur.px[0], bex, aex, tEyx);
                    tEzx = cpml_pre(f.psi_out[0][1], cur.qx, cur.px[1], bex, aex, tEzx);
                }
                if (cur.qz >= 0) {
                    const float bez = __ldg(f.cb_e[2] + k), aez = __ldg(f.ca_e[2] + k);
                    tExz = cpml_pre(f.psi_out[2][0], cur.qz, cur.pz[0], bez, aez, tExz);
                    tEyz = cpml_pre(f.psi_out[2][1], cur.qz, cur.pz[1], bez, aez, tEyz);
                }
            }
            if (EPS) {  // eps dE/dt = curl H - J (Eq. consteps)
                f.En[0][o] = cur.e0 + cur.ie * (c2dt * (tExy - tExz) - dte * jx);
                f.En[1][o] = cur.e1 + cur.ie * (c2dt * (tEyz - tEyx) - dte * jy);
                f.En[2][o] = cur.e2 + cur.ie * (c2dt * (tEzx - tEzy) - dte * jz);
            } else {
                f.En[0][o] = cur.e0 + c2dt * (tExy - tExz) - dte * jx;
                f.En[1][o] = cur.e1 + c2dt * (tEyz - tEyx) - dte * jy;
                f.En[2][o] = cur.e2 + c2dt * (tEzx - tEzy) - dte * jz;
            }
            bxm = cur.bx;
            bym = cur.by;
            cur = nxt;
        }
    }
    if (jdirty) {
        __syncthreads();
        if (threadIdx.x == 0) f.jdirty_clear[bflag] = 0;
    }
}

}  // namespace

cudaError_t launch_field_b(const GridP &g, const FieldP &f, cudaStream_t s) {
    if (f.blk[0]) {  // each launch over its compact block list
        const int nl = f.nblk[f.tma_b ? 1 : 3], np = f.nblk[2];
        if (g.dims == 3) {
            if (nl > 0) field_b_kernel<3, false><<<nl, BX * BY, 0, s>>>(g, f);
            if (np > 0) field_b_kernel<3, true><<<np, BX * BY, 0, s>>>(g, f);
        } else {
            if (nl > 0) field_b_kernel<2, false><<<nl, BX * BY, 0, s>>>(g, f);
            if (np > 0) field_b_kernel<2, true><<<np, BX * BY, 0, s>>>(g, f);
        }
        return cudaGetLastError();
    }
    dim3 grid((g.n[0] + BX - 1) / BX, (g.n[1] + BY - 1) / BY,
              g.dims == 3 ? (g.n[2] + f.zchunk - 1) / f.zchunk : 1);
    const bool pml = f.pml[0] || f.pml[1] || f.pml[2];
    if (g.dims == 3) {
        field_b_kernel<3, false><<<grid, BX * BY, 0, s>>>(g, f);
        if (pml) field_b_kernel<3, true><<<grid, BX * BY, 0, s>>>(g, f);
    } else {
        field_b_kernel<2, false><<<grid, BX * BY, 0, s>>>(g, f);
        if (pml) field_b_kernel<2, true><<<grid, BX * BY, 0, s>>>(g, f);
    }
    return cudaGetLastError();
}

cudaError_t launch_field_e(const GridP &g, const FieldP &f, const float *inv_eps, cudaStream_t s) {
    if (f.blk[0]) {  // each launch over its compact block list
        const int nl = f.nblk[3], np = f.nblk[2];
        if (g.dims == 3) {
            if (inv_eps) {
                if (nl > 0) field_e_kernel<3, false, true><<<nl, BX * BY, 0, s>>>(g, f, inv_eps);
                if (np > 0) field_e_kernel<3, true, true><<<np, BX * BY, 0, s>>>(g, f, inv_eps);
            } else {
                if (nl > 0) field_e_kernel<3, false, false><<<nl, BX * BY, 0, s>>>(g, f, nullptr);
                if (np > 0) field_e_kernel<3, true, false><<<np, BX * BY, 0, s>>>(g, f, nullptr);
            }
        } else {
            if (inv_eps) {
                if (nl > 0) field_e_kernel<2, false, true><<<nl, BX * BY, 0, s>>>(g, f, inv_eps);
                if (np > 0) field_e_kernel<2, true, true><<<np, BX * BY, 0, s>>>(g, f, inv_eps);
            } else {
                if (nl > 0) field_e_kernel<2, false, false><<<nl, BX * BY, 0, s>>>(g, f, nullptr);
                if (np > 0) field_e_kernel<2, true, false><<<np, BX * BY, 0, s>>>(g, f, nullptr);
            }
        }
        return cudaGetLastError();
    }
    dim3 grid((g.n[0] + BX - 1) / BX, (g.n[1] + BY - 1) / BY,
              g.dims == 3 ? (g.n[2] + f.zchunk - 1) / f.zchunk : 1);
    const bool pml = f.pml[0] || f.pml[1] || f.pml[2];
    if (g.dims == 3) {
        if (inv_eps) {
            field_e_kernel<3, false, true><<<grid, BX * BY, 0, s>>>(g, f, inv_eps);
            if (pml) field_e_kernel<3, true, true><<<grid, BX * BY, 0, s>>>(g, f, inv_eps);
        } else {
            field_e_kernel<3, false, false><<<grid, BX * BY, 0, s>>>(g, f, nullptr);
            if (pml) field_e_kernel<3, true, false><<<grid, BX * BY, 0, s>>>(g, f, nullptr);
        }
    } else {
        if (inv_eps) {
            field_e_kernel<2, false, true><<<grid, BX * BY, 0, s>>>(g, f, inv_eps);
            if (pml) field_e_kernel<2, true, true><<<grid, BX * BY, 0, s>>>(g, f, inv_eps);
        } else {
            field_e_kernel<2, false, false><<<grid, BX * BY, 0, s>>>(g, f, nullptr);
            if (pml) field_e_kernel<2, true, false><<<grid, BX * BY, 0, s>>>(g, f, nullptr);
        }
    }
    return cudaGetLastError();
}

}  // namespace pic
