// k_field_stream.cu -- the Yee + CPML + source update in one streaming pass.
//
//   B^{n+1/2} = B^{n-1/2} - dt (curl E^n + psi_B)
//   E^{n+1}   = E^n + c^2 dt (curl B^{n+1/2} + psi_E) - (dt/eps0) (J^{n+1/2} + source)
// (Maxwell's curl equations on the Yee stagger, Sec. 4.1; Eq. consteps with
// eps = eps0; CPML after Roden & Gedney with kappa = 1, alpha = 0.)
//
// One thread per (i, j) column marches up a chunk of z planes and updates
// both fields of its cells, so each cell's E and B are read and written once
// (48 B per cell, as the fused kernels of k_field.cu / k_field_tma.cu) without
// shared memory or CTA barriers (as the split passes of k_field_split.cu).
// The E update at (i, j, k) needs B^{n+1/2} at the cell and at its -x, -y and
// -z neighbours:
//   -x  B_y, B_z from lane - 1 by a warp shuffle (lane 0 recomputes them);
//   -y  B_x, B_z recomputed by the thread from E^n, B^{n-1/2} of the row below
//       (those loads hit L1: they are the neighbouring warp's own values);
//   -z  B_x, B_y of the previous plane, kept in registers (the first plane of
//       a chunk recomputes the plane below).
// Every B^{n+1/2} value, stored or recomputed, comes from the same operations
// on the same inputs with each operation rounded on its own (no contraction),
// so a recomputed neighbour equals the value its owner stores bit for bit and
// div B, div(curl) stay what the two-pass update gives.  CPML memory terms are
// written by the owner only; a recomputation reads the old term.
//
// The CTA grid is the field-block grid (32 x 8 columns x field_zchunk planes),
// so the particle kernel's block flags index it unchanged.
#include "pic_internal.cuh"

namespace pic {

namespace {

constexpr int BX = kFieldBX, BY = kFieldBY;
static_assert(BX == 32, "one warp per row of a field block");

__device__ inline int slab_of(int i, int n, int P) {
    if (i < P) return i;
    if (i >= n - P) return i - (n - 2 * P);
    return -1;
}

// slab offsets of the memory terms of cell (i, j, k): x slab [nz][ny][2P],
// y slab [nz][2P][nx], z slab [2P][ny][nx]; -1 outside a slab
struct SlabQ {
    int qx, qy, qz;
};

template <int DIM>
__device__ inline SlabQ slab_q(const GridP &g, const FieldP &f, int i, int j, int k) {
    SlabQ q;
    const int nx = g.n[0], ny = g.n[1], P = f.P;
    const int sx = f.pml[0] ? slab_of(i, nx, P) : -1;
    const int sy = f.pml[1] ? slab_of(j, ny, P) : -1;
    const int sz = (DIM == 3 && f.pml[2]) ? slab_of(k, g.n[2], P) : -1;
    q.qx = sx >= 0 ? (k * ny + j) * 2 * P + sx : -1;
    q.qy = sy >= 0 ? (k * 2 * P + sy) * nx + i : -1;
    q.qz = sz >= 0 ? (sz * ny + j) * nx + i : -1;
    return q;
}

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

// (hi - lo) / d, each operation rounded on its own
__device__ inline float dd(float hi, float lo, float inv_d) {
    return __fmul_rn(__fsub_rn(hi, lo), inv_d);
}

// a derivative with its memory term: psi = b old + c d; returns d + psi
template <bool OWN>
__device__ inline float with_psi(float d, const float *psi_in, float *psi_out, int q, float b,
                                 float c) {
    const float psi = __fadd_rn(__fmul_rn(b, __ldg(psi_in + q)), __fmul_rn(c, d));
    if (OWN) psi_out[q] = psi;
    return __fadd_rn(d, psi);
}

// B^{n+1/2} from B^{n-1/2} and the two curl terms
__device__ inline float bnew(float bold, float t1, float t2, float dt) {
    return __fsub_rn(bold, __fmul_rn(dt, __fsub_rn(t1, t2)));
}

// ---- the three B components of a cell (i, j, k), from the E^n values they
// need.  Memory-term slots: x slab dEz/dx -> 2, dEy/dx -> 3; y slab dEz/dy
// -> 2, dEx/dy -> 3; z slab dEy/dz -> 2, dEx/dz -> 3.

// B_x = B_x - dt (dEz/dy - dEy/dz)
template <int DIM, bool PML, bool OWN>
__device__ inline float bx_of(const GridP &g, const FieldP &f, const SlabQ &q, int j, int k,
                              float bold, float ez, float ez_yp, float ey, float ey_kp) {
    float t1 = dd(ez_yp, ez, g.inv_d[1]);
    float t2 = DIM == 3 ? dd(ey_kp, ey, g.inv_d[2]) : 0.f;
    if (PML) {
        if (q.qy >= 0)
            t1 = with_psi<OWN>(t1, f.psi_in[1][2], f.psi_out[1][2], q.qy, __ldg(f.cb_h[1] + j),
                               __ldg(f.ca_h[1] + j));
        if (q.qz >= 0)
            t2 = with_psi<OWN>(t2, f.psi_in[2][2], f.psi_out[2][2], q.qz, __ldg(f.cb_h[2] + k),
                               __ldg(f.ca_h[2] + k));
    }
    return bnew(bold, t1, t2, g.dt);
}

// B_y = B_y - dt (dEx/dz - dEz/dx)
template <int DIM, bool PML, bool OWN>
__device__ inline float by_of(const GridP &g, const FieldP &f, const SlabQ &q, int i, int k,
                              float bold, float ex, float ex_kp, float ez, float ez_xp) {
    float t1 = DIM == 3 ? dd(ex_kp, ex, g.inv_d[2]) : 0.f;
    float t2 = dd(ez_xp, ez, g.inv_d[0]);
    if (PML) {
        if (q.qz >= 0)
            t1 = with_psi<OWN>(t1, f.psi_in[2][3], f.psi_out[2][3], q.qz, __ldg(f.cb_h[2] + k),
                               __ldg(f.ca_h[2] + k));
        if (q.qx >= 0)
            t2 = with_psi<OWN>(t2, f.psi_in[0][2], f.psi_out[0][2], q.qx, __ldg(f.cb_h[0] + i),
                               __ldg(f.ca_h[0] + i));
    }
    return bnew(bold, t1, t2, g.dt);
}

// B_z = B_z - dt (dEy/dx - dEx/dy)
template <bool PML, bool OWN>
__device__ inline float bz_of(const GridP &g, const FieldP &f, const SlabQ &q, int i, int j,
                              float bold, float ey, float ey_xp, float ex, float ex_yp) {
    float t1 = dd(ey_xp, ey, g.inv_d[0]);
    float t2 = dd(ex_yp, ex, g.inv_d[1]);
    if (PML) {
        if (q.qx >= 0)
            t1 = with_psi<OWN>(t1, f.psi_in[0][3], f.psi_out[0][3], q.qx, __ldg(f.cb_h[0] + i),
                               __ldg(f.ca_h[0] + i));
        if (q.qy >= 0)
            t2 = with_psi<OWN>(t2, f.psi_in[1][3], f.psi_out[1][3], q.qy, __ldg(f.cb_h[1] + j),
                               __ldg(f.ca_h[1] + j));
    }
    return bnew(bold, t1, t2, g.dt);
}

__device__ inline float ld_or0(const float *p, long long o, bool ok) { return ok ? __ldg(p + o) : 0.f; }

// Geometry of a column: its own offset, its neighbours' offsets and which of
// them exist (beyond a wall E = B = 0).
struct Col {
    long long dxp, dxm, dyp, dym, pl;
    int ic, jc, im, jm;
    bool hxp, hxm, hyp, hym, xp_ld, xm_ld;
};

// Everything plane k needs from memory, issued one plane ahead: E^n and
// B^{n-1/2} of the own cell and of the row below (for the -y neighbour's
// B^{n+1/2}), E^n of the +y cell and of the plane above, J in flagged blocks,
// and the edge lanes' extra values (lane 31: its +x column; lane 0: what the
// -x neighbour's B^{n+1/2} needs).
struct PlaneIn {
    float ez, ex_kp, ey_kp, ex_yp, ez_yp, bx0, by0, bz0;
    float ex_ym, ez_ym, eykp_ym, bx0_ym, bz0_ym;
    float ey_xp, ez_xp, eyym_xp;              // +x column (lane 31 / ragged edge)
    float exm, eym, ezm, exm_kp, exm_yp, bym0, bzm0;  // -x column (lane 0)
    float jx, jy, jz;
    bool hkp;
    long long okp;
};

template <int DIM>
__device__ inline void plane_in(const GridP &g, const FieldP &f, const Col &c, long long o, int k,
                                bool jdirty, PlaneIn &L) {
    const int nz = g.n[2];
    L.hkp = DIM == 3 && (k + 1 < nz || g.per[2]);
    L.okp = DIM == 3 ? (k + 1 < nz ? o + c.pl : o - (long long)(nz - 1) * c.pl) : o;
    L.ez = __ldg(f.E[2] + o);
    L.ex_kp = DIM == 3 ? ld_or0(f.E[0], L.okp, L.hkp) : 0.f;
    L.ey_kp = DIM == 3 ? ld_or0(f.E[1], L.okp, L.hkp) : 0.f;
    L.ex_yp = ld_or0(f.E[0], o + c.dyp, c.hyp);
    L.ez_yp = ld_or0(f.E[2], o + c.dyp, c.hyp);
    L.bx0 = __ldg(f.B[0] + o);
    L.by0 = __ldg(f.B[1] + o);
    L.bz0 = __ldg(f.B[2] + o);
    L.ex_ym = ld_or0(f.E[0], o + c.dym, c.hym);
    L.ez_ym = ld_or0(f.E[2], o + c.dym, c.hym);
    L.eykp_ym = DIM == 3 ? ld_or0(f.E[1], L.okp + c.dym, L.hkp && c.hym) : 0.f;
    L.bx0_ym = ld_or0(f.B[0], o + c.dym, c.hym);
    L.bz0_ym = ld_or0(f.B[2], o + c.dym, c.hym);
    if (c.xp_ld) {
        L.ey_xp = ld_or0(f.E[1], o + c.dxp, c.hxp);
        L.ez_xp = ld_or0(f.E[2], o + c.dxp, c.hxp);
        L.eyym_xp = ld_or0(f.E[1], o + c.dym + c.dxp, c.hxp && c.hym);
    }
    if (c.xm_ld) {
        const long long om = o + c.dxm;
        L.exm = __ldg(f.E[0] + om);
        L.eym = __ldg(f.E[1] + om);
        L.ezm = __ldg(f.E[2] + om);
        L.exm_kp = DIM == 3 ? ld_or0(f.E[0], L.okp + c.dxm, L.hkp) : 0.f;
        L.exm_yp = ld_or0(f.E[0], om + c.dyp, c.hyp);
        L.bym0 = __ldg(f.B[1] + om);
        L.bzm0 = __ldg(f.B[2] + om);
    }
    L.jx = L.jy = L.jz = 0.f;
    if (jdirty) {
        L.jx = __ldcg(f.J[0] + o);
        L.jy = __ldcg(f.J[1] + o);
        L.jz = __ldcg(f.J[2] + o);
    }
}

template <int DIM, bool PML>
__global__ void __launch_bounds__(BX * BY) field_stream_kernel(GridP g, FieldP f) {
    if (block_has_pml<DIM>(g, f) != PML) return;  // the other instantiation's block
    __shared__ float s_src;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long long bflag = ((long long)blockIdx.z * f.nby + blockIdx.y) * f.nbx + blockIdx.x;
    const bool jdirty = !f.splitJ && f.jdirty[bflag] != 0;
    float src = 0.f;
    if (f.src_on) {
        if (f.src_host) {
            src = f.src_val;
        } else {
            if (threadIdx.x == 0) {
                const long long n = *f.step_counter - 1;  // the particle phase of step n ran
                const double t = ((double)n + 0.5) * f.dt64 - f.src_t0;
                s_src = (float)(f.src_amp *
                                exp(-2.0 * 0.6931471805599453 * t * t / (f.src_tau * f.src_tau)) *
                                sin(f.src_omega * t));
            }
            __syncthreads();
            src = s_src;
        }
    }
    const int lane = threadIdx.x % BX;
    const int i = blockIdx.x * BX + lane;
    const int j = blockIdx.y * BY + threadIdx.x / BX;
    // threads beyond the grid keep shuffling (with clamped, unused values)
    const bool live = i < nx && j < ny;
    Col c;
    c.ic = min(i, nx - 1);
    c.jc = min(j, ny - 1);
    c.hxp = c.ic + 1 < nx || g.per[0];
    c.hxm = c.ic > 0 || g.per[0];
    c.hyp = c.jc + 1 < ny || g.per[1];
    c.hym = c.jc > 0 || g.per[1];
    const int ip = c.ic + 1 < nx ? c.ic + 1 : 0, jp = c.jc + 1 < ny ? c.jc + 1 : 0;
    c.im = c.ic > 0 ? c.ic - 1 : nx - 1;
    c.jm = c.jc > 0 ? c.jc - 1 : ny - 1;
    c.dxp = ip - c.ic;
    c.dxm = c.im - c.ic;
    c.dyp = (long long)(jp - c.jc) * nx;
    c.dym = (long long)(c.jm - c.jc) * nx;
    c.pl = (long long)nx * ny;
    // E(i+1) by shuffle where lane + 1 holds column i + 1, else loaded; B(i-1)
    // by shuffle from lane - 1, recomputed by lane 0
    c.xp_ld = !(lane < BX - 1 && c.ic + 1 < nx);
    c.xm_ld = lane == 0 && c.hxm;
    const int ic = c.ic, jc = c.jc, im = c.im, jm = c.jm;
    const int k0 = DIM == 3 ? blockIdx.z * f.zchunk : 0;
    const int k1 = DIM == 3 ? min(k0 + f.zchunk, nz) : 1;
    const float c2dt = f.c2dt, dte = f.dt_eps0;
    const float idx_ = g.inv_d[0], idy = g.inv_d[1], idz = g.inv_d[2];
    const int spos = f.inc == 0 ? i : (f.inc == 1 ? j : -1);
    const bool clearJ = jdirty && !f.keepJ;
    const unsigned full = 0xffffffffu;

    long long o = ((long long)k0 * ny + jc) * nx + ic;
    // E_x, E_y of the own column at plane k (carried), E_y of the row below
    float ex = __ldg(f.E[0] + o), ey = __ldg(f.E[1] + o);
    float ey_ym = ld_or0(f.E[1], o + c.dym, c.hym);
    PlaneIn cur, nxt;
    plane_in<DIM>(g, f, c, o, k0, jdirty, cur);
    // B_x, B_y of plane k0 - 1 (the -z neighbours of the first plane)
    float bx_km = 0.f, by_km = 0.f;
    if (DIM == 3 && (k0 > 0 || g.per[2])) {
        const int km = k0 > 0 ? k0 - 1 : nz - 1;
        const long long om = ((long long)km * ny + jc) * nx + ic;
        const float exm = __ldg(f.E[0] + om), eym = __ldg(f.E[1] + om), ezm = __ldg(f.E[2] + om);
        const float ezm_yp = ld_or0(f.E[2], om + c.dyp, c.hyp);
        float ezm_xp = __shfl_down_sync(full, ezm, 1);
        if (c.xp_ld) ezm_xp = ld_or0(f.E[2], om + c.dxp, c.hxp);
        // plane km + 1 is k0 (or 0 when km wraps): E_x, E_y of the own column there
        const SlabQ qm = PML ? slab_q<DIM>(g, f, ic, jc, km) : SlabQ{-1, -1, -1};
        bx_km = bx_of<DIM, PML, false>(g, f, qm, jc, km, __ldg(f.B[0] + om), ezm, ezm_yp, eym, ey);
        by_km = by_of<DIM, PML, false>(g, f, qm, ic, km, __ldg(f.B[1] + om), exm, ex, ezm, ezm_xp);
    }
    for (int k = k0; k < k1; ++k, o += c.pl) {
        if (k + 1 < k1) plane_in<DIM>(g, f, c, o + c.pl, k + 1, jdirty, nxt);
        const float ez = cur.ez;
        // +x neighbours
        float ey_xp = __shfl_down_sync(full, ey, 1);
        float ez_xp = __shfl_down_sync(full, ez, 1);
        float eyym_xp = __shfl_down_sync(full, ey_ym, 1);
        if (c.xp_ld) {
            ey_xp = cur.ey_xp;
            ez_xp = cur.ez_xp;
            eyym_xp = cur.eyym_xp;
        }
        // B^{n+1/2} of the own cell (stored) ...
        const SlabQ q = PML ? slab_q<DIM>(g, f, ic, jc, k) : SlabQ{-1, -1, -1};
        float bx = 0.f, by = 0.f, bz = 0.f;
        if (live) {
            bx = bx_of<DIM, PML, true>(g, f, q, jc, k, cur.bx0, ez, cur.ez_yp, ey, cur.ey_kp);
            by = by_of<DIM, PML, true>(g, f, q, ic, k, cur.by0, ex, cur.ex_kp, ez, ez_xp);
            bz = bz_of<PML, true>(g, f, q, ic, jc, cur.bz0, ey, ey_xp, ex, cur.ex_yp);
            f.Bn[0][o] = bx;
            f.Bn[1][o] = by;
            f.Bn[2][o] = bz;
        }
        // ... of the -y neighbour (recomputed) ...
        float bx_ym = 0.f, bz_ym = 0.f;
        if (c.hym) {
            const SlabQ qy = PML ? slab_q<DIM>(g, f, ic, jm, k) : SlabQ{-1, -1, -1};
            bx_ym = bx_of<DIM, PML, false>(g, f, qy, jm, k, cur.bx0_ym, cur.ez_ym, ez, ey_ym,
                                           cur.eykp_ym);
            bz_ym = bz_of<PML, false>(g, f, qy, ic, jm, cur.bz0_ym, ey_ym, eyym_xp, cur.ex_ym, ex);
        }
        // ... and of the -x neighbour (lane - 1, or recomputed by lane 0)
        float by_xm = __shfl_up_sync(full, by, 1);
        float bz_xm = __shfl_up_sync(full, bz, 1);
        if (lane == 0) {
            by_xm = bz_xm = 0.f;
            if (c.xm_ld) {
                const SlabQ qx = PML ? slab_q<DIM>(g, f, im, jc, k) : SlabQ{-1, -1, -1};
                by_xm = by_of<DIM, PML, false>(g, f, qx, im, k, cur.bym0, cur.exm, cur.exm_kp,
                                               cur.ezm, ez);
                bz_xm = bz_of<PML, false>(g, f, qx, im, jc, cur.bzm0, cur.eym, ey, cur.exm,
                                          cur.exm_yp);
            }
        }
        if (live) {
            float jx = cur.jx, jy = cur.jy, jz = cur.jz;
            if (clearJ) {
                __stcg(f.J[0] + o, 0.f);
                __stcg(f.J[1] + o, 0.f);
                __stcg(f.J[2] + o, 0.f);
            }
            if (f.src_on && (f.inc == 2 ? k : spos) == f.src_index) {
                if (f.pol == 0) jx += src;
                else if (f.pol == 1) jy += src;
                else jz += src;
            }
            float tExy = (bz - bz_ym) * idy;
            float tEzy = (bx - bx_ym) * idy;
            float tEyx = (bz - bz_xm) * idx_;
            float tEzx = (by - by_xm) * idx_;
            float tExz = 0.f, tEyz = 0.f;
            if (DIM == 3) {
                tExz = (by - by_km) * idz;
                tEyz = (bx - bx_km) * idz;
            }
            if (PML) {
                // E memory terms: x slab E_y, E_z (slots 0, 1); y slab E_x, E_z;
                // z slab E_x, E_y
                if (q.qy >= 0) {
                    const float b = __ldg(f.cb_e[1] + jc), cc = __ldg(f.ca_e[1] + jc);
                    tExy = with_psi<true>(tExy, f.psi_in[1][0], f.psi_out[1][0], q.qy, b, cc);
                    tEzy = with_psi<true>(tEzy, f.psi_in[1][1], f.psi_out[1][1], q.qy, b, cc);
                }
                if (q.qx >= 0) {
                    const float b = __ldg(f.cb_e[0] + ic), cc = __ldg(f.ca_e[0] + ic);
                    tEyx = with_psi<true>(tEyx, f.psi_in[0][0], f.psi_out[0][0], q.qx, b, cc);
                    tEzx = with_psi<true>(tEzx, f.psi_in[0][1], f.psi_out[0][1], q.qx, b, cc);
                }
                if (q.qz >= 0) {
                    const float b = __ldg(f.cb_e[2] + k), cc = __ldg(f.ca_e[2] + k);
                    tExz = with_psi<true>(tExz, f.psi_in[2][0], f.psi_out[2][0], q.qz, b, cc);
                    tEyz = with_psi<true>(tEyz, f.psi_in[2][1], f.psi_out[2][1], q.qz, b, cc);
                }
            }
            f.En[0][o] = ex + c2dt * (tExy - tExz) - dte * jx;
            f.En[1][o] = ey + c2dt * (tEyz - tEyx) - dte * jy;
            f.En[2][o] = ez + c2dt * (tEzx - tEzy) - dte * jz;
        }
        bx_km = bx;
        by_km = by;
        ex = cur.ex_kp;
        ey = cur.ey_kp;
        ey_ym = cur.eykp_ym;
        cur = nxt;
    }
    if (jdirty) {
        __syncthreads();
        if (threadIdx.x == 0) f.jdirty_clear[bflag] = 0;
    }
}

}  // namespace

cudaError_t launch_field_stream(const GridP &g, const FieldP &f, cudaStream_t s) {
    dim3 grid((g.n[0] + BX - 1) / BX, (g.n[1] + BY - 1) / BY,
              g.dims == 3 ? (g.n[2] + f.zchunk - 1) / f.zchunk : 1);
    const bool pml = f.pml[0] || f.pml[1] || f.pml[2];
    if (g.dims == 3) {
        field_stream_kernel<3, false><<<grid, BX * BY, 0, s>>>(g, f);
        if (pml) field_stream_kernel<3, true><<<grid, BX * BY, 0, s>>>(g, f);
    } else {
        field_stream_kernel<2, false><<<grid, BX * BY, 0, s>>>(g, f);
        if (pml) field_stream_kernel<2, true><<<grid, BX * BY, 0, s>>>(g, f);
    }
    return cudaGetLastError();
}

}  // namespace pic
