// k_particle_lean.cu -- the particle phase of a 3D step with CIC shapes on
// the default tile of 8 x 8 x 4 cells (and on 16 x 8 x 1, for one-cell
// sheets): the same gather, push, drift and
// Esirkepov deposit as particle_kernel<3> (k_particle.cu; Sec. 4.1 and
// Appendix A of the paper), organised around the common case.
//
//  * The staged box (13 x 13 x 9 nodes per component for 8 x 8 x 4) has
//    compile-time dimensions, so the gather reaches the eight nodes of a component from
//    one base index by constant offsets, and all nine components (E, B^n, J)
//    from one shared-memory base.
//  * Each thread loads its next particle before it works on the current one
//    (the loads of particle p + 256 are in flight during the gather, push
//    and deposit of particle p).
//  * The loop body is the move that stays in its cell (99.7 % of the moves
//    on the nanosphere workload).  A particle whose move crosses a cell face
//    (the reflection at material edges included), or that fails the drift
//    check, is not finished there: its index joins a per-tile list in shared
//    memory and, after the loop, the CTA completes the list with the generic
//    particle code of k_particle.cuh (one item per warp, so that their long
//    dependency chains run side by side).  Nothing of the particle was
//    written in the loop; the generic code gathers and pushes it again from
//    the same box.
//  * A particle outside the tile's core (drifted more than a cell out of its
//    tile since the last re-sort), and the overflow of the shared list, go
//    to a global list that particle_deferred_kernel completes after this
//    kernel with global gathers and global atomics.
//  * The box is staged by asynchronous copies (cp.async), all of a thread's
//    issued before it waits once.
//  * Tiles whose box lies inside the grid stage and flush without the
//    periodic wrap and flag the field blocks under the box as a whole (the
//    flags mean "J may be non-zero there").
#include "k_particle.cuh"

namespace pic {

namespace {

constexpr int LH = kHalo;        // box = local cells [-2, T + 2]
constexpr int kDeferCap = 256;  // per-tile list of crossing moves

// A tile shape of the lean kernel: T0 x T1 x T2 cells, its box B0 x B1 x B2
// nodes (BN per component).  Instantiated for the default 3D tile 8 x 8 x 4
// and for 16 x 8 x 1, the shape of a one-cell sheet (the graphene workload:
// twice the sheet cells of an 8 x 8 x 4 tile under a box of about the same
// size).
template <int A, int B, int C>
struct LeanTile {
    static constexpr int T0 = A, T1 = B, T2 = C;
    static constexpr int B0 = A + 2 * LH + 1, B1 = B + 2 * LH + 1, B2 = C + 2 * LH + 1;
    static constexpr int B01 = B0 * B1, BN = B01 * B2;
};
using TileCube = LeanTile<8, 8, 4>;
using TileSheet = LeanTile<16, 8, 1>;

// the tile constants of TL under the names the kernel code uses
#define LEAN_CONSTS(TL)                                                                     \
    [[maybe_unused]] constexpr int LT0 = TL::T0, LT1 = TL::T1, LT2 = TL::T2;                \
    [[maybe_unused]] constexpr int LB0 = TL::B0, LB1 = TL::B1, LB2 = TL::B2;                \
    [[maybe_unused]] constexpr int LB01 = TL::B01, LBN = TL::BN

template <class TL>
__device__ __forceinline__ int lidx(int x, int y, int z) {
    LEAN_CONSTS(TL);
    return (z + LH) * LB01 + (y + LH) * LB0 + (x + LH);
}

// The box with constant strides, for deposit_nocross_acc / cellj_flush.
template <class TL>
struct LeanBox {
    static constexpr int b0 = TL::B0, b01 = TL::B01;
    struct JRef {
        float *base;
        __device__ __forceinline__ float *operator[](int c) const { return base + (6 + c) * TL::BN; }
    };
    JRef J;
    __device__ __forceinline__ int idx(int x, int y, int z) const { return lidx<TL>(x, y, z); }
};

// Trilinear interpolation over the eight nodes from p (node (0, 0, 0)) with
// the weights x1, y1, z1 of the upper nodes; the same association as
// interp() of the generic kernel.
template <class TL>
__device__ __forceinline__ float tri(const float *p, float x1, float y1, float z1) {
    LEAN_CONSTS(TL);
    const float x0 = 1.f - x1, y0 = 1.f - y1, z0 = 1.f - z1;
    const float a0 = y0 * (x0 * p[0] + x1 * p[1]) + y1 * (x0 * p[LB0] + x1 * p[LB0 + 1]);
    const float a1 = y0 * (x0 * p[LB01] + x1 * p[LB01 + 1]) +
                     y1 * (x0 * p[LB01 + LB0] + x1 * p[LB01 + LB0 + 1]);
    return z0 * a0 + z1 * a1;
}

// CIC gather of E^n, B^n on the Yee stagger (as gather<3>): integer-staggered
// axes take the node l with the weight f of node l + 1; half-staggered ones
// the node m + 1/2 below the particle, m = l (weight f - 1/2) when f >= 1/2,
// else m = l - 1 (weight f + 1/2).
template <class TL>
__device__ __forceinline__ void lean_gather(const float *sm, const int *lc, const float *f,
                                            float *E, float *B) {
    LEAN_CONSTS(TL);
    const int e = lidx<TL>(lc[0], lc[1], lc[2]);
    float wh[3];
    int oh[3];
    const int step[3] = {1, LB0, LB01};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float u = f[a] - 0.5f;
        const bool up = u >= 0.f;
        wh[a] = up ? u : u + 1.0f;
        oh[a] = up ? 0 : -step[a];
    }
    E[0] = tri<TL>(sm + 0 * LBN + e + oh[0], wh[0], f[1], f[2]);
    E[1] = tri<TL>(sm + 1 * LBN + e + oh[1], f[0], wh[1], f[2]);
    E[2] = tri<TL>(sm + 2 * LBN + e + oh[2], f[0], f[1], wh[2]);
    B[0] = tri<TL>(sm + 3 * LBN + e + oh[1] + oh[2], f[0], wh[1], wh[2]);
    B[1] = tri<TL>(sm + 4 * LBN + e + oh[0] + oh[2], wh[0], f[1], wh[2]);
    B[2] = tri<TL>(sm + 5 * LBN + e + oh[0] + oh[1], wh[0], wh[1], f[2]);
}

// the core of the box: local cells [-1, T] on every axis (as in_core<3>)
template <class TL>
__device__ __forceinline__ bool lean_core(const int *c) {
    LEAN_CONSTS(TL);
    return c[0] >= -1 && c[0] <= LT0 && c[1] >= -1 && c[1] <= LT1 && c[2] >= -1 && c[2] <= LT2;
}

enum : int { kDone = 0, kDeferTile = 1, kDeferGlobal = 2 };



// Free electron or Dirac carrier whose move stays in its cell: gather, push,
// drift, deposit into the register sum, store.  Anything else is deferred
// with nothing written.
struct MobIn {
    uint32_t pc;
    float o[3], v[3];
};
__device__ __forceinline__ void load_mob(const SpeciesP &s, int p, MobIn &m) {
    m.pc = s.cell[p];
    m.o[0] = s.o[0][p];
    m.o[1] = s.o[1][p];
    m.o[2] = s.o[2][p];
    m.v[0] = s.v[0][p];
    m.v[1] = s.v[1][p];
    m.v[2] = s.v[2][p];
}
template <class TL>
__device__ __forceinline__ int lean_mobile(const ParticleLaunch &P, const SpeciesP &s, bool dirac,
                                           int p, const MobIn &m, const int *org, float *sm,
                                           CellJ &acc) {
    LEAN_CONSTS(TL);
    const uint32_t pc = m.pc;
    const int gc[3] = {cell_x(pc), cell_y(pc), cell_z(pc)};
    int lc[3];
    local_cell<3>(P, gc, org, lc);
    if (!lean_core<TL>(lc)) return kDeferGlobal;
    float v[3] = {m.v[0], m.v[1], m.v[2]};
    const float f0[3] = {m.o[0], m.o[1], m.o[2]};
    float E[3], B[3];
    lean_gather<TL>(sm, lc, f0, E, B);
    if (dirac) dirac_push(v, E, B, s);
    else boris(v, E, B, s.hq);
    float f1[3], dF[3];
    bool stay = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dF[a] = s.dtd[a] * v[a];  // the move in cells, which the current takes (as push_mobile)
        f1[a] = f0[a] + dF[a];
        stay = stay && f1[a] >= 0.f && f1[a] < 1.f;
    }
    if (!stay) return kDeferTile;
    LeanBox<TL> box{{sm}};
    deposit_nocross_acc<3>(box, lc, f0, dF, s.jfac, v[2], acc);
    s.o[0][p] = f1[0];
    s.o[1][p] = f1[1];
    s.o[2][p] = f1[2];
    s.v[0][p] = v[0];
    s.v[1][p] = v[1];
    s.v[2][p] = v[2];
    return kDone;
}

// Bound electron (isotropic damping) whose move stays in its cell (as
// push_bound<3, false>).
struct BndIn {
    uint32_t pc;
    float an[3], D[3], v[3];
};
__device__ __forceinline__ void load_bnd(const SpeciesP &s, int p, BndIn &m) {
    m.pc = s.cell[p];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        m.an[a] = s.anchor32[a][p];
        m.D[a] = s.disp[a][p];
        m.v[a] = s.v[a][p];
    }
}
template <class TL>
__device__ __forceinline__ int lean_bound(const ParticleLaunch &P, const SpeciesP &s, int p,
                                          const BndIn &m, const int *org, float *sm, CellJ &acc) {
    LEAN_CONSTS(TL);
    const GridP &g = P.g;
    const uint32_t pc = m.pc;
    const int gc[3] = {cell_x(pc), cell_y(pc), cell_z(pc)};
    int lc[3];
    local_cell<3>(P, gc, org, lc);
    float D[3] = {m.D[0], m.D[1], m.D[2]};
    int c0[3];
    float f0[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float xa = m.an[a] + D[a] * g.inv_d[a];
        const float fl = floorf(xa);
        c0[a] = lc[a] + (int)fl;
        f0[a] = clamp_below_one(xa - fl);
    }
    if (!lean_core<TL>(c0)) return kDeferGlobal;
    float v[3] = {m.v[0], m.v[1], m.v[2]};
    float E[3], B[3];
    lean_gather<TL>(sm, c0, f0, E, B);
    bound_push<false>(v, D, E, B, s);
    float dF[3];
    bool stay = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dF[a] = s.dt * v[a] * g.inv_d[a];
        const float x = f0[a] + dF[a];
        stay = stay && x >= 0.f && x < 1.f;
    }
    if (!stay) return kDeferTile;
    LeanBox<TL> box{{sm}};
    deposit_nocross_acc<3>(box, c0, f0, dF, s.jfac, v[2], acc);
    s.disp[0][p] = D[0];
    s.disp[1][p] = D[1];
    s.disp[2][p] = D[2];
    s.v[0][p] = v[0];
    s.v[1][p] = v[1];
    s.v[2][p] = v[2];
    return kDone;
}

__device__ __forceinline__ void lean_defer(const ParticleLaunch &P, int code, int si, int p,
                                           int2 *s_def, int *s_ndef) {
    if (code == kDeferTile) {
        const int k = atomicAdd(s_ndef, 1);
        if (k < kDeferCap) {
            s_def[k] = make_int2(si, p);
            return;
        }
    }
    const int k = atomicAdd(P.defer_count, 1);
    P.defer[k] = make_int2(si, p);
}

// global index of box node (bx, by, bz) of a tile at org; -1 outside a
// non-periodic edge
__device__ __forceinline__ long long lean_node(const GridP &g, const int *org, int bx, int by,
                                               int bz) {
    const int gx = wrap_or_neg(org[0] + bx - LH, g.n[0], g.per[0]);
    const int gy = wrap_or_neg(org[1] + by - LH, g.n[1], g.per[1]);
    const int gz = wrap_or_neg(org[2] + bz - LH, g.n[2], g.per[2]);
    if (gx < 0 || gy < 0 || gz < 0) return -1;
    return ((long long)gz * g.n[1] + gy) * g.n[0] + gx;
}

// Box element e -> (bx, by, bz) with constant box dims, advanced by the CTA
// width.
template <class TL>
struct LeanWalk {
    static constexpr int LB0 = TL::B0, LB1 = TL::B1, LB01 = TL::B01;
    int bx, by, bz, e;
    static constexpr int kDz = kThreads / LB01, kDy = (kThreads - kDz * LB01) / LB0,
                         kDx = kThreads - kDz * LB01 - kDy * LB0;
    __device__ __forceinline__ void start(int e0) {
        e = e0;
        bz = e0 / LB01;
        by = (e0 - bz * LB01) / LB0;
        bx = e0 - bz * LB01 - by * LB0;
    }
    __device__ __forceinline__ void next() {
        e += kThreads;
        bx += kDx;
        by += kDy;
        bz += kDz;
        if (bx >= LB0) { bx -= LB0; ++by; }
        if (by >= LB1) { by -= LB1; ++bz; }
    }
};

template <class TL>
__device__ void lean_tile(const ParticleLaunch &P, const int t, float *sm, unsigned *s_refl,
                          int2 *s_def, int *s_ndef) {
    LEAN_CONSTS(TL);
    const TileP &tp = P.tp;
    const GridP &g = P.g;
    const float hdt = 0.5f * g.dt;
    const int tx = t % tp.nt[0], ty = (t / tp.nt[0]) % tp.nt[1], tz = t / (tp.nt[0] * tp.nt[1]);
    const int org[3] = {tx * LT0, ty * LT1, tz * LT2};
    // the box lies inside the grid: no wrap, no edge
    const bool inner = org[0] >= LH && org[0] + LT0 + LH < g.n[0] && org[1] >= LH &&
                       org[1] + LT1 + LH < g.n[1] && org[2] >= LH && org[2] + LT2 + LH < g.n[2];
    const int nx = g.n[0];
    const int plane = g.n[0] * g.n[1];
    const long long base =
        ((long long)(org[2] - LH) * g.n[1] + (org[1] - LH)) * g.n[0] + (org[0] - LH);
    __syncthreads();  // the previous tile's flush is done with the box and the list
    if (threadIdx.x == 0) *s_ndef = 0;
    // stage E^n, B^{n-1/2}; zero J
    {
        LeanWalk<TL> w;
        for (w.start(threadIdx.x); w.e < LBN; w.next()) {
            long long o;
            if (inner) o = base + (long long)(w.bz * plane + w.by * nx + w.bx);
            else o = lean_node(g, org, w.bx, w.by, w.bz);
            const bool in = o >= 0;
            if (!in) o = 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                cp_async4(&sm[c * LBN + w.e], P.E[c] + o, in);
                cp_async4(&sm[(3 + c) * LBN + w.e], P.B[c] + o, in);
                sm[(6 + c) * LBN + w.e] = 0.f;
            }
        }
        cp_async_wait_all();
    }
    __syncthreads();
    // B^n = B^{n-1/2} - (dt/2) curl E^n on every node a gather can reach
    {
        LeanWalk<TL> w;
        for (w.start(threadIdx.x); w.e < LBN; w.next()) {
            const int e = w.e;
            if (w.bx + 1 >= LB0 || w.by + 1 >= LB1 || w.bz + 1 >= LB2) continue;  // never gathered
            if (!inner && lean_node(g, org, w.bx, w.by, w.bz) < 0) {
                sm[3 * LBN + e] = sm[4 * LBN + e] = sm[5 * LBN + e] = 0.f;
                continue;
            }
            const float *Ex = sm, *Ey = sm + LBN, *Ez = sm + 2 * LBN;
            const float dEz_dy = (Ez[e + LB0] - Ez[e]) * g.inv_d[1];
            const float dEx_dy = (Ex[e + LB0] - Ex[e]) * g.inv_d[1];
            const float dEz_dx = (Ez[e + 1] - Ez[e]) * g.inv_d[0];
            const float dEy_dx = (Ey[e + 1] - Ey[e]) * g.inv_d[0];
            const float dEy_dz = (Ey[e + LB01] - Ey[e]) * g.inv_d[2];
            const float dEx_dz = (Ex[e + LB01] - Ex[e]) * g.inv_d[2];
            sm[3 * LBN + e] -= hdt * (dEz_dy - dEy_dz);
            sm[4 * LBN + e] -= hdt * (dEx_dz - dEz_dx);
            sm[5 * LBN + e] -= hdt * (dEy_dx - dEx_dy);
        }
    }
    __syncthreads();
    CellJ acc;
    acc.e = -1;
    for (int si = 0; si < P.nsp; ++si) {
        const SpeciesP &s = P.sp[si];
        const int a = s.tile_start[t], b = s.tile_start[t + 1];
        if (s.kind == PIC_BOUND) {
            BndIn nxt;
            int p = a + threadIdx.x;
            if (p < b) load_bnd(s, p, nxt);
            for (; p < b; p += kThreads) {
                const BndIn cur = nxt;
                if (p + kThreads < b) load_bnd(s, p + kThreads, nxt);
                const int r = lean_bound<TL>(P, s, p, cur, org, sm, acc);
                if (r != kDone) lean_defer(P, r, si, p, s_def, s_ndef);
            }
        } else {
            const bool dirac = s.kind == PIC_DIRAC;
            MobIn nxt;
            int p = a + threadIdx.x;
            if (p < b) load_mob(s, p, nxt);
            for (; p < b; p += kThreads) {
                const MobIn cur = nxt;
                if (p + kThreads < b) load_mob(s, p + kThreads, nxt);
                const int r = lean_mobile<TL>(P, s, dirac, p, cur, org, sm, acc);
                if (r != kDone) lean_defer(P, r, si, p, s_def, s_ndef);
            }
        }
    }
    {
        LeanBox<TL> box{{sm}};
        cellj_flush<3>(box, acc);
    }
    __syncthreads();
    // the crossing moves of this tile, with the generic code on the same box
    const int nd = min(*s_ndef, kDeferCap);
    if (nd > 0) {
        BoxAcc box;
        for (int c = 0; c < 6; ++c) box.F[c] = sm + c * LBN;
        for (int c = 0; c < 3; ++c) box.J[c] = sm + (6 + c) * LBN;
        box.b0 = LB0;
        box.b01 = LB01;
        box.hz = LH;
        GlobalAcc<3, false> glob;
        glob.g = &P.g;
        glob.E = P.E;
        glob.B = P.B;
        glob.Eext = P.Eext;
        glob.J = P.J;
        glob.jdirty = P.jdirty;
        glob.nbx = P.nbx;
        glob.nby = P.nby;
        glob.zchunk = P.zchunk;
        CellJ unused;
        unused.e = -1;
        // item i to lane i / 8 of warp i % 8: the few items run on separate warps
        for (int i = (threadIdx.x & 31) * (kThreads / 32) + (threadIdx.x >> 5); i < nd; i += kThreads) {
            const int2 d = s_def[i];
            const SpeciesP &s = P.sp[d.x];
            if (s.kind == PIC_BOUND) {
                push_bound<3, false>(P, s, d.y, org, box, glob, unused);
            } else if (push_mobile<3, false>(P, s, d.x, s.kind == PIC_DIRAC, d.y, org, box, glob,
                                             unused)) {
                atomicAdd(&s_refl[d.x], 1u);
            }
        }
        __syncthreads();
    }
    // flush the J box
    if (inner) {
        LeanWalk<TL> w;
        for (w.start(threadIdx.x); w.e < LBN; w.next()) {
            const int e = w.e;
            const float jx = sm[6 * LBN + e], jy = sm[7 * LBN + e], jz = sm[8 * LBN + e];
            const long long o = base + (long long)(w.bz * plane + w.by * nx + w.bx);
            if (jx != 0.f) atomicAdd(P.J[0] + o, jx);
            if (jy != 0.f) atomicAdd(P.J[1] + o, jy);
            if (jz != 0.f) atomicAdd(P.J[2] + o, jz);
        }
        // flag the field blocks under the box (at most 2 x 3 x 2)
        const int x0 = (org[0] - LH) / kFieldBX, x1 = (org[0] + LT0 + LH) / kFieldBX;
        const int y0 = (org[1] - LH) / kFieldBY, y1 = (org[1] + LT1 + LH) / kFieldBY;
        const int z0 = (org[2] - LH) / P.zchunk, z1 = (org[2] + LT2 + LH) / P.zchunk;
        const int nbx = x1 - x0 + 1, nby = y1 - y0 + 1, nbz = z1 - z0 + 1;
        const int q = threadIdx.x;
        if (q < nbx * nby * nbz) {
            const int bx = x0 + q % nbx, by = y0 + (q / nbx) % nby, bz = z0 + q / (nbx * nby);
            P.jdirty[((long long)bz * P.nby + by) * P.nbx + bx] = 1;
        }
    } else {
        const int lane = threadIdx.x & 31;
        LeanWalk<TL> w;
        w.start(threadIdx.x);
        for (int e0 = 0; e0 < LBN; e0 += kThreads, w.next()) {
            long long blk = -1;
            if (w.e < LBN) {
                const int e = w.e;
                const float jx = sm[6 * LBN + e], jy = sm[7 * LBN + e], jz = sm[8 * LBN + e];
                if (jx != 0.f || jy != 0.f || jz != 0.f) {
                    const int gx = wrap_or_neg(org[0] + w.bx - LH, g.n[0], g.per[0]);
                    const int gy = wrap_or_neg(org[1] + w.by - LH, g.n[1], g.per[1]);
                    const int gz = wrap_or_neg(org[2] + w.bz - LH, g.n[2], g.per[2]);
                    if (gx >= 0 && gy >= 0 && gz >= 0) {
                        const long long o = ((long long)gz * g.n[1] + gy) * g.n[0] + gx;
                        if (jx != 0.f) atomicAdd(P.J[0] + o, jx);
                        if (jy != 0.f) atomicAdd(P.J[1] + o, jy);
                        if (jz != 0.f) atomicAdd(P.J[2] + o, jz);
                        blk = ((long long)(gz / P.zchunk) * P.nby + gy / kFieldBY) * P.nbx +
                              gx / kFieldBX;
                    }
                }
            }
            const unsigned same = __match_any_sync(0xffffffffu, blk);
            if (blk >= 0 && lane == __ffs(same) - 1) P.jdirty[blk] = 1;
        }
    }
}

}  // namespace

// Resident CTAs per SM the lean kernel's registers are sized for (as the
// plain kernel's: three beside the B pass).
template <class TL>
__global__ void __launch_bounds__(kThreads, 3) particle_kernel_lean(ParticleLaunch P) {
    extern __shared__ float smem[];
    __shared__ unsigned s_refl[kMaxSpecies];
    __shared__ int2 s_def[kDeferCap];
    __shared__ int s_ndef, s_next;
    if (threadIdx.x < kMaxSpecies) s_refl[threadIdx.x] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && P.step_counter) *P.step_counter += 1;
    const int nact = *P.nactive;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(&P.sched[0], 1);
        __syncthreads();
        const int it = s_next;
        if (it >= nact) break;
        lean_tile<TL>(P, P.active[it], smem, s_refl, s_def, &s_ndef);
    }
    __syncthreads();
    if (threadIdx.x < P.nsp && s_refl[threadIdx.x])
        atomicAdd(P.sp[threadIdx.x].nrefl, (unsigned long long)s_refl[threadIdx.x]);
    if (threadIdx.x == 0) {
        // the last CTA to finish resets the tile counters for the next launch
        __threadfence();
        if (atomicAdd(&P.sched[1], 1) == (int)gridDim.x - 1) {
            P.sched[0] = 0;
            P.sched[1] = 0;
        }
    }
}

// The particles the lean kernel deferred to the global list: the generic
// particle code with global gathers (B^n formed from E^n and B^{n-1/2} at
// the particle) and global atomics.  The last CTA resets the list.
__global__ void __launch_bounds__(kThreads) particle_deferred_kernel(ParticleLaunch P) {
    const int n = *P.defer_count;
    GlobalAcc<3, false> glob;
    glob.g = &P.g;
    glob.E = P.E;
    glob.B = P.B;
    glob.Eext = P.Eext;
    glob.J = P.J;
    glob.jdirty = P.jdirty;
    glob.nbx = P.nbx;
    glob.nby = P.nby;
    glob.zchunk = P.zchunk;
    BoxAcc none{};
    CellJ unused;
    unused.e = -1;
    const int org[3] = {0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int2 d = P.defer[i];
        const SpeciesP &s = P.sp[d.x];
        if (s.kind == PIC_BOUND) {
            push_bound<3, false, false, BoxAcc, true>(P, s, d.y, org, none, glob, unused);
        } else if (push_mobile<3, false, 1, false, BoxAcc, true>(P, s, d.x, s.kind == PIC_DIRAC,
                                                                 d.y, org, none, glob, unused)) {
            atomicAdd(s.nrefl, 1ull);
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(P.defer_sched, 1) == (int)gridDim.x - 1) {
            *P.defer_count = 0;
            *P.defer_sched = 0;
        }
    }
}

template <class TL>
bool lean_tile_is(const TileP &tp) {
    return tp.T[0] == TL::T0 && tp.T[1] == TL::T1 && tp.T[2] == TL::T2;
}

bool particle_lean_fits(const ParticleLaunch &pl) {
    return pl.g.dims == 3 && pl.shape == 1 &&
           (lean_tile_is<TileCube>(pl.tp) || lean_tile_is<TileSheet>(pl.tp)) &&
           pl.defer != nullptr && !particle_launch_ext(pl);
}

cudaError_t particle_lean_setup() {
    cudaError_t e = allow_max_dynamic_smem(particle_kernel_lean<TileCube>);
    if (e != cudaSuccess) return e;
    return allow_max_dynamic_smem(particle_kernel_lean<TileSheet>);
}

cudaError_t launch_particles_lean(const ParticleLaunch &pl, int nctas, int ndefer_ctas,
                                  cudaStream_t s) {
    if (nctas < 1) nctas = 1;
    if (ndefer_ctas < 1) ndefer_ctas = 1;
    if (lean_tile_is<TileSheet>(pl.tp))
        particle_kernel_lean<TileSheet>
            <<<nctas, kThreads, (size_t)9 * TileSheet::BN * sizeof(float), s>>>(pl);
    else
        particle_kernel_lean<TileCube>
            <<<nctas, kThreads, (size_t)9 * TileCube::BN * sizeof(float), s>>>(pl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    particle_deferred_kernel<<<ndefer_ctas, kThreads, 0, s>>>(pl);
    return cudaGetLastError();
}

}  // namespace pic
