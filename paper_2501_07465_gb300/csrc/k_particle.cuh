// k_particle.cuh -- device code of the particle phase (see k_particle.cu),
// shared by the translation units that instantiate it: k_particle.cu (the
// plain kernels and the batch kernel), k_particle_ext.cu (the kernels with
// the boundary variants of Sec. 3) and k_particle_tsc.cu (TSC shapes for
// the free and Dirac particles), compiled in parallel.
#pragma once

#include "pic_internal.cuh"

namespace pic {

namespace {

constexpr int kThreads = kParticleThreads;  // the chunk of the cell-interleaved order
constexpr int kHalo = 2;  // box covers local cells [-2, T+2]

__device__ inline float clamp_below_one(float f) {
    return f < 1.0f ? f : 0x1.fffffep-1f;
}

// 4-byte asynchronous copy global -> shared (zero-filled when !valid); the
// staging issues the whole box before it waits once
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

__device__ inline int wrap_or_neg(int i, int n, int per) {
    if (i >= 0 && i < n) return i;
    if (!per) return -1;
    int r = i % n;
    return r < 0 ? r + n : r;
}

// ---------------------------------------------------------------------------
// field access: shared-memory box (fast path) or global memory (slow path)
// ---------------------------------------------------------------------------

// Components: 0..2 E, 3..5 B^n.  Coordinates are "local" integers: box
// coordinates (local cell + 2) for the box, global cell indices (possibly
// outside [0,n)) for the global accessor.
// H: halo of the box in cells (2; 3 for the TSC kernel, whose three-node
// gather and four-node deposit reach one node further)
template <int H>
struct BoxAccT {
    float *F[6];
    float *J[3];
    int b0, b01;
    int hz;  // halo along z: H in 3D, 0 in 2D
    // local cell coordinates (relative to the tile origin) -> box index
    __device__ inline int idx(int x, int y, int z) const {
        return (z + hz) * b01 + (y + H) * b0 + (x + H);
    }
    __device__ inline float get(int c, int x, int y, int z) const { return F[c][idx(x, y, z)]; }
    __device__ inline void add(int c, int x, int y, int z, float v) const {
        atomicAdd(&J[c][idx(x, y, z)], v);
    }
};
using BoxAcc = BoxAccT<kHalo>;

template <int DIM, bool X>
struct GlobalAcc {
    const GridP *g;
    const float *const *E;
    const float *const *B;
    const float *const *Eext;  // external field (X only), Eext[0] null: none
    float *const *J;
    uint8_t *jdirty;
    int nbx, nby, zchunk;
    __device__ inline long long off(int x, int y, int z) const {
        int gx = wrap_or_neg(x, g->n[0], g->per[0]);
        int gy = wrap_or_neg(y, g->n[1], g->per[1]);
        int gz = DIM == 3 ? wrap_or_neg(z, g->n[2], g->per[2]) : 0;
        if (gx < 0 || gy < 0 || gz < 0) return -1;
        return ((long long)gz * g->n[1] + gy) * g->n[0] + gx;
    }
    __device__ inline float e(int c, int x, int y, int z) const {
        long long o = off(x, y, z);
        return o < 0 ? 0.f : __ldg(E[c] + o);
    }
    __device__ inline float get(int c, int x, int y, int z) const {
        if (c < 3) {
            if (X && Eext[0]) {
                // the particles see E^n plus the external field (Sec. 3);
                // the curl below takes the Maxwell E alone
                long long o = off(x, y, z);
                return o < 0 ? 0.f : __ldg(E[c] + o) + __ldg(Eext[c] + o);
            }
            return e(c, x, y, z);
        }
        long long o = off(x, y, z);
        if (o < 0) return 0.f;
        const float h = 0.5f * g->dt;
        float b = __ldg(B[c - 3] + o);
        if (c == 3) {
            float dEz_dy = (e(2, x, y + 1, z) - e(2, x, y, z)) * g->inv_d[1];
            float dEy_dz = DIM == 3 ? (e(1, x, y, z + 1) - e(1, x, y, z)) * g->inv_d[2] : 0.f;
            return b - h * (dEz_dy - dEy_dz);
        } else if (c == 4) {
            float dEx_dz = DIM == 3 ? (e(0, x, y, z + 1) - e(0, x, y, z)) * g->inv_d[2] : 0.f;
            float dEz_dx = (e(2, x + 1, y, z) - e(2, x, y, z)) * g->inv_d[0];
            return b - h * (dEx_dz - dEz_dx);
        } else {
            float dEy_dx = (e(1, x + 1, y, z) - e(1, x, y, z)) * g->inv_d[0];
            float dEx_dy = (e(0, x, y + 1, z) - e(0, x, y, z)) * g->inv_d[1];
            return b - h * (dEy_dx - dEx_dy);
        }
    }
    // (the flagged block from the wrapped coordinates, not by dividing the
    // offset: a form that skipped off() made the compiler copy the whole
    // launch block to local memory in the boundary-variant kernel, 2.5 KB a
    // thread, and doubled its time)
    __device__ inline void add(int c, int x, int y, int z, float v) const {
        long long o = off(x, y, z);
        if (o < 0) return;  // deposits beyond a wall are dropped
        atomicAdd(J[c] + o, v);
        const int gx = wrap_or_neg(x, g->n[0], g->per[0]);
        const int gy = wrap_or_neg(y, g->n[1], g->per[1]);
        const int gz = DIM == 3 ? wrap_or_neg(z, g->n[2], g->per[2]) : 0;
        const int bz = DIM == 3 ? gz / zchunk : 0;
        jdirty[((long long)bz * nby + gy / kFieldBY) * nbx + gx / kFieldBX] = 1;
    }
};

// ---------------------------------------------------------------------------
// CIC gather on the Yee stagger
// ---------------------------------------------------------------------------

// Per axis: integer-staggered nodes (base, weight of base+1) and
// half-staggered nodes.
struct AxisW {
    int bi, bh;
    float wi, wh;
};

__device__ inline AxisW axis_weights(int l, float f) {
    AxisW a;
    a.bi = l;
    a.wi = f;
    float u = f - 0.5f;
    if (u >= 0.f) {
        a.bh = l;
        a.wh = u;
    } else {
        a.bh = l - 1;
        a.wh = u + 1.0f;
    }
    return a;
}

template <int DIM, class Acc>
__device__ inline float interp(const Acc &A, int c, const AxisW *w, bool hx, bool hy, bool hz) {
    int bx = hx ? w[0].bh : w[0].bi, by = hy ? w[1].bh : w[1].bi;
    float x1 = hx ? w[0].wh : w[0].wi, y1 = hy ? w[1].wh : w[1].wi;
    float x0 = 1.f - x1, y0 = 1.f - y1;
    if (DIM == 2) {
        return y0 * (x0 * A.get(c, bx, by, 0) + x1 * A.get(c, bx + 1, by, 0)) +
               y1 * (x0 * A.get(c, bx, by + 1, 0) + x1 * A.get(c, bx + 1, by + 1, 0));
    }
    int bz = hz ? w[2].bh : w[2].bi;
    float z1 = hz ? w[2].wh : w[2].wi, z0 = 1.f - z1;
    float a0 = y0 * (x0 * A.get(c, bx, by, bz) + x1 * A.get(c, bx + 1, by, bz)) +
               y1 * (x0 * A.get(c, bx, by + 1, bz) + x1 * A.get(c, bx + 1, by + 1, bz));
    float a1 = y0 * (x0 * A.get(c, bx, by, bz + 1) + x1 * A.get(c, bx + 1, by, bz + 1)) +
               y1 * (x0 * A.get(c, bx, by + 1, bz + 1) + x1 * A.get(c, bx + 1, by + 1, bz + 1));
    return z0 * a0 + z1 * a1;
}

// E^n, B^n at a particle in cell (l[0..2]) with offsets f[0..2].
template <int DIM, class Acc>
__device__ inline void gather(const Acc &A, const int *l, const float *f, float *E, float *B) {
    AxisW w[3];
    w[0] = axis_weights(l[0], f[0]);
    w[1] = axis_weights(l[1], f[1]);
    w[2] = axis_weights(DIM == 3 ? l[2] : 0, DIM == 3 ? f[2] : 0.f);
    E[0] = interp<DIM>(A, 0, w, true, false, false);
    E[1] = interp<DIM>(A, 1, w, false, true, false);
    E[2] = interp<DIM>(A, 2, w, false, false, true);
    B[0] = interp<DIM>(A, 3, w, false, true, true);
    B[1] = interp<DIM>(A, 4, w, true, false, true);
    B[2] = interp<DIM>(A, 5, w, true, true, false);
}

// ---------------------------------------------------------------------------
// TSC (order 2) gather: three nodes per axis around the nearest one
// ---------------------------------------------------------------------------

// First node n and the three weights for an offset x in [-1/2, 1/2) from
// the nearest node n + 1: (1/2 - x)^2 / 2, 3/4 - x^2, (1/2 + x)^2 / 2.
struct AxisT {
    int n;
    float w[3];
};

__device__ inline AxisT tsc_axis(int nearest, float x) {
    AxisT a;
    a.n = nearest - 1;
    const float l = 0.5f - x, r = 0.5f + x;
    a.w[0] = 0.5f * l * l;
    a.w[1] = 0.75f - x * x;
    a.w[2] = 0.5f * r * r;
    return a;
}

// integer-staggered nodes: nearest of l + f; half-staggered (at m + 1/2): m = l
__device__ inline AxisT tsc_int(int l, float f) {
    return f >= 0.5f ? tsc_axis(l + 1, f - 1.f) : tsc_axis(l, f);
}
__device__ inline AxisT tsc_half(int l, float f) { return tsc_axis(l, f - 0.5f); }

template <int DIM, class Acc>
__device__ inline float interp_tsc(const Acc &A, int c, const AxisT &ax, const AxisT &ay,
                                   const AxisT &az) {
    float acc = 0.f;
    const int kn = DIM == 3 ? 3 : 1;
#pragma unroll
    for (int k = 0; k < kn; ++k) {
        float pl = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int z = DIM == 3 ? az.n + k : 0;
            const float row = ax.w[0] * A.get(c, ax.n, ay.n + j, z) +
                              ax.w[1] * A.get(c, ax.n + 1, ay.n + j, z) +
                              ax.w[2] * A.get(c, ax.n + 2, ay.n + j, z);
            pl += ay.w[j] * row;
        }
        acc += DIM == 3 ? az.w[k] * pl : pl;
    }
    return acc;
}

// E^n, B^n at a particle with TSC weights on each component's stagger.
template <int DIM, class Acc>
__device__ inline void gather_tsc(const Acc &A, const int *l, const float *f, float *E,
                                  float *B) {
    const AxisT ix = tsc_int(l[0], f[0]), hx = tsc_half(l[0], f[0]);
    const AxisT iy = tsc_int(l[1], f[1]), hy = tsc_half(l[1], f[1]);
    const AxisT iz = DIM == 3 ? tsc_int(l[2], f[2]) : ix;
    const AxisT hz = DIM == 3 ? tsc_half(l[2], f[2]) : ix;
    E[0] = interp_tsc<DIM>(A, 0, hx, iy, iz);
    E[1] = interp_tsc<DIM>(A, 1, ix, hy, iz);
    E[2] = interp_tsc<DIM>(A, 2, ix, iy, hz);
    B[0] = interp_tsc<DIM>(A, 3, ix, hy, hz);
    B[1] = interp_tsc<DIM>(A, 4, hx, iy, hz);
    B[2] = interp_tsc<DIM>(A, 5, hx, hy, iz);
}

// Change of the three TSC weights around one nearest node for a move from
// offset x by d (x and x + d within [-1/2, 1/2]), without cancellation:
// -d (1/2 - x - d/2), -d (2x + d), d (1/2 + x + d/2) (they sum to zero).
__device__ inline void tsc_delta(float x, float d, float *o) {
    o[0] = -d * (0.5f - x - 0.5f * d);
    o[1] = -d * (2.f * x + d);
    o[2] = d * (0.5f + x + 0.5f * d);
}

// Esirkepov deposit with TSC shapes for a move from cell c0 + offset f0 to
// cell c1 + offset f1 (less than one cell per axis): on each axis the start
// and end shapes live on the four nodes lo .. lo + 3, lo = min(nearest) - 1;
// the weight changes DS are formed from the displacement (a move that
// changes the nearest node is split at the half-integer point between the
// two), so a small move keeps its relative precision in FP32.  W as in the
// CIC deposit, and J_a at face i + 1/2 is the running sum of W_a along a up
// to node i (the flux through the last face is zero).
template <int DIM, class Acc>
__device__ inline void deposit_tsc(const Acc &A, const int *c0, const float *f0, const int *c1,
                                   const float *f1, const float *jfac, float vz) {
    int lo[3] = {0, 0, 0};
    float S0[3][4] = {}, DS[3][4] = {};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const bool u0 = f0[a] >= 0.5f, u1 = f1[a] >= 0.5f;
        const int n0 = c0[a] + (u0 ? 1 : 0), n1 = c1[a] + (u1 ? 1 : 0);
        const float x0 = u0 ? f0[a] - 1.f : f0[a];
        const float x1 = u1 ? f1[a] - 1.f : f1[a];
        const AxisT t0 = tsc_axis(n0, x0);
        float da[3], db[3];
        if (n1 == n0) {
            lo[a] = n0 - 1;
            tsc_delta(x0, x1 - x0, da);
            S0[a][0] = t0.w[0]; S0[a][1] = t0.w[1]; S0[a][2] = t0.w[2]; S0[a][3] = 0.f;
            DS[a][0] = da[0]; DS[a][1] = da[1]; DS[a][2] = da[2]; DS[a][3] = 0.f;
        } else if (n1 > n0) {
            // up to the point n0 + 1/2, then on around n0 + 1
            lo[a] = n0 - 1;
            tsc_delta(x0, 0.5f - x0, da);
            tsc_delta(-0.5f, x1 + 0.5f, db);
            S0[a][0] = t0.w[0]; S0[a][1] = t0.w[1]; S0[a][2] = t0.w[2]; S0[a][3] = 0.f;
            DS[a][0] = da[0]; DS[a][1] = da[1] + db[0]; DS[a][2] = da[2] + db[1];
            DS[a][3] = db[2];
        } else {
            // down to the point n0 - 1/2, then on around n0 - 1
            lo[a] = n0 - 2;
            tsc_delta(x0, -0.5f - x0, da);
            tsc_delta(0.5f, x1 - 0.5f, db);
            S0[a][0] = 0.f; S0[a][1] = t0.w[0]; S0[a][2] = t0.w[1]; S0[a][3] = t0.w[2];
            DS[a][0] = db[0]; DS[a][1] = db[1] + da[0]; DS[a][2] = db[2] + da[1];
            DS[a][3] = da[2];
        }
    }
    const float third = 1.0f / 3.0f;
    if (DIM == 3) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float run = 0.f;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    run += DS[0][i] * (S0[1][j] * S0[2][k] + 0.5f * DS[1][j] * S0[2][k] +
                                       0.5f * S0[1][j] * DS[2][k] + DS[1][j] * DS[2][k] * third);
                    if (run != 0.f) A.add(0, lo[0] + i, lo[1] + j, lo[2] + k, jfac[0] * run);
                }
            }
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float run = 0.f;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    run += DS[1][j] * (S0[0][i] * S0[2][k] + 0.5f * DS[0][i] * S0[2][k] +
                                       0.5f * S0[0][i] * DS[2][k] + DS[0][i] * DS[2][k] * third);
                    if (run != 0.f) A.add(1, lo[0] + i, lo[1] + j, lo[2] + k, jfac[1] * run);
                }
            }
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float run = 0.f;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    run += DS[2][k] * (S0[0][i] * S0[1][j] + 0.5f * DS[0][i] * S0[1][j] +
                                       0.5f * S0[0][i] * DS[1][j] + DS[0][i] * DS[1][j] * third);
                    if (run != 0.f) A.add(2, lo[0] + i, lo[1] + j, lo[2] + k, jfac[2] * run);
                }
            }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float run = 0.f;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                run += DS[0][i] * (S0[1][j] + 0.5f * DS[1][j]);
                if (run != 0.f) A.add(0, lo[0] + i, lo[1] + j, 0, jfac[0] * run);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float run = 0.f;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                run += DS[1][j] * (S0[0][i] + 0.5f * DS[0][i]);
                if (run != 0.f) A.add(1, lo[0] + i, lo[1] + j, 0, jfac[1] * run);
            }
        }
        const float fz = jfac[2] * vz;
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float W = S0[0][i] * S0[1][j] + 0.5f * DS[0][i] * S0[1][j] +
                                0.5f * S0[0][i] * DS[1][j] + DS[0][i] * DS[1][j] * third;
                if (W != 0.f) A.add(2, lo[0] + i, lo[1] + j, 0, fz * W);
            }
    }
}

// ---------------------------------------------------------------------------
// Esirkepov deposit (order 1)
// ---------------------------------------------------------------------------

// Shape values on the three nodes lo, lo+1, lo+2 of one axis, at the start
// (S0) and their change (DS) for a move from (c0, f0) to (c1, f1), |c1-c0| <= 1.
__device__ inline void shape3(int c0, float f0, int c1, float f1, int lo, float *S0, float *DS) {
    float s1[3];
    if (c0 == lo) { S0[0] = 1.f - f0; S0[1] = f0; S0[2] = 0.f; }
    else { S0[0] = 0.f; S0[1] = 1.f - f0; S0[2] = f0; }
    if (c0 == c1) {
        float d = f1 - f0;
        if (c0 == lo) { DS[0] = -d; DS[1] = d; DS[2] = 0.f; }
        else { DS[0] = 0.f; DS[1] = -d; DS[2] = d; }
        return;
    }
    if (c1 == lo) { s1[0] = 1.f - f1; s1[1] = f1; s1[2] = 0.f; }
    else { s1[0] = 0.f; s1[1] = 1.f - f1; s1[2] = f1; }
    for (int m = 0; m < 3; ++m) DS[m] = s1[m] - S0[m];
}

template <int DIM, class Acc>
__device__ inline void deposit_w(const Acc &A, const int *lo, const float (*S0)[3],
                                 const float (*DS)[3], const float *jf, float vz);

template <int DIM, class Acc>
__device__ inline void deposit(const Acc &A, const int *c0, const float *f0, const int *c1,
                               const float *f1, const float *jf, float vz) {
    float S0[3][3], DS[3][3];
    int lo[3];
    for (int a = 0; a < DIM; ++a) {
        lo[a] = min(c0[a], c1[a]);
        shape3(c0[a], f0[a], c1[a], f1[a], lo[a], S0[a], DS[a]);
    }
    deposit_w<DIM>(A, lo, S0, DS, jf, vz);
}

// Esirkepov sums for given node bases lo, start shapes S0 and shape changes DS
// on the three nodes lo .. lo+2 of each axis.
template <int DIM, class Acc>
__device__ inline void deposit_w(const Acc &A, const int *lo, const float (*S0)[3],
                                 const float (*DS)[3], const float *jf, float vz) {
    const float third = 1.0f / 3.0f;
    if (DIM == 3) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                float T = S0[1][j] * S0[2][k] + 0.5f * DS[1][j] * S0[2][k] +
                          0.5f * S0[1][j] * DS[2][k] + third * DS[1][j] * DS[2][k];
                if (T == 0.f) continue;
                float r0 = DS[0][0] * T, r1 = (DS[0][0] + DS[0][1]) * T;
                if (r0 != 0.f) A.add(0, lo[0], lo[1] + j, lo[2] + k, jf[0] * r0);
                if (r1 != 0.f) A.add(0, lo[0] + 1, lo[1] + j, lo[2] + k, jf[0] * r1);
            }
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                float T = S0[0][i] * S0[2][k] + 0.5f * DS[0][i] * S0[2][k] +
                          0.5f * S0[0][i] * DS[2][k] + third * DS[0][i] * DS[2][k];
                if (T == 0.f) continue;
                float r0 = DS[1][0] * T, r1 = (DS[1][0] + DS[1][1]) * T;
                if (r0 != 0.f) A.add(1, lo[0] + i, lo[1], lo[2] + k, jf[1] * r0);
                if (r1 != 0.f) A.add(1, lo[0] + i, lo[1] + 1, lo[2] + k, jf[1] * r1);
            }
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                float T = S0[0][i] * S0[1][j] + 0.5f * DS[0][i] * S0[1][j] +
                          0.5f * S0[0][i] * DS[1][j] + third * DS[0][i] * DS[1][j];
                if (T == 0.f) continue;
                float r0 = DS[2][0] * T, r1 = (DS[2][0] + DS[2][1]) * T;
                if (r0 != 0.f) A.add(2, lo[0] + i, lo[1] + j, lo[2], jf[2] * r0);
                if (r1 != 0.f) A.add(2, lo[0] + i, lo[1] + j, lo[2] + 1, jf[2] * r1);
            }
    } else {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float T = S0[1][j] + 0.5f * DS[1][j];
            if (T == 0.f) continue;
            float r0 = DS[0][0] * T, r1 = (DS[0][0] + DS[0][1]) * T;
            if (r0 != 0.f) A.add(0, lo[0], lo[1] + j, 0, jf[0] * r0);
            if (r1 != 0.f) A.add(0, lo[0] + 1, lo[1] + j, 0, jf[0] * r1);
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            float T = S0[0][i] + 0.5f * DS[0][i];
            if (T == 0.f) continue;
            float r0 = DS[1][0] * T, r1 = (DS[1][0] + DS[1][1]) * T;
            if (r0 != 0.f) A.add(1, lo[0] + i, lo[1], 0, jf[1] * r0);
            if (r1 != 0.f) A.add(1, lo[0] + i, lo[1] + 1, 0, jf[1] * r1);
        }
        const float fz = jf[2] * vz;
        if (fz != 0.f) {
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    float W = S0[0][i] * S0[1][j] + 0.5f * DS[0][i] * S0[1][j] +
                              0.5f * S0[0][i] * DS[1][j] + third * DS[0][i] * DS[1][j];
                    if (W != 0.f) A.add(2, lo[0] + i, lo[1] + j, 0, fz * W);
                }
        }
    }
}

// ---------------------------------------------------------------------------
// pushers
// ---------------------------------------------------------------------------

// Boris (Appendix A.1): v- = v + h E; v+ = [(1-|b|^2) v- + 2 b (v-.b) +
// 2 v- x b] / (1 + |b|^2), b = h B; v = v+ + h E; h = q dt / (2m).
__device__ inline void boris(float *v, const float *E, const float *B, float h) {
    float vm0 = v[0] + h * E[0], vm1 = v[1] + h * E[1], vm2 = v[2] + h * E[2];
    float b0 = h * B[0], b1 = h * B[1], b2 = h * B[2];
    float bb = b0 * b0 + b1 * b1 + b2 * b2;
    float vb = vm0 * b0 + vm1 * b1 + vm2 * b2;
    float c0 = vm1 * b2 - vm2 * b1, c1 = vm2 * b0 - vm0 * b2, c2 = vm0 * b1 - vm1 * b0;
    float inv = 1.0f / (1.0f + bb);
    float s = 1.0f - bb;
    v[0] = (s * vm0 + 2.f * (b0 * vb + c0)) * inv + h * E[0];
    v[1] = (s * vm1 + 2.f * (b1 * vb + c1)) * inv + h * E[1];
    v[2] = (s * vm2 + 2.f * (b2 * vb + c2)) * inv + h * E[2];
}

// Modified Boris for bound species (Appendix A.2):
// kick = h E - (dt/2) w0^2 D; v- = v + kick; solve
// (1 + G) v+ - v+ x b = (1 - G) v- + v- x b, G = diag(gamma_a dt / 2), i.e.
// (diag(a) + [b]x) v+ = w with a = 1 + G, w = (1 - G) v- + v- x b;
// v = v+ + kick; D += dt v.  Isotropic gamma (the plain kernel, and the
// variant kernel when the entries are equal): the closed form
// v+ = (a^2 w + a (w x b) + (w.b) b) / (a (a^2 + |b|^2)).  Diagonal gamma
// (variant kernel only): v+ = adj(M) w / det(M), M = diag(a) + [b]x.
// The kick and the isotropic solve are written with explicitly rounded
// operations (__fmaf_rn and friends), so that every kernel that inlines them
// computes the same bits whatever the compiler contracts around them.
template <bool X>
__device__ inline void bound_push(float *v, float *D, const float *E, const float *B,
                                  const SpeciesP &s) {
    const float h = s.hq;
    float k0 = __fmaf_rn(-s.hw0sq[0], D[0], __fmul_rn(h, E[0]));
    float k1 = __fmaf_rn(-s.hw0sq[1], D[1], __fmul_rn(h, E[1]));
    float k2 = __fmaf_rn(-s.hw0sq[2], D[2], __fmul_rn(h, E[2]));
    if (X && s.tensor) {
        // off-diagonal entries of the binding tensor (xy, xz, yz) x dt / 2
        k0 -= s.hw0off[0] * D[1] + s.hw0off[1] * D[2];
        k1 -= s.hw0off[0] * D[0] + s.hw0off[2] * D[2];
        k2 -= s.hw0off[1] * D[0] + s.hw0off[2] * D[1];
    }
    const float vm0 = __fadd_rn(v[0], k0), vm1 = __fadd_rn(v[1], k1), vm2 = __fadd_rn(v[2], k2);
    const float b0 = __fmul_rn(h, B[0]), b1 = __fmul_rn(h, B[1]), b2 = __fmul_rn(h, B[2]);
    if (X && s.aniso) {
        const float a0 = 1.f + s.gdt2v[0], a1 = 1.f + s.gdt2v[1], a2 = 1.f + s.gdt2v[2];
        const float w0 = (1.f - s.gdt2v[0]) * vm0 + (vm1 * b2 - vm2 * b1);
        const float w1 = (1.f - s.gdt2v[1]) * vm1 + (vm2 * b0 - vm0 * b2);
        const float w2 = (1.f - s.gdt2v[2]) * vm2 + (vm0 * b1 - vm1 * b0);
        const float inv = 1.0f / (a0 * a1 * a2 + a0 * b0 * b0 + a1 * b1 * b1 + a2 * b2 * b2);
        const float p0 = ((a1 * a2 + b0 * b0) * w0 + (b0 * b1 + a2 * b2) * w1 +
                          (b0 * b2 - a1 * b1) * w2) * inv;
        const float p1 = ((b0 * b1 - a2 * b2) * w0 + (a0 * a2 + b1 * b1) * w1 +
                          (b1 * b2 + a0 * b0) * w2) * inv;
        const float p2 = ((b0 * b2 + a1 * b1) * w0 + (b1 * b2 - a0 * b0) * w1 +
                          (a0 * a1 + b2 * b2) * w2) * inv;
        v[0] = p0 + k0;
        v[1] = p1 + k1;
        v[2] = p2 + k2;
        D[0] += s.dt * v[0];
        D[1] += s.dt * v[1];
        D[2] += s.dt * v[2];
        return;
    }
    // u x b component by component: p q - r t, one rounding for p q
    auto cross = [](float p, float q, float r, float t) { return __fmaf_rn(p, q, -__fmul_rn(r, t)); };
    const float a = __fadd_rn(1.f, s.gdt2), cc = __fsub_rn(1.f, s.gdt2);
    const float w0 = __fmaf_rn(cc, vm0, cross(vm1, b2, vm2, b1));
    const float w1 = __fmaf_rn(cc, vm1, cross(vm2, b0, vm0, b2));
    const float w2 = __fmaf_rn(cc, vm2, cross(vm0, b1, vm1, b0));
    const float wb = __fmaf_rn(w2, b2, __fmaf_rn(w1, b1, __fmul_rn(w0, b0)));
    const float bb = __fmaf_rn(b2, b2, __fmaf_rn(b1, b1, __fmul_rn(b0, b0)));
    const float a2 = __fmul_rn(a, a);
    const float inv = __fdiv_rn(1.0f, __fmul_rn(a, __fadd_rn(a2, bb)));
    const float p0 = __fmul_rn(__fmaf_rn(wb, b0, __fmaf_rn(a, cross(w1, b2, w2, b1), __fmul_rn(a2, w0))), inv);
    const float p1 = __fmul_rn(__fmaf_rn(wb, b1, __fmaf_rn(a, cross(w2, b0, w0, b2), __fmul_rn(a2, w1))), inv);
    const float p2 = __fmul_rn(__fmaf_rn(wb, b2, __fmaf_rn(a, cross(w0, b1, w1, b0), __fmul_rn(a2, w2))), inv);
    v[0] = __fadd_rn(p0, k0);
    v[1] = __fadd_rn(p1, k1);
    v[2] = __fadd_rn(p2, k2);
    D[0] = __fmaf_rn(s.dt, v[0], D[0]);
    D[1] = __fmaf_rn(s.dt, v[1], D[1]);
    D[2] = __fmaf_rn(s.dt, v[2], D[2]);
}

// Dirac carriers (Sec. 5): Boris with the transverse mass, v_z = 0 (sheet in
// the x-y plane), then |v| = v_F; a zero intermediate keeps the old direction.
__device__ inline void dirac_push(float *v, const float *E, const float *B, const SpeciesP &s) {
    float old0 = v[0], old1 = v[1], old2 = v[2];
    boris(v, E, B, s.hq);
    v[2] = 0.f;
    float n2 = v[0] * v[0] + v[1] * v[1];
    if (n2 > 0.f) {
        float sc = s.vF / sqrtf(n2);
        v[0] *= sc;
        v[1] *= sc;
    } else {
        v[0] = old0;
        v[1] = old1;
        v[2] = old2;
    }
}

// ---------------------------------------------------------------------------
// Esirkepov deposit for a move that stays in its cell (the common case)
// ---------------------------------------------------------------------------

// With S0 = (1 - f0, f0) and DS = (-dF, dF) on the two nodes of each axis,
// Esirkepov's transverse factor S0y S0z + (DSy S0z + S0y DSz)/2 +
// DSy DSz/3 equals my mz + DSy DSz / 12, where m = S0 + DS/2 holds the
// midpoint weights (1 - fm, fm), fm = f0 + dF/2.  Only the first node of the
// move axis receives current.
template <int DIM, class Acc>
__device__ inline void deposit_nocross(const Acc &A, const int *c, const float *f0, const float *dF,
                                       const float *jf, float vz) {
    const float k12 = 1.0f / 12.0f;
    float m0[2], m1[2], m2[2] = {1.f, 0.f};
    {
        float fm = f0[0] + 0.5f * dF[0];
        m0[0] = 1.f - fm;
        m0[1] = fm;
        fm = f0[1] + 0.5f * dF[1];
        m1[0] = 1.f - fm;
        m1[1] = fm;
        if (DIM == 3) {
            fm = f0[2] + 0.5f * dF[2];
            m2[0] = 1.f - fm;
            m2[1] = fm;
        }
    }
    if (DIM == 3) {
        if (dF[0] != 0.f) {
            const float cx = -jf[0] * dF[0], e = dF[1] * dF[2] * k12;
            A.add(0, c[0], c[1], c[2], cx * (m1[0] * m2[0] + e));
            A.add(0, c[0], c[1], c[2] + 1, cx * (m1[0] * m2[1] - e));
            A.add(0, c[0], c[1] + 1, c[2], cx * (m1[1] * m2[0] - e));
            A.add(0, c[0], c[1] + 1, c[2] + 1, cx * (m1[1] * m2[1] + e));
        }
        if (dF[1] != 0.f) {
            const float cy = -jf[1] * dF[1], e = dF[0] * dF[2] * k12;
            A.add(1, c[0], c[1], c[2], cy * (m0[0] * m2[0] + e));
            A.add(1, c[0], c[1], c[2] + 1, cy * (m0[0] * m2[1] - e));
            A.add(1, c[0] + 1, c[1], c[2], cy * (m0[1] * m2[0] - e));
            A.add(1, c[0] + 1, c[1], c[2] + 1, cy * (m0[1] * m2[1] + e));
        }
        if (dF[2] != 0.f) {
            const float cz = -jf[2] * dF[2], e = dF[0] * dF[1] * k12;
            A.add(2, c[0], c[1], c[2], cz * (m0[0] * m1[0] + e));
            A.add(2, c[0], c[1] + 1, c[2], cz * (m0[0] * m1[1] - e));
            A.add(2, c[0] + 1, c[1], c[2], cz * (m0[1] * m1[0] - e));
            A.add(2, c[0] + 1, c[1] + 1, c[2], cz * (m0[1] * m1[1] + e));
        }
    } else {
        if (dF[0] != 0.f) {
            const float cx = -jf[0] * dF[0];
            A.add(0, c[0], c[1], 0, cx * m1[0]);
            A.add(0, c[0], c[1] + 1, 0, cx * m1[1]);
        }
        if (dF[1] != 0.f) {
            const float cy = -jf[1] * dF[1];
            A.add(1, c[0], c[1], 0, cy * m0[0]);
            A.add(1, c[0] + 1, c[1], 0, cy * m0[1]);
        }
        const float fz = jf[2] * vz;
        if (fz != 0.f) {
            const float e = dF[0] * dF[1] * k12;
            A.add(2, c[0], c[1], 0, fz * (m0[0] * m1[0] + e));
            A.add(2, c[0], c[1] + 1, 0, fz * (m0[0] * m1[1] - e));
            A.add(2, c[0] + 1, c[1], 0, fz * (m0[1] * m1[0] - e));
            A.add(2, c[0] + 1, c[1] + 1, 0, fz * (m0[1] * m1[1] + e));
        }
    }
}

// The no-crossing current of a thread's consecutive particles in one cell,
// summed in registers before it reaches the shared J tile: with the
// cell-interleaved order a thread meets the particles of a cell in a row, so
// one flush of (up to) 12 shared atomics serves all of them.  Slots: J_x at
// the cell's (y, z) corners (0,0) (0,1) (1,0) (1,1); J_y at the (x, z)
// corners; J_z at the (x, y) corners (2D: the z = 0 corners only).
struct CellJ {
    int e;  // box index of the summed cell, -1: none
    float j[12];
};

template <int DIM, class Box>
__device__ inline void cellj_flush(const Box &box, CellJ &a) {
    if (a.e < 0) return;
    const int e = a.e, sy = box.b0, sz = box.b01;
    auto put = [&](int c, int o, float v) {
        if (v != 0.f) atomicAdd(&box.J[c][e + o], v);
    };
    put(0, 0, a.j[0]);
    put(0, sy, a.j[2]);
    put(1, 0, a.j[4]);
    put(1, 1, a.j[6]);
    put(2, 0, a.j[8]);
    put(2, sy, a.j[9]);
    put(2, 1, a.j[10]);
    put(2, 1 + sy, a.j[11]);
    if (DIM == 3) {
        put(0, sz, a.j[1]);
        put(0, sy + sz, a.j[3]);
        put(1, sz, a.j[5]);
        put(1, 1 + sz, a.j[7]);
    }
    a.e = -1;
}

// deposit_nocross into the register sum of the particle's cell (box index
// of local cell c), flushing the previous cell's sum first.  The same
// contributions as deposit_nocross, summed in another order.
template <int DIM, class Box>
__device__ inline void deposit_nocross_acc(const Box &box, const int *c, const float *f0,
                                           const float *dF, const float *jf, float vz, CellJ &a) {
    const int e = box.idx(c[0], c[1], c[2]);
    if (e != a.e) {
        cellj_flush<DIM>(box, a);
        a.e = e;
#pragma unroll
        for (int k = 0; k < 12; ++k) a.j[k] = 0.f;
    }
    const float k12 = 1.0f / 12.0f;
    float m0[2], m1[2], m2[2] = {1.f, 0.f};
    {
        float fm = f0[0] + 0.5f * dF[0];
        m0[0] = 1.f - fm;
        m0[1] = fm;
        fm = f0[1] + 0.5f * dF[1];
        m1[0] = 1.f - fm;
        m1[1] = fm;
        if (DIM == 3) {
            fm = f0[2] + 0.5f * dF[2];
            m2[0] = 1.f - fm;
            m2[1] = fm;
        }
    }
    if (DIM == 3) {
        const float cx = -jf[0] * dF[0], ex = dF[1] * dF[2] * k12;
        a.j[0] += cx * (m1[0] * m2[0] + ex);
        a.j[1] += cx * (m1[0] * m2[1] - ex);
        a.j[2] += cx * (m1[1] * m2[0] - ex);
        a.j[3] += cx * (m1[1] * m2[1] + ex);
        const float cy = -jf[1] * dF[1], ey = dF[0] * dF[2] * k12;
        a.j[4] += cy * (m0[0] * m2[0] + ey);
        a.j[5] += cy * (m0[0] * m2[1] - ey);
        a.j[6] += cy * (m0[1] * m2[0] - ey);
        a.j[7] += cy * (m0[1] * m2[1] + ey);
        const float cz = -jf[2] * dF[2], ez = dF[0] * dF[1] * k12;
        a.j[8] += cz * (m0[0] * m1[0] + ez);
        a.j[9] += cz * (m0[0] * m1[1] - ez);
        a.j[10] += cz * (m0[1] * m1[0] - ez);
        a.j[11] += cz * (m0[1] * m1[1] + ez);
    } else {
        const float cx = -jf[0] * dF[0];
        a.j[0] += cx * m1[0];
        a.j[2] += cx * m1[1];
        const float cy = -jf[1] * dF[1];
        a.j[4] += cy * m0[0];
        a.j[6] += cy * m0[1];
        const float fz = jf[2] * vz, ez = dF[0] * dF[1] * k12;
        a.j[8] += fz * (m0[0] * m1[0] + ez);
        a.j[9] += fz * (m0[0] * m1[1] - ez);
        a.j[10] += fz * (m0[1] * m1[0] - ez);
        a.j[11] += fz * (m0[1] * m1[1] + ez);
    }
}

// the no-crossing deposit into the box: through the register sum (ACC) or
// straight into the box's accessor
template <int DIM, bool ACC, class Box>
__device__ inline void deposit_nocross_box(const Box &box, const int *c, const float *f0,
                                           const float *dF, const float *jf, float vz, CellJ &acc) {
    if constexpr (ACC) deposit_nocross_acc<DIM>(box, c, f0, dF, jf, vz, acc);
    else deposit_nocross<DIM>(box, c, f0, dF, jf, vz);
}

// ---------------------------------------------------------------------------
// one particle
// ---------------------------------------------------------------------------

__device__ inline int mask_at(const ParticleLaunch &P, int x, int y, int z, bool &outside) {
    const GridP &g = P.g;
    int gx = wrap_or_neg(x, g.n[0], g.per[0]);
    int gy = wrap_or_neg(y, g.n[1], g.per[1]);
    int gz = g.dims == 3 ? wrap_or_neg(z, g.n[2], g.per[2]) : 0;
    outside = gx < 0 || gy < 0 || gz < 0;
    if (outside) return 0;
    if (!P.mask) return 1;
    return __ldg(P.mask + ((long long)gz * g.n[1] + gy) * g.n[0] + gx) != 0;
}

// local cell of a particle relative to the tile origin, unwrapped across
// periodic edges (so that a particle that drifted over the edge stays near
// its tile)
template <int DIM>
__device__ inline void local_cell(const ParticleLaunch &P, const int *gc, const int *org, int *lc) {
    for (int a = 0; a < 3; ++a) {
        int l = gc[a] - org[a];
        if (a < DIM && P.g.per[a]) {
            const int n = P.g.n[a];
            if (l < -kHalo) l += n;
            else if (l > P.tp.T[a] + kHalo) l -= n;
        }
        lc[a] = a < DIM ? l : 0;
    }
}

// The staged box serves a particle in local cell c in [-1, T]: CIC with the
// box of local cells -2 .. T+2; TSC (its three-node gather and four-node
// deposit reach one node further) with the box of cells -3 .. T+3.
template <int DIM>
__device__ inline bool in_core(const ParticleLaunch &P, const int *c) {
    bool ok = true;
    for (int a = 0; a < DIM; ++a) ok = ok && c[a] >= -1 && c[a] <= P.tp.T[a];
    return ok;
}

// Uniform in [0, 1) from the top 24 bits of a Philox word (exact in FP32).
__device__ inline float u24(uint32_t w) { return (float)(w >> 8) * 0x1p-24f; }

// Diffuse re-emission (Sec. 3) of a particle that crossed the face normal to
// axis ax moving along sgn (+1 / -1): the speed is kept, the direction is
// drawn from Lambert's cosine law about the inward normal -sgn e_ax --
// cos(theta) = sqrt(u1), azimuth 2 pi u2 from the next axis (x -> y -> z);
// Dirac carriers: the in-plane law sin(theta) = 2 u1 - 1, v_z = 0.
__device__ inline void diffuse_velocity(bool dirac, float *v, int ax, int sgn, float u1,
                                        float u2) {
    const float speed = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const float vn = sgn > 0 ? -speed : speed;
    if (dirac) {
        const float st = 2.f * u1 - 1.f;
        const float ct = sqrtf((1.f - st) * (1.f + st));
        const float a = vn * ct, b = speed * st;
        if (ax == 0) { v[0] = a; v[1] = b; }
        else { v[1] = a; v[0] = b; }
        v[2] = 0.f;
    } else {
        const float ct = sqrtf(u1), st = sqrtf(1.f - u1);
        float sn, cs;
        sincospif(2.f * u2, &sn, &cs);
        const float a = vn * ct, t1 = speed * st * cs, t2 = speed * st * sn;
        if (ax == 0) { v[0] = a; v[1] = t1; v[2] = t2; }
        else if (ax == 1) { v[1] = a; v[2] = t1; v[0] = t2; }
        else { v[2] = a; v[0] = t1; v[1] = t2; }
    }
}

// Free electrons and Dirac carriers (species index si, dirac: the species is
// PIC_DIRAC -- one loop body for both kinds, which differ only in the push,
// keeps the kernel's code small), shape order S.
// ACC: a fast no-crossing move's current goes to the register sum acc.
// GONLY: always the global accessors (the pass over particles deferred out of
// a tile by the lean kernel, k_particle_lean.cu); the box is not read.
template <int DIM, bool X, int S = 1, bool ACC = false, class Box = BoxAcc, bool GONLY = false>
__device__ inline unsigned push_mobile(const ParticleLaunch &P, const SpeciesP &s, int si,
                                       bool dirac, int p, const int *org, const Box &box,
                                       const GlobalAcc<DIM, X> &glob, CellJ &acc) {
    const GridP &g = P.g;
    const uint32_t pc = s.cell[p];
    const int gc[3] = {cell_x(pc), cell_y(pc), DIM == 3 ? cell_z(pc) : 0};
    int lc[3];
    local_cell<DIM>(P, gc, org, lc);
    float v[3] = {s.v[0][p], s.v[1][p], s.v[2][p]};
    float f0[3] = {s.o[0][p], s.o[1][p], DIM == 3 ? s.o[2][p] : 0.f};
    float E[3], B[3];
    const bool fast = !GONLY && in_core<DIM>(P, lc);
    if constexpr (S == 2) {
        if (fast) gather_tsc<DIM>(box, lc, f0, E, B);
        else gather_tsc<DIM>(glob, gc, f0, E, B);
    } else {
        if (fast) gather<DIM>(box, lc, f0, E, B);
        else gather<DIM>(glob, gc, f0, E, B);
    }

    if (dirac) dirac_push(v, E, B, s);
    else boris(v, E, B, s.hq);

    // drift; at most one cell per axis per step.  mv: the move in cells
    float f1[3] = {f0[0], f0[1], f0[2]};
    float mv[3] = {0.f, 0.f, 0.f};
    int sh[3] = {0, 0, 0};
    for (int a = 0; a < DIM; ++a) {
        mv[a] = s.dtd[a] * v[a];
        float x = f0[a] + mv[a];
        if (!(x > -1.f && x < 2.f)) {
            // more than one cell in one step (or NaN): record and stay put
            atomicOr(P.status, kStatusBounds);
            x = f0[a];
            mv[a] = 0.f;
        }
        if (x >= 1.f) { sh[a] = 1; x -= 1.f; }
        else if (x < 0.f) { sh[a] = -1; x += 1.f; }
        f1[a] = clamp_below_one(x);
    }
    unsigned refl = 0;
    const bool moved = (sh[0] | sh[1] | sh[2]) != 0;
    if (moved) {
        bool out1, out0;
        int m1 = mask_at(P, gc[0] + sh[0], gc[1] + sh[1], gc[2] + sh[2], out1);
        int m0 = mask_at(P, gc[0], gc[1], gc[2], out0);
        if (out1 || (m0 && !m1)) {
            // reflection at the crossed faces (Sec. 3): positions mirrored;
            // specular, or -- at a material edge crossed through a single
            // face, with probability p_diffuse -- diffuse
            bool diffuse = false;
            if (X && !out1 && P.p_diffuse > 0.f) {
                const int ncross = (sh[0] != 0) + (sh[1] != 0) + (sh[2] != 0);
                const int ax = sh[0] ? 0 : sh[1] ? 1 : 2;
                if (ncross == 1 && !(dirac && ax == 2)) {
                    uint32_t x[4] = {s.pid[p], P.rng_step, (uint32_t)si, kDiffuseStream};
                    philox4x32_10(x, P.diff_key[0], P.diff_key[1]);
                    diffuse = u24(x[0]) < P.p_diffuse;
                    if (diffuse)
                        diffuse_velocity(dirac, v, ax, sh[0] + sh[1] + sh[2], u24(x[1]),
                                         u24(x[2]));
                }
            }
            for (int a = 0; a < DIM; ++a) {
                if (sh[a] == 0) continue;
                f1[a] = clamp_below_one(1.f - f1[a]);
                if (!diffuse) v[a] = -v[a];
                sh[a] = 0;
            }
            refl = 1;
        }
    }
    if constexpr (S == 2) {
        const int c1l[3] = {lc[0] + sh[0], lc[1] + sh[1], lc[2] + sh[2]};
        if (fast) deposit_tsc<DIM>(box, lc, f0, c1l, f1, s.jfac, v[2]);
        else {
            const int g1[3] = {gc[0] + sh[0], gc[1] + sh[1], gc[2] + sh[2]};
            deposit_tsc<DIM>(glob, gc, f0, g1, f1, s.jfac, v[2]);
        }
        if (sh[0] | sh[1] | sh[2]) {
            int nxc[3];
            for (int a = 0; a < 3; ++a) {
                nxc[a] = gc[a] + sh[a];
                if (a < DIM && g.per[a]) nxc[a] = wrap_or_neg(nxc[a], g.n[a], 1);
            }
            s.cell[p] = pack_cell(nxc[0], nxc[1], nxc[2]);
        }
    } else if (!(sh[0] | sh[1] | sh[2])) {
        // ends in its cell.  A move that stayed there takes the move itself,
        // not the difference of the stored offsets (an FP32 offset near 1 has
        // an ulp of 6e-8 cell, a few 1e-5 of a typical move of 1e-3 cell);
        // the offset's rounding leaves a charge-continuity defect of at most
        // half an ulp of the offset per move.  A move mirrored back into its
        // cell takes the difference of the offsets.
        float dF[3];
        for (int a = 0; a < 3; ++a)
            dF[a] = a >= DIM ? 0.f : refl ? f1[a] - f0[a] : mv[a];
        if (fast) deposit_nocross_box<DIM, ACC>(box, lc, f0, dF, s.jfac, v[2], acc);
        else deposit_nocross<DIM>(glob, gc, f0, dF, s.jfac, v[2]);
    } else {
        int c1l[3] = {lc[0] + sh[0], lc[1] + sh[1], lc[2] + sh[2]};
        if (fast) deposit<DIM>(box, lc, f0, c1l, f1, s.jfac, v[2]);
        else {
            int g1[3] = {gc[0] + sh[0], gc[1] + sh[1], gc[2] + sh[2]};
            deposit<DIM>(glob, gc, f0, g1, f1, s.jfac, v[2]);
        }
        int nxc[3];
        for (int a = 0; a < 3; ++a) {
            nxc[a] = gc[a] + sh[a];
            if (a < DIM && g.per[a]) nxc[a] = wrap_or_neg(nxc[a], g.n[a], 1);
        }
        s.cell[p] = pack_cell(nxc[0], nxc[1], nxc[2]);
    }
    s.o[0][p] = f1[0];
    s.o[1][p] = f1[1];
    if (DIM == 3) s.o[2][p] = f1[2];
    s.v[0][p] = v[0];
    s.v[1][p] = v[1];
    s.v[2][p] = v[2];
    return refl;
}

// Bound electrons.  Position = anchor cell + anchor offset + D / d.  The hot
// loop reads the FP32 copy of the anchor offset (the FP64 anchor is the
// stored rest position).  The current uses the move dt v / d of this step
// directly: it is far below an FP32 ulp of the offset, and the displacement D
// itself is ~100x the per-step move, so differences of stored values would
// lose most of its bits.
template <int DIM, bool X, bool ACC = false, class Box = BoxAcc, bool GONLY = false>
__device__ inline void push_bound(const ParticleLaunch &P, const SpeciesP &s, int p,
                                  const int *org, const Box &box,
                                  const GlobalAcc<DIM, X> &glob, CellJ &acc) {
    const GridP &g = P.g;
    const uint32_t pc = s.cell[p];
    const int gc[3] = {cell_x(pc), cell_y(pc), DIM == 3 ? cell_z(pc) : 0};
    int lc[3];
    local_cell<DIM>(P, gc, org, lc);
    float v[3] = {s.v[0][p], s.v[1][p], s.v[2][p]};
    float D[3] = {s.disp[0][p], s.disp[1][p], s.disp[2][p]};
    float an[3];
    int c0[3] = {0, 0, 0}, c1[3] = {0, 0, 0};
    float f0[3] = {0.f, 0.f, 0.f}, f1[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < DIM; ++a) {
        an[a] = s.anchor32[a][p];
        float xa = an[a] + D[a] * g.inv_d[a];
        float fl = floorf(xa);
        c0[a] = lc[a] + (int)fl;
        f0[a] = clamp_below_one(xa - fl);
    }
    float E[3], B[3];
    const bool fast = !GONLY && in_core<DIM>(P, c0);
    if (fast) gather<DIM>(box, c0, f0, E, B);
    else {
        int gg[3] = {c0[0] + org[0], c0[1] + org[1], c0[2] + org[2]};
        gather<DIM>(glob, gg, f0, E, B);
    }
    bound_push<X>(v, D, E, B, s);
    float dF[3] = {0.f, 0.f, 0.f};
    int sh[3] = {0, 0, 0};
    bool jump = false;
    for (int a = 0; a < DIM; ++a) {
        dF[a] = s.dt * v[a] * g.inv_d[a];
        const float x = f0[a] + dF[a];
        sh[a] = x >= 1.f ? 1 : (x < 0.f ? -1 : 0);
        jump = jump || !(x > -1.f && x < 2.f);
    }
    (void)c1;
    (void)f1;
    if (jump) {
        // more than one cell in one step (or NaN): record, deposit nothing
        atomicOr(P.status, kStatusBounds);
    } else if (!(sh[0] | sh[1] | sh[2])) {
        if (fast) deposit_nocross_box<DIM, ACC>(box, c0, f0, dF, s.jfac, v[2], acc);
        else {
            int g0[3] = {c0[0] + org[0], c0[1] + org[1], c0[2] + org[2]};
            deposit_nocross<DIM>(glob, g0, f0, dF, s.jfac, v[2]);
        }
    } else {
        // shapes on the nodes lo .. lo+2 written from (f0, dF) so that the
        // small move is not rounded against offsets near 1
        float S0[3][3], DS[3][3];
        int lo[3];
        for (int a = 0; a < DIM; ++a) {
            const float f = f0[a], d = dF[a];
            if (sh[a] == 0) {
                lo[a] = c0[a];
                S0[a][0] = 1.f - f; S0[a][1] = f; S0[a][2] = 0.f;
                DS[a][0] = -d; DS[a][1] = d; DS[a][2] = 0.f;
            } else if (sh[a] > 0) {
                const float e0 = 1.f - f, f1u = d - e0;
                lo[a] = c0[a];
                S0[a][0] = e0; S0[a][1] = f; S0[a][2] = 0.f;
                DS[a][0] = -e0; DS[a][1] = e0 - f1u; DS[a][2] = f1u;
            } else {
                const float x = f + d;
                lo[a] = c0[a] - 1;
                S0[a][0] = 0.f; S0[a][1] = 1.f - f; S0[a][2] = f;
                DS[a][0] = -x; DS[a][1] = x + f; DS[a][2] = -f;
            }
        }
        if (fast) deposit_w<DIM>(box, lo, S0, DS, s.jfac, v[2]);
        else {
            int g0[3] = {lo[0] + org[0], lo[1] + org[1], lo[2] + org[2]};
            deposit_w<DIM>(glob, g0, S0, DS, s.jfac, v[2]);
        }
    }
    s.disp[0][p] = D[0];
    s.disp[1][p] = D[1];
    s.disp[2][p] = D[2];
    s.v[0][p] = v[0];
    s.v[1][p] = v[1];
    s.v[2][p] = v[2];
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------

// Box element e -> (bx, by, bz), advanced by the CTA width without divisions.
struct BoxWalk {
    int bx, by, bz, e;
    int dx, dy, dz;  // the step decomposed over the box
    __device__ inline void start(int b0, int b1, int e0, int step) {
        const int b01 = b0 * b1;
        e = e0;
        bz = e0 / b01;
        by = (e0 - bz * b01) / b0;
        bx = e0 - bz * b01 - by * b0;
        dz = step / b01;
        dy = (step - dz * b01) / b0;
        dx = step - dz * b01 - dy * b0;
    }
    __device__ inline void next(int b0, int b1, int step) {
        e += step;
        bx += dx;
        by += dy;
        bz += dz;
        if (bx >= b0) { bx -= b0; ++by; }
        if (by >= b1) { by -= b1; ++bz; }
    }
};

// One tile of one simulation: stage the field box, push every particle of
// the tile (all species), flush the J box.  P must live in parameter or shared
// memory (not global), so that the compiler keeps its fields in registers
// across the particle stores.
// ACC: sum each thread's no-crossing current per cell in registers (the
// particles are in the cell-interleaved order).
template <int DIM, bool X, int S = 1, bool ACC = false>
__device__ void tile_pass(const ParticleLaunch &P, const int t, float *smem, unsigned *s_refl) {
    constexpr int H = S == 2 ? 3 : kHalo;  // box halo (cells)
    const TileP &tp = P.tp;
    const int bn = tp.boxn;
    const int B0 = tp.box[0], B1 = tp.box[1];
    BoxAccT<H> box;
    for (int c = 0; c < 6; ++c) box.F[c] = smem + c * bn;
    for (int c = 0; c < 3; ++c) box.J[c] = smem + (6 + c) * bn;
    box.b0 = B0;
    box.b01 = B0 * B1;
    box.hz = DIM == 3 ? H : 0;
    GlobalAcc<DIM, X> glob;
    glob.g = &P.g;
    glob.E = P.E;
    glob.B = P.B;
    glob.Eext = P.Eext;
    glob.J = P.J;
    glob.jdirty = P.jdirty;
    glob.nbx = P.nbx;
    glob.nby = P.nby;
    glob.zchunk = P.zchunk;
    const GridP &g = P.g;
    const float hdt = 0.5f * g.dt;
    const int tx = t % tp.nt[0], ty = (t / tp.nt[0]) % tp.nt[1], tz = t / (tp.nt[0] * tp.nt[1]);
    const int org[3] = {tx * tp.T[0], ty * tp.T[1], DIM == 3 ? tz * tp.T[2] : 0};
    const int step = blockDim.x;
    __syncthreads();  // previous tile's flush is done with the box
    // stage E^n, B^{n-1/2} of the box; zero J
    {
        BoxWalk w;
        for (w.start(B0, B1, threadIdx.x, step); w.e < bn; w.next(B0, B1, step)) {
            int gx = wrap_or_neg(org[0] + w.bx - H, g.n[0], g.per[0]);
            int gy = wrap_or_neg(org[1] + w.by - H, g.n[1], g.per[1]);
            int gz = DIM == 3 ? wrap_or_neg(org[2] + w.bz - H, g.n[2], g.per[2]) : 0;
            bool in = gx >= 0 && gy >= 0 && gz >= 0;
            long long o = in ? ((long long)gz * g.n[1] + gy) * g.n[0] + gx : 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                cp_async4(&box.F[c][w.e], P.E[c] + o, in);
                cp_async4(&box.F[3 + c][w.e], P.B[c] + o, in);
                box.J[c][w.e] = 0.f;
            }
        }
        cp_async_wait_all();
    }
    __syncthreads();
    // B^n = B^{n-1/2} - (dt/2) curl E^n (plain Yee curl); zero outside
    {
        BoxWalk w;
        for (w.start(B0, B1, threadIdx.x, step); w.e < bn; w.next(B0, B1, step)) {
            const int e = w.e;
            const bool hx = w.bx + 1 < B0, hy = w.by + 1 < B1;
            const bool hz = DIM == 2 || w.bz + 1 < tp.box[2];
            if (!(hx && hy && hz)) continue;  // never gathered
            int gx = wrap_or_neg(org[0] + w.bx - H, g.n[0], g.per[0]);
            int gy = wrap_or_neg(org[1] + w.by - H, g.n[1], g.per[1]);
            int gz = DIM == 3 ? wrap_or_neg(org[2] + w.bz - H, g.n[2], g.per[2]) : 0;
            if (gx < 0 || gy < 0 || gz < 0) {
                box.F[3][e] = box.F[4][e] = box.F[5][e] = 0.f;
                continue;
            }
            const int sx = 1, sy = box.b0, sz = box.b01;
            float dEz_dy = (box.F[2][e + sy] - box.F[2][e]) * g.inv_d[1];
            float dEx_dy = (box.F[0][e + sy] - box.F[0][e]) * g.inv_d[1];
            float dEz_dx = (box.F[2][e + sx] - box.F[2][e]) * g.inv_d[0];
            float dEy_dx = (box.F[1][e + sx] - box.F[1][e]) * g.inv_d[0];
            float dEy_dz = 0.f, dEx_dz = 0.f;
            if (DIM == 3) {
                dEy_dz = (box.F[1][e + sz] - box.F[1][e]) * g.inv_d[2];
                dEx_dz = (box.F[0][e + sz] - box.F[0][e]) * g.inv_d[2];
            }
            box.F[3][e] -= hdt * (dEz_dy - dEy_dz);
            box.F[4][e] -= hdt * (dEx_dz - dEz_dx);
            box.F[5][e] -= hdt * (dEy_dx - dEx_dy);
        }
    }
    __syncthreads();
    if (X && P.Eext[0]) {
        // the external field joins the gathered E after the B^n pass, which
        // takes the curl of the Maxwell E alone
        BoxWalk w;
        for (w.start(B0, B1, threadIdx.x, step); w.e < bn; w.next(B0, B1, step)) {
            int gx = wrap_or_neg(org[0] + w.bx - H, g.n[0], g.per[0]);
            int gy = wrap_or_neg(org[1] + w.by - H, g.n[1], g.per[1]);
            int gz = DIM == 3 ? wrap_or_neg(org[2] + w.bz - H, g.n[2], g.per[2]) : 0;
            if (gx < 0 || gy < 0 || gz < 0) continue;
            const long long o = ((long long)gz * g.n[1] + gy) * g.n[0] + gx;
#pragma unroll
            for (int c = 0; c < 3; ++c) box.F[c][w.e] += __ldg(P.Eext[c] + o);
        }
        __syncthreads();
    }
    CellJ acc;
    acc.e = -1;
    for (int si = 0; si < P.nsp; ++si) {
        const SpeciesP &s = P.sp[si];
        // particle indices of a simulation fit int32 (tile_start is int)
        const int a = s.tile_start[t], b = s.tile_start[t + 1];
        unsigned r = 0;
        if (s.kind == PIC_BOUND) {
            for (int p = a + threadIdx.x; p < b; p += blockDim.x)
                push_bound<DIM, X, ACC>(P, s, p, org, box, glob, acc);
        } else {
            const bool dirac = s.kind == PIC_DIRAC;
            for (int p = a + threadIdx.x; p < b; p += blockDim.x)
                r += push_mobile<DIM, X, S, ACC>(P, s, si, dirac, p, org, box, glob, acc);
        }
        if (r) atomicAdd(&s_refl[si], r);
    }
    if (ACC) cellj_flush<DIM>(box, acc);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    // flush the J box; mark the field blocks that received current (lanes of
    // a warp with the same block elect one to store the flag)
    BoxWalk w;
    w.start(B0, B1, threadIdx.x, step);
    for (int e0 = 0; e0 < bn; e0 += step, w.next(B0, B1, step)) {
        long long blk = -1;
        if (w.e < bn) {
            const int e = w.e;
            const float jx = box.J[0][e], jy = box.J[1][e], jz = box.J[2][e];
            if (jx != 0.f || jy != 0.f || jz != 0.f) {
                int gx = wrap_or_neg(org[0] + w.bx - H, g.n[0], g.per[0]);
                int gy = wrap_or_neg(org[1] + w.by - H, g.n[1], g.per[1]);
                int gz = DIM == 3 ? wrap_or_neg(org[2] + w.bz - H, g.n[2], g.per[2]) : 0;
                if (gx >= 0 && gy >= 0 && gz >= 0) {
                    const long long o = ((long long)gz * g.n[1] + gy) * g.n[0] + gx;
                    if (jx != 0.f) atomicAdd(P.J[0] + o, jx);
                    if (jy != 0.f) atomicAdd(P.J[1] + o, jy);
                    if (jz != 0.f) atomicAdd(P.J[2] + o, jz);
                    const int bz = DIM == 3 ? gz / P.zchunk : 0;
                    blk = ((long long)bz * P.nby + gy / kFieldBY) * P.nbx + gx / kFieldBX;
                }
            }
        }
        const unsigned same = __match_any_sync(0xffffffffu, blk);
        if (blk >= 0 && lane == __ffs(same) - 1) P.jdirty[blk] = 1;
    }
}

// One particle phase: the persistent CTAs take tiles from the active list.
template <int DIM, bool X, int S = 1, bool ACC = false>
__device__ __forceinline__ void particle_phase(const ParticleLaunch &P) {
    extern __shared__ float smem[];
    __shared__ unsigned s_refl[kMaxSpecies];
    __shared__ int s_next;
    if (threadIdx.x < kMaxSpecies) s_refl[threadIdx.x] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && P.step_counter) *P.step_counter += 1;
    const int nact = *P.nactive;
    // take tiles from the list (largest first) as this CTA becomes free; the
    // read of s_next happens before tile_pass's first barrier, its next write
    // after tile_pass
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(&P.sched[0], 1);
        __syncthreads();
        const int it = s_next;
        if (it >= nact) break;
        tile_pass<DIM, X, S, ACC>(P, P.active[it], smem, s_refl);
    }
    __syncthreads();
    if (threadIdx.x < P.nsp && s_refl[threadIdx.x])
        atomicAdd(P.sp[threadIdx.x].nrefl, (unsigned long long)s_refl[threadIdx.x]);
    if (threadIdx.x == 0) {
        // the last CTA to finish (every CTA has made its final take) resets
        // the counters for the next launch
        __threadfence();
        if (atomicAdd(&P.sched[1], 1) == (int)gridDim.x - 1) {
            P.sched[0] = 0;
            P.sched[1] = 0;
        }
    }
}

// Resident CTAs per SM the plain kernel's registers are sized for.
#ifndef PIC_PARTICLE_MINBLOCKS
#define PIC_PARTICLE_MINBLOCKS 3
#endif

template <int DIM>
__global__ void __launch_bounds__(kThreads, PIC_PARTICLE_MINBLOCKS) particle_kernel(ParticleLaunch P) {
    particle_phase<DIM, false, 1, true>(P);
}

// The kernel with the boundary variants is held to the plain kernel's 64
// registers (as if 4 CTAs of 256 threads shared an SM): beside the B pass of
// the overlapped step 3 CTAs per SM run, and the registers they leave free
// are what lets the B pass co-run.
template <int DIM>
__global__ void __launch_bounds__(kThreads, 4) particle_kernel_ext(ParticleLaunch P) {
    particle_phase<DIM, true>(P);
}

// Many simulations in one persistent launch: items[i] = (simulation, tile),
// tile < 0 = padding.  Each simulation's parameter block (two variants, one
// per field ping-pong parity) is copied to shared memory for its items.
// X: the variant with the external field, diffuse reflection and the
// anisotropic bound push (k_particle_ext.cu), launched when a member has one
// of them; S = 2: TSC members (k_particle_tsc.cu).  The diffuse draws are
// keyed on the step index: a member's block holds the index of its first
// group step in rng_step, and the member's device step count done[] (set
// by the step's begin pass) is added here, so a captured epoch draws afresh
// at every step.
template <int DIM, bool X = false, int S = 1>
__global__ void __launch_bounds__(kThreads, S == 2 ? 2 : 3)
    batch_particle_kernel(const ParticleLaunch *descs, const int *fpar, const int *active,
                          const int2 *items, int nitems, int *sched, const long long *done) {
    extern __shared__ float smem[];
    __shared__ unsigned s_refl[kMaxSpecies];
    __shared__ ParticleLaunch sP;
    __shared__ int s_sim, s_next;
    if (threadIdx.x == 0) s_sim = -1;
    // items are taken through an atomic counter as the CTA becomes free
    for (;;) {
        __syncthreads();  // previous item finished with sP / s_refl / s_next
        if (threadIdx.x == 0) s_next = atomicAdd(&sched[0], 1);
        __syncthreads();
        const int it = s_next;
        if (it >= nitems) break;
        const int2 w = items[it];
        if (w.y < 0 || !active[w.x]) continue;  // uniform over the CTA
        const bool fresh = s_sim != w.x;
        if (fresh) {
            const int *src = reinterpret_cast<const int *>(descs + 2 * w.x + fpar[w.x]);
            int *dst = reinterpret_cast<int *>(&sP);
            for (int q = threadIdx.x; q < (int)(sizeof(ParticleLaunch) / 4); q += blockDim.x)
                dst[q] = src[q];
        }
        if (threadIdx.x < kMaxSpecies) s_refl[threadIdx.x] = 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            if (fresh) sP.rng_step += (uint32_t)done[w.x];
            s_sim = w.x;
        }
        tile_pass<DIM, X, S>(sP, w.y, smem, s_refl);
        __syncthreads();
        if (threadIdx.x < sP.nsp && s_refl[threadIdx.x])
            atomicAdd(sP.sp[threadIdx.x].nrefl, (unsigned long long)s_refl[threadIdx.x]);
    }
    if (threadIdx.x == 0) {
        // the last CTA to finish resets the counters for the next launch
        __threadfence();
        if (atomicAdd(&sched[1], 1) == (int)gridDim.x - 1) {
            sched[0] = 0;
            sched[1] = 0;
        }
    }
}

}  // namespace

// the kernels with the boundary variants (k_particle_ext.cu)
cudaError_t particle_ext_setup(int dims, size_t smem, int *ctas_per_sm);
cudaError_t launch_particles_ext(const ParticleLaunch &pl, int nctas, size_t smem,
                                 cudaStream_t s);
// the batch kernel with the boundary variants and the anisotropic bound push
// (k_particle_ext.cu)
cudaError_t launch_batch_particles_ext(int dims, const ParticleLaunch *descs, const int *fpar,
                                       const int *active, const int2 *items, int nitems,
                                       int *sched, const long long *done, int nctas, size_t smem,
                                       cudaStream_t s);
// the batch kernel of TSC members (k_particle_tsc.cu)
cudaError_t launch_batch_particles_tsc(int dims, const ParticleLaunch *descs, const int *fpar,
                                       const int *active, const int2 *items, int nitems,
                                       int *sched, const long long *done, int nctas, size_t smem,
                                       cudaStream_t s);
// the TSC kernels (k_particle_tsc.cu), boundary variants included
cudaError_t particle_tsc_setup(int dims, size_t smem, int *ctas_per_sm);
cudaError_t launch_particles_tsc(const ParticleLaunch &pl, int nctas, size_t smem,
                                 cudaStream_t s);

}  // namespace pic
