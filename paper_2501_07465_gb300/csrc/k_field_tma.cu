// k_field_tma.cu -- the fused Yee + CPML + source update of k_field.cu, fed by
// the Tensor Memory Accelerator.
//
//   B^{n+1/2} = B^{n-1/2} - dt (curl E^n + psi_B)
//   E^{n+1}   = E^n + dt (c^2 (curl B^{n+1/2} + psi_E) - J^{n+1/2} / eps0)
// (Maxwell's curl equations on the Yee stagger, Sec. 4.1; Eq. consteps with
// eps = eps0; CPML after Roden & Gedney with kappa = 1, alpha = 0.)
//
// Same decomposition as k_field.cu (a CTA owns a 32 x 8 column of cells and
// marches up a chunk of z planes), but the planes arrive by TMA: one elected
// thread issues cp.async.bulk.tensor loads of E^n (box 40 x 10: x from i0-4 so
// the start is 16-byte aligned, y from j0-1), B^{n-1/2} (36 x 9) and, where
// the block holds current, J (32 x 8) into a ring of S stages, each guarded
// by an mbarrier with expect_tx.  Loads run S - 1 planes ahead of the
// compute, so the kernel streams at HBM speed instead of waiting on two
// dependent global round trips per plane.  Outside a non-periodic face the
// TMA fill value (zero) is the wall; across a periodic face the few halo
// entries the box cannot wrap are patched with plain loads.
//
// Every mbarrier wait is bounded: a wait that gives up latches
// PIC_ETIMEOUT in the status word, waits (bounded) for the copies still in
// flight and ends the CTA.
#include <cuda.h>

#include <type_traits>

#include "pic_internal.cuh"

namespace pic {

namespace {

constexpr int BX = kFieldBX, BY = kFieldBY, NT = BX * BY;
constexpr int S = 4;                       // pipeline stages
constexpr int EW = 40, EH = 10;            // E tile: x in [i0-4, i0+36), y in [j0-1, j0+9)
constexpr int BW = 36, BH = 9;             // B tile: x in [i0-4, i0+32), y in [j0-1, j0+8)
constexpr int JW = BX, JH = BY;            // J tile: the own cells
constexpr uint32_t E_BYTES = EW * EH * 4, B_BYTES = BW * BH * 4, J_BYTES = JW * JH * 4;
constexpr int E_PAD = 1664, B_PAD = 1408, J_PAD = 1024;  // 128-byte aligned component slots
constexpr int STAGE = 3 * (E_PAD + B_PAD + J_PAD);
constexpr int SB_FLOATS = 3 * (BY + 1) * (BX + 1);
constexpr int SB_BYTES = (SB_FLOATS * 4 + 127) / 128 * 128;

__device__ inline uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ inline void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ inline void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ inline bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ inline bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; false = gave up.  A limit below the default (the tests'
// knob) polls with the non-blocking test_wait, so that the limit counts
// polls and not the hardware's own suspension inside try_wait.
__device__ inline bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit = kWaitPolls) {
    if (limit < kWaitPolls) {
        for (long long it = 0; it < limit; ++it)
            if (mbar_test_wait(bar, parity)) return true;
        return false;
    }
    for (long long it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 32) __nanosleep(64);
    }
    return false;
}

__device__ inline void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                   uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ inline void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ inline int wrap_or_neg(int i, int n, int per) {
    if (i >= 0 && i < n) return i;
    if (!per) return -1;
    int r = i % n;
    return r < 0 ? r + n : r;
}

__device__ inline int slab_idx(int i, int n, int P) {
    if (i < P) return i;
    if (i >= n - P) return i - (n - 2 * P);
    return -1;
}

__device__ inline long long psi_index(const GridP &g, const FieldP &f, int a, int i, int j, int k) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], P = f.P;
    if (!f.pml[a]) return -1;
    if (a == 0) {
        int s = slab_idx(i, nx, P);
        return s < 0 ? -1 : ((long long)k * ny + j) * (2 * P) + s;
    } else if (a == 1) {
        int s = slab_idx(j, ny, P);
        return s < 0 ? -1 : ((long long)k * (2 * P) + s) * nx + i;
    }
    int s = slab_idx(k, nz, P);
    return s < 0 ? -1 : ((long long)s * ny + j) * nx + i;
}

__device__ inline float cpml_term(const FieldP &f, int a, int slot, long long pidx, int pos,
                                  bool half, float deriv, bool write) {
    if (pidx < 0) return deriv;
    float b = half ? __ldg(f.cb_h[a] + pos) : __ldg(f.cb_e[a] + pos);
    float c = half ? __ldg(f.ca_h[a] + pos) : __ldg(f.ca_e[a] + pos);
    float psi = b * __ldg(f.psi_in[a][slot] + pidx) + c * deriv;
    if (write) f.psi_out[a][slot][pidx] = psi;
    return deriv + psi;
}

struct Stage {
    float *E[3];
    float *B[3];
    float *J[3];
};

// tile coordinates: E/B tiles start at (i0-4, j0-1): local (lx, ly) -> (lx+4, ly+1)
__device__ inline float te(const Stage &s, int c, int lx, int ly) {
    return s.E[c][(ly + 1) * EW + lx + 4];
}
__device__ inline float tb(const Stage &s, int c, int lx, int ly) {
    return s.B[c][(ly + 1) * BW + lx + 4];
}

// CPML position of one column of cells (fixed gi, gj for the whole z march):
// slab index along x and y (-1 outside) and the offsets of the cell's memory
// terms in the x-, y- and z-slab arrays for plane 0 / slab plane 0.  The
// slab arrays are [nz][ny][2P] (x), [nz][2P][nx] (y) and [2P][ny][nx] (z);
// the host keeps the TMA kernel to grids of fewer than 2^31 cells, so 32-bit
// offsets suffice.
struct ColPml {
    int sx, sy;
    int ox, oy, oz;
};

__device__ inline ColPml col_pml(const GridP &g, const FieldP &f, bool valid, int gi, int gj) {
    ColPml c;
    const int nx = g.n[0], ny = g.n[1], P = f.P;
    c.sx = (valid && f.pml[0]) ? slab_idx(gi, nx, P) : -1;
    c.sy = (valid && f.pml[1]) ? slab_idx(gj, ny, P) : -1;
    c.ox = gj * (2 * P) + c.sx;
    c.oy = c.sy * nx + gi;
    c.oz = gj * nx + gi;
    return c;
}

// per-plane strides of the three slab arrays
struct SlabStride {
    int x, y, z;
};

// CPML memory terms of one cell for one plane, loaded together at the start
// of the plane so that their latencies overlap.  Slot order per axis (see
// FieldP): x: E_y, E_z, B_y, B_z; y: E_x, E_z, B_x, B_z; z: E_x, E_y, B_x, B_y.
struct PsiCell {
    int idx[3];         // offset in the axis' slab arrays, or -1
    float v[3][4];      // psi_in values
};

template <int DIM>
__device__ inline void psi_load(const FieldP &f, const ColPml &cp, int k, int zs,
                                const SlabStride &st, PsiCell &pc) {
    pc.idx[0] = cp.sx >= 0 ? cp.ox + k * st.x : -1;
    pc.idx[1] = cp.sy >= 0 ? cp.oy + k * st.y : -1;
    pc.idx[2] = (DIM == 3 && zs >= 0) ? cp.oz + zs * st.z : -1;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q)
            pc.v[a][q] = pc.idx[a] >= 0 ? __ldg(f.psi_in[a][q] + pc.idx[a]) : 0.f;
}

// derivative + updated memory term, with psi_in preloaded
__device__ inline float cpml_pre(const FieldP &f, const PsiCell &pc, int a, int slot, int pos,
                                 bool half, float deriv) {
    if (pc.idx[a] < 0) return deriv;
    float b = half ? __ldg(f.cb_h[a] + pos) : __ldg(f.cb_e[a] + pos);
    float c = half ? __ldg(f.ca_h[a] + pos) : __ldg(f.ca_e[a] + pos);
    float psi = b * pc.v[a][slot] + c * deriv;
    f.psi_out[a][slot][pc.idx[a]] = psi;
    return deriv + psi;
}

// B^{n+1/2} of a halo cell (low-x column: comps 6, low-y row: comps 5) in a
// CPML plane: the memory terms are read, not advanced (their own CTA does that)
template <int DIM>
__device__ inline void compute_B_halo_pml(const GridP &g, const FieldP &f, const Stage &cur,
                                          const Stage &nxt, int lx, int ly, int gi, int gj, int k,
                                          int zs, const ColPml &cp, const SlabStride &st,
                                          int comps, float *out) {
    const float dt = g.dt;
    const int ix = cp.sx >= 0 ? cp.ox + k * st.x : -1;
    const int iy = cp.sy >= 0 ? cp.oy + k * st.y : -1;
    const int iz = (DIM == 3 && zs >= 0) ? cp.oz + zs * st.z : -1;
    auto term = [&](int a, int slot, int idx, int pos, float deriv) {
        if (idx < 0) return deriv;
        const float b = __ldg(f.cb_h[a] + pos), c = __ldg(f.ca_h[a] + pos);
        const float psi = b * __ldg(f.psi_in[a][slot] + idx) + c * deriv;
        return deriv + psi;
    };
    if (comps & 1) {  // B_x
        float dEz_dy = (te(cur, 2, lx, ly + 1) - te(cur, 2, lx, ly)) * g.inv_d[1];
        float t1 = term(1, 2, iy, gj, dEz_dy);
        float t2 = 0.f;
        if (DIM == 3) {
            float dEy_dz = (te(nxt, 1, lx, ly) - te(cur, 1, lx, ly)) * g.inv_d[2];
            t2 = term(2, 2, iz, k, dEy_dz);
        }
        out[0] = tb(cur, 0, lx, ly) - dt * (t1 - t2);
    }
    if (comps & 2) {  // B_y
        float t1 = 0.f;
        if (DIM == 3) {
            float dEx_dz = (te(nxt, 0, lx, ly) - te(cur, 0, lx, ly)) * g.inv_d[2];
            t1 = term(2, 3, iz, k, dEx_dz);
        }
        float dEz_dx = (te(cur, 2, lx + 1, ly) - te(cur, 2, lx, ly)) * g.inv_d[0];
        float t2 = term(0, 2, ix, gi, dEz_dx);
        out[1] = tb(cur, 1, lx, ly) - dt * (t1 - t2);
    }
    if (comps & 4) {  // B_z
        float dEy_dx = (te(cur, 1, lx + 1, ly) - te(cur, 1, lx, ly)) * g.inv_d[0];
        float dEx_dy = (te(cur, 0, lx, ly + 1) - te(cur, 0, lx, ly)) * g.inv_d[1];
        float t1 = term(0, 3, ix, gi, dEy_dx);
        float t2 = term(1, 3, iy, gj, dEx_dy);
        out[2] = tb(cur, 2, lx, ly) - dt * (t1 - t2);
    }
}

// B^{n+1/2} of an own cell in a CPML plane, memory terms preloaded
template <int DIM>
__device__ inline void compute_B_own_pml(const GridP &g, const FieldP &f, const Stage &cur,
                                         const Stage &nxt, int lx, int ly, int gi, int gj, int k,
                                         const PsiCell &pc, float *out) {
    const float dt = g.dt;
    float dEz_dy = (te(cur, 2, lx, ly + 1) - te(cur, 2, lx, ly)) * g.inv_d[1];
    float t1 = cpml_pre(f, pc, 1, 2, gj, true, dEz_dy);
    float t2 = 0.f;
    if (DIM == 3) {
        float dEy_dz = (te(nxt, 1, lx, ly) - te(cur, 1, lx, ly)) * g.inv_d[2];
        t2 = cpml_pre(f, pc, 2, 2, k, true, dEy_dz);
    }
    out[0] = tb(cur, 0, lx, ly) - dt * (t1 - t2);
    t1 = 0.f;
    if (DIM == 3) {
        float dEx_dz = (te(nxt, 0, lx, ly) - te(cur, 0, lx, ly)) * g.inv_d[2];
        t1 = cpml_pre(f, pc, 2, 3, k, true, dEx_dz);
    }
    float dEz_dx = (te(cur, 2, lx + 1, ly) - te(cur, 2, lx, ly)) * g.inv_d[0];
    t2 = cpml_pre(f, pc, 0, 2, gi, true, dEz_dx);
    out[1] = tb(cur, 1, lx, ly) - dt * (t1 - t2);
    float dEy_dx = (te(cur, 1, lx + 1, ly) - te(cur, 1, lx, ly)) * g.inv_d[0];
    float dEx_dy = (te(cur, 0, lx, ly + 1) - te(cur, 0, lx, ly)) * g.inv_d[1];
    t1 = cpml_pre(f, pc, 0, 3, gi, true, dEy_dx);
    t2 = cpml_pre(f, pc, 1, 3, gj, true, dEx_dy);
    out[2] = tb(cur, 2, lx, ly) - dt * (t1 - t2);
}

__device__ inline Stage stage_ptrs(unsigned char *smem, int slot) {
    Stage st;
    unsigned char *base = smem + (size_t)slot * STAGE;
    for (int c = 0; c < 3; ++c) {
        st.E[c] = reinterpret_cast<float *>(base + c * E_PAD);
        st.B[c] = reinterpret_cast<float *>(base + 3 * E_PAD + c * B_PAD);
        st.J[c] = reinterpret_cast<float *>(base + 3 * E_PAD + 3 * B_PAD + c * J_PAD);
    }
    return st;
}

// B^{n+1/2} at local (lx, ly) of plane k (global gi, gj, k in the domain).
// PML = false: no cell of the CTA's plane lies in a CPML slab, the memory
// terms vanish and the plain Yee update is used.
template <int DIM, bool PML>
__device__ inline void compute_B(const GridP &g, const FieldP &f, const Stage &cur,
                                 const Stage &nxt, int lx, int ly, int gi, int gj, int k, int comps,
                                 bool write_psi, float *out) {
    const float dt = g.dt;
    const long long px = PML ? psi_index(g, f, 0, gi, gj, k) : -1;
    const long long py = PML ? psi_index(g, f, 1, gi, gj, k) : -1;
    const long long pz = (PML && DIM == 3) ? psi_index(g, f, 2, gi, gj, k) : -1;
    if (comps & 1) {  // B_x at (i, j+1/2, k+1/2)
        float dEz_dy = (te(cur, 2, lx, ly + 1) - te(cur, 2, lx, ly)) * g.inv_d[1];
        float t1 = (PML ? cpml_term(f, 1, 2, py, gj, true, dEz_dy, write_psi) : dEz_dy);
        float t2 = 0.f;
        if (DIM == 3) {
            float dEy_dz = (te(nxt, 1, lx, ly) - te(cur, 1, lx, ly)) * g.inv_d[2];
            t2 = PML ? cpml_term(f, 2, 2, pz, k, true, dEy_dz, write_psi) : dEy_dz;
        }
        out[0] = tb(cur, 0, lx, ly) - dt * (t1 - t2);
    }
    if (comps & 2) {  // B_y at (i+1/2, j, k+1/2)
        float t1 = 0.f;
        if (DIM == 3) {
            float dEx_dz = (te(nxt, 0, lx, ly) - te(cur, 0, lx, ly)) * g.inv_d[2];
            t1 = PML ? cpml_term(f, 2, 3, pz, k, true, dEx_dz, write_psi) : dEx_dz;
        }
        float dEz_dx = (te(cur, 2, lx + 1, ly) - te(cur, 2, lx, ly)) * g.inv_d[0];
        float t2 = PML ? cpml_term(f, 0, 2, px, gi, true, dEz_dx, write_psi) : dEz_dx;
        out[1] = tb(cur, 1, lx, ly) - dt * (t1 - t2);
    }
    if (comps & 4) {  // B_z at (i+1/2, j+1/2, k)
        float dEy_dx = (te(cur, 1, lx + 1, ly) - te(cur, 1, lx, ly)) * g.inv_d[0];
        float dEx_dy = (te(cur, 0, lx, ly + 1) - te(cur, 0, lx, ly)) * g.inv_d[1];
        float t1 = PML ? cpml_term(f, 0, 3, px, gi, true, dEy_dx, write_psi) : dEy_dx;
        float t2 = PML ? cpml_term(f, 1, 3, py, gj, true, dEx_dy, write_psi) : dEx_dy;
        out[2] = tb(cur, 2, lx, ly) - dt * (t1 - t2);
    }
}

template <int DIM>
__global__ void __launch_bounds__(NT, 4)
    field_kernel_tma(GridP g, FieldP f, const __grid_constant__ TmaMaps maps, int cur_buf,
                     int *status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // 128-byte aligned base (the allocation carries 128 spare bytes)
    unsigned char *smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    float *sB = reinterpret_cast<float *>(smem + (size_t)S * STAGE);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)S * STAGE + SB_BYTES);
    __shared__ double s_src;
    __shared__ int s_abort;

    const int tx = threadIdx.x % BX, ty = threadIdx.x / BX;
    const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int i = i0 + tx, j = j0 + ty;
    const bool own = (i < nx) && (j < ny);
    const int k0 = DIM == 3 ? blockIdx.z * f.zchunk : 0;
    const int k1 = DIM == 3 ? min(k0 + f.zchunk, nz) : 1;
    const int kfirst = DIM == 3 ? k0 - 1 : 0;  // first plane loaded
    const int klast = DIM == 3 ? k1 : 0;       // last plane loaded
    const long long bflag = ((long long)blockIdx.z * f.nby + blockIdx.y) * f.nbx + blockIdx.x;
    const bool jdirty = !f.splitJ && f.jdirty[bflag] != 0;
    const bool fixx = g.per[0] && (i0 == 0 || i0 + BX >= nx);
    const bool fixy = g.per[1] && (j0 == 0 || j0 + BY >= ny);

    auto zplane = [&](int p) -> int {  // global z of plane p, or -1 outside a wall
        return DIM == 3 ? wrap_or_neg(p, nz, g.per[2]) : 0;
    };
    auto slot_of = [&](int p) { return (int)((unsigned)(p - kfirst) % S); };  // p >= kfirst
    auto parity_of = [&](int p) { return ((unsigned)(p - kfirst) / S) & 1u; };
    auto want_B = [&](int p) { return DIM == 2 || p < k1; };
    auto want_J = [&](int p) { return jdirty && (DIM == 2 || (p >= k0 && p < k1)); };

    auto issue = [&](int p) {  // thread 0 only
        const int slot = slot_of(p);
        Stage st = stage_ptrs(smem, slot);
        const bool wb = want_B(p), wj = want_J(p);
        const uint32_t bytes = 3 * E_BYTES + (wb ? 3 * B_BYTES : 0) + (wj ? 3 * J_BYTES : 0);
        mbar_expect_tx(&bars[slot], bytes);
        int zc = zplane(p);
        if (zc < 0) zc = p;  // outside a wall: the whole box is fill (zero)
        for (int c = 0; c < 3; ++c)
            tma_load_3d(st.E[c], &maps.E[cur_buf][c], i0 - 4, j0 - 1, zc, &bars[slot]);
        if (wb)
            for (int c = 0; c < 3; ++c)
                tma_load_3d(st.B[c], &maps.B[cur_buf][c], i0 - 4, j0 - 1, zc, &bars[slot]);
        if (wj)
            for (int c = 0; c < 3; ++c) tma_load_3d(st.J[c], &maps.J[c], i0, j0, zc, &bars[slot]);
    };

    // patch halo entries that lie across a periodic x / y face
    auto fixup = [&](int p) {
        if (!(fixx || fixy)) return;
        const int zz = zplane(p);
        if (zz < 0) return;
        Stage st = stage_ptrs(smem, slot_of(p));
        for (int e = threadIdx.x; e < EW * EH; e += NT) {
            const int gx = i0 - 4 + e % EW, gy = j0 - 1 + e / EW;
            const bool ox = gx < 0 || gx >= nx, oy = gy < 0 || gy >= ny;
            if (!(ox || oy) || (ox && !g.per[0]) || (oy && !g.per[1])) continue;
            const long long o = ((long long)zz * ny + wrap_or_neg(gy, ny, 1)) * nx +
                                wrap_or_neg(gx, nx, 1);
            for (int c = 0; c < 3; ++c) st.E[c][e] = __ldg(f.E[c] + o);
        }
        if (want_B(p)) {
            for (int e = threadIdx.x; e < BW * BH; e += NT) {
                const int gx = i0 - 4 + e % BW, gy = j0 - 1 + e / BW;
                const bool ox = gx < 0 || gx >= nx, oy = gy < 0 || gy >= ny;
                if (!(ox || oy) || (ox && !g.per[0]) || (oy && !g.per[1])) continue;
                const long long o = ((long long)zz * ny + wrap_or_neg(gy, ny, 1)) * nx +
                                    wrap_or_neg(gx, nx, 1);
                for (int c = 0; c < 3; ++c) st.B[c][e] = __ldg(f.B[c] + o);
            }
        }
        fence_proxy_async();  // generic writes before the stage is refilled by TMA
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        double v = 0.0;
        if (f.src_on) {
            long long n = *f.step_counter - (f.splitJ ? 0 : 1);
            double t = ((double)n + 0.5) * f.dt64 - f.src_t0;
            v = f.src_amp * exp(-2.0 * 0.6931471805599453 * t * t / (f.src_tau * f.src_tau)) *
                sin(f.src_omega * t);
        }
        s_src = v;
        s_abort = 0;
    }
    __syncthreads();
    int issued = kfirst - 1;  // meaningful in thread 0
    if (threadIdx.x == 0) {
        for (int p = kfirst; p <= klast && p < kfirst + S; ++p) {
            issue(p);
            issued = p;
        }
    }
    int waited = kfirst - 1;

    // halo work items: column lx = -1 (B_z, B_y) and row ly = -1 (B_z, B_x)
    const int hid = threadIdx.x;
    const bool halo_col = hid < BY;
    const bool halo_row = hid >= BY && hid < BY + BX;
    const int hlx = halo_col ? -1 : hid - BY, hly = halo_col ? hid : -1;
    const int hgi = wrap_or_neg(i0 + hlx, nx, g.per[0]);
    const int hgj = wrap_or_neg(j0 + hly, ny, g.per[1]);
    const bool halo_valid = (halo_col && j0 + hly < ny && hgi >= 0) ||
                            (halo_row && i0 + hlx < nx && hgj >= 0);

    // CPML decisions: the halo work takes the CPML path when any cell the CTA
    // reads lies in an x or y slab (CTA-uniform); an own row (one warp) when
    // the CTA's columns touch an x slab or the row lies in a y slab; every
    // plane of a z slab takes it for all.  Cells outside every slab compute
    // the same values on either path.
    const int P = f.P;
    const bool xyslab = (f.pml[0] && (i0 - 1 < P || i0 + BX > nx - P)) ||
                        (f.pml[1] && (j0 - 1 < P || j0 + BY > ny - P));
    const bool x_own = f.pml[0] && (i0 < P || i0 + BX > nx - P);
    const bool y_own = f.pml[1] && (j < P || j >= ny - P);  // warp-uniform: j = j0 + warp
    const ColPml cp_own = col_pml(g, f, own, i, j);
    const ColPml cp_halo = col_pml(g, f, halo_valid, hgi, hgj);
    const SlabStride sst{ny * 2 * P, 2 * P * nx, nx * ny};

    float Bx_prev = 0.f, By_prev = 0.f;
    bool ok = true;
    if (DIM == 3) {
        ok = mbar_wait(&bars[slot_of(kfirst)], parity_of(kfirst)) &&
             mbar_wait(&bars[slot_of(k0)], parity_of(k0));
        if (!ok) s_abort = 1;
        else {
            fixup(kfirst);
            fixup(k0);
        }
        waited = k0;
        __syncthreads();
        if (!s_abort) {
            const int km1 = zplane(kfirst);
            if (own && km1 >= 0) {
                float b[3];
                compute_B<DIM, true>(g, f, stage_ptrs(smem, slot_of(kfirst)),
                                     stage_ptrs(smem, slot_of(k0)), tx, ty, i, j, km1, 3, false, b);
                Bx_prev = b[0];
                By_prev = b[1];
            }
        }
    }

    for (int k = k0; k < k1 && !s_abort; ++k) {
        if (DIM == 3) {
            if (!mbar_wait(&bars[slot_of(k + 1)], parity_of(k + 1))) s_abort = 1;
            else fixup(k + 1);
            waited = k + 1;
        } else {
            if (!mbar_wait(&bars[slot_of(0)], parity_of(0))) s_abort = 1;
            else fixup(0);
            waited = 0;
        }
        __syncthreads();  // A: stage k+1 ready; iteration k-1 finished
        if (s_abort) break;
        if (DIM == 3 && threadIdx.x == 0 && k - 1 + S <= klast && k - 1 + S > issued) {
            issue(k - 1 + S);  // refill the slot plane k-1 used
            issued = k - 1 + S;
        }
        const Stage sc = stage_ptrs(smem, slot_of(k));
        const Stage sn = DIM == 3 ? stage_ptrs(smem, slot_of(k + 1)) : sc;
        const long long o = ((long long)k * ny + j) * nx + i;
        const int zs = (DIM == 3 && f.pml[2]) ? slab_idx(k, nz, P) : -1;  // uniform
        const bool own_pml = x_own || y_own || zs >= 0;                     // warp-uniform
        float bown[3] = {0.f, 0.f, 0.f};
        PsiCell pc;
        if (own_pml) {
            if (own) {
                psi_load<DIM>(f, cp_own, k, zs, sst, pc);
                compute_B_own_pml<DIM>(g, f, sc, sn, tx, ty, i, j, k, pc, bown);
            }
        } else if (own) {
            compute_B<DIM, false>(g, f, sc, sn, tx, ty, i, j, k, 7, true, bown);
        }
        if (own) {
            f.Bn[0][o] = bown[0];
            f.Bn[1][o] = bown[1];
            f.Bn[2][o] = bown[2];
        }
        sB[(0 * (BY + 1) + ty + 1) * (BX + 1) + tx + 1] = bown[0];
        sB[(1 * (BY + 1) + ty + 1) * (BX + 1) + tx + 1] = bown[1];
        sB[(2 * (BY + 1) + ty + 1) * (BX + 1) + tx + 1] = bown[2];
        if (halo_col || halo_row) {
            float hb[3] = {0.f, 0.f, 0.f};
            if (halo_valid) {
                if (xyslab || zs >= 0)
                    compute_B_halo_pml<DIM>(g, f, sc, sn, hlx, hly, hgi, hgj, k, zs, cp_halo, sst,
                                            halo_col ? 6 : 5, hb);
                else
                    compute_B<DIM, false>(g, f, sc, sn, hlx, hly, hgi, hgj, k, halo_col ? 6 : 5,
                                          false, hb);
            }
            for (int c = 0; c < 3; ++c) sB[(c * (BY + 1) + hly + 1) * (BX + 1) + hlx + 1] = hb[c];
        }
        __syncthreads();  // B: sB of plane k complete
        if (own) {
            auto SB = [&](int c, int ly, int lx) {
                return sB[(c * (BY + 1) + ly + 1) * (BX + 1) + lx + 1];
            };
            float jx = 0.f, jy = 0.f, jz = 0.f;
            if (jdirty) {
                jx = sc.J[0][ty * JW + tx];
                jy = sc.J[1][ty * JW + tx];
                jz = sc.J[2][ty * JW + tx];
                if (!f.keepJ) {
                    f.J[0][o] = 0.f;
                    f.J[1][o] = 0.f;
                    f.J[2][o] = 0.f;
                }
            }
            if (f.src_on) {
                const int pos = f.inc == 0 ? i : (f.inc == 1 ? j : k);
                if (pos == f.src_index) {
                    const float sv = (float)s_src;
                    if (f.pol == 0) jx += sv;
                    else if (f.pol == 1) jy += sv;
                    else jz += sv;
                }
            }
            const float bx = SB(0, ty, tx), by = SB(1, ty, tx), bz = SB(2, ty, tx);
            float tExy = (bz - SB(2, ty - 1, tx)) * g.inv_d[1];
            float tExz = 0.f, tEyz = 0.f;
            if (DIM == 3) {
                tExz = (by - By_prev) * g.inv_d[2];
                tEyz = (bx - Bx_prev) * g.inv_d[2];
            }
            float tEyx = (bz - SB(2, ty, tx - 1)) * g.inv_d[0];
            float tEzx = (by - SB(1, ty, tx - 1)) * g.inv_d[0];
            float tEzy = (bx - SB(0, ty - 1, tx)) * g.inv_d[1];
            if (own_pml) {
                tExy = cpml_pre(f, pc, 1, 0, j, false, tExy);
                if (DIM == 3) {
                    tExz = cpml_pre(f, pc, 2, 0, k, false, tExz);
                    tEyz = cpml_pre(f, pc, 2, 1, k, false, tEyz);
                }
                tEyx = cpml_pre(f, pc, 0, 0, i, false, tEyx);
                tEzx = cpml_pre(f, pc, 0, 1, i, false, tEzx);
                tEzy = cpml_pre(f, pc, 1, 1, j, false, tEzy);
            }
            f.En[0][o] = te(sc, 0, tx, ty) + f.c2dt * (tExy - tExz) - f.dt_eps0 * jx;
            f.En[1][o] = te(sc, 1, tx, ty) + f.c2dt * (tEyz - tEyx) - f.dt_eps0 * jy;
            f.En[2][o] = te(sc, 2, tx, ty) + f.c2dt * (tEzx - tEzy) - f.dt_eps0 * jz;
            Bx_prev = bx;
            By_prev = by;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_abort) {
            atomicOr(status, kStatusTimeout);
            // let the copies still in flight land before the CTA's memory goes
            for (int p = waited + 1; p <= issued; ++p) mbar_wait(&bars[slot_of(p)], parity_of(p));
        }
        if (jdirty) f.jdirty_clear[bflag] = 0;
    }
}


// ---------------------------------------------------------------------------
// The B pass of the split update, TMA-fed:
//   B^{n+1/2} = B^{n-1/2} - dt curl E^n
// on the blocks field_b_tma_block admits (no CPML slab, no halo to wrap).
// One elected thread streams the planes k0 .. k1 of the E^n tile (40 x 10:
// the own columns and their +x / +y neighbours) and planes k0 .. k1 - 1 of
// the B^{n-1/2} tile into a ring of SBP stages; a stage is refilled once every
// thread has arrived on its "empty" barrier after the plane that reads it
// last.  The copies in flight wait in shared memory, not in registers, so the
// pass keeps its bandwidth with one resident CTA per SM, e.g. beside the
// particle phase.  Every wait is bounded as in the fused kernel.
// ---------------------------------------------------------------------------

constexpr int SBP = 5;                        // stages
constexpr int BSTAGE = 3 * (E_PAD + B_PAD);   // bytes per stage

__device__ inline void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__global__ void __launch_bounds__(NT) field_b_kernel_tma(GridP g, FieldP f,
                                                         const __grid_constant__ TmaMaps maps,
                                                         int cur_buf, int *status) {
    int bx = blockIdx.x, by = blockIdx.y, bz = blockIdx.z;
    if (f.blk[0]) field_list_block(f, 0, bx, by, bz);
    else if (!field_b_tma_block(g, f, bx, by, bz)) return;  // CTA-uniform
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)SBP * BSTAGE);
    uint64_t *empty = full + SBP;
    __shared__ int s_abort;
    const int tx = threadIdx.x % BX, ty = threadIdx.x / BX;
    const int i0 = bx * BX, j0 = by * BY;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int k0 = bz * f.zchunk, k1 = min(k0 + f.zchunk, nz);
    const int np = k1 - k0 + 1;  // planes k0 .. k1; the top one for E only
    if (threadIdx.x == 0) {
        for (int s = 0; s < SBP; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NT);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    __syncthreads();
    auto issue = [&](int p) {  // thread 0 only
        const int s = p % SBP;
        int z = k0 + p;
        if (z >= nz && g.per[2]) z -= nz;  // beyond a wall the box is fill (zero)
        unsigned char *base = smem + (size_t)s * BSTAGE;
        const bool wb = p < np - 1;
        mbar_expect_tx(&full[s], 3 * E_BYTES + (wb ? 3 * B_BYTES : 0));
        for (int c = 0; c < 3; ++c)
            tma_load_3d(base + c * E_PAD, &maps.E[cur_buf][c], i0 - 4, j0 - 1, z, &full[s]);
        if (wb)
            for (int c = 0; c < 3; ++c)
                tma_load_3d(base + 3 * E_PAD + c * B_PAD, &maps.B[cur_buf][c], i0 - 4, j0 - 1, z,
                            &full[s]);
    };
    int issued = -1, waited = -1;
    if (threadIdx.x == 0)
        for (int p = 0; p < np && p < SBP; ++p) {
            issue(p);
            issued = p;
        }
    const float dt = g.dt, idx_ = g.inv_d[0], idy = g.inv_d[1], idz = g.inv_d[2];
    const int e = (ty + 1) * EW + tx + 4, b = (ty + 1) * BW + tx + 4;
    const long long pl = (long long)nx * ny;
    long long o = ((long long)k0 * ny + j0 + ty) * nx + i0 + tx;
    const long long lim = f.wait_polls;
    bool ok = mbar_wait(&full[0], 0, lim);
    if (ok) waited = 0;
    for (int p = 0; ok && p < np - 1; ++p, o += pl) {
        const int s = p % SBP, s1 = (p + 1) % SBP;
        if (!mbar_wait(&full[s1], ((p + 1) / SBP) & 1, lim)) {
            ok = false;
            break;
        }
        waited = p + 1;
        const float *E = reinterpret_cast<const float *>(smem + (size_t)s * BSTAGE);
        const float *Ek = reinterpret_cast<const float *>(smem + (size_t)s1 * BSTAGE);
        const float *Bt = reinterpret_cast<const float *>(smem + (size_t)s * BSTAGE + 3 * E_PAD);
        const int ep = E_PAD / 4, bp = B_PAD / 4;  // component stride in floats
        const float ex = E[e], ey = E[ep + e], ez = E[2 * ep + e];
        const float dEz_dy = (E[2 * ep + e + EW] - ez) * idy;
        const float dEx_dy = (E[e + EW] - ex) * idy;
        const float dEz_dx = (E[2 * ep + e + 1] - ez) * idx_;
        const float dEy_dx = (E[ep + e + 1] - ey) * idx_;
        const float dEy_dz = (Ek[ep + e] - ey) * idz;
        const float dEx_dz = (Ek[e] - ex) * idz;
        const float bx = Bt[b], by = Bt[bp + b], bz = Bt[2 * bp + b];
        f.Bn[0][o] = bx - dt * (dEz_dy - dEy_dz);
        f.Bn[1][o] = by - dt * (dEx_dz - dEz_dx);
        f.Bn[2][o] = bz - dt * (dEy_dx - dEx_dy);
        // plane p is the last reader of stage s: release it, refill it
        mbar_arrive(&empty[s]);
        if (threadIdx.x == 0 && p + SBP < np) {
            if (!mbar_wait(&empty[s], (p / SBP) & 1, lim)) {
                ok = false;
                s_abort = 1;
                break;
            }
            issue(p + SBP);
            issued = p + SBP;
        }
    }
    if (!ok) s_abort = 1;
    __syncthreads();
    if (threadIdx.x == 0 && s_abort) {
        atomicOr(status, kStatusTimeout);
        // let the copies still in flight land before the CTA's memory goes
        for (int p = waited + 1; p <= issued; ++p) mbar_wait(&full[p % SBP], (p / SBP) & 1);
    }
}

}  // namespace

size_t field_tma_smem_bytes() { return (size_t)S * STAGE + SB_BYTES + S * 8 + 128; }

cudaError_t field_tma_setup() {
    cudaError_t e = cudaFuncSetAttribute(field_kernel_tma<3>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)field_tma_smem_bytes());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(field_kernel_tma<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)field_tma_smem_bytes());
}

size_t field_b_tma_smem_bytes() { return (size_t)SBP * BSTAGE + 2 * SBP * 8 + 128; }

cudaError_t launch_field_b_tma(const GridP &g, const FieldP &f, const TmaMaps &maps, int cur_buf,
                               int *status, cudaStream_t s) {
    if (!f.tma_b || g.dims != 3) return cudaSuccess;
    if (f.blk[0]) {
        if (f.nblk[0] > 0)
            field_b_kernel_tma<<<f.nblk[0], NT, field_b_tma_smem_bytes(), s>>>(g, f, maps, cur_buf,
                                                                               status);
        return cudaGetLastError();
    }
    dim3 grid((g.n[0] + BX - 1) / BX, (g.n[1] + BY - 1) / BY, (g.n[2] + f.zchunk - 1) / f.zchunk);
    field_b_kernel_tma<<<grid, NT, field_b_tma_smem_bytes(), s>>>(g, f, maps, cur_buf, status);
    return cudaGetLastError();
}

cudaError_t launch_field_tma(const GridP &g, const FieldP &f, const TmaMaps &maps, int cur_buf,
                             int *status, cudaStream_t s) {
    dim3 block(NT);
    const size_t smem = field_tma_smem_bytes();
    if (g.dims == 3) {
        dim3 grid((g.n[0] + BX - 1) / BX, (g.n[1] + BY - 1) / BY, (g.n[2] + f.zchunk - 1) / f.zchunk);
        field_kernel_tma<3><<<grid, block, smem, s>>>(g, f, maps, cur_buf, status);
    } else {
        dim3 grid((g.n[0] + BX - 1) / BX, (g.n[1] + BY - 1) / BY, 1);
        field_kernel_tma<2><<<grid, block, smem, s>>>(g, f, maps, cur_buf, status);
    }
    return cudaGetLastError();
}

// Tensor maps of every field array: FP32 [nz][ny][nx], strides nx*4 and
// nx*ny*4 bytes (hence nx % 4 == 0), zero fill outside the tensor.
bool encode_field_maps(const GridP &g, float *const E[2][3], float *const B[2][3],
                       float *const J[3], TmaMaps *maps) {
    if (g.n[0] % 4 != 0) return false;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[3] = {(cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2]};
    const cuuint64_t strides[2] = {(cuuint64_t)g.n[0] * 4, (cuuint64_t)g.n[0] * g.n[1] * 4};
    const cuuint32_t estr[3] = {1, 1, 1};
    auto enc = [&](CUtensorMap *m, float *base, cuuint32_t bw, cuuint32_t bh) {
        const cuuint32_t box[3] = {bw, bh, 1};
        return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    for (int b = 0; b < 2; ++b)
        for (int c = 0; c < 3; ++c) {
            if (!enc(&maps->E[b][c], E[b][c], EW, EH)) return false;
            if (!enc(&maps->B[b][c], B[b][c], BW, BH)) return false;
        }
    for (int c = 0; c < 3; ++c)
        if (!enc(&maps->J[c], J[c], JW, JH)) return false;
    return true;
}

}  // namespace pic
