// pic_internal.cuh -- device-side data layout and kernel parameter blocks of
// the PIC step.  Shared by the CUDA translation units of libpic.so only.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pic.h"

namespace pic {

// SI constants (exact c; eps0 from CODATA 2018; mu0 from c and eps0).
constexpr double kC = 299792458.0;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kKB = 1.380649e-23;
constexpr double kPi = 3.14159265358979323846;

// Particle cells are packed (x | y << 11 | z << 22): no integer division in
// the hot loop.  Hence nx, ny <= 2048 and nz <= 1024.
constexpr int kPackBitsX = 11, kPackBitsY = 11;
__host__ __device__ inline uint32_t pack_cell(int x, int y, int z) {
    return (uint32_t)x | ((uint32_t)y << kPackBitsX) | ((uint32_t)z << (kPackBitsX + kPackBitsY));
}
__host__ __device__ inline int cell_x(uint32_t c) { return (int)(c & 2047u); }
__host__ __device__ inline int cell_y(uint32_t c) { return (int)((c >> 11) & 2047u); }
__host__ __device__ inline int cell_z(uint32_t c) { return (int)(c >> 22); }

// Device status word bits (latched, read at sync points).
enum : int { kStatusBounds = 1, kStatusTimeout = 2 };

// Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw, SC'11):
// ten rounds of the Philox S-box on the counter x with key (k0, k1).
__device__ inline void philox4x32_10(uint32_t *x, uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, x[0]), lo0 = 0xD2511F53u * x[0];
        uint32_t hi1 = __umulhi(0xCD9E8D57u, x[2]), lo1 = 0xCD9E8D57u * x[2];
        uint32_t y0 = hi1 ^ x[1] ^ k0, y2 = hi0 ^ x[3] ^ k1;
        x[0] = y0;
        x[1] = lo1;
        x[2] = y2;
        x[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Fourth counter word of the diffuse-reflection draws (particle id, step,
// species, kDiffuseStream).
constexpr uint32_t kDiffuseStream = 0x44494655u;

struct GridP {
    int dims;
    int n[3];
    int per[3];          // 1 = periodic axis
    float d[3];          // cell size (m)
    float inv_d[3];
    float dt;
    long long ncell;
};

// Per-species parameters of the particle kernel (FP32 coefficients are
// formed on the host in FP64 and rounded once).
struct SpeciesP {
    int kind;
    long long n;
    uint32_t *cell;               // packed cell (anchor cell for bound)
    float *o[3];                  // in-cell offset (free, Dirac)
    float *v[3];                  // velocity (m/s)
    const double *anchor[3];      // bound: anchor offset in [0,1), FP64 (the stored rest position)
    const float *anchor32[3];     // bound: the same offset rounded to FP32 (read by the step)
    float *disp[3];               // bound: displacement from the anchor (m)
    const int *tile_start;        // [ntiles + 1]
    float hq;                     // q dt / (2 m)
    float hw0sq[3];               // (dt/2) omega0^2 per axis
    float gdt2;                   // gamma dt / 2 (isotropic gamma)
    float gdt2v[3];               // gamma_a dt / 2 per axis
    int aniso;                    // bound with unequal gamma entries: the general solve
    float hw0off[3];              // (dt/2) x off-diagonal binding tensor entries (xy, xz, yz)
    int tensor;                   // bound with a full binding tensor
    float vF;
    float dt;
    float dtd[3];                 // dt / d_a
    float jfac[3];                // Esirkepov factors -q w / (d_b d_c dt); 2D J_z: q w / V
    unsigned long long *nrefl;    // device reflection counter
    const uint32_t *pid;          // particle id (load order), keys the diffuse draws
};

struct FieldP {
    const float *E[3];   // E^n (read)
    const float *B[3];   // B^{n-1/2} (read)
    float *En[3];        // E^{n+1} (write)
    float *Bn[3];        // B^{n+1/2} (write)
    float *J[3];         // J^{n+1/2}, zeroed after use unless keepJ
    const uint8_t *jdirty;   // field-block flags: J may be non-zero
    uint8_t *jdirty_clear;   // same array, cleared after use
    // CPML: per PML axis a, slab arrays psi[a][c] (c = 0..3) ping-pong
    //   axis x: E_y, E_z, B_y, B_z ; axis y: E_x, E_z, B_x, B_z ; axis z: E_x, E_y, B_x, B_y
    const float *psi_in[3][4];
    float *psi_out[3][4];
    int pml[3];          // 1 = PML axis
    int P;               // slab thickness
    const float *cb_e[3], *ca_e[3], *cb_h[3], *ca_h[3];   // per-axis coefficients (length n_a)
    // source
    int src_on, inc, pol, src_index;
    double src_amp;      // -2 E0 / (eta0 d_inc)
    double src_omega, src_tau, src_t0;
    const long long *step_counter;   // particle phases completed (step n -> n + 1)
    int src_host;        // 1: src_val holds this step's source current (set by the host)
    float src_val;
    double dt64;
    float c2dt;          // c^2 dt
    float dt_eps0;       // dt / eps0
    int keepJ;
    int splitJ;          // 1: J is applied by the separate current pass (overlapped step):
                         //    the update ignores J and the block flags, and the step
                         //    counter has not advanced yet when it runs
    int zchunk;
    int nbx, nby, nbz;   // field-block grid (for jdirty)
    int tma_b;           // 1: the TMA-fed B pass takes the blocks field_b_tma_block admits
    long long wait_polls;  // bounded waits of the TMA-fed passes (kWaitPolls by default)
    const float *inv_eps;  // 1 / eps_r per cell (Eq. consteps) for the fused update, null: vacuum
    // Compact lists of field blocks (linear index (bz * nby + by) * nbx + bx),
    // so that each launch of the split passes runs its own blocks only:
    // [0] the TMA-fed B pass's, [1] the other blocks without a CPML slab,
    // [2] the blocks with one, [3] all blocks without one.  blk[0] null:
    // every launch covers the whole block grid and skips the others' blocks.
    const int *blk[4];
    int nblk[4];
};

// Polls of a bounded mbarrier wait before it gives up (~0.5 s with the
// back-off); the drain of copies in flight always uses this bound.
constexpr long long kWaitPolls = 1LL << 23;

constexpr int kFieldBX = 32, kFieldBY = 8;

// Field blocks (32 x 8 columns x zchunk planes) that the TMA-fed B pass
// updates when it is on: 3D, no cell in a CPML slab, and the +x / +y
// neighbour columns inside the grid (no halo to wrap).  The scalar B pass
// skips exactly these.
__host__ __device__ inline bool field_b_tma_block(const GridP &g, const FieldP &f, int bx, int by,
                                                  int bz) {
    if (!f.tma_b || g.dims != 3) return false;
    const int i0 = bx * kFieldBX, j0 = by * kFieldBY, k0 = bz * f.zchunk;
    const int k1 = k0 + f.zchunk < g.n[2] ? k0 + f.zchunk : g.n[2];
    if (i0 + kFieldBX >= g.n[0] || j0 + kFieldBY >= g.n[1]) return false;
    const int P = f.P;
    const bool pml = (f.pml[0] && (i0 < P || i0 + kFieldBX > g.n[0] - P)) ||
                     (f.pml[1] && (j0 < P || j0 + kFieldBY > g.n[1] - P)) ||
                     (f.pml[2] && (k0 < P || k1 > g.n[2] - P));
    return !pml;
}

// Does field block (bx, by, bz) hold a cell of a CPML slab?
__host__ __device__ inline bool field_block_pml(const GridP &g, const FieldP &f, int bx, int by,
                                                int bz) {
    const int P = f.P;
    const int i0 = bx * kFieldBX, j0 = by * kFieldBY;
    bool r = (f.pml[0] && (i0 < P || i0 + kFieldBX > g.n[0] - P)) ||
             (f.pml[1] && (j0 < P || j0 + kFieldBY > g.n[1] - P));
    if (g.dims == 3 && f.pml[2]) {
        const int k0 = bz * f.zchunk, k1 = k0 + f.zchunk < g.n[2] ? k0 + f.zchunk : g.n[2];
        r = r || k0 < P || k1 > g.n[2] - P;
    }
    return r;
}

// Block (bx, by, bz) of a launch over the compact list `kind`
__device__ inline void field_list_block(const FieldP &f, int kind, int &bx, int &by, int &bz) {
    const int q = f.blk[kind][blockIdx.x];
    bx = q % f.nbx;
    by = (q / f.nbx) % f.nby;
    bz = q / (f.nbx * f.nby);
}

// Particle tiling.
struct TileP {
    int T[3];        // tile dims (cells)
    int nt[3];       // tiles per axis
    int ntiles;
    int box[3];      // staged box dims = T + 5 (3D) / T + 5, T + 5, 1 (2D); T + 7 for TSC
    int boxn;        // product
};

constexpr int kMaxSpecies = PIC_MAX_SPECIES;

struct ParticleLaunch {
    GridP g;
    TileP tp;
    int nsp;
    SpeciesP sp[kMaxSpecies];
    const float *E[3];
    const float *B[3];       // B^{n-1/2}
    float *J[3];
    const uint8_t *mask;     // may be null (all material, or open material edges)
    // particle boundary variants (Sec. 3); read by the extended kernel only
    const float *Eext[3];    // external field on the E stagger, null: none
    float p_diffuse;         // probability of a diffuse material-edge reflection
    uint32_t diff_key[2];    // Philox key of the diffuse draws
    uint32_t rng_step;       // step index of this particle phase (mod 2^32)
    int shape;               // free / Dirac shape order: 1 CIC, 2 TSC (bound: CIC)
    uint8_t *jdirty;
    int nbx, nby, nbz, zchunk;
    const int *active;       // active tile list, largest particle count first
    const int *nactive;
    int *sched;              // [2]: next list entry to take, CTAs finished (reset by the last)
    long long *step_counter;
    int *status;
    // lean kernel (k_particle_lean.cu): particles deferred to the global list
    // as (species, index), capacity the simulation's particle count; its
    // length; the finished-CTA count of the kernel that completes it.  Null
    // defer: the lean kernel is not used.
    int2 *defer;
    int *defer_count;
    int *defer_sched;
};

// Let `func` take as much dynamic shared memory as the device allows (the
// opt-in limit less its static shared memory).  The limit is a property of
// the function, shared by every simulation of the process: setting it to one
// simulation's size would refuse the launches of another with a larger box.
template <class F>
inline cudaError_t allow_max_dynamic_smem(F *func) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes a{};
    e = cudaFuncGetAttributes(&a, func);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)a.sharedSizeBytes);
}

// TMA descriptors of the field arrays (ping-pong E and B, J)
struct TmaMaps {
    CUtensorMap E[2][3];
    CUtensorMap B[2][3];
    CUtensorMap J[3];
};

// ---------------------------------------------------------------------------
// host-side launch wrappers (defined in the kernel translation units)
// ---------------------------------------------------------------------------
cudaError_t launch_field(const GridP &g, const FieldP &f, cudaStream_t s);
cudaError_t launch_field_b(const GridP &g, const FieldP &f, cudaStream_t s);
// inv_eps: 1 / eps_r per cell (Eq. consteps), or null: vacuum
cudaError_t launch_field_e(const GridP &g, const FieldP &f, const float *inv_eps, cudaStream_t s);
cudaError_t launch_field_stream(const GridP &g, const FieldP &f, cudaStream_t s);
// E^{n+1} -= (dt / eps0) J (x 1/eps_r where inv_eps is set) over the flagged
// blocks, J and the flags cleared; counter advanced (the step's particle phase ran)
cudaError_t launch_japply(const GridP &g, const FieldP &f, const float *inv_eps, long long *counter,
                          cudaStream_t s);
cudaError_t launch_batch_field(int dims, const GridP *grids, const FieldP *fdescs, const int *fpar,
                               const int *active, const int4 *items, int nitems, cudaStream_t s);
bool encode_field_maps(const GridP &g, float *const E[2][3], float *const B[2][3],
                       float *const J[3], TmaMaps *maps);
cudaError_t field_tma_setup();
size_t field_tma_smem_bytes();
cudaError_t launch_field_b_tma(const GridP &g, const FieldP &f, const TmaMaps &maps, int cur_buf,
                               int *status, cudaStream_t s);
cudaError_t launch_field_tma(const GridP &g, const FieldP &f, const TmaMaps &maps, int cur_buf,
                             int *status, cudaStream_t s);
cudaError_t launch_particles(const ParticleLaunch &pl, int nctas, size_t smem, cudaStream_t s);
// ext: launch the batch kernel with the boundary variants and the
// anisotropic bound push (some member has one); shape 2: the TSC batch
// kernel (the group's members all have TSC shapes); done: the members'
// device step counts (the diffuse draws' step index)
cudaError_t launch_batch_particles(int dims, const ParticleLaunch *descs, const int *fpar,
                                  const int *active, const int2 *items, int nitems, int *sched,
                                  const long long *done, int nctas, size_t smem, bool ext,
                                  int shape, cudaStream_t s);
size_t particle_smem_bytes(const TileP &tp);
// the lean 3D CIC kernel of the default tile (k_particle_lean.cu): whether a
// launch can take it, its shared-memory limit, and the launch of it plus the
// kernel that completes the particles it deferred (two launches)
bool particle_lean_fits(const ParticleLaunch &pl);
cudaError_t particle_lean_setup();
cudaError_t launch_particles_lean(const ParticleLaunch &pl, int nctas, int ndefer_ctas,
                                  cudaStream_t s);
// kernels one launch_particles call starts
inline int particle_launches(const ParticleLaunch &pl) { return particle_lean_fits(pl) ? 2 : 1; }
// ctas_per_sm: the plain kernel; ctas_per_sm_ext: the one with the boundary
// variants (external field, diffuse reflection)
cudaError_t particle_kernel_setup(int dims, size_t smem, int *ctas_per_sm, int *ctas_per_sm_ext,
                                  int *ctas_per_sm_tsc = nullptr);
// true when the launch needs the kernel with the boundary variants (or the
// anisotropic bound push)
inline bool particle_launch_ext(const ParticleLaunch &pl) {
    bool aniso = false;
    for (int i = 0; i < pl.nsp; ++i) aniso = aniso || pl.sp[i].aniso || pl.sp[i].tensor;
    return pl.Eext[0] != nullptr || pl.p_diffuse > 0.f || aniso;
}

// boundary variants (k_boundary.cu): the work-function barrier field of
// height W_eV from the mask (null: all material) into E[3] on the E stagger
cudaError_t launch_work_function(const GridP &g, const uint8_t *mask, double W_eV,
                                 float *const E[3], cudaStream_t s);

// sort (k_sort.cu)
cudaError_t launch_tile_histogram(const GridP &g, const TileP &tp, const uint32_t *cell,
                                  long long n, int *count, int *rank, cudaStream_t s);
cudaError_t launch_scan_int(const int *in, int *out_excl, long long n, int *tmp,
                            long long tmp_len, cudaStream_t s);
long long scan_tmp_len(long long n);
int scan_kernel_count(long long n);
cudaError_t launch_tile_scatter(const GridP &g, const TileP &tp, const SpeciesP &src,
                                const uint32_t *pid_src, SpeciesP &dst, uint32_t *pid_dst,
                                const int *start, const int *rank, bool spread, cudaStream_t s);
// cell-interleaved order inside each tile, in chunks of `chunk` cells (src
// tile-grouped -> dst); rank: per-particle scratch
cudaError_t launch_tile_interleave(const TileP &tp, const SpeciesP &src, const uint32_t *pid_src,
                                   SpeciesP &dst, uint32_t *pid_dst, const int *start, int *rank,
                                   int chunk, cudaStream_t s);
// threads of a particle-kernel CTA (the chunk of the interleaved order)
constexpr int kParticleThreads = 256;
long long active_tiles_work_len(long long ntiles);
int active_tiles_kernel_count(long long ntiles);
cudaError_t launch_active_tiles_work(const TileP &tp, const int *const *starts_dev, int nsp,
                                     int *active, int *nactive, int *work, cudaStream_t s);
cudaError_t launch_cell_histogram(const GridP &g, const SpeciesP &sp, int *counts,
                                  cudaStream_t s);

// batch engine (k_batch.cu)
struct SortSeg {           // one mobile species of one member
    SpeciesP src;          // its current buffer (sorted in place)
    SpeciesP tmp;          // its other buffer, scratch
    const uint32_t *pid_src;
    uint32_t *pid_tmp;
    TileP tp;
    int *count;            // [ntiles + 1] scratch
    int *tile_start;       // [ntiles + 1]
    int *rank;             // this segment's part of the rank scratch
    long long poff;        // first particle of the segment in the batch index space
};
struct SimTiles {          // one member for the active-tile item list
    int sim, ntiles, nsp, ioff;
    const int *starts[kMaxSpecies];
};
cudaError_t launch_begin_step(int n, const int *member, int *active, int *fpar, long long *done,
                              const long long *target, long long *const *counters, cudaStream_t s);
cudaError_t launch_finalize(int n, int *active, int *fpar, long long *done, cudaStream_t s);
cudaError_t launch_batch_sort(const SortSeg *segs, int nseg, long long total, cudaStream_t s,
                              int *nlaunch);
cudaError_t launch_batch_items(const SimTiles *sims, int nsims, int2 *items, cudaStream_t s);

// loader (k_fd.cu)
struct FDRequest {
    int kind, dims, ppc, quiet;
    double m, mu, kT, vF;
    uint64_t seed;
    uint32_t stream;
};
constexpr int kFDPanels = 4096;
double fd_pmax(const FDRequest &r);
cudaError_t launch_fd_table(const FDRequest &r, double *table, double pmax, cudaStream_t s);
cudaError_t launch_fd_particles(const GridP &g, const FDRequest &r, const int *mat_cells,
                                long long np, const double *table, double pmax, SpeciesP out,
                                uint32_t *pid, cudaStream_t s);
cudaError_t launch_material_cells(const GridP &g, const uint8_t *mask, const int *rank,
                                  int *mat_cells, cudaStream_t s);
cudaError_t launch_mask_to_int(const uint8_t *mask, long long n, int *out, cudaStream_t s);

// diagnostics (k_diag.cu)
struct DiagAcc {
    double kinetic[kMaxSpecies];
    double e2, b2;
    unsigned long long gauss_max_bits, rho_max_bits;
    double gauss_sum2;
};
cudaError_t launch_kinetic(const SpeciesP &sp, double mw_half, double *acc, cudaStream_t s);
cudaError_t launch_energy_histogram(const SpeciesP &sp, double half_m, double e_max, int nbins,
                                    unsigned long long *out, cudaStream_t s);
cudaError_t launch_field_energy(const GridP &g, const float *const *E, const float *const *B,
                                DiagAcc *acc, cudaStream_t s);
// order: 1 CIC, 2 TSC
cudaError_t launch_rho_deposit(const GridP &g, const SpeciesP &sp, double qw_over_V, int order,
                               double *rho, cudaStream_t s);
cudaError_t launch_gauss(const GridP &g, const float *const *E, const float *inv_eps,
                         const double *rho, const double *rho_bg, DiagAcc *acc, cudaStream_t s);
cudaError_t launch_add_uniform(double *rho, long long n, double v, cudaStream_t s);

// readback helpers (k_diag.cu)
cudaError_t launch_unsort(const GridP &g, const SpeciesP &sp, const uint32_t *pid,
                          int32_t *cell_out, float *off_out, float *v_out, double *anchor_out,
                          float *disp_out, cudaStream_t s);
cudaError_t launch_pack_explicit(const GridP &g, long long n, const int32_t *cell_lin,
                                 uint32_t *cell_packed, uint32_t *pid, cudaStream_t s);
cudaError_t launch_f32_to_f64(const float *in, double *out, long long n, cudaStream_t s);
cudaError_t launch_f64_to_f32(const double *in, float *out, long long n, cudaStream_t s);

}  // namespace pic
