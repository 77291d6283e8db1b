/*
 * pic.h -- C ABI of the GB300-native particle-in-cell step for quantum
 * plasmas (Ngirmang, Do, Liu, Bosman & Wu, "Particle-In-Cell Simulations of
 * Quantum Plasmas", arXiv 2501.07465).
 *
 * One simulation = a Yee grid (E on integer steps, B on half steps, Sec. 4.1),
 * an optional material mask (Sec. 3) and up to PIC_MAX_SPECIES particle
 * species of three kinds:
 *   PIC_FREE  -- free carriers, Boris push (Appendix A.1, Eq. borisscheme),
 *                optionally loaded from a Fermi-Dirac law (Sec. 2, Eq. fddist);
 *   PIC_BOUND -- bound electrons on a damped harmonic tether (Sec. 4, Eq.
 *                modlorentz), modified Boris push (Appendix A.2);
 *   PIC_DIRAC -- massless Dirac carriers of a sheet in the x-y plane (Sec. 5):
 *                Boris push with the transverse mass, |v| renormalised to v_F.
 * A step gathers E^n and B^n to every particle (CIC, or TSC for free and
 * Dirac particles: pic_set_shape_order), pushes it, applies the surface rule
 * at the material edges (specular or diffuse reflection, or open edges, with
 * an optional work-function barrier: pic_set_particle_bc,
 * pic_set_work_function, pic_set_external_field), deposits the current with
 * Esirkepov's charge-conserving scheme and advances the fields with Yee FDTD
 * (CPML layers, a soft plane-wave current sheet and a per-cell permittivity
 * optional).  Bound species may carry per-axis damping and a full binding
 * tensor (pic_set_binding_tensor).
 *
 * Conventions for every call:
 *  - Units are SI.  Cells are indexed x fastest: c = (k*ny + j)*nx + i.
 *  - Host pointers are owned by the caller and only read or written during
 *    the call.  Device state is owned by the simulation handle and freed by
 *    pic_destroy.
 *  - Calls never throw and never abort; they return a pic_status.  Work is
 *    enqueued on the simulation's stream; errors found on the device (a
 *    particle outside the domain, a wait that timed out) are latched and
 *    returned by the next pic_sync, pic_diagnostics, pic_read_* call.
 *  - A handle is not thread-safe: one host thread per handle at a time.
 *  - Precision: fields, velocities and in-cell offsets are FP32; cell indices
 *    int32; bound-particle anchors FP64; the loader's CDF inversion and the
 *    diagnostics reductions FP64.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_MAX_SPECIES 8

typedef enum pic_status {
    PIC_OK = 0,
    PIC_EINVAL = 1,    /* bad argument (size, kind, layout) */
    PIC_ENOMEM = 2,    /* device allocation failed */
    PIC_EDTLIMIT = 3,  /* dt violates the stability limit of Eq. dtlimit */
    PIC_ECUDA = 4,     /* a CUDA call failed; see pic_last_error */
    PIC_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
    PIC_ESTATE = 6,    /* call not valid in the handle's state */
    PIC_EBOUNDS = 7,   /* a device-side bounds check fired */
    PIC_EBUDGET = 8    /* a group's HBM budget would be exceeded */
} pic_status;

enum { PIC_BC_PERIODIC = 0, PIC_BC_PML = 1 };
enum { PIC_FREE = 0, PIC_BOUND = 1, PIC_DIRAC = 2 };
/* Fixed neutralising ions, used only by the Gauss-law diagnostic (ions carry
   no current): none, at the loaded positions (anchors for bound species), or
   uniform over the domain. */
enum { PIC_BG_NONE = 0, PIC_BG_AT_PARTICLES = 1, PIC_BG_UNIFORM = 2 };
/* bits of the `which` argument of pic_read_fields / pic_write_fields */
enum {
    PIC_EX = 1 << 0, PIC_EY = 1 << 1, PIC_EZ = 1 << 2,
    PIC_BX = 1 << 3, PIC_BY = 1 << 4, PIC_BZ = 1 << 5,
    PIC_JX = 1 << 6, PIC_JY = 1 << 7, PIC_JZ = 1 << 8,
    /* the external field of pic_set_external_field (pic_read_fields only) */
    PIC_EXTX = 1 << 9, PIC_EXTY = 1 << 10, PIC_EXTZ = 1 << 11
};
/* particle boundary rule at material edges (pic_set_particle_bc) */
enum { PIC_EDGE_REFLECT = 0, PIC_EDGE_OPEN = 1 };

typedef struct pic_sim pic_sim;     /* opaque, owned by the library */
typedef struct pic_group pic_group; /* opaque batch of simulations */

/* Grid, time step and boundaries (Sec. 4.1).  2D runs are 2D3V in the x-y
   plane (nz must be 1; dz is the slab depth used for densities).  Limits:
   nx, ny <= 2048, nz <= 1024. */
typedef struct pic_grid_desc {
    int dims;           /* 2 or 3 */
    int nx, ny, nz;     /* cells */
    double dx, dy, dz;  /* cell size, m */
    double dt;          /* time step, s; checked against Eq. dtlimit */
    int bc[3];          /* PIC_BC_PERIODIC or PIC_BC_PML per axis (z ignored in 2D) */
    int pml_cells;      /* CPML thickness on PML axes (cells) */
    double pml_R0;      /* CPML target reflection; <= 0 selects 1e-8 */
    int pml_order;      /* CPML grading exponent; <= 0 selects 3 */
    /* Soft plane-wave drive: a one-cell current sheet normal to inc_axis at
       index src_index carrying J_pol = -2 E0 g(t) / (eta0 d_inc), which
       radiates E_pol = E0 g(t - |x - x_s|/c) to both sides, with
       g(t) = exp(-2 ln2 (t - t0)^2 / tau^2) sin(omega (t - t0)). */
    int src_on;
    int inc_axis, pol_axis, src_index;
    double E0, omega, tau, t0;
} pic_grid_desc;

/* One species.  q, m in C and kg; weight = physical particles per
   macro-particle (ignored by the Fermi-Dirac loader, which sets it to
   density * cell volume / ppc).  omega0 / gamma: binding frequency and
   damping of PIC_BOUND per axis (Eq. modlorentz with diagonal tensors;
   gamma finite and >= 0, PIC_EINVAL otherwise; unequal gamma entries take
   the general 3x3 solve of the modified Boris rotation in the kernel with
   the boundary variants, single or batch).  v_F: Fermi velocity of PIC_DIRAC (m is then the averaged
   transverse mass p_F / (2 v_F) of Sec. 5).  background: PIC_BG_*. */
typedef struct pic_species_desc {
    int kind;
    double q, m, weight;
    double omega0[3], gamma[3];
    double v_F;
    int background;
} pic_species_desc;

/* Particles of one species, either given explicitly (cell != NULL) or drawn
   by the Fermi-Dirac loader (cell == NULL).
   Explicit: n particles; cell[n] linear cell index; off[3n] in-cell offset in
   [0,1) (x,y,z interleaved; free and Dirac); v[3n] velocity at t = -dt/2 (m/s);
   for PIC_BOUND anchor_off[3n] (FP64, [0,1)) is the rest position inside
   `cell` and disp[3n] (may be NULL = 0) the displacement from it in metres.
   Loader (Sec. 2): every material cell (mask != 0, all cells without a
   mask) gets ppc particles, particle id = material-cell rank * ppc + j;
   Philox-4x32-10 with key = seed and counter (id_lo, id_hi, call, stream)
   gives six uniforms per particle (position, |p|, direction); positions are
   uniform in the cell, or the j-th point of an m^dims lattice when quiet
   (m^dims = ppc); |p| follows the FD law with mu = E_F up to mu + 40 kT
   (3D density p^2 f for free, 2D p f for Dirac); bound particles start at
   rest.  density (m^-3) also feeds the plasma term of the dt check. */
typedef struct pic_particles {
    int64_t n;
    const int32_t *cell;
    const float *off;
    const float *v;
    const double *anchor_off;
    const float *disp;
    double density;
    double E_F;   /* J */
    double T;     /* K */
    int ppc;
    int quiet;
    uint64_t seed;
    uint32_t stream;
} pic_particles;

/* Tuning of one simulation (defaults in brackets; 0 keeps the default). */
typedef struct pic_tuning {
    int tile[3];        /* particle tile, cells [8,8,4 in 3D; 32,32,1 in 2D].  In 3D with
                           CIC shapes and the plain surface rule, 8,8,4 and 16,8,1 (the
                           shape for one-cell sheets) run a kernel specialised to the
                           tile; any other tile runs the general one */
    int sort_interval;  /* steps between tile re-sorts [32] */
    int field_zchunk;   /* z planes per field-kernel CTA [16] */
    int particle_ctas;  /* persistent particle CTAs [SMs x occupancy, one CTA per SM
                           fewer when the field work runs beside the particle phase] */
    int keep_J;         /* 1: J of the last step stays readable (tests) [0] */
    int timing;         /* 1: time every kernel launch with CUDA events [0] */
    int field_plain;    /* 1: field kernel with plain loads even where TMA applies [0] */
    int tile_order;     /* particles inside a tile: 0 cells interleaved (rank inside the
                           cell, then cell: a warp's lanes in consecutive cells), 1 arrival
                           order, 2 spread over the cells by a multiplicative permutation [0] */
    int no_overlap;     /* 0: the field work that does not need this step's current runs
                           beside the particle phase on a second stream of the handle --
                           the B pass (field_mode 2), or the whole fused update with the
                           current applied afterwards by a short pass over the field
                           blocks the deposit touched (field_mode 1); 1: the particle
                           phase, then the field update, on one stream [0] */
    int field_mode;     /* 1: fused field update (one pass, 48 B/cell; TMA-fed where nx % 4
                           == 0); 2: two streaming passes, B then E (36 B/cell each, no
                           shared memory or barriers); 3: one streaming pass (48 B/cell,
                           no shared memory or barriers: the -x neighbour's B by warp
                           shuffle, the -y one recomputed); 0: keep the current mode [2] */
    int64_t wait_polls; /* polls after which a TMA-fed field pass stops waiting for a copy
                           and latches PIC_ETIMEOUT [2^23, about 0.5 s]; copies already in
                           flight are always waited for in full before a CTA exits.  A
                           small value makes the waits give up (tests of the timeout path) */
    int field_overlap;  /* field_mode 2 with overlap: 1 the B pass runs beside the particle
                           phase, the E pass after it; 2 both passes run beside it (the E
                           pass without this step's current) and a short pass over the field
                           blocks the deposit touched then subtracts (dt / eps0) J from
                           E^{n+1}; 0: keep the current choice [1] */
} pic_tuning;

/* Results of pic_diagnostics (FP64 reductions on the device). */
typedef struct pic_diag {
    int64_t step;                            /* steps taken */
    double time;                             /* step * dt, s */
    int nspecies;
    int64_t count[PIC_MAX_SPECIES];          /* particles per species */
    uint64_t reflections[PIC_MAX_SPECIES];   /* reflections so far (specular or diffuse) */
    double kinetic[PIC_MAX_SPECIES];         /* sum 1/2 m w |v|^2, J */
    double field_E;                          /* sum eps0 E^2 / 2 dV, J */
    double field_B;                          /* sum B^2 / (2 mu0) dV, J (B on the half step) */
    double gauss_max;                        /* max |div E - rho/eps0| over nodes */
    double gauss_rms;                        /* RMS of the same */
    double rho_max;                          /* max |rho / eps0| */
} pic_diag;

/* Kernel timing totals since the last query (pic_tuning.timing = 1). */
typedef struct pic_timing {
    double particle_ms, field_ms, sort_ms;       /* summed CUDA-event durations */
    int64_t particle_launches, field_launches, sort_launches;  /* timed phases */
    int64_t kernel_launches;                     /* all kernels pic_step launched */
    double fieldb_ms;                            /* field_mode 1: the B pass (field_ms: E pass) */
    int64_t fieldb_launches;
} pic_timing;

/* Device memory hooks.  alloc returns a device pointer of `bytes` usable on
   `stream`, aligned to 256 bytes (NULL on failure; a misaligned pointer is
   handed back to free and the call that needed it fails with PIC_ENOMEM);
   free releases it.  Without hooks the library uses cudaMalloc / cudaFree.
   Set before creating simulations. */
typedef void *(*pic_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*pic_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
pic_status pic_set_allocator(pic_alloc_fn alloc, pic_free_fn release, void *ctx);

/* Create a simulation on the current CUDA device.  stream: a cudaStream_t
   (NULL = the legacy default stream).  Checks dt against Eq. dtlimit with
   no plasma yet (PIC_EDTLIMIT).  *out receives the handle. */
pic_status pic_create(const pic_grid_desc *grid, void *stream, pic_sim **out);

/* Free all device state of the handle (NULL is accepted). */
pic_status pic_destroy(pic_sim *sim);

/* Material mask (Sec. 3): n = number of cells, 1 = material, 0 = vacuum.
   Must precede pic_load_species. */
pic_status pic_set_material_mask(pic_sim *sim, const uint8_t *mask, size_t n);

/* Relative permittivity per cell (Eq. consteps, eps = eps0 eps_r, the
   material's background response; the bound species add the Lorentz part):
   the E update becomes E^{n+1} = E^n + (dt / eps_r) (c^2 curl B - J / eps0),
   each E component taking the eps_r of the cell its node belongs to, and the
   Gauss residual of pic_diagnostics is taken on D = eps0 eps_r E.  eps_r:
   n = number of cells values [nz][ny][nx], finite, 1e-6 .. 1e6 (else
   PIC_EINVAL; the library keeps its own copy of 1 / eps_r); NULL returns to
   vacuum.  Needs field_mode 2 (PIC_ESTATE otherwise; pic_set_tuning then
   refuses modes 1 and 3); in a group the batched field update applies it. */
pic_status pic_set_permittivity(pic_sim *sim, const float *eps_r, size_t n);

/* External electrostatic field (Sec. 3, the work-function model): a static
   field in V/m on the E stagger of the Yee grid (E_x of cell (i, j, k) at
   (i+1/2, j, k), E_y at (i, j+1/2, k), E_z at (i, j, k+1/2)) that the
   particle push adds to the gathered E^n of every species and that the
   Maxwell update never sees (it enters neither curl E, the E update nor the
   Gauss diagnostic).  ex, ey, ez: n = number of cells finite doubles each,
   [nz][ny][nx] (PIC_EINVAL otherwise); the library keeps an FP32 copy, read
   back with PIC_EXT* in pic_read_fields.  ex == NULL removes the field.
   Not while the simulation belongs to a group (PIC_ESTATE); a member with a
   field steps in its group with the variant batch kernel. */
pic_status pic_set_external_field(pic_sim *sim, const double *ex, const double *ey,
                                  const double *ez, size_t n);

/* The work-function barrier of height W_eV (eV) built on the device from the
   material mask and set as the external field: node potential
   phi = -(W / e) f, f the vacuum fraction of the cells that share the node
   (cells i-1..i, j-1..j, k-1..k; in 2D the four cells of the plane; cells
   beyond a non-periodic face do not count), and E = -grad phi on the Yee
   stagger, E_a of cell (i, j, k) = -(phi(node + e_a) - phi(node)) / d_a with
   node = (i, j, k), E_z = 0 in 2D; an electron gains potential energy W on
   leaving the material.  Uses the mask set at the time of the call (no mask:
   all material, the field is removed).  W_eV = 0 removes the field;
   |W_eV| <= 1e3 and finite (PIC_EINVAL otherwise). */
pic_status pic_set_work_function(pic_sim *sim, double W_eV);

/* Particle boundary rule at material edges (Sec. 3).
   PIC_EDGE_REFLECT (default): a free or Dirac particle that moves from a
   material cell into a vacuum cell is reflected; on every axis whose cell
   index changed the position is mirrored about the crossed face.  The
   reflection is specular (those velocity components change sign) or, with
   probability p_diffuse when a single face was crossed, diffuse: the speed
   is kept and the direction is drawn from Lambert's cosine law about the
   inward normal -- cos(theta) = sqrt(u1) and azimuth 2 pi u2 (measured from
   the next axis in x -> y -> z order) for 3D velocities; for Dirac carriers
   the in-plane law sin(theta) = 2 u1 - 1 with v_z = 0.  The draws are
   Philox-4x32-10 with key (seed low word, seed high word) and counter
   (particle id, step index mod 2^32, species index, 0x44494655);
   u_i = (word_i >> 8) / 2^24, and the reflection is diffuse when
   u0 < p_diffuse rounded to FP32.
   PIC_EDGE_OPEN: particles cross material edges freely (the open surface;
   with pic_set_work_function, the potential-wall surface); p_diffuse must
   be 0.
   Non-periodic domain faces reflect specularly under either rule.  edges
   outside the enum or p_diffuse outside [0, 1]: PIC_EINVAL.  In a group the
   step index of the draws is the member's own (its device step count), so
   the draws equal those of the simulation stepped alone. */
pic_status pic_set_particle_bc(pic_sim *sim, int edges, double p_diffuse, uint64_t seed);

/* Shape function W of Sec. 4.1 for the free and Dirac particles: order 1
   CIC (default), 2 TSC (the quadratic B-spline: 3/4 - r^2 for r < 1/2,
   (3/2 - r)^2 / 2 for r < 3/2; gather from the three nodes around the
   nearest one on each component's stagger, Esirkepov deposit over four
   nodes per axis, and the charge density of the Gauss diagnostic with the
   same shape).  Bound particles keep CIC.  Must precede pic_load_species
   (PIC_ESTATE otherwise: a species' ion background is deposited with its
   shape); other orders: PIC_EINVAL.  A group's members share one shape
   order (pic_group_add refuses a member of the other order). */
pic_status pic_set_shape_order(pic_sim *sim, int order);

/* Full symmetric binding tensor of bound species `species` (Eq. modlorentz
   with a tensor restoring force): Omega^2 = diag(omega0^2) plus the
   off-diagonal entries w2off = (xy, xz, yz) in s^-2, so the Hooke term of
   the push is Omega^2 D (a rotated anisotropic medium).  The tensor must be
   positive definite and finite (PIC_EINVAL), dt within the limit of Eq.
   dtlimit with the largest eigenvalue (bounded by Gershgorin's discs) as
   the binding frequency squared (PIC_EDTLIMIT), the species bound
   (PIC_EINVAL), the simulation not in a group (PIC_ESTATE).  Such a species runs in the kernel with the boundary
   variants (single or batch). */
pic_status pic_set_binding_tensor(pic_sim *sim, int species, const double *w2off);

/* Add a species (explicit particles or the Fermi-Dirac loader) and sort it
   into tiles.  Re-checks Eq. dtlimit with the plasma and binding frequencies
   of all species so far (PIC_EDTLIMIT).  *species_id receives its index. */
pic_status pic_load_species(pic_sim *sim, const pic_species_desc *desc,
                            const pic_particles *parts, int *species_id);

/* Set tuning; call before the first pic_step. */
pic_status pic_set_tuning(pic_sim *sim, const pic_tuning *tuning);

/* Enqueue nsteps PIC steps on the simulation's stream (asynchronous). */
pic_status pic_step(pic_sim *sim, int nsteps);

/* Wait for the stream; return a latched device error, if any. */
pic_status pic_sync(pic_sim *sim);

/* Copy fields to/from host FP64 arrays (converted from/to the FP32 device
   fields).  which = OR of PIC_E*, PIC_B*, PIC_J* (and, for reading, PIC_EXT*:
   the external field, PIC_ESTATE if none is set); the arrays of the selected
   components follow one another in bit order, each ncell long; n = total
   doubles.  J is readable only with keep_J.  Synchronous. */
pic_status pic_read_fields(pic_sim *sim, int which, double *host_out, size_t n);
pic_status pic_write_fields(pic_sim *sim, int which, const double *host_in, size_t n);

/* Copy one species back in load order (particle id order): cell[n] linear
   cell index, off[3n], v[3n]; for PIC_BOUND anchor_off[3n] and disp[3n]
   (pass NULL for unused arrays).  n must equal the species count. */
pic_status pic_read_species(pic_sim *sim, int species, int32_t *cell, float *off, float *v,
                            double *anchor_off, float *disp, size_t n);

/* Particles per cell of one species (current positions), int32[ncell]. */
pic_status pic_cell_counts(pic_sim *sim, int species, int32_t *host_out, size_t n);

/* FP64 diagnostics (kinetic and field energy, Gauss residual, counts). */
pic_status pic_diagnostics(pic_sim *sim, pic_diag *out);

/* Histogram of the kinetic energy E = m |v|^2 / 2 of one species'
   macro-particles (the relaxation study of Sec. 2 fits its high-energy
   tail): host_out[b], b < nbins, counts E in [b D, (b+1) D) with
   D = e_max / nbins; host_out[nbins] counts E >= e_max.  E is formed in FP64
   from the FP32 velocities as (0.5 m) ((vx vx + vy vy) + vz vz) and the bin
   as floor(E / D), each operation rounded once, so for given velocities the
   counts are exact.  nbins 1 .. 2^20, e_max finite and > 0,
   n = nbins + 1 (PIC_EINVAL otherwise).  Synchronous. */
pic_status pic_energy_histogram(pic_sim *sim, int species, double e_max, int nbins,
                                uint64_t *host_out, size_t n);

/* Kernel timing totals since the last call; resets them.  Synchronous. */
pic_status pic_get_timing(pic_sim *sim, pic_timing *out);

/* Device bytes held by the handle. */
pic_status pic_memory_bytes(const pic_sim *sim, size_t *bytes);

/* Text of the last error on this handle (never NULL). */
const char *pic_last_error(const pic_sim *sim);

/* ------------------------------------------------------------------------
   Batch engine: many independent simulations (for example nanostructures of
   uneven size) advanced by the same launches.
   A group holds up to `capacity` simulations of one dimensionality, one
   particle tile size and one shape order (the first member fixes them; a
   member may carry a permittivity, a boundary variant of Sec. 3 or an
   anisotropic bound species).  pic_group_step advances
   every member that has steps left -- a member added with nsteps stops after
   nsteps -- with one persistent launch for the particle phase of all members
   and one launch for their field phase per step; the tile re-sorts of all
   members run in a few batched launches every sort_interval steps (the first
   member's interval).  With use_graph the steps between re-sorts are captured
   once into a CUDA graph and replayed; finished members are skipped on the
   device.  While in a group a member cannot be stepped on its own, nor take
   a mask, species or tuning (PIC_ESTATE); pic_read_*, pic_write_fields,
   pic_diagnostics and pic_sync on a member wait for the group's stream, and
   pic_destroy on a member removes it first.  Admission: the device bytes of
   all members must stay within hbm_budget (0 = no limit; PIC_EBUDGET
   otherwise, also when all `capacity` slots are taken).
   stream: the CUDA stream all group work is queued on; NULL makes the group
   create (and later destroy) a non-blocking stream of its own, since the
   legacy default stream cannot be captured into a graph.  The group keeps
   small device tables (parameter blocks, work-item lists, sort scratch of one
   int per mobile particle) that it allocates through the pic_set_allocator
   hooks when membership changes.
   ------------------------------------------------------------------------ */
pic_status pic_group_create(int capacity, size_t hbm_budget, void *stream, int use_graph,
                            pic_group **out);
/* Free the group; members are released (their handles stay valid). */
pic_status pic_group_destroy(pic_group *g);
/* Add a simulation that will advance nsteps more steps with the group. */
pic_status pic_group_add(pic_group *g, pic_sim *sim, int64_t nsteps);
/* Remove a member (after waiting for the group's stream). */
pic_status pic_group_remove(pic_group *g, pic_sim *sim);
/* Enqueue nsteps group steps (asynchronous). */
pic_status pic_group_step(pic_group *g, int nsteps);
/* Wait for the group's stream; return a latched device error of any member. */
pic_status pic_group_sync(pic_group *g);
/* Steps a member has taken in the group and steps it has left. */
pic_status pic_group_progress(pic_group *g, const pic_sim *sim, int64_t *steps_done,
                              int64_t *steps_left);
/* Members, device bytes held by members, kernels launched since creation. */
pic_status pic_group_info(pic_group *g, int *members, size_t *member_bytes, int64_t *launches);

/* Largest grid (cells) pic_cell_counts_noalloc accepts: 2^22 cells, i.e. a
   16 MiB int32 array built into the library. */
#define PIC_NOALLOC_MAX_CELLS (1 << 22)

/* pic_cell_counts without any device allocation.  (No counterpart in the
   paper: this is a service of the library.)
   pic_cell_counts asks for a temporary device buffer on every call.  Some
   callers cannot allow that: code that records work into a CUDA graph (a
   cudaMalloc cannot be captured), hosts that hand all device memory to a
   fixed pool or another framework up front, and serving loops where
   cudaMalloc / cudaFree would synchronise the device and stall other work.
   This variant counts into a fixed device array of PIC_NOALLOC_MAX_CELLS
   int32 that lives in the library itself; every device that has loaded the
   library's code for this call keeps those 16 MiB until the process exits.
   Arguments and output are those of pic_cell_counts; grids larger than
   PIC_NOALLOC_MAX_CELLS cells are rejected with PIC_EINVAL.  The first call
   on a device looks up the array's device address (cudaGetSymbolAddress);
   make that first call before any stream capture.  All calls share the one
   array and clear it at the start: calls that run at the same time on the
   GPU (several streams or threads) race and must be serialised by the
   caller.  Synchronous: it waits for the simulation's stream. */
pic_status pic_cell_counts_noalloc(pic_sim *sim, int species, int32_t *host_out, size_t n);

#ifdef __cplusplus
}
#endif

#endif /* PIC_H */
