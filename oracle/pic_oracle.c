/*
 * pic_oracle.c -- plain, slow FP64 CPU oracle for the quantum-plasma PIC step
 * of Ngirmang, Do, Liu, Bosman & Wu, "Particle-In-Cell Simulations of Quantum
 * Plasmas" (arXiv 2501.07465).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no source, header, table or constant with the
 * CUDA library; the two meet only through plain arrays handed to both by the
 * tests.
 *
 * Everything is FP64 and written to be checked against the paper by eye:
 * positions are kept in cell units (X = x / dx), velocities in m/s, fields in
 * SI units on the Yee stagger, one particle at a time, one cell at a time, no
 * blocking and no fusion.
 *
 * Step order (the PIC cycle of Sec. 4.1 / Appendix A):
 *   1. B at the integer time for the gather: B^n = B^{n-1/2} - (dt/2) curl E^n
 *      (plain Yee curl; the paper stores B on half steps, Sec. 4.1).
 *   2. Per particle: CIC gather of E^n, B^n (shape function W, Sec. 4.1);
 *      push -- free: Boris (Eqs. discrlorentz/borisscheme, R of Eq.
 *      borisrotsol); bound: modified Boris (Eqs. modborisvpm, modborisBrot;
 *      the 3x3 implicit-midpoint system solved by Cramer's rule); Dirac:
 *      Boris with the transverse mass then |v| renormalised to v_F (Sec. 5);
 *      plus an optional external electrostatic field that only the particles
 *      see (the work-function barrier of Sec. 3); the particle boundary rule
 *      of Sec. 3: conditional specular or diffusive reflection at material
 *      edges, or open edges;
 *      Esirkepov charge-conserving current deposit.
 *   3. Soft plane-wave current sheet added to J.
 *   4. Yee: B^{n+1/2} = B^{n-1/2} - dt (curl E^n + CPML psi),
 *      E^{n+1} = E^n + (dt / eps_r) (c^2 (curl B^{n+1/2} + CPML psi) - J / eps0)
 *      (Sec. 4.1 Maxwell curl equations; Eq. consteps with eps = eps0 eps_r,
 *      eps_r a per-cell relative permittivity, 1 unless set; E_x at
 *      (i+1/2, j, k) and the other components of cell (i, j, k) take the
 *      cell's eps_r).
 *
 * Threads: compiled with -fopenmp (a separate library used only to time the
 * oracle on all host cores), the cell loops of steps 1 and 4 and the particle
 * loop of step 2 run in parallel and the deposit's additions to J are atomic;
 * the arithmetic of every particle and every cell is unchanged, only the
 * order in which J's FP64 contributions are summed differs.  The test suite
 * uses the serial build, where these directives are absent.
 *
 * Parity pins: every function below is pinned by a CPU test against a closed
 * form, an invariant or a brute-force check (tests/test_oracle_pins.py).  The
 * CPML absorption quality is the one part checked only for decay, not against
 * a closed form ("parity unpinned" for the absorption coefficient).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA SI constants (exact c; eps0 from CODATA 2018; mu0 from c and eps0). */
static const double C_LIGHT = 299792458.0;
static const double EPS0 = 8.8541878128e-12;
static const double KB = 1.380649e-23;
static const double PI = 3.14159265358979323846;
static double mu0(void) { return 1.0 / (EPS0 * C_LIGHT * C_LIGHT); }

enum { KIND_FREE = 0, KIND_BOUND = 1, KIND_DIRAC = 2 };
enum { BC_PERIODIC = 0, BC_PML = 1 };
#define MAX_SPECIES 8
/* fourth Philox counter word of the diffuse-reflection draws */
#define DIFFUSE_STREAM 0x44494655u

void orc_philox(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out);

typedef struct {
    int kind;
    double q, m, w;
    double omega0[3], gamma[3];
    /* off-diagonal entries of the binding tensor Omega^2 (xy, xz, yz, s^-2;
       the diagonal is omega0^2), used when has_off */
    double w2off[3];
    int has_off;
    double vF;
    long n;
    double *X; /* 3n: position (free, Dirac) or anchor (bound), cell units */
    double *D; /* 3n: bound displacement from the anchor, metres */
    double *V; /* 3n: velocity at the half step, m/s */
    long long nrefl;
} orc_species;

typedef struct {
    int dims;
    int n[3];
    double d[3];
    double dt;
    int bc[3];
    int P;         /* CPML thickness in cells */
    double R0;     /* CPML normal-incidence reflection target */
    int order;     /* CPML grading exponent */
    /* soft plane-wave source (a current sheet) */
    int src_on, inc, pol, src_idx;
    double E0, omega, tau, t0;

    long ncell;
    double *E[3], *B[3], *J[3], *Bn[3], *Jlast[3];
    /* CPML psi, full-size arrays (one per component and derivative axis);
       only allocated for PML axes. psiE[a][c]: E component c, derivative along a. */
    double *psiE[3][3], *psiB[3][3];
    /* CPML coefficients per axis: e = integer positions, h = half positions */
    double *be[3], *ae[3], *bh[3], *ah[3];
    uint8_t *mask;
    double *eps_r; /* per-cell relative permittivity (NULL: vacuum) */
    /* external electrostatic field on the E stagger, seen by the particles
       only (NULL: none) */
    double *Eext[3];
    /* particle boundary at material edges: open_edges = 1 lets particles
       leave the material; otherwise a fraction p_diffuse of the single-face
       reflections is diffuse (Philox key diff_seed) */
    int open_edges;
    double p_diffuse;
    uint64_t diff_seed;
    /* shape order of the free and Dirac particles: 1 CIC, 2 TSC (bound
       particles are always CIC) */
    int shape_order;
    double *rho_bg;
    long step;
    int nsp;
    orc_species sp[MAX_SPECIES];
} orc_sim;

/* ------------------------------------------------------------------------ */
/* indexing and boundary rule                                                 */
/* ------------------------------------------------------------------------ */

static long idx3(const orc_sim *s, int i, int j, int k) {
    return ((long)k * s->n[1] + j) * s->n[0] + i;
}

/* Map (i,j,k) into the domain.  Periodic axes wrap; on a non-periodic axis an
   index outside [0,n) is outside the domain (fields there are zero, a
   perfectly conducting wall behind the CPML).  In 2D the z index is always 0. */
static int wrap_index(const orc_sim *s, int *ijk) {
    for (int a = 0; a < 3; ++a) {
        if (a == 2 && s->dims == 2) { ijk[2] = 0; continue; }
        int n = s->n[a];
        if (ijk[a] < 0 || ijk[a] >= n) {
            if (s->bc[a] != BC_PERIODIC) return 0;
            ijk[a] = ((ijk[a] % n) + n) % n;
        }
    }
    return 1;
}

static double fget(const orc_sim *s, const double *F, int i, int j, int k) {
    int c[3] = {i, j, k};
    if (!wrap_index(s, c)) return 0.0;
    return F[idx3(s, c[0], c[1], c[2])];
}

static void fadd(const orc_sim *s, double *F, int i, int j, int k, double v) {
    int c[3] = {i, j, k};
    if (!wrap_index(s, c)) return; /* deposits beyond a wall are dropped */
#ifdef _OPENMP
#pragma omp atomic
#endif
    F[idx3(s, c[0], c[1], c[2])] += v;
}

/* material mask at a cell; outside the domain (non-periodic axis) = vacuum */
static int mask_at(const orc_sim *s, int i, int j, int k) {
    int c[3] = {i, j, k};
    if (!wrap_index(s, c)) return 0;
    if (!s->mask) return 1;
    return s->mask[idx3(s, c[0], c[1], c[2])] != 0;
}

/* ------------------------------------------------------------------------ */
/* creation                                                                   */
/* ------------------------------------------------------------------------ */

/* CPML profile (Roden & Gedney 2000, kappa = 1, alpha = 0): sigma grows as
   (depth/P)^order inside the P-cell slabs at both ends of a PML axis;
   b = exp(-sigma dt / eps0), a = b - 1.  pos = cell-unit position. */
static void cpml_coeff(const orc_sim *s, int a, double pos, double *b, double *c) {
    int n = s->n[a], P = s->P;
    double depth = 0.0;
    if (pos < P) depth = P - pos;
    else if (pos > n - P) depth = pos - (n - P);
    double eta0 = mu0() * C_LIGHT;
    double smax = -(s->order + 1) * log(s->R0) / (2.0 * eta0 * P * s->d[a]);
    double sigma = smax * pow(depth / P, s->order);
    *b = exp(-sigma * s->dt / EPS0);
    *c = *b - 1.0;
}

void *orc_create(int dims, const int *n, const double *d, double dt, const int *bc,
                 int pml_cells, double R0, int order, int src_on, int inc, int pol,
                 int src_idx, double E0, double omega, double tau, double t0) {
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->dims = dims;
    for (int a = 0; a < 3; ++a) { s->n[a] = n[a]; s->d[a] = d[a]; s->bc[a] = bc[a]; }
    if (dims == 2) { s->n[2] = 1; s->bc[2] = BC_PERIODIC; }
    s->dt = dt;
    s->P = pml_cells; s->R0 = R0; s->order = order;
    s->src_on = src_on; s->inc = inc; s->pol = pol; s->src_idx = src_idx;
    s->E0 = E0; s->omega = omega; s->tau = tau; s->t0 = t0;
    s->ncell = (long)s->n[0] * s->n[1] * s->n[2];
    s->shape_order = 1;
    for (int c = 0; c < 3; ++c) {
        s->E[c] = (double *)calloc(s->ncell, sizeof(double));
        s->B[c] = (double *)calloc(s->ncell, sizeof(double));
        s->J[c] = (double *)calloc(s->ncell, sizeof(double));
        s->Bn[c] = (double *)calloc(s->ncell, sizeof(double));
        s->Jlast[c] = (double *)calloc(s->ncell, sizeof(double));
    }
    for (int a = 0; a < 3; ++a) {
        if (s->bc[a] != BC_PML) continue;
        for (int c = 0; c < 3; ++c) {
            if (c == a) continue; /* no derivative of a component along itself */
            s->psiE[a][c] = (double *)calloc(s->ncell, sizeof(double));
            s->psiB[a][c] = (double *)calloc(s->ncell, sizeof(double));
        }
        int na = s->n[a];
        s->be[a] = (double *)calloc(na, sizeof(double));
        s->ae[a] = (double *)calloc(na, sizeof(double));
        s->bh[a] = (double *)calloc(na, sizeof(double));
        s->ah[a] = (double *)calloc(na, sizeof(double));
        for (int i = 0; i < na; ++i) {
            cpml_coeff(s, a, (double)i, &s->be[a][i], &s->ae[a][i]);
            cpml_coeff(s, a, i + 0.5, &s->bh[a][i], &s->ah[a][i]);
        }
    }
    return s;
}

void orc_destroy(void *h) {
    orc_sim *s = (orc_sim *)h;
    if (!s) return;
    for (int c = 0; c < 3; ++c) {
        free(s->E[c]); free(s->B[c]); free(s->J[c]); free(s->Bn[c]); free(s->Jlast[c]);
    }
    for (int a = 0; a < 3; ++a) {
        for (int c = 0; c < 3; ++c) { free(s->psiE[a][c]); free(s->psiB[a][c]); }
        free(s->be[a]); free(s->ae[a]); free(s->bh[a]); free(s->ah[a]);
    }
    for (int k = 0; k < s->nsp; ++k) { free(s->sp[k].X); free(s->sp[k].D); free(s->sp[k].V); }
    for (int c = 0; c < 3; ++c) free(s->Eext[c]);
    free(s->mask); free(s->eps_r); free(s->rho_bg);
    free(s);
}

void orc_set_mask(void *h, const uint8_t *mask) {
    orc_sim *s = (orc_sim *)h;
    if (!s->mask) s->mask = (uint8_t *)malloc(s->ncell);
    memcpy(s->mask, mask, s->ncell);
}

/* Relative permittivity per cell (Eq. consteps, eps = eps0 eps_r); NULL
   restores vacuum. */
void orc_set_permittivity(void *h, const double *eps_r) {
    orc_sim *s = (orc_sim *)h;
    if (!eps_r) {
        free(s->eps_r);
        s->eps_r = NULL;
        return;
    }
    if (!s->eps_r) s->eps_r = (double *)malloc(s->ncell * sizeof(double));
    memcpy(s->eps_r, eps_r, s->ncell * sizeof(double));
}

/* External electrostatic field (V/m) on the E stagger, added to the gathered
   E of every particle and never seen by the Maxwell update (the work-function
   model of Sec. 3).  ex == NULL removes it. */
void orc_set_external_field(void *h, const double *ex, const double *ey, const double *ez) {
    orc_sim *s = (orc_sim *)h;
    const double *in[3] = {ex, ey, ez};
    for (int c = 0; c < 3; ++c) {
        free(s->Eext[c]);
        s->Eext[c] = NULL;
    }
    if (!ex) return;
    for (int c = 0; c < 3; ++c) {
        s->Eext[c] = (double *)malloc(s->ncell * sizeof(double));
        memcpy(s->Eext[c], in[c], s->ncell * sizeof(double));
    }
}

/* Vacuum fraction of the cells that share grid node (i, j, k): cells
   i-1..i, j-1..j, k-1..k (the four cells of the plane in 2D); cells beyond a
   non-periodic face do not count.  No mask: all material. */
static double node_vacuum(const orc_sim *s, int i, int j, int k) {
    int nin = 0, nvac = 0;
    int kn = s->dims == 3 ? 2 : 1;
    for (int dk = 0; dk < kn; ++dk)
        for (int dj = 0; dj < 2; ++dj)
            for (int di = 0; di < 2; ++di) {
                int c[3] = {i - 1 + di, j - 1 + dj, s->dims == 3 ? k - 1 + dk : 0};
                if (!wrap_index(s, c)) continue;
                ++nin;
                if (s->mask && !s->mask[idx3(s, c[0], c[1], c[2])]) ++nvac;
            }
    return nin ? (double)nvac / nin : 0.0;
}

/* Work-function barrier (Sec. 3): the electrostatic potential on the grid
   nodes is phi = -(W / e) f, f the node's vacuum fraction, so an electron
   (charge -e) gains potential energy W on leaving the material.  The field
   E = -grad phi is taken on the Yee stagger: E_a of cell (i, j, k) is
   -(phi(node + e_a) - phi(node)) / d_a, node = (i, j, k); E_z = 0 in 2D.
   W in eV; writes ex, ey, ez (ncell each). */
void orc_work_function_field(void *h, double W_eV, double *ex, double *ey, double *ez) {
    orc_sim *s = (orc_sim *)h;
    double *out[3] = {ex, ey, ez};
    for (int k = 0; k < s->n[2]; ++k)
        for (int j = 0; j < s->n[1]; ++j)
            for (int i = 0; i < s->n[0]; ++i) {
                long c = idx3(s, i, j, k);
                double phi0 = -W_eV * node_vacuum(s, i, j, k);
                for (int a = 0; a < 3; ++a) {
                    if (a == 2 && s->dims == 2) { out[a][c] = 0.0; continue; }
                    int nb[3] = {i + (a == 0), j + (a == 1), k + (a == 2)};
                    double phi1 = -W_eV * node_vacuum(s, nb[0], nb[1], nb[2]);
                    out[a][c] = -(phi1 - phi0) / s->d[a];
                }
            }
}

/* Particle boundary rule at material edges (Sec. 3): open = 1 lets the
   particles cross; otherwise a reflection across a single face is diffuse
   with probability p_diffuse (Philox key = seed), specular otherwise. */
void orc_set_particle_bc(void *h, int open, double p_diffuse, uint64_t seed) {
    orc_sim *s = (orc_sim *)h;
    s->open_edges = open;
    s->p_diffuse = p_diffuse;
    s->diff_seed = seed;
}

/* ------------------------------------------------------------------------ */
/* shape function (CIC, order 1) and charge density                          */
/* ------------------------------------------------------------------------ */

/* CIC weight of the node at integer position `node` for a particle at X */
static double cic(double X, int node) {
    double r = fabs(X - node);
    return r < 1.0 ? 1.0 - r : 0.0;
}

/* TSC (quadratic B-spline, order 2) weight of the node at integer position
   `node` for a particle at X: 3/4 - r^2 for r < 1/2, (3/2 - r)^2 / 2 for
   1/2 <= r < 3/2, r = |X - node|. */
static double tsc(double X, int node) {
    double r = fabs(X - node);
    if (r < 0.5) return 0.75 - r * r;
    if (r < 1.5) {
        double t = 1.5 - r;
        return 0.5 * t * t;
    }
    return 0.0;
}

static double shape(int order, double X, int node) {
    return order == 2 ? tsc(X, node) : cic(X, node);
}

/* first of the nodes a particle at X touches: CIC floor(X) (2 nodes), TSC
   the nearest node - 1 (3 nodes) */
static int first_node(int order, double X) {
    return order == 2 ? (int)floor(X + 0.5) - 1 : (int)floor(X);
}

/* shape order of species sp (bound particles keep CIC) */
static int species_order(const orc_sim *s, const orc_species *sp) {
    return sp->kind == KIND_BOUND ? 1 : s->shape_order;
}

/* Deposit the charge density of one macro-particle (charge qw) at X onto the
   integer nodes (Gauss-law nodes of the Yee grid) with the shape of the
   given order. */
static void deposit_rho(const orc_sim *s, int order, double *rho, const double *X, double qw) {
    double V = s->d[0] * s->d[1] * s->d[2];
    int nn = order + 1;
    int i0 = first_node(order, X[0]), j0 = first_node(order, X[1]), k0 = first_node(order, X[2]);
    int kn = s->dims == 3 ? nn : 1;
    for (int k = 0; k < kn; ++k)
        for (int j = 0; j < nn; ++j)
            for (int i = 0; i < nn; ++i) {
                double wz = s->dims == 3 ? shape(order, X[2], k0 + k) : 1.0;
                double w = shape(order, X[0], i0 + i) * shape(order, X[1], j0 + j) * wz;
                fadd(s, rho, i0 + i, j0 + j, s->dims == 3 ? k0 + k : 0, qw / V * w);
            }
}

/* current position (cell units) of particle p of species sp */
static void particle_pos(const orc_sim *s, const orc_species *sp, long p, double *X) {
    for (int a = 0; a < 3; ++a) {
        X[a] = sp->X[3 * p + a];
        if (sp->kind == KIND_BOUND) X[a] += sp->D[3 * p + a] / s->d[a];
    }
}

/* rho of all species at their current positions, plus the fixed background */
void orc_rho(void *h, double *rho) {
    orc_sim *s = (orc_sim *)h;
    memset(rho, 0, s->ncell * sizeof(double));
    for (int k = 0; k < s->nsp; ++k) {
        orc_species *sp = &s->sp[k];
        for (long p = 0; p < sp->n; ++p) {
            double X[3];
            particle_pos(s, sp, p, X);
            deposit_rho(s, species_order(s, sp), rho, X, sp->q * sp->w);
        }
    }
    if (s->rho_bg)
        for (long c = 0; c < s->ncell; ++c) rho[c] += s->rho_bg[c];
}

/* ------------------------------------------------------------------------ */
/* species                                                                    */
/* ------------------------------------------------------------------------ */

/* bg_mode: 0 no neutralising background; 1 fixed ions at the loaded positions
   (anchors for bound species); 2 a uniform background over the whole domain. */
int orc_add_species(void *h, int kind, double q, double m, double w, const double *omega0,
                    const double *gamma, double vF, long n, const double *X, const double *V,
                    const double *D, int bg_mode) {
    orc_sim *s = (orc_sim *)h;
    if (s->nsp >= MAX_SPECIES) return -1;
    orc_species *sp = &s->sp[s->nsp];
    sp->kind = kind; sp->q = q; sp->m = m; sp->w = w; sp->vF = vF;
    for (int a = 0; a < 3; ++a) { sp->omega0[a] = omega0[a]; sp->gamma[a] = gamma[a]; }
    sp->n = n;
    size_t bytes = (size_t)(3 * (n > 0 ? n : 1)) * sizeof(double);
    sp->X = (double *)malloc(bytes);
    sp->V = (double *)malloc(bytes);
    sp->D = (double *)calloc(3 * (n > 0 ? n : 1), sizeof(double));
    if (n > 0) {
        memcpy(sp->X, X, 3 * n * sizeof(double));
        memcpy(sp->V, V, 3 * n * sizeof(double));
        if (kind == KIND_BOUND && D) memcpy(sp->D, D, 3 * n * sizeof(double));
    }
    sp->nrefl = 0;
    if (bg_mode != 0) {
        if (!s->rho_bg) s->rho_bg = (double *)calloc(s->ncell, sizeof(double));
        if (bg_mode == 1) {
            /* ions at the loaded positions; for bound species at the anchors */
            for (long p = 0; p < n; ++p)
                deposit_rho(s, species_order(s, sp), s->rho_bg, &sp->X[3 * p], -q * w);
        } else {
            double V = s->d[0] * s->d[1] * s->d[2];
            double total = q * w * (double)n;
            for (long c = 0; c < s->ncell; ++c) s->rho_bg[c] -= total / (V * s->ncell);
        }
    }
    return s->nsp++;
}

/* ------------------------------------------------------------------------ */
/* pushers                                                                    */
/* ------------------------------------------------------------------------ */

/* Free species: Boris scheme (Appendix A.1).  Half electric kick (Eq.
   borisvpm), rotation v+ = R v- with R of Eq. borisrotsol, second half kick
   (Eq. borisscheme).  eps(b) u is the cross product u x b. */
void orc_push_free(double *v, const double *E, const double *B, double q, double m, double dt) {
    double h = q * dt / (2.0 * m);
    double b[3] = {h * B[0], h * B[1], h * B[2]};
    double bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    double vm[3], vp[3];
    for (int a = 0; a < 3; ++a) vm[a] = v[a] + h * E[a];
    double vmxb[3] = {vm[1] * b[2] - vm[2] * b[1], vm[2] * b[0] - vm[0] * b[2],
                      vm[0] * b[1] - vm[1] * b[0]};
    double vmdb = vm[0] * b[0] + vm[1] * b[1] + vm[2] * b[2];
    for (int a = 0; a < 3; ++a)
        vp[a] = ((1.0 - bb) * vm[a] + 2.0 * b[a] * vmdb + 2.0 * vmxb[a]) / (1.0 + bb);
    for (int a = 0; a < 3; ++a) v[a] = vp[a] + h * E[a];
}

static double det3(const double M[3][3]) {
    return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
           M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
           M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}

/* Bound species: modified Boris scheme (Appendix A.2).  Kick with the Lorentz
   force plus the Hooke term: v- = v + (dt/2)((q/m)E - w0^2 D) (Eq.
   modborisvpm), then the implicit-midpoint rotation with damping (Eq.
   modborisBrot read as (v+ - v-)/dt = [(q/m) eps(B) - Gamma](v+ + v-)/2),
   i.e. (I + (dt/2)Gamma - eps(b)) v+ = (I - (dt/2)Gamma + eps(b)) v-, solved
   here by Cramer's rule; second kick; drift D += dt v (Eq. discrvel).
   D is the displacement from the anchor in metres. */
/* The same with a full symmetric binding tensor: the Hooke term becomes
   Omega^2 D with Omega^2 = diag(omega0^2) + the off-diagonal entries w2off
   (xy, xz, yz); w2off == NULL is the diagonal case. */
void orc_push_bound_tensor(double *v, double *D, const double *E, const double *B, double q,
                           double m, double dt, const double *omega0, const double *w2off,
                           const double *gamma);

void orc_push_bound(double *v, double *D, const double *E, const double *B, double q, double m,
                    double dt, const double *omega0, const double *gamma) {
    orc_push_bound_tensor(v, D, E, B, q, m, dt, omega0, NULL, gamma);
}

void orc_push_bound_tensor(double *v, double *D, const double *E, const double *B, double q,
                           double m, double dt, const double *omega0, const double *w2off,
                           const double *gamma) {
    double h = q * dt / (2.0 * m);
    double b[3] = {h * B[0], h * B[1], h * B[2]};
    double kick[3], vm[3];
    for (int a = 0; a < 3; ++a) {
        double hooke = omega0[a] * omega0[a] * D[a];
        if (w2off) {
            /* off-diagonal entries of row a: (0,1) xy, (0,2) xz, (1,2) yz */
            const double o1 = a == 0 ? w2off[0] : a == 1 ? w2off[0] : w2off[1];
            const double o2 = a == 0 ? w2off[1] : a == 1 ? w2off[2] : w2off[2];
            const int b1 = a == 0 ? 1 : 0, b2 = a == 2 ? 1 : 2;
            hooke += o1 * D[b1] + o2 * D[b2];
        }
        kick[a] = 0.5 * dt * (q / m * E[a] - hooke);
        vm[a] = v[a] + kick[a];
    }
    /* matrix of u -> u x b */
    double X[3][3] = {{0.0, b[2], -b[1]}, {-b[2], 0.0, b[0]}, {b[1], -b[0], 0.0}};
    double L[3][3], rhs[3];
    for (int r = 0; r < 3; ++r) {
        rhs[r] = (1.0 - 0.5 * dt * gamma[r]) * vm[r];
        for (int c = 0; c < 3; ++c) {
            L[r][c] = (r == c ? 1.0 + 0.5 * dt * gamma[r] : 0.0) - X[r][c];
            rhs[r] += X[r][c] * vm[c];
        }
    }
    double det = det3(L);
    double vp[3];
    for (int c = 0; c < 3; ++c) {
        double M[3][3];
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) M[r][cc] = (cc == c) ? rhs[r] : L[r][cc];
        vp[c] = det3(M) / det;
    }
    for (int a = 0; a < 3; ++a) {
        v[a] = vp[a] + kick[a];
        D[a] += dt * v[a];
    }
}

/* Dirac carriers (Sec. 5): Boris push with the transverse mass m, the
   in-plane reading (carriers of a 2D sheet in the x-y plane carry no z
   momentum, so v_z is set to zero), then |v| renormalised to v_F.  A zero
   intermediate velocity keeps the previous direction. */
void orc_push_dirac(double *v, const double *E, const double *B, double q, double m, double dt,
                    double vF) {
    double vold[3] = {v[0], v[1], v[2]};
    orc_push_free(v, E, B, q, m, dt);
    v[2] = 0.0;
    double nrm = sqrt(v[0] * v[0] + v[1] * v[1]);
    if (nrm == 0.0) {
        for (int a = 0; a < 3; ++a) v[a] = vold[a];
        return;
    }
    v[0] = vF * v[0] / nrm;
    v[1] = vF * v[1] / nrm;
}

/* ------------------------------------------------------------------------ */
/* gather                                                                     */
/* ------------------------------------------------------------------------ */

/* Yee stagger (in cell units) of each component: E_x at (i+1/2, j, k), ...,
   B_x at (i, j+1/2, k+1/2), ... */
static const double STAG_E[3][3] = {{0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5}};
static const double STAG_B[3][3] = {{0, 0.5, 0.5}, {0.5, 0, 0.5}, {0.5, 0.5, 0}};

static double interp(const orc_sim *s, int order, const double *F, const double *stag,
                     const double *X) {
    double u[3];
    int i0[3];
    int nn = order + 1;
    for (int a = 0; a < 3; ++a) {
        u[a] = X[a] - stag[a];
        i0[a] = first_node(order, u[a]);
    }
    double acc = 0.0;
    int kn = s->dims == 3 ? nn : 1;
    for (int k = 0; k < kn; ++k)
        for (int j = 0; j < nn; ++j)
            for (int i = 0; i < nn; ++i) {
                double wz = s->dims == 3 ? shape(order, u[2], i0[2] + k) : 1.0;
                double w = shape(order, u[0], i0[0] + i) * shape(order, u[1], i0[1] + j) * wz;
                acc += w * fget(s, F, i0[0] + i, i0[1] + j, s->dims == 3 ? i0[2] + k : 0);
            }
    return acc;
}

/* E^n and B^n at a particle on the Yee stagger with the shape function W
   of Sec. 4.1 (CIC, or TSC for order 2). */
static void gather(const orc_sim *s, int order, const double *X, double *E, double *B) {
    for (int c = 0; c < 3; ++c) {
        E[c] = interp(s, order, s->E[c], STAG_E[c], X);
        if (s->Eext[c]) E[c] += interp(s, order, s->Eext[c], STAG_E[c], X);
        B[c] = interp(s, order, s->Bn[c], STAG_B[c], X);
    }
}

/* gather with the shape of the free particles (the simulation's order) */
void orc_gather(void *h, const double *X, double *E, double *B) {
    const orc_sim *s = (const orc_sim *)h;
    gather(s, s->shape_order, X, E, B);
}

/* Off-diagonal entries (xy, xz, yz, s^-2) of bound species k's binding
   tensor Omega^2 (Eq. modlorentz with a full symmetric tensor; the diagonal
   stays omega0^2). */
void orc_set_binding_offdiag(void *h, int k, const double *w2off) {
    orc_species *sp = &((orc_sim *)h)->sp[k];
    for (int a = 0; a < 3; ++a) sp->w2off[a] = w2off[a];
    sp->has_off = 1;
}

/* Shape order of the free and Dirac particles (1 CIC, 2 TSC); bound
   particles stay CIC.  Call before orc_add_species (the ion background of a
   species is deposited with its shape). */
void orc_set_shape_order(void *h, int order) {
    ((orc_sim *)h)->shape_order = order == 2 ? 2 : 1;
}

/* ------------------------------------------------------------------------ */
/* Esirkepov charge-conserving deposit (order 1)                              */
/* ------------------------------------------------------------------------ */

/* Current of one macro-particle (charge qw) moving on a straight line from X0
   to X1 (cell units, |X1 - X0| < 1 per axis) during dt.  Esirkepov's density
   decomposition W; J_x(i+1/2) - J_x(i-1/2) = -(qw / (dy dz dt)) W_x(i), so
   J_x(i+1/2) is minus the running sum of W_x.  vz is the out-of-plane velocity
   used by the 2D3V form. */
static void esirkepov(orc_sim *s, int order, const double *X0, const double *X1, double qw,
                      double vz) {
    const double dt = s->dt;
    const double *d = s->d;
    /* nodes touched by the start and end shapes: CIC 3, TSC 4 per axis */
    const int NS = order + 2;
    int lo[3];
    double S0[3][4], DS[3][4];
    int na = s->dims;
    for (int a = 0; a < na; ++a) {
        int c0 = first_node(order, X0[a]), c1 = first_node(order, X1[a]);
        lo[a] = c0 < c1 ? c0 : c1;
        for (int m = 0; m < NS; ++m) {
            S0[a][m] = shape(order, X0[a], lo[a] + m);
            DS[a][m] = shape(order, X1[a], lo[a] + m) - S0[a][m];
        }
    }
    if (s->dims == 3) {
        double fx = -qw / (d[1] * d[2] * dt);
        double fy = -qw / (d[0] * d[2] * dt);
        double fz = -qw / (d[0] * d[1] * dt);
        for (int k = 0; k < NS; ++k)
            for (int j = 0; j < NS; ++j) {
                double run = 0.0;
                for (int i = 0; i < NS; ++i) {
                    double W = DS[0][i] * (S0[1][j] * S0[2][k] + 0.5 * DS[1][j] * S0[2][k] +
                                           0.5 * S0[1][j] * DS[2][k] + DS[1][j] * DS[2][k] / 3.0);
                    run += W;
                    if (run != 0.0) fadd(s, s->J[0], lo[0] + i, lo[1] + j, lo[2] + k, fx * run);
                }
            }
        for (int k = 0; k < NS; ++k)
            for (int i = 0; i < NS; ++i) {
                double run = 0.0;
                for (int j = 0; j < NS; ++j) {
                    double W = DS[1][j] * (S0[0][i] * S0[2][k] + 0.5 * DS[0][i] * S0[2][k] +
                                           0.5 * S0[0][i] * DS[2][k] + DS[0][i] * DS[2][k] / 3.0);
                    run += W;
                    if (run != 0.0) fadd(s, s->J[1], lo[0] + i, lo[1] + j, lo[2] + k, fy * run);
                }
            }
        for (int j = 0; j < NS; ++j)
            for (int i = 0; i < NS; ++i) {
                double run = 0.0;
                for (int k = 0; k < NS; ++k) {
                    double W = DS[2][k] * (S0[0][i] * S0[1][j] + 0.5 * DS[0][i] * S0[1][j] +
                                           0.5 * S0[0][i] * DS[1][j] + DS[0][i] * DS[1][j] / 3.0);
                    run += W;
                    if (run != 0.0) fadd(s, s->J[2], lo[0] + i, lo[1] + j, lo[2] + k, fz * run);
                }
            }
    } else {
        double fx = -qw / (d[1] * d[2] * dt);
        double fy = -qw / (d[0] * d[2] * dt);
        double fz = qw * vz / (d[0] * d[1] * d[2]);
        for (int j = 0; j < NS; ++j) {
            double run = 0.0;
            for (int i = 0; i < NS; ++i) {
                run += DS[0][i] * (S0[1][j] + 0.5 * DS[1][j]);
                if (run != 0.0) fadd(s, s->J[0], lo[0] + i, lo[1] + j, 0, fx * run);
            }
        }
        for (int i = 0; i < NS; ++i) {
            double run = 0.0;
            for (int j = 0; j < NS; ++j) {
                run += DS[1][j] * (S0[0][i] + 0.5 * DS[0][i]);
                if (run != 0.0) fadd(s, s->J[1], lo[0] + i, lo[1] + j, 0, fy * run);
            }
        }
        for (int j = 0; j < NS; ++j)
            for (int i = 0; i < NS; ++i) {
                double W = S0[0][i] * S0[1][j] + 0.5 * DS[0][i] * S0[1][j] +
                           0.5 * S0[0][i] * DS[1][j] + DS[0][i] * DS[1][j] / 3.0;
                if (W != 0.0) fadd(s, s->J[2], lo[0] + i, lo[1] + j, 0, fz * W);
            }
    }
}

/* one deposit with the shape of the free particles */
void orc_deposit_one(void *h, const double *X0, const double *X1, double qw, double vz) {
    orc_sim *s = (orc_sim *)h;
    esirkepov(s, s->shape_order, X0, X1, qw, vz);
}

/* ------------------------------------------------------------------------ */
/* material-edge reflection (Sec. 3, fully specular scattering)              */
/* ------------------------------------------------------------------------ */

/* Uniform in [0, 1) from the top 24 bits of a Philox word: exact in FP32, so
   a comparison with an FP32 probability decides alike in any precision. */
static double u24(uint32_t x) { return (double)(x >> 8) / 16777216.0; }

/* Particle boundary rule (Sec. 3).  A particle that leaves the domain across
   a non-periodic face is reflected specularly.  A particle that leaves a
   material cell for a vacuum cell is reflected there too, unless the edges
   are open.  Reflection: for every axis a whose cell index changed, the
   position is mirrored about the crossed face; specular reflection also
   changes the sign of v_a.  A material-edge reflection across a single face
   is diffuse with probability p: the speed is kept and the new direction is
   drawn from Lambert's cosine law about the inward normal n -- cos(theta) =
   sqrt(u1), azimuth 2 pi u2 for 3D velocities; for the in-plane Dirac
   carriers the 2D law sin(theta) = 2 u1 - 1 in the sheet (v_z stays 0).  The
   draw of particle p of species k at step n is Philox-4x32-10 with key =
   seed and counter (p, n, k, DIFFUSE_STREAM): u0 decides (u0 < p, p rounded
   to FP32), u1 and u2 give the direction.  Returns 1 if reflected. */
static int reflect(const orc_sim *s, const orc_species *sp, int k, long p, const double *X0,
                   double *X1, double *v) {
    int c0[3], c1[3], moved = 0, ncross = 0, axis = 0;
    int na = s->dims;
    for (int a = 0; a < 3; ++a) {
        c0[a] = (int)floor(X0[a]);
        c1[a] = (a < na) ? (int)floor(X1[a]) : c0[a];
        if (c1[a] != c0[a]) { moved = 1; ++ncross; axis = a; }
    }
    if (!moved) return 0;
    int outside = 0;
    for (int a = 0; a < na; ++a)
        if (s->bc[a] != BC_PERIODIC && (c1[a] < 0 || c1[a] >= s->n[a])) outside = 1;
    int edge = !outside && !s->open_edges &&
               mask_at(s, c0[0], c0[1], c0[2]) && !mask_at(s, c1[0], c1[1], c1[2]);
    if (!outside && !edge) return 0;
    int diffuse = 0;
    double u1 = 0.0, u2 = 0.0;
    if (edge && ncross == 1 && s->p_diffuse > 0.0 && !(sp->kind == KIND_DIRAC && axis == 2)) {
        uint32_t ctr[4] = {(uint32_t)p, (uint32_t)s->step, (uint32_t)k, DIFFUSE_STREAM};
        uint32_t key[2] = {(uint32_t)s->diff_seed, (uint32_t)(s->diff_seed >> 32)};
        uint32_t r[4];
        orc_philox(ctr, key, r);
        diffuse = u24(r[0]) < (double)(float)s->p_diffuse;
        u1 = u24(r[1]);
        u2 = u24(r[2]);
    }
    for (int a = 0; a < na; ++a) {
        if (c1[a] == c0[a]) continue;
        double face = (double)(c1[a] > c0[a] ? c1[a] : c0[a]);
        X1[a] = 2.0 * face - X1[a];
        if (!diffuse) v[a] = -v[a];
    }
    if (diffuse) {
        const double nin = c1[axis] > c0[axis] ? -1.0 : 1.0; /* inward normal along axis */
        const double speed = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (sp->kind == KIND_DIRAC) {
            const double st = 2.0 * u1 - 1.0, ct = sqrt(1.0 - st * st);
            v[axis] = nin * speed * ct;
            v[1 - axis] = speed * st;
            v[2] = 0.0;
        } else {
            const double ct = sqrt(u1), st = sqrt(1.0 - u1), ph = 2.0 * PI * u2;
            v[axis] = nin * speed * ct;
            v[(axis + 1) % 3] = speed * st * cos(ph);
            v[(axis + 2) % 3] = speed * st * sin(ph);
        }
    }
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Yee field update with CPML and the soft source                            */
/* ------------------------------------------------------------------------ */

/* B^n = B^{n-1/2} - (dt/2) curl E^n with the plain Yee curl. */
static void compute_Bn(orc_sim *s) {
    const double *dd = s->d;
    double hdt = 0.5 * s->dt;
    int D3 = s->dims == 3;
#ifdef _OPENMP
#pragma omp parallel for collapse(2) schedule(static)
#endif
    for (int k = 0; k < s->n[2]; ++k)
        for (int j = 0; j < s->n[1]; ++j)
            for (int i = 0; i < s->n[0]; ++i) {
                long c = idx3(s, i, j, k);
                double dEz_dy = (fget(s, s->E[2], i, j + 1, k) - fget(s, s->E[2], i, j, k)) / dd[1];
                double dEy_dz = D3 ? (fget(s, s->E[1], i, j, k + 1) - fget(s, s->E[1], i, j, k)) / dd[2] : 0.0;
                double dEx_dz = D3 ? (fget(s, s->E[0], i, j, k + 1) - fget(s, s->E[0], i, j, k)) / dd[2] : 0.0;
                double dEz_dx = (fget(s, s->E[2], i + 1, j, k) - fget(s, s->E[2], i, j, k)) / dd[0];
                double dEy_dx = (fget(s, s->E[1], i + 1, j, k) - fget(s, s->E[1], i, j, k)) / dd[0];
                double dEx_dy = (fget(s, s->E[0], i, j + 1, k) - fget(s, s->E[0], i, j, k)) / dd[1];
                s->Bn[0][c] = s->B[0][c] - hdt * (dEz_dy - dEy_dz);
                s->Bn[1][c] = s->B[1][c] - hdt * (dEx_dz - dEz_dx);
                s->Bn[2][c] = s->B[2][c] - hdt * (dEy_dx - dEx_dy);
            }
}

/* Derivative of a field along axis a plus its CPML memory term.  psi is
   updated in place: psi = b psi + a * deriv (Roden-Gedney recursive
   convolution, kappa = 1).  coef_b/coef_a are the per-axis profiles at the
   component's position along a; pos_index indexes them. */
static double with_psi(const orc_sim *s, int a, double *psi, long c, const double *coef_b,
                       const double *coef_a, int pos_index, double deriv) {
    if (s->bc[a] != BC_PML || !psi) return deriv;
    psi[c] = coef_b[pos_index] * psi[c] + coef_a[pos_index] * deriv;
    return deriv + psi[c];
}

static void source_current(orc_sim *s) {
    if (!s->src_on) return;
    double t = (s->step + 0.5) * s->dt;
    double tt = t - s->t0;
    double g = exp(-2.0 * log(2.0) * tt * tt / (s->tau * s->tau)) * sin(s->omega * tt);
    double eta0 = mu0() * C_LIGHT;
    double Js = -2.0 * s->E0 / (eta0 * s->d[s->inc]) * g;
    for (int k = 0; k < s->n[2]; ++k)
        for (int j = 0; j < s->n[1]; ++j)
            for (int i = 0; i < s->n[0]; ++i) {
                int ijk[3] = {i, j, k};
                if (ijk[s->inc] == s->src_idx) s->J[s->pol][idx3(s, i, j, k)] += Js;
            }
}

static void yee_update(orc_sim *s) {
    const double *dd = s->d;
    const double dt = s->dt;
    const double c2 = C_LIGHT * C_LIGHT;
    int D3 = s->dims == 3;
    /* B^{n+1/2} from E^n */
#ifdef _OPENMP
#pragma omp parallel for collapse(2) schedule(static)
#endif
    for (int k = 0; k < s->n[2]; ++k)
        for (int j = 0; j < s->n[1]; ++j)
            for (int i = 0; i < s->n[0]; ++i) {
                long c = idx3(s, i, j, k);
                double dEz_dy = (fget(s, s->E[2], i, j + 1, k) - fget(s, s->E[2], i, j, k)) / dd[1];
                double dEy_dz = D3 ? (fget(s, s->E[1], i, j, k + 1) - fget(s, s->E[1], i, j, k)) / dd[2] : 0.0;
                double dEx_dz = D3 ? (fget(s, s->E[0], i, j, k + 1) - fget(s, s->E[0], i, j, k)) / dd[2] : 0.0;
                double dEz_dx = (fget(s, s->E[2], i + 1, j, k) - fget(s, s->E[2], i, j, k)) / dd[0];
                double dEy_dx = (fget(s, s->E[1], i + 1, j, k) - fget(s, s->E[1], i, j, k)) / dd[0];
                double dEx_dy = (fget(s, s->E[0], i, j + 1, k) - fget(s, s->E[0], i, j, k)) / dd[1];
                /* B_x at (i, j+1/2, k+1/2): d/dy at half position j, d/dz at half k */
                double tBxy = with_psi(s, 1, s->psiB[1][0], c, s->bh[1], s->ah[1], j, dEz_dy);
                double tBxz = D3 ? with_psi(s, 2, s->psiB[2][0], c, s->bh[2], s->ah[2], k, dEy_dz) : 0.0;
                /* B_y at (i+1/2, j, k+1/2) */
                double tByz = D3 ? with_psi(s, 2, s->psiB[2][1], c, s->bh[2], s->ah[2], k, dEx_dz) : 0.0;
                double tByx = with_psi(s, 0, s->psiB[0][1], c, s->bh[0], s->ah[0], i, dEz_dx);
                /* B_z at (i+1/2, j+1/2, k) */
                double tBzx = with_psi(s, 0, s->psiB[0][2], c, s->bh[0], s->ah[0], i, dEy_dx);
                double tBzy = with_psi(s, 1, s->psiB[1][2], c, s->bh[1], s->ah[1], j, dEx_dy);
                s->B[0][c] -= dt * (tBxy - tBxz);
                s->B[1][c] -= dt * (tByz - tByx);
                s->B[2][c] -= dt * (tBzx - tBzy);
            }
    /* E^{n+1} from B^{n+1/2} and J^{n+1/2} */
#ifdef _OPENMP
#pragma omp parallel for collapse(2) schedule(static)
#endif
    for (int k = 0; k < s->n[2]; ++k)
        for (int j = 0; j < s->n[1]; ++j)
            for (int i = 0; i < s->n[0]; ++i) {
                long c = idx3(s, i, j, k);
                double dBz_dy = (fget(s, s->B[2], i, j, k) - fget(s, s->B[2], i, j - 1, k)) / dd[1];
                double dBy_dz = D3 ? (fget(s, s->B[1], i, j, k) - fget(s, s->B[1], i, j, k - 1)) / dd[2] : 0.0;
                double dBx_dz = D3 ? (fget(s, s->B[0], i, j, k) - fget(s, s->B[0], i, j, k - 1)) / dd[2] : 0.0;
                double dBz_dx = (fget(s, s->B[2], i, j, k) - fget(s, s->B[2], i - 1, j, k)) / dd[0];
                double dBy_dx = (fget(s, s->B[1], i, j, k) - fget(s, s->B[1], i - 1, j, k)) / dd[0];
                double dBx_dy = (fget(s, s->B[0], i, j, k) - fget(s, s->B[0], i, j - 1, k)) / dd[1];
                /* E_x at (i+1/2, j, k): d/dy at integer j, d/dz at integer k */
                double tExy = with_psi(s, 1, s->psiE[1][0], c, s->be[1], s->ae[1], j, dBz_dy);
                double tExz = D3 ? with_psi(s, 2, s->psiE[2][0], c, s->be[2], s->ae[2], k, dBy_dz) : 0.0;
                double tEyz = D3 ? with_psi(s, 2, s->psiE[2][1], c, s->be[2], s->ae[2], k, dBx_dz) : 0.0;
                double tEyx = with_psi(s, 0, s->psiE[0][1], c, s->be[0], s->ae[0], i, dBz_dx);
                double tEzx = with_psi(s, 0, s->psiE[0][2], c, s->be[0], s->ae[0], i, dBy_dx);
                double tEzy = with_psi(s, 1, s->psiE[1][2], c, s->be[1], s->ae[1], j, dBx_dy);
                /* eps dE/dt = curl H - J (Eq. consteps) */
                double er = s->eps_r ? s->eps_r[c] : 1.0;
                s->E[0][c] += dt / er * (c2 * (tExy - tExz) - s->J[0][c] / EPS0);
                s->E[1][c] += dt / er * (c2 * (tEyz - tEyx) - s->J[1][c] / EPS0);
                s->E[2][c] += dt / er * (c2 * (tEzx - tEzy) - s->J[2][c] / EPS0);
            }
}

/* ------------------------------------------------------------------------ */
/* one PIC step                                                               */
/* ------------------------------------------------------------------------ */

static void push_species(orc_sim *s, orc_species *sp, int k) {
    const double dt = s->dt;
    long long nrefl = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(+ : nrefl)
#endif
    for (long p = 0; p < sp->n; ++p) {
        double X0[3], X1[3], E[3], B[3];
        double *v = &sp->V[3 * p];
        particle_pos(s, sp, p, X0);
        const int order = species_order(s, sp);
        gather(s, order, X0, E, B);
        if (sp->kind == KIND_BOUND) {
            double *D = &sp->D[3 * p];
            orc_push_bound_tensor(v, D, E, B, sp->q, sp->m, dt, sp->omega0,
                                  sp->has_off ? sp->w2off : NULL, sp->gamma);
            particle_pos(s, sp, p, X1);
        } else {
            if (sp->kind == KIND_FREE) orc_push_free(v, E, B, sp->q, sp->m, dt);
            else orc_push_dirac(v, E, B, sp->q, sp->m, dt, sp->vF);
            for (int a = 0; a < 3; ++a) X1[a] = X0[a] + (a < s->dims ? dt * v[a] / s->d[a] : 0.0);
            nrefl += reflect(s, sp, k, p, X0, X1, v);
        }
        esirkepov(s, order, X0, X1, sp->q * sp->w, v[2]);
        if (sp->kind != KIND_BOUND) {
            for (int a = 0; a < s->dims; ++a) {
                if (s->bc[a] == BC_PERIODIC) {
                    double n = s->n[a];
                    X1[a] = fmod(X1[a], n);
                    if (X1[a] < 0.0) X1[a] += n;
                    if (X1[a] >= n) X1[a] -= n;
                }
                sp->X[3 * p + a] = X1[a];
            }
        }
    }
    sp->nrefl += nrefl;
}

/* threads the step uses (1 in the serial build) */
int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_step(void *h, int nsteps) {
    orc_sim *s = (orc_sim *)h;
    for (int it = 0; it < nsteps; ++it) {
        compute_Bn(s);
        for (int k = 0; k < s->nsp; ++k) push_species(s, &s->sp[k], k);
        source_current(s);
        yee_update(s);
        for (int c = 0; c < 3; ++c) {
            memcpy(s->Jlast[c], s->J[c], s->ncell * sizeof(double));
            memset(s->J[c], 0, s->ncell * sizeof(double));
        }
        s->step++;
    }
}

/* ------------------------------------------------------------------------ */
/* access and diagnostics                                                     */
/* ------------------------------------------------------------------------ */

/* comp 0..2: E, 3..5: B (half step), 6..8: J of the last step, 9..11: B^n of
   the last gather */
void orc_get_field(void *h, int comp, double *out) {
    orc_sim *s = (orc_sim *)h;
    const double *src = comp < 3 ? s->E[comp] : comp < 6 ? s->B[comp - 3]
                      : comp < 9 ? s->Jlast[comp - 6] : s->Bn[comp - 9];
    memcpy(out, src, s->ncell * sizeof(double));
}

void orc_set_field(void *h, int comp, const double *in) {
    orc_sim *s = (orc_sim *)h;
    double *dst = comp < 3 ? s->E[comp] : s->B[comp - 3];
    memcpy(dst, in, s->ncell * sizeof(double));
}

/* J accumulated since the last step (for single-deposit tests) */
void orc_get_J(void *h, int comp, double *out) {
    orc_sim *s = (orc_sim *)h;
    memcpy(out, s->J[comp], s->ncell * sizeof(double));
}

void orc_clear_J(void *h) {
    orc_sim *s = (orc_sim *)h;
    for (int c = 0; c < 3; ++c) memset(s->J[c], 0, s->ncell * sizeof(double));
}

long orc_species_count(void *h, int k) { return ((orc_sim *)h)->sp[k].n; }

void orc_get_species(void *h, int k, double *X, double *V, double *D, long long *nrefl) {
    orc_sim *s = (orc_sim *)h;
    orc_species *sp = &s->sp[k];
    if (sp->n > 0) {
        memcpy(X, sp->X, 3 * sp->n * sizeof(double));
        memcpy(V, sp->V, 3 * sp->n * sizeof(double));
        memcpy(D, sp->D, 3 * sp->n * sizeof(double));
    }
    *nrefl = sp->nrefl;
}

/* Histogram of the kinetic energy E = m |v|^2 / 2 of species k's particles
   (the relaxation study of Sec. 2 fits the high-energy tail of this
   histogram): out[b], b < nbins, counts E in [b D, (b+1) D), D = e_max /
   nbins; out[nbins] counts E >= e_max.  E is formed as
   0.5 m ((vx vx + vy vy) + vz vz) and the bin as floor(E / D), each
   operation rounded once. */
void orc_energy_histogram(void *h, int k, double e_max, int nbins, uint64_t *out) {
    orc_sim *s = (orc_sim *)h;
    orc_species *sp = &s->sp[k];
    const double D = e_max / nbins;
    memset(out, 0, (size_t)(nbins + 1) * sizeof(uint64_t));
    for (long p = 0; p < sp->n; ++p) {
        const double *v = &sp->V[3 * p];
        double E = 0.5 * sp->m * ((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
        long b;
        if (E >= e_max) b = nbins;
        else {
            b = (long)floor(E / D);
            if (b > nbins - 1) b = nbins - 1;
        }
        out[b] += 1;
    }
}

/* Particles per cell (cell of the current position), x fastest. */
void orc_cell_counts(void *h, int k, int32_t *out) {
    orc_sim *s = (orc_sim *)h;
    orc_species *sp = &s->sp[k];
    memset(out, 0, s->ncell * sizeof(int32_t));
    for (long p = 0; p < sp->n; ++p) {
        double X[3];
        particle_pos(s, sp, p, X);
        int c[3] = {(int)floor(X[0]), (int)floor(X[1]), s->dims == 3 ? (int)floor(X[2]) : 0};
        if (!wrap_index(s, c)) continue;
        out[idx3(s, c[0], c[1], c[2])] += 1;
    }
}

/* eps_r E_a at the E_a node of cell (i, j, k), with the boundary rule of fget */
static double dget(const orc_sim *s, int a, int i, int j, int k) {
    int ijk[3] = {i, j, k};
    if (!wrap_index(s, ijk)) return 0.0;
    long c = idx3(s, ijk[0], ijk[1], ijk[2]);
    return (s->eps_r ? s->eps_r[c] : 1.0) * s->E[a][c];
}

/* out[0..nsp-1]: kinetic energy sum(1/2 m w |v|^2) per species (J);
   out[8]: electric field energy, out[9]: magnetic (B at the half step) (J);
   out[10]: max |div (eps_r E) - rho/eps0|, out[11]: RMS of the same, out[12]: max |rho/eps0|. */
void orc_diag(void *h, double *out) {
    orc_sim *s = (orc_sim *)h;
    for (int k = 0; k < 13; ++k) out[k] = 0.0;
    for (int k = 0; k < s->nsp; ++k) {
        orc_species *sp = &s->sp[k];
        double e = 0.0;
        for (long p = 0; p < sp->n; ++p) {
            const double *v = &sp->V[3 * p];
            e += 0.5 * sp->m * sp->w * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        }
        out[k] = e;
    }
    double V = s->d[0] * s->d[1] * s->d[2];
    double ue = 0.0, ub = 0.0;
    for (long c = 0; c < s->ncell; ++c)
        for (int a = 0; a < 3; ++a) {
            ue += 0.5 * EPS0 * s->E[a][c] * s->E[a][c] * V;
            ub += 0.5 / mu0() * s->B[a][c] * s->B[a][c] * V;
        }
    out[8] = ue; out[9] = ub;
    double *rho = (double *)malloc(s->ncell * sizeof(double));
    orc_rho(s, rho);
    double rmax = 0.0, rsum = 0.0, qmax = 0.0;
    for (int k = 0; k < s->n[2]; ++k)
        for (int j = 0; j < s->n[1]; ++j)
            for (int i = 0; i < s->n[0]; ++i) {
                long c = idx3(s, i, j, k);
                /* Gauss's law for D = eps0 eps_r E (eps_r 1 in vacuum) */
                double div = (dget(s, 0, i, j, k) - dget(s, 0, i - 1, j, k)) / s->d[0] +
                             (dget(s, 1, i, j, k) - dget(s, 1, i, j - 1, k)) / s->d[1];
                if (s->dims == 3)
                    div += (dget(s, 2, i, j, k) - dget(s, 2, i, j, k - 1)) / s->d[2];
                double r = div - rho[c] / EPS0;
                if (fabs(r) > rmax) rmax = fabs(r);
                rsum += r * r;
                if (fabs(rho[c] / EPS0) > qmax) qmax = fabs(rho[c] / EPS0);
            }
    out[10] = rmax;
    out[11] = sqrt(rsum / s->ncell);
    out[12] = qmax;
    free(rho);
}

/* ------------------------------------------------------------------------ */
/* paper formulas used for input checks                                       */
/* ------------------------------------------------------------------------ */

/* Fermi energy of a 3D electron gas of density n (Sec. 2), with the exponent
   read as 2/3: E_F = hbar^2 / (2m) (3 pi^2 n)^(2/3). */
double orc_fermi_energy(double n, double m) {
    const double HBAR = 1.054571817e-34;
    return HBAR * HBAR / (2.0 * m) * pow(3.0 * PI * PI * n, 2.0 / 3.0);
}

/* Time-step stability limit of the modified Boris scheme coupled to Yee
   (Eq. dtlimit); in 2D only the in-plane cell sizes enter. */
double orc_dt_limit(int dims, const double *d, double omega_b, double omega_p) {
    double inv = 1.0 / (d[0] * d[0]) + 1.0 / (d[1] * d[1]);
    if (dims == 3) inv += 1.0 / (d[2] * d[2]);
    return 1.0 / sqrt(0.25 * omega_b * omega_b + 0.25 * omega_p * omega_p +
                      C_LIGHT * C_LIGHT * inv);
}

/* ------------------------------------------------------------------------ */
/* Fermi-Dirac loader (Sec. 2, Eq. fddist)                                    */
/* ------------------------------------------------------------------------ */

/* Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw,
   "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of the
   Philox S-box with multipliers 0xD2511F53 / 0xCD9E8D57 and the Weyl key
   increments 0x9E3779B9 / 0xBB67AE85. */
void orc_philox(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out) {
    uint32_t x[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * x[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * x[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x[1] ^ k0;
        uint32_t y2 = hi0 ^ x[3] ^ k1;
        x[0] = y0; x[1] = lo1; x[2] = y2; x[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    for (int i = 0; i < 4; ++i) out[i] = x[i];
}

/* uniform double in (0,1) from two 32-bit words: 53 bits, half-ulp offset */
static double u53(uint32_t a, uint32_t b) {
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6) + 0.5) / 9007199254740992.0;
}

/* The six uniforms of particle `id`: u[0..2] position, u[3] |p|, u[4] cos
   theta, u[5] azimuth.  Counter (id_lo, id_hi, call, stream), key = seed. */
void orc_particle_uniforms(uint64_t seed, uint32_t stream, uint64_t id, double *u) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint32_t call = 0; call < 3; ++call) {
        uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), call, stream};
        uint32_t r[4];
        orc_philox(ctr, key, r);
        u[2 * call] = u53(r[0], r[1]);
        u[2 * call + 1] = u53(r[2], r[3]);
    }
}

/* Radial FD density of |p|: 3D (free/bound electrons) p^2 f(p^2/2m); the 2D
   Dirac sheet p f(v_F p), f(E) = 1 / (1 + exp((E - mu)/kT)) with mu = E_F. */
typedef struct { int dirac; double m, mu, kT, vF, pmax; } fd_law;

static double fd_g(const fd_law *L, double p) {
    double E = L->dirac ? L->vF * p : p * p / (2.0 * L->m);
    double f = 1.0 / (1.0 + exp((E - L->mu) / L->kT));
    return (L->dirac ? p : p * p) * f;
}

/* Composite Simpson on [a,b] with one panel */
static double simpson1(const fd_law *L, double a, double b) {
    return (b - a) / 6.0 * (fd_g(L, a) + 4.0 * fd_g(L, 0.5 * (a + b)) + fd_g(L, b));
}

#define FD_PANELS 65536
/* Invert F(p) = int_0^p g / int_0^pmax g at the given uniforms.  The
   cumulative integral is tabulated by Simpson's rule on 65536 panels, the
   panel holding the target is found by bisection on the table and the
   position inside it by bisection on a single-panel Simpson integral.
   Momentum range (the paper leaves it open): [0, pmax] with the carrier
   energy at pmax equal to mu + 40 kT.  At T = 0 the closed form is used. */
void orc_fd_invert(int dirac, double m, double EF, double T, double vF, long n,
                   const double *u, double *p_out) {
    fd_law L = {dirac, m, EF, KB * T, vF, 0.0};
    if (T <= 0.0) {
        double pF = dirac ? EF / vF : sqrt(2.0 * m * EF);
        for (long i = 0; i < n; ++i) p_out[i] = dirac ? pF * sqrt(u[i]) : pF * cbrt(u[i]);
        return;
    }
    double Emax = EF + 40.0 * L.kT;
    L.pmax = dirac ? Emax / vF : sqrt(2.0 * m * Emax);
    double h = L.pmax / FD_PANELS;
    double *F = (double *)malloc((FD_PANELS + 1) * sizeof(double));
    F[0] = 0.0;
    for (int k = 0; k < FD_PANELS; ++k) F[k + 1] = F[k] + simpson1(&L, k * h, (k + 1) * h);
    for (long i = 0; i < n; ++i) {
        double target = u[i] * F[FD_PANELS];
        int lo = 0, hi = FD_PANELS;
        while (hi - lo > 1) {
            int mid = (lo + hi) / 2;
            if (F[mid] <= target) lo = mid; else hi = mid;
        }
        double a = lo * h, b = (lo + 1) * h;
        for (int it = 0; it < 64; ++it) {
            double mid = 0.5 * (a + b);
            if (F[lo] + simpson1(&L, lo * h, mid) <= target) a = mid; else b = mid;
        }
        p_out[i] = 0.5 * (a + b);
    }
    free(F);
}

/* The loader (module I of the paper): for every material cell in linear
   order (x fastest) and every one of its ppc particles, particle id =
   rank * ppc + j draws its six uniforms; the position is uniform in the cell
   (or, when quiet, the j-th point of an m^dims lattice, m^dims = ppc), the
   direction is isotropic in 3D (cos theta = 2u - 1, azimuth 2 pi u) or
   in-plane for Dirac carriers, |p| follows the FD law above, v = p/m for free
   electrons, v = v_F p/|p| for Dirac carriers, v = 0 for bound electrons.
   Positions go out as cell index + offset in [0,1) like the ABI takes them.
   Returns the number of particles written (or the count needed when cell is
   NULL). */
long orc_fd_load(int dims, const int *n, const uint8_t *mask, int kind, double m, double EF,
                 double T, double vF, int ppc, int quiet, uint64_t seed, uint32_t stream,
                 int32_t *cell, double *off, double *V) {
    long ncell = (long)n[0] * n[1] * (dims == 3 ? n[2] : 1);
    long nmat = 0;
    for (long c = 0; c < ncell; ++c) nmat += (mask == NULL || mask[c] != 0);
    long np = nmat * ppc;
    if (!cell) return np;
    int lat = 0;
    if (quiet) {
        lat = (int)lround(pow((double)ppc, 1.0 / dims));
        long t = 1;
        for (int a = 0; a < dims; ++a) t *= lat;
        if (t != ppc) return -1;
    }
    double *u = (double *)malloc(6 * (np > 0 ? np : 1) * sizeof(double));
    double *up = (double *)malloc((np > 0 ? np : 1) * sizeof(double));
    double *pm = (double *)malloc((np > 0 ? np : 1) * sizeof(double));
    for (long id = 0; id < np; ++id) {
        orc_particle_uniforms(seed, stream, (uint64_t)id, &u[6 * id]);
        up[id] = u[6 * id + 3];
    }
    if (kind != KIND_BOUND) orc_fd_invert(kind == KIND_DIRAC, m, EF, T, vF, np, up, pm);
    long rank = 0;
    for (long c = 0; c < ncell; ++c) {
        if (mask && !mask[c]) continue;
        for (int j = 0; j < ppc; ++j) {
            long id = rank * ppc + j;
            const double *ui = &u[6 * id];
            cell[id] = (int32_t)c;
            if (quiet) {
                int a0 = j % lat, a1 = (j / lat) % lat, a2 = j / (lat * lat);
                off[3 * id + 0] = (a0 + 0.5) / lat;
                off[3 * id + 1] = (a1 + 0.5) / lat;
                off[3 * id + 2] = dims == 3 ? (a2 + 0.5) / lat : 0.5;
            } else {
                off[3 * id + 0] = ui[0];
                off[3 * id + 1] = ui[1];
                off[3 * id + 2] = ui[2];
            }
            double *v = &V[3 * id];
            if (kind == KIND_BOUND) {
                v[0] = v[1] = v[2] = 0.0;
            } else if (kind == KIND_DIRAC) {
                double phi = 2.0 * PI * ui[5];
                v[0] = vF * cos(phi);
                v[1] = vF * sin(phi);
                v[2] = 0.0;
            } else {
                double ct = 2.0 * ui[4] - 1.0;
                double st = sqrt(fmax(0.0, 1.0 - ct * ct));
                double phi = 2.0 * PI * ui[5];
                double sp = pm[id] / m;
                v[0] = sp * st * cos(phi);
                v[1] = sp * st * sin(phi);
                v[2] = sp * ct;
            }
        }
        ++rank;
    }
    free(u); free(up); free(pm);
    return np;
}
