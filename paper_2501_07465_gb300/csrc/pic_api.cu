// pic_api.cu -- the C ABI of include/pic.h: argument checks, device memory,
// the step schedule (sort every K steps, particle kernel, field kernel) and
// the copies between host arrays and the device layout.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "pic_sim.h"

namespace {

struct Allocator {
    pic_alloc_fn alloc = nullptr;
    pic_free_fn release = nullptr;
    void *ctx = nullptr;
};
Allocator g_alloc;
thread_local std::string g_err;

}  // namespace

namespace pic {

pic_status fail(pic_sim *s, pic_status st, const std::string &msg) {
    if (s) s->err = msg;
    g_err = msg;
    return st;
}



void *dalloc(pic_sim *s, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void *p = nullptr;
    if (g_alloc.alloc) {
        p = g_alloc.alloc(bytes, (void *)s->stream, g_alloc.ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p && ((uintptr_t)p & 255u)) {
        // field arrays feed TMA tensor maps (16-byte aligned at least): a
        // caller's allocator must align to 256 bytes
        if (g_alloc.release) g_alloc.release(p, bytes, (void *)s->stream, g_alloc.ctx);
        s->err = "allocator returned memory not aligned to 256 bytes";
        p = nullptr;
    }
    if (p) {
        s->bufs.push_back({p, bytes});
        s->bytes += bytes;
    }
    return p;
}

void *raw_alloc(size_t bytes, cudaStream_t stream) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void *p = nullptr;
    if (g_alloc.alloc) return g_alloc.alloc(bytes, (void *)stream, g_alloc.ctx);
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void raw_free(void *p, size_t bytes, cudaStream_t stream) {
    if (!p) return;
    bytes = (bytes + 255) & ~(size_t)255;
    if (g_alloc.release) g_alloc.release(p, bytes, (void *)stream, g_alloc.ctx);
    else cudaFree(p);
}

void dfree(pic_sim *s, void *p) {
    if (!p) return;
    for (size_t i = 0; i < s->bufs.size(); ++i) {
        if (s->bufs[i].p != p) continue;
        if (g_alloc.release) g_alloc.release(p, s->bufs[i].bytes, (void *)s->stream, g_alloc.ctx);
        else cudaFree(p);
        s->bytes -= s->bufs[i].bytes;
        s->bufs.erase(s->bufs.begin() + i);
        return;
    }
}


double dt_limit(const pic_sim *s, double wb2, double wp2) {
    double inv = 1.0 / (s->gd.dx * s->gd.dx) + 1.0 / (s->gd.dy * s->gd.dy);
    if (s->gd.dims == 3) inv += 1.0 / (s->gd.dz * s->gd.dz);
    return 1.0 / sqrt(0.25 * wb2 + 0.25 * wp2 + kC * kC * inv);
}

// CPML profile (Roden & Gedney, kappa = 1, alpha = 0, polynomial grading)
void cpml_profile(const pic_sim *s, int a, double pos, double *b, double *c) {
    const int n = s->g.n[a], P = s->gd.pml_cells;
    double depth = 0.0;
    if (pos < P) depth = P - pos;
    else if (pos > n - P) depth = pos - (n - P);
    const double eta0 = 1.0 / (kEps0 * kC);
    const double d = a == 0 ? s->gd.dx : a == 1 ? s->gd.dy : s->gd.dz;
    double smax = -(s->gd.pml_order + 1) * log(s->gd.pml_R0) / (2.0 * eta0 * P * d);
    double sigma = smax * pow(depth / P, s->gd.pml_order);
    *b = exp(-sigma * s->gd.dt / kEps0);
    *c = *b - 1.0;
}

pic_status setup_tiles(pic_sim *s) {
    TileP &tp = s->tp;
    const int dims = s->g.dims;
    for (int a = 0; a < 3; ++a) {
        int T = s->tun.tile[a];
        if (a == 2 && dims == 2) T = 1;
        if (T < 1) return fail(s, PIC_EINVAL, "tile dims must be >= 1");
        tp.T[a] = T;
        tp.nt[a] = (s->g.n[a] + T - 1) / T;
        // staged box: the tile plus a halo of 2 cells (3 for TSC shapes)
        const int halo = s->shape_order == 2 ? 3 : 2;
        tp.box[a] = (a == 2 && dims == 2) ? 1 : T + 2 * halo + 1;
    }
    tp.ntiles = tp.nt[0] * tp.nt[1] * tp.nt[2];
    tp.boxn = tp.box[0] * tp.box[1] * tp.box[2];
    s->psmem = particle_smem_bytes(tp);
    if (s->psmem > 227 * 1024 - 1024)
        return fail(s, PIC_EINVAL, "particle tile too large for shared memory");
    int per_sm = 0, per_sm_ext = 0, per_sm_tsc = 0;
    CK(s, particle_kernel_setup(dims, s->psmem, &per_sm, &per_sm_ext, &per_sm_tsc));
    if (per_sm < 1 || per_sm_ext < 1 || per_sm_tsc < 1)
        return fail(s, PIC_EINVAL, "particle tile does not fit on an SM");
    // beside the field work, one CTA per SM fewer leaves it room when the
    // kernel fits four (3 of 4 measured best); the plain kernel at three
    // CTAs per SM keeps all three (2 of 3 measured slower: 0.536 against
    // 0.496 ms per step on the 256^3 sphere)
    const int use_sm = (!s->tun.no_overlap && per_sm > 3) ? per_sm - 1 : per_sm;
    const int use_sm_ext = (!s->tun.no_overlap && per_sm_ext > 1) ? per_sm_ext - 1 : per_sm_ext;
    s->particle_ctas = s->tun.particle_ctas > 0 ? s->tun.particle_ctas : use_sm * s->num_sms;
    s->particle_ctas_ext =
        s->tun.particle_ctas > 0 ? s->tun.particle_ctas : use_sm_ext * s->num_sms;
    // the TSC kernel holds ~127 registers a thread: 2 CTAs fill an SM's
    // registers, so none is held back for the B pass
    const int use_sm_tsc = (!s->tun.no_overlap && per_sm_tsc > 2) ? per_sm_tsc - 1 : per_sm_tsc;
    s->particle_ctas_tsc =
        s->tun.particle_ctas > 0 ? s->tun.particle_ctas : use_sm_tsc * s->num_sms;
    // tile-indexed buffers
    dfree(s, s->active);
    dfree(s, s->nactive);
    dfree(s, s->tile_work);
    dfree(s, s->sort_count);
    const long long nt = tp.ntiles;
    // nactive holds the list length, then the particle kernel's tile counter
    // and finished-CTA count, the lean kernel's deferred-list length and the
    // finished-CTA count of the kernel that completes it (zero between
    // launches)
    if (!alloc_zero(s, &s->active, nt + 1) || !alloc_zero(s, &s->nactive, 8) ||
        !alloc_zero(s, &s->tile_work, active_tiles_work_len(nt)) ||
        !alloc_zero(s, &s->sort_count, nt + 1))
        return fail(s, PIC_ENOMEM, "tile buffers");
    for (int i = 0; i < s->nsp; ++i) {
        dfree(s, s->sp[i].tile_start);
        if (!alloc_zero(s, &s->sp[i].tile_start, nt + 1)) return fail(s, PIC_ENOMEM, "tile_start");
    }
    return PIC_OK;
}

SpeciesP species_params(const pic_sim *s, const Species &sp, int buf) {
    SpeciesP p{};
    const pic_species_desc &d = sp.desc;
    const double dt = s->gd.dt;
    const double dd[3] = {s->gd.dx, s->gd.dy, s->gd.dz};
    p.kind = d.kind;
    p.n = sp.n;
    p.cell = sp.cell[buf];
    for (int a = 0; a < 3; ++a) {
        p.o[a] = sp.o[buf][a];
        p.v[a] = sp.v[buf][a];
        p.anchor[a] = sp.anchor[buf][a];
        p.anchor32[a] = sp.anchor32[buf][a];
        p.disp[a] = sp.disp[buf][a];
        p.hw0sq[a] = (float)(0.5 * dt * d.omega0[a] * d.omega0[a]);
        p.dtd[a] = (float)(dt / dd[a]);
    }
    p.tile_start = sp.tile_start;
    p.hq = (float)(d.q * dt / (2.0 * d.m));
    p.gdt2 = (float)(0.5 * d.gamma[0] * dt);
    for (int a = 0; a < 3; ++a) p.gdt2v[a] = (float)(0.5 * d.gamma[a] * dt);
    p.aniso = d.kind == PIC_BOUND && !(d.gamma[0] == d.gamma[1] && d.gamma[1] == d.gamma[2]);
    for (int a = 0; a < 3; ++a) p.hw0off[a] = (float)(0.5 * dt * sp.w2off[a]);
    p.tensor = sp.has_off ? 1 : 0;
    p.vF = (float)d.v_F;
    p.dt = (float)dt;
    const double qw = d.q * sp.weight;
    p.jfac[0] = (float)(-qw / (dd[1] * dd[2] * dt));
    p.jfac[1] = (float)(-qw / (dd[0] * dd[2] * dt));
    p.jfac[2] = s->g.dims == 3 ? (float)(-qw / (dd[0] * dd[1] * dt))
                               : (float)(qw / (dd[0] * dd[1] * dd[2]));
    p.nrefl = sp.nrefl;
    p.pid = sp.pid[buf];
    return p;
}

pic_status ensure_rank_cap(pic_sim *s, long long n) {
    if (n <= s->rank_cap) return PIC_OK;
    dfree(s, s->sort_rank);
    if (!alloc_zero(s, &s->sort_rank, n)) return fail(s, PIC_ENOMEM, "sort rank buffer");
    s->rank_cap = n;
    return PIC_OK;
}

// counting sort of species i by tile: buffer cur -> 1 - cur
pic_status sort_species(pic_sim *s, int i) {
    Species &sp = s->sp[i];
    const TileP &tp = s->tp;
    pic_status st = ensure_rank_cap(s, sp.n);
    if (st != PIC_OK) return st;
    if (!s->scan_tmp) {
        long long need = std::max<long long>(scan_tmp_len(tp.ntiles), scan_tmp_len(s->g.ncell));
        if (!alloc_zero(s, &s->scan_tmp, need)) return fail(s, PIC_ENOMEM, "scan tmp");
    }
    CK(s, cudaMemsetAsync(s->sort_count, 0, (tp.ntiles + 1) * sizeof(int), s->stream));
    SpeciesP src = species_params(s, sp, sp.cur);
    SpeciesP dst = species_params(s, sp, 1 - sp.cur);
    CK(s, launch_tile_histogram(s->g, tp, src.cell, sp.n, s->sort_count, s->sort_rank, s->stream));
    CK(s, launch_scan_int(s->sort_count, sp.tile_start, tp.ntiles, s->scan_tmp, 0, s->stream));
    CK(s, launch_tile_scatter(s->g, tp, src, sp.pid[sp.cur], dst, sp.pid[1 - sp.cur],
                              sp.tile_start, s->sort_rank, s->tun.tile_order == 2, s->stream));
    s->launches += 2 + scan_kernel_count(tp.ntiles);
    if (s->tun.tile_order == 0) {
        // cell-interleaved order inside each tile, back into the first buffer
        CK(s, launch_tile_interleave(tp, dst, sp.pid[1 - sp.cur], src, sp.pid[sp.cur],
                                     sp.tile_start, s->sort_rank, kParticleThreads, s->stream));
        s->launches += 1;
        return PIC_OK;
    }
    sp.cur = 1 - sp.cur;
    return PIC_OK;
}

pic_status rebuild_active(pic_sim *s) {
    if (!s->starts_dev) {
        s->starts_dev = (int **)dalloc(s, kMaxSpecies * sizeof(int *));
        if (!s->starts_dev) return fail(s, PIC_ENOMEM, "starts");
    }
    int *h[kMaxSpecies] = {};
    for (int i = 0; i < s->nsp; ++i) h[i] = s->sp[i].tile_start;
    CK(s, cudaMemcpyAsync(s->starts_dev, h, sizeof(h), cudaMemcpyHostToDevice, s->stream));
    // the host array must outlive the copy: synchronise (setup path only)
    CK(s, cudaStreamSynchronize(s->stream));
    CK(s, launch_active_tiles_work(s->tp, s->starts_dev, s->nsp, s->active, s->nactive,
                                   s->tile_work, s->stream));
    CK(s, cudaMemsetAsync(s->nactive + 1, 0, 2 * sizeof(int), s->stream));
    return PIC_OK;
}

pic_status sort_all(pic_sim *s, bool include_bound) {
    for (int i = 0; i < s->nsp; ++i) {
        if (!include_bound && s->sp[i].desc.kind == PIC_BOUND) continue;
        if (s->sp[i].n == 0) continue;
        pic_status st = sort_species(s, i);
        if (st != PIC_OK) return st;
    }
    s->since_sort = 0;
    return PIC_OK;
}

void record(pic_sim *s, int which, bool start, cudaStream_t on = nullptr) {
    if (!s->tun.timing) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, on ? on : s->stream);
    (start ? s->ev[which].start : s->ev[which].stop).push_back(e);
}

FieldP field_params(pic_sim *s) {
    FieldP f{};
    const int c = s->fcur, nx = 1 - c;
    for (int a = 0; a < 3; ++a) {
        f.E[a] = s->E[c][a];
        f.B[a] = s->B[c][a];
        f.En[a] = s->E[nx][a];
        f.Bn[a] = s->B[nx][a];
        f.J[a] = s->J[a];
        f.pml[a] = s->gd.bc[a] == PIC_BC_PML && (a < 2 || s->g.dims == 3);
        for (int q = 0; q < 4; ++q) {
            f.psi_in[a][q] = s->psi[c][a][q];
            f.psi_out[a][q] = s->psi[nx][a][q];
        }
        f.cb_e[a] = s->cb_e[a];
        f.ca_e[a] = s->ca_e[a];
        f.cb_h[a] = s->cb_h[a];
        f.ca_h[a] = s->ca_h[a];
    }
    f.jdirty = s->jdirty;
    f.jdirty_clear = s->jdirty;
    f.P = s->gd.pml_cells;
    f.src_on = s->gd.src_on;
    f.inc = s->gd.inc_axis;
    f.pol = s->gd.pol_axis;
    f.src_index = s->gd.src_index;
    const double dinc = s->gd.inc_axis == 0 ? s->gd.dx : s->gd.inc_axis == 1 ? s->gd.dy : s->gd.dz;
    const double eta0 = 1.0 / (kEps0 * kC);
    f.src_amp = -2.0 * s->gd.E0 / (eta0 * dinc);
    f.src_omega = s->gd.omega;
    f.src_tau = s->gd.tau;
    f.src_t0 = s->gd.t0;
    f.step_counter = s->step_counter;
    f.dt64 = s->gd.dt;
    f.c2dt = (float)(kC * kC * s->gd.dt);
    f.dt_eps0 = (float)(s->gd.dt / kEps0);
    f.keepJ = s->tun.keep_J;
    f.zchunk = s->tun.field_zchunk;
    f.nbx = s->nbx;
    f.nby = s->nby;
    f.nbz = s->nbz;
    // the split B pass feeds its interior blocks by TMA where the maps exist
    f.tma_b = (s->tun.field_mode == 2 && s->use_tma && !s->tun.field_plain && s->g.dims == 3) ? 1 : 0;
    f.wait_polls = s->tun.wait_polls > 0 ? s->tun.wait_polls : kWaitPolls;
    f.inv_eps = s->inv_eps;
    for (int k = 0; k < 4; ++k) {
        f.blk[k] = s->blk_lists ? s->blk_lists + s->blk_off[k] : nullptr;
        f.nblk[k] = s->blk_n[k];
    }
    return f;
}

ParticleLaunch particle_params(pic_sim *s) {
    ParticleLaunch P{};
    P.g = s->g;
    P.tp = s->tp;
    P.nsp = s->nsp;
    for (int i = 0; i < s->nsp; ++i) P.sp[i] = species_params(s, s->sp[i], s->sp[i].cur);
    for (int a = 0; a < 3; ++a) {
        P.E[a] = s->E[s->fcur][a];
        P.B[a] = s->B[s->fcur][a];
        P.J[a] = s->J[a];
    }
    P.mask = s->open_edges ? nullptr : s->mask_d;
    for (int a = 0; a < 3; ++a) P.Eext[a] = s->Eext[a];
    P.p_diffuse = (float)s->p_diffuse;
    P.diff_key[0] = (uint32_t)s->diff_seed;
    P.diff_key[1] = (uint32_t)(s->diff_seed >> 32);
    P.rng_step = (uint32_t)s->steps;
    P.shape = s->shape_order;
    P.jdirty = s->jdirty;
    P.nbx = s->nbx;
    P.nby = s->nby;
    P.nbz = s->nbz;
    P.zchunk = s->tun.field_zchunk;
    P.active = s->active;
    P.nactive = s->nactive;
    P.sched = s->nactive + 1;
    P.step_counter = s->step_counter;
    P.status = s->status;
    P.defer = s->defer;
    P.defer_count = s->nactive + 3;
    P.defer_sched = s->nactive + 4;
    return P;
}

bool alloc_external_field(pic_sim *s) {
    for (int c = 0; c < 3; ++c)
        if (!s->Eext[c] && !(s->Eext[c] = (float *)dalloc(s, s->g.ncell * sizeof(float))))
            return false;
    return true;
}

int particle_ctas_for(const pic_sim *s, const ParticleLaunch &P) {
    if (P.shape == 2) return s->particle_ctas_tsc;
    return particle_launch_ext(P) ? s->particle_ctas_ext : s->particle_ctas;
}

pic_status check_device_status(pic_sim *s) {
    int st = 0;
    if (s->group_stream) CK(s, cudaStreamSynchronize(s->group_stream));
    CK(s, cudaMemcpy(&st, s->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & kStatusTimeout) return fail(s, PIC_ETIMEOUT, "device wait timed out");
    if (st & kStatusBounds) return fail(s, PIC_EBOUNDS, "device bounds check fired");
    return PIC_OK;
}

}  // namespace pic

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------

extern "C" {

pic_status pic_set_allocator(pic_alloc_fn alloc, pic_free_fn release, void *ctx) {
    if ((alloc == nullptr) != (release == nullptr))
        return fail(nullptr, PIC_EINVAL, "alloc and free hooks must be set together");
    g_alloc.alloc = alloc;
    g_alloc.release = release;
    g_alloc.ctx = ctx;
    return PIC_OK;
}

const char *pic_last_error(const pic_sim *sim) {
    return sim ? sim->err.c_str() : g_err.c_str();
}

pic_status pic_create(const pic_grid_desc *gd, void *stream, pic_sim **out) {
    if (!gd || !out) return fail(nullptr, PIC_EINVAL, "null argument");
    *out = nullptr;
    const pic_grid_desc &d = *gd;
    if (d.dims != 2 && d.dims != 3) return fail(nullptr, PIC_EINVAL, "dims must be 2 or 3");
    if (d.nx < 1 || d.ny < 1 || d.nz < 1 || d.nx > 2048 || d.ny > 2048 || d.nz > 1024)
        return fail(nullptr, PIC_EINVAL, "grid size out of range (nx, ny <= 2048, nz <= 1024)");
    if (d.dims == 2 && d.nz != 1) return fail(nullptr, PIC_EINVAL, "2D grids need nz = 1");
    if (!(d.dx > 0 && d.dy > 0 && d.dz > 0 && d.dt > 0))
        return fail(nullptr, PIC_EINVAL, "cell sizes and dt must be positive");
    for (int a = 0; a < d.dims; ++a) {
        if (d.bc[a] != PIC_BC_PERIODIC && d.bc[a] != PIC_BC_PML)
            return fail(nullptr, PIC_EINVAL, "bc must be PIC_BC_PERIODIC or PIC_BC_PML");
        const int n = a == 0 ? d.nx : a == 1 ? d.ny : d.nz;
        if (d.bc[a] == PIC_BC_PML && (d.pml_cells < 1 || n < 2 * d.pml_cells + 1))
            return fail(nullptr, PIC_EINVAL, "PML axis needs n >= 2 * pml_cells + 1, pml_cells >= 1");
    }
    if (d.src_on) {
        if (d.inc_axis < 0 || d.inc_axis >= d.dims || d.pol_axis < 0 || d.pol_axis > 2 ||
            d.pol_axis == d.inc_axis)
            return fail(nullptr, PIC_EINVAL, "source axes invalid");
        const int n = d.inc_axis == 0 ? d.nx : d.inc_axis == 1 ? d.ny : d.nz;
        if (d.src_index < 0 || d.src_index >= n || !(d.tau > 0))
            return fail(nullptr, PIC_EINVAL, "source index or duration invalid");
    }
    pic_sim *s = new pic_sim();
    s->gd = d;
    if (s->gd.pml_R0 <= 0) s->gd.pml_R0 = 1e-8;
    if (s->gd.pml_order <= 0) s->gd.pml_order = 3;
    if (d.dims == 2) s->gd.bc[2] = PIC_BC_PERIODIC;
    if (dt_limit(s, 0.0, 0.0) <= d.dt) {
        delete s;
        return fail(nullptr, PIC_EDTLIMIT, "dt exceeds the Yee stability limit (Eq. dtlimit)");
    }
    s->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) !=
            cudaSuccess) {
        std::string m = cudaGetErrorString(cudaGetLastError());
        delete s;
        return fail(nullptr, PIC_ECUDA, "no CUDA device: " + m);
    }
    GridP &g = s->g;
    g.dims = d.dims;
    g.n[0] = d.nx;
    g.n[1] = d.ny;
    g.n[2] = d.nz;
    const double dd[3] = {d.dx, d.dy, d.dz};
    for (int a = 0; a < 3; ++a) {
        g.per[a] = s->gd.bc[a] == PIC_BC_PERIODIC;
        g.d[a] = (float)dd[a];
        g.inv_d[a] = (float)(1.0 / dd[a]);
    }
    g.dt = (float)d.dt;
    g.ncell = (long long)d.nx * d.ny * d.nz;
    // default tuning
    s->tun.tile[0] = d.dims == 3 ? 8 : 32;
    s->tun.tile[1] = d.dims == 3 ? 8 : 32;
    s->tun.tile[2] = d.dims == 3 ? 4 : 1;
    s->tun.sort_interval = 32;
    s->tun.field_mode = 2;
    s->tun.field_overlap = 1;
    s->tun.field_zchunk = 16;
    const long long nc = g.ncell;
    bool ok = true;
    for (int b = 0; b < 2; ++b)
        for (int c = 0; c < 3; ++c) {
            ok = ok && alloc_zero(s, &s->E[b][c], nc);
            ok = ok && alloc_zero(s, &s->B[b][c], nc);
        }
    for (int c = 0; c < 3; ++c) ok = ok && alloc_zero(s, &s->J[c], nc);
    s->nbx = (d.nx + kFieldBX - 1) / kFieldBX;
    s->nby = (d.ny + kFieldBY - 1) / kFieldBY;
    s->nbz = d.dims == 3 ? (d.nz + s->tun.field_zchunk - 1) / s->tun.field_zchunk : 1;
    ok = ok && alloc_zero(s, &s->jdirty, (size_t)s->nbx * s->nby * s->nbz);
    ok = ok && alloc_zero(s, &s->step_counter, 1) && alloc_zero(s, &s->status, 1);
    ok = ok && alloc_zero(s, &s->diag_acc, 1);
    if (!ok) {
        pic_destroy(s);
        return fail(nullptr, PIC_ENOMEM, "field allocation failed");
    }
    // CPML slabs and coefficients
    const int P = s->gd.pml_cells;
    for (int a = 0; a < d.dims; ++a) {
        if (s->gd.bc[a] != PIC_BC_PML) continue;
        long long slab = 2LL * P * (nc / g.n[a]);
        for (int b = 0; b < 2; ++b)
            for (int q = 0; q < 4; ++q) ok = ok && alloc_zero(s, &s->psi[b][a][q], slab);
        const int n = g.n[a];
        std::vector<float> be(n), ae(n), bh(n), ah(n);
        for (int i = 0; i < n; ++i) {
            double bb, cc;
            cpml_profile(s, a, (double)i, &bb, &cc);
            be[i] = (float)bb;
            ae[i] = (float)cc;
            cpml_profile(s, a, i + 0.5, &bb, &cc);
            bh[i] = (float)bb;
            ah[i] = (float)cc;
        }
        ok = ok && (s->cb_e[a] = (float *)dalloc(s, n * 4)) && (s->ca_e[a] = (float *)dalloc(s, n * 4)) &&
             (s->cb_h[a] = (float *)dalloc(s, n * 4)) && (s->ca_h[a] = (float *)dalloc(s, n * 4));
        if (!ok) break;
        cudaMemcpy(s->cb_e[a], be.data(), n * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(s->ca_e[a], ae.data(), n * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(s->cb_h[a], bh.data(), n * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(s->ca_h[a], ah.data(), n * 4, cudaMemcpyHostToDevice);
    }
    if (!ok) {
        pic_destroy(s);
        return fail(nullptr, PIC_ENOMEM, "CPML allocation failed");
    }
    pic_status st = setup_tiles(s);
    if (st != PIC_OK) {
        std::string m = s->err;
        pic_destroy(s);
        return fail(nullptr, st, m);
    }
    // TMA-fed field kernel where the layout allows it (row pitch a multiple of
    // 16 B; 32-bit offsets into the CPML slab arrays)
    if (g.ncell < (1LL << 31) && encode_field_maps(g, s->E, s->B, s->J, &s->maps) &&
        field_tma_setup() == cudaSuccess)
        s->use_tma = true;
    cudaGetLastError();
    if (build_block_lists(s) != PIC_OK) {
        std::string m = s->err;
        pic_destroy(s);
        return fail(nullptr, PIC_ENOMEM, m);
    }
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) {
        std::string m = cudaGetErrorString(cudaGetLastError());
        pic_destroy(s);
        return fail(nullptr, PIC_ECUDA, m);
    }
    *out = s;
    return PIC_OK;
}

pic_status pic_destroy(pic_sim *s) {
    if (!s) return PIC_OK;
    if (s->group) pic_group_remove(s->group, s);
    cudaStreamSynchronize(s->stream);
    if (s->aux) {
        cudaStreamSynchronize(s->aux);
        cudaStreamDestroy(s->aux);
        cudaEventDestroy(s->ev_fork);
        cudaEventDestroy(s->ev_join);
    }
    for (auto &b : s->bufs) {
        if (g_alloc.release) g_alloc.release(b.p, b.bytes, (void *)s->stream, g_alloc.ctx);
        else cudaFree(b.p);
    }
    for (auto &te : s->ev) {
        for (auto e : te.start) cudaEventDestroy(e);
        for (auto e : te.stop) cudaEventDestroy(e);
    }
    delete s;
    return PIC_OK;
}

pic_status pic_set_material_mask(pic_sim *s, const uint8_t *mask, size_t n) {
    if (!s || !mask) return fail(s, PIC_EINVAL, "null argument");
    if (s->group) return fail(s, PIC_ESTATE, "the simulation belongs to a group");
    if ((long long)n != s->g.ncell) return fail(s, PIC_EINVAL, "mask size must equal the cell count");
    if (s->nsp > 0) return fail(s, PIC_ESTATE, "set the mask before loading species");
    if (!s->mask_d && !(s->mask_d = (uint8_t *)dalloc(s, n))) return fail(s, PIC_ENOMEM, "mask");
    s->mask_h.assign(mask, mask + n);
    CK(s, cudaMemcpy(s->mask_d, mask, n, cudaMemcpyHostToDevice));
    return PIC_OK;
}

pic_status pic_set_tuning(pic_sim *s, const pic_tuning *t) {
    if (!s || !t) return fail(s, PIC_EINVAL, "null argument");
    if (s->steps > 0) return fail(s, PIC_ESTATE, "tuning must precede the first step");
    if (s->group) return fail(s, PIC_ESTATE, "the simulation belongs to a group");
    if (s->inv_eps && (t->field_mode == 1 || t->field_mode == 3))
        return fail(s, PIC_EINVAL, "a permittivity needs field_mode 2 (the split passes)");
    return pic::apply_tuning(s, t);
}

pic_status pic_set_permittivity(pic_sim *s, const float *eps_r, size_t n) {
    if (!s) return fail(s, PIC_EINVAL, "null handle");
    if (s->group) return fail(s, PIC_ESTATE, "the simulation belongs to a group");
    if (!eps_r) {  // back to vacuum
        dfree(s, s->inv_eps);
        s->inv_eps = nullptr;
        return PIC_OK;
    }
    if ((long long)n != s->g.ncell)
        return fail(s, PIC_EINVAL, "permittivity size must equal the cell count");
    if (s->tun.field_mode != 2)
        return fail(s, PIC_ESTATE, "a permittivity needs field_mode 2 (the split passes)");
    std::vector<float> inv(n);
    for (size_t c = 0; c < n; ++c) {
        if (!(eps_r[c] >= 1e-6f && eps_r[c] <= 1e6f))  // also rejects NaN
            return fail(s, PIC_EINVAL, "eps_r must be finite and positive (1e-6 .. 1e6)");
        inv[c] = 1.0f / eps_r[c];
    }
    if (!s->inv_eps && !(s->inv_eps = (float *)dalloc(s, n * sizeof(float))))
        return fail(s, PIC_ENOMEM, "permittivity");
    CK(s, cudaMemcpy(s->inv_eps, inv.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    return PIC_OK;
}

pic_status pic_set_external_field(pic_sim *s, const double *ex, const double *ey,
                                  const double *ez, size_t n) {
    if (!s) return fail(s, PIC_EINVAL, "null handle");
    if (s->group) return fail(s, PIC_ESTATE, "the simulation belongs to a group");
    if (!ex) {
        CK(s, cudaStreamSynchronize(s->stream));
        for (int c = 0; c < 3; ++c) {
            dfree(s, s->Eext[c]);
            s->Eext[c] = nullptr;
        }
        return PIC_OK;
    }
    if (!ey || !ez) return fail(s, PIC_EINVAL, "ex, ey and ez must all be given");
    if ((long long)n != s->g.ncell)
        return fail(s, PIC_EINVAL, "external field size must equal the cell count");
    const double *in[3] = {ex, ey, ez};
    std::vector<float> tmp(n);
    for (int c = 0; c < 3; ++c)
        for (size_t i = 0; i < n; ++i)
            if (!std::isfinite(in[c][i]) || std::fabs(in[c][i]) > 3e38)
                return fail(s, PIC_EINVAL, "external field must be finite");
    if (!alloc_external_field(s)) return fail(s, PIC_ENOMEM, "external field");
    CK(s, cudaStreamSynchronize(s->stream));
    for (int c = 0; c < 3; ++c) {
        for (size_t i = 0; i < n; ++i) tmp[i] = (float)in[c][i];
        CK(s, cudaMemcpy(s->Eext[c], tmp.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    }
    return PIC_OK;
}

pic_status pic_set_work_function(pic_sim *s, double W_eV) {
    if (!s) return fail(s, PIC_EINVAL, "null handle");
    if (s->group) return fail(s, PIC_ESTATE, "the simulation belongs to a group");
    if (!(std::fabs(W_eV) <= 1e3)) return fail(s, PIC_EINVAL, "|W| must be finite, <= 1e3 eV");
    if (W_eV == 0.0 || !s->mask_d) return pic_set_external_field(s, nullptr, nullptr, nullptr, 0);
    if (!alloc_external_field(s)) return fail(s, PIC_ENOMEM, "external field");
    CK(s, launch_work_function(s->g, s->mask_d, W_eV, s->Eext, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    return PIC_OK;
}

pic_status pic_set_binding_tensor(pic_sim *s, int k, const double *w2off) {
    if (!s || !w2off) return fail(s, PIC_EINVAL, "null argument");
    if (s->group) return fail(s, PIC_ESTATE, "the simulation belongs to a group");
    if (k < 0 || k >= s->nsp || s->sp[k].desc.kind != PIC_BOUND)
        return fail(s, PIC_EINVAL, "not a bound species");
    const double *w0 = s->sp[k].desc.omega0;
    const double xx = w0[0] * w0[0], yy = w0[1] * w0[1], zz = w0[2] * w0[2];
    const double xy = w2off[0], xz = w2off[1], yz = w2off[2];
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(w2off[a])) return fail(s, PIC_EINVAL, "entries must be finite");
    // positive definite (Sylvester): a restoring force in every direction
    const double m2 = xx * yy - xy * xy;
    const double m3 = xx * (yy * zz - yz * yz) - xy * (xy * zz - yz * xz) + xz * (xy * yz - yy * xz);
    if (!(xx > 0 && m2 > 0 && m3 > 0))
        return fail(s, PIC_EINVAL, "the binding tensor must be positive definite");
    // Eq. dtlimit with the largest eigenvalue bounded by Gershgorin's discs
    const double lam = std::max({xx + std::fabs(xy) + std::fabs(xz),
                                 yy + std::fabs(xy) + std::fabs(yz),
                                 zz + std::fabs(xz) + std::fabs(yz)});
    if (!(dt_limit(s, std::max(s->omega_b2, lam), s->omega_p2) > s->gd.dt))
        return fail(s, PIC_EDTLIMIT, "dt exceeds the stability limit of Eq. dtlimit with this tensor");
    for (int a = 0; a < 3; ++a) s->sp[k].w2off[a] = w2off[a];
    s->sp[k].has_off = true;
    // later species are checked against the tensor's bound too
    s->omega_b2 = std::max(s->omega_b2, lam);
    return PIC_OK;
}

pic_status pic_set_shape_order(pic_sim *s, int order) {
    if (!s) return fail(s, PIC_EINVAL, "null handle");
    if (s->group) return fail(s, PIC_ESTATE, "the simulation belongs to a group");
    if (order != 1 && order != 2) return fail(s, PIC_EINVAL, "order must be 1 (CIC) or 2 (TSC)");
    if (s->nsp > 0) return fail(s, PIC_ESTATE, "set the shape order before loading species");
    s->shape_order = order;
    return setup_tiles(s);  // the staged box grows by a cell on each side for TSC
}

pic_status pic_set_particle_bc(pic_sim *s, int edges, double p_diffuse, uint64_t seed) {
    if (!s) return fail(s, PIC_EINVAL, "null handle");
    if (s->group) return fail(s, PIC_ESTATE, "the simulation belongs to a group");
    if (edges != PIC_EDGE_REFLECT && edges != PIC_EDGE_OPEN)
        return fail(s, PIC_EINVAL, "edges must be PIC_EDGE_REFLECT or PIC_EDGE_OPEN");
    if (!(p_diffuse >= 0.0 && p_diffuse <= 1.0))
        return fail(s, PIC_EINVAL, "p_diffuse must lie in [0, 1]");
    if (edges == PIC_EDGE_OPEN && p_diffuse != 0.0)
        return fail(s, PIC_EINVAL, "open edges take no diffuse share");
    s->open_edges = edges == PIC_EDGE_OPEN;
    s->p_diffuse = p_diffuse;
    s->diff_seed = seed;
    return PIC_OK;
}

}  // extern "C"

namespace pic {

// Kernels the split passes launch for one step: one per non-empty block
// list (launch_field_b_tma, launch_field_b, launch_field_e skip empty ones).
int split_field_launches(const FieldP &f) {
    if (!f.blk[0]) {
        const bool pml = f.pml[0] || f.pml[1] || f.pml[2];
        return (pml ? 4 : 2) + (f.tma_b ? 1 : 0);
    }
    return (f.tma_b && f.nblk[0] > 0) + (f.nblk[f.tma_b ? 1 : 3] > 0) + 2 * (f.nblk[2] > 0) +
           (f.nblk[3] > 0);
}

// The field blocks of each launch of the split passes (FieldP.blk): [0] the
// TMA-fed B pass's, [1] the other blocks without a CPML slab, [2] those with
// one, [3] all without one.  They follow the block grid, the CPML slabs and
// whether the TMA-fed B pass is on, so they are rebuilt with the tuning.
pic_status build_block_lists(pic_sim *s) {
    dfree(s, s->blk_lists);
    s->blk_lists = nullptr;
    const FieldP f = field_params(s);
    std::vector<int> lists[4];
    for (int bz = 0; bz < s->nbz; ++bz)
        for (int by = 0; by < s->nby; ++by)
            for (int bx = 0; bx < s->nbx; ++bx) {
                const int q = (bz * s->nby + by) * s->nbx + bx;
                if (field_block_pml(s->g, f, bx, by, bz)) {
                    lists[2].push_back(q);
                    continue;
                }
                lists[3].push_back(q);
                lists[field_b_tma_block(s->g, f, bx, by, bz) ? 0 : 1].push_back(q);
            }
    std::vector<int> all;
    for (int k = 0; k < 4; ++k) {
        s->blk_off[k] = (int)all.size();
        s->blk_n[k] = (int)lists[k].size();
        all.insert(all.end(), lists[k].begin(), lists[k].end());
    }
    if (!(s->blk_lists = (int *)dalloc(s, std::max<size_t>(all.size(), 1) * sizeof(int))))
        return fail(s, PIC_ENOMEM, "field block lists");
    CK(s, cudaMemcpyAsync(s->blk_lists, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice,
                          s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    return PIC_OK;
}

pic_status apply_tuning(pic_sim *s, const pic_tuning *t) {
    pic_tuning nt = s->tun;
    for (int a = 0; a < 3; ++a)
        if (t->tile[a] > 0) nt.tile[a] = t->tile[a];
    if (t->sort_interval > 0) nt.sort_interval = t->sort_interval;
    if (t->particle_ctas > 0) nt.particle_ctas = t->particle_ctas;
    nt.keep_J = t->keep_J;
    nt.timing = t->timing;
    nt.field_plain = t->field_plain;
    nt.tile_order = t->tile_order;
    nt.no_overlap = t->no_overlap;
    if (t->field_mode >= 1 && t->field_mode <= 3) nt.field_mode = t->field_mode;
    if (t->wait_polls < 0) return fail(s, PIC_EINVAL, "wait_polls must be >= 0");
    nt.wait_polls = t->wait_polls;
    if (t->field_overlap < 0 || t->field_overlap > 2)
        return fail(s, PIC_EINVAL, "field_overlap must be 0, 1 or 2");
    if (t->field_overlap > 0) nt.field_overlap = t->field_overlap;
    if (t->field_zchunk > 0 && t->field_zchunk != s->tun.field_zchunk) {
        nt.field_zchunk = t->field_zchunk;
        s->nbz = s->g.dims == 3 ? (s->g.n[2] + nt.field_zchunk - 1) / nt.field_zchunk : 1;
        dfree(s, s->jdirty);
        if (!alloc_zero(s, &s->jdirty, (size_t)s->nbx * s->nby * s->nbz))
            return fail(s, PIC_ENOMEM, "jdirty");
    }
    s->tun = nt;
    pic_status st = setup_tiles(s);
    if (st != PIC_OK) return st;
    if ((st = build_block_lists(s)) != PIC_OK) return st;
    if (s->nsp > 0) {
        st = sort_all(s, true);
        if (st != PIC_OK) return st;
        st = rebuild_active(s);
        if (st != PIC_OK) return st;
    }
    CK(s, cudaStreamSynchronize(s->stream));
    return PIC_OK;
}

}  // namespace pic

extern "C" {

pic_status pic_load_species(pic_sim *s, const pic_species_desc *d, const pic_particles *pp,
                            int *species_id) {
    if (!s || !d || !pp) return fail(s, PIC_EINVAL, "null argument");
    if (s->group) return fail(s, PIC_ESTATE, "the simulation belongs to a group");
    if (s->nsp >= kMaxSpecies) return fail(s, PIC_EINVAL, "too many species");
    if (d->kind != PIC_FREE && d->kind != PIC_BOUND && d->kind != PIC_DIRAC)
        return fail(s, PIC_EINVAL, "unknown species kind");
    if (!(d->m > 0) || d->q == 0) return fail(s, PIC_EINVAL, "mass must be > 0 and charge != 0");
    for (int a = 0; a < 3; ++a)
        if (!(d->gamma[a] >= 0.0 && d->gamma[a] < 1e300))  // also rejects NaN
            return fail(s, PIC_EINVAL, "gamma must be finite and >= 0");
    if (d->kind == PIC_DIRAC && !(d->v_F > 0)) return fail(s, PIC_EINVAL, "Dirac species need v_F > 0");
    if (d->background < PIC_BG_NONE || d->background > PIC_BG_UNIFORM)
        return fail(s, PIC_EINVAL, "unknown background mode");
    const bool loader = pp->cell == nullptr;
    const GridP &g = s->g;
    const double V = s->gd.dx * s->gd.dy * s->gd.dz;
    long long n = 0;
    double weight = d->weight;
    long long nmat = 0;
    if (loader) {
        if (pp->ppc < 1) return fail(s, PIC_EINVAL, "ppc must be >= 1");
        if (!(pp->density > 0)) return fail(s, PIC_EINVAL, "loader needs density > 0");
        if (pp->T < 0) return fail(s, PIC_EINVAL, "temperature must be >= 0");
        if (d->kind != PIC_BOUND && !(pp->E_F > 0)) return fail(s, PIC_EINVAL, "loader needs E_F > 0");
        if (pp->quiet) {
            int lat = (int)llround(pow((double)pp->ppc, 1.0 / g.dims));
            long long t = 1;
            for (int a = 0; a < g.dims; ++a) t *= lat;
            if (t != pp->ppc) return fail(s, PIC_EINVAL, "quiet loading needs ppc = m^dims");
        }
        if (s->mask_h.empty()) nmat = g.ncell;
        else
            for (uint8_t m : s->mask_h) nmat += m != 0;
        n = nmat * pp->ppc;
        if (n > 0x7fffffffLL) return fail(s, PIC_EINVAL, "too many particles for one species");
        weight = pp->density * V / pp->ppc;
    } else {
        n = pp->n;
        if (n < 0 || n > 0x7fffffffLL) return fail(s, PIC_EINVAL, "particle count out of range");
        if (n > 0 && !pp->v) return fail(s, PIC_EINVAL, "v array missing");
        if (n > 0 && d->kind == PIC_BOUND && !pp->anchor_off)
            return fail(s, PIC_EINVAL, "bound species need anchor_off");
        if (n > 0 && d->kind != PIC_BOUND && !pp->off) return fail(s, PIC_EINVAL, "off array missing");
        for (long long p = 0; p < n; ++p) {
            if (pp->cell[p] < 0 || pp->cell[p] >= g.ncell)
                return fail(s, PIC_EINVAL, "cell index out of range");
            for (int a = 0; a < 3; ++a) {
                double f = d->kind == PIC_BOUND ? pp->anchor_off[3 * p + a] : pp->off[3 * p + a];
                if (!(f >= 0.0 && f < 1.0)) return fail(s, PIC_EINVAL, "offsets must lie in [0,1)");
            }
        }
    }
    // stability limit with this species added (Eq. dtlimit)
    double wp2 = s->omega_p2, wb2 = s->omega_b2;
    double dens = pp->density;
    if (!(dens > 0) && n > 0) dens = n * weight / (V * (double)g.ncell);
    wp2 += d->q * d->q * dens / (d->m * kEps0);
    if (d->kind == PIC_BOUND)
        for (int a = 0; a < 3; ++a) wb2 = std::max(wb2, d->omega0[a] * d->omega0[a]);
    if (dt_limit(s, wb2, wp2) <= s->gd.dt)
        return fail(s, PIC_EDTLIMIT, "dt exceeds the stability limit of Eq. dtlimit with this species");

    const int id = s->nsp;
    Species &sp = s->sp[id];
    sp = Species();
    sp.desc = *d;
    sp.n = n;
    sp.weight = weight;
    const long long na = std::max<long long>(n, 1);
    bool ok = alloc_zero(s, &sp.nrefl, 1) && alloc_zero(s, &sp.tile_start, s->tp.ntiles + 1);
    for (int b = 0; b < 2 && ok; ++b) {
        ok = ok && alloc_zero(s, &sp.cell[b], na) && alloc_zero(s, &sp.pid[b], na);
        for (int a = 0; a < 3 && ok; ++a) {
            ok = ok && alloc_zero(s, &sp.v[b][a], na);
            if (d->kind == PIC_BOUND)
                ok = ok && alloc_zero(s, &sp.anchor[b][a], na) && alloc_zero(s, &sp.disp[b][a], na) &&
                     alloc_zero(s, &sp.anchor32[b][a], na);
            else ok = ok && alloc_zero(s, &sp.o[b][a], na);
        }
    }
    if (!ok) return fail(s, PIC_ENOMEM, "species allocation failed");
    // the lean kernel's deferred list holds each particle at most once a step
    long long total = 0;
    for (int i = 0; i <= id; ++i) total += s->sp[i].n;
    if (total > s->defer_cap) {
        dfree(s, s->defer);
        if (!alloc_zero(s, &s->defer, std::max<long long>(total, 1))) {
            s->defer = nullptr;
            s->defer_cap = 0;
            return fail(s, PIC_ENOMEM, "deferred-particle list");
        }
        s->defer_cap = total;
    }
    SpeciesP dst = species_params(s, sp, 0);
    if (loader) {
        FDRequest r{};
        r.kind = d->kind;
        r.dims = g.dims;
        r.ppc = pp->ppc;
        r.quiet = pp->quiet;
        r.m = d->m;
        r.mu = pp->E_F;
        r.kT = kKB * pp->T;
        r.vF = d->v_F;
        r.seed = pp->seed;
        r.stream = pp->stream;
        double *table = nullptr;
        int *mat = nullptr, *flags = nullptr, *rank = nullptr;
        double pmax = 0.0;
        if (d->kind == PIC_FREE && pp->T > 0) {
            pmax = fd_pmax(r);
            if (!alloc_zero(s, &table, kFDPanels + 1)) return fail(s, PIC_ENOMEM, "fd table");
            CK(s, launch_fd_table(r, table, pmax, s->stream));
        }
        if (s->mask_d) {
            if (!alloc_zero(s, &flags, g.ncell) || !alloc_zero(s, &rank, g.ncell + 1) ||
                !alloc_zero(s, &mat, std::max<long long>(nmat, 1)))
                return fail(s, PIC_ENOMEM, "loader buffers");
            int *tmp = nullptr;
            if (!alloc_zero(s, &tmp, scan_tmp_len(g.ncell))) return fail(s, PIC_ENOMEM, "scan tmp");
            CK(s, launch_mask_to_int(s->mask_d, g.ncell, flags, s->stream));
            CK(s, launch_scan_int(flags, rank, g.ncell, tmp, 0, s->stream));
            CK(s, launch_material_cells(g, s->mask_d, rank, mat, s->stream));
            CK(s, launch_fd_particles(g, r, mat, n, table, pmax, dst, sp.pid[0], s->stream));
            CK(s, cudaStreamSynchronize(s->stream));
            dfree(s, tmp);
        } else {
            CK(s, launch_fd_particles(g, r, nullptr, n, table, pmax, dst, sp.pid[0], s->stream));
        }
        CK(s, cudaStreamSynchronize(s->stream));
        dfree(s, table);
        dfree(s, flags);
        dfree(s, rank);
        dfree(s, mat);
    } else if (n > 0) {
        int32_t *lin = nullptr;
        if (!alloc_zero(s, &lin, n)) return fail(s, PIC_ENOMEM, "staging");
        CK(s, cudaMemcpy(lin, pp->cell, n * sizeof(int32_t), cudaMemcpyHostToDevice));
        CK(s, launch_pack_explicit(g, n, lin, sp.cell[0], sp.pid[0], s->stream));
        std::vector<float> hv(n);
        std::vector<double> hd(n);
        for (int a = 0; a < 3; ++a) {
            for (long long p = 0; p < n; ++p) hv[p] = pp->v[3 * p + a];
            CK(s, cudaMemcpy(sp.v[0][a], hv.data(), n * 4, cudaMemcpyHostToDevice));
            if (d->kind == PIC_BOUND) {
                for (long long p = 0; p < n; ++p) hd[p] = pp->anchor_off[3 * p + a];
                CK(s, cudaMemcpy(sp.anchor[0][a], hd.data(), n * 8, cudaMemcpyHostToDevice));
                for (long long p = 0; p < n; ++p) {
                    float f = (float)hd[p];
                    hv[p] = f < 1.0f ? f : 0x1.fffffep-1f;
                }
                CK(s, cudaMemcpy(sp.anchor32[0][a], hv.data(), n * 4, cudaMemcpyHostToDevice));
                for (long long p = 0; p < n; ++p) hv[p] = pp->disp ? pp->disp[3 * p + a] : 0.f;
                CK(s, cudaMemcpy(sp.disp[0][a], hv.data(), n * 4, cudaMemcpyHostToDevice));
            } else {
                for (long long p = 0; p < n; ++p) hv[p] = pp->off[3 * p + a];
                CK(s, cudaMemcpy(sp.o[0][a], hv.data(), n * 4, cudaMemcpyHostToDevice));
            }
        }
        CK(s, cudaStreamSynchronize(s->stream));
        dfree(s, lin);
    }
    sp.cur = 0;
    s->omega_p2 = wp2;
    s->omega_b2 = wb2;
    // neutralising background for the Gauss diagnostic
    if (d->background != PIC_BG_NONE && n > 0) {
        if (!s->rho_bg && !alloc_zero(s, &s->rho_bg, g.ncell)) return fail(s, PIC_ENOMEM, "rho_bg");
        if (d->background == PIC_BG_AT_PARTICLES) {
            SpeciesP at = species_params(s, sp, 0);
            if (d->kind == PIC_BOUND) {
                // ions sit at the anchors: deposit with zero displacement
                float *zero[3];
                for (int a = 0; a < 3; ++a) {
                    if (!alloc_zero(s, &zero[a], n)) return fail(s, PIC_ENOMEM, "bg");
                    at.disp[a] = zero[a];
                }
                CK(s, launch_rho_deposit(g, at, -d->q * weight / V, 1, s->rho_bg, s->stream));
                CK(s, cudaStreamSynchronize(s->stream));
                for (int a = 0; a < 3; ++a) dfree(s, zero[a]);
            } else {
                CK(s, launch_rho_deposit(g, at, -d->q * weight / V, s->shape_order, s->rho_bg,
                                         s->stream));
            }
        } else {
            CK(s, launch_add_uniform(s->rho_bg, g.ncell, -d->q * weight * n / (V * g.ncell),
                                     s->stream));
        }
    }
    s->nsp++;
    pic_status st = PIC_OK;
    if (n > 0) st = sort_species(s, id);
    if (st == PIC_OK) st = rebuild_active(s);
    if (st != PIC_OK) return st;
    CK(s, cudaStreamSynchronize(s->stream));
    if (species_id) *species_id = id;
    return PIC_OK;
}

pic_status pic_step(pic_sim *s, int nsteps) {
    if (!s) return fail(s, PIC_EINVAL, "null handle");
    if (s->group) return fail(s, PIC_ESTATE, "the simulation steps through its group");
    if (nsteps < 0) return fail(s, PIC_EINVAL, "nsteps must be >= 0");
    const long long nc = s->g.ncell;
    for (int it = 0; it < nsteps; ++it) {
        if (s->since_sort >= s->tun.sort_interval) {
            record(s, 2, true);
            pic_status st = sort_all(s, false);
            if (st != PIC_OK) return st;
            // tile_start pointers do not move between sorts: starts_dev stays valid
            CK(s, launch_active_tiles_work(s->tp, s->starts_dev, s->nsp, s->active, s->nactive,
                                           s->tile_work, s->stream));
            s->launches += active_tiles_kernel_count(s->tp.ntiles);
            record(s, 2, false);
        }
        if (s->tun.keep_J)
            for (int c = 0; c < 3; ++c) CK(s, cudaMemsetAsync(s->J[c], 0, nc * 4, s->stream));
        ParticleLaunch P = particle_params(s);
        FieldP f = field_params(s);
        const bool tma = s->use_tma && !s->tun.field_plain;
        if (!s->tun.no_overlap && !s->aux) {
            CK(s, cudaStreamCreateWithFlags(&s->aux, cudaStreamNonBlocking));
            CK(s, cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming));
            CK(s, cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming));
        }
        const bool stream = s->tun.field_mode == 3;
        const int fl = (f.pml[0] || f.pml[1] || f.pml[2]) ? 2 : 1;  // launches of a pass
        if (s->tun.field_mode != 1 && s->gd.src_on) {
            // this step's source current, formed on the host
            const double t = ((double)s->steps + 0.5) * s->gd.dt - f.src_t0;
            f.src_val = (float)(f.src_amp * exp(-2.0 * 0.6931471805599453 * t * t /
                                                (f.src_tau * f.src_tau)) *
                                sin(f.src_omega * t));
            f.src_host = 1;
        }
        if (s->tun.field_mode == 2 && !s->tun.no_overlap && s->tun.field_overlap == 2) {
            // both passes beside the particle phase: the E pass takes
            // B^{n+1/2} from the B pass before it and leaves the current (and
            // the block flags) to the current pass after the join, which also
            // advances the step counter
            P.step_counter = nullptr;
            f.splitJ = 1;
            CK(s, cudaEventRecord(s->ev_fork, s->stream));
            record(s, 0, true);
            CK(s, launch_particles(P, particle_ctas_for(s, P), s->psmem, s->stream));
            record(s, 0, false);
            CK(s, cudaStreamWaitEvent(s->aux, s->ev_fork, 0));
            record(s, 3, true, s->aux);
            CK(s, launch_field_b_tma(s->g, f, s->maps, s->fcur, s->status, s->aux));
            CK(s, launch_field_b(s->g, f, s->aux));
            record(s, 3, false, s->aux);
            record(s, 1, true, s->aux);
            CK(s, launch_field_e(s->g, f, s->inv_eps, s->aux));
            record(s, 1, false, s->aux);
            CK(s, cudaEventRecord(s->ev_join, s->aux));
            CK(s, cudaStreamWaitEvent(s->stream, s->ev_join, 0));
            CK(s, launch_japply(s->g, f, s->inv_eps, s->step_counter, s->stream));
            s->launches += 1 + particle_launches(P) + split_field_launches(f);
        } else if (s->tun.field_mode == 2) {
            // two streaming passes; the B pass reads only E^n, B^{n-1/2} and
            // writes the other ping-pong half, so with overlap it runs beside
            // the particle phase
            if (!s->tun.no_overlap) {
                CK(s, cudaEventRecord(s->ev_fork, s->stream));
                record(s, 0, true);
                CK(s, launch_particles(P, particle_ctas_for(s, P), s->psmem, s->stream));
                record(s, 0, false);
                CK(s, cudaStreamWaitEvent(s->aux, s->ev_fork, 0));
                record(s, 3, true, s->aux);
                CK(s, launch_field_b_tma(s->g, f, s->maps, s->fcur, s->status, s->aux));
                CK(s, launch_field_b(s->g, f, s->aux));
                record(s, 3, false, s->aux);
                CK(s, cudaEventRecord(s->ev_join, s->aux));
                CK(s, cudaStreamWaitEvent(s->stream, s->ev_join, 0));
            } else {
                record(s, 0, true);
                CK(s, launch_particles(P, particle_ctas_for(s, P), s->psmem, s->stream));
                record(s, 0, false);
                record(s, 3, true);
                CK(s, launch_field_b_tma(s->g, f, s->maps, s->fcur, s->status, s->stream));
                CK(s, launch_field_b(s->g, f, s->stream));
                record(s, 3, false);
            }
            record(s, 1, true);
            CK(s, launch_field_e(s->g, f, s->inv_eps, s->stream));
            record(s, 1, false);
            s->launches += particle_launches(P) + split_field_launches(f);
        } else if (!s->tun.no_overlap) {
            // E^n, B^{n-1/2} are only read by both launches and the update
            // writes the other ping-pong half, so the two can run together;
            // the current pass after the join adds J and advances the counter
            P.step_counter = nullptr;
            f.splitJ = 1;
            CK(s, cudaEventRecord(s->ev_fork, s->stream));
            record(s, 0, true);
            CK(s, launch_particles(P, particle_ctas_for(s, P), s->psmem, s->stream));
            record(s, 0, false);
            CK(s, cudaStreamWaitEvent(s->aux, s->ev_fork, 0));
            record(s, 1, true, s->aux);
            if (stream) CK(s, launch_field_stream(s->g, f, s->aux));
            else if (tma) CK(s, launch_field_tma(s->g, f, s->maps, s->fcur, s->status, s->aux));
            else CK(s, launch_field(s->g, f, s->aux));
            record(s, 1, false, s->aux);
            CK(s, cudaEventRecord(s->ev_join, s->aux));
            CK(s, cudaStreamWaitEvent(s->stream, s->ev_join, 0));
            CK(s, launch_japply(s->g, f, s->inv_eps, s->step_counter, s->stream));
            s->launches += 1 + particle_launches(P) + (stream ? fl : 1);
        } else {
            record(s, 0, true);
            CK(s, launch_particles(P, particle_ctas_for(s, P), s->psmem, s->stream));
            record(s, 0, false);
            record(s, 1, true);
            if (stream) CK(s, launch_field_stream(s->g, f, s->stream));
            else if (tma) CK(s, launch_field_tma(s->g, f, s->maps, s->fcur, s->status, s->stream));
            else CK(s, launch_field(s->g, f, s->stream));
            record(s, 1, false);
            s->launches += particle_launches(P) + (stream ? fl : 1);
        }
        s->fcur ^= 1;
        s->steps++;
        s->since_sort++;
    }
    return PIC_OK;
}

pic_status pic_sync(pic_sim *s) {
    if (!s) return fail(s, PIC_EINVAL, "null handle");
    CK(s, cudaStreamSynchronize(s->stream));
    return check_device_status(s);
}

pic_status pic_read_fields(pic_sim *s, int which, double *out, size_t n) {
    if (s && s->group_stream) CK(s, cudaStreamSynchronize(s->group_stream));
    if (!s || !out) return fail(s, PIC_EINVAL, "null argument");
    const long long nc = s->g.ncell;
    int cnt = 0;
    for (int b = 0; b < 12; ++b) cnt += (which >> b) & 1;
    if (which <= 0 || which >= (1 << 12) || (long long)n != cnt * nc)
        return fail(s, PIC_EINVAL, "which/n mismatch");
    if ((which & (PIC_JX | PIC_JY | PIC_JZ)) && !s->tun.keep_J)
        return fail(s, PIC_ESTATE, "J is readable only with keep_J");
    if ((which & (PIC_EXTX | PIC_EXTY | PIC_EXTZ)) && !s->Eext[0])
        return fail(s, PIC_ESTATE, "no external field is set");
    CK(s, cudaStreamSynchronize(s->stream));
    std::vector<float> tmp(nc);
    size_t off = 0;
    for (int b = 0; b < 12; ++b) {
        if (!((which >> b) & 1)) continue;
        const float *src = b < 3   ? s->E[s->fcur][b]
                           : b < 6 ? s->B[s->fcur][b - 3]
                           : b < 9 ? s->J[b - 6]
                                   : s->Eext[b - 9];
        CK(s, cudaMemcpy(tmp.data(), src, nc * 4, cudaMemcpyDeviceToHost));
        for (long long i = 0; i < nc; ++i) out[off + i] = tmp[i];
        off += nc;
    }
    return check_device_status(s);
}

pic_status pic_write_fields(pic_sim *s, int which, const double *in, size_t n) {
    if (s && s->group_stream) CK(s, cudaStreamSynchronize(s->group_stream));
    if (!s || !in) return fail(s, PIC_EINVAL, "null argument");
    const long long nc = s->g.ncell;
    int cnt = 0;
    for (int b = 0; b < 6; ++b) cnt += (which >> b) & 1;
    if (which <= 0 || which >= (1 << 6) || (long long)n != cnt * nc)
        return fail(s, PIC_EINVAL, "which/n mismatch (E and B only)");
    CK(s, cudaStreamSynchronize(s->stream));
    std::vector<float> tmp(nc);
    size_t off = 0;
    for (int b = 0; b < 6; ++b) {
        if (!((which >> b) & 1)) continue;
        for (long long i = 0; i < nc; ++i) tmp[i] = (float)in[off + i];
        float *dst = b < 3 ? s->E[s->fcur][b] : s->B[s->fcur][b - 3];
        CK(s, cudaMemcpy(dst, tmp.data(), nc * 4, cudaMemcpyHostToDevice));
        off += nc;
    }
    return PIC_OK;
}

pic_status pic_read_species(pic_sim *s, int k, int32_t *cell, float *off, float *v,
                            double *anchor_off, float *disp, size_t n) {
    if (s && s->group_stream) CK(s, cudaStreamSynchronize(s->group_stream));
    if (!s) return fail(s, PIC_EINVAL, "null handle");
    if (k < 0 || k >= s->nsp) return fail(s, PIC_EINVAL, "no such species");
    Species &sp = s->sp[k];
    if ((long long)n != sp.n) return fail(s, PIC_EINVAL, "n must equal the species count");
    if (n == 0) return PIC_OK;
    const bool bound = sp.desc.kind == PIC_BOUND;
    int32_t *dc = nullptr;
    float *doff = nullptr, *dv = nullptr, *ddisp = nullptr;
    double *danc = nullptr;
    bool ok = alloc_zero(s, &dc, n) && alloc_zero(s, &dv, 3 * n);
    if (bound) ok = ok && alloc_zero(s, &danc, 3 * n) && alloc_zero(s, &ddisp, 3 * n);
    else ok = ok && alloc_zero(s, &doff, 3 * n);
    if (!ok) return fail(s, PIC_ENOMEM, "readback buffers");
    CK(s, launch_unsort(s->g, species_params(s, sp, sp.cur), sp.pid[sp.cur], dc, doff, dv, danc,
                        ddisp, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    if (cell) CK(s, cudaMemcpy(cell, dc, n * 4, cudaMemcpyDeviceToHost));
    if (v) CK(s, cudaMemcpy(v, dv, 3 * n * 4, cudaMemcpyDeviceToHost));
    if (off && !bound) CK(s, cudaMemcpy(off, doff, 3 * n * 4, cudaMemcpyDeviceToHost));
    if (anchor_off && bound) CK(s, cudaMemcpy(anchor_off, danc, 3 * n * 8, cudaMemcpyDeviceToHost));
    if (disp && bound) CK(s, cudaMemcpy(disp, ddisp, 3 * n * 4, cudaMemcpyDeviceToHost));
    dfree(s, dc);
    dfree(s, dv);
    dfree(s, doff);
    dfree(s, danc);
    dfree(s, ddisp);
    return check_device_status(s);
}

pic_status pic_cell_counts(pic_sim *s, int k, int32_t *out, size_t n) {
    if (s && s->group_stream) CK(s, cudaStreamSynchronize(s->group_stream));
    if (!s || !out) return fail(s, PIC_EINVAL, "null argument");
    if (k < 0 || k >= s->nsp) return fail(s, PIC_EINVAL, "no such species");
    if ((long long)n != s->g.ncell) return fail(s, PIC_EINVAL, "n must equal the cell count");
    int *d = nullptr;
    if (!alloc_zero(s, &d, n)) return fail(s, PIC_ENOMEM, "counts");
    Species &sp = s->sp[k];
    CK(s, launch_cell_histogram(s->g, species_params(s, sp, sp.cur), d, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    CK(s, cudaMemcpy(out, d, n * 4, cudaMemcpyDeviceToHost));
    dfree(s, d);
    return check_device_status(s);
}

pic_status pic_energy_histogram(pic_sim *s, int k, double e_max, int nbins, uint64_t *out,
                                size_t n) {
    if (s && s->group_stream) CK(s, cudaStreamSynchronize(s->group_stream));
    if (!s || !out) return fail(s, PIC_EINVAL, "null argument");
    if (k < 0 || k >= s->nsp) return fail(s, PIC_EINVAL, "no such species");
    if (nbins < 1 || nbins > (1 << 20)) return fail(s, PIC_EINVAL, "nbins must be 1 .. 2^20");
    if (!(e_max > 0.0 && e_max < 1e300)) return fail(s, PIC_EINVAL, "e_max must be finite and > 0");
    if (n != (size_t)nbins + 1) return fail(s, PIC_EINVAL, "n must equal nbins + 1");
    unsigned long long *d = nullptr;
    if (!alloc_zero(s, &d, n)) return fail(s, PIC_ENOMEM, "histogram");
    Species &sp = s->sp[k];
    CK(s, launch_energy_histogram(species_params(s, sp, sp.cur), 0.5 * sp.desc.m, e_max, nbins, d,
                                  s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    CK(s, cudaMemcpy(out, d, n * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    dfree(s, d);
    return check_device_status(s);
}

pic_status pic_diagnostics(pic_sim *s, pic_diag *out) {
    if (s && s->group_stream) CK(s, cudaStreamSynchronize(s->group_stream));
    if (!s || !out) return fail(s, PIC_EINVAL, "null argument");
    const GridP &g = s->g;
    const double V = s->gd.dx * s->gd.dy * s->gd.dz;
    CK(s, cudaMemsetAsync(s->diag_acc, 0, sizeof(DiagAcc), s->stream));
    for (int i = 0; i < s->nsp; ++i) {
        Species &sp = s->sp[i];
        double mw = 0.5 * sp.desc.m * sp.weight;
        CK(s, launch_kinetic(species_params(s, sp, sp.cur), mw, &s->diag_acc->kinetic[i],
                             s->stream));
    }
    const float *E[3] = {s->E[s->fcur][0], s->E[s->fcur][1], s->E[s->fcur][2]};
    const float *B[3] = {s->B[s->fcur][0], s->B[s->fcur][1], s->B[s->fcur][2]};
    CK(s, launch_field_energy(g, E, B, s->diag_acc, s->stream));
    if (!s->rho && !alloc_zero(s, &s->rho, g.ncell)) return fail(s, PIC_ENOMEM, "rho");
    CK(s, cudaMemsetAsync(s->rho, 0, g.ncell * 8, s->stream));
    for (int i = 0; i < s->nsp; ++i) {
        Species &sp = s->sp[i];
        CK(s, launch_rho_deposit(g, species_params(s, sp, sp.cur), sp.desc.q * sp.weight / V,
                                 sp.desc.kind == PIC_BOUND ? 1 : s->shape_order, s->rho,
                                 s->stream));
    }
    CK(s, launch_gauss(g, E, s->inv_eps, s->rho, s->rho_bg, s->diag_acc, s->stream));
    DiagAcc acc;
    CK(s, cudaStreamSynchronize(s->stream));
    CK(s, cudaMemcpy(&acc, s->diag_acc, sizeof(acc), cudaMemcpyDeviceToHost));
    memset(out, 0, sizeof(*out));
    out->step = s->steps;
    out->time = s->steps * s->gd.dt;
    out->nspecies = s->nsp;
    for (int i = 0; i < s->nsp; ++i) {
        out->count[i] = s->sp[i].n;
        out->kinetic[i] = acc.kinetic[i];
        unsigned long long r = 0;
        CK(s, cudaMemcpy(&r, s->sp[i].nrefl, 8, cudaMemcpyDeviceToHost));
        out->reflections[i] = r;
    }
    const double mu0 = 1.0 / (kEps0 * kC * kC);
    out->field_E = 0.5 * kEps0 * acc.e2 * V;
    out->field_B = 0.5 / mu0 * acc.b2 * V;
    double gm, qm;
    memcpy(&gm, &acc.gauss_max_bits, 8);
    memcpy(&qm, &acc.rho_max_bits, 8);
    out->gauss_max = gm;
    out->gauss_rms = sqrt(acc.gauss_sum2 / (double)g.ncell);
    out->rho_max = qm;
    return check_device_status(s);
}

pic_status pic_get_timing(pic_sim *s, pic_timing *out) {
    if (!s || !out) return fail(s, PIC_EINVAL, "null argument");
    CK(s, cudaStreamSynchronize(s->stream));
    double ms[4] = {0, 0, 0, 0};
    int64_t cnt[4] = {0, 0, 0, 0};
    for (int w = 0; w < 4; ++w) {
        TimedEvents &te = s->ev[w];
        for (size_t i = 0; i < te.start.size() && i < te.stop.size(); ++i) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, te.start[i], te.stop[i]) == cudaSuccess) {
                ms[w] += t;
                cnt[w]++;
            }
        }
        for (auto e : te.start) cudaEventDestroy(e);
        for (auto e : te.stop) cudaEventDestroy(e);
        te.start.clear();
        te.stop.clear();
    }
    out->particle_ms = ms[0];
    out->field_ms = ms[1];
    out->sort_ms = ms[2];
    out->particle_launches = cnt[0];
    out->field_launches = cnt[1];
    out->sort_launches = cnt[2];
    out->kernel_launches = s->launches;
    out->fieldb_ms = ms[3];
    out->fieldb_launches = cnt[3];
    s->launches = 0;
    return PIC_OK;
}

pic_status pic_memory_bytes(const pic_sim *s, size_t *bytes) {
    if (!s || !bytes) return fail(nullptr, PIC_EINVAL, "null argument");
    *bytes = s->bytes;
    return PIC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Per-cell counts that allocate nothing (pic_cell_counts_noalloc)
// ---------------------------------------------------------------------------

// The counts live in this fixed array instead of a per-call buffer.  In host
// code the name only stands for the array; the kernel gets the device address
// obtained once per device with cudaGetSymbolAddress.
static __device__ __align__(256) int g_noalloc_counts[PIC_NOALLOC_MAX_CELLS];

namespace {
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
int *g_noalloc_ptr[kNoallocMaxDevices] = {};
}  // namespace

extern "C" pic_status pic_cell_counts_noalloc(pic_sim *s, int k, int32_t *out, size_t n) {
    // a group member's particles move on the group's stream: wait for it, as
    // every other reader does
    if (s && s->group_stream) CK(s, cudaStreamSynchronize(s->group_stream));
    if (!s || !out) return fail(s, PIC_EINVAL, "null argument");
    if (k < 0 || k >= s->nsp) return fail(s, PIC_EINVAL, "no such species");
    if ((long long)n != s->g.ncell) return fail(s, PIC_EINVAL, "n must equal the cell count");
    if (n > (size_t)PIC_NOALLOC_MAX_CELLS)
        return fail(s, PIC_EINVAL,
                    "grid has " + std::to_string(n) + " cells; pic_cell_counts_noalloc holds at most " +
                        std::to_string(PIC_NOALLOC_MAX_CELLS) + " (use pic_cell_counts)");
    // the array's address is looked up on the simulation's own device, which
    // must be the current one (the stream and the kernel run there)
    const int dev = s->device;
    int cur = -1;
    CK(s, cudaGetDevice(&cur));
    if (cur != dev)
        return fail(s, PIC_EINVAL, "current device " + std::to_string(cur) +
                                       " is not the simulation's device " + std::to_string(dev));
    if (dev < 0 || dev >= kNoallocMaxDevices) return fail(s, PIC_EINVAL, "device index too large");
    int *counts = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_counts);
            if (e != cudaSuccess || !p)
                return fail(s, PIC_ECUDA,
                            std::string("cudaGetSymbolAddress(counts): ") + cudaGetErrorString(e));
            g_noalloc_ptr[dev] = (int *)p;
        }
        counts = g_noalloc_ptr[dev];
    }
    Species &sp = s->sp[k];
    CK(s, cudaMemsetAsync(counts, 0, n * sizeof(int), s->stream));
    CK(s, launch_cell_histogram(s->g, species_params(s, sp, sp.cur), counts, s->stream));
    CK(s, cudaMemcpyAsync(out, counts, n * sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    return check_device_status(s);
}
