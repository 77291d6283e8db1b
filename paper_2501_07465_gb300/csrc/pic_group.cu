// pic_group.cu -- host side of the batch engine (pic_group_* of include/pic.h).
//
// The group keeps device tables for its member slots: each member's
// particle and field parameter blocks (two variants, one per field ping-pong
// parity), its grid, step counts and target, and the work-item lists of the
// batched particle and field launches.  Tables are rebuilt when membership
// changes; a step is then begin_step + batched particle launch + batched
// field launch, with the batched sort at the start of every epoch of
// sort_interval steps.  The host mirrors each member's step count and field
// parity exactly (a member steps while done < target), so the handles stay
// consistent for later single-simulation calls.
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "pic_sim.h"

struct pic_group {
    int capacity = 0;
    size_t budget = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;  // created here because the caller passed none
    int use_graph = 0;
    int dims = 0;
    int tile[3] = {0, 0, 0};
    int sort_interval = 32;
    size_t psmem = 0;
    int pctas = 1;
    bool ext = false;  // some member has a boundary variant or anisotropic gamma
    int shape = 0;     // the members' shape order (1 CIC, 2 TSC); 0 before the first
    std::vector<pic_sim *> slots;
    std::vector<long long> done, target;  // host mirrors
    bool dirty = true;
    int epoch_pos = 0;
    long long launches = 0;
    std::string err;
    // device tables
    struct Buf {
        void *p = nullptr;
        size_t bytes = 0;
    };
    std::vector<Buf> bufs;
    ParticleLaunch *pdesc = nullptr;
    GridP *grids = nullptr;
    FieldP *fdesc = nullptr;
    int *member = nullptr, *active = nullptr, *fpar = nullptr;
    long long *ddone = nullptr, *dtarget = nullptr;
    long long **counters = nullptr;
    int2 *pitems = nullptr;
    int npitems = 0;
    int *psched = nullptr;  // particle items: next to take, CTAs finished
    int4 *fitems = nullptr;
    int nfitems = 0;
    SortSeg *segs = nullptr;
    int nseg = 0;
    long long total = 0;
    SimTiles *simtiles = nullptr;
    int nsimtiles = 0;
    cudaGraphExec_t exec = nullptr;
    int graph_launches = 0;  // kernels in one captured epoch
};

namespace {

pic_status gfail(pic_group *g, pic_status st, const std::string &m) {
    if (g) g->err = m;
    pic::fail(nullptr, st, m);
    return st;
}

#define GCK(g, call)                                                                           \
    do {                                                                                       \
        cudaError_t _e = (call);                                                               \
        if (_e != cudaSuccess)                                                                 \
            return gfail(g, PIC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e));    \
    } while (0)

template <class T>
T *galloc(pic_group *g, size_t count) {
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    void *p = pic::raw_alloc(bytes, g->stream);
    if (p) g->bufs.push_back({p, bytes});
    return (T *)p;
}

void gfree_all(pic_group *g) {
    for (auto &b : g->bufs) pic::raw_free(b.p, b.bytes, g->stream);
    g->bufs.clear();
}

void drop_graph(pic_group *g) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
    g->graph_launches = 0;
}

size_t member_bytes(const pic_group *g) {
    size_t b = 0;
    for (auto *s : g->slots)
        if (s) b += s->bytes;
    return b;
}

// host mirror of one group step
void mirror_step(pic_group *g) {
    for (size_t k = 0; k < g->slots.size(); ++k) {
        pic_sim *s = g->slots[k];
        if (!s || g->done[k] >= g->target[k]) continue;
        g->done[k] += 1;
        s->steps += 1;
        s->fcur ^= 1;
    }
}

// (Re)build every device table from the current membership.
pic_status rebuild(pic_group *g) {
    drop_graph(g);
    GCK(g, cudaStreamSynchronize(g->stream));
    gfree_all(g);
    const int cap = g->capacity;
    std::vector<ParticleLaunch> hp(2 * cap);
    std::vector<GridP> hg(cap);
    std::vector<FieldP> hf(2 * cap);
    std::vector<int> hmember(cap, 0), hfpar(cap, 0), hzero(cap, 0);
    std::vector<long long> hdone(cap, 0), htarget(cap, 0);
    std::vector<long long *> hcnt(cap, nullptr);
    std::vector<int4> hfitems;
    std::vector<SortSeg> hsegs;
    std::vector<SimTiles> hsims;
    long long total = 0;
    int ioff = 0;
    bool ext = false;
    for (int k = 0; k < cap; ++k) {
        pic_sim *s = g->slots[k];
        if (!s) continue;
        const int keep = s->fcur;
        for (int par = 0; par < 2; ++par) {
            s->fcur = par;
            hp[2 * k + par] = pic::particle_params(s);
            hp[2 * k + par].step_counter = nullptr;  // begin_step sets the counter
            // the step index of the member's first group step: the kernel adds
            // the member's device step count (the diffuse draws' key)
            hp[2 * k + par].rng_step = (uint32_t)(s->steps - g->done[k]);
            ext = ext || pic::particle_launch_ext(hp[2 * k + par]);
            hf[2 * k + par] = pic::field_params(s);
        }
        s->fcur = keep;
        hg[k] = s->g;
        hmember[k] = 1;
        hfpar[k] = s->fcur;
        hdone[k] = g->done[k];
        htarget[k] = g->target[k];
        hcnt[k] = s->step_counter;
        const int nbz = s->g.dims == 3 ? s->nbz : 1;
        for (int bz = 0; bz < nbz; ++bz)
            for (int by = 0; by < s->nby; ++by)
                for (int bx = 0; bx < s->nbx; ++bx) hfitems.push_back(make_int4(k, bx, by, bz));
        SimTiles st{};
        st.sim = k;
        st.ntiles = s->tp.ntiles;
        st.nsp = s->nsp;
        st.ioff = ioff;
        for (int q = 0; q < s->nsp; ++q) st.starts[q] = s->sp[q].tile_start;
        hsims.push_back(st);
        ioff += s->tp.ntiles;
        for (int q = 0; q < s->nsp; ++q) {
            Species &sp = s->sp[q];
            if (sp.desc.kind == PIC_BOUND || sp.n == 0) continue;
            SortSeg sg{};
            sg.src = pic::species_params(s, sp, sp.cur);
            sg.tmp = pic::species_params(s, sp, 1 - sp.cur);
            sg.pid_src = sp.pid[sp.cur];
            sg.pid_tmp = sp.pid[1 - sp.cur];
            sg.tp = s->tp;
            sg.tile_start = sp.tile_start;
            sg.poff = total;
            total += sp.n;
            hsegs.push_back(sg);
        }
    }
    // the batched tile histogram keys a particle by (segment << 20) | tile
    for (auto &sg : hsegs)
        if (sg.tp.ntiles >= (1 << 20)) return gfail(g, PIC_EINVAL, "member has 2^20 tiles or more");
    if (hsegs.size() >= (1u << 12)) return gfail(g, PIC_EINVAL, "more than 4095 sorted species");
    // scratch for the batched sort: counts per segment, ranks per particle
    long long ncount = 0;
    for (auto &sg : hsegs) ncount += sg.tp.ntiles + 1;
    int *counts = galloc<int>(g, ncount);
    int *ranks = galloc<int>(g, total);
    if (!counts || !ranks) return gfail(g, PIC_ENOMEM, "batch sort scratch");
    long long co = 0;
    for (auto &sg : hsegs) {
        sg.count = counts + co;
        co += sg.tp.ntiles + 1;
        sg.rank = ranks + sg.poff;
    }
    g->pdesc = galloc<ParticleLaunch>(g, 2 * cap);
    g->grids = galloc<GridP>(g, cap);
    g->fdesc = galloc<FieldP>(g, 2 * cap);
    g->member = galloc<int>(g, cap);
    g->active = galloc<int>(g, cap);
    g->fpar = galloc<int>(g, cap);
    g->ddone = galloc<long long>(g, cap);
    g->dtarget = galloc<long long>(g, cap);
    g->counters = galloc<long long *>(g, cap);
    g->pitems = galloc<int2>(g, ioff);
    g->psched = galloc<int>(g, 2);
    g->fitems = galloc<int4>(g, hfitems.size());
    g->segs = galloc<SortSeg>(g, hsegs.size());
    g->simtiles = galloc<SimTiles>(g, hsims.size());
    if (!g->pdesc || !g->grids || !g->fdesc || !g->member || !g->active || !g->fpar || !g->ddone ||
        !g->dtarget || !g->counters || !g->pitems || !g->psched || !g->fitems || !g->segs ||
        !g->simtiles)
        return gfail(g, PIC_ENOMEM, "batch tables");
    auto up = [&](void *dst, const void *src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, g->stream)
                     : cudaSuccess;
    };
    g->ext = ext;
    GCK(g, up(g->pdesc, hp.data(), hp.size() * sizeof(ParticleLaunch)));
    GCK(g, up(g->grids, hg.data(), hg.size() * sizeof(GridP)));
    GCK(g, up(g->fdesc, hf.data(), hf.size() * sizeof(FieldP)));
    GCK(g, up(g->member, hmember.data(), cap * sizeof(int)));
    GCK(g, up(g->active, hzero.data(), cap * sizeof(int)));
    GCK(g, up(g->fpar, hfpar.data(), cap * sizeof(int)));
    GCK(g, up(g->ddone, hdone.data(), cap * sizeof(long long)));
    GCK(g, up(g->dtarget, htarget.data(), cap * sizeof(long long)));
    GCK(g, up(g->counters, hcnt.data(), cap * sizeof(long long *)));
    GCK(g, up(g->fitems, hfitems.data(), hfitems.size() * sizeof(int4)));
    GCK(g, up(g->segs, hsegs.data(), hsegs.size() * sizeof(SortSeg)));
    GCK(g, up(g->simtiles, hsims.data(), hsims.size() * sizeof(SimTiles)));
    GCK(g, cudaMemsetAsync(g->psched, 0, 2 * sizeof(int), g->stream));
    GCK(g, cudaStreamSynchronize(g->stream));  // host vectors go out of scope
    g->npitems = ioff;
    g->nfitems = (int)hfitems.size();
    g->nseg = (int)hsegs.size();
    g->total = total;
    g->nsimtiles = (int)hsims.size();
    g->dirty = false;
    g->epoch_pos = 0;  // a fresh table starts with a sort
    return PIC_OK;
}

pic_status enqueue_sort(pic_group *g) {
    int n = 0;
    GCK(g, pic::launch_batch_sort(g->segs, g->nseg, g->total, g->stream, &n));
    GCK(g, pic::launch_batch_items(g->simtiles, g->nsimtiles, g->pitems, g->stream));
    g->launches += n + (g->nsimtiles > 0 ? 1 : 0);
    return PIC_OK;
}

pic_status enqueue_step(pic_group *g) {
    if (g->epoch_pos == 0) {
        pic_status st = enqueue_sort(g);
        if (st != PIC_OK) return st;
    }
    GCK(g, pic::launch_begin_step(g->capacity, g->member, g->active, g->fpar, g->ddone, g->dtarget,
                                  g->counters, g->stream));
    GCK(g, pic::launch_batch_particles(g->dims, g->pdesc, g->fpar, g->active, g->pitems,
                                       g->npitems, g->psched, g->ddone, g->pctas, g->psmem,
                                       g->ext, g->shape, g->stream));
    GCK(g, pic::launch_batch_field(g->dims, g->grids, g->fdesc, g->fpar, g->active, g->fitems,
                                   g->nfitems, g->stream));
    g->launches += 3;
    g->epoch_pos = (g->epoch_pos + 1) % g->sort_interval;
    return PIC_OK;
}

int slot_of(const pic_group *g, const pic_sim *s) {
    for (size_t k = 0; k < g->slots.size(); ++k)
        if (g->slots[k] == s) return (int)k;
    return -1;
}

}  // namespace

extern "C" {

pic_status pic_group_create(int capacity, size_t hbm_budget, void *stream, int use_graph,
                            pic_group **out) {
    if (!out || capacity < 1) return gfail(nullptr, PIC_EINVAL, "capacity must be >= 1");
    pic_group *g = new pic_group();
    g->capacity = capacity;
    g->budget = hbm_budget;
    g->stream = (cudaStream_t)stream;
    if (!g->stream) {  // the legacy default stream cannot be captured into a graph
        cudaError_t e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete g;
            return gfail(nullptr, PIC_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
        }
        g->own_stream = true;
    }
    g->use_graph = use_graph;
    g->slots.assign(capacity, nullptr);
    g->done.assign(capacity, 0);
    g->target.assign(capacity, 0);
    *out = g;
    return PIC_OK;
}

pic_status pic_group_destroy(pic_group *g) {
    if (!g) return PIC_OK;
    cudaStreamSynchronize(g->stream);
    // release the members (their step counts and field parity are already exact)
    for (auto *s : g->slots) {
        if (!s) continue;
        s->group = nullptr;
        s->group_slot = -1;
        s->group_stream = nullptr;
        s->since_sort = s->tun.sort_interval;  // re-sort before its next own step
    }
    drop_graph(g);
    gfree_all(g);
    if (g->own_stream) cudaStreamDestroy(g->stream);
    delete g;
    return PIC_OK;
}

pic_status pic_group_add(pic_group *g, pic_sim *s, int64_t nsteps) {
    if (!g || !s) return gfail(g, PIC_EINVAL, "null argument");
    if (s->group) return gfail(g, PIC_ESTATE, "simulation already belongs to a group");
    if (nsteps < 0) return gfail(g, PIC_EINVAL, "nsteps must be >= 0");
    if (g->dims == 0) {
        g->dims = s->g.dims;
        for (int a = 0; a < 3; ++a) g->tile[a] = s->tp.T[a];
        g->sort_interval = std::max(1, s->tun.sort_interval);
        g->shape = s->shape_order;
        g->psmem = s->psmem;  // the staged box of the shape (TSC: one cell more a side)
        int per_sm = 0, per_sm_ext = 0, per_sm_tsc = 0;
        GCK(g, pic::particle_kernel_setup(g->dims, g->psmem, &per_sm, &per_sm_ext, &per_sm_tsc));
        g->pctas = std::max(1, g->shape == 2 ? per_sm_tsc : per_sm) * s->num_sms;
    }
    if (s->g.dims != g->dims) return gfail(g, PIC_EINVAL, "members must share dims");
    if (s->shape_order != g->shape)
        return gfail(g, PIC_EINVAL, "members must share the shape order (CIC or TSC)");
    for (int a = 0; a < 3; ++a)
        if (s->tp.T[a] != g->tile[a]) return gfail(g, PIC_EINVAL, "members must share the particle tile");
    if (g->budget && member_bytes(g) + s->bytes > g->budget)
        return gfail(g, PIC_EBUDGET, "HBM budget of the group exceeded");
    int k = -1;
    for (int q = 0; q < g->capacity; ++q)
        if (!g->slots[q]) {
            k = q;
            break;
        }
    if (k < 0) return gfail(g, PIC_EBUDGET, "group is full");
    GCK(g, cudaStreamSynchronize(s->stream));
    GCK(g, cudaStreamSynchronize(g->stream));
    g->slots[k] = s;
    g->done[k] = 0;
    g->target[k] = nsteps;
    s->group = g;
    s->group_slot = k;
    s->group_stream = g->stream;
    g->dirty = true;
    return PIC_OK;
}

pic_status pic_group_remove(pic_group *g, pic_sim *s) {
    if (!g || !s) return gfail(g, PIC_EINVAL, "null argument");
    const int k = slot_of(g, s);
    if (k < 0) return gfail(g, PIC_EINVAL, "not a member of this group");
    GCK(g, cudaStreamSynchronize(g->stream));
    g->slots[k] = nullptr;
    s->group = nullptr;
    s->group_slot = -1;
    s->group_stream = nullptr;
    s->since_sort = s->tun.sort_interval;  // re-sort before its next own step
    g->dirty = true;
    return PIC_OK;
}

pic_status pic_group_step(pic_group *g, int nsteps) {
    if (!g || nsteps < 0) return gfail(g, PIC_EINVAL, "bad argument");
    if (g->dims == 0 || nsteps == 0) return PIC_OK;
    if (g->dirty) {
        pic_status st = rebuild(g);
        if (st != PIC_OK) return st;
    }
    int left = nsteps;
    // direct launches up to the next epoch boundary
    while (left > 0 && (g->epoch_pos != 0 || !g->use_graph || left < g->sort_interval)) {
        pic_status st = enqueue_step(g);
        if (st != PIC_OK) return st;
        mirror_step(g);
        --left;
    }
    // whole epochs from a captured graph
    if (left >= g->sort_interval) {
        if (!g->exec) {
            cudaGraph_t graph = nullptr;
            GCK(g, cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
            const long long l0 = g->launches;
            for (int q = 0; q < g->sort_interval; ++q) {
                pic_status st = enqueue_step(g);
                if (st != PIC_OK) {
                    cudaStreamEndCapture(g->stream, &graph);
                    if (graph) cudaGraphDestroy(graph);
                    return st;
                }
            }
            GCK(g, cudaStreamEndCapture(g->stream, &graph));
            g->graph_launches = (int)(g->launches - l0);
            g->launches = l0;
            cudaError_t e = cudaGraphInstantiate(&g->exec, graph, 0);
            cudaGraphDestroy(graph);
            GCK(g, e);
        }
        while (left >= g->sort_interval) {
            GCK(g, cudaGraphLaunch(g->exec, g->stream));
            g->launches += g->graph_launches;
            for (int q = 0; q < g->sort_interval; ++q) mirror_step(g);
            left -= g->sort_interval;
        }
    }
    while (left > 0) {
        pic_status st = enqueue_step(g);
        if (st != PIC_OK) return st;
        mirror_step(g);
        --left;
    }
    GCK(g, pic::launch_finalize(g->capacity, g->active, g->fpar, g->ddone, g->stream));
    g->launches += 1;
    return PIC_OK;
}

pic_status pic_group_sync(pic_group *g) {
    if (!g) return gfail(g, PIC_EINVAL, "null argument");
    GCK(g, cudaStreamSynchronize(g->stream));
    for (auto *s : g->slots) {
        if (!s) continue;
        pic_status st = pic::check_device_status(s);
        if (st != PIC_OK) return gfail(g, st, s->err);
    }
    return PIC_OK;
}

pic_status pic_group_progress(pic_group *g, const pic_sim *s, int64_t *steps_done,
                              int64_t *steps_left) {
    if (!g || !s) return gfail(g, PIC_EINVAL, "null argument");
    const int k = slot_of(g, s);
    if (k < 0) return gfail(g, PIC_EINVAL, "not a member of this group");
    if (steps_done) *steps_done = g->done[k];
    if (steps_left) *steps_left = std::max<long long>(0, g->target[k] - g->done[k]);
    return PIC_OK;
}

pic_status pic_group_info(pic_group *g, int *members, size_t *bytes, int64_t *launches) {
    if (!g) return gfail(g, PIC_EINVAL, "null argument");
    int m = 0;
    for (auto *s : g->slots) m += s != nullptr;
    if (members) *members = m;
    if (bytes) *bytes = member_bytes(g);
    if (launches) *launches = g->launches;
    return PIC_OK;
}

}  // extern "C"
