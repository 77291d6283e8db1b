// pic_sim.h -- host-side state of one simulation handle and the helpers the
// C ABI (pic_api.cu) and the batch engine (pic_group.cu) share.
#pragma once

#include <string>
#include <vector>

#include "pic_internal.cuh"

namespace pic {

struct DevBuf {
    void *p;
    size_t bytes;
};

struct Species {
    pic_species_desc desc{};
    long long n = 0;
    double weight = 0;
    int cur = 0;
    uint32_t *cell[2] = {nullptr, nullptr};
    uint32_t *pid[2] = {nullptr, nullptr};
    float *o[2][3] = {};
    float *v[2][3] = {};
    double *anchor[2][3] = {};
    float *anchor32[2][3] = {};
    float *disp[2][3] = {};
    int *tile_start = nullptr;
    unsigned long long *nrefl = nullptr;
    double w2off[3] = {0, 0, 0};  // off-diagonal binding tensor entries (xy, xz, yz), s^-2
    bool has_off = false;
};

struct TimedEvents {
    std::vector<cudaEvent_t> start, stop;
};

}  // namespace pic

using namespace pic;

struct pic_sim {
    struct pic_group *group = nullptr;  // batch this simulation belongs to, if any
    int group_slot = -1;
    cudaStream_t group_stream = nullptr;
    int device = 0;
    int num_sms = 148;
    cudaStream_t stream = nullptr;
    pic_grid_desc gd{};
    GridP g{};
    TileP tp{};
    pic_tuning tun{};
    std::vector<pic::DevBuf> bufs;
    size_t bytes = 0;
    float *E[2][3] = {};
    float *B[2][3] = {};
    float *J[3] = {};
    int fcur = 0;
    float *psi[2][3][4] = {};
    float *cb_e[3] = {}, *ca_e[3] = {}, *cb_h[3] = {}, *ca_h[3] = {};
    uint8_t *mask_d = nullptr;
    float *inv_eps = nullptr;  // 1 / eps_r per cell, null: vacuum
    // particle boundary variants (Sec. 3)
    float *Eext[3] = {};       // external field seen by the particles only, null: none
    int open_edges = 0;        // 1: particles cross material edges
    double p_diffuse = 0.0;    // share of diffuse material-edge reflections
    uint64_t diff_seed = 0;    // Philox key of the diffuse draws
    int shape_order = 1;       // free and Dirac particles: 1 CIC, 2 TSC
    std::vector<uint8_t> mask_h;
    uint8_t *jdirty = nullptr;
    int nbx = 1, nby = 1, nbz = 1;
    int *blk_lists = nullptr;  // the split passes' compact block lists (FieldP.blk)
    int blk_off[4] = {0, 0, 0, 0}, blk_n[4] = {0, 0, 0, 0};
    double *rho_bg = nullptr, *rho = nullptr;
    long long *step_counter = nullptr;
    int *status = nullptr;
    DiagAcc *diag_acc = nullptr;
    // sort / tiles
    int *active = nullptr, *nactive = nullptr;
    int *tile_work = nullptr;
    int *sort_count = nullptr, *sort_rank = nullptr, *scan_tmp = nullptr;
    long long rank_cap = 0;
    int2 *defer = nullptr;    // the lean kernel's deferred-particle list
    long long defer_cap = 0;  // its capacity: the particles of all species
    int **starts_dev = nullptr;
    int particle_ctas = 1;
    int particle_ctas_ext = 1;  // the same for the kernel with the boundary variants
    int particle_ctas_tsc = 1;  // and for the TSC kernel
    size_t psmem = 0;
    int nsp = 0;
    pic::Species sp[kMaxSpecies];
    long long steps = 0;
    int since_sort = 0;
    double omega_p2 = 0.0, omega_b2 = 0.0;
    std::string err;
    pic::TimedEvents ev[4];  // particle, field (E pass), sort, B pass
    long long launches = 0;  // kernels launched by pic_step since the last timing query
    TmaMaps maps;            // TMA descriptors of the field arrays
    bool use_tma = false;    // TMA field kernel (needs nx % 4 == 0)
    // overlapped step: the field update runs on `aux` while the particle
    // phase runs on `stream`; fork / join events order them
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace pic {

pic_status fail(pic_sim *s, pic_status st, const std::string &msg);
void *dalloc(pic_sim *s, size_t bytes);
void dfree(pic_sim *s, void *p);
template <class T>
bool alloc_zero(pic_sim *s, T **out, size_t count) {
    *out = (T *)dalloc(s, count * sizeof(T));
    if (!*out) return false;
    return cudaMemsetAsync(*out, 0, count * sizeof(T), s->stream) == cudaSuccess;
}
SpeciesP species_params(const pic_sim *s, const Species &sp, int buf);
FieldP field_params(pic_sim *s);
ParticleLaunch particle_params(pic_sim *s);
pic_status check_device_status(pic_sim *s);
pic_status sort_all(pic_sim *s, bool include_bound);
pic_status apply_tuning(pic_sim *s, const pic_tuning *t);
void *raw_alloc(size_t bytes, cudaStream_t stream);
void raw_free(void *p, size_t bytes, cudaStream_t stream);
pic_status rebuild_active(pic_sim *s);
pic_status build_block_lists(pic_sim *s);
int split_field_launches(const FieldP &f);

}  // namespace pic

#define CK(sim, call)                                                                          \
    do {                                                                                       \
        cudaError_t _e = (call);                                                               \
        if (_e != cudaSuccess)                                                                 \
            return pic::fail(sim, PIC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
    } while (0)
