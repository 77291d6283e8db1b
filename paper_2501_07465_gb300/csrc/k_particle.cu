// k_particle.cu -- the particle phase of one PIC step, fused in one kernel:
// CIC gather of E^n, B^n -> push (free: Boris; bound: modified Boris;
// Dirac: Boris + |v| renormalised to v_F) -> reflection at material edges
// -> Esirkepov charge-conserving current deposit.
//
// Two instantiations per dimensionality: the plain kernel (specular
// reflection, open edges by a null mask) and the one with the boundary
// variants of Sec. 3 -- an external electrostatic field added to the
// gathered E (the work-function barrier), and diffuse reflection drawn from
// Philox keyed on (particle id, step, species).
//
// Paper passages: gather and deposit with the shape function W (Sec. 4.1);
// free push Appendix A.1 (Eqs. borisvpm, borisrotsol, borisscheme); bound
// push Sec. 4 Eq. modlorentz and Appendix A.2 (Eqs. modborisvpm,
// modborisrotsol, modborisBrot); Dirac push Sec. 5; material boundary Sec. 3.
//
// Work decomposition: particles are sorted by tile (T0 x T1 x T2 cells).  The
// persistent CTAs take tiles from the active-tile list (largest particle
// count first) through an atomic counter as they become free; for each tile it
// stages E^n and B^{n-1/2} of the tile plus a halo (cells -2 .. T+2 on each
// axis) in shared memory, turns B^{n-1/2} into B^n = B^{n-1/2} - (dt/2)
// curl E^n in place, zeroes a J tile of the same extent, and then streams the
// tile's particles of every species: reads are coalesced SoA loads, the
// gather reads shared memory, the deposit accumulates in the shared J tile
// (shared-memory atomics: the per-tile reduction), and the J tile is flushed
// to global memory with one atomic per non-zero entry.  A particle that has
// drifted more than one cell out of its tile since the last sort takes a
// slow path (global gather, global atomics), so correctness never depends on
// how often the particles are re-sorted.
#include "k_particle.cuh"

namespace pic {

size_t particle_smem_bytes(const TileP &tp) { return (size_t)9 * tp.boxn * sizeof(float); }

template <int DIM>
cudaError_t particle_setup_dim(size_t smem, int *ctas_per_sm) {
    cudaError_t e = allow_max_dynamic_smem(batch_particle_kernel<DIM>);
    if (e != cudaSuccess) return e;
    e = allow_max_dynamic_smem(particle_kernel<DIM>);
    if (e != cudaSuccess) return e;
    if (DIM == 3 && (e = particle_lean_setup()) != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, particle_kernel<DIM>,
                                                         kThreads, smem);
}

cudaError_t particle_kernel_setup(int dims, size_t smem, int *ctas_per_sm, int *ctas_per_sm_ext,
                                  int *ctas_per_sm_tsc) {
    cudaError_t e = dims == 3 ? particle_setup_dim<3>(smem, ctas_per_sm)
                              : particle_setup_dim<2>(smem, ctas_per_sm);
    if (e != cudaSuccess) return e;
    if (ctas_per_sm_ext && (e = particle_ext_setup(dims, smem, ctas_per_sm_ext)) != cudaSuccess)
        return e;
    if (ctas_per_sm_tsc) return particle_tsc_setup(dims, smem, ctas_per_sm_tsc);
    return cudaSuccess;
}

cudaError_t launch_batch_particles(int dims, const ParticleLaunch *descs, const int *fpar,
                                  const int *active, const int2 *items, int nitems, int *sched,
                                  const long long *done, int nctas, size_t smem, bool ext,
                                  int shape, cudaStream_t s) {
    if (shape == 2)
        return launch_batch_particles_tsc(dims, descs, fpar, active, items, nitems, sched, done,
                                          nctas, smem, s);
    if (ext)
        return launch_batch_particles_ext(dims, descs, fpar, active, items, nitems, sched, done,
                                          nctas, smem, s);
    if (nctas < 1) nctas = 1;
    if (dims == 3)
        batch_particle_kernel<3><<<nctas, kThreads, smem, s>>>(descs, fpar, active, items, nitems,
                                                               sched, done);
    else
        batch_particle_kernel<2><<<nctas, kThreads, smem, s>>>(descs, fpar, active, items, nitems,
                                                               sched, done);
    return cudaGetLastError();
}

cudaError_t launch_particles(const ParticleLaunch &pl, int nctas, size_t smem, cudaStream_t s) {
    if (nctas < 1) nctas = 1;
    if (pl.shape == 2) return launch_particles_tsc(pl, nctas, smem, s);
    if (particle_launch_ext(pl)) return launch_particles_ext(pl, nctas, smem, s);
    // the completion of the deferred particles: a small grid (its list is
    // empty on most steps, and then each CTA only reads the length)
    if (particle_lean_fits(pl)) return launch_particles_lean(pl, nctas, (nctas + 11) / 12, s);
    if (pl.g.dims == 3) particle_kernel<3><<<nctas, kThreads, smem, s>>>(pl);
    else particle_kernel<2><<<nctas, kThreads, smem, s>>>(pl);
    return cudaGetLastError();
}

}  // namespace pic
