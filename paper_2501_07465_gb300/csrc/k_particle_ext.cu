// k_particle_ext.cu -- the particle kernels with the boundary variants of
// Sec. 3 (external electrostatic field, diffuse reflection) and the
// anisotropic bound push, single-simulation and batch, instantiated apart
// from the plain ones so that the two compile in parallel.
#include "k_particle.cuh"

namespace pic {

namespace {

template <int DIM>
cudaError_t ext_setup_dim(size_t smem, int *ctas_per_sm) {
    cudaError_t e = allow_max_dynamic_smem(particle_kernel_ext<DIM>);
    if (e != cudaSuccess) return e;
    e = allow_max_dynamic_smem(batch_particle_kernel<DIM, true>);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, particle_kernel_ext<DIM>,
                                                         kThreads, smem);
}

}  // namespace

cudaError_t particle_ext_setup(int dims, size_t smem, int *ctas_per_sm) {
    return dims == 3 ? ext_setup_dim<3>(smem, ctas_per_sm) : ext_setup_dim<2>(smem, ctas_per_sm);
}

cudaError_t launch_batch_particles_ext(int dims, const ParticleLaunch *descs, const int *fpar,
                                       const int *active, const int2 *items, int nitems,
                                       int *sched, const long long *done, int nctas, size_t smem,
                                       cudaStream_t s) {
    if (nctas < 1) nctas = 1;
    if (dims == 3)
        batch_particle_kernel<3, true><<<nctas, kThreads, smem, s>>>(descs, fpar, active, items,
                                                                     nitems, sched, done);
    else
        batch_particle_kernel<2, true><<<nctas, kThreads, smem, s>>>(descs, fpar, active, items,
                                                                     nitems, sched, done);
    return cudaGetLastError();
}

cudaError_t launch_particles_ext(const ParticleLaunch &pl, int nctas, size_t smem,
                                 cudaStream_t s) {
    if (nctas < 1) nctas = 1;
    if (pl.g.dims == 3) particle_kernel_ext<3><<<nctas, kThreads, smem, s>>>(pl);
    else particle_kernel_ext<2><<<nctas, kThreads, smem, s>>>(pl);
    return cudaGetLastError();
}

}  // namespace pic
