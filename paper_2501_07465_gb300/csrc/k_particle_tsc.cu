// k_particle_tsc.cu -- the particle kernels with TSC (order-2) shapes for
// the free and Dirac particles (gather from three nodes per axis on each
// component's stagger, Esirkepov deposit over four; the shape function W of
// Sec. 4.1 at the next order), the boundary variants of Sec. 3 included.
// Bound particles keep CIC.  Single-simulation and batch kernels,
// instantiated apart so the plain kernels keep their registers and compile in
// parallel.
#include "k_particle.cuh"

namespace pic {

namespace {

template <int DIM>
__global__ void __launch_bounds__(kThreads) particle_kernel_tsc(const __grid_constant__ ParticleLaunch P) {
    particle_phase<DIM, true, 2>(P);
}

template <int DIM>
cudaError_t tsc_setup_dim(size_t smem, int *ctas_per_sm) {
    cudaError_t e = allow_max_dynamic_smem(particle_kernel_tsc<DIM>);
    if (e != cudaSuccess) return e;
    e = allow_max_dynamic_smem(batch_particle_kernel<DIM, true, 2>);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, particle_kernel_tsc<DIM>,
                                                         kThreads, smem);
}

}  // namespace

cudaError_t particle_tsc_setup(int dims, size_t smem, int *ctas_per_sm) {
    return dims == 3 ? tsc_setup_dim<3>(smem, ctas_per_sm) : tsc_setup_dim<2>(smem, ctas_per_sm);
}

cudaError_t launch_batch_particles_tsc(int dims, const ParticleLaunch *descs, const int *fpar,
                                       const int *active, const int2 *items, int nitems,
                                       int *sched, const long long *done, int nctas, size_t smem,
                                       cudaStream_t s) {
    if (nctas < 1) nctas = 1;
    if (dims == 3)
        batch_particle_kernel<3, true, 2><<<nctas, kThreads, smem, s>>>(descs, fpar, active, items,
                                                                        nitems, sched, done);
    else
        batch_particle_kernel<2, true, 2><<<nctas, kThreads, smem, s>>>(descs, fpar, active, items,
                                                                        nitems, sched, done);
    return cudaGetLastError();
}

cudaError_t launch_particles_tsc(const ParticleLaunch &pl, int nctas, size_t smem,
                                 cudaStream_t s) {
    if (nctas < 1) nctas = 1;
    if (pl.g.dims == 3) particle_kernel_tsc<3><<<nctas, kThreads, smem, s>>>(pl);
    else particle_kernel_tsc<2><<<nctas, kThreads, smem, s>>>(pl);
    return cudaGetLastError();
}

}  // namespace pic
