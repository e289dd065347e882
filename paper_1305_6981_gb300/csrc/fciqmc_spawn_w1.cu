// Spawning kernels for one-word determinants (up to 32 spatial orbitals).
#include "fciqmc_spawn_impl.cuh"

namespace fq {

void launch_sweep_w1(int mode, int grid, cudaStream_t s, const Params &P) { launch_sweep_impl<1>(mode, grid, s, P); }
void launch_heavy_w1(int mode, int grid, cudaStream_t s, const Params &P) { launch_heavy_impl<1>(mode, grid, s, P); }
cudaError_t sweep_occupancy_w1(int n_elec, int *blocks_per_sm) {
    cudaError_t e = configure_spawn_impl<1>();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_sweep<1, 0>, kTile, sweep_bytes<1>(n_elec));
}

}  // namespace fq
