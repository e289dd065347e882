// Spawning kernels for two-word determinants (33 to 64 spatial orbitals).
#include "fciqmc_spawn_impl.cuh"

namespace fq {

void launch_sweep_w2(int mode, int grid, cudaStream_t s, const Params &P) { launch_sweep_impl<2>(mode, grid, s, P); }
void launch_heavy_w2(int mode, int grid, cudaStream_t s, const Params &P) { launch_heavy_impl<2>(mode, grid, s, P); }
cudaError_t sweep_occupancy_w2(int n_elec, int *blocks_per_sm) {
    cudaError_t e = configure_spawn_impl<2>();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_sweep<2, 0>, kTile, sweep_bytes<2>(n_elec));
}

}  // namespace fq
