// Launchers of the spawning kernels (k_sweep, k_heavy), defined in one translation unit per determinant
// width so that their instantiations (plain, permitted space, spin-coupled functions, both) compile in
// parallel with the rest of the library. mode: bit 0 permitted space, bit 1 spin-coupled functions.
#pragma once

#include <cuda_runtime.h>

namespace fq {

struct Params;

void launch_sweep_w1(int mode, int grid, cudaStream_t s, const Params &P);
void launch_heavy_w1(int mode, int grid, cudaStream_t s, const Params &P);
cudaError_t sweep_occupancy_w1(int n_elec, int *blocks_per_sm);  // also sets the kernels' shared-memory limits
void launch_sweep_w2(int mode, int grid, cudaStream_t s, const Params &P);
void launch_heavy_w2(int mode, int grid, cudaStream_t s, const Params &P);
cudaError_t sweep_occupancy_w2(int n_elec, int *blocks_per_sm);

}  // namespace fq
