// Shared body of the per-width spawning launchers (included by fciqmc_spawn_w1.cu and _w2.cu).
#pragma once

#include "fciqmc_kernels.cuh"
#include "fciqmc_spawn.h"

namespace fq {

template <int W>
void launch_sweep_impl(int mode, int grid, cudaStream_t s, const Params &P) {
    switch (mode) {
        case 0: k_sweep<W, 0><<<grid, kTile, 0, s>>>(P); break;
        case 1: k_sweep<W, 1><<<grid, kTile, 0, s>>>(P); break;
        case 2: k_sweep<W, 2><<<grid, kTile, 0, s>>>(P); break;
        default: k_sweep<W, 3><<<grid, kTile, 0, s>>>(P); break;
    }
}

template <int W>
void launch_heavy_impl(int mode, int grid, cudaStream_t s, const Params &P) {
    switch (mode) {
        case 0: k_heavy<W, 0><<<grid, kTile, 0, s>>>(P); break;
        case 1: k_heavy<W, 1><<<grid, kTile, 0, s>>>(P); break;
        case 2: k_heavy<W, 2><<<grid, kTile, 0, s>>>(P); break;
        default: k_heavy<W, 3><<<grid, kTile, 0, s>>>(P); break;
    }
}

}  // namespace fq
