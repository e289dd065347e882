// Shared body of the per-width spawning launchers (included by fciqmc_spawn_w1.cu and _w2.cu).
#pragma once

#include "fciqmc_kernels.cuh"
#include "fciqmc_spawn.h"

namespace fq {

// dynamic shared memory of both spawning kernels: one spawn queue per warp
template <int W>
constexpr size_t queue_bytes() { return sizeof(SpawnQueue<W>) * (kTile / 32); }

template <int W>
cudaError_t configure_spawn_impl() {
    const int b = (int)queue_bytes<W>();
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *f) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    };
    set((const void *)k_sweep<W, 0>); set((const void *)k_sweep<W, 1>);
    set((const void *)k_sweep<W, 2>); set((const void *)k_sweep<W, 3>);
    set((const void *)k_heavy<W, 0>); set((const void *)k_heavy<W, 1>);
    set((const void *)k_heavy<W, 2>); set((const void *)k_heavy<W, 3>);
    return e;
}

template <int W>
void launch_sweep_impl(int mode, int grid, cudaStream_t s, const Params &P) {
    const size_t b = queue_bytes<W>();
    switch (mode) {
        case 0: k_sweep<W, 0><<<grid, kTile, b, s>>>(P); break;
        case 1: k_sweep<W, 1><<<grid, kTile, b, s>>>(P); break;
        case 2: k_sweep<W, 2><<<grid, kTile, b, s>>>(P); break;
        default: k_sweep<W, 3><<<grid, kTile, b, s>>>(P); break;
    }
}

template <int W>
void launch_heavy_impl(int mode, int grid, cudaStream_t s, const Params &P) {
    const size_t b = queue_bytes<W>();
    switch (mode) {
        case 0: k_heavy<W, 0><<<grid, kTile, b, s>>>(P); break;
        case 1: k_heavy<W, 1><<<grid, kTile, b, s>>>(P); break;
        case 2: k_heavy<W, 2><<<grid, kTile, b, s>>>(P); break;
        default: k_heavy<W, 3><<<grid, kTile, b, s>>>(P); break;
    }
}

}  // namespace fq
