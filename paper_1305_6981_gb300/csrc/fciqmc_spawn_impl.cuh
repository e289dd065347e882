// Shared body of the per-width spawning launchers (included by fciqmc_spawn_w1.cu and _w2.cu).
#pragma once

#include "fciqmc_kernels.cuh"
#include "fciqmc_spawn.h"

namespace fq {

// dynamic shared memory of both spawning kernels: one spawn queue per warp; the sweep's also the occupied
// lists of its tile
template <int W>
constexpr size_t queue_bytes() { return sizeof(SpawnQueue<W>) * (kTile / 32); }
template <int W>
size_t sweep_bytes(int n_elec) { return queue_bytes<W>() + (size_t)kTile * occ_stride(n_elec); }

template <int W>
cudaError_t configure_spawn_impl() {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *f, size_t b) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
    };
    const size_t bs = sweep_bytes<W>(MAXN), bh = queue_bytes<W>();
    set((const void *)k_sweep<W, 0>, bs); set((const void *)k_sweep<W, 1>, bs);
    set((const void *)k_sweep<W, 2>, bs); set((const void *)k_sweep<W, 3>, bs);
    set((const void *)k_heavy<W, 0>, bh); set((const void *)k_heavy<W, 1>, bh);
    set((const void *)k_heavy<W, 2>, bh); set((const void *)k_heavy<W, 3>, bh);
    return e;
}

template <int W>
void launch_sweep_impl(int mode, int grid, cudaStream_t s, const Params &P) {
    const size_t b = sweep_bytes<W>(P.n_elec);
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
