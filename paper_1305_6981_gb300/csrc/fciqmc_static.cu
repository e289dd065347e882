// Estimators of a caller-supplied walker list with scratch in a static device array.
//
// This is the one entry point of the library that needs neither a handle nor a workspace: its
// scratch (one partial sum per 256-determinant tile, four integer accumulators) lives in the
// file-scope array g_scratch below, so a caller that may not allocate device memory at the time
// of the call can still evaluate N_w, N_d, C_0 and the projected-energy numerator of a list it
// already holds on the device. The declaration and the contract are in include/fciqmc.h.
#include <cuda_runtime.h>

#include <mutex>

#include "fciqmc.h"
#include "fciqmc_device.cuh"

namespace {

constexpr int kStaticTile = 256;
constexpr long long kStaticMaxTiles = FCIQMC_STATIC_MAX_DETS / kStaticTile;
constexpr int kStaticMaxDevices = 64;

struct StaticScratch {
    unsigned long long nw, nd;
    long long c0;
    unsigned long long bad;  // entries skipped as invalid
    double partial[kStaticMaxTiles];
};

// Scratch shared by every call on a device; it keeps the last call's contents.
static __device__ __align__(256) StaticScratch g_scratch;

std::mutex g_mutex;
StaticScratch *g_addr[kStaticMaxDevices] = {};

__device__ __forceinline__ double warp_sum_f64(double x) {
    for (int o = 16; o > 0; o >>= 1) x = __dadd_rn(x, __shfl_down_sync(0xFFFFFFFFu, x, o));
    return x;
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
    return x;
}

__global__ void k_static_clear(StaticScratch *s) {
    if (threadIdx.x == 0) {
        s->nw = 0;
        s->nd = 0;
        s->c0 = 0;
        s->bad = 0;
    }
}

// An entry the estimator can use: n_elec occupied spin orbitals, none at or beyond n_so, a population that
// negates within int32; for spin-coupled functions also M_s = 0 and the stored (smaller) determinant of the
// pair. Checked before any integral is read, so an invalid entry never indexes the integral arrays.
template <int W>
__device__ __forceinline__ bool static_entry_ok(const fq::Params &P, const unsigned long long (&d)[W], int c) {
    int cnt = 0;
    bool ok = c != (-2147483647 - 1);
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int hi = P.n_so - 64 * w;
        if (hi < 64 && (hi <= 0 ? d[w] != 0ull : (d[w] >> hi) != 0ull)) ok = false;
        cnt += __popcll(d[w]);
    }
    if (cnt != P.n_elec) ok = false;
    if (P.hphf) {
        unsigned long long db[W];
        fq::flip_spins<W>(d, db);
        int na = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) na += __popcll(d[w] & fq::kEven);
        if (fq::det_less<W>(db, d) || 2 * na != P.n_elec) ok = false;
    }
    return ok;
}

// One tile of 256 determinants per block iteration; each tile's FP64 sum is stored in its own slot
// (lane tree, then warps in order), so the result does not depend on the grid.
template <int W>
__global__ void __launch_bounds__(kStaticTile) k_static_estimate(fq::Params P, const unsigned long long *dets,
                                                                  const int *pops, long long n, StaticScratch *s) {
    __shared__ unsigned char s_ref_occ[fq::MAXN];
    __shared__ double s_red[kStaticTile / 32];
    __shared__ unsigned long long s_cnt[3][kStaticTile / 32];
    if (threadIdx.x == 0) {
        int m = 0;
        for (int k = 0; k < P.n_so; ++k)
            if ((P.ref[k >> 6] >> (k & 63)) & 1ull) s_ref_occ[m++] = (unsigned char)k;
    }
    __syncthreads();
    P.ref_occ = s_ref_occ;
    const long long ntiles = (n + kStaticTile - 1) / kStaticTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long nw = 0, nd = 0, bad = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long i = t * kStaticTile + threadIdx.x;
        double num = 0.0;
        if (i < n) {
            const int c = pops[i];
            if (c != 0) {
                unsigned long long d[W];
#pragma unroll
                for (int w = 0; w < W; ++w) d[w] = dets[i * W + w];
                if (!static_entry_ok<W>(P, d, c)) {
                    bad += 1;
                } else {
                    nw += (unsigned)(c < 0 ? -c : c);
                    nd += 1;
                    unsigned long long xd = 0;
                    int diff = 0;
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        xd |= d[w] ^ P.ref[w];
                        diff += __popcll(d[w] ^ P.ref[w]);
                    }
                    if (xd == 0) {
                        s->c0 = c;
                    } else if (diff == 2 || diff == 4) {
                        double h0 = fq::h0i<W>(P, d);
                        if (P.hphf && fq::n_open<W>(d) > 0) h0 = __dmul_rn(h0, fq::kSqrt2);  // closed reference, open function
                        num = __dmul_rn(h0, (double)c);
                    }
                }
            }
        }
        num = warp_sum_f64(num);
        if (lane == 0) s_red[warp] = num;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int w = 0; w < kStaticTile / 32; ++w) tot = __dadd_rn(tot, s_red[w]);
            s->partial[t] = tot;
        }
        __syncthreads();
    }
    nw = warp_sum_u64(nw);
    nd = warp_sum_u64(nd);
    bad = warp_sum_u64(bad);
    if (lane == 0) {
        s_cnt[0][warp] = nw;
        s_cnt[1][warp] = nd;
        s_cnt[2][warp] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0, b = 0, x = 0;
        for (int w = 0; w < kStaticTile / 32; ++w) {
            a += s_cnt[0][w];
            b += s_cnt[1][w];
            x += s_cnt[2][w];
        }
        if (a) atomicAdd(&s->nw, a);
        if (b) atomicAdd(&s->nd, b);
        if (x) atomicAdd(&s->bad, x);
    }
}

__global__ void k_static_finish(const StaticScratch *s, long long ntiles, double *out) {
    if (threadIdx.x != 0) return;
    double num = 0.0;
    for (long long t = 0; t < ntiles; ++t) num = __dadd_rn(num, s->partial[t]);
    out[0] = (double)s->nw;
    out[1] = (double)s->nd;
    out[2] = (double)s->c0;
    out[3] = num;
    out[4] = (double)s->bad;
}

// Device address of g_scratch for the current device, looked up on the first call per device.
int scratch_address(StaticScratch **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FCIQMC_ERR_CUDA;
    if (dev < 0 || dev >= kStaticMaxDevices) return FCIQMC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return FCIQMC_ERR_CUDA;
        g_addr[dev] = static_cast<StaticScratch *>(p);
    }
    *out = g_addr[dev];
    return FCIQMC_OK;
}

}  // namespace

extern "C" int fciqmc_estimate_list_static(const double *h_dev, const double *eri_dev, int n_elec, int n_orb,
                                           const uint64_t *reference, const uint64_t *dets_dev,
                                           const int32_t *pops_dev, int64_t n_dets, int32_t flags,
                                           double *out_dev, void *cuda_stream) {
    if (n_orb < 1 || n_orb > 64 || n_elec < 1 || n_elec > fq::MAXN || n_elec >= 2 * n_orb) return FCIQMC_ERR_UNSUPPORTED;
    if (!h_dev || !eri_dev || !reference || !out_dev || n_dets < 0 || (n_dets > 0 && (!dets_dev || !pops_dev)))
        return FCIQMC_ERR_INVALID_ARG;
    if ((flags & ~FCIQMC_STATIC_SPIN_COUPLED) != 0) return FCIQMC_ERR_INVALID_ARG;
    if (n_dets > FCIQMC_STATIC_MAX_DETS) return FCIQMC_ERR_CAPACITY;
    const int W = (2 * n_orb + 63) / 64;
    int nref = 0;
    for (int w = 0; w < W; ++w) {
        const int hi = 2 * n_orb - 64 * w;  // bits [hi, 64) of word w lie beyond the basis
        if (hi < 64 && (reference[w] >> hi) != 0ull) return FCIQMC_ERR_INVALID_ARG;
        nref += __builtin_popcountll(reference[w]);
    }
    if (nref != n_elec) return FCIQMC_ERR_INVALID_ARG;
    const bool spin_coupled = (flags & FCIQMC_STATIC_SPIN_COUPLED) != 0;
    if (spin_coupled)  // the reference of spin-coupled functions is closed-shell
        for (int w = 0; w < W; ++w)
            if (((reference[w] ^ (reference[w] >> 1)) & 0x5555555555555555ull) != 0ull) return FCIQMC_ERR_INVALID_ARG;
    StaticScratch *s = nullptr;
    int rc = scratch_address(&s);
    if (rc != FCIQMC_OK) return rc;
    fq::Params P{};
    P.n_elec = n_elec;
    P.n_orb = n_orb;
    P.n_so = 2 * n_orb;
    P.h = h_dev;
    P.eri = eri_dev;
    P.ref[0] = reference[0];
    P.ref[1] = W == 2 ? reference[1] : 0ull;
    P.hphf = spin_coupled ? 1 : 0;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const long long ntiles = (n_dets + kStaticTile - 1) / kStaticTile;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FCIQMC_ERR_CUDA;
    const long long grid = ntiles > 0 ? (ntiles < 8LL * sms ? ntiles : 8LL * sms) : 1;
    k_static_clear<<<1, 32, 0, st>>>(s);
    if (W == 1) k_static_estimate<1><<<(unsigned)grid, kStaticTile, 0, st>>>(P, reinterpret_cast<const unsigned long long *>(dets_dev), pops_dev, n_dets, s);
    else k_static_estimate<2><<<(unsigned)grid, kStaticTile, 0, st>>>(P, reinterpret_cast<const unsigned long long *>(dets_dev), pops_dev, n_dets, s);
    k_static_finish<<<1, 32, 0, st>>>(s, ntiles, out_dev);
    return cudaGetLastError() == cudaSuccess ? FCIQMC_OK : FCIQMC_ERR_CUDA;
}
