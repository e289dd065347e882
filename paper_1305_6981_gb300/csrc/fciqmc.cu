// C ABI of the FCIQMC walker cycle: workspace layout, setup, iteration launch, read-back.
// The declarations and the contract of every entry point are in include/fciqmc.h.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "fciqmc.h"
#include "fciqmc_cycle.cuh"
#include "fciqmc_spawn.h"

using fq::DevState;
using fq::Params;

namespace {

#define FQ_CUDA(call)                                     \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return FCIQMC_ERR_CUDA;    \
    } while (0)

// NVTX range over a library call (a no-op unless a profiler is attached), so a timeline attributes the
// graph launches, loads and read-backs to the call that issued them.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr size_t kAlign = 256;
constexpr int kMaxGrid = 4096;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
long long next_pow2(long long x) {
    long long p = 1;
    while (p < x) p <<= 1;
    return p;
}
int log2_exact(long long x) {
    int b = 0;
    while ((1LL << b) < x) ++b;
    return b;
}

struct Sizes {
    int W, n_so, npairs, n_parts, part, ostride;
    long long n_eri, cap, idx_cap, mt_cap, hist_cap, heavy_cap, ref_cap, ob_cap;
};

bool sizes_of(int n_elec, int n_orb, const fciqmc_options &o, Sizes &z) {
    if (n_orb < 1 || n_orb > 64 || n_elec < 1 || n_elec > fq::MAXN || n_elec >= 2 * n_orb) return false;
    z.W = (2 * n_orb + 63) / 64;
    z.n_so = 2 * n_orb;
    z.ostride = fq::occ_stride(n_elec);
    z.npairs = n_elec * (n_elec - 1) / 2;
    long long npair = (long long)n_orb * (n_orb + 1) / 2;
    z.n_eri = npair * (npair + 1) / 2;
    z.cap = std::max<long long>(o.main_capacity > 0 ? o.main_capacity : (1LL << 20), 1024);
    if (z.cap > (1LL << 31) - 2) return false;
    const double load = (o.index_load > 0.0 && o.index_load < 1.0) ? o.index_load : 0.5;
    z.idx_cap = next_pow2(std::max<long long>((long long)std::ceil((double)z.cap / load), 1 << 12));
    z.mt_cap = next_pow2(std::max<long long>(o.spawn_capacity > 0 ? o.spawn_capacity : z.cap / 2, 1 << 12));
    if (z.mt_cap > (1LL << 32)) return false;
    // records of determinants with |C| > 256 (a run that needs more stops with FCIQMC_ERR_CAPACITY)
    z.heavy_cap = std::max<long long>(1 << 14, std::min<long long>(z.cap / 2, 1 << 22));
    z.hist_cap = std::max<long long>(o.history_capacity > 0 ? o.history_capacity : (1LL << 16), 16);
    // the reference's double excitations: at most npairs x virtuals x virtuals choices
    const long long nv = z.n_so - n_elec;
    z.ref_cap = std::min<long long>((long long)z.npairs * nv * nv, 1LL << 22);
    // hash partitioning: one outbox per destination partition
    z.n_parts = o.n_partitions > 1 ? o.n_partitions : 1;
    z.part = o.n_partitions > 1 ? o.partition_index : 0;
    z.ob_cap = z.n_parts > 1 ? (o.outbox_capacity > 0 ? o.outbox_capacity : std::max<long long>(z.mt_cap / 4, 1024)) : 0;
    return true;
}

struct Layout {
    size_t state, h, h_f, eri, eri_f, wpair, map1, cmask, unionm, irrep, pairs, recip, rcpf, ref_occ, facts, e0;
    size_t det[2], hd[2], hdf[2], pop[2][2], pre[2], occa[2], idx, mt, merged, heavy, heavy_occ, heavy_base, heavy_att, partial, hist;
    size_t ref_pinfo, ref_off2, ref_exc, outbox;
    size_t total;
};

Layout layout_of(const Sizes &z, int n_orb) {
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    L.state = take(sizeof(DevState));
    L.h = take(sizeof(double) * n_orb * n_orb);
    L.h_f = take(sizeof(float) * n_orb * n_orb);
    L.eri = take(sizeof(double) * z.n_eri);
    L.eri_f = take(sizeof(float) * z.n_eri);
    L.wpair = take(sizeof(double) * 2 * n_orb * n_orb);
    L.map1 = take(sizeof(unsigned long long) * fq::MAXSO);
    L.cmask = take(sizeof(unsigned long long) * fq::NCLASS * fq::MAXW);
    L.unionm = take(sizeof(unsigned long long) * 2 * 256 * fq::MAXW);
    L.irrep = take(fq::MAXSO);
    L.pairs = take(sizeof(unsigned short) * std::max(z.npairs, 1));
    L.recip = take(sizeof(double) * (2 * fq::MAXSO + 2));
    L.rcpf = take(sizeof(float) * (2 * fq::MAXSO + 2));
    L.ref_occ = take(fq::MAXN);
    L.facts = take(sizeof(long long) * 4);
    L.e0 = take(sizeof(double));
    for (int b = 0; b < 2; ++b) {
        L.det[b] = take(sizeof(unsigned long long) * z.W * z.cap);
        L.hd[b] = take(sizeof(double) * z.cap);
        L.hdf[b] = take(sizeof(float) * z.cap);
        L.pop[b][0] = take(sizeof(int) * z.cap);
        L.pop[b][1] = take(sizeof(int) * z.cap);
        L.pre[b] = take(sizeof(unsigned long long) * fq::PRE_WORDS * z.cap);
        L.occa[b] = take((size_t)z.ostride * z.cap);
    }
    const int stride = z.W == 1 ? 2 : 4;
    L.idx = take(sizeof(unsigned long long) * stride * z.idx_cap);
    L.mt = take(sizeof(unsigned long long) * stride * z.mt_cap);
    L.merged = take(sizeof(unsigned) * z.mt_cap);
    L.heavy = take(sizeof(fq::DetView<2>) * z.heavy_cap);
    L.heavy_occ = take((size_t)fq::MAXN * z.heavy_cap);
    L.heavy_base = take(sizeof(unsigned) * z.heavy_cap);
    L.heavy_att = take(sizeof(unsigned) * z.heavy_cap);
    L.partial = take(sizeof(double) * (std::max<long long>((z.cap + fq::kTile - 1) / fq::kTile, kMaxGrid) + fq::kTileSums));
    L.hist = take(sizeof(fciqmc_row) * z.hist_cap);
    L.ref_pinfo = take(sizeof(unsigned) * std::max(z.npairs, 1));
    L.ref_off2 = take(sizeof(unsigned) * std::max<long long>((long long)z.npairs * z.n_so, 1));
    L.ref_exc = take(sizeof(fq::RefExc) * std::max<long long>(z.ref_cap, 1));
    L.outbox = take(sizeof(unsigned long long) * stride * z.n_parts * z.ob_cap);
    L.total = off;
    return L;
}

// Host copies of the orbital map and fingerprint of Algorithm 1 (the device computes the same in k_setup and
// fingerprint<W>): Philox4x32-10 (Salmon et al., SC'11) with 64-bit products.
void host_philox(const unsigned ctr_in[4], const unsigned key_in[2], unsigned out[4]) {
    unsigned c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3], k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = 0xD2511F53ull * c0, p1 = 0xCD9E8D57ull * c2;
        const unsigned n0 = (unsigned)(p1 >> 32) ^ c1 ^ k0, n2 = (unsigned)(p0 >> 32) ^ c3 ^ k1;
        c0 = n0;
        c1 = (unsigned)p1;
        c2 = n2;
        c3 = (unsigned)p0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}
unsigned long long host_map1(int k) {
    const unsigned ctr[4] = {(unsigned)k, 0u, 0u, 0u}, key[2] = {0x46434951u, 0x4D415031u};
    unsigned o[4];
    host_philox(ctr, key, o);
    return (unsigned long long)o[0] | ((unsigned long long)o[1] << 32);
}
unsigned long long host_fingerprint(const uint64_t *d, int W, const unsigned long long *map1) {
    unsigned long long h = 0, n = 0;
    for (int w = 0; w < W; ++w)
        for (int b = 0; b < 64; ++b)
            if ((d[w] >> b) & 1ull) h = 1099511628211ull * h + map1[64 * w + b] * (++n);
    return h;
}

}  // namespace

struct fciqmc_handle {
    Params P;
    Sizes z;
    Layout L;
    char *ws;
    cudaStream_t stream;
    fciqmc_info info;
    int sweep_grid, heavy_grid, ann_grid, diag_grid, small_grid;
    size_t smem_w;
    double e_core;
    cudaGraph_t graph_tmpl;  // one iteration, kept for composing batch graphs
    cudaGraphExec_t graph;
    bool graph_ready;
    int grid_request;
    fciqmc_options opt;      // as created (checked when partitions are grouped)
    double tau;
    int32_t init_thr;
    cudaStream_t aux, aux2;  // helper streams of set_walkers (created on first use), joined by events
    cudaEvent_t ev_fork, ev_join, ev_join2, ev_chunk[8];
};

namespace {

template <typename T>
T *at(fciqmc_handle *h, size_t off) {
    return reinterpret_cast<T *>(h->ws + off);
}

template <int W>
int configure_kernels(fciqmc_handle *h) {
    FQ_CUDA(cudaFuncSetAttribute(fq::k_new_diag<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->smem_w));
    FQ_CUDA(cudaFuncSetAttribute(fq::k_prepare_list<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->smem_w));
    FQ_CUDA(cudaFuncSetAttribute(fq::k_reference_energy<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->smem_w));
    int dev = 0, sms = 0, per_sm = 0;
    FQ_CUDA(cudaGetDevice(&dev));
    FQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    FQ_CUDA(W == 1 ? fq::sweep_occupancy_w1(h->P.n_elec, &per_sm) : fq::sweep_occupancy_w2(h->P.n_elec, &per_sm));
    h->sweep_grid = std::min(kMaxGrid, std::max(1, sms * std::max(per_sm, 1)));
    FQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fq::k_annihilate<W>, 256, 0));
    h->ann_grid = std::min(kMaxGrid, std::max(1, sms * std::max(per_sm, 1)));
    // k_new_diag: as many blocks as fit at once (one new slot per thread up to that many; each thread's H_ii
    // is a long chain of dependent FP64 adds, so more resident warps hide its latency; blocks with no new
    // slot return before loading the pair terms)
    FQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fq::k_new_diag<W>, 256, h->smem_w));
    h->diag_grid = std::min(kMaxGrid, std::max(1, sms * std::max(per_sm, 1)));
    h->heavy_grid = std::min(kMaxGrid, sms * 4);
    if (h->grid_request > 0) {
        const int g = std::min(kMaxGrid, h->grid_request);
        h->sweep_grid = std::min(h->sweep_grid, g);
        h->ann_grid = std::min(h->ann_grid, g);
        h->diag_grid = std::min(h->diag_grid, g);
        h->heavy_grid = std::min(h->heavy_grid, g);
    }
    h->P.heavy_warps = (long long)h->heavy_grid * (fq::kTile / 32);
    h->P.sweep_blocks = h->sweep_grid;
    h->small_grid = std::min(kMaxGrid, sms * 8);
    h->info.num_sms = sms;
    h->info.grid_blocks = h->sweep_grid;
    h->P.sweep_grid = h->sweep_grid;
    return FCIQMC_OK;
}

// The spawning kernels, instantiated with the permitted-space test only for runs that have one.
int spawn_mode(const fciqmc_handle *h) { return (h->P.space ? 1 : 0) | (h->P.hphf ? 2 : 0); }
template <int W>
void launch_sweep(fciqmc_handle *h, cudaStream_t s) {
    if (W == 1) fq::launch_sweep_w1(spawn_mode(h), h->sweep_grid, s, h->P);
    else fq::launch_sweep_w2(spawn_mode(h), h->sweep_grid, s, h->P);
}
template <int W>
void launch_heavy(fciqmc_handle *h, cudaStream_t s) {
    if (W == 1) fq::launch_heavy_w1(spawn_mode(h), h->heavy_grid, s, h->P);
    else fq::launch_heavy_w2(spawn_mode(h), h->heavy_grid, s, h->P);
}
template <int W>
void launch_spawning(fciqmc_handle *h, cudaStream_t s) {
    launch_sweep<W>(h, s);
    launch_heavy<W>(h, s);
    // the sweep tiles' numerators are summed after k_heavy, which does not need them: the 32-block sum then
    // does not sit between the two spawning kernels
    fq::k_tile_sum<<<fq::kTileSums, 256, 0, s>>>(h->P);
}

template <int W>
void enqueue_iteration(fciqmc_handle *h, cudaStream_t s) {
    const Params &P = h->P;
    fq::k_compact_copy<W><<<h->small_grid, 256, 0, s>>>(P);
    fq::k_index_clear<<<h->small_grid, 256, 0, s>>>(P, 0);
    fq::k_index_locate_old<W><<<h->small_grid, 256, 0, s>>>(P);
    fq::k_index_clear_old<W><<<h->small_grid, 256, 0, s>>>(P);
    fq::k_index_fill<W><<<h->small_grid, 256, 0, s>>>(P, 0);
    fq::k_compact_finish<<<1, 32, 0, s>>>(P);
    launch_spawning<W>(h, s);
    fq::k_annihilate<W><<<h->ann_grid, 256, 0, s>>>(P);
    fq::k_new_diag<W><<<h->diag_grid, 256, h->smem_w, s>>>(P);
    if (P.occ_units > 1) fq::k_round<W><<<h->small_grid, 256, 0, s>>>(P);
    fq::k_finish<<<1, 32, 0, s>>>(P);
}

void enqueue(fciqmc_handle *h, cudaStream_t s) {
    if (h->z.W == 1) enqueue_iteration<1>(h, s);
    else enqueue_iteration<2>(h, s);
}

int build_graph(fciqmc_handle *h) {
    cudaStream_t cs;
    FQ_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        enqueue(h, cs);
        e = cudaStreamEndCapture(cs, &g);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph, g, 0);
    if (e == cudaSuccess) h->graph_tmpl = g;
    else if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    h->graph_ready = (e == cudaSuccess);
    cudaGetLastError();
    return FCIQMC_OK;
}

template <int W>
void launch_index_rebuild(fciqmc_handle *h) {
    fq::k_index_clear<<<h->small_grid, 256, 0, h->stream>>>(h->P, 1);
    fq::k_index_fill<W><<<h->small_grid, 256, 0, h->stream>>>(h->P, 1);
}

template <int W>
void launch_prepare(fciqmc_handle *h, int b, long long n, int compute) {  // slots [0, n)
    long long blocks = std::min<long long>((n + 255) / 256, h->small_grid);
    if (blocks < 1) blocks = 1;
    fq::k_prepare_list<W><<<(unsigned)blocks, 256, h->smem_w, h->stream>>>(h->P, b, 0, n, compute);
}

// The helper streams of set_walkers and their events, created together (nothing is kept if one fails).
int create_helper_stream(fciqmc_handle *h) {
    static_assert(sizeof(fciqmc_handle::ev_chunk) == 8 * sizeof(cudaEvent_t), "eight chunk events");
    cudaStream_t a = nullptr, a2 = nullptr;
    cudaEvent_t ev[11] = {};
    bool ok = cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&a2, cudaStreamNonBlocking) == cudaSuccess;
    for (cudaEvent_t &e : ev) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (a) cudaStreamDestroy(a);
        if (a2) cudaStreamDestroy(a2);
        cudaGetLastError();
        return FCIQMC_ERR_CUDA;
    }
    h->ev_fork = ev[0];
    h->ev_join = ev[1];
    h->ev_join2 = ev[2];
    for (int k = 0; k < 8; ++k) h->ev_chunk[k] = ev[3 + k];
    h->aux = a;
    h->aux2 = a2;
    return FCIQMC_OK;
}

// Copy, check, index and derived-data work of load_list, up to the join of the helper streams; bad receives
// the outcome of the check and of the inserts (1 invalid entry, 2 repeated determinant, 3 index full).
template <int W>
int load_stage(fciqmc_handle *h, const DevState &cur, const uint64_t *dets, const int32_t *pops,
               const double *hdiag, long long n, int &bad) {
    cudaStream_t s = h->stream, a = h->aux;
    const Params &P = h->P;
    const int b = cur.lb ^ 1;
    const unsigned blocks = (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, h->small_grid));
    const bool sparse = cur.status == 0 && cur.list_len >= 0 && cur.list_len * 16 <= h->z.idx_cap &&
                        h->z.idx_cap <= (1LL << 31);  // positions held as int
    int *pos = P.pop[cur.lb][cur.pp ^ 1];  // the old list's idle population buffer
    const unsigned ob = (unsigned)std::max<long long>(1, std::min<long long>((cur.list_len + 255) / 256, h->small_grid));
    FQ_CUDA(cudaMemsetAsync(&P.st->check_bad, 0, sizeof(int), s));
    FQ_CUDA(cudaEventRecord(h->ev_fork, s));
    FQ_CUDA(cudaStreamWaitEvent(a, h->ev_fork, 0));
    if (sparse && cur.list_len > 0) {
        fq::k_index_locate<W><<<ob, 256, 0, a>>>(P, cur.lb, cur.list_len, pos);
        fq::k_index_clear_at<W><<<ob, 256, 0, a>>>(P, pos, cur.list_len);
    } else if (!sparse) {
        fq::k_index_clear<<<h->small_grid, 256, 0, a>>>(P, 1);
    }
    const int nchunk = (int)std::min<long long>(8, std::max<long long>(1, n >> 20));  // >= 2^20 keys a chunk
    for (int k = 0; k < nchunk; ++k) {
        const long long lo = n * k / nchunk, hi = n * (k + 1) / nchunk;
        if (hi > lo) {
            FQ_CUDA(cudaMemcpyAsync(P.det[b] + W * lo, dets + W * lo, sizeof(uint64_t) * W * (hi - lo),
                                    cudaMemcpyHostToDevice, s));
            FQ_CUDA(cudaEventRecord(h->ev_chunk[k], s));
            FQ_CUDA(cudaStreamWaitEvent(a, h->ev_chunk[k], 0));
            const unsigned ib = (unsigned)std::max<long long>(1, std::min<long long>((hi - lo + 255) / 256, h->small_grid));
            fq::k_index_insert<W><<<ib, 256, 0, a>>>(P, b, lo, hi);
            // the chunk's derived words on the second helper stream, beside the index work
            FQ_CUDA(cudaStreamWaitEvent(h->aux2, h->ev_chunk[k], 0));
            fq::k_prepare_list<W><<<ib, 256, 0, h->aux2>>>(P, b, lo, hi, 0);
        }
    }
    FQ_CUDA(cudaGetLastError());
    FQ_CUDA(cudaEventRecord(h->ev_join, a));
    FQ_CUDA(cudaEventRecord(h->ev_join2, h->aux2));
    if (n > 0) {
        FQ_CUDA(cudaMemcpyAsync(P.pop[b][0], pops, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
        if (hdiag) FQ_CUDA(cudaMemcpyAsync(P.hd[b], hdiag, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    }
    fq::k_check_list<W><<<blocks, 256, 0, s>>>(P, b, n, hdiag ? 1 : 0);
    FQ_CUDA(cudaGetLastError());
    FQ_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));
    FQ_CUDA(cudaStreamWaitEvent(s, h->ev_join2, 0));
    FQ_CUDA(cudaMemcpyAsync(&bad, &P.st->check_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    FQ_CUDA(cudaStreamSynchronize(s));
    return FCIQMC_OK;
}

// Loads a list into buffer b; on success makes it the active list with the state st0. The index work
// runs on a helper stream while the list is copied in: the old list's entries are emptied (located first,
// or the whole index for a dense index or after a failed step), then each chunk of new keys is inserted as
// soon as it has arrived; a second helper stream derives each chunk's per-slot data (fingerprint, class
// counts, occupied list) meanwhile. The check of the new entries (and the float copies of given diagonal
// elements) runs on the caller's stream. A rejected list (invalid entries, a repeated determinant) or a
// failed copy leaves the run as it was: the index is rebuilt from the current list and the state is not
// replaced.
template <int W>
int load_list(fciqmc_handle *h, const DevState &cur, DevState &st0, const uint64_t *dets, const int32_t *pops,
              const double *hdiag, long long n) {
    cudaStream_t s = h->stream;
    const Params &P = h->P;
    if (!h->aux && create_helper_stream(h) != FCIQMC_OK) return FCIQMC_ERR_CUDA;
    int bad = 0;
    const int rc = load_stage<W>(h, cur, dets, pops, hdiag, n, bad);
    if (rc != FCIQMC_OK || bad) {
        cudaStreamSynchronize(h->aux);
        cudaStreamSynchronize(h->aux2);
        cudaStreamSynchronize(s);
        fq::k_index_clear<<<h->small_grid, 256, 0, s>>>(P, 1);
        fq::k_index_fill<W><<<h->small_grid, 256, 0, s>>>(P, 1);
        FQ_CUDA(cudaGetLastError());
        FQ_CUDA(cudaStreamSynchronize(s));
        if (rc != FCIQMC_OK) return rc;
        return bad == 3 ? FCIQMC_ERR_CAPACITY : FCIQMC_ERR_INVALID_ARG;
    }
    const int b = cur.lb ^ 1;
    st0.lb = b;
    st0.pp = 0;
    FQ_CUDA(cudaMemcpyAsync(P.st, &st0, sizeof(st0), cudaMemcpyHostToDevice, s));
    if (!hdiag) launch_prepare<W>(h, b, n, 1);
    // a failed step may have left claimed entries in the spawn table
    if (cur.status != 0) fq::k_mt_clear<<<h->small_grid, 256, 0, s>>>(P, W);
    FQ_CUDA(cudaGetLastError());
    return FCIQMC_OK;
}

int read_state(fciqmc_handle *h, DevState &st) {
    FQ_CUDA(cudaMemcpyAsync(&st, h->P.st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    FQ_CUDA(cudaStreamSynchronize(h->stream));
    return FCIQMC_OK;
}

}  // namespace

extern "C" {

void fciqmc_default_options(fciqmc_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->shift_damping = 0.05;
    opt->shift_period = 10;
    opt->initial_population = 10;
    opt->initial_shift = 0.0;
    opt->target_walkers = 1LL << 62;
    opt->seed = 1;
    opt->p_double = 0.0;
    opt->main_capacity = 1LL << 20;
    opt->spawn_capacity = 0;
    opt->history_capacity = 1LL << 16;
    opt->reference = nullptr;
}

size_t fciqmc_workspace_bytes(int n_elec, int n_orb, const fciqmc_options *opt) {
    fciqmc_options o;
    if (opt) o = *opt;
    else fciqmc_default_options(&o);
    Sizes z;
    if (!sizes_of(n_elec, n_orb, o, z)) return 0;
    return layout_of(z, n_orb).total;
}

const char *fciqmc_strerror(int status) {
    switch (status) {
        case FCIQMC_OK: return "ok";
        case FCIQMC_ERR_INVALID_ARG: return "invalid argument";
        case FCIQMC_ERR_CAPACITY: return "capacity exceeded (main list, hash index or spawn table)";
        case FCIQMC_ERR_NUMERIC: return "population or spawn count outside int32";
        case FCIQMC_ERR_TIMEOUT: return "bounded device wait timed out";
        case FCIQMC_ERR_CUDA: return "CUDA runtime error";
        case FCIQMC_ERR_UNSUPPORTED: return "unsupported size (n_orb <= 64, n_elec <= 64)";
        case FCIQMC_ERR_WORKSPACE: return "workspace too small or not 256-byte aligned";
        case FCIQMC_ERR_BOUNDS: return "device index out of range (debug build check)";
        default: return "unknown status";
    }
}

int fciqmc_create(const double *h1, const double *eri_s8, double e_core, int n_elec, int n_orb, int ms2,
                  const int32_t *orb_irrep, double tau, int32_t initiator_threshold, const fciqmc_options *opt,
                  void *workspace, size_t workspace_bytes, void *cuda_stream, fciqmc_handle **out) {
    if (!out) return FCIQMC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!h1 || !eri_s8 || !(tau > 0.0) || !std::isfinite(tau)) return FCIQMC_ERR_INVALID_ARG;
    fciqmc_options o;
    if (opt) o = *opt;
    else fciqmc_default_options(&o);
    if (o.shift_period < 1 || o.initial_population == 0 || o.target_walkers < 0) return FCIQMC_ERR_INVALID_ARG;
    if (o.n_partitions < 0 || o.n_partitions > fq::MAXPARTS || o.outbox_capacity < 0 ||
        (o.n_partitions > 1 && (o.partition_index < 0 || o.partition_index >= o.n_partitions)))
        return FCIQMC_ERR_INVALID_ARG;
    // hybrid walkers: populations, the initiator threshold and the target in units of 2^-bits walkers
    if (o.walker_fraction_bits < 0 || o.walker_fraction_bits > 20) return FCIQMC_ERR_INVALID_ARG;
    const int fbits = o.walker_fraction_bits;
    const double unit_scale = std::ldexp(1.0, fbits);
    const double occ_units = std::nearbyint((o.occupation_threshold > 0.0 ? o.occupation_threshold : 1.0) * unit_scale);
    if (!(occ_units >= 1.0) || occ_units > 2147483647.0 ||
        std::fabs((double)o.initial_population) * unit_scale > 2147483647.0 ||
        (initiator_threshold >= 0 && (double)initiator_threshold * unit_scale > 2147483647.0))
        return FCIQMC_ERR_INVALID_ARG;
    Sizes z;
    if (!sizes_of(n_elec, n_orb, o, z)) return FCIQMC_ERR_UNSUPPORTED;
    Layout L = layout_of(z, n_orb);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0 || workspace_bytes < L.total)
        return FCIQMC_ERR_WORKSPACE;
    // reference determinant
    uint64_t ref[2] = {0, 0};
    if (o.reference) {
        ref[0] = o.reference[0];
        if (z.W == 2) ref[1] = o.reference[1];
    } else {
        if ((n_elec + ms2) % 2 != 0 || ms2 < -n_elec || ms2 > n_elec) return FCIQMC_ERR_INVALID_ARG;
        int na = (n_elec + ms2) / 2, nb = (n_elec - ms2) / 2;
        if (na > n_orb || nb > n_orb) return FCIQMC_ERR_INVALID_ARG;
        for (int p = 0; p < na; ++p) ref[(2 * p) >> 6] |= 1ull << ((2 * p) & 63);
        for (int p = 0; p < nb; ++p) ref[(2 * p + 1) >> 6] |= 1ull << ((2 * p + 1) & 63);
    }
    int max_irrep = 0;
    if (orb_irrep) {
        for (int p = 0; p < n_orb; ++p) {
            if (orb_irrep[p] < 0 || orb_irrep[p] > 7) return FCIQMC_ERR_INVALID_ARG;
            max_irrep = std::max(max_irrep, (int)orb_irrep[p]);
        }
    }

    fciqmc_handle *h = new (std::nothrow) fciqmc_handle();
    if (!h) return FCIQMC_ERR_INVALID_ARG;
    h->z = z;
    h->L = L;
    h->ws = static_cast<char *>(workspace);
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->e_core = e_core;
    h->graph_ready = false;
    h->graph_tmpl = nullptr;
    h->grid_request = o.grid_blocks;
    h->smem_w = sizeof(double) * (2 * n_orb * n_orb + n_orb);
    h->opt = o;
    h->tau = tau;
    h->init_thr = initiator_threshold < 0 ? -1 : initiator_threshold;

    Params &P = h->P;
    std::memset(&P, 0, sizeof(P));
    P.n_elec = n_elec;
    P.ostride = z.ostride;
    P.n_orb = n_orb;
    P.n_so = z.n_so;
    P.npairs = z.npairs;
    P.n_irrep_used = max_irrep + 1;
    P.init_thr = initiator_threshold < 0 ? -1 : (int)((long long)initiator_threshold << fbits);
    P.seed = (unsigned)(o.seed & 0xFFFFFFFFull);
    P.tau = tau * unit_scale;  // spawning probabilities in units (exact: a power of two)
    P.period = o.shift_period;
    P.target = o.target_walkers > (LLONG_MAX >> fbits) ? LLONG_MAX : (o.target_walkers << fbits);
    P.c_shift = o.shift_damping / ((double)o.shift_period * tau);
    P.tau_f = (float)P.tau;
    P.tau_death = tau;
    P.tau_death_f = (float)tau;
    P.frac_bits = fbits;
    P.frac_scale = std::ldexp(1.0, -fbits);
    P.occ_units = (int)occ_units;
    P.h = at<double>(h, L.h);
    P.eri = at<double>(h, L.eri);
    P.eri_f = at<float>(h, L.eri_f);
    P.h_f = at<float>(h, L.h_f);
    P.wpair = at<double>(h, L.wpair);
    P.map1 = at<unsigned long long>(h, L.map1);
    P.cmask = at<unsigned long long>(h, L.cmask);
    P.unionm = at<unsigned long long>(h, L.unionm);
    P.irrep = at<unsigned char>(h, L.irrep);
    P.pairs = at<unsigned short>(h, L.pairs);
    P.recip = at<double>(h, L.recip);
    P.ref[0] = ref[0];
    P.ref[1] = ref[1];
    P.ref_occ = at<unsigned char>(h, L.ref_occ);
    for (int b = 0; b < 2; ++b) {
        P.det[b] = at<unsigned long long>(h, L.det[b]);
        P.hd[b] = at<double>(h, L.hd[b]);
        P.hdf[b] = at<float>(h, L.hdf[b]);
        P.pre[b] = at<unsigned long long>(h, L.pre[b]);
        P.occa[b] = at<unsigned char>(h, L.occa[b]);
        P.pop[b][0] = at<int>(h, L.pop[b][0]);
        P.pop[b][1] = at<int>(h, L.pop[b][1]);
    }
    P.cap = z.cap;
    P.idx = at<unsigned long long>(h, L.idx);
    P.idx_cap = z.idx_cap;
    P.idx_bits = log2_exact(z.idx_cap);
    P.idx_stride = z.W == 1 ? 2 : 4;
    P.mt = at<unsigned long long>(h, L.mt);
    P.mt_cap = z.mt_cap;
    P.mt_bits = log2_exact(z.mt_cap);
    P.merged = at<unsigned>(h, L.merged);
    P.heavy = h->ws + L.heavy;
    P.heavy_occ = at<unsigned char>(h, L.heavy_occ);
    P.heavy_base = at<unsigned>(h, L.heavy_base);
    P.heavy_att = at<unsigned>(h, L.heavy_att);
    P.heavy_cap = z.heavy_cap;
    P.rcpf = at<float>(h, L.rcpf);
    P.partial = at<double>(h, L.partial);
    P.tiles_cap = std::max<long long>((z.cap + fq::kTile - 1) / fq::kTile, kMaxGrid);
    P.hist = at<fciqmc_row>(h, L.hist);
    P.hist_cap = z.hist_cap;
    P.st = at<DevState>(h, L.state);
    P.n_eri = z.n_eri;
    P.n_parts = z.n_parts;
    P.part = z.part;
    P.outbox = z.n_parts > 1 ? at<unsigned long long>(h, L.outbox) : nullptr;
    P.ob_cap = z.ob_cap;

    int rc = FCIQMC_OK;
    cudaStream_t s = h->stream;
    // host-side tables: class masks, irreps, electron pairs, reference occupations
    std::vector<unsigned long long> cmask(fq::NCLASS * fq::MAXW, 0ull);
    std::vector<unsigned char> irr(fq::MAXSO, 0);
    for (int k = 0; k < z.n_so; ++k) {
        int g = orb_irrep ? orb_irrep[k >> 1] : 0;
        int cl = g * 2 + (k & 1);
        cmask[cl * fq::MAXW + (k >> 6)] |= 1ull << (k & 63);
    }
    for (int p = 0; p < n_orb; ++p) irr[p] = orb_irrep ? (unsigned char)orb_irrep[p] : 0;
    std::vector<unsigned long long> unionm(2 * 256 * fq::MAXW, 0ull);
    for (int sp = 0; sp < 2; ++sp)
        for (int set = 0; set < 256; ++set)
            for (int g = 0; g < 8; ++g)
                if ((set >> g) & 1)
                    for (int w = 0; w < fq::MAXW; ++w)
                        unionm[(sp * 256 + set) * fq::MAXW + w] |= cmask[(g * 2 + sp) * fq::MAXW + w];
    std::vector<unsigned short> pairs(std::max(z.npairs, 1), 0);
    for (int j = 1, k = 0; j < n_elec; ++j)
        for (int i = 0; i < j; ++i) pairs[k++] = (unsigned short)(i | (j << 8));
    std::vector<unsigned char> ref_occ(fq::MAXN, 0);
    {
        int n = 0;
        for (int k = 0; k < z.n_so; ++k)
            if ((ref[k >> 6] >> (k & 63)) & 1ull) {
                if (n < fq::MAXN) ref_occ[n] = (unsigned char)k;
                ++n;
            }
        if (n != n_elec) { delete h; return FCIQMC_ERR_INVALID_ARG; }
    }
    if (z.W == 1 && ref[1] != 0) { delete h; return FCIQMC_ERR_INVALID_ARG; }
    // permitted space; the reference must lie in it
    P.space = (int)(o.space_flags & 3u) | (o.frozen_occupied || o.frozen_empty ? 4 : 0);
    P.max_exc = o.max_excitation;
    P.max_sen = o.max_seniority;
    for (int w = 0; w < z.W; ++w) {
        P.froz_occ[w] = o.frozen_occupied ? o.frozen_occupied[w] : 0ull;
        P.froz_emp[w] = o.frozen_empty ? o.frozen_empty[w] : 0ull;
        if (((ref[w] & P.froz_emp[w]) | (~ref[w] & P.froz_occ[w])) != 0ull) { delete h; return FCIQMC_ERR_INVALID_ARG; }
    }
    if (((P.space & 1) && P.max_exc < 0) || ((P.space & 2) && P.max_sen < 0)) { delete h; return FCIQMC_ERR_INVALID_ARG; }
    if (o.hphf) {  // spin-coupled functions: M_s = 0 and a closed-shell reference
        if (ms2 != 0) { delete h; return FCIQMC_ERR_INVALID_ARG; }
        for (int w = 0; w < z.W; ++w)
            if (((ref[w] ^ (ref[w] >> 1)) & 0x5555555555555555ull) != 0ull) { delete h; return FCIQMC_ERR_INVALID_ARG; }
        P.hphf = 1;
    }
    if (P.space & 2) {
        int sen = 0;
        for (int w = 0; w < z.W; ++w) sen += __builtin_popcountll((ref[w] ^ (ref[w] >> 1)) & 0x5555555555555555ull);
        if (sen > P.max_sen) { delete h; return FCIQMC_ERR_INVALID_ARG; }
    }

#define FQ_TRY(call)                               \
    do {                                           \
        if ((call) != cudaSuccess) {               \
            rc = FCIQMC_ERR_CUDA;                  \
            goto fail;                             \
        }                                          \
    } while (0)
    {
        FQ_TRY(cudaMemsetAsync(P.st, 0, sizeof(DevState), s));
        FQ_TRY(cudaMemcpyAsync(const_cast<double *>(P.h), h1, sizeof(double) * n_orb * n_orb, cudaMemcpyHostToDevice, s));
        FQ_TRY(cudaMemcpyAsync(const_cast<double *>(P.eri), eri_s8, sizeof(double) * z.n_eri, cudaMemcpyHostToDevice, s));
        FQ_TRY(cudaMemcpyAsync(const_cast<unsigned long long *>(P.cmask), cmask.data(), sizeof(unsigned long long) * cmask.size(), cudaMemcpyHostToDevice, s));
        FQ_TRY(cudaMemcpyAsync(const_cast<unsigned long long *>(P.unionm), unionm.data(), sizeof(unsigned long long) * unionm.size(), cudaMemcpyHostToDevice, s));
        FQ_TRY(cudaMemcpyAsync(const_cast<unsigned char *>(P.irrep), irr.data(), irr.size(), cudaMemcpyHostToDevice, s));
        FQ_TRY(cudaMemcpyAsync(const_cast<unsigned short *>(P.pairs), pairs.data(), sizeof(unsigned short) * pairs.size(), cudaMemcpyHostToDevice, s));
        FQ_TRY(cudaMemcpyAsync(const_cast<unsigned char *>(P.ref_occ), ref_occ.data(), ref_occ.size(), cudaMemcpyHostToDevice, s));
        // nearest floats of h and of 1/L
        std::vector<float> hf32((size_t)n_orb * n_orb);
        for (size_t k = 0; k < hf32.size(); ++k) hf32[k] = (float)h1[k];
        FQ_TRY(cudaMemcpyAsync(const_cast<float *>(P.h_f), hf32.data(), sizeof(float) * hf32.size(), cudaMemcpyHostToDevice, s));
        std::vector<float> rcpf(2 * fq::MAXSO + 2, 0.f);
        for (int l = 1; l < 2 * fq::MAXSO + 2; ++l) rcpf[l] = (float)(1.0 / l);
        FQ_TRY(cudaMemcpyAsync(const_cast<float *>(P.rcpf), rcpf.data(), sizeof(float) * rcpf.size(), cudaMemcpyHostToDevice, s));
        long long *facts = at<long long>(h, L.facts);
        double *e0 = at<double>(h, L.e0);
        if (z.W == 1) {
            if (configure_kernels<1>(h) != FCIQMC_OK) { rc = FCIQMC_ERR_CUDA; goto fail; }
            fq::k_setup<1><<<1, 256, 0, s>>>(P, z.n_eri, const_cast<unsigned long long *>(P.map1), const_cast<double *>(P.wpair),
                                             const_cast<float *>(P.eri_f), const_cast<double *>(P.recip), facts, e0);
            fq::k_reference_energy<1><<<1, 256, h->smem_w, s>>>(P, e0);
        } else {
            if (configure_kernels<2>(h) != FCIQMC_OK) { rc = FCIQMC_ERR_CUDA; goto fail; }
            fq::k_setup<2><<<1, 256, 0, s>>>(P, z.n_eri, const_cast<unsigned long long *>(P.map1), const_cast<double *>(P.wpair),
                                             const_cast<float *>(P.eri_f), const_cast<double *>(P.recip), facts, e0);
            fq::k_reference_energy<2><<<1, 256, h->smem_w, s>>>(P, e0);
        }
        FQ_TRY(cudaGetLastError());
        long long hf[4];
        double E0;
        FQ_TRY(cudaMemcpyAsync(hf, facts, sizeof(hf), cudaMemcpyDeviceToHost, s));
        FQ_TRY(cudaMemcpyAsync(&E0, e0, sizeof(double), cudaMemcpyDeviceToHost, s));
        FQ_TRY(cudaStreamSynchronize(s));
        // P_double from the reference's allowed excitations (Sec. VI), realised exactly by the draw
        double pd = o.p_double > 0.0 ? o.p_double : (double)hf[1] / (double)(hf[0] + hf[1]);
        if (pd > 1.0) pd = 1.0;
        unsigned long long d53 = (unsigned long long)(pd * 0x1.0p53);
        double p_double = (double)d53 * 0x1.0p-53;
        double p_single = 1.0 - p_double;
        P.d53 = d53;
        P.E0 = E0;
        P.cs = P.tau / p_single;
        P.cd = P.tau / p_double;
        P.p_double_d = p_double;
        P.p_single_d = p_single;
        P.p_double_f = (float)p_double;
        P.p_single_f = (float)p_single;
        P.cdn_f = (float)(P.cd * (double)z.npairs);
        P.d53_d = (double)d53;
        P.d53_f = (float)d53;
        P.cs_f = (float)P.cs;
        P.srange_f = (float)(0x1.0p53 - (double)d53);
        // the float single-excitation element sums at most 2N - 1 terms, each rounded to float once
        // (relative 2^-24), with at most 2N - 2 float additions; the FP64 sum adds far less
        P.serr_f = (float)((2.0 * n_elec + 2.0) * 0x1.0p-24 * (1.0 + 0x1.0p-6));
        // the reference's double excitations with their p (plain runs), read by its spawning attempts
        P.ref_tab = 0;
        long long n_ref_exc = 0;
        if (z.ref_cap > 0 && z.npairs > 0) {
            unsigned *pinfo = at<unsigned>(h, L.ref_pinfo), *off2 = at<unsigned>(h, L.ref_off2);
            fq::RefExc *ex = at<fq::RefExc>(h, L.ref_exc);
            if (z.W == 1) fq::k_ref_table<1><<<1, 256, 0, s>>>(P, pinfo, off2, ex, z.ref_cap, facts + 2);
            else fq::k_ref_table<2><<<1, 256, 0, s>>>(P, pinfo, off2, ex, z.ref_cap, facts + 2);
            FQ_TRY(cudaGetLastError());
            FQ_TRY(cudaMemcpyAsync(&n_ref_exc, facts + 2, sizeof(long long), cudaMemcpyDeviceToHost, s));
            FQ_TRY(cudaStreamSynchronize(s));
            if (n_ref_exc >= 0) {
                P.ref_n = n_ref_exc;
                P.ref_pinfo = pinfo;
                P.ref_off2 = off2;
                P.ref_exc = ex;
                P.ref_tab = 1;
            } else {
                n_ref_exc = 0;
            }
        }
        // initial state: the reference with the initial population (in a partitioned run, on the reference's
        // own partition; the others start empty)
        bool owns_ref = true;
        if (z.n_parts > 1) {
            std::vector<unsigned long long> m1(z.n_so);
            FQ_TRY(cudaMemcpyAsync(m1.data(), P.map1, sizeof(unsigned long long) * z.n_so, cudaMemcpyDeviceToHost, s));
            FQ_TRY(cudaStreamSynchronize(s));
            owns_ref = (int)(host_fingerprint(ref, z.W, m1.data()) % (unsigned long long)z.n_parts) == z.part;
        }
        DevState st0;
        std::memset(&st0, 0, sizeof(st0));
        st0.iter = 0;
        st0.shift = o.initial_shift;
        st0.list_len = owns_ref ? 1 : 0;
        st0.claim = owns_ref ? 1 : 0;
        FQ_TRY(cudaMemcpyAsync(P.st, &st0, sizeof(st0), cudaMemcpyHostToDevice, s));
        FQ_TRY(cudaMemcpyAsync(P.det[0], ref, sizeof(uint64_t) * z.W, cudaMemcpyHostToDevice, s));
        int p0 = (int)((long long)o.initial_population << fbits);
        FQ_TRY(cudaMemcpyAsync(P.pop[0][0], &p0, sizeof(int), cudaMemcpyHostToDevice, s));
        if (z.W == 1) {
            launch_prepare<1>(h, 0, 1, 1);
            launch_index_rebuild<1>(h);
        } else {
            launch_prepare<2>(h, 0, 1, 1);
            launch_index_rebuild<2>(h);
        }
        FQ_TRY(cudaGetLastError());
        // empty spawn table: EMPTY keys, zero payloads
        fq::k_mt_clear<<<h->small_grid, 256, 0, s>>>(P, z.W);
        FQ_TRY(cudaGetLastError());
        DevState chk;
        if (read_state(h, chk) != FCIQMC_OK) { rc = FCIQMC_ERR_CUDA; goto fail; }
        if (chk.status != 0) { rc = chk.status; goto fail; }

        fciqmc_info &I = h->info;
        I.n_elec = n_elec;
        I.n_orb = n_orb;
        I.words = z.W;
        I.e0 = E0;
        I.e_core = e_core;
        I.p_double = p_double;
        I.d53 = d53;
        I.n_single_ref = hf[0];
        I.n_double_ref = hf[1];
        I.reference[0] = ref[0];
        I.reference[1] = ref[1];
        I.main_capacity = z.cap;
        I.index_capacity = z.idx_cap;
        I.spawn_capacity = z.mt_cap;
        I.history_capacity = z.hist_cap;
        I.workspace_bytes = L.total;
        I.reference_excitations = n_ref_exc;
        build_graph(h);
    }
#undef FQ_TRY
    *out = h;
    return FCIQMC_OK;
fail:
    delete h;
    return rc;
}

int fciqmc_step(fciqmc_handle *h, int32_t n_iterations) {
    if (!h || n_iterations < 0 || h->z.n_parts > 1) return FCIQMC_ERR_INVALID_ARG;
    NvtxRange range("fciqmc_step");
    for (int i = 0; i < n_iterations; ++i) {
        if (h->graph_ready) FQ_CUDA(cudaGraphLaunch(h->graph, h->stream));
        else enqueue(h, h->stream);
    }
    FQ_CUDA(cudaGetLastError());
    return FCIQMC_OK;
}

int fciqmc_profile(fciqmc_handle *h, int32_t n_iterations, double *kernel_ms) {
    if (!h || !kernel_ms || n_iterations < 0 || h->z.n_parts > 1) return FCIQMC_ERR_INVALID_ARG;
    cudaEvent_t ev[FCIQMC_N_KERNELS + 1];
    for (int k = 0; k <= FCIQMC_N_KERNELS; ++k) FQ_CUDA(cudaEventCreate(&ev[k]));
    const Params &P = h->P;
    cudaStream_t s = h->stream;
    static const char *const kNames[FCIQMC_N_KERNELS] = {"compact_copy", "index_clear", "index_fill", "compact_finish",
                                                         "sweep", "heavy", "annihilate", "finish"};
    for (int it = 0; it < n_iterations; ++it) {
        cudaEventRecord(ev[0], s);
        for (int k = 0; k < FCIQMC_N_KERNELS; ++k) {
            NvtxRange range(kNames[k]);
            if (h->z.W == 1) {
                switch (k) {
                    case 0: fq::k_compact_copy<1><<<h->small_grid, 256, 0, s>>>(P); break;
                    case 1:
                        fq::k_index_clear<<<h->small_grid, 256, 0, s>>>(P, 0);
                        fq::k_index_locate_old<1><<<h->small_grid, 256, 0, s>>>(P);
                        fq::k_index_clear_old<1><<<h->small_grid, 256, 0, s>>>(P);
                        break;
                    case 2: fq::k_index_fill<1><<<h->small_grid, 256, 0, s>>>(P, 0); break;
                    case 3: fq::k_compact_finish<<<1, 32, 0, s>>>(P); break;
                    case 4:
                        launch_sweep<1>(h, s);
                        fq::k_tile_sum<<<fq::kTileSums, 256, 0, s>>>(P);
                        break;
                    case 5: launch_heavy<1>(h, s); break;
                    case 6:
                        fq::k_annihilate<1><<<h->ann_grid, 256, 0, s>>>(P);
                        fq::k_new_diag<1><<<h->diag_grid, 256, h->smem_w, s>>>(P);
                        if (P.occ_units > 1) fq::k_round<1><<<h->small_grid, 256, 0, s>>>(P);
                        break;
                    default: fq::k_finish<<<1, 32, 0, s>>>(P); break;
                }
            } else {
                switch (k) {
                    case 0: fq::k_compact_copy<2><<<h->small_grid, 256, 0, s>>>(P); break;
                    case 1:
                        fq::k_index_clear<<<h->small_grid, 256, 0, s>>>(P, 0);
                        fq::k_index_locate_old<2><<<h->small_grid, 256, 0, s>>>(P);
                        fq::k_index_clear_old<2><<<h->small_grid, 256, 0, s>>>(P);
                        break;
                    case 2: fq::k_index_fill<2><<<h->small_grid, 256, 0, s>>>(P, 0); break;
                    case 3: fq::k_compact_finish<<<1, 32, 0, s>>>(P); break;
                    case 4:
                        launch_sweep<2>(h, s);
                        fq::k_tile_sum<<<fq::kTileSums, 256, 0, s>>>(P);
                        break;
                    case 5: launch_heavy<2>(h, s); break;
                    case 6:
                        fq::k_annihilate<2><<<h->ann_grid, 256, 0, s>>>(P);
                        fq::k_new_diag<2><<<h->diag_grid, 256, h->smem_w, s>>>(P);
                        if (P.occ_units > 1) fq::k_round<2><<<h->small_grid, 256, 0, s>>>(P);
                        break;
                    default: fq::k_finish<<<1, 32, 0, s>>>(P); break;
                }
            }
            cudaEventRecord(ev[k + 1], s);
        }
        FQ_CUDA(cudaGetLastError());
        FQ_CUDA(cudaEventSynchronize(ev[FCIQMC_N_KERNELS]));
        for (int k = 0; k < FCIQMC_N_KERNELS; ++k) {
            float ms = 0.f;
            FQ_CUDA(cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
            kernel_ms[k] += ms;
        }
    }
    for (int k = 0; k <= FCIQMC_N_KERNELS; ++k) cudaEventDestroy(ev[k]);
    return FCIQMC_OK;
}

int fciqmc_sync(fciqmc_handle *h) {
    if (!h) return FCIQMC_ERR_INVALID_ARG;
    int status = 0;
    FQ_CUDA(cudaMemcpyAsync(&status, &h->P.st->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    FQ_CUDA(cudaStreamSynchronize(h->stream));
    return status;
}

int fciqmc_estimators(fciqmc_handle *h, fciqmc_estimates *out) {
    if (!h || !out) return FCIQMC_ERR_INVALID_ARG;
    NvtxRange range("fciqmc_estimators");
    DevState *st = h->P.st;
    FQ_CUDA(cudaMemsetAsync(&st->est_nw, 0, sizeof(unsigned long long) * 2 + sizeof(long long), h->stream));
    const int blocks = std::min(h->small_grid, kMaxGrid);
    if (h->z.W == 1) fq::k_estimate<1><<<blocks, 256, 0, h->stream>>>(h->P);
    else fq::k_estimate<2><<<blocks, 256, 0, h->stream>>>(h->P);
    fq::k_estimate_finish<<<1, 32, 0, h->stream>>>(h->P, blocks);
    FQ_CUDA(cudaGetLastError());
    DevState s;
    int rc = read_state(h, s);
    if (rc != FCIQMC_OK) return rc;
    std::memset(out, 0, sizeof(*out));
    out->iteration = s.iter;
    out->shift = s.shift;
    out->e_ref = h->P.E0 + h->e_core;
    out->e_shift = out->e_ref + s.shift;
    out->proj_num = s.est_num;
    out->c0 = s.est_c0;
    out->n_walkers = (int64_t)s.est_nw;
    out->n_dets = (int64_t)s.est_nd;
    out->e_proj = s.est_c0 != 0 ? out->e_ref + s.est_num / (double)s.est_c0 : NAN;
    out->vary_shift = s.vary;
    out->status = s.status;
    out->list_slots = s.list_len;
    out->compactions = s.compactions;
    out->exact_spawns = (int64_t)s.exact_spawn;
    out->exact_deaths = (int64_t)s.exact_death;
    return s.status;
}

int fciqmc_history(fciqmc_handle *h, fciqmc_row *rows, int64_t max_rows, int64_t *n_rows) {
    if (!h || !n_rows || max_rows < 0 || (max_rows > 0 && !rows)) return FCIQMC_ERR_INVALID_ARG;
    DevState s;
    int rc = read_state(h, s);
    if (rc != FCIQMC_OK) return rc;
    const long long avail = std::min<long long>(s.hist_n, h->z.hist_cap);
    const long long n = std::min<long long>(avail, max_rows);
    for (long long k = 0; k < n; ++k) {
        long long idx = (s.hist_n - n + k) % h->z.hist_cap;
        FQ_CUDA(cudaMemcpyAsync(rows + k, h->P.hist + idx, sizeof(fciqmc_row), cudaMemcpyDeviceToHost, h->stream));
    }
    FQ_CUDA(cudaStreamSynchronize(h->stream));
    *n_rows = n;
    return FCIQMC_OK;
}

int fciqmc_n_dets(fciqmc_handle *h, int64_t *n_dets) {
    fciqmc_estimates e;
    int rc = fciqmc_estimators(h, &e);
    if (n_dets) *n_dets = e.n_dets;
    return rc == e.status ? FCIQMC_OK : rc;
}

int fciqmc_get_walkers(fciqmc_handle *h, uint64_t *dets, int32_t *pops, double *hdiag, int64_t cap, int64_t *n) {
    if (!h || !n || cap < 0 || (cap > 0 && (!dets || !pops))) return FCIQMC_ERR_INVALID_ARG;
    NvtxRange range("fciqmc_get_walkers");
    DevState *st = h->P.st;
    const Params &P = h->P;
    DevState s0;
    int rc = read_state(h, s0);
    if (rc != FCIQMC_OK) return rc;
    // the occupied entries gathered into the idle list buffer, then copied out (a gather writing page-locked
    // host memory itself was slower than the copy engines)
    const int other = s0.lb ^ 1;
    unsigned long long *od = P.det[other];
    int *op = P.pop[other][s0.pp];
    double *oh = P.hd[other];
    FQ_CUDA(cudaMemsetAsync(&st->new_len, 0, sizeof(unsigned long long), h->stream));
    if (h->z.W == 1) fq::k_gather<1><<<h->small_grid, 256, 0, h->stream>>>(P, od, op, oh, h->z.cap);
    else fq::k_gather<2><<<h->small_grid, 256, 0, h->stream>>>(P, od, op, oh, h->z.cap);
    FQ_CUDA(cudaGetLastError());
    unsigned long long cnt_u = 0;
    FQ_CUDA(cudaMemcpyAsync(&cnt_u, &st->new_len, sizeof(cnt_u), cudaMemcpyDeviceToHost, h->stream));
    FQ_CUDA(cudaStreamSynchronize(h->stream));
    const long long cnt = (long long)cnt_u;
    *n = cnt;
    if (cnt > cap) {
        FQ_CUDA(cudaMemsetAsync(&st->new_len, 0, sizeof(unsigned long long), h->stream));
        FQ_CUDA(cudaStreamSynchronize(h->stream));
        return FCIQMC_ERR_CAPACITY;
    }
    if (cnt > 0) {
        FQ_CUDA(cudaMemcpyAsync(dets, od, sizeof(uint64_t) * h->z.W * cnt, cudaMemcpyDeviceToHost, h->stream));
        FQ_CUDA(cudaMemcpyAsync(pops, op, sizeof(int32_t) * cnt, cudaMemcpyDeviceToHost, h->stream));
        if (hdiag) FQ_CUDA(cudaMemcpyAsync(hdiag, oh, sizeof(double) * cnt, cudaMemcpyDeviceToHost, h->stream));
    }
    FQ_CUDA(cudaMemsetAsync(&st->new_len, 0, sizeof(unsigned long long), h->stream));
    FQ_CUDA(cudaStreamSynchronize(h->stream));
    return FCIQMC_OK;
}

int fciqmc_set_walkers(fciqmc_handle *h, const uint64_t *dets, const int32_t *pops, const double *hdiag, int64_t n,
                       const fciqmc_state *stin) {
    if (!h || n < 0 || (n > 0 && (!dets || !pops))) return FCIQMC_ERR_INVALID_ARG;
    if (n > h->z.cap) return FCIQMC_ERR_CAPACITY;
    NvtxRange range("fciqmc_set_walkers");
    DevState cur;
    int rc = read_state(h, cur);
    if (rc != FCIQMC_OK) return rc;
    DevState st0;
    std::memset(&st0, 0, sizeof(st0));
    if (stin) {
        st0.iter = stin->iteration;
        st0.shift = stin->shift;
        st0.vary = stin->vary_shift;
        st0.n_since = stin->shift_counter;
        st0.nw_prev = stin->nw_last_update;
    } else {
        st0.iter = cur.iter;
        st0.shift = cur.shift;
        st0.vary = cur.vary;
        st0.n_since = cur.n_since;
        st0.nw_prev = cur.nw_prev;
    }
    st0.list_len = n;
    st0.claim = (unsigned long long)n;
    rc = h->z.W == 1 ? load_list<1>(h, cur, st0, dets, pops, hdiag, n) : load_list<2>(h, cur, st0, dets, pops, hdiag, n);
    if (rc != FCIQMC_OK) return rc;
    return fciqmc_sync(h);
}

int fciqmc_get_state(fciqmc_handle *h, fciqmc_state *out) {
    if (!h || !out) return FCIQMC_ERR_INVALID_ARG;
    DevState s;
    int rc = read_state(h, s);
    if (rc != FCIQMC_OK) return rc;
    out->iteration = s.iter;
    out->shift = s.shift;
    out->vary_shift = s.vary;
    out->shift_counter = s.n_since;
    out->nw_last_update = s.nw_prev;
    return FCIQMC_OK;
}

int fciqmc_get_info(const fciqmc_handle *h, fciqmc_info *info) {
    if (!h || !info) return FCIQMC_ERR_INVALID_ARG;
    *info = h->info;
    return FCIQMC_OK;
}

void fciqmc_destroy(fciqmc_handle *h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    if (h->aux) {
        cudaStreamSynchronize(h->aux);
        cudaStreamSynchronize(h->aux2);
        cudaStreamDestroy(h->aux);
        cudaStreamDestroy(h->aux2);
        cudaEventDestroy(h->ev_fork);
        cudaEventDestroy(h->ev_join);
        cudaEventDestroy(h->ev_join2);
        for (cudaEvent_t e : h->ev_chunk) cudaEventDestroy(e);
    }
    if (h->graph_ready) cudaGraphExecDestroy(h->graph);
    if (h->graph_tmpl) cudaGraphDestroy(h->graph_tmpl);
    delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------------------
// Throughput of the attempt's random numbers: one Philox4x32-10 block per (thread, k), keyed like a spawning
// attempt's block. The accumulated words are stored only if they hit a value the generator's output cannot
// be forced to (so the blocks are not optimised away and nothing is written in practice).
namespace {
__device__ unsigned long long g_rng_sink;

__global__ void __launch_bounds__(256) k_rng_throughput(long long per_thread) {
    const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long acc = 0;
    for (long long k = 0; k < per_thread; ++k) {
        unsigned long long w0, w1;
        fq::draw2((unsigned)k, 0u, 0x9E3779B97F4A7C15ull ^ tid, 1u, tid, w0, w1);
        acc ^= w0 + w1;
    }
    if (acc == 0x0123456789ABCDEFull) g_rng_sink = acc;
}
}  // namespace

extern "C" int fciqmc_rng_throughput(int64_t n_blocks, void *cuda_stream, double *blocks_per_s) {
    if (!blocks_per_s || n_blocks < 1) return FCIQMC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0, per_sm = 0;
    FQ_CUDA(cudaGetDevice(&dev));
    FQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    FQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rng_throughput, 256, 0));
    const long long threads = (long long)sms * std::max(per_sm, 1) * 256;
    const long long per_thread = std::max<long long>(1, (n_blocks + threads - 1) / threads);
    const unsigned grid = (unsigned)(threads / 256);
    cudaEvent_t e0, e1;
    FQ_CUDA(cudaEventCreate(&e0));
    FQ_CUDA(cudaEventCreate(&e1));
    k_rng_throughput<<<grid, 256, 0, s>>>(std::max<long long>(1, per_thread / 8));  // warm-up
    cudaEventRecord(e0, s);
    k_rng_throughput<<<grid, 256, 0, s>>>(per_thread);
    cudaEventRecord(e1, s);
    int rc = FCIQMC_OK;
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f))
        rc = FCIQMC_ERR_CUDA;
    else
        *blocks_per_s = (double)per_thread * (double)threads / (ms * 1e-3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

struct fciqmc_batch {
    std::vector<fciqmc_handle *> runs;
    std::vector<cudaEvent_t> run_events;
    cudaEvent_t done;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaStream_t last_stream;
};

extern "C" {

int fciqmc_batch_create(fciqmc_handle *const *runs, int n_runs, int32_t iterations_per_launch, fciqmc_batch **out) {
    if (!out || !runs || n_runs < 1 || iterations_per_launch < 1) return FCIQMC_ERR_INVALID_ARG;
    *out = nullptr;
    for (int r = 0; r < n_runs; ++r) {
        if (!runs[r] || !runs[r]->graph_ready || !runs[r]->graph_tmpl || runs[r]->z.n_parts > 1)
            return FCIQMC_ERR_INVALID_ARG;
        for (int q = 0; q < r; ++q)
            if (runs[q] == runs[r]) return FCIQMC_ERR_INVALID_ARG;
    }
    fciqmc_batch *b = new (std::nothrow) fciqmc_batch();
    if (!b) return FCIQMC_ERR_INVALID_ARG;
    b->runs.assign(runs, runs + n_runs);
    b->last_stream = nullptr;
    b->graph = nullptr;
    b->exec = nullptr;
    int rc = FCIQMC_OK;
    if (cudaGraphCreate(&b->graph, 0) != cudaSuccess) rc = FCIQMC_ERR_CUDA;
    for (int r = 0; r < n_runs && rc == FCIQMC_OK; ++r) {
        // each run: a chain of iterations_per_launch copies of its one-iteration graph
        cudaGraphNode_t prev = nullptr;
        for (int it = 0; it < iterations_per_launch; ++it) {
            cudaGraphNode_t node;
            if (cudaGraphAddChildGraphNode(&node, b->graph, prev ? &prev : nullptr, prev ? 1 : 0,
                                           runs[r]->graph_tmpl) != cudaSuccess) {
                rc = FCIQMC_ERR_CUDA;
                break;
            }
            prev = node;
        }
    }
    if (rc == FCIQMC_OK && cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) rc = FCIQMC_ERR_CUDA;
    if (rc == FCIQMC_OK) {
        b->run_events.resize(n_runs);
        for (int r = 0; r < n_runs && rc == FCIQMC_OK; ++r)
            if (cudaEventCreateWithFlags(&b->run_events[r], cudaEventDisableTiming) != cudaSuccess) rc = FCIQMC_ERR_CUDA;
        if (rc == FCIQMC_OK && cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess) rc = FCIQMC_ERR_CUDA;
    }
    if (rc != FCIQMC_OK) {
        cudaGetLastError();
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        delete b;
        return rc;
    }
    *out = b;
    return FCIQMC_OK;
}

int fciqmc_batch_step(fciqmc_batch *b, int32_t n_launches, void *cuda_stream) {
    if (!b || n_launches < 0) return FCIQMC_ERR_INVALID_ARG;
    NvtxRange range("fciqmc_batch_step");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    for (size_t r = 0; r < b->runs.size(); ++r) {
        FQ_CUDA(cudaEventRecord(b->run_events[r], b->runs[r]->stream));
        FQ_CUDA(cudaStreamWaitEvent(s, b->run_events[r], 0));
    }
    for (int k = 0; k < n_launches; ++k) FQ_CUDA(cudaGraphLaunch(b->exec, s));
    FQ_CUDA(cudaEventRecord(b->done, s));
    for (size_t r = 0; r < b->runs.size(); ++r) FQ_CUDA(cudaStreamWaitEvent(b->runs[r]->stream, b->done, 0));
    b->last_stream = s;
    return FCIQMC_OK;
}

void fciqmc_batch_destroy(fciqmc_batch *b) {
    if (!b) return;
    if (b->last_stream) cudaStreamSynchronize(b->last_stream);
    for (cudaEvent_t e : b->run_events) cudaEventDestroy(e);
    if (!b->run_events.empty()) cudaEventDestroy(b->done);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    delete b;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------------------
// Hash-partitioned runs (Sec. V A).
struct fciqmc_group {
    std::vector<fciqmc_handle *> parts;
    std::vector<cudaEvent_t> part_events;
    cudaEvent_t done;
    cudaStream_t stream;
    fq::PartLink *links;      // device
    fq::GroupDev *gdev;       // device
    fciqmc_row *ghist;        // device ring
    long long hist_cap;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

namespace {

struct GroupLayout {
    size_t gdev, links, hist, total;
};
GroupLayout group_layout(int n, long long hist_cap) {
    GroupLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    L.gdev = take(sizeof(fq::GroupDev));
    L.links = take(sizeof(fq::PartLink) * n);
    L.hist = take(sizeof(fciqmc_row) * hist_cap);
    L.total = off;
    return L;
}

template <int W>
void enqueue_group_iteration(fciqmc_group *g, cudaStream_t s) {
    const int n = (int)g->parts.size();
    for (fciqmc_handle *h : g->parts) {
        const Params &P = h->P;
        fq::k_compact_copy<W><<<h->small_grid, 256, 0, s>>>(P);
        fq::k_index_clear<<<h->small_grid, 256, 0, s>>>(P, 0);
        fq::k_index_locate_old<W><<<h->small_grid, 256, 0, s>>>(P);
        fq::k_index_clear_old<W><<<h->small_grid, 256, 0, s>>>(P);
        fq::k_index_fill<W><<<h->small_grid, 256, 0, s>>>(P, 0);
        fq::k_compact_finish<<<1, 32, 0, s>>>(P);
    }
    for (fciqmc_handle *h : g->parts) launch_spawning<W>(h, s);
    // the exchange: each partition merges the spawns the others routed to it
    for (fciqmc_handle *h : g->parts) fq::k_receive<W><<<h->ann_grid, 256, 0, s>>>(h->P, g->links);
    for (fciqmc_handle *h : g->parts) {
        fq::k_annihilate<W><<<h->ann_grid, 256, 0, s>>>(h->P);
        fq::k_new_diag<W><<<h->diag_grid, 256, h->smem_w, s>>>(h->P);
        if (h->P.occ_units > 1) fq::k_round<W><<<h->small_grid, 256, 0, s>>>(h->P);
    }
    const Params &P0 = g->parts[0]->P;
    fq::k_group_finish<<<1, 32, 0, s>>>(g->links, n, g->gdev, g->ghist, g->hist_cap, P0.target, P0.period, P0.c_shift);
}

bool same_run(const fciqmc_handle *a, const fciqmc_handle *b) {
    const fciqmc_options &x = a->opt, &y = b->opt;
    return a->z.W == b->z.W && a->P.n_elec == b->P.n_elec && a->P.n_orb == b->P.n_orb && a->tau == b->tau &&
           a->init_thr == b->init_thr && a->P.d53 == b->P.d53 && a->P.E0 == b->P.E0 && a->P.ref[0] == b->P.ref[0] &&
           a->P.ref[1] == b->P.ref[1] && x.shift_damping == y.shift_damping && x.shift_period == y.shift_period &&
           x.initial_shift == y.initial_shift && x.target_walkers == y.target_walkers &&
           (x.seed & 0xFFFFFFFFull) == (y.seed & 0xFFFFFFFFull) && a->P.space == b->P.space &&
           a->P.max_exc == b->P.max_exc && a->P.max_sen == b->P.max_sen && a->P.hphf == b->P.hphf &&
           a->P.froz_occ[0] == b->P.froz_occ[0] && a->P.froz_occ[1] == b->P.froz_occ[1] &&
           a->P.froz_emp[0] == b->P.froz_emp[0] && a->P.froz_emp[1] == b->P.froz_emp[1] &&
           a->z.n_parts == b->z.n_parts && a->P.frac_bits == b->P.frac_bits && a->P.occ_units == b->P.occ_units;
}

}  // namespace

extern "C" {

size_t fciqmc_group_workspace_bytes(int32_t n_partitions, int64_t history_capacity) {
    if (n_partitions < 2 || n_partitions > fq::MAXPARTS || history_capacity < 0) return 0;
    return group_layout(n_partitions, history_capacity > 0 ? history_capacity : (1LL << 16)).total;
}

int fciqmc_group_create(fciqmc_handle *const *parts, int32_t n_partitions, int64_t history_capacity, void *workspace,
                        size_t workspace_bytes, void *cuda_stream, fciqmc_group **out) {
    if (!out) return FCIQMC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!parts || n_partitions < 2 || n_partitions > fq::MAXPARTS || history_capacity < 0) return FCIQMC_ERR_INVALID_ARG;
    for (int r = 0; r < n_partitions; ++r) {
        const fciqmc_handle *h = parts[r];
        if (!h || h->z.n_parts != n_partitions || h->z.part != r || !same_run(h, parts[0])) return FCIQMC_ERR_INVALID_ARG;
    }
    const long long hist_cap = history_capacity > 0 ? history_capacity : (1LL << 16);
    const GroupLayout L = group_layout(n_partitions, hist_cap);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0 || workspace_bytes < L.total)
        return FCIQMC_ERR_WORKSPACE;
    fciqmc_group *g = new (std::nothrow) fciqmc_group();
    if (!g) return FCIQMC_ERR_INVALID_ARG;
    char *ws = static_cast<char *>(workspace);
    g->parts.assign(parts, parts + n_partitions);
    g->stream = static_cast<cudaStream_t>(cuda_stream);
    g->gdev = reinterpret_cast<fq::GroupDev *>(ws + L.gdev);
    g->links = reinterpret_cast<fq::PartLink *>(ws + L.links);
    g->ghist = reinterpret_cast<fciqmc_row *>(ws + L.hist);
    g->hist_cap = hist_cap;
    g->graph = nullptr;
    g->exec = nullptr;
    std::vector<fq::PartLink> links(n_partitions);
    for (int r = 0; r < n_partitions; ++r) {
        const Params &P = parts[r]->P;
        links[r].st = P.st;
        links[r].outbox = P.outbox;
        links[r].ob_cap = P.ob_cap;
        links[r].partial = P.partial + P.tiles_cap;
        links[r].hist = P.hist;
        links[r].hist_cap = P.hist_cap;
        links[r].cap = P.cap;
        links[r].heavy_warps = P.heavy_warps;
        links[r].sweep_blocks = P.sweep_blocks;
        links[r].frac_bits = P.frac_bits;
    }
    int rc = FCIQMC_OK;
    cudaStream_t cs = nullptr;
    do {
        // the partitions' own streams finish their work (creation, loads) before the group starts
        for (fciqmc_handle *h : g->parts)
            if (cudaStreamSynchronize(h->stream) != cudaSuccess) { rc = FCIQMC_ERR_CUDA; break; }
        if (rc != FCIQMC_OK) break;
        if (cudaMemsetAsync(g->gdev, 0, sizeof(fq::GroupDev), g->stream) != cudaSuccess ||
            cudaMemcpyAsync(g->links, links.data(), sizeof(fq::PartLink) * n_partitions, cudaMemcpyHostToDevice,
                            g->stream) != cudaSuccess ||
            cudaStreamSynchronize(g->stream) != cudaSuccess) { rc = FCIQMC_ERR_CUDA; break; }
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) { rc = FCIQMC_ERR_CUDA; break; }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            if (parts[0]->z.W == 1) enqueue_group_iteration<1>(g, cs);
            else enqueue_group_iteration<2>(g, cs);
            e = cudaStreamEndCapture(cs, &graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, graph, 0);
        if (e == cudaSuccess) g->graph = graph;
        else if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) { rc = FCIQMC_ERR_CUDA; break; }
        g->part_events.resize(n_partitions);
        for (int r = 0; r < n_partitions && rc == FCIQMC_OK; ++r)
            if (cudaEventCreateWithFlags(&g->part_events[r], cudaEventDisableTiming) != cudaSuccess) rc = FCIQMC_ERR_CUDA;
        if (rc == FCIQMC_OK && cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming) != cudaSuccess)
            rc = FCIQMC_ERR_CUDA;
    } while (false);
    if (cs) cudaStreamDestroy(cs);
    if (rc != FCIQMC_OK) {
        cudaGetLastError();
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return rc;
    }
    *out = g;
    return FCIQMC_OK;
}

int fciqmc_group_step(fciqmc_group *g, int32_t n_iterations) {
    if (!g || n_iterations < 0) return FCIQMC_ERR_INVALID_ARG;
    NvtxRange range("fciqmc_group_step");
    for (size_t r = 0; r < g->parts.size(); ++r) {
        FQ_CUDA(cudaEventRecord(g->part_events[r], g->parts[r]->stream));
        FQ_CUDA(cudaStreamWaitEvent(g->stream, g->part_events[r], 0));
    }
    for (int k = 0; k < n_iterations; ++k) FQ_CUDA(cudaGraphLaunch(g->exec, g->stream));
    FQ_CUDA(cudaEventRecord(g->done, g->stream));
    for (fciqmc_handle *h : g->parts) FQ_CUDA(cudaStreamWaitEvent(h->stream, g->done, 0));
    return FCIQMC_OK;
}

int fciqmc_group_sync(fciqmc_group *g) {
    if (!g) return FCIQMC_ERR_INVALID_ARG;
    fq::GroupDev d;
    FQ_CUDA(cudaMemcpyAsync(&d, g->gdev, sizeof(d), cudaMemcpyDeviceToHost, g->stream));
    FQ_CUDA(cudaStreamSynchronize(g->stream));
    return d.status;
}

int fciqmc_group_history(fciqmc_group *g, fciqmc_row *rows, int64_t max_rows, int64_t *n_rows) {
    if (!g || !n_rows || max_rows < 0 || (max_rows > 0 && !rows)) return FCIQMC_ERR_INVALID_ARG;
    fq::GroupDev d;
    FQ_CUDA(cudaMemcpyAsync(&d, g->gdev, sizeof(d), cudaMemcpyDeviceToHost, g->stream));
    FQ_CUDA(cudaStreamSynchronize(g->stream));
    const long long avail = std::min<long long>(d.hist_n, g->hist_cap);
    const long long n = std::min<long long>(avail, max_rows);
    for (long long k = 0; k < n; ++k) {
        const long long idx = (d.hist_n - n + k) % g->hist_cap;
        FQ_CUDA(cudaMemcpyAsync(rows + k, g->ghist + idx, sizeof(fciqmc_row), cudaMemcpyDeviceToHost, g->stream));
    }
    FQ_CUDA(cudaStreamSynchronize(g->stream));
    *n_rows = n;
    return FCIQMC_OK;
}

void fciqmc_group_destroy(fciqmc_group *g) {
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    for (cudaEvent_t e : g->part_events) cudaEventDestroy(e);
    if (!g->part_events.empty()) cudaEventDestroy(g->done);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

int fciqmc_owner(int n_orb, const uint64_t *dets, int64_t n, int32_t n_partitions, int32_t *owner) {
    if (n_orb < 1 || n_orb > 64 || n < 0 || n_partitions < 1 || (n > 0 && (!dets || !owner))) return FCIQMC_ERR_INVALID_ARG;
    const int W = (2 * n_orb + 63) / 64;
    unsigned long long map1[fq::MAXSO];
    for (int k = 0; k < 2 * n_orb; ++k) map1[k] = host_map1(k);
    for (int k = 2 * n_orb; k < fq::MAXSO; ++k) map1[k] = 0ull;
    for (int64_t x = 0; x < n; ++x)
        owner[x] = (int32_t)(host_fingerprint(dets + x * W, W, map1) % (unsigned long long)n_partitions);
    return FCIQMC_OK;
}

}  // extern "C"
