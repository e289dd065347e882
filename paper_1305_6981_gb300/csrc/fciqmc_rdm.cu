// Energy functional E(h, V; c) = c^T H c / c^T c over a fixed determinant list, and its gradient with
// respect to the one- and two-electron integrals (the 1- and 2-RDMs of c divided by c^T c).
//
// Pairs of determinants that H connects (differing in at most two spin orbitals) are found without a
// sort: every determinant I emits, for each pair {x, y} of its occupied spin orbitals, the key
// I - {x, y}. Two distinct determinants share a key exactly when they differ by a double excitation
// (one shared key, their hole sets removed) or a single excitation (one shared key per common
// electron; the pair is kept only in the bucket of the lowest common electron). Keys are grouped in
// an open-addressing table (128-bit compare-and-swap for two-word determinants), buckets with two or
// more members get contiguous member segments (sorted by determinant index, so sums are
// deterministic), and each thread then evaluates one candidate pair.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>

#include "fciqmc.h"
#include "fciqmc_device.cuh"

namespace {

using fq::Params;

constexpr int kThreads = 256;
constexpr int kMaxGrid = 4096;
constexpr unsigned long long kSaltKey = 0x2545F4914F6CDD1Dull;

struct RdmLayout {
    size_t dets, c, keys, counts, cursor, moff, poff, members, bsum, partial, state, gh, ge, npair_tab, wpair, scan_tmp;
    size_t total;
};

struct RdmState {
    unsigned long long n_buckets;
    unsigned long long n_members;  // members of buckets with two or more entries
    unsigned long long n_pairs;    // candidate pairs
    unsigned long long n_single, n_double;
    double norm;
    int status;
    int pad;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }
long long next_pow2(long long x) {
    long long p = 1;
    while (p < x) p <<= 1;
    return p;
}
int log2i(long long x) {
    int b = 0;
    while ((1LL << b) < x) ++b;
    return b;
}

struct Dims {
    int n_elec, n_orb, W, npairs;
    long long n, n_keys, kcap, n_eri;
};

bool dims_of(int n_elec, int n_orb, long long n, Dims &d) {
    if (n_orb < 1 || n_orb > 64 || n_elec < 2 || n_elec > fq::MAXN || n_elec >= 2 * n_orb || n < 1 || n > (1LL << 30))
        return false;
    d.n_elec = n_elec;
    d.n_orb = n_orb;
    d.W = (2 * n_orb + 63) / 64;
    d.npairs = n_elec * (n_elec - 1) / 2;
    d.n = n;
    d.n_keys = n * d.npairs;
    d.kcap = next_pow2(std::max<long long>(2 * d.n_keys, 1 << 12));
    long long np = (long long)n_orb * (n_orb + 1) / 2;
    d.n_eri = np * (np + 1) / 2;
    return d.n_keys < (1LL << 31);
}

RdmLayout layout_of(const Dims &d) {
    RdmLayout L{};
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off = align256(off + b);
        return o;
    };
    const int stride = d.W == 1 ? 2 : 4;
    L.dets = take(sizeof(unsigned long long) * d.W * d.n);
    L.c = take(sizeof(double) * d.n);
    L.keys = take(sizeof(unsigned long long) * stride * d.kcap);
    L.counts = take(sizeof(unsigned) * d.n_keys);
    L.cursor = take(sizeof(unsigned) * d.n_keys);
    L.moff = take(sizeof(unsigned long long) * (d.n_keys + 1));
    L.poff = take(sizeof(unsigned long long) * (d.n_keys + 1));
    L.members = take(sizeof(unsigned long long) * d.n_keys);
    L.bsum = take(sizeof(unsigned long long) * 2 * (kMaxGrid + 1));
    L.partial = take(sizeof(double) * 4 * kMaxGrid);
    L.state = take(sizeof(RdmState));
    L.gh = take(sizeof(double) * d.n_orb * d.n_orb);
    L.ge = take(sizeof(double) * d.n_eri);
    L.npair_tab = take(sizeof(double) * 2 * fq::MAXSO * fq::MAXSO);
    L.wpair = take(sizeof(double) * 2 * d.n_orb * d.n_orb);
    L.scan_tmp = take(sizeof(unsigned long long) * 4);
    L.total = off;
    return L;
}

// ------------------------------------------------------------------------------------ device helpers
template <int W>
__device__ __forceinline__ void load_det(const unsigned long long *dets, long long i, unsigned long long (&d)[W]) {
#pragma unroll
    for (int w = 0; w < W; ++w) d[w] = dets[i * W + w];
}

// x-th occupied spin orbital (ascending) of d
template <int W>
__device__ __forceinline__ int nth_occ(const unsigned long long (&d)[W], int x) {
    return fq::select_bit<W>(d, x);
}

// member word: determinant index (bits 0..31), removed orbitals x (32..39) and y (40..47)
__device__ __forceinline__ unsigned long long pack_member(unsigned I, int x, int y) {
    return (unsigned long long)I | ((unsigned long long)x << 32) | ((unsigned long long)y << 40);
}

template <int W>
__device__ __forceinline__ long long key_lookup(const unsigned long long *tab, long long kcap, int kbits,
                                                const unsigned long long (&key)[W]) {
    constexpr int S = fq::Stride<W>::v;
    unsigned long long h = fq::table_hash<W>(key, kSaltKey) >> (64 - kbits);
    for (long long probe = 0; probe < kcap; ++probe) {
        const unsigned long long *e = tab + h * S;
        bool match = true, empty = true;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            match = match && (e[w] == key[w]);
            empty = empty && (e[w] == fq::EMPTY);
        }
        if (match) return (long long)h;
        if (empty) return -1;
        h = (h + 1ull) & ((unsigned long long)kcap - 1ull);
    }
    return -1;
}

// ------------------------------------------------------------------------------------ construction kernels
// Empty key table: EMPTY key words, zero payloads.
__global__ void k_key_init(unsigned long long *tab, long long kcap, int W) {
    const int S = W == 1 ? 2 : 4;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < kcap; e += (long long)gridDim.x * blockDim.x) {
        for (int w = 0; w < W; ++w) tab[e * S + w] = fq::EMPTY;
        tab[e * S + W] = 0ull;
    }
}

// Key table entries: key words, then (bucket id << 32) + number of determinants with that key.
template <int W>
__global__ void k_keys(const unsigned long long *dets, long long n, int n_elec, unsigned long long *tab, long long kcap,
                       int kbits, RdmState *st) {
    constexpr int S = fq::Stride<W>::v;
    const int npairs = n_elec * (n_elec - 1) / 2;
    const long long total = n * npairs;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const long long I = t / npairs;
        int k = (int)(t - I * npairs);
        int y = 1;
        while ((y + 1) * y / 2 <= k) ++y;
        const int x = k - y * (y - 1) / 2;
        unsigned long long d[W];
        load_det<W>(dets, I, d);
        unsigned long long key[W];
#pragma unroll
        for (int w = 0; w < W; ++w) key[w] = d[w];
        fq::flip<W>(key, nth_occ<W>(d, x));
        fq::flip<W>(key, nth_occ<W>(d, y));
        unsigned long long h = fq::table_hash<W>(key, kSaltKey) >> (64 - kbits);
        bool done = false;
        for (long long probe = 0; probe < kcap && !done; ++probe) {
            unsigned long long *e = tab + h * S;
            int r = fq::probe_key<W>(e, key);
            if (r == 1) {
                atomicAdd(e + W, 1ull);
                done = true;
            } else if (r == 2) {
                bool claimed;
                if (fq::claim_key<W>(e, key, claimed)) {
                    unsigned long long add = 1ull;
                    if (claimed) add += atomicAdd(&st->n_buckets, 1ull) << 32;
                    atomicAdd(e + W, add);
                    done = true;
                }
            }
            if (!done) h = (h + 1ull) & ((unsigned long long)kcap - 1ull);
        }
        if (!done) atomicCAS(&st->status, 0, FCIQMC_ERR_CAPACITY);
    }
}

template <int W>
__global__ void k_counts(const unsigned long long *tab, long long kcap, unsigned *counts) {
    constexpr int S = fq::Stride<W>::v;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < kcap; e += (long long)gridDim.x * blockDim.x) {
        bool empty = true;
#pragma unroll
        for (int w = 0; w < W; ++w) empty = empty && (tab[e * S + w] == fq::EMPTY);
        if (empty) continue;
        const unsigned long long v = tab[e * S + W];
        counts[v >> 32] = (unsigned)(v & 0xFFFFFFFFull);
    }
}

// Exclusive scans over buckets b < nb of m_b = count if count >= 2 else 0 (member offsets) and of
// p_b = C(m_b, 2) (pair offsets), in three passes: per-block sums, a scan of the block sums, then
// per-element offsets. Both outputs have nb + 1 entries.
__global__ void k_scan_blocks(const unsigned *counts, long long nb, long long per_block, unsigned long long *bsum) {
    __shared__ unsigned long long s_m[kThreads], s_p[kThreads];
    const long long lo = (long long)blockIdx.x * per_block, hi = min(lo + per_block, nb);
    unsigned long long m = 0, p = 0;
    for (long long b = lo + threadIdx.x; b < hi; b += blockDim.x) {
        const unsigned long long c = counts[b] >= 2 ? counts[b] : 0;
        m += c;
        p += c * (c - 1) / 2;
    }
    s_m[threadIdx.x] = m;
    s_p[threadIdx.x] = p;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s_m[threadIdx.x] += s_m[threadIdx.x + o];
            s_p[threadIdx.x] += s_p[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        bsum[2 * blockIdx.x] = s_m[0];
        bsum[2 * blockIdx.x + 1] = s_p[0];
    }
}

__global__ void k_scan_top(unsigned long long *bsum, int nblocks, RdmState *st) {
    if (threadIdx.x != 0) return;
    unsigned long long m = 0, p = 0;
    for (int b = 0; b < nblocks; ++b) {
        const unsigned long long bm = bsum[2 * b], bp = bsum[2 * b + 1];
        bsum[2 * b] = m;
        bsum[2 * b + 1] = p;
        m += bm;
        p += bp;
    }
    st->n_members = m;
    st->n_pairs = p;
}

__global__ void k_scan_out(const unsigned *counts, long long nb, long long per_block, const unsigned long long *bsum,
                           unsigned long long *moff, unsigned long long *poff, const RdmState *st) {
    if (threadIdx.x != 0) return;  // one thread per block walks its range in order
    const long long lo = (long long)blockIdx.x * per_block, hi = min(lo + per_block, nb);
    unsigned long long m = bsum[2 * blockIdx.x], p = bsum[2 * blockIdx.x + 1];
    for (long long b = lo; b < hi; ++b) {
        moff[b] = m;
        poff[b] = p;
        const unsigned long long c = counts[b] >= 2 ? counts[b] : 0;
        m += c;
        p += c * (c - 1) / 2;
    }
    if (hi == nb && lo < hi) {
        moff[nb] = st->n_members;
        poff[nb] = st->n_pairs;
    }
}

template <int W>
__global__ void k_members(const unsigned long long *dets, long long n, int n_elec, const unsigned long long *tab,
                          long long kcap, int kbits, const unsigned *counts, unsigned *cursor,
                          const unsigned long long *moff, unsigned long long *members) {
    constexpr int S = fq::Stride<W>::v;
    const int npairs = n_elec * (n_elec - 1) / 2;
    const long long total = n * npairs;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const long long I = t / npairs;
        int k = (int)(t - I * npairs);
        int y = 1;
        while ((y + 1) * y / 2 <= k) ++y;
        const int x = k - y * (y - 1) / 2;
        unsigned long long d[W];
        load_det<W>(dets, I, d);
        unsigned long long key[W];
#pragma unroll
        for (int w = 0; w < W; ++w) key[w] = d[w];
        const int ox = nth_occ<W>(d, x), oy = nth_occ<W>(d, y);
        fq::flip<W>(key, ox);
        fq::flip<W>(key, oy);
        const long long e = key_lookup<W>(tab, kcap, kbits, key);
        if (e < 0) continue;
        const unsigned long long b = tab[e * S + W] >> 32;
        if (counts[b] < 2) continue;
        const unsigned pos = atomicAdd(&cursor[b], 1u);
        members[moff[b] + pos] = pack_member((unsigned)I, ox, oy);
    }
}

// Sorts each bucket's members by determinant index (insertion sort; buckets are small).
__global__ void k_sort_members(long long nb, const unsigned *counts, const unsigned long long *moff,
                               unsigned long long *members) {
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (long long)gridDim.x * blockDim.x) {
        const unsigned c = counts[b];
        if (c < 2) continue;
        unsigned long long *m = members + moff[b];
        for (unsigned i = 1; i < c; ++i) {
            const unsigned long long v = m[i];
            unsigned j = i;
            while (j > 0 && (m[j - 1] & 0xFFFFFFFFull) > (v & 0xFFFFFFFFull)) {
                m[j] = m[j - 1];
                --j;
            }
            m[j] = v;
        }
    }
}

__global__ void k_norm(const double *c, long long n, double *partial) {
    __shared__ double s[kThreads];
    double v = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v = __dadd_rn(v, __dmul_rn(c[i], c[i]));
    s[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kThreads; ++k) t = __dadd_rn(t, s[k]);
        partial[blockIdx.x] = t;
    }
}

__global__ void k_sum_partials(const double *partial, int n, double *out) {
    if (threadIdx.x != 0) return;
    double t = 0.0;
    for (int b = 0; b < n; ++b) t = __dadd_rn(t, partial[b]);
    *out = t;
}

// ------------------------------------------------------------------------------------ compensated sums
// Sum and running error of a sequence of FP64 additions (Knuth's TwoSum per addition, Neumaier's
// compensated summation): the result is the rounded exact sum up to a few ulp whatever the number of
// terms, so finite differences of E are not swamped by accumulated rounding.
struct CSum {
    double s, c;
};
__device__ __forceinline__ void csum_add(CSum &a, double x) {
    const double t = __dadd_rn(a.s, x);
    const double bb = __dsub_rn(t, a.s);
    const double err = __dadd_rn(__dsub_rn(a.s, __dsub_rn(t, bb)), __dsub_rn(x, bb));
    a.s = t;
    a.c = __dadd_rn(a.c, err);
}
__device__ __forceinline__ void csum_merge(CSum &a, const CSum &b) {
    csum_add(a, b.s);
    a.c = __dadd_rn(a.c, b.c);
}

// Fixed-tree merges (the same order in every run): lanes pairwise by shuffles, then the warps' results.
__device__ __forceinline__ CSum warp_csum(CSum a) {
    for (int o = 16; o > 0; o >>= 1) {
        const CSum b{__shfl_down_sync(0xFFFFFFFFu, a.s, o), __shfl_down_sync(0xFFFFFFFFu, a.c, o)};
        csum_merge(a, b);
    }
    return a;  // lane 0 holds the warp's sum
}
// Block sum of every thread's acc into out[0] (sum) and out[1] (running error); s: kThreads / 32 slots.
__device__ __forceinline__ void block_csum(CSum acc, CSum *s, double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    acc = warp_csum(acc);
    if (lane == 0) s[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        CSum x = lane < kThreads / 32 ? s[lane] : CSum{0.0, 0.0};
        x = warp_csum(x);
        if (lane == 0) {
            out[0] = x.s;
            out[1] = x.c;
        }
    }
}

// ------------------------------------------------------------------------------------ pairs
struct PairInfo {
    long long I, J;
    int kind;            // 0: skip, 1: single i -> a (from I), 2: double (i<j) -> (a<b) (from I)
    int i, j, a, b;
};

// Last bucket b in [lo, hi] with poff[b] <= x.
__device__ __forceinline__ long long bucket_search(const unsigned long long *poff, unsigned long long x, long long lo,
                                                   long long hi) {
    while (lo < hi) {
        const long long mid = (lo + hi + 1) >> 1;
        if (poff[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Bucket of pair k * 2^kPairIndexShift for every k (the coarse index of the bucket search).
constexpr int kPairIndexShift = 8;
__global__ void k_pair_index(const unsigned long long *poff, long long nb, const RdmState *st, unsigned *idx) {
    const unsigned long long nk = (st->n_pairs >> kPairIndexShift) + 1;
    for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < nk;
         k += (unsigned long long)gridDim.x * blockDim.x)
        idx[k] = (unsigned)bucket_search(poff, k << kPairIndexShift, 0, nb - 1);
}

// Candidate pair t: bucket by binary search over pair offsets, narrowed by the coarse index when there is
// one, (u < v) by inverse triangular index (the float square root is a first guess that the integer
// steps correct).
template <int W>
__device__ __forceinline__ PairInfo pair_of(unsigned long long t, unsigned long long np, long long nb,
                                            const unsigned long long *poff, const unsigned *pidx,
                                            const unsigned long long *moff, const unsigned long long *members,
                                            const unsigned long long *dets, unsigned long long (&dI)[W],
                                            unsigned long long (&dJ)[W]) {
    PairInfo P{};
    long long b_lo = 0, b_hi = nb - 1;
    if (pidx) {
        const unsigned long long k = t >> kPairIndexShift;
        b_lo = pidx[k];
        if (((k + 1) << kPairIndexShift) < np) b_hi = pidx[k + 1];
    }
    const long long lo = bucket_search(poff, t, b_lo, b_hi);
    const unsigned long long l = t - poff[lo];
    unsigned long long v = (unsigned long long)((1.0f + sqrtf(1.0f + 8.0f * (float)l)) * 0.5f);
    while (v > 1 && v * (v - 1) / 2 > l) --v;
    while ((v + 1) * v / 2 <= l) ++v;
    const unsigned long long u = l - v * (v - 1) / 2;
    const unsigned long long mu = members[moff[lo] + u], mv = members[moff[lo] + v];
    P.I = (long long)(mu & 0xFFFFFFFFull);
    P.J = (long long)(mv & 0xFFFFFFFFull);
    load_det<W>(dets, P.I, dI);
    load_det<W>(dets, P.J, dJ);
    int nd = 0;
    unsigned long long holes[W], parts[W], common[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        holes[w] = dI[w] & ~dJ[w];
        parts[w] = dJ[w] & ~dI[w];
        common[w] = dI[w] & dJ[w];
        nd += __popcll(holes[w]);
    }
    if (nd == 2) {
        P.kind = 2;
        P.i = fq::select_bit<W>(holes, 0);
        P.j = fq::select_bit<W>(holes, 1);
        P.a = fq::select_bit<W>(parts, 0);
        P.b = fq::select_bit<W>(parts, 1);
    } else if (nd == 1) {
        // single: kept only in the bucket whose shared removed orbital is the lowest common electron
        const int xu = (int)((mu >> 32) & 0xFF), yu = (int)((mu >> 40) & 0xFF);
        const int hole = fq::select_bit<W>(holes, 0);
        const int shared = xu == hole ? yu : xu;
        if (shared == fq::select_bit<W>(common, 0)) {
            P.kind = 1;
            P.i = hole;
            P.a = fq::select_bit<W>(parts, 0);
        }
    }
    return P;
}

template <int W>
__device__ __forceinline__ double single_h(const Params &P, const unsigned long long (&d)[W], int i, int a) {
    const int I = i >> 1, A = a >> 1;
    double v = P.h[I * P.n_orb + A];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        unsigned long long m = d[w];
        while (m) {
            const int j = 64 * w + __ffsll((long long)m) - 1;
            m &= m - 1;
            if (j == i) continue;
            const int J = j >> 1;
            v = __dadd_rn(v, fq::eri_d(P, I, A, J, J));
            if ((j & 1) == (i & 1)) v = __dsub_rn(v, fq::eri_d(P, I, J, J, A));
        }
    }
    return (fq::count_between<W>(d, i, a) & 1) ? -v : v;
}

// Single-excitation pairs are a few percent of the candidates, and each costs an O(N) FP64 loop: a warp
// queues its lanes' singles (pair I, J and orbitals i -> a) and evaluates them 32 at a time, so the loop
// never runs for one lane while 31 wait. The queue order is fixed by the warp's schedule.
struct SingleQueue {
    unsigned long long ij[64];  // I | J << 32
    unsigned short ia[64];      // i | a << 8
    unsigned n;
};
__device__ __forceinline__ void queue_single(SingleQueue &q, bool single, const PairInfo &p) {
    const unsigned m = __ballot_sync(0xFFFFFFFFu, single);
    const int lane = threadIdx.x & 31;
    const unsigned n = q.n;
    if (single) {
        const unsigned k = n + __popc(m & ((1u << lane) - 1u));
        q.ij[k] = (unsigned long long)p.I | ((unsigned long long)p.J << 32);
        q.ia[k] = (unsigned short)(p.i | (p.a << 8));
    }
    __syncwarp();
    if (lane == 0) q.n = n + __popc(m);
    __syncwarp();
}
// Takes up to 32 queued singles (all when `all`, else only once 32 are queued): lane k gets entry k
// (take = false for the others); the rest moves to the front.
__device__ __forceinline__ bool pop_single(SingleQueue &q, bool all, long long &I, long long &J, int &i, int &a) {
    const int lane = threadIdx.x & 31;
    const unsigned n = q.n;
    if (n == 0 || (!all && n < 32)) return false;
    const unsigned take = min(n, 32u);
    bool got = false;
    if ((unsigned)lane < take) {
        I = (long long)(q.ij[lane] & 0xFFFFFFFFull);
        J = (long long)(q.ij[lane] >> 32);
        i = q.ia[lane] & 0xFF;
        a = q.ia[lane] >> 8;
        got = true;
    }
    __syncwarp();
    const unsigned rest = n - take;
    if ((unsigned)lane < rest) {
        q.ij[lane] = q.ij[take + lane];
        q.ia[lane] = q.ia[take + lane];
    }
    __syncwarp();
    if (lane == 0) q.n = rest;
    __syncwarp();
    return got;
}

// 2 c_I c_J H_IJ summed over candidate pairs, per block in a fixed order (compensated).
template <int W>
__global__ void __launch_bounds__(kThreads) k_pair_energy(Params P, const unsigned long long *dets, const double *c,
                                                          long long nb, const unsigned long long *poff,
                                                          const unsigned *pidx, const unsigned long long *moff,
                                                          const unsigned long long *members, const RdmState *st,
                                                          double *partial) {
    __shared__ CSum s[kThreads / 32];
    __shared__ SingleQueue s_q[kThreads / 32];
    SingleQueue &sq = s_q[threadIdx.x >> 5];
    if ((threadIdx.x & 31) == 0) sq.n = 0;
    __syncwarp();
    const unsigned long long np = st->n_pairs;
    CSum acc{0.0, 0.0};
    auto add_single = [&](bool all) {
        long long I = 0, J = 0;
        int i = 0, a = 0;
        if (pop_single(sq, all, I, J, i, a)) {
            unsigned long long dI[W];
            load_det<W>(dets, I, dI);
            csum_add(acc, __dmul_rn(__dmul_rn(2.0, __dmul_rn(c[I], c[J])), single_h<W>(P, dI, i, a)));
        }
    };
    // warp-uniform loop: lane k takes pair base + k
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < np;
         base += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long t = base + (threadIdx.x & 31);
        PairInfo q{};
        if (t < np) {
            unsigned long long dI[W], dJ[W];
            q = pair_of<W>(t, np, nb, poff, pidx, moff, members, dets, dI, dJ);
            if (q.kind == 2)
                csum_add(acc, __dmul_rn(__dmul_rn(2.0, __dmul_rn(c[q.I], c[q.J])),
                                        fq::hij_double<W>(P, dI, q.i, q.j, q.a, q.b)));
        }
        queue_single(sq, q.kind == 1, q);
        add_single(false);
    }
    add_single(true);  // fewer than 32 remain
    block_csum(acc, s, partial + 2 * blockIdx.x);
}

// c_I^2 H_II per block (pair-term table in shared memory, compensated).
template <int W>
__global__ void __launch_bounds__(kThreads) k_diag_energy(Params P, const unsigned long long *dets, const double *c,
                                                          long long n, double *partial) {
    extern __shared__ double s_w[];
    __shared__ CSum s[kThreads / 32];
    const int M = P.n_orb;
    for (int k = threadIdx.x; k < 2 * M * M; k += blockDim.x) s_w[k] = P.wpair[k];
    for (int k = threadIdx.x; k < M; k += blockDim.x) s_w[2 * M * M + k] = P.h[k * M + k];
    __syncthreads();
    CSum acc{0.0, 0.0};
    for (long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x; I < n; I += (long long)gridDim.x * blockDim.x) {
        unsigned long long d[W];
        load_det<W>(dets, I, d);
        csum_add(acc, __dmul_rn(__dmul_rn(c[I], c[I]), fq::hdiag<W>(P, d, s_w, s_w + 2 * M * M)));
    }
    block_csum(acc, s, partial + 2 * blockIdx.x);
}

// One warp: lane k merges the block partials k, k + 32, ... (diagonal, then pairs), then a fixed tree.
__global__ void k_energy_finish(const double *pp, int npp, const double *pd, int npd, const RdmState *st, double *e) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32) return;
    CSum tot{0.0, 0.0};
    for (int b = lane; b < npd; b += 32) csum_merge(tot, CSum{pd[2 * b], pd[2 * b + 1]});
    for (int b = lane; b < npp; b += 32) csum_merge(tot, CSum{pp[2 * b], pp[2 * b + 1]});
    tot = warp_csum(tot);
    if (lane == 0) *e = __ddiv_rn(__dadd_rn(tot.s, tot.c), st->norm);
}

__global__ void k_pair_wpair(Params P, double *wpair) {
    const int M = P.n_orb;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M * M; k += gridDim.x * blockDim.x) {
        const int p = k / M, q = k % M;
        const double j = fq::eri_d(P, p, p, q, q);
        wpair[k] = j;
        wpair[M * M + k] = __dsub_rn(j, fq::eri_d(P, p, q, q, p));
    }
}

// Gradient contributions of the connected pairs (atomics into the unscaled RDM arrays).
template <int W>
__global__ void __launch_bounds__(kThreads) k_pair_grad(int n_orb, const unsigned long long *dets, const double *c,
                                                        long long nb, const unsigned long long *poff,
                                                        const unsigned *pidx, const unsigned long long *moff,
                                                        const unsigned long long *members, RdmState *st, double *gh,
                                                        double *ge) {
    __shared__ SingleQueue s_q[kThreads / 32];
    SingleQueue &sq = s_q[threadIdx.x >> 5];
    if ((threadIdx.x & 31) == 0) sq.n = 0;
    __syncwarp();
    const unsigned long long np = st->n_pairs;
    unsigned long long ns = 0, ndb = 0;
    auto add_single = [&](bool all) {
        long long Id = 0, Jd = 0;
        int i = 0, a = 0;
        if (pop_single(sq, all, Id, Jd, i, a)) {
            ++ns;
            unsigned long long dI[W];
            load_det<W>(dets, Id, dI);
            const double cc = c[Id] * c[Jd];
            const double sg = (fq::count_between<W>(dI, i, a) & 1) ? -cc : cc;
            const int I = i >> 1, A = a >> 1;
            atomicAdd(&gh[I * n_orb + A], sg);
            atomicAdd(&gh[A * n_orb + I], sg);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                unsigned long long m = dI[w];
                while (m) {
                    const int j = 64 * w + __ffsll((long long)m) - 1;
                    m &= m - 1;
                    if (j == i) continue;
                    const int J = j >> 1;
                    atomicAdd(&ge[fq::eidx(I, A, J, J)], 2.0 * sg);
                    if ((j & 1) == (i & 1)) atomicAdd(&ge[fq::eidx(I, J, J, A)], -2.0 * sg);
                }
            }
        }
    };
    // warp-uniform loop: lane k takes pair base + k
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < np;
         base += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long t = base + (threadIdx.x & 31);
        PairInfo q{};
        unsigned long long dI[W], dJ[W];
        if (t < np) q = pair_of<W>(t, np, nb, poff, pidx, moff, members, dets, dI, dJ);
        queue_single(sq, q.kind == 1, q);
        add_single(false);
        if (q.kind == 2) {
            const double cc = c[q.I] * c[q.J];
            ++ndb;
            const double sg = fq::double_parity<W>(dI, q.i, q.j, q.a, q.b) ? -cc : cc;
            if ((q.i & 1) == (q.a & 1) && (q.j & 1) == (q.b & 1))
                atomicAdd(&ge[fq::eidx(q.i >> 1, q.a >> 1, q.j >> 1, q.b >> 1)], 2.0 * sg);
            if ((q.i & 1) == (q.b & 1) && (q.j & 1) == (q.a & 1))
                atomicAdd(&ge[fq::eidx(q.i >> 1, q.b >> 1, q.j >> 1, q.a >> 1)], -2.0 * sg);
        }
    }
    add_single(true);  // fewer than 32 remain
    if (ns) atomicAdd(&st->n_single, ns);
    if (ndb) atomicAdd(&st->n_double, ndb);
}

// Diagonal contributions: occupation-pair sums O_pq = sum_I c_I^2 n_p n_q over spin orbitals p <= q
// (p == q gives sum_I c_I^2 n_p). Each thread walks the occupied pairs of its determinants and adds c_I^2
// into a block copy of the triangle in shared memory (index q (q + 1) / 2 + p), flushed once per block.
// O is stored at p * n_so + q.
template <int W>
__global__ void __launch_bounds__(kThreads) k_diag_grad(int n_so, const unsigned long long *dets, const double *c,
                                                        long long n, double *occ_pair) {
    extern __shared__ double s_o[];
    const int nent = n_so * (n_so + 1) / 2;
    for (int k = threadIdx.x; k < nent; k += blockDim.x) s_o[k] = 0.0;
    __syncthreads();
    for (long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x; I < n; I += (long long)gridDim.x * blockDim.x) {
        unsigned long long d[W];
        load_det<W>(dets, I, d);
        const double c2 = c[I] * c[I];
#pragma unroll
        for (int wq = 0; wq < W; ++wq) {
            unsigned long long mq = d[wq];
            while (mq) {
                const int q = 64 * wq + __ffsll((long long)mq) - 1;
                mq &= mq - 1;
                const int row = q * (q + 1) / 2;
#pragma unroll
                for (int wp = 0; wp <= wq; ++wp) {
                    unsigned long long mp = d[wp];
                    if (wp == wq) mp &= (q & 63) == 63 ? ~0ull : ((2ull << (q & 63)) - 1ull);  // p <= q
                    while (mp) {
                        const int p = 64 * wp + __ffsll((long long)mp) - 1;
                        mp &= mp - 1;
                        atomicAdd(&s_o[row + p], c2);
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nent; k += blockDim.x) {
        const double v = s_o[k];
        if (v != 0.0) {
            int q = 0;
            while ((q + 1) * (q + 2) / 2 <= k) ++q;
            atomicAdd(&occ_pair[(k - q * (q + 1) / 2) * n_so + q], v);
        }
    }
}

// Maps the occupation-pair sums onto h and the packed ERIs and scales the whole RDM by 1 / c^T c.
__global__ void k_diag_finish(int n_orb, const double *occ_pair, double *gh, double *ge, const RdmState *st) {
    if (blockIdx.x != 0) return;
    const int n_so = 2 * n_orb;
    for (int e = threadIdx.x; e < n_so * n_so; e += blockDim.x) {
        const int p = e / n_so, q = e % n_so;
        if (q < p) continue;
        const double v = occ_pair[e];
        if (v == 0.0) continue;
        const int P = p >> 1, Q = q >> 1;
        if (p == q) {
            atomicAdd(&gh[P * n_orb + P], v);
        } else {
            atomicAdd(&ge[fq::eidx(P, P, Q, Q)], v);
            if ((p & 1) == (q & 1)) atomicAdd(&ge[fq::eidx(P, Q, Q, P)], -v);
        }
    }
}

__global__ void k_scale_out(const double *gh, const double *ge, long long n_h, long long n_e, const double *scale,
                            const RdmState *st, double *out_h, double *out_e) {
    const double f = __ddiv_rn(*scale, st->norm);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n_h + n_e; k += (long long)gridDim.x * blockDim.x) {
        if (k < n_h) out_h[k] = __dmul_rn(gh[k], f);
        else out_e[k - n_h] = __dmul_rn(ge[k - n_h], f);
    }
}

}  // namespace

struct fciqmc_rdm {
    Dims d;
    RdmLayout L;
    char *ws;
    cudaStream_t s;
    int grid;
    int sms;
    long long nb;  // buckets (host copy after construction)
    bool pidx_ok;  // the coarse index of the bucket search is built (in the member-cursor buffer)
    RdmState host;
    bool rdm_ready;  // unscaled density matrices computed
};

namespace {
template <typename T>
T *ptr(fciqmc_rdm *r, size_t off) {
    return reinterpret_cast<T *>(r->ws + off);
}
Params params_for(fciqmc_rdm *r, const double *h, const double *eri) {
    Params P{};
    P.n_elec = r->d.n_elec;
    P.n_orb = r->d.n_orb;
    P.n_so = 2 * r->d.n_orb;
    P.h = h;
    P.eri = eri;
    P.wpair = ptr<double>(r, r->L.wpair);
    return P;
}

template <int W>
int construct(fciqmc_rdm *r) {
    const Dims &d = r->d;
    cudaStream_t s = r->s;
    const int stride = W == 1 ? 2 : 4;
    const int g = r->grid;
    RdmState *st = ptr<RdmState>(r, r->L.state);
    unsigned long long *tab = ptr<unsigned long long>(r, r->L.keys);
    (void)stride;
    k_key_init<<<g, kThreads, 0, s>>>(tab, d.kcap, W);
    cudaMemsetAsync(st, 0, sizeof(RdmState), s);
    k_keys<W><<<g, kThreads, 0, s>>>(ptr<unsigned long long>(r, r->L.dets), d.n, d.n_elec, tab, d.kcap, log2i(d.kcap), st);
    if (cudaMemcpyAsync(&r->host, st, sizeof(RdmState), cudaMemcpyDeviceToHost, s) != cudaSuccess) return FCIQMC_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FCIQMC_ERR_CUDA;
    if (r->host.status) return r->host.status;
    const long long nb = (long long)r->host.n_buckets;
    r->nb = nb;
    unsigned *counts = ptr<unsigned>(r, r->L.counts);
    k_counts<W><<<g, kThreads, 0, s>>>(tab, d.kcap, counts);
    const int nblk = (int)std::min<long long>(kMaxGrid, std::max<long long>(1, (nb + 4095) / 4096));
    const long long per_block = (nb + nblk - 1) / nblk;
    unsigned long long *bsum = ptr<unsigned long long>(r, r->L.bsum);
    unsigned long long *moff = ptr<unsigned long long>(r, r->L.moff), *poff = ptr<unsigned long long>(r, r->L.poff);
    k_scan_blocks<<<nblk, kThreads, 0, s>>>(counts, nb, per_block, bsum);
    k_scan_top<<<1, 32, 0, s>>>(bsum, nblk, st);
    k_scan_out<<<nblk, 32, 0, s>>>(counts, nb, per_block, bsum, moff, poff, st);
    unsigned *cursor = ptr<unsigned>(r, r->L.cursor);
    cudaMemsetAsync(cursor, 0, sizeof(unsigned) * nb, s);
    unsigned long long *members = ptr<unsigned long long>(r, r->L.members);
    k_members<W><<<g, kThreads, 0, s>>>(ptr<unsigned long long>(r, r->L.dets), d.n, d.n_elec, tab, d.kcap, log2i(d.kcap),
                                        counts, cursor, moff, members);
    k_sort_members<<<g, kThreads, 0, s>>>(nb, counts, moff, members);
    double *partial = ptr<double>(r, r->L.partial);
    k_norm<<<g, kThreads, 0, s>>>(ptr<double>(r, r->L.c), d.n, partial);
    k_sum_partials<<<1, 32, 0, s>>>(partial, g, &st->norm);
    if (cudaGetLastError() != cudaSuccess) return FCIQMC_ERR_CUDA;
    if (cudaMemcpyAsync(&r->host, st, sizeof(RdmState), cudaMemcpyDeviceToHost, s) != cudaSuccess) return FCIQMC_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FCIQMC_ERR_CUDA;
    // coarse index of the bucket search, in the member cursors (no longer needed)
    r->pidx_ok = r->host.status == 0 && nb > 0 &&
                 (long long)(r->host.n_pairs >> kPairIndexShift) + 2 <= d.n_keys;
    if (r->pidx_ok) {
        k_pair_index<<<g, kThreads, 0, s>>>(poff, nb, st, cursor);
        if (cudaGetLastError() != cudaSuccess) return FCIQMC_ERR_CUDA;
    }
    return r->host.status;
}

template <int W>
void launch_energy(fciqmc_rdm *r, const Params &P, double *e) {
    const Dims &d = r->d;
    cudaStream_t s = r->s;
    const int g = r->grid;
    RdmState *st = ptr<RdmState>(r, r->L.state);
    double *partial = ptr<double>(r, r->L.partial);
    const int gd = std::min(g, kMaxGrid / 2);
    const size_t smem = sizeof(double) * (2 * d.n_orb * d.n_orb + d.n_orb);
    k_pair_wpair<<<8, kThreads, 0, s>>>(P, const_cast<double *>(P.wpair));
    k_diag_energy<W><<<gd, kThreads, smem, s>>>(P, ptr<unsigned long long>(r, r->L.dets), ptr<double>(r, r->L.c), d.n,
                                                partial);
    const unsigned *pidx = r->pidx_ok ? ptr<unsigned>(r, r->L.cursor) : nullptr;
    k_pair_energy<W><<<gd, kThreads, 0, s>>>(P, ptr<unsigned long long>(r, r->L.dets), ptr<double>(r, r->L.c), r->nb,
                                             ptr<unsigned long long>(r, r->L.poff), pidx,
                                             ptr<unsigned long long>(r, r->L.moff),
                                             ptr<unsigned long long>(r, r->L.members), st, partial + 2 * gd);
    k_energy_finish<<<1, 32, 0, s>>>(partial + 2 * gd, gd, partial, gd, st, e);
}

template <int W>
void launch_rdm(fciqmc_rdm *r) {
    const Dims &d = r->d;
    cudaStream_t s = r->s;
    const int g = r->grid;
    RdmState *st = ptr<RdmState>(r, r->L.state);
    double *gh = ptr<double>(r, r->L.gh), *ge = ptr<double>(r, r->L.ge);
    double *occ_pair = ptr<double>(r, r->L.npair_tab);
    cudaMemsetAsync(gh, 0, sizeof(double) * d.n_orb * d.n_orb, s);
    cudaMemsetAsync(ge, 0, sizeof(double) * d.n_eri, s);
    cudaMemsetAsync(occ_pair, 0, sizeof(double) * 4 * d.n_orb * d.n_orb, s);
    const unsigned *pidx = r->pidx_ok ? ptr<unsigned>(r, r->L.cursor) : nullptr;
    k_pair_grad<W><<<g, kThreads, 0, s>>>(d.n_orb, ptr<unsigned long long>(r, r->L.dets), ptr<double>(r, r->L.c), r->nb,
                                          ptr<unsigned long long>(r, r->L.poff), pidx, ptr<unsigned long long>(r, r->L.moff),
                                          ptr<unsigned long long>(r, r->L.members), st, gh, ge);
    k_diag_grad<W><<<std::min<long long>(g, (d.n + kThreads - 1) / kThreads), kThreads,
                     sizeof(double) * d.n_orb * (2 * d.n_orb + 1), s>>>(
        2 * d.n_orb, ptr<unsigned long long>(r, r->L.dets), ptr<double>(r, r->L.c), d.n, occ_pair);
    k_diag_finish<<<1, kThreads, 0, s>>>(d.n_orb, occ_pair, gh, ge, st);
}
}  // namespace

extern "C" {

size_t fciqmc_rdm_workspace_bytes(int n_elec, int n_orb, int64_t n_dets) {
    Dims d;
    if (!dims_of(n_elec, n_orb, n_dets, d)) return 0;
    return layout_of(d).total;
}

int fciqmc_rdm_create(int n_elec, int n_orb, const uint64_t *dets_dev, const double *c_dev, int64_t n_dets,
                      void *workspace, size_t workspace_bytes, void *cuda_stream, fciqmc_rdm **out) {
    if (!out) return FCIQMC_ERR_INVALID_ARG;
    *out = nullptr;
    Dims d;
    if (!dims_of(n_elec, n_orb, n_dets, d)) return FCIQMC_ERR_UNSUPPORTED;
    if (!dets_dev || !c_dev) return FCIQMC_ERR_INVALID_ARG;
    RdmLayout L = layout_of(d);
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % 256) != 0 || workspace_bytes < L.total)
        return FCIQMC_ERR_WORKSPACE;
    fciqmc_rdm *r = new (std::nothrow) fciqmc_rdm();
    if (!r) return FCIQMC_ERR_INVALID_ARG;
    r->d = d;
    r->L = L;
    r->ws = static_cast<char *>(workspace);
    r->s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&r->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete r;
        return FCIQMC_ERR_CUDA;
    }
    r->grid = std::min(kMaxGrid, r->sms * 8);
    const size_t smem = sizeof(double) * (2 * d.n_orb * d.n_orb + d.n_orb);
    const size_t smem_o = sizeof(double) * d.n_orb * (2 * d.n_orb + 1);  // occupation-pair triangle
    if (cudaFuncSetAttribute(k_diag_energy<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_diag_energy<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_diag_grad<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_o) != cudaSuccess ||
        cudaFuncSetAttribute(k_diag_grad<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_o) != cudaSuccess) {
        delete r;
        return FCIQMC_ERR_CUDA;
    }
    if (cudaMemcpyAsync(ptr<unsigned long long>(r, L.dets), dets_dev, sizeof(uint64_t) * d.W * d.n, cudaMemcpyDeviceToDevice, r->s) != cudaSuccess ||
        cudaMemcpyAsync(ptr<double>(r, L.c), c_dev, sizeof(double) * d.n, cudaMemcpyDeviceToDevice, r->s) != cudaSuccess) {
        delete r;
        return FCIQMC_ERR_CUDA;
    }
    const int rc = d.W == 1 ? construct<1>(r) : construct<2>(r);
    if (rc != FCIQMC_OK) {
        delete r;
        return rc;
    }
    *out = r;
    return FCIQMC_OK;
}

int fciqmc_rdm_energy(fciqmc_rdm *r, const double *h_dev, const double *eri_dev, double *e_dev) {
    if (!r || !h_dev || !eri_dev || !e_dev) return FCIQMC_ERR_INVALID_ARG;
    Params P = params_for(r, h_dev, eri_dev);
    if (r->d.W == 1) launch_energy<1>(r, P, e_dev);
    else launch_energy<2>(r, P, e_dev);
    return cudaGetLastError() == cudaSuccess ? FCIQMC_OK : FCIQMC_ERR_CUDA;
}

int fciqmc_rdm_gradient(fciqmc_rdm *r, const double *scale_dev, double *grad_h_dev, double *grad_eri_dev) {
    if (!r || !scale_dev || !grad_h_dev || !grad_eri_dev) return FCIQMC_ERR_INVALID_ARG;
    RdmState *st = ptr<RdmState>(r, r->L.state);
    if (!r->rdm_ready) {
        if (r->d.W == 1) launch_rdm<1>(r);
        else launch_rdm<2>(r);
        r->rdm_ready = true;
    }
    const long long nh = (long long)r->d.n_orb * r->d.n_orb;
    k_scale_out<<<std::min(r->grid, 1024), kThreads, 0, r->s>>>(ptr<double>(r, r->L.gh), ptr<double>(r, r->L.ge), nh,
                                                                r->d.n_eri, scale_dev, st, grad_h_dev, grad_eri_dev);
    return cudaGetLastError() == cudaSuccess ? FCIQMC_OK : FCIQMC_ERR_CUDA;
}

int fciqmc_rdm_info(fciqmc_rdm *r, int64_t *counts) {
    if (!r || !counts) return FCIQMC_ERR_INVALID_ARG;
    RdmState h;
    if (cudaMemcpyAsync(&h, ptr<RdmState>(r, r->L.state), sizeof(RdmState), cudaMemcpyDeviceToHost, r->s) != cudaSuccess ||
        cudaStreamSynchronize(r->s) != cudaSuccess)
        return FCIQMC_ERR_CUDA;
    counts[0] = (int64_t)h.n_buckets;
    counts[1] = (int64_t)h.n_members;
    counts[2] = (int64_t)h.n_pairs;
    counts[3] = (int64_t)h.n_single;
    counts[4] = (int64_t)h.n_double;
    return h.status;
}

void fciqmc_rdm_destroy(fciqmc_rdm *r) {
    if (!r) return;
    cudaStreamSynchronize(r->s);
    delete r;
}

}  // extern "C"
