// Kernels of one FCIQMC iteration (sm_103a).
//
// Per iteration, on the caller's stream (or as one CUDA graph):
//   [compaction, only when flagged]  k_compact_copy -> k_index_clear -> k_index_fill -> k_compact_finish
//   k_sweep        estimators of the incoming list, death/cloning (Eq. 4), and every spawning
//                  attempt (Eq. 3, Sec. VI) of determinants with |C_i| <= kHeavy, merged on the fly
//                  into the spawn table (sum of signed amounts, initiator flags counted)
//   k_heavy        the attempts of determinants with |C_i| > kHeavy, split into chunks
//   k_annihilate   the merged spawns against the post-death main list through the hash index, with
//                  the initiator filter and H_ii on insertion (Sec. V B)
//   k_finish       deterministic reduction of the projected-energy numerator, history row, shift
//                  update, population parity flip
#pragma once

#include "fciqmc_device.cuh"

namespace fq {

constexpr int kTile = 256;          // determinants per sweep tile = threads per sweep block
constexpr int kTileSums = 32;       // range sums of the per-tile numerators (blocks of k_tile_sum)
#ifndef FQ_SWEEP_MIN_BLOCKS
#define FQ_SWEEP_MIN_BLOCKS 5          // resident sweep blocks per SM the register budget is sized for
#endif
#ifndef FQ_HEAVY_THRESHOLD
#define FQ_HEAVY_THRESHOLD 256
#endif
constexpr int kHeavy = FQ_HEAVY_THRESHOLD;  // |C_i| above this: attempts go to the chunked heavy path
constexpr int kHeavyShort = 32;  // the threshold for lists with fewer tiles than a quarter of the sweep's blocks
#ifndef FQ_HEAVY_CHUNK
#define FQ_HEAVY_CHUNK 512
#endif
constexpr int kChunk = FQ_HEAVY_CHUNK;  // smallest heavy chunk in attempts (one warp task)
#ifndef FQ_CHUNK_GROWTH
#define FQ_CHUNK_GROWTH 4
#endif
constexpr int kChunkGrowth = FQ_CHUNK_GROWTH;  // chunks grow to at most kChunkGrowth kChunk with the walkers
constexpr int kChunksPerWarp = 12;       // the chunk size keeps at least this many chunks per k_heavy warp
#ifndef FQ_CHUNK_BATCH
#define FQ_CHUNK_BATCH 32
#endif
constexpr int kChunkBatch = FQ_CHUNK_BATCH;  // most consecutive chunks a warp takes at a time (guided, see k_heavy)
constexpr unsigned long long kSaltMerge = 0x5851F42D4C957F2Dull;
constexpr unsigned long long kSaltIndex = 0x14057B7EF767814Full;
constexpr unsigned long long kFlagUnit = 1ull << 40;  // merge payload: (#initiator spawns << 40) + amount

enum { C_ATTEMPTS = 0, C_NULLS, C_EVENTS, C_SPAWNED, C_DEATH, C_CLONE, C_MERGED, C_ABORTED, C_INSERTED, C_HEAVY };

// Per-determinant data used by every attempt from it, kept in shared memory (its occupied list separately, so
// the sweep's tile of views takes only the bytes the run's electron count needs).
template <int W>
struct DetView {
    unsigned long long d[W];
    unsigned long long fp;
    unsigned long long okm;     // bit x: electron x has at least one symmetry-allowed single
    unsigned long long cb8[2];  // byte g of cb8[s]: unoccupied spin orbitals of class (irrep g, spin s)
    unsigned char cnt[NCLASS];  // the same counts by class index 2 g + s
    int c;
    unsigned char nok;          // electrons with at least one symmetry-allowed single (N - delta_s)
    unsigned char flag;         // initiator
    unsigned char isref;        // the reference determinant
};  // the occupied spin orbitals (ascending) are kept beside the view, n_elec bytes

// Occupied spin orbitals of d in ascending order (for the exact FP64 paths, which run rarely); returns their
// number.
template <int W>
__device__ __forceinline__ int decode_occ(const unsigned long long (&d)[W], unsigned char *occ) {
    int n = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        unsigned long long m = d[w];
        while (m && n < MAXN) {
            occ[n++] = (unsigned char)(64 * w + __ffsll((long long)m) - 1);
            m &= m - 1;
        }
    }
    return n;
}

// Bytes of one occupied list in the sweep's tile (the electron count rounded up to 4).
__host__ __device__ constexpr int occ_stride(int n_elec) { return (n_elec + 3) & ~3; }

struct Tables {
    unsigned long long map1[MAXSO];
    unsigned long long mask[NCLASS * MAXW];
    // spin orbitals of spin s in the irreps of a 4-bit set, for irreps 0..3 (half 0) and 4..7 (half 1):
    // uh[((s * 2 + half) * 16 + set) * MAXW + w]
    unsigned long long uh[2 * 2 * 16 * MAXW];
    unsigned char irrep[MAXSO / 2];
    unsigned short pairs[MAXPAIRS];
};

__device__ __forceinline__ void load_tables(const Params &P, Tables &T) {
    for (int k = threadIdx.x; k < P.n_so; k += blockDim.x) T.map1[k] = P.map1[k];
    for (int k = threadIdx.x; k < NCLASS * MAXW; k += blockDim.x) T.mask[k] = P.cmask[k];
    for (int k = threadIdx.x; k < 2 * 2 * 16 * MAXW; k += blockDim.x) {
        const int w = k % MAXW, set = (k / MAXW) % 16, half = (k / (16 * MAXW)) % 2, s = k / (32 * MAXW);
        unsigned long long u = 0ull;
        for (int b = 0; b < 4; ++b)
            if ((set >> b) & 1) u |= P.cmask[((4 * half + b) * 2 + s) * MAXW + w];
        T.uh[k] = u;
    }
    for (int k = threadIdx.x; k < P.n_orb; k += blockDim.x) T.irrep[k] = P.irrep[k];
    for (int k = threadIdx.x; k < P.npairs; k += blockDim.x) T.pairs[k] = P.pairs[k];
}

// ---------------------------------------------------------------------------- float bounds
// Decisions n = floor(p) + [u < p - floor(p)] are first tried with float bounds lo <= p_d <= hi of the
// value p_d the exact FP64 expression would give; only undecided cases evaluate p_d. Bounds use
// round-to-nearest float arithmetic with explicit margins: an input rounded to the nearest float f
// lies within |f| 2^-24 of it, every float operation adds at most 2^-24 relative, and the final
// factors (1 +- 2^-18) cover those roundings and the FP64 rounding of p_d with room to spare.
constexpr float kUp = 1.0f + 0x1p-18f;
constexpr float kDown = 1.0f - 0x1p-18f;

// n = floor(x) + [u < x - floor(x)] for u = (r >> 11) 2^-53 (death draw) and an FP64 value x >= 0 known
// only to lie in [lo, hi]: n, or -1 when the bounds do not decide it. hi - m and max(lo, 0) - m are
// exact (Sterbenz), and u_lo <= u < u_lo + 2^-24 exactly.
__device__ __forceinline__ int decide_death(float lo, float hi, unsigned long long r) {
    if (!(hi < 0x1p22f)) return -1;
    const float l = fmaxf(lo, 0.f);
    const float m = floorf(l);
    if (floorf(hi) != m) return -1;
    const float u_lo = (float)(unsigned)(r >> 40) * 0x1p-24f;
    if (u_lo >= hi - m) return (int)m;
    if (u_lo + 0x1p-24f <= l - m) return (int)m + 1;
    return -1;
}

__device__ __forceinline__ double unit53(unsigned long long r) { return __dmul_rn(__ull2double_rn(r >> 11), 0x1p-53); }

// ---------------------------------------------------------------------------- spawn merge table
template <int W>
__device__ __forceinline__ bool merge_insert(const Params &P, const unsigned long long (&key)[W], unsigned long long val,
                                             unsigned &pos) {
    constexpr int S = Stride<W>::v;
    const unsigned long long mask = (unsigned long long)P.mt_cap - 1ull;
    unsigned long long h = table_hash<W>(key, kSaltMerge) >> (64 - P.mt_bits);
    for (long long probe = 0; probe < P.mt_cap; ++probe) {
        unsigned long long *e = P.mt + h * S;
        int r = probe_key<W>(e, key);
        if (r == 1) {
            atomicAdd(e + W, val);
            return false;
        }
        if (r == 2) {
            bool claimed;
            if (claim_key<W>(e, key, claimed)) {
                atomicAdd(e + W, val);
                if (claimed) pos = (unsigned)h;
                return claimed;
            }
        }
        h = (h + 1ull) & mask;
    }
    set_status(P.st, FCIQMC_ERR_CAPACITY);
    return false;
}

// ---------------------------------------------------------------------------- per-determinant preparation
// Nonzero bytes of a byte-packed count word as an 8-bit set.
__device__ __forceinline__ unsigned nonzero_bytes(unsigned long long x) {
    const unsigned long long bits = ((x + 0x7F7F7F7F7F7F7F7Full) & 0x8080808080808080ull) >> 7;
    return (unsigned)((bits * 0x0102040810204080ull) >> 56);
}

// What the spawning kernels need of a determinant beyond its bits, a function of the bits alone (stored per
// slot when the determinant enters the list): PRE_FP the fingerprint of Algorithm 1, PRE_OKM bit x set when
// electron x has an allowed single (its class keeps an unoccupied orbital), PRE_CB0 / PRE_CB1 byte g the
// unoccupied spin orbitals of class (irrep g, spin 0 / 1); beside them the occupied list.
enum { PRE_FP = 0, PRE_OKM, PRE_CB0, PRE_CB1, PRE_WORDS };

// Class counts first (population counts against the class masks); then one pass over the occupied spin
// orbitals in ascending order gives the occupied list, the electrons with an allowed single and the
// fingerprint.
template <int W>
__device__ __forceinline__ void derive_det(const Params &P, const Tables &T, const unsigned long long (&d)[W],
                                           unsigned long long (&pre)[PRE_WORDS], unsigned char *occ) {
    unsigned long long cb0 = 0, cb1 = 0;
    for (int g = 0; g < P.n_irrep_used; ++g) {
        int u0 = 0, u1 = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            u0 += __popcll(~d[w] & T.mask[(2 * g) * MAXW + w]);
            u1 += __popcll(~d[w] & T.mask[(2 * g + 1) * MAXW + w]);
        }
        cb0 |= (unsigned long long)u0 << (8 * g);
        cb1 |= (unsigned long long)u1 << (8 * g);
    }
    const unsigned set0 = nonzero_bytes(cb0), set1 = nonzero_bytes(cb1);
    unsigned long long ok[W];
#pragma unroll
    for (int w = 0; w < W; ++w)
        ok[w] = __ldg(P.unionm + (set0 * MAXW + w)) | __ldg(P.unionm + ((256 + set1) * MAXW + w));
    int n = 0;
    unsigned long long okm = 0, h = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        unsigned long long m = d[w];
        while (m) {
            const int b = __ffsll((long long)m) - 1;
            const int k = 64 * w + b;
            if (!FQ_CHECK(n < MAXN, P.st)) break;
            occ[n] = (unsigned char)k;
            okm |= ((ok[w] >> b) & 1ull) << n;
            h = 1099511628211ull * h + T.map1[k] * (unsigned long long)(n + 1);
            ++n;
            m &= m - 1;
        }
    }
    pre[PRE_FP] = h;
    pre[PRE_OKM] = okm;
    pre[PRE_CB0] = cb0;
    pre[PRE_CB1] = cb1;
}

// The per-determinant view from the derived words, the population and the run's reference and initiator rule.
template <int W>
__device__ __forceinline__ void fill_view(const Params &P, DetView<W> &v, const unsigned long long (&pre)[PRE_WORDS],
                                          int c) {
    const unsigned long long cb0 = pre[PRE_CB0], cb1 = pre[PRE_CB1];
    v.cb8[0] = cb0;
    v.cb8[1] = cb1;
    unsigned *cw = reinterpret_cast<unsigned *>(v.cnt);
#pragma unroll
    for (int j = 0; j < NCLASS / 4; ++j)  // class 2g + s: bytes (g = 2j, s = 0), (2j, 1), (2j + 1, 0), (2j + 1, 1)
        cw[j] = __byte_perm((unsigned)(cb0 >> (16 * j)), (unsigned)(cb1 >> (16 * j)), 0x5140u);
    v.okm = pre[PRE_OKM];
    v.nok = (unsigned char)__popcll(pre[PRE_OKM]);
    v.fp = pre[PRE_FP];
    v.c = c;
    int ac = c < 0 ? -c : c;
    bool is_ref = det_eq<W>(v.d, P.ref);
    v.flag = (P.init_thr < 0 || ac > P.init_thr || is_ref) ? 1 : 0;
    v.isref = is_ref ? 1 : 0;
}

// The view of v.d (its bits already set), derived on the spot.
template <int W>
__device__ __forceinline__ void prepare_det(const Params &P, const Tables &T, DetView<W> &v, unsigned char *occ,
                                            int c) {
    unsigned long long pre[PRE_WORDS];
    derive_det<W>(P, T, v.d, pre, occ);
    fill_view<W>(P, v, pre, c);
}

// Derived words and occupied list of slot s of list buffer b, computed and stored.
template <int W>
__device__ __forceinline__ void store_derived(const Params &P, const Tables &T, int b, long long s,
                                              const unsigned long long (&d)[W]) {
    unsigned long long pre[PRE_WORDS];
    unsigned char occ[MAXN] = {};
    derive_det<W>(P, T, d, pre, occ);
    ulonglong2 *dst = reinterpret_cast<ulonglong2 *>(P.pre[b] + s * PRE_WORDS);
    dst[0] = make_ulonglong2(pre[0], pre[1]);
    dst[1] = make_ulonglong2(pre[2], pre[3]);
    unsigned *od = reinterpret_cast<unsigned *>(P.occa[b] + s * P.ostride);
    for (int k = 0; k < P.ostride / 4; ++k)
        od[k] = (unsigned)occ[4 * k] | ((unsigned)occ[4 * k + 1] << 8) | ((unsigned)occ[4 * k + 2] << 16) |
                ((unsigned)occ[4 * k + 3] << 24);
}

// ---------------------------------------------------------------------------- one spawning attempt
// Spawns accepted by the lanes of one warp, inserted into the merge table together (flush_queue) so that
// the table's round trips are shared by the lanes instead of stalling the warp once per accepting lane.
#ifndef FQ_QUEUE_FLUSH
#define FQ_QUEUE_FLUSH 16
#endif
constexpr int kQueueFlush = FQ_QUEUE_FLUSH;  // flushed from this many entries on
constexpr int kQueue = kQueueFlush + 32;     // capacity: a round adds at most 32 to fewer than kQueueFlush
template <int W>
struct SpawnQueue {
    unsigned long long key[kQueue][W];
    unsigned long long val[kQueue];
    unsigned n;
    unsigned pad[3];
};

// Inserts queued spawns into the merge table (all 32 lanes; every lane inserts one entry): everything
// when all is set, else up to 32 entries once at least kQueueFlush are queued. Merge-table positions
// newly claimed go to the merged list. In a hash-partitioned run (Sec. V A) an entry whose determinant
// belongs to another partition (its fingerprint mod the partition count; map1 the orbital map) is
// appended to that partition's outbox instead, to be merged there after the exchange.
template <int W>
__device__ __forceinline__ void flush_queue(const Params &P, SpawnQueue<W> &q, bool all,
                                            const unsigned long long *map1) {
    __syncwarp();
    const unsigned n = q.n;
    if (n == 0 || (!all && n < (unsigned)kQueueFlush)) return;
    const int lane = threadIdx.x & 31;
    unsigned done = 0;
    do {
        const unsigned take = min(n - done, 32u);
        const unsigned e = done + lane;
        bool claimed = false;
        unsigned pos = 0;
        if (lane < (int)take) {
            unsigned long long key[W];
#pragma unroll
            for (int w = 0; w < W; ++w) key[w] = q.key[e][w];
            const unsigned long long val = q.val[e];
            int dest = P.part;
            if (P.n_parts > 1) dest = (int)(fingerprint<W>(key, map1) % (unsigned long long)P.n_parts);
            if (dest == P.part) {
                claimed = merge_insert<W>(P, key, val, pos);
            } else {
                const unsigned long long slot = atomicAdd(&P.st->ob_n[dest], 1ull);
                if (slot < (unsigned long long)P.ob_cap) {
                    unsigned long long *o = P.outbox + ((unsigned long long)dest * (unsigned long long)P.ob_cap + slot) * Stride<W>::v;
#pragma unroll
                    for (int w = 0; w < W; ++w) o[w] = key[w];
                    o[W] = val;
                } else {
                    set_status(P.st, FCIQMC_ERR_CAPACITY);
                }
            }
        }
        const long long slot = warp_append(&P.st->n_merged, claimed);
        if (claimed && slot < P.mt_cap) P.merged[slot] = pos;
        done += take;
    } while (all && done < n);
    __syncwarp();
    const unsigned rest = n - done;  // fewer than kQueueFlush, below the entries just taken
    if (lane < (int)rest) {
#pragma unroll
        for (int w = 0; w < W; ++w) q.key[lane][w] = q.key[done + lane][w];
        q.val[lane] = q.val[done + lane];
    }
    __syncwarp();
    if (lane == 0) q.n = rest;
    __syncwarp();
}

// Exact float of a small nonnegative integer (x < 2^23) without a conversion instruction.
__device__ __forceinline__ float small_f(unsigned x) { return __int_as_float(0x4B000000 | x) - 8388608.0f; }

// Tables of one heavily populated determinant, built by the warp that takes it up and used for all of
// that warp's attempts from it: for each double-excitation entry (spin case of the pair: 0 alpha alpha,
// 1 beta beta, 2 mixed; times 8, plus the irrep product of the pair) the "good" first virtuals a of
// Sec. VI B in ascending order and their number G; for each (irrep, spin) class its unoccupied spin
// orbitals in ascending order, and the position of each unoccupied spin orbital in its class list.
// Rows are padded by one 32-bit word so that the same position in different rows falls in different
// shared-memory banks (the lanes of a warp read random rows).
struct HeavyTab {
    unsigned char glist[24][MAXSO + 4];
    unsigned char ulist[NCLASS][MAXSO / 2 + 4];
    unsigned char urank[MAXSO];
    unsigned char occ[MAXN];  // the determinant's occupied spin orbitals, ascending
    unsigned short G[24];
};

// Good a-orbitals for one (spin case, pair irrep): a of spin sa in irrep g is good when its class has
// an unoccupied orbital and the class of b (irrep g ^ gij, spin sb = si + sj - sa) has one left besides
// a. All eight irreps of a spin are tested at once on the byte-packed class counts (counts <= 64, so no
// byte carries); the union of the good classes' orbitals comes from a table indexed by the irrep set.
template <int W>
__device__ __forceinline__ unsigned good_set(const Params &P, const DetView<W> &v, int si, int sj, int gij,
                                             unsigned long long (&gm)[W]) {
    constexpr unsigned long long kOnes = 0x0101010101010101ull, kHigh = 0x8080808080808080ull;
    unsigned G = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) gm[w] = 0ull;
#pragma unroll
    for (int sa = 0; sa < 2; ++sa) {
        if (si == sj && sa != si) continue;
        const int sb = si + sj - sa;
        const unsigned long long A = v.cb8[sa];
        unsigned long long B = v.cb8[sb];
        if (gij & 4) B = (B >> 32) | (B << 32);
        const unsigned sel = 0x3210u ^ (0x1111u * (unsigned)(gij & 3));  // byte g <- byte g ^ (gij & 3)
        B = ((unsigned long long)__byte_perm((unsigned)(B >> 32), 0u, sel) << 32) | __byte_perm((unsigned)B, 0u, sel);
        const unsigned long long need = (sa == sb && gij == 0) ? 2ull : 1ull;  // a and b from one class
        const unsigned long long cond = (A + 0x7F * kOnes) & (B + (0x80 - need) * kOnes) & kHigh;
        const unsigned long long bits = cond >> 7;
        G += (unsigned)(((A & (bits * 0xFFull)) * kOnes) >> 56);
        const unsigned set = (unsigned)((bits * 0x0102040810204080ull) >> 56);
#pragma unroll
        for (int w = 0; w < W; ++w) gm[w] |= __ldg(P.unionm + ((sa * 256 + set) * MAXW + w));
    }
#pragma unroll
    for (int w = 0; w < W; ++w) gm[w] &= ~v.d[w];
    return G;
}

// good_set with the union of the good classes' orbitals from the block's shared tables (two 4-irrep halves)
// instead of the global 8-bit-set table.
template <int W>
__device__ __forceinline__ unsigned good_set_t(const Tables &T, const DetView<W> &v, int si, int sj, int gij,
                                               unsigned long long (&gm)[W]) {
    constexpr unsigned long long kOnes = 0x0101010101010101ull, kHigh = 0x8080808080808080ull;
    unsigned G = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) gm[w] = 0ull;
#pragma unroll
    for (int sa = 0; sa < 2; ++sa) {
        if (si == sj && sa != si) continue;
        const int sb = si + sj - sa;
        const unsigned long long A = v.cb8[sa];
        unsigned long long B = v.cb8[sb];
        if (gij & 4) B = (B >> 32) | (B << 32);
        const unsigned sel = 0x3210u ^ (0x1111u * (unsigned)(gij & 3));  // byte g <- byte g ^ (gij & 3)
        B = ((unsigned long long)__byte_perm((unsigned)(B >> 32), 0u, sel) << 32) | __byte_perm((unsigned)B, 0u, sel);
        const unsigned long long need = (sa == sb && gij == 0) ? 2ull : 1ull;  // a and b from one class
        const unsigned long long cond = (A + 0x7F * kOnes) & (B + (0x80 - need) * kOnes) & kHigh;
        const unsigned long long bits = cond >> 7;
        G += (unsigned)(((A & (bits * 0xFFull)) * kOnes) >> 56);
        const unsigned set = (unsigned)((bits * 0x0102040810204080ull) >> 56);
        const unsigned long long *lo = T.uh + ((sa * 2) * 16 + (set & 15u)) * MAXW;
        const unsigned long long *hi = T.uh + ((sa * 2 + 1) * 16 + (set >> 4)) * MAXW;
#pragma unroll
        for (int w = 0; w < W; ++w) gm[w] |= lo[w] | hi[w];
    }
#pragma unroll
    for (int w = 0; w < W; ++w) gm[w] &= ~v.d[w];
    return G;
}

// Builds tab for determinant v; called by all 32 lanes of a warp. Lanes 0..23 take one entry each,
// lanes 24..31 two classes each.
template <int W>
__device__ __forceinline__ void build_heavy_tab(const Params &P, const Tables &T, const DetView<W> &v, HeavyTab &tab,
                                                int lane) {
    if (lane < 24) {
        const int sc = lane >> 3, gij = lane & 7;
        const int si = sc == 1 ? 1 : 0, sj = sc == 0 ? 0 : 1;
        unsigned long long gm[W];
        tab.G[lane] = (unsigned short)good_set<W>(P, v, si, sj, gij, gm);
        int n = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            unsigned long long m = gm[w];
            while (m) {
                tab.glist[lane][n++] = (unsigned char)(64 * w + __ffsll((long long)m) - 1);
                m &= m - 1;
            }
        }
    } else {
        for (int c = lane - 24; c < NCLASS; c += 8) {
            int n = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                unsigned long long m = ~v.d[w] & T.mask[c * MAXW + w];
                while (m) {
                    const int so = 64 * w + __ffsll((long long)m) - 1;
                    tab.ulist[c][n] = (unsigned char)so;
                    tab.urank[so] = (unsigned char)n;
                    ++n;
                    m &= m - 1;
                }
            }
        }
    }
    __syncwarp();
}

// n = floor(p) + [q < (p - floor(p)) R] for an FP64 value p known only to lie in [p_lo, p_hi], an integer
// q < 2^53 and R given as its nearest float rf: n, or -1 when the bounds do not decide it. p - m and
// max(p_lo, 0) - m are exact (Sterbenz); the products round to nearest within the kUp/kDown margins.
__device__ __forceinline__ int decide_spawn(float p_lo, float p_hi, unsigned long long q, float rf) {
    if (!(p_hi < 0x1p22f)) return -1;
    const float pl = fmaxf(p_lo, 0.f);
    const float m = floorf(pl);
    if (floorf(p_hi) != m) return -1;
    const float th_hi = (p_hi - m) * rf * kUp, th_lo = (pl - m) * rf * kDown;
    const float q_lo = small_f((unsigned)(q >> 30)) * 0x1p30f;  // q_lo <= q < q_lo + 2^30, exact
    if (q_lo >= th_hi) return (int)m;
    if (q_lo + 0x1p30f <= th_lo) return (int)m + 1;
    return -1;
}

// Counters and queued merge-table entry of an attempt that spawns n > 0 walkers onto child.
template <int W>
__device__ __forceinline__ void emit_spawn(const Params &P, const DetView<W> &v, const unsigned long long (&child)[W],
                                           int n, int sgn_h, unsigned long long *cnt, SpawnQueue<W> &out) {
    cnt[C_EVENTS]++;
    cnt[C_SPAWNED] += (unsigned long long)n;
    const long long amt = -(long long)(v.c > 0 ? 1 : -1) * sgn_h * (long long)n;
    const unsigned slot = atomicAdd(&out.n, 1u);
    if (!FQ_CHECK(slot < (unsigned)kQueue, P.st)) return;
#pragma unroll
    for (int w = 0; w < W; ++w) out.key[slot][w] = child[w];
    out.val[slot] = (v.flag ? kFlagUnit : 0ull) + (unsigned long long)amt;
}

// Probability that one attempt from v generates the determinant x (the closed forms the generator of
// Sec. VI A, B realises; 0 when it cannot produce x), in the FP64 order
//   single: P_single / (M_allow (N - delta_s)); double: (P_double (M^(b|a) + M^(a|b))) / (npairs G M^(b|a) M^(a|b)).
template <int W>
__device__ double gen_prob(const Params &P, const DetView<W> &v, const unsigned long long (&x)[W]) {
    unsigned long long holes[W], parts[W];
    int nh = 0, np = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        holes[w] = v.d[w] & ~x[w];
        parts[w] = x[w] & ~v.d[w];
        nh += __popcll(holes[w]);
        np += __popcll(parts[w]);
    }
    if (nh != np || nh == 0 || nh > 2) return 0.0;
    if (nh == 1) {
        const int i = select_bit<W>(holes, 0), a = select_bit<W>(parts, 0);
        const int ci = (int)__ldg(P.irrep + (i >> 1)) * 2 + (i & 1), ca = (int)__ldg(P.irrep + (a >> 1)) * 2 + (a & 1);
        if (ci != ca) return 0.0;
        return __ddiv_rn(P.p_single_d, (double)((long long)v.cnt[ci] * (long long)v.nok));
    }
    const int i = select_bit<W>(holes, 0), j = select_bit<W>(holes, 1);
    const int a = select_bit<W>(parts, 0), b = select_bit<W>(parts, 1);
    const int si = i & 1, sj = j & 1;
    if ((a & 1) + (b & 1) != si + sj) return 0.0;
    const int gi = __ldg(P.irrep + (i >> 1)), gj = __ldg(P.irrep + (j >> 1));
    const int ga = __ldg(P.irrep + (a >> 1)), gb = __ldg(P.irrep + (b >> 1));
    if ((ga ^ gb) != (gi ^ gj)) return 0.0;
    if (si == sj && ((a & 1) != si || (b & 1) != si)) return 0.0;
    unsigned long long gm[W];
    const long long G = good_set<W>(P, v, si, sj, gi ^ gj, gm);
    const int ca = ga * 2 + (a & 1), cb = gb * 2 + (b & 1);
    const long long m_ba = (long long)v.cnt[cb] - (ca == cb ? 1 : 0);
    const long long m_ab = (long long)v.cnt[ca] - (ca == cb ? 1 : 0);
    return __ddiv_rn(__dmul_rn(P.p_double_d, (double)(m_ba + m_ab)), (double)((long long)P.npairs * G * m_ba * m_ab));
}

// <Phi_a|H|Phi_b> between the spin-coupled functions stored on v (a) and b != a: both open:
// <a|H|b> + sigma pi_b <a|H|bbar>; one closed: sqrt(2) <a|H|b>; both closed: <a|H|b> (the flip symmetry folds
// the four determinant couplings).
template <int W>
__device__ double hphf_hij(const Params &P, const DetView<W> &v, const unsigned long long (&b)[W]) {
    unsigned long long ab[W], bb[W], a[W];
#pragma unroll
    for (int w = 0; w < W; ++w) a[w] = v.d[w];
    flip_spins<W>(a, ab);
    flip_spins<W>(b, bb);
    const bool a_open = !det_same<W>(a, ab), b_open = !det_same<W>(b, bb);
    unsigned char occ[MAXN];
    decode_occ<W>(v.d, occ);
    const double hab = hij_any<W>(P, a, occ, b);
    if (a_open && b_open) return __dadd_rn(hab, __dmul_rn(pair_sign(n_open<W>(b)), hij_any<W>(P, a, occ, bb)));
    if (a_open || b_open) return __dmul_rn(hab, kSqrt2);
    return hab;
}

// Float bounds of the two quantities of a spin-coupled double-excitation attempt (the same forms as in
// gen_prob and hij_double): the generation probability of a double excitation y of v (0 if the generator
// cannot produce it), within 4 roundings of float, and the matrix element <y|H|v> for a double
// difference, |H - value| <= err.
template <int W>
__device__ float gen_prob_double_f(const Params &P, const DetView<W> &v, const HeavyTab *tab, int i, int j, int a,
                                   int b) {
    const int si = i & 1, sj = j & 1;
    if ((a & 1) + (b & 1) != si + sj) return 0.f;
    const int gi = __ldg(P.irrep + (i >> 1)), gj = __ldg(P.irrep + (j >> 1));
    const int ga = __ldg(P.irrep + (a >> 1)), gb = __ldg(P.irrep + (b >> 1));
    if ((ga ^ gb) != (gi ^ gj)) return 0.f;
    if (si == sj && ((a & 1) != si || (b & 1) != si)) return 0.f;
    long long G;
    if (tab) {  // the determinant's tables hold the good-set sizes
        G = tab->G[(si == sj ? si : 2) * 8 + (gi ^ gj)];
    } else {
        unsigned long long gm[W];
        G = good_set<W>(P, v, si, sj, gi ^ gj, gm);
    }
    const int ca = ga * 2 + (a & 1), cb = gb * 2 + (b & 1);
    const long long m_ba = (long long)v.cnt[cb] - (ca == cb ? 1 : 0);
    const long long m_ab = (long long)v.cnt[ca] - (ca == cb ? 1 : 0);
    return __fdiv_rn(P.p_double_f * small_f((unsigned)(m_ba + m_ab)), (float)((long long)P.npairs * G * m_ba * m_ab));
}
template <int W>
__device__ __forceinline__ float hdouble_f_at(const Params &P, const unsigned long long (&d)[W], int i, int j, int a,
                                              int b, unsigned long long pol, float &err) {
    const float xf = ((i & 1) == (a & 1) && (j & 1) == (b & 1)) ? eri_f(P, i >> 1, a >> 1, j >> 1, b >> 1, pol) : 0.f;
    const float yf = ((i & 1) == (b & 1) && (j & 1) == (a & 1)) ? eri_f(P, i >> 1, b >> 1, j >> 1, a >> 1, pol) : 0.f;
    err = fmaf(fabsf(xf) + fabsf(yf), 0x1p-22f, 1e-30f);
    const float h = xf - yf;
    return double_parity<W>(d, i, j, a, b) ? -h : h;
}

// The FP64 evaluation of a spin-coupled attempt that generated x (flip xb) from v, target function stored
// on b: p = (tau |H_AB|) / (P(x) + P(xb)), then floor(p) plus one with the Bernoulli part of the type word.
template <int W>
__device__ __forceinline__ void hphf_exact(const Params &P, const DetView<W> &v, const unsigned long long (&x)[W],
                                           const unsigned long long (&xb)[W], const unsigned long long (&b)[W],
                                           unsigned long long t, bool single, unsigned long long *cnt,
                                           SpawnQueue<W> &out) {
    const double hv = hphf_hij<W>(P, v, b);
    if (hv == 0.0) return;
    double g = gen_prob<W>(P, v, x);
    if (!det_same<W>(xb, x)) g = __dadd_rn(g, gen_prob<W>(P, v, xb));
    const double p = __ddiv_rn(__dmul_rn(P.tau, fabs(hv)), g);
    const double fl = floor(p);
    if (fl >= 2147483647.0) { set_status(P.st, FCIQMC_ERR_NUMERIC); return; }
    const unsigned long long off = single ? P.d53 : 0ull;
    const double range = single ? __dsub_rn(9007199254740992.0, P.d53_d) : P.d53_d;
    const int n = (int)fl + (__ull2double_rn(t - off) < __dmul_rn(__dsub_rn(p, fl), range) ? 1 : 0);
    if (n == 0) return;
    emit_spawn<W>(P, v, b, n, hv > 0.0 ? 1 : -1, cnt, out);
}

// Completes a double-excitation attempt on spin-coupled functions (Sec. VI C) that generated the
// determinant x from the stored determinant v: the target function holds x and its flip, its generation
// probability is the sum of theirs, p = tau |H_AB| / (P(x) + P(xbar)), the Bernoulli part from the type
// word as for determinants. The attempt is first decided from float bounds of H_AB and of the generation
// probability (gx: the float form of x's); a flip that is a single of v and undecided cases evaluate
// everything in FP64. For a closed-shell v the flip of x has the same class counts, so the same
// generation probability, and H_AB needs only the element to the stored determinant. (Singles are
// completed by hphf_single_end.)
template <int W, bool SP>
__device__ void hphf_attempt_end(const Params &P, const DetView<W> &v, const HeavyTab *tab,
                                 const unsigned long long (&x)[W], unsigned long long t, float gx, int oi, int oj,
                                 int oa, int ob, unsigned long long *cnt, SpawnQueue<W> &out) {
    unsigned long long xb[W], b[W];
    flip_spins<W>(x, xb);
    const bool fl_less = det_less<W>(xb, x);
#pragma unroll
    for (int w = 0; w < W; ++w) b[w] = fl_less ? xb[w] : x[w];
    bool same = true;
#pragma unroll
    for (int w = 0; w < W; ++w) same = same && b[w] == v.d[w];
    if (same || (SP && !in_space<W>(P, b))) { cnt[C_NULLS]++; return; }
    {
        unsigned long long hb[W], pb[W], a[W], ab[W], bb[W];
        int lb = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            a[w] = v.d[w];
            hb[w] = v.d[w] & ~xb[w];
            pb[w] = xb[w] & ~v.d[w];
            lb += __popcll(hb[w]);
        }
        if (lb != 1) {
            const unsigned long long pol = keep_policy();
            flip_spins<W>(a, ab);
            flip_spins<W>(b, bb);
            const bool a_open = !det_same<W>(a, ab), b_open = !det_same<W>(b, bb);
            // (oi, oj) -> (oa, ob), ascending: the double that generated x
            float hab, habbar = 0.f, e1, e2 = 0.f;
            int bi = 0, bj = 0, ba = 0, bbo = 0;  // a -> xbar when it is a double
            if (a_open && lb == 2) {
                bi = select_bit<W>(hb, 0);
                bj = select_bit<W>(hb, 1);
                ba = select_bit<W>(pb, 0);
                bbo = select_bit<W>(pb, 1);
            }
            if (a_open) {
                float ex, exb = 0.f;
                const float hxf = hdouble_f_at<W>(P, a, oi, oj, oa, ob, pol, ex);
                const float hxbf = lb == 2 ? hdouble_f_at<W>(P, a, bi, bj, ba, bbo, pol, exb) : 0.f;  // beyond doubles: 0
                hab = fl_less ? hxbf : hxf;
                habbar = fl_less ? hxf : hxbf;
                e1 = fl_less ? exb : ex;
                e2 = fl_less ? ex : exb;
            } else if (fl_less) {  // a = abar: the flip of x is the flipped double of a
                const int fi = oi ^ 1, fj = oj ^ 1, fa = oa ^ 1, fb = ob ^ 1;
                hab = hdouble_f_at<W>(P, a, min(fi, fj), max(fi, fj), min(fa, fb), max(fa, fb), pol, e1);
            } else {
                hab = hdouble_f_at<W>(P, a, oi, oj, oa, ob, pol, e1);
            }
            float vf, ev;
            if (a_open && b_open) {
                vf = hab + (float)pair_sign(n_open<W>(b)) * habbar;
                ev = e1 + e2 + fabsf(vf) * 0x1p-21f;
            } else if (a_open || b_open) {
                vf = hab * (float)kSqrt2;
                ev = 1.5f * e1 + fabsf(vf) * 0x1p-21f;
            } else {
                vf = hab;
                ev = e1;
            }
            float g = gx;
            if (lb == 2 && !det_same<W>(xb, x)) g = a_open ? g + gen_prob_double_f<W>(P, v, tab, bi, bj, ba, bbo) : g + g;
            const float ah_lo = fabsf(vf) - ev, ah_hi = fabsf(vf) + ev;
            const int n = decide_spawn(__fdiv_rn(ah_lo * P.tau_f, g) * kDown, __fdiv_rn(ah_hi * P.tau_f, g) * kUp, t,
                                       P.d53_f);
            if (n == 0) return;
            if (n > 0) {
                emit_spawn<W>(P, v, b, n, vf > 0.f ? 1 : -1, cnt, out);  // |vf| > ev: the sign of H_AB
                return;
            }
            atomicAdd(&P.st->exact_spawn, 1ull);  // undecided by the float bounds
        }
    }
    hphf_exact<W>(P, v, x, xb, b, t, false, cnt, out);
}

// First part of attempt a from determinant v (Eq. 3 with the generator of Sec. VI). Random numbers:
// one Philox block keyed by (seed, iteration), counter (a, tag 0, fingerprint), words (r0, r1). The
// type word t = r0 >> 11 also realises the Bernoulli part of the spawn: given the type, t is uniform on
// [0, d53) for a double and on [d53, 2^53) for a single. The other 75 bits, r1 2^11 + (r0 mod 2^11),
// give the choices as mixed-radix digits (rank_next). A double is completed here; a single is
// selected (electron i, virtual ao) and returned pending (true) for the warp to evaluate its element.
template <int W, bool TAB, int MODE>
__device__ __forceinline__ bool attempt_begin(const Params &P, const Tables &T, const DetView<W> &v,
                                              const unsigned char *occ, const HeavyTab *tab, const float *rcpf, unsigned a, unsigned iter,
                                              unsigned long long pol, unsigned long long *cnt, SpawnQueue<W> &out,
                                              int &i_out, int &a_out, unsigned &mallow_out, unsigned long long &q_out,
                                              int &i1_out, int &a1_out, int &i2_out, int &a2_out, bool rtab) {
    unsigned long long r0, rh;
    draw2(a, 0u, v.fp, P.seed, iter, r0, rh);
    const unsigned long long t = r0 >> 11;
    unsigned rl = (unsigned)r0 & 0x7FFu;  // choice word R = rh 2^11 + rl
    if (t >= P.d53) {
        // single excitation (Sec. VI A): i uniform over the N - delta_s electrons with M_allow > 0, a
        // uniform over the unoccupied spin orbitals of i's class
        if (v.nok == 0) { cnt[C_NULLS]++; return false; }
        const int i = occ[select64(v.okm, (int)rank_next(rh, rl, v.nok))];
        const int ci = T.irrep[i >> 1] * 2 + (i & 1);
        const unsigned mallow = v.cnt[ci];
        const int k2 = (int)rank_next(rh, rl, mallow);
        int ao;
        if (TAB) {
            ao = tab->ulist[ci][k2];
        } else {
            unsigned long long um[W];
#pragma unroll
            for (int w = 0; w < W; ++w) um[w] = ~v.d[w] & T.mask[ci * MAXW + w];
            ao = select_bit<W>(um, k2);
        }
        if (MODE & 2) {  // spin-coupled functions: the single elements H_AB needs are evaluated by the warp
            unsigned long long x[W], xb[W], b[W], sb[W];
#pragma unroll
            for (int w = 0; w < W; ++w) x[w] = v.d[w];
            flip<W>(x, i);
            flip<W>(x, ao);
            flip_spins<W>(x, xb);
            const bool fl_less = det_less<W>(xb, x);
#pragma unroll
            for (int w = 0; w < W; ++w) b[w] = fl_less ? xb[w] : x[w];
            if (det_same<W>(b, v.d) || ((MODE & 1) && !in_space<W>(P, b))) { cnt[C_NULLS]++; return false; }
            flip_spins<W>(v.d, sb);
            i1_out = i;
            a1_out = ao;
            i2_out = -1;
            a2_out = -1;
            if (det_same<W>(v.d, sb)) {  // closed source: only the element to b, a single (flipped when b = xb)
                if (fl_less) {
                    i1_out = i ^ 1;
                    a1_out = ao ^ 1;
                }
            } else if (!det_same<W>(x, xb)) {  // the element to x, and the one to xb when that is a single as well
                unsigned long long hb[W], pb[W];
                int lb = 0;
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    hb[w] = v.d[w] & ~xb[w];
                    pb[w] = xb[w] & ~v.d[w];
                    lb += __popcll(hb[w]);
                }
                if (lb == 1) {
                    i2_out = select_bit<W>(hb, 0);
                    a2_out = select_bit<W>(pb, 0);
                }
            }
            i_out = i;
            a_out = ao;
            mallow_out = mallow;
            q_out = t - P.d53;
            return true;
        }
        if (MODE & 1) {  // outside the permitted space: a null excitation (Sec. VI)
            unsigned long long ch[W];
#pragma unroll
            for (int w = 0; w < W; ++w) ch[w] = v.d[w];
            flip<W>(ch, i);
            flip<W>(ch, ao);
            if (!in_space<W>(P, ch)) { cnt[C_NULLS]++; return false; }
        }
        i_out = i1_out = i;
        a_out = a1_out = ao;
        i2_out = a2_out = -1;
        mallow_out = mallow;
        q_out = t - P.d53;
        return true;
    }
    // double excitation (Sec. VI B): pair by inverse triangular index, a among the "good" unoccupied
    // orbitals of allowed spin, b from the class fixed by symmetry (Eq. sym1) and spin
    if (P.npairs == 0) { cnt[C_NULLS]++; return false; }
    if (TAB && rtab) {  // the reference: the same choices, read with p from its table
        const unsigned pi = __ldg(P.ref_pinfo + rank_next(rh, rl, (unsigned)P.npairs));
        const unsigned G = pi & 0xFFu;
        if (G == 0) { cnt[C_NULLS]++; return false; }
        const unsigned o2 = __ldg(P.ref_off2 + (pi >> 8) + rank_next(rh, rl, G));
        const unsigned ei = (o2 >> 7) + rank_next(rh, rl, o2 & 0x7Fu);
        if (!FQ_CHECK((long long)ei < P.ref_n, P.st)) return false;
        const RefExc *e = P.ref_exc + ei;
        const float2 pb = __ldg(reinterpret_cast<const float2 *>(e));
        if (MODE & 1) {
            if (pb.x < 0.f) { cnt[C_NULLS]++; return false; }  // the target lies outside the permitted space
        }
        const double ps = __ldg(&e->ps);
        int n = decide_spawn(pb.x, pb.y, t, P.d53_f);
        if (n < 0) {
            atomicAdd(&P.st->exact_spawn, 1ull);
            const double p = fabs(ps);
            const double fl = floor(p);
            if (fl >= 2147483647.0) { set_status(P.st, FCIQMC_ERR_NUMERIC); return false; }
            n = (int)fl + (__ull2double_rn(t) < __dmul_rn(__dsub_rn(p, fl), P.d53_d) ? 1 : 0);
        }
        if (n == 0) return false;
        const uchar4 o = __ldg(reinterpret_cast<const uchar4 *>(&e->i));
        unsigned long long child[W];
#pragma unroll
        for (int w = 0; w < W; ++w) child[w] = v.d[w];
        flip<W>(child, o.x);
        flip<W>(child, o.y);
        flip<W>(child, o.z);
        flip<W>(child, o.w);
        emit_spawn<W>(P, v, child, n, ps > 0.0 ? 1 : -1, cnt, out);
        return false;
    }
    const unsigned short pr = T.pairs[rank_next(rh, rl, (unsigned)P.npairs)];
    const int i = occ[pr & 0xFF], j = occ[pr >> 8];
    const int si = i & 1, sj = j & 1;
    const int gij = T.irrep[i >> 1] ^ T.irrep[j >> 1];
    unsigned G;
    int ao;
    if (TAB) {
        const int e = (si == sj ? si : 2) * 8 + gij;
        G = tab->G[e];
        if (G == 0) { cnt[C_NULLS]++; return false; }
        const unsigned k2 = rank_next(rh, rl, G);
        if (!FQ_CHECK(k2 < (unsigned)MAXSO, P.st)) return false;
        ao = tab->glist[e][k2];
    } else {
        unsigned long long gm[W];
        G = good_set_t<W>(T, v, si, sj, gij, gm);
        if (G == 0) { cnt[C_NULLS]++; return false; }
        ao = select_bit<W>(gm, (int)rank_next(rh, rl, G));
    }
    const int ga = T.irrep[ao >> 1];
    const int ca = ga * 2 + (ao & 1);
    const int cb = (gij ^ ga) * 2 + (si + sj - (ao & 1));
    const unsigned same = ca == cb ? 1u : 0u;
    const unsigned m_ba = v.cnt[cb] - same;
    const unsigned m_ab = v.cnt[ca] - same;
    int k3 = (int)rank_next(rh, rl, m_ba);
    int bo;
    if (TAB) {
        if (same && k3 >= tab->urank[ao]) ++k3;  // the list of class cb still holds a
        if (!FQ_CHECK(k3 < MAXSO / 2, P.st)) return false;
        bo = tab->ulist[cb][k3];
    } else {
        unsigned long long bm[W];
#pragma unroll
        for (int w = 0; w < W; ++w) bm[w] = ~v.d[w] & T.mask[cb * MAXW + w];
        clear_bit<W>(bm, ao);
        bo = select_bit<W>(bm, k3);
    }
    if (MODE & 2) {  // spin-coupled functions
        unsigned long long ch[W];
#pragma unroll
        for (int w = 0; w < W; ++w) ch[w] = v.d[w];
        flip<W>(ch, i);
        flip<W>(ch, j);
        flip<W>(ch, ao);
        flip<W>(ch, bo);
        // generation probability of this double from the quantities of its selection (as gen_prob_double_f)
        const float gx = __fdiv_rn(P.p_double_f * small_f(m_ba + m_ab),
                                   (float)((long long)P.npairs * (long long)G * (long long)m_ba * (long long)m_ab));
        hphf_attempt_end<W, (MODE & 1) != 0>(P, v, tab, ch, t, gx, i, j, min(ao, bo), max(ao, bo), cnt, out);
        return false;
    }
    if (MODE & 1) {  // outside the permitted space: a null excitation (Sec. VI)
        unsigned long long ch[W];
#pragma unroll
        for (int w = 0; w < W; ++w) ch[w] = v.d[w];
        flip<W>(ch, i);
        flip<W>(ch, j);
        flip<W>(ch, ao);
        flip<W>(ch, bo);
        if (!in_space<W>(P, ch)) { cnt[C_NULLS]++; return false; }
    }
    const int A = min(ao, bo), B = max(ao, bo);
    const unsigned L = m_ba + m_ab;
    const bool t1 = ((i & 1) == (A & 1)) && ((j & 1) == (B & 1));
    const bool t2 = ((i & 1) == (B & 1)) && ((j & 1) == (A & 1));
    // bounds of p = |H| tau / P_gen from the float copy of the integrals
    const float xf = t1 ? eri_f(P, i >> 1, A >> 1, j >> 1, B >> 1, pol) : 0.f;
    const float yf = t2 ? eri_f(P, i >> 1, B >> 1, j >> 1, A >> 1, pol) : 0.f;
    const float hf = xf - yf;
    const float eh = fmaf(fabsf(xf) + fabsf(yf), 0x1p-22f, 1e-30f);  // >= |H - hf| with a factor 2
    const float ah_lo = fabsf(hf) - eh, ah_hi = fabsf(hf) + eh;
    const float F = P.cdn_f * small_f(G) * small_f(m_ba) * small_f(m_ab) * rcpf[L];
    int n = decide_spawn(ah_lo * F * kDown, ah_hi * F * kUp, t, P.d53_f);
    int sgn_h;
    if (n >= 0) {
        if (n == 0) return false;
        sgn_h = hf > 0.f ? 1 : -1;  // |hf| > eh: same sign as H
        if (double_parity<W>(v.d, i, j, A, B)) sgn_h = -sgn_h;
    } else {
        atomicAdd(&P.st->exact_spawn, 1ull);
        const double hd = hij_double<W>(P, v.d, i, j, A, B);
        if (hd == 0.0) return false;
        // p = ((|H| (tau / P_double)) (npairs G M^(b|a) M^(a|b))) (1 / (M^(b|a) + M^(a|b)))
        const long long K = (long long)P.npairs * (long long)G * (long long)m_ba * (long long)m_ab;
        const double p = __dmul_rn(__dmul_rn(__dmul_rn(fabs(hd), P.cd), (double)K), P.recip[L]);
        const double fl = floor(p);
        if (fl >= 2147483647.0) { set_status(P.st, FCIQMC_ERR_NUMERIC); return false; }
        n = (int)fl + (__ull2double_rn(t) < __dmul_rn(__dsub_rn(p, fl), P.d53_d) ? 1 : 0);
        sgn_h = hd > 0.0 ? 1 : -1;
        if (n == 0) return false;
    }
    unsigned long long child[W];
#pragma unroll
    for (int w = 0; w < W; ++w) child[w] = v.d[w];
    flip<W>(child, i);
    flip<W>(child, j);
    flip<W>(child, ao);
    flip<W>(child, bo);
    emit_spawn<W>(P, v, child, n, sgn_h, cnt, out);
    return false;
}

// Float value and sum of absolute terms of the single-excitation element h_ia + sum_j [(ia|jj) -
// delta_spin (ij|ja)] (without the parity sign) for every lane with a pending single, each evaluated by
// the whole warp: lane x takes electrons x, x + 32. Called by all 32 lanes.
template <int W>
__device__ __forceinline__ void single_elements_warp(const Params &P, const unsigned char *occp, bool pend, int i,
                                                     int a, unsigned long long pol, float &hs, float &hab) {
    unsigned need = __ballot_sync(0xFFFFFFFFu, pend);
    const int lane = threadIdx.x & 31;
    while (need) {
        const int src = __ffs(need) - 1;
        need &= need - 1;
        const unsigned char *so = reinterpret_cast<const unsigned char *>(
            __shfl_sync(0xFFFFFFFFu, reinterpret_cast<unsigned long long>(occp), src));
        const int ii = __shfl_sync(0xFFFFFFFFu, i, src), aa = __shfl_sync(0xFFFFFFFFu, a, src);
        const int I = ii >> 1, A = aa >> 1;
        float s = 0.f, b = 0.f;
        for (int x = lane; x < P.n_elec; x += 32) {
            const int j = so[x];
            if (j != ii) {
                const int J = j >> 1;
                const float u = eri_f(P, I, A, J, J, pol);
                s += u;
                b += fabsf(u);
                if ((j & 1) == (ii & 1)) {
                    const float w = eri_f(P, I, J, J, A, pol);
                    s -= w;
                    b += fabsf(w);
                }
            }
        }
        if (lane == 0) {
            const float hh = __ldg(P.h_f + I * P.n_orb + A);
            s += hh;
            b += fabsf(hh);
        }
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_down_sync(0xFFFFFFFFu, s, o);
            b += __shfl_down_sync(0xFFFFFFFFu, b, o);
        }
        s = __shfl_sync(0xFFFFFFFFu, s, 0);
        b = __shfl_sync(0xFFFFFFFFu, b, 0);
        if (lane == src) {
            hs = s;
            hab = b;
        }
    }
}

// Completes a pending single i -> ao: |H - hs| <= hab serr (float sum of at most 2N - 1 rounded terms,
// and the FP64 sum), so most decisions need no FP64; the rest evaluate H in FP64.
template <int W>
__device__ __forceinline__ void attempt_single_end(const Params &P, const DetView<W> &v, const unsigned char *occ,
                                                   int i, int ao, unsigned mallow,
                                                   unsigned long long q, float hs, float hab, unsigned long long *cnt,
                                                   SpawnQueue<W> &out) {
    const float eh = fmaf(hab, P.serr_f, 1e-30f);
    const float ah_lo = fabsf(hs) - eh, ah_hi = fabsf(hs) + eh;
    const float F = P.cs_f * small_f(mallow * v.nok);
    int n = decide_spawn(ah_lo * F * kDown, ah_hi * F * kUp, q, P.srange_f);
    int sgn_h;
    if (n >= 0) {
        if (n == 0) return;
        sgn_h = hs > 0.f ? 1 : -1;
        if (count_between<W>(v.d, i, ao) & 1) sgn_h = -sgn_h;
    } else {
        atomicAdd(&P.st->exact_spawn, 1ull);
        const double hv = hij_single<W>(P, v.d, occ, i, ao);
        if (hv == 0.0) return;
        // p = (|H| (tau / P_single)) (M_allow (N - delta_s))
        const double p = __dmul_rn(__dmul_rn(fabs(hv), P.cs), (double)((long long)mallow * (long long)v.nok));
        const double fl = floor(p);
        if (fl >= 2147483647.0) { set_status(P.st, FCIQMC_ERR_NUMERIC); return; }
        const double range = __dsub_rn(9007199254740992.0, P.d53_d);
        n = (int)fl + (__ull2double_rn(q) < __dmul_rn(__dsub_rn(p, fl), range) ? 1 : 0);
        sgn_h = hv > 0.0 ? 1 : -1;
        if (n == 0) return;
    }
    unsigned long long child[W];
#pragma unroll
    for (int w = 0; w < W; ++w) child[w] = v.d[w];
    flip<W>(child, i);
    flip<W>(child, ao);
    emit_spawn<W>(P, v, child, n, sgn_h, cnt, out);
}

// Completes a pending spin-coupled single i -> ao from v (x and its flip xb; target stored on b) from the
// warp's float sums of the single elements (i1, a1) and, for an open-shell v whose xb is a single as well,
// (i2, a2): H_AB and the generation probability in float with error bounds, the same decision as for
// determinants; undecided cases evaluate everything in FP64.
template <int W>
__device__ __forceinline__ void hphf_single_end(const Params &P, const DetView<W> &v, const HeavyTab *tab, int i,
                                                int ao, int i1, int a1,
                                                int i2, int a2, unsigned mallow, unsigned long long q, float hs,
                                                float hab, float hs2, float hab2, unsigned long long *cnt,
                                                SpawnQueue<W> &out) {
    unsigned long long a[W], ab[W], x[W], xb[W], b[W], bb[W];
#pragma unroll
    for (int w = 0; w < W; ++w) a[w] = x[w] = v.d[w];
    flip<W>(x, i);
    flip<W>(x, ao);
    flip_spins<W>(x, xb);
    const bool fl_less = det_less<W>(xb, x);
#pragma unroll
    for (int w = 0; w < W; ++w) b[w] = fl_less ? xb[w] : x[w];
    flip_spins<W>(a, ab);
    flip_spins<W>(b, bb);
    const bool a_open = !det_same<W>(a, ab), b_open = !det_same<W>(b, bb);
    const float h1 = (count_between<W>(a, i1, a1) & 1) ? -hs : hs;  // signed element to (i1, a1)
    const float e1 = fmaf(hab, P.serr_f, 1e-30f);
    const float gx = __fdiv_rn(P.p_single_f, small_f(mallow * v.nok));
    float vf, ev, g;
    if (!a_open) {  // closed v: b is open, H_AB = sqrt(2) <a|H|b>, and P(xb) = P(x)
        vf = h1 * (float)kSqrt2;
        ev = 1.5f * e1 + fabsf(vf) * 0x1p-21f;
        g = gx + gx;
    } else {
        float h2 = 0.f, e2 = 0.f, g2 = 0.f;  // the element to xb and its generation probability
        if (i2 >= 0) {
            h2 = (count_between<W>(a, i2, a2) & 1) ? -hs2 : hs2;
            e2 = fmaf(hab2, P.serr_f, 1e-30f);
            const int c2 = (int)__ldg(P.irrep + (i2 >> 1)) * 2 + (i2 & 1);
            const int c2a = (int)__ldg(P.irrep + (a2 >> 1)) * 2 + (a2 & 1);
            g2 = c2 == c2a ? __fdiv_rn(P.p_single_f, small_f((unsigned)v.cnt[c2] * v.nok)) : 0.f;
        } else {
            unsigned long long hb[W], pb[W];
            int lb = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                hb[w] = a[w] & ~xb[w];
                pb[w] = xb[w] & ~a[w];
                lb += __popcll(hb[w]);
            }
            if (lb == 2) {  // beyond a double both stay 0
                const int bi = select_bit<W>(hb, 0), bj = select_bit<W>(hb, 1);
                const int ba = select_bit<W>(pb, 0), bbo = select_bit<W>(pb, 1);
                h2 = hdouble_f_at<W>(P, a, bi, bj, ba, bbo, keep_policy(), e2);
                g2 = gen_prob_double_f<W>(P, v, tab, bi, bj, ba, bbo);
            }
        }
        const float hb_f = fl_less ? h2 : h1, hbb_f = fl_less ? h1 : h2;
        const float eb = fl_less ? e2 : e1, ebb = fl_less ? e1 : e2;
        if (b_open) {
            vf = hb_f + (float)pair_sign(n_open<W>(b)) * hbb_f;
            ev = eb + ebb + fabsf(vf) * 0x1p-21f;
        } else {
            vf = hb_f * (float)kSqrt2;
            ev = 1.5f * eb + fabsf(vf) * 0x1p-21f;
        }
        g = det_same<W>(xb, x) ? gx : gx + g2;
    }
    const float ah_lo = fabsf(vf) - ev, ah_hi = fabsf(vf) + ev;
    const int n = decide_spawn(__fdiv_rn(ah_lo * P.tau_f, g) * kDown, __fdiv_rn(ah_hi * P.tau_f, g) * kUp, q,
                               P.srange_f);
    if (n == 0) return;
    if (n > 0) {
        emit_spawn<W>(P, v, b, n, vf > 0.f ? 1 : -1, cnt, out);  // |vf| > ev: the sign of H_AB
        return;
    }
    atomicAdd(&P.st->exact_spawn, 1ull);  // undecided by the float bounds
    hphf_exact<W>(P, v, x, xb, b, q + P.d53, true, cnt, out);
}

// One spawning attempt per lane (active lanes only); called by all 32 lanes of a warp.
template <int W, bool TAB, int MODE>
__device__ __forceinline__ void spawn_attempt(const Params &P, const Tables &T, const DetView<W> &v,
                                              const unsigned char *occ, const HeavyTab *tab, const float *rcpf, bool active, unsigned a,
                                              unsigned iter, unsigned long long *cnt, SpawnQueue<W> &out,
                                              bool rtab = false) {
    const unsigned long long pol = keep_policy();
    int i = 0, ao = 0, i1 = 0, a1 = 0, i2 = -1, a2 = -1;
    unsigned mallow = 0;
    unsigned long long q = 0;
    bool pend = false;
    if (active)
        pend = attempt_begin<W, TAB, MODE>(P, T, v, occ, tab, rcpf, a, iter, pol, cnt, out, i, ao, mallow, q, i1, a1, i2, a2,
                                           rtab);
    float hs = 0.f, hab = 0.f;
    single_elements_warp<W>(P, occ, pend, i1, a1, pol, hs, hab);
    if (MODE & 2) {
        float hs2 = 0.f, hab2 = 0.f;
        single_elements_warp<W>(P, occ, pend && i2 >= 0, i2, a2, pol, hs2, hab2);
        if (pend) hphf_single_end<W>(P, v, tab, i, ao, i1, a1, i2, a2, mallow, q, hs, hab, hs2, hab2, cnt, out);
    } else if (pend) {
        attempt_single_end<W>(P, v, occ, i, ao, mallow, q, hs, hab, cnt, out);
    }
}

// ---------------------------------------------------------------------------- death / cloning (Eq. 4)
// r = (tau ((H_ii - E0) - S)) |C|; n = floor(|r|) + [u < frac |r|]; C -= sign(C) n for r >= 0, += for r < 0.
template <int W>
__device__ __forceinline__ int death_step(const Params &P, const DetView<W> &v, float hdf, const double *hd_ptr,
                                          double S, float S_f, unsigned iter, unsigned long long *cnt) {
    const int c = v.c;
    const unsigned ac = (unsigned)(c < 0 ? -c : c);
    unsigned long long u, unused;
    draw2(0u, 3u, v.fp, P.seed, iter, u, unused);
    const float tf = hdf - S_f;
    const float et = fmaf(fabsf(hdf) + fabsf(S_f), 0x1p-22f, 1e-30f);  // >= |(H_ii - E0 - S) - tf|
    const float acf = __uint2float_rn(ac);
    const float at_lo = fabsf(tf) - et, at_hi = fabsf(tf) + et;
    const float r_hi = at_hi * P.tau_death_f * acf * kUp, r_lo = at_lo * P.tau_death_f * acf * kDown;
    const int dec = decide_death(r_lo, r_hi, u);
    int nd;
    bool positive;
    if (dec == 0) {
        return c;
    } else if (dec > 0) {
        nd = dec;
        positive = tf > 0.f;  // r_lo > 0, so at_lo > 0: the sign of tf is the sign of r
    } else {
        atomicAdd(&P.st->exact_death, 1ull);
        double hd = *hd_ptr;
        double r = __dmul_rn(__dmul_rn(P.tau_death, __dsub_rn(hd, S)), (double)ac);
        double arr = fabs(r);
        double fl = floor(arr);
        if (fl >= 2147483647.0) { set_status(P.st, FCIQMC_ERR_NUMERIC); return c; }
        nd = (int)fl + (unit53(u) < __dsub_rn(arr, fl) ? 1 : 0);
        positive = r >= 0.0;
    }
    long long sc = c > 0 ? 1 : -1;
    long long nc;
    if (positive) { nc = (long long)c - sc * nd; cnt[C_DEATH] += (unsigned long long)nd; }
    else { nc = (long long)c + sc * nd; cnt[C_CLONE] += (unsigned long long)nd; }
    if (nc > 2147483647LL || nc < -2147483647LL) { set_status(P.st, FCIQMC_ERR_NUMERIC); return c; }
    return (int)nc;
}

// ---------------------------------------------------------------------------- reductions
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
    return x;
}
__device__ __forceinline__ double warp_sum_f64(double x) {
    for (int o = 16; o > 0; o >>= 1) x = __dadd_rn(x, __shfl_down_sync(0xFFFFFFFFu, x, o));
    return x;
}
// Block-wide sums of NV per-thread counters with one barrier; thread k adds counter k to *dst[k].
template <int NT, int NV>
__device__ __forceinline__ void flush_counters(unsigned long long (&v)[NV], unsigned long long *const (&dst)[NV],
                                               unsigned long long *s_red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        unsigned long long x = warp_sum_u64(v[k]);
        if (lane == 0) s_red[warp * NV + k] = x;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        unsigned long long t = 0;
        for (int w = 0; w < NT / 32; ++w) t += s_red[w * NV + threadIdx.x];
        if (t) atomicAdd(dst[threadIdx.x], t);
    }
}
// Deterministic block sum of an FP64 value (lane tree, then warps in order), returned to thread 0.
template <int NT>
__device__ __forceinline__ double block_sum_f64(double v, double *s_red) {
    v = warp_sum_f64(v);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w) t = __dadd_rn(t, s_red[w]);
    return t;
}

// ---------------------------------------------------------------------------- kernels
// Nearest floats of 1/L for the spawn bound, copied to shared memory.
__device__ __forceinline__ void load_rcpf(const Params &P, float *s_rcpf) {
    for (int k = threadIdx.x; k < 2 * MAXSO + 2; k += blockDim.x) s_rcpf[k] = P.rcpf[k];
}

// MODE bit 0: the run has a permitted space; bit 1: walkers on spin-coupled functions (the code of
// each is compiled in only for runs that use it).
template <int W, int MODE>
__global__ void __launch_bounds__(kTile, FQ_SWEEP_MIN_BLOCKS) k_sweep(Params P) {
    DevState *st = P.st;
    if (st->status) return;
    // dynamic: one SpawnQueue per warp, then the tile's occupied lists (occ_stride bytes each)
    extern __shared__ __align__(16) unsigned char s_queue[];
    unsigned char *const s_occ = s_queue + sizeof(SpawnQueue<W>) * (kTile / 32);
    const int ostride = occ_stride(P.n_elec);
    __shared__ Tables T;
    __shared__ DetView<W> s_dv[kTile];
    __shared__ unsigned s_off[kTile];
    __shared__ unsigned s_wsum[kTile / 32];
    __shared__ float s_rcpf[2 * MAXSO + 2];
    __shared__ unsigned long long s_red[(kTile / 32) * (NCNT + 4)];
    load_tables(P, T);
    load_rcpf(P, s_rcpf);
    const int lb = st->lb, pp = st->pp;
    const long long len = st->list_len;
    const unsigned iter = (unsigned)st->iter;
    const double S = st->shift;
    const float S_f = __double2float_rn(S);
    const unsigned long long *det = P.det[lb];
    const float *hdf = P.hdf[lb];
    const double *hd = P.hd[lb];
    const int *pop_in = P.pop[lb][pp];
    int *pop_out = P.pop[lb][pp ^ 1];
    DetView<W> *heavy = reinterpret_cast<DetView<W> *>(P.heavy);
    const unsigned chunk = st->heavy_chunk ? st->heavy_chunk : (unsigned)kChunk;
    const unsigned heavy_thr = st->heavy_thr ? st->heavy_thr : (unsigned)kHeavy;
    __syncthreads();

    unsigned long long acc[NCNT + 4];  // counters, then nw, nd, d_nw, d_nd
#pragma unroll
    for (int k = 0; k < NCNT + 4; ++k) acc[k] = 0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    SpawnQueue<W> &sq = reinterpret_cast<SpawnQueue<W> *>(s_queue)[warp];
    if (lane == 0) sq.n = 0;
    __syncwarp();

    // tiles are handed out dynamically (one atomic per tile): per-tile costs vary with the populations, and a
    // static assignment left the blocks' last tiles as a tail. The next tile is claimed while this one is
    // worked on (two slots), so a tile takes three block barriers: after the per-determinant work, after the
    // attempt offsets, and after the attempts.
    __shared__ long long s_tile[2];
    __shared__ double s_numw[kTile / 32];
    if (tid == 0) s_tile[0] = (long long)atomicAdd(&st->sweep_next, 1ull) * kTile;
    __syncthreads();
    for (int slot = 0;; slot ^= 1) {
        const long long tb = s_tile[slot];
        if (tb >= len) break;
        double num = 0.0;  // this tile's share of the Eq. 2 numerator
        const long long s = tb + tid;
        unsigned att = 0;
        if (s < len) {
            const int c = __ldcs(pop_in + s);
            if (c == 0) {
                pop_out[s] = 0;
            } else {
                DetView<W> &v = s_dv[tid];
                if (W == 2) {
                    ulonglong2 dd = __ldcs(reinterpret_cast<const ulonglong2 *>(det) + s);
                    v.d[0] = dd.x;
                    v.d[W - 1] = dd.y;
                } else {
                    v.d[0] = __ldcs(det + s);
                }
                const float hf = __ldcs(hdf + s);
                // the determinant's derived words and occupied list, stored when it entered the list
                unsigned char *occ = s_occ + tid * ostride;
                unsigned long long pre[PRE_WORDS];
                {
                    const ulonglong2 *ps = reinterpret_cast<const ulonglong2 *>(P.pre[lb] + s * PRE_WORDS);
                    const ulonglong2 p0 = __ldcs(ps), p1 = __ldcs(ps + 1);
                    pre[0] = p0.x;
                    pre[1] = p0.y;
                    pre[2] = p1.x;
                    pre[3] = p1.y;
                    const unsigned *os = reinterpret_cast<const unsigned *>(P.occa[lb] + s * ostride);
                    for (int k = 0; k < ostride / 4; ++k) reinterpret_cast<unsigned *>(occ)[k] = __ldcs(os + k);
                }
                fill_view<W>(P, v, pre, c);
                const unsigned ac = (unsigned)(c < 0 ? -c : c);
                acc[NCNT] += ac;
                acc[NCNT + 1] += 1;
                unsigned long long xd = 0;
                int diff = 0;
#pragma unroll
                for (int w = 0; w < W; ++w) { xd |= v.d[w] ^ P.ref[w]; diff += __popcll(v.d[w] ^ P.ref[w]); }
                if (xd == 0) st->c0_in = c;
                else if (diff == 2 || diff == 4) {
                    double h0 = h0i<W>(P, v.d);
                    if ((MODE & 2) && n_open<W>(v.d) > 0) h0 = __dmul_rn(h0, kSqrt2);  // closed reference, open function
                    num = __dadd_rn(num, __dmul_rn(h0, (double)c));
                }
                const int nc = death_step<W>(P, v, hf, hd + s, S, S_f, iter, acc);
                pop_out[s] = nc;
                acc[NCNT + 2] += (unsigned long long)((long long)(nc < 0 ? -nc : nc) - (long long)ac);
                if (nc == 0) acc[NCNT + 3] += (unsigned long long)(-1LL);
                // attempts: one per walker; with hybrid walkers the |C| 2^-b walkers rounded stochastically
                // (floor, plus one with the probability of the fraction; draw tag 4)
                unsigned natt = ac;
                if (P.frac_bits) {
                    natt = ac >> P.frac_bits;
                    const unsigned frac = ac & ((1u << P.frac_bits) - 1u);
                    if (frac) {
                        unsigned long long u, unused;
                        draw2(0u, 4u, v.fp, P.seed, iter, u, unused);
                        if (unit53(u) < __dmul_rn((double)frac, P.frac_scale)) ++natt;
                    }
                }
                acc[C_ATTEMPTS] += natt;
                if (natt > heavy_thr) {
                    // heavily populated determinant: a record for k_heavy, whose warps take chunks of `chunk`
                    // attempts; record index and first chunk are claimed by one atomic, so the first
                    // chunks are nondecreasing in the record index
                    acc[C_HEAVY] += natt;
                    const unsigned nch = (natt + chunk - 1) / chunk;
                    const unsigned long long old = atomicAdd(&st->heavy_packed, (1ull << 40) | nch);
                    const unsigned long long hidx = old >> 40;
                    if (hidx >= (unsigned long long)P.heavy_cap) {
                        set_status(st, FCIQMC_ERR_CAPACITY);
                    } else {
                        heavy[hidx] = v;
                        for (int k = 0; k < P.n_elec; ++k) P.heavy_occ[hidx * MAXN + k] = occ[k];
                        P.heavy_base[hidx] = (unsigned)(old & ((1ull << 40) - 1ull));
                        P.heavy_att[hidx] = natt;
                    }
                } else {
                    att = natt;
                }
            }
        }
        // exclusive scan of attempts over the tile: within each warp, then every thread adds the totals of the
        // warps before its own; the tile's numerator from the warps' sums added in warp order
        unsigned x = att;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        const double wnum = warp_sum_f64(num);
        if (lane == 31) s_wsum[warp] = x;
        if (lane == 0) s_numw[warp] = wnum;
        if (tid == 0) s_tile[slot ^ 1] = (long long)atomicAdd(&st->sweep_next, 1ull) * kTile;
        __syncthreads();
        unsigned woff = 0, total = 0;
#pragma unroll
        for (int w = 0; w < kTile / 32; ++w) {
            const unsigned ws = s_wsum[w];
            woff += w < warp ? ws : 0u;
            total += ws;
        }
        s_off[tid] = x - att + woff;
        if (tid == 0) {
            // the tile's numerator, summed in a fixed order, so the run's total does not depend on which block
            // took which tile
            double bs = 0.0;
            for (int w = 0; w < kTile / 32; ++w) bs = __dadd_rn(bs, s_numw[w]);
            if (FQ_CHECK(tb / kTile < P.tiles_cap, P.st)) P.partial[tb / kTile] = bs;
        }
        __syncthreads();
        for (unsigned base = 0; base < total; base += kTile) {
            const unsigned k = base + tid;
            const bool act = k < total;
            int lo = 0;
            if (act) {
                int hi = kTile - 1;  // last d with s_off[d] <= k
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (s_off[mid] <= k) lo = mid; else hi = mid - 1;
                }
            }
            spawn_attempt<W, false, MODE>(P, T, s_dv[lo], s_occ + lo * ostride, nullptr, s_rcpf, act, k - s_off[lo],
                                          iter, acc, sq);
            flush_queue<W>(P, sq, false, T.map1);
        }
        __syncthreads();  // the tile's views and offsets are free again; the next tile's index is visible
    }
    flush_queue<W>(P, sq, true, T.map1);
    unsigned long long *const dst[NCNT + 4] = {&st->cnt[0], &st->cnt[1], &st->cnt[2], &st->cnt[3], &st->cnt[4],
                                               &st->cnt[5], &st->cnt[6], &st->cnt[7], &st->cnt[8], &st->cnt[9],
                                               &st->nw_in, &st->nd_in, &st->d_nw, &st->d_nd};
    flush_counters<kTile, NCNT + 4>(acc, dst, s_red);
}

// Attempts of heavily populated determinants, split into chunks of kChunk attempts: warps take batches of
// consecutive chunks from a counter (guided: a share of what is left, at most kChunkBatch), so a warp meets
// few determinants, and build a determinant's tables once when they reach it.
template <int W, int MODE>
__global__ void __launch_bounds__(kTile, 4) k_heavy(Params P) {
    DevState *st = P.st;
    if (st->status) return;
    extern __shared__ __align__(16) unsigned char s_queue[];  // one SpawnQueue per warp
    constexpr int NW = kTile / 32;
    __shared__ Tables T;
    __shared__ DetView<W> s_v[NW];
    __shared__ HeavyTab s_tab[NW];
    __shared__ float s_rcpf[2 * MAXSO + 2];
    __shared__ unsigned long long s_red[NW * NCNT];
    load_tables(P, T);
    load_rcpf(P, s_rcpf);
    const unsigned long long packed = st->heavy_packed;
    const long long nh = min((long long)(packed >> 40), P.heavy_cap);
    const unsigned long long nch = nh > 0 ? (packed & ((1ull << 40) - 1ull)) : 0ull;
    const unsigned iter = (unsigned)st->iter;
    const unsigned chunk = st->heavy_chunk ? st->heavy_chunk : (unsigned)kChunk;
    const DetView<W> *heavy = reinterpret_cast<const DetView<W> *>(P.heavy);
    unsigned long long cnt[NCNT];
#pragma unroll
    for (int k = 0; k < NCNT; ++k) cnt[k] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long cur = -1;
    DetView<W> &v = s_v[warp];
    HeavyTab &tab = s_tab[warp];
    SpawnQueue<W> &sq = reinterpret_cast<SpawnQueue<W> *>(s_queue)[warp];
    if (lane == 0) sq.n = 0;
    __syncwarp();
    // warps take batches of consecutive chunks from a counter: consecutive chunks mostly belong to one
    // determinant, so a warp still builds few tables, and no warp is left with a tail of work
    unsigned long long q = 0, qend = 0;
    for (;;) {
        bool fresh = false;
        if (q >= qend) {
            // guided self-scheduling: a share of what is left, so batches are long while much is left (few
            // determinant switches) and single chunks at the end (no tail); lane 0 decides, so every lane of
            // the warp holds the same batch
            unsigned long long b = 0, size = 1;
            if (lane == 0) {
                const unsigned long long taken = *(volatile unsigned long long *)&st->heavy_next;
                const unsigned long long nwarps = (unsigned long long)gridDim.x * NW;
                if (taken < nch)
                    size = max(1ull, min((unsigned long long)kChunkBatch, (nch - taken) / (2ull * nwarps)));
                b = atomicAdd(&st->heavy_next, size);
            }
            b = __shfl_sync(0xFFFFFFFFu, b, 0);
            size = __shfl_sync(0xFFFFFFFFu, size, 0);
            if (b >= nch) break;
            q = b;
            qend = min(b + size, nch);
            fresh = true;
        }
        // record holding chunk q: last record whose first chunk is <= q (searched at the start of a batch)
        long long r;
        if (cur < 0 || fresh) {
            long long lo = 0, hi = nh - 1;
            while (lo < hi) {
                const long long mid = (lo + hi + 1) >> 1;
                if ((unsigned long long)P.heavy_base[mid] <= q) lo = mid; else hi = mid - 1;
            }
            r = lo;
        } else {
            r = cur;
            while (r + 1 < nh && (unsigned long long)P.heavy_base[r + 1] <= q) ++r;
        }
        if (r != cur) {
            const unsigned long long *src = reinterpret_cast<const unsigned long long *>(heavy + r);
            unsigned long long *dstv = reinterpret_cast<unsigned long long *>(&v);
            for (int k = lane; k < (int)(sizeof(DetView<W>) / 8); k += 32) dstv[k] = src[k];
            for (int k = lane; k < P.n_elec; k += 32) tab.occ[k] = P.heavy_occ[r * MAXN + k];
            __syncwarp();
            build_heavy_tab<W>(P, T, v, tab, lane);
            cur = r;
        }
        const unsigned a0 = (unsigned)(q - P.heavy_base[r]) * chunk;
        const unsigned a1 = min(a0 + chunk, P.heavy_att[r]);
        const bool rtab = P.ref_tab && v.isref;
        for (unsigned base = a0; base < a1; base += 32) {
            const unsigned a = base + lane;
            spawn_attempt<W, true, MODE>(P, T, v, tab.occ, &tab, s_rcpf, a < a1, a, iter, cnt, sq, rtab);
            flush_queue<W>(P, sq, false, T.map1);
        }
        __syncwarp();
        ++q;
    }
    flush_queue<W>(P, sq, true, T.map1);
    unsigned long long *const dst[NCNT] = {&st->cnt[0], &st->cnt[1], &st->cnt[2], &st->cnt[3], &st->cnt[4],
                                           &st->cnt[5], &st->cnt[6], &st->cnt[7], &st->cnt[8], &st->cnt[9]};
    cnt[C_ATTEMPTS] = 0;  // attempts are counted by the sweep
    flush_counters<kTile, NCNT>(cnt, dst, s_red);
}

}  // namespace fq
