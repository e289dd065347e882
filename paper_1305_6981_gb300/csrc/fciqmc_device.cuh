// Device building blocks of the FCIQMC walker cycle (sm_103a).
//
// Determinants are W uint64 words (W = 1 or 2); spin orbital k is bit k & 63
// of word k >> 6, spatial orbital k >> 1, spin k & 1 (Sec. III bit strings).
// Floating-point expressions that decide walker counts are written with
// explicit round-to-nearest intrinsics (__dadd_rn, __dmul_rn, ...), which the
// compiler never contracts into FMAs, so the values are the IEEE results of
// the operation order stated next to each one.
#pragma once

#include <cstdint>
#include <math_constants.h>

#include "fciqmc.h"

namespace fq {

constexpr int MAXW = 2;
constexpr int MAXN = 64;     // electrons
constexpr int MAXSO = 128;   // spin orbitals
constexpr int NCLASS = 16;   // 8 irreps x 2 spins
constexpr int MAXPAIRS = MAXN * (MAXN - 1) / 2;
constexpr unsigned long long EMPTY = ~0ull;
constexpr int NCNT = 10;     // per-iteration counters, same order as fciqmc_row from `attempts`
constexpr int MAXPARTS = 64; // partitions of a hash-partitioned run

// ---------------------------------------------------------------------------
// Shared state of one run, in device memory.
struct DevState {
    long long iter;            // iterations completed (keys the random numbers of the next one)
    double shift;
    int vary, n_since;
    long long nw_prev;
    int lb, pp;                // active list buffer, population parity
    long long list_len;        // slots in use (live + vacated) in the active list
    unsigned long long claim;  // slot claim counter during annihilation
    int status;                // sticky error status (0 = OK)
    int compact_pending;
    unsigned long long n_merged;
    unsigned long long heavy_packed;  // (heavy determinants << 40) | chunks, claimed together
    unsigned long long nw_in, nd_in;
    long long c0_in;
    unsigned long long d_nw, d_nd;  // two's-complement signed changes
    unsigned long long cnt[NCNT];
    unsigned long long new_len;
    unsigned long long exact_spawn, exact_death;  // exact-path evaluations (diagnostics)
    long long hist_n;
    long long compactions;
    // last estimator sweep
    unsigned long long est_nw, est_nd;
    long long est_c0;
    double est_num;
    int check_bad;             // set by the check of a list being loaded
    unsigned long long n_new;  // determinants placed in new slots this iteration (diagonal elements pending)
    unsigned long long sweep_next;  // next sweep tile to hand out (tiles are taken dynamically by the blocks)
    unsigned long long heavy_next;  // next batch of heavy chunks to hand out (taken dynamically by the warps)
    unsigned heavy_chunk;           // attempts per heavy chunk this iteration (0: the smallest size)
    unsigned heavy_thr;             // attempts above which a determinant takes the heavy path (0: kHeavy)
    unsigned long long ob_n[MAXPARTS];  // partitioned runs: spawns routed to each other partition this iteration
};

// One double excitation of the reference determinant as the generator selects it (pair, good a, b),
// with its spawning probability p = tau |H| / P_gen in the FP64 order of the exact path: p_lo <= p <= p_hi
// as floats, ps = p with the sign of H (0 when H = 0), and the spin orbitals i < j (occupied), a, b.
struct RefExc {
    float p_lo, p_hi;
    double ps;
    unsigned char i, j, a, b;
    unsigned pad;
};

// Uniform parameters of a run, passed by value to every kernel.
struct Params {
    int n_elec, n_orb, n_so, npairs, n_irrep_used;
    int init_thr;
    unsigned seed;
    unsigned long long d53;
    double tau, cs, cd, E0, c_shift;
    float tau_f, cdn_f, d53_f;             // nearest floats of tau, cd * npairs and d53
    float cs_f, srange_f;                  // nearest floats of cs and 2^53 - d53
    float serr_f;                          // relative error bound of the float single-excitation element
    double d53_d;                          // (double)d53, exact
    int period;
    int sweep_grid;                        // blocks of k_sweep
    long long tiles_cap;                   // partial[0, tiles_cap): the Eq. 2 numerator of each sweep tile;
                                           // partial[tiles_cap, + kTileSums): their fixed-order range sums
    int idx_stride;                        // 64-bit words per index entry
    long long target;
    // read-only tables
    const double *h;        // n_orb x n_orb
    const double *eri;      // packed 8-fold
    const float *eri_f;     // same, rounded to float
    const float *h_f;       // h rounded to float
    const double *wpair;    // [2][n_orb][n_orb]: [0] opposite spin (pp|qq), [1] same spin (pp|qq) - (pq|qp)
    const unsigned long long *map1;   // n_so, orbital map of Algorithm 1
    const unsigned long long *cmask;  // [NCLASS][MAXW] spin orbitals of each (irrep, spin) class
    const unsigned long long *unionm; // [2][256][MAXW] spin orbitals of spin s in the irreps of an 8-bit set
    const unsigned char *irrep;       // n_orb
    const unsigned short *pairs;      // npairs: (i | j << 8), i < j electron indices
    const double *recip;              // recip[L] = 1.0 / L, L < 2 * MAXSO + 2
    const float *rcpf;                // nearest float of 1 / L
    unsigned long long ref[MAXW];
    const unsigned char *ref_occ;     // n_elec ascending spin orbitals of the reference
    // permitted space: bit 0 excitation limit, bit 1 seniority limit, bit 2 frozen spin orbitals
    int space, max_exc, max_sen;
    unsigned long long froz_occ[MAXW], froz_emp[MAXW];
    int hphf;                         // walkers on spin-coupled functions (Sec. VI C)
    double p_single_d, p_double_d;    // P_single, P_double as realised by the draw
    // the reference's double excitations, for runs with neither a permitted space nor spin coupling:
    // pair k -> (first good-a slot << 8) | G; good-a slot -> (first excitation << 7) | M^(b|a)
    const unsigned *ref_pinfo;
    const unsigned *ref_off2;
    const RefExc *ref_exc;
    int ref_tab;                      // 1 when those tables are built
    float p_double_f, p_single_f;     // nearest floats of P_double, P_single
    // main list, two buffers for compaction, two population arrays per buffer
    unsigned long long *det[2];
    double *hd[2];
    float *hdf[2];
    int *pop[2][2];
    long long cap;
    // hash index: det -> slot
    unsigned long long *idx;
    long long idx_cap;
    int idx_bits;
    // spawn merge table
    unsigned long long *mt;
    long long mt_cap;
    int mt_bits;
    unsigned *merged;
    void *heavy;                      // DetView records of heavily populated determinants
    unsigned char *heavy_occ;         // their occupied lists (MAXN bytes each)
    unsigned *heavy_base;             // first chunk of each (nondecreasing in the record index)
    unsigned *heavy_att;              // attempts of each
    long long heavy_cap;
    long long heavy_warps;            // warps of a k_heavy launch (chooses the chunk size)
    long long sweep_blocks;           // blocks of a k_sweep launch (chooses the heavy threshold)
    double *partial;
    fciqmc_row *hist;
    long long hist_cap;
    DevState *st;
    // hash-partitioned runs (Sec. V A): this list holds the determinants whose fingerprint mod n_parts is
    // part; spawns onto the others go to outbox[dest][ob_cap] (entries of Stride<W> words: key, payload)
    int n_parts, part;
    unsigned long long *outbox;
    long long ob_cap;
    long long n_eri, ref_n;           // packed ERIs; entries of the reference's table (debug checks)
    // real/integer hybrid walkers: populations in units of 2^-frac_bits walkers; tau, tau_f, cs, cd, cs_f and
    // cdn_f above carry the factor 2^frac_bits (spawn counts in units), death uses tau_death
    int frac_bits;
    double frac_scale;                // 2^-frac_bits
    int occ_units;                    // occupation threshold in units (1: none)
    double tau_death;
    float tau_death_f;
    // per slot of each list buffer, what the spawning kernels need of a determinant beyond its bits, derived
    // once when it enters the list: PRE_WORDS words, and its occupied spin orbitals (ostride bytes)
    unsigned long long *pre[2];
    unsigned char *occa[2];
    int ostride;
};

__device__ __forceinline__ void set_status(DevState *st, int code) { atomicCAS(&st->status, 0, code); }

// Debug build (-DFCIQMC_DEBUG): indices that the algorithm keeps in range by construction are checked before
// the access they guard; a violation sets FCIQMC_ERR_BOUNDS (sticky like the other device errors) and the
// access is skipped. In the normal build the check is the constant true.
#ifdef FCIQMC_DEBUG
#define FQ_CHECK(cond, st) ((cond) ? true : (::fq::set_status((st), FCIQMC_ERR_BOUNDS), false))
#else
#define FQ_CHECK(cond, st) true
#endif

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Two 64-bit words keyed by (seed, iteration), counter (attempt, tag, fingerprint).
__device__ __forceinline__ void draw2(unsigned a, unsigned tag, unsigned long long fp, unsigned seed, unsigned iter,
                                      unsigned long long &w0, unsigned long long &w1) {
    uint4 o = philox4x32_10(make_uint4(a, tag, (unsigned)fp, (unsigned)(fp >> 32)), make_uint2(seed, iter));
    w0 = (unsigned long long)o.x | ((unsigned long long)o.y << 32);
    w1 = (unsigned long long)o.z | ((unsigned long long)o.w << 32);
}

// The choices of an attempt are the successive digits of its 75-bit choice word R = rh 2^11 + rl (rl < 2^11)
// in mixed radix: k = floor(R n / 2^75), uniform in [0, n), and R becomes R n mod 2^75. With
// S = rh n + floor(rl n / 2^11) (at most 85 bits), k = floor(S / 2^64), the new rh = S mod 2^64 and the new
// rl = rl n mod 2^11. Every radix is below 2^12 (at most MAXPAIRS = 2016 electron pairs, MAXSO spin
// orbitals), so rl n fits 32 bits and (rh >> 32) n + 2^33 fits 64.
static_assert(MAXPAIRS < 4096 && MAXSO < 4096, "choice radices must stay below 2^12");
__device__ __forceinline__ unsigned rank_next(unsigned long long &rh, unsigned &rl, unsigned n) {
    const unsigned long long lo = (unsigned long long)(unsigned)rh * n;
    const unsigned long long hi = (unsigned long long)(unsigned)(rh >> 32) * n;
    const unsigned q = rl * n;
    const unsigned long long s0 = (lo & 0xFFFFFFFFull) + (q >> 11);
    const unsigned long long sh = hi + (lo >> 32) + (s0 >> 32);
    rh = (sh << 32) | (s0 & 0xFFFFFFFFull);
    rl = q & 0x7FFu;
    return (unsigned)(sh >> 32);
}

// ---------------------------------------------------------------------------
// bit-string helpers
// Word selection by comparison rather than by a computed index keeps W-word arrays in registers.
template <int W>
__device__ __forceinline__ int bit_of(const unsigned long long (&d)[W], int k) {
    const unsigned long long w = (W == 1 || k < 64) ? d[0] : d[W - 1];
    return (int)((w >> (k & 63)) & 1ull);
}
template <int W>
__device__ __forceinline__ void flip(unsigned long long (&d)[W], int k) {
    const unsigned long long b = 1ull << (k & 63);
    if (W == 1 || k < 64) d[0] ^= b;
    else d[W - 1] ^= b;
}
template <int W>
__device__ __forceinline__ void clear_bit(unsigned long long (&d)[W], int k) {
    const unsigned long long b = ~(1ull << (k & 63));
    if (W == 1 || k < 64) d[0] &= b;
    else d[W - 1] &= b;
}
// bits [0, n) of a 64-bit word, n in [0, 64]
__device__ __forceinline__ unsigned long long low_bits(int n) {
    return n >= 64 ? ~0ull : ((1ull << n) - 1ull);
}
// occupied spin orbitals strictly between k and l
template <int W>
__device__ __forceinline__ int count_between(const unsigned long long (&d)[W], int k, int l) {
    int lo = min(k, l) + 1, hi = max(k, l);
    int c = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        int a = max(lo - 64 * w, 0), b = min(hi - 64 * w, 64);
        if (b > a) c += __popcll(d[w] & low_bits(b) & ~low_bits(a));
    }
    return c;
}
// position of the k-th (0-based) set bit of a word (k < popc(x)): the half holding it is chosen by a
// population count, down to single bits; one word is searched, on 32-bit operations
__device__ __forceinline__ int select32(unsigned x, int k) {
    int pos = 0, c;
    c = __popc(x & 0xFFFFu);
    if (k >= c) { k -= c; x >>= 16; pos += 16; }
    c = __popc(x & 0xFFu);
    if (k >= c) { k -= c; x >>= 8; pos += 8; }
    c = __popc(x & 0xFu);
    if (k >= c) { k -= c; x >>= 4; pos += 4; }
    c = __popc(x & 0x3u);
    if (k >= c) { k -= c; x >>= 2; pos += 2; }
    return pos + (k >= (int)(x & 1u) ? 1 : 0);
}
__device__ __forceinline__ int select64(unsigned long long x, int k) {
    const unsigned lo = (unsigned)x, hi = (unsigned)(x >> 32);
    const int c = __popc(lo);
    const bool up = k >= c;
    return (up ? 32 : 0) + select32(up ? hi : lo, up ? k - c : k);
}
template <int W>
__device__ __forceinline__ int select_bit(const unsigned long long (&m)[W], int k) {
    if (W == 1) return select64(m[0], k);
    const int c0 = __popcll(m[0]);
    const bool up = k >= c0;
    return (up ? 64 : 0) + select64(up ? m[W - 1] : m[0], up ? k - c0 : k);
}
template <int W>
__device__ __forceinline__ bool det_eq(const unsigned long long (&a)[W], const unsigned long long *b) {
    bool e = true;
#pragma unroll
    for (int w = 0; w < W; ++w) e = e && (a[w] == b[w]);
    return e;
}

// Algorithm 1 (Sec. V) over the occupied spin orbitals in ascending order, electrons counted from 1, uint64
// wraparound: the fingerprint that keys the random numbers and, mod the partition count, a determinant's
// partition (map1: the orbital map).
template <int W>
__device__ __forceinline__ unsigned long long fingerprint(const unsigned long long (&d)[W], const unsigned long long *map1) {
    unsigned long long h = 0;
    unsigned n = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        unsigned long long m = d[w];
        while (m) {
            const int k = 64 * w + __ffsll((long long)m) - 1;
            h = 1099511628211ull * h + map1[k] * (unsigned long long)(++n);
            m &= m - 1;
        }
    }
    return h;
}

// Permitted space (Sec. VI): at most max_exc reference spin orbitals empty, at most max_sen spatial
// orbitals singly occupied (spin orbitals 2p and 2p + 1 share a word), frozen spin orbitals kept.
template <int W>
__device__ __forceinline__ bool in_space(const Params &P, const unsigned long long (&d)[W]) {
    int exc = 0, sen = 0;
    bool ok = true;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        exc += __popcll(P.ref[w] & ~d[w]);
        sen += __popcll((d[w] ^ (d[w] >> 1)) & 0x5555555555555555ull);
        ok = ok && (d[w] & P.froz_emp[w]) == 0ull && (~d[w] & P.froz_occ[w]) == 0ull;
    }
    if (P.space & 1) ok = ok && exc <= P.max_exc;
    if (P.space & 2) ok = ok && sen <= P.max_sen;
    return ok;
}

// ---------------------------------------------------------------------------
// integrals
__device__ __forceinline__ int pidx(int p, int q) { return p >= q ? p * (p + 1) / 2 + q : q * (q + 1) / 2 + p; }
__device__ __forceinline__ int eidx(int p, int q, int r, int s) {
    int a = pidx(p, q), b = pidx(r, s);
    return a >= b ? a * (a + 1) / 2 + b : b * (b + 1) / 2 + a;
}
__device__ __forceinline__ double eri_d(const Params &P, int p, int q, int r, int s) {
    return __ldg(P.eri + eidx(p, q, r, s));
}
// L2 policy that keeps the integral tables resident while the walker list streams past them.
__device__ __forceinline__ unsigned long long keep_policy() {
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ float ld_keep(const float *p, unsigned long long pol) {
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float eri_f(const Params &P, int p, int q, int r, int s, unsigned long long pol) {
    const int k = eidx(p, q, r, s);
    if (!FQ_CHECK(k >= 0 && k < P.n_eri, P.st)) return 0.f;
    return ld_keep(P.eri_f + k, pol);
}

// Slater-Condon, single i -> a from source d (occupied list occ of d), exact FP64 in ascending order.
template <int W>
__device__ double hij_single(const Params &P, const unsigned long long (&d)[W], const unsigned char *occ, int i, int a) {
    int I = i >> 1, A = a >> 1;
    double v = __ldg(P.h + I * P.n_orb + A);
    for (int x = 0; x < P.n_elec; ++x) {
        int j = occ[x];
        if (j == i) continue;
        int J = j >> 1;
        v = __dadd_rn(v, eri_d(P, I, A, J, J));
        if ((j & 1) == (i & 1)) v = __dsub_rn(v, eri_d(P, I, J, J, A));
    }
    return (count_between<W>(d, i, a) & 1) ? -v : v;
}

// Parity of i -> a then j -> b (i < j, a < b) applied to d.
template <int W>
__device__ __forceinline__ int double_parity(const unsigned long long (&d)[W], int i, int j, int a, int b) {
    unsigned long long t[W];
#pragma unroll
    for (int w = 0; w < W; ++w) t[w] = d[w];
    int par = count_between<W>(t, i, a);
    flip<W>(t, i);
    flip<W>(t, a);
    par += count_between<W>(t, j, b);
    return par & 1;
}

// Slater-Condon, double (i<j) -> (a<b), exact FP64: 0 + (ia|jb) - (ib|ja) with spin deltas.
template <int W>
__device__ __forceinline__ double hij_double(const Params &P, const unsigned long long (&d)[W], int i, int j, int a, int b) {
    double v = 0.0;
    if ((i & 1) == (a & 1) && (j & 1) == (b & 1)) v = __dadd_rn(v, eri_d(P, i >> 1, a >> 1, j >> 1, b >> 1));
    if ((i & 1) == (b & 1) && (j & 1) == (a & 1)) v = __dsub_rn(v, eri_d(P, i >> 1, b >> 1, j >> 1, a >> 1));
    return double_parity<W>(d, i, j, a, b) ? -v : v;
}

// <D|H|D_0> from the reference side (projected-energy numerator, Eq. 2); 0 beyond doubles.
template <int W>
__device__ double h0i(const Params &P, const unsigned long long (&d)[W]) {
    unsigned long long ref[W], holes[W], parts[W];
    int nd = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        ref[w] = P.ref[w];
        holes[w] = ref[w] & ~d[w];
        parts[w] = d[w] & ~ref[w];
        nd += __popcll(holes[w]) + __popcll(parts[w]);
    }
    if (nd == 2) {
        int i = select_bit<W>(holes, 0), a = select_bit<W>(parts, 0);
        return hij_single<W>(P, ref, P.ref_occ, i, a);
    }
    if (nd == 4) {
        int i = select_bit<W>(holes, 0), j = select_bit<W>(holes, 1);
        int a = select_bit<W>(parts, 0), b = select_bit<W>(parts, 1);
        return hij_double<W>(P, ref, i, j, a, b);
    }
    return 0.0;
}

// ---------------------------------------------------------------------------
// spin-coupled functions (Sec. VI C). For M_s = 0 the spin flip F maps |D> to pi(D) |Dbar>, Dbar with spin
// orbitals 2p and 2p + 1 exchanged, pi(D) = (-1)^(doubly occupied spatial orbitals); F commutes with H. A
// function is |D> (closed shell) or (|D> + sigma pi(D) |Dbar>) / sqrt(2), sigma = pi(reference), stored
// on the smaller of D, Dbar; sigma pi(D) = (-1)^(n_open / 2).
constexpr double kSqrt2 = 0x1.6a09e667f3bcdp+0;  // sqrt(2) rounded to nearest
constexpr unsigned long long kEven = 0x5555555555555555ull;

template <int W>
__device__ __forceinline__ void flip_spins(const unsigned long long (&d)[W], unsigned long long (&o)[W]) {
#pragma unroll
    for (int w = 0; w < W; ++w) o[w] = ((d[w] & kEven) << 1) | ((d[w] >> 1) & kEven);
}
template <int W>
__device__ __forceinline__ int n_open(const unsigned long long (&d)[W]) {
    int c = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) c += __popcll((d[w] ^ (d[w] >> 1)) & kEven);
    return c;
}
template <int W>
__device__ __forceinline__ bool det_less(const unsigned long long (&a)[W], const unsigned long long (&b)[W]) {
    if (W == 2 && a[W - 1] != b[W - 1]) return a[W - 1] < b[W - 1];
    return a[0] < b[0];
}
template <int W>
__device__ __forceinline__ bool det_same(const unsigned long long (&a)[W], const unsigned long long (&b)[W]) {
    bool e = true;
#pragma unroll
    for (int w = 0; w < W; ++w) e = e && a[w] == b[w];
    return e;
}
__device__ __forceinline__ double pair_sign(int nopen) { return (nopen / 2) % 2 ? -1.0 : 1.0; }

// <dst|H|src> for a single or double difference, evaluated from the source side; 0 otherwise
// (occ: the source's ascending occupied list, for the spectator sum of a single).
template <int W>
__device__ double hij_any(const Params &P, const unsigned long long (&src)[W], const unsigned char *occ,
                          const unsigned long long (&dst)[W]) {
    unsigned long long holes[W], parts[W];
    int nd = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        holes[w] = src[w] & ~dst[w];
        parts[w] = dst[w] & ~src[w];
        nd += __popcll(holes[w]);
    }
    if (nd == 1) return hij_single<W>(P, src, occ, select_bit<W>(holes, 0), select_bit<W>(parts, 0));
    if (nd == 2)
        return hij_double<W>(P, src, select_bit<W>(holes, 0), select_bit<W>(holes, 1), select_bit<W>(parts, 0),
                             select_bit<W>(parts, 1));
    return 0.0;
}

// Diagonal: sum_p h_pp (ascending) then, for p < q ascending, the pair term
// (pp|qq) - delta_spin (pq|qp) added to the running sum. w: wpair table in shared memory.
template <int W>
__device__ double hdiag(const Params &P, const unsigned long long (&d)[W], const double *w, const double *hdiag_tab) {
    const int M = P.n_orb;
    double v = 0.0;
#pragma unroll
    for (int wa = 0; wa < W; ++wa) {
        unsigned long long m = d[wa];
        while (m) {
            int k = 64 * wa + __ffsll((long long)m) - 1;
            m &= m - 1;
            v = __dadd_rn(v, hdiag_tab[k >> 1]);
        }
    }
#pragma unroll
    for (int wa = 0; wa < W; ++wa) {
        unsigned long long m = d[wa];
        while (m) {
            int p = 64 * wa + __ffsll((long long)m) - 1;
            m &= m - 1;
            const double *row_same = w + M * M + (p >> 1) * M;
            const double *row_diff = w + (p >> 1) * M;
            // q > p: the rest of this word, then the following words
            unsigned long long m2 = m;
            int wb = wa;
            while (true) {
                while (m2) {
                    int q = 64 * wb + __ffsll((long long)m2) - 1;
                    m2 &= m2 - 1;
                    double t = ((p & 1) == (q & 1)) ? row_same[q >> 1] : row_diff[q >> 1];
                    v = __dadd_rn(v, t);
                }
                if (++wb >= W) break;
                m2 = d[wb];
            }
        }
    }
    return v;
}

// <Phi_d|H|Phi_d> of a stored spin-coupled function: H_dd + sigma pi_d <d|H|dbar>, the second term only
// for two open shells (d and dbar then differ by a double excitation).
template <int W>
__device__ double hphf_hdiag(const Params &P, const unsigned long long (&d)[W], const double *w, const double *hdiag_tab) {
    double v = hdiag<W>(P, d, w, hdiag_tab);
    const int no = n_open<W>(d);
    if (no == 2) {
        unsigned long long db[W];
        flip_spins<W>(d, db);
        v = __dadd_rn(v, __dmul_rn(pair_sign(no), hij_any<W>(P, d, nullptr, db)));
    }
    return v;
}

// ---------------------------------------------------------------------------
// hash tables
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
    x ^= x >> 31;
    x *= 0x7FB5D329728EA185ull;
    x ^= x >> 27;
    x *= 0x81DADEF4BC2DD44Dull;
    x ^= x >> 33;
    return x;
}
template <int W>
__device__ __forceinline__ unsigned long long table_hash(const unsigned long long (&d)[W], unsigned long long salt) {
    unsigned long long x = mix64(d[0] ^ salt);
    if (W == 2) x = mix64(x ^ (d[W - 1] * 0x9E3779B97F4A7C15ull));
    return x;
}

__device__ __forceinline__ void cas128(unsigned long long *addr, unsigned long long c0, unsigned long long c1,
                                       unsigned long long n0, unsigned long long n1, unsigned long long &o0,
                                       unsigned long long &o1) {
    asm volatile(
        "{\n\t.reg .b128 c, n, o;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 n, {%4, %5};\n\t"
        "atom.global.cas.b128 o, [%6], c, n;\n\t"
        "mov.b128 {%0, %1}, o;\n\t}"
        : "=l"(o0), "=l"(o1)
        : "l"(c0), "l"(c1), "l"(n0), "l"(n1), "l"(addr)
        : "memory");
}

// Atomically claim an EMPTY key slot for `key` or report what is there: returns true if the slot now
// holds `key` (claimed by us when *claimed is set).
template <int W>
__device__ __forceinline__ bool claim_key(unsigned long long *e, const unsigned long long (&key)[W], bool &claimed) {
    claimed = false;
    if (W == 1) {
        unsigned long long old = atomicCAS(e, EMPTY, key[0]);
        if (old == EMPTY) { claimed = true; return true; }
        return old == key[0];
    } else {
        unsigned long long o0, o1;
        cas128(e, EMPTY, EMPTY, key[0], key[W - 1], o0, o1);
        if (o0 == EMPTY && o1 == EMPTY) { claimed = true; return true; }
        return o0 == key[0] && o1 == key[W - 1];
    }
}

// Volatile read of a key; `maybe_torn` is set when some word is still EMPTY (another thread may be
// in the middle of writing it), in which case only an atomic CAS can tell what is there.
template <int W>
__device__ __forceinline__ int probe_key(const unsigned long long *e, const unsigned long long (&key)[W]) {
    // 0: different key, 1: our key, 2: EMPTY or possibly being written
    unsigned long long k0 = *(volatile const unsigned long long *)e;
    if (W == 1) return k0 == key[0] ? 1 : (k0 == EMPTY ? 2 : 0);
    unsigned long long k1 = *(volatile const unsigned long long *)(e + 1);
    if (k0 == key[0] && k1 == key[W - 1]) return 1;
    if (k0 == EMPTY || k1 == EMPTY) return 2;
    return 0;
}

// Index/merge entry strides in 64-bit words (key words + one payload word, padded to a power of two)
template <int W>
struct Stride { static constexpr int v = (W == 1) ? 2 : 4; };

// Warp-aggregated append: all 32 lanes must call it. Returns the position for lanes with want, else -1.
__device__ __forceinline__ long long warp_append(unsigned long long *ctr, bool want) {
    const unsigned full = 0xFFFFFFFFu;
    unsigned m = __ballot_sync(full, want);
    if (m == 0) return -1;
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(ctr, (unsigned long long)__popc(m));
    base = __shfl_sync(full, base, leader);
    if (!want) return -1;
    return (long long)(base + __popc(m & ((1u << lane) - 1u)));
}



}  // namespace fq
