// Kernels of one FCIQMC iteration after spawning (annihilation, finish, compaction) and of loading,
// reading back and setting up a run. Included by the host translation unit only; the spawning kernels
// are in fciqmc_kernels.cuh.
#pragma once

#include "fciqmc_kernels.cuh"

namespace fq {

// New determinants get a slot, their population and an index entry here; their diagonal elements are
// computed by k_new_diag over the list of new slots, where every lane of a warp has one (inserting lanes
// are a minority of each warp here, and H_ii is a long FP64 sum).
template <int W>
__global__ void __launch_bounds__(256) k_annihilate(Params P) {
    __shared__ unsigned long long s_red[(256 / 32) * 4];
    DevState *st = P.st;
    if (st->status) return;
    constexpr int S = Stride<W>::v;
    const unsigned long long nm = st->n_merged;
    const long long len = st->list_len;
    // every block sees the same values, so either all blocks proceed or none changes anything
    if (nm > (unsigned long long)(P.mt_cap / 4 * 3) || (long long)nm + len > P.cap ||
        (long long)nm + len > P.idx_cap / 4 * 3) {
        set_status(st, FCIQMC_ERR_CAPACITY);
        return;
    }
    const int lb = st->lb, pp = st->pp;
    int *pop_out = P.pop[lb][pp ^ 1];
    int *new_slots = P.pop[lb][pp];  // the iteration's input populations, no longer read after the sweep
    unsigned long long *det = P.det[lb];
    const unsigned long long imask = (unsigned long long)P.idx_cap - 1ull;
    unsigned long long dnw = 0, dnd = 0, aborted = 0, inserted = 0;

    for (unsigned long long i0 = (unsigned long long)blockIdx.x * blockDim.x; i0 < nm;
         i0 += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long i = i0 + threadIdx.x;
        bool want = false;
        unsigned long long key[W];
        long long amt = 0;
        unsigned long long h = 0;
        if (i < nm) {
            const unsigned pos = P.merged[i];
            unsigned long long *e = P.mt + (unsigned long long)pos * S;
#pragma unroll
            for (int w = 0; w < W; ++w) key[w] = e[w];
            const unsigned long long val = e[W];
#pragma unroll
            for (int w = 0; w < W; ++w) e[w] = EMPTY;
            e[W] = 0ull;
            // payload = (#initiator spawns << 40) + signed amount
            unsigned long long low = val & (kFlagUnit - 1ull);
            amt = (low & (1ull << 39)) ? (long long)low - (long long)kFlagUnit : (long long)low;
            const bool flag = ((val - (unsigned long long)amt) >> 40) != 0ull;
            if (amt != 0) {
                h = table_hash<W>(key, kSaltIndex) >> (64 - P.idx_bits);
                long long slot = -1;
                for (long long probe = 0; probe < P.idx_cap; ++probe) {
                    const unsigned long long *x = P.idx + h * S;
                    bool match = true, empty = true;
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        unsigned long long kw = __ldcg(x + w);
                        match = match && (kw == key[w]);
                        empty = empty && (kw == EMPTY);
                    }
                    if (match) { slot = (long long)__ldcg(x + W); break; }
                    if (empty) break;
                    h = (h + 1ull) & imask;
                }
                const bool allow = P.init_thr < 0 || flag;
                const unsigned long long aa = (unsigned long long)(amt < 0 ? -amt : amt);
                if (slot >= 0) {
                    const int old = pop_out[slot];
                    if (old != 0) {
                        long long nv = (long long)old + amt;
                        if (nv > 2147483647LL || nv < -2147483647LL) set_status(st, FCIQMC_ERR_NUMERIC);
                        pop_out[slot] = (int)nv;
                        dnw += (unsigned long long)((nv < 0 ? -nv : nv) - (long long)(old < 0 ? -old : old));
                        if (nv == 0) dnd += (unsigned long long)(-1LL);
                    } else if (allow) {
                        if (amt > 2147483647LL || amt < -2147483647LL) set_status(st, FCIQMC_ERR_NUMERIC);
                        pop_out[slot] = (int)amt;
                        dnw += aa;
                        dnd += 1;
                        inserted += 1;
                    } else {
                        aborted += aa;
                    }
                } else if (allow) {
                    want = true;
                } else {
                    aborted += aa;
                }
            }
        }
        const long long ns = warp_append(&st->claim, want);
        const long long nk = warp_append(&st->n_new, want);
        if (want) {
            if (amt > 2147483647LL || amt < -2147483647LL) set_status(st, FCIQMC_ERR_NUMERIC);
#pragma unroll
            for (int w = 0; w < W; ++w) det[ns * W + w] = key[w];
            pop_out[ns] = (int)amt;
            new_slots[nk] = (int)ns;
            // publish in the index (distinct keys only: no other thread inserts this determinant)
            for (long long probe = 0; probe < P.idx_cap; ++probe) {
                unsigned long long *x = P.idx + h * S;
                bool claimed;
                if (claim_key<W>(x, key, claimed)) {
                    x[W] = (unsigned long long)ns;
                    break;
                }
                h = (h + 1ull) & imask;
            }
            dnw += (unsigned long long)(amt < 0 ? -amt : amt);
            dnd += 1;
            inserted += 1;
        }
    }
    unsigned long long accv[4] = {dnw, dnd, aborted, inserted};
    unsigned long long *const dst[4] = {&st->d_nw, &st->d_nd, &st->cnt[C_ABORTED], &st->cnt[C_INSERTED]};
    flush_counters<256, 4>(accv, dst, s_red);
}

// H_ii - E0 (and its nearest float) of the slots placed by k_annihilate this iteration, one per thread in
// the FP64 order of hdiag / hphf_hdiag, with the pair terms in shared memory.
template <int W>
__global__ void __launch_bounds__(256) k_new_diag(Params P) {
    extern __shared__ double s_w[];  // [2][M][M] pair terms, then M diagonal h_pp
    DevState *st = P.st;
    if (st->status) return;
    const long long n = (long long)st->n_new;
    if ((long long)blockIdx.x * blockDim.x >= n) return;
    const int M = P.n_orb;
    __shared__ Tables T;
    load_tables(P, T);
    for (int k = threadIdx.x; k < 2 * M * M; k += blockDim.x) s_w[k] = P.wpair[k];
    for (int k = threadIdx.x; k < M; k += blockDim.x) s_w[2 * M * M + k] = P.h[k * M + k];
    __syncthreads();
    const int lb = st->lb, pp = st->pp;
    const int *new_slots = P.pop[lb][pp];
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const long long s = new_slots[k];
        unsigned long long key[W];
#pragma unroll
        for (int w = 0; w < W; ++w) key[w] = P.det[lb][s * W + w];
        const double v = P.hphf ? hphf_hdiag<W>(P, key, s_w, s_w + 2 * M * M) : hdiag<W>(P, key, s_w, s_w + 2 * M * M);
        const double hdv = __dsub_rn(v, P.E0);
        P.hd[lb][s] = hdv;
        P.hdf[lb][s] = __double2float_rn(hdv);
        store_derived<W>(P, T, lb, s, key);
    }
}

// Occupation threshold of hybrid walkers: after annihilation every amplitude below occ_units units is rounded
// stochastically to +-occ_units (probability |C| / occ_units, draw tag 5) or removed, which keeps the list's
// expectation (Eq. 1). Launched only for runs with a threshold above one unit.
template <int W>
__global__ void __launch_bounds__(256) k_round(Params P) {
    __shared__ unsigned long long s_red[(256 / 32) * 2];
    DevState *st = P.st;
    if (st->status) return;
    const int lb = st->lb, pp = st->pp;
    int *pop_out = P.pop[lb][pp ^ 1];
    const long long n = (long long)st->claim;
    const unsigned iter = (unsigned)st->iter;
    unsigned long long dnw = 0, dnd = 0;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int c = pop_out[s];
        const unsigned ac = (unsigned)(c < 0 ? -c : c);
        if (c == 0 || ac >= (unsigned)P.occ_units) continue;
        unsigned long long d[W];
#pragma unroll
        for (int w = 0; w < W; ++w) d[w] = P.det[lb][s * W + w];
        unsigned long long u, unused;
        draw2(0u, 5u, fingerprint<W>(d, P.map1), P.seed, iter, u, unused);
        const bool keep = unit53(u) < __ddiv_rn((double)ac, (double)P.occ_units);
        pop_out[s] = keep ? (c > 0 ? P.occ_units : -P.occ_units) : 0;
        dnw += (unsigned long long)((long long)(keep ? P.occ_units : 0) - (long long)ac);
        if (!keep) dnd += (unsigned long long)(-1LL);
    }
    unsigned long long accv[2] = {dnw, dnd};
    unsigned long long *const dst[2] = {&st->d_nw, &st->d_nd};
    flush_counters<256, 2>(accv, dst, s_red);
}

// Natural logarithm from the atanh series (shift update); same operation order as the oracle's.
__device__ double own_log(double x) {
    const double LN2_HI = 0x1.62e42fe800000p-1;
    const double LN2_LO = 0x1.e8e7bcd5e4f1ep-31;
    const double SQRT2 = 0x1.6a09e667f3bcdp+0;
    if (!(x > 0.0)) return x == 0.0 ? -CUDART_INF : CUDART_NAN;
    if (isinf(x)) return x;
    int e = 0;
    if (x < 0x1.0p-1022) { x = __dmul_rn(x, 0x1.0p54); e = -54; }
    unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    e += (int)((bits >> 52) & 0x7FFull) - 1023;
    bits = (bits & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;
    double m = __longlong_as_double((long long)bits);
    if (m > SQRT2) { m = __dmul_rn(m, 0.5); e += 1; }
    double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
    double z = __dmul_rn(s, s);
    double poly = __ddiv_rn(1.0, 23.0);
    for (int k = 10; k >= 0; --k) poly = __dadd_rn(__dmul_rn(poly, z), __ddiv_rn(1.0, (double)(2 * k + 1)));
    double t = __dmul_rn(s, poly);
    double lnm = __dadd_rn(t, t);
    double de = (double)e;
    double r = __dadd_rn(lnm, __dmul_rn(de, LN2_LO));
    return __dadd_rn(__dmul_rn(de, LN2_HI), r);
}

// The iteration's row for one list: its estimators (start of the iteration) and counters; num is the
// Eq. 2 numerator of the list.
__device__ __forceinline__ fciqmc_row list_row(const DevState *st, double num) {
    fciqmc_row row;
    const long long nw_in = (long long)st->nw_in, nd_in = (long long)st->nd_in;
    row.iteration = st->iter;
    row.shift = st->shift;
    row.nw_in = nw_in;
    row.nd_in = nd_in;
    row.c0_in = st->c0_in;
    row.num_in = num;
    row.nw_out = nw_in + (long long)st->d_nw;
    row.nd_out = nd_in + (long long)st->d_nd;
    row.attempts = (long long)st->cnt[C_ATTEMPTS];
    row.nulls = (long long)st->cnt[C_NULLS];
    row.spawn_events = (long long)st->cnt[C_EVENTS];
    row.spawned_walkers = (long long)st->cnt[C_SPAWNED];
    row.death_walkers = (long long)st->cnt[C_DEATH];
    row.clone_walkers = (long long)st->cnt[C_CLONE];
    row.merged_entries = (long long)st->n_merged;
    row.aborted_walkers = (long long)st->cnt[C_ABORTED];
    row.inserted_dets = (long long)st->cnt[C_INSERTED];
    row.heavy_attempts = (long long)st->cnt[C_HEAVY];
    return row;
}

// Shift update of the run: S <- S - zeta/(A tau) ln(N_w(n) / N_w(n-A)) every A iterations once N_w reached
// the target (nw_out: the whole run's walkers after the iteration).
__device__ __forceinline__ void shift_update(DevState *st, long long nw_out, long long target, int period, double c_shift) {
    if (!st->vary) {
        if (nw_out >= target) { st->vary = 1; st->nw_prev = nw_out; st->n_since = 0; }
    } else {
        st->n_since++;
        if (st->n_since == period) {
            double ratio = __ddiv_rn((double)nw_out, (double)st->nw_prev);
            st->shift = __dsub_rn(st->shift, __dmul_rn(c_shift, own_log(ratio)));
            st->nw_prev = nw_out;
            st->n_since = 0;
        }
    }
}

// Heavy chunk size for the next iteration from its expected attempts: kChunk doubled while every k_heavy warp
// still gets kChunksPerWarp chunks, up to kChunkGrowth kChunk (larger chunks: fewer table builds and batch
// claims; small ones when the walkers are few, so that every warp has work).
__device__ __forceinline__ unsigned next_chunk(long long attempts, long long warps) {
    unsigned c = kChunk;
    while (c < (unsigned)(kChunkGrowth * kChunk) && attempts >= 2ll * c * kChunksPerWarp * warps) c *= 2u;
    return c;
}

// Makes the iteration's list the current one (new slots included, populations' parity flipped), decides a
// compaction and the heavy chunk size for the next iteration (attempts: its expected spawning attempts) and
// clears the per-iteration counters.
__device__ __forceinline__ void commit_list(DevState *st, long long nd_out, long long cap, long long attempts,
                                            long long heavy_warps, long long sweep_blocks) {
    const long long new_len = (long long)st->claim;
    st->list_len = new_len;
    st->pp ^= 1;
    st->iter++;
    const long long vacated = new_len - nd_out;
    if ((vacated > 64 && vacated * 4 > new_len) || (vacated > 0 && new_len * 4 > cap * 3))
        st->compact_pending = 1;
    st->n_merged = 0;
    st->heavy_packed = 0;
    st->nw_in = st->nd_in = 0;
    st->c0_in = 0;
    st->d_nw = st->d_nd = 0;
    st->n_new = 0;
    st->sweep_next = 0;
    st->heavy_next = 0;
    st->heavy_chunk = next_chunk(attempts, heavy_warps);
    // a short list leaves most sweep blocks without a tile, and each tile's light attempts run in one block:
    // then the heavy path, whose chunks spread over every warp, takes determinants from 32 walkers on
    st->heavy_thr = (new_len + kTile - 1) / kTile * 4 < sweep_blocks ? (unsigned)kHeavyShort : (unsigned)kHeavy;
    for (int k = 0; k < NCNT; ++k) st->cnt[k] = 0;
    for (int k = 0; k < MAXPARTS; ++k) st->ob_n[k] = 0;
}

// Range sums of the sweep tiles' numerators (after k_sweep): block b adds the tiles of its fixed range
// [b n / kTileSums, (b + 1) n / kTileSums) in a fixed order (thread t takes tiles t, t + 256, ... of the range,
// then the block's fixed tree), so the run's numerator is the same in every run; the FP64 adds are spread
// over kTileSums SMs.
__global__ void __launch_bounds__(256) k_tile_sum(Params P) {
    __shared__ double s_red[256 / 32];
    DevState *st = P.st;
    if (st->status) return;
    const long long n = (st->list_len + kTile - 1) / kTile;
    const long long lo = n * blockIdx.x / kTileSums, hi = n * (blockIdx.x + 1) / kTileSums;
    double v = 0.0;
    for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) v = __dadd_rn(v, P.partial[t]);
    const double bs = block_sum_f64<256>(v, s_red);
    if (threadIdx.x == 0) P.partial[P.tiles_cap + blockIdx.x] = bs;
}

// Eq. 2 numerator of one list: the kTileSums range sums added by one warp in a fixed order (lane k takes sum
// k, then a fixed shuffle tree); lane 0 holds it.
__device__ __forceinline__ double list_numerator(const double *range_sums) {
    const int lane = threadIdx.x & 31;
    double part = 0.0;
    for (int b = lane; b < kTileSums; b += 32) part = __dadd_rn(part, range_sums[b]);
    return warp_sum_f64(part);
}

__global__ void k_finish(Params P) {
    DevState *st = P.st;
    if (st->status) return;
    const double num = list_numerator(P.partial + P.tiles_cap);
    if (threadIdx.x != 0) return;
    const fciqmc_row row = list_row(st, num);
    P.hist[st->hist_n % P.hist_cap] = row;
    st->hist_n++;
    shift_update(st, row.nw_out, P.target, P.period, P.c_shift);
    commit_list(st, row.nd_out, P.cap, row.nw_out >> P.frac_bits, P.heavy_warps, P.sweep_blocks);
}

// ---------------------------------------------------------------------------- hash-partitioned runs
// What a partition's kernels need of the other partitions of its run (device array, one entry per partition).
struct PartLink {
    DevState *st;
    unsigned long long *outbox;  // [n_parts][ob_cap] entries
    long long ob_cap;
    const double *partial;       // range sums of the sweep tiles' numerators (kTileSums)
    fciqmc_row *hist;            // the partition's own rows (its list's counters)
    long long hist_cap, cap;
    long long heavy_warps;       // warps of the partition's k_heavy launch
    long long sweep_blocks;      // blocks of the partition's k_sweep launch
    int frac_bits;               // hybrid walkers: populations in units of 2^-frac_bits
};
struct GroupDev {
    long long hist_n;            // rows written to hist
    int status;                  // first error of any partition (sticky)
};

// The exchange of Sec. V A, receiving side: the entries the other partitions routed to this one are merged
// into its spawn table (sum of signed amounts, initiator flags counted) as its own spawns were.
template <int W>
__global__ void __launch_bounds__(256) k_receive(Params P, const PartLink *links) {
    DevState *st = P.st;
    if (st->status) return;
    constexpr int S = Stride<W>::v;
    for (int r = 0; r < P.n_parts; ++r) {
        if (r == P.part) continue;
        const long long n = min((long long)links[r].st->ob_n[P.part], links[r].ob_cap);
        const unsigned long long *src = links[r].outbox + (unsigned long long)P.part * (unsigned long long)links[r].ob_cap * S;
        for (long long i0 = (long long)blockIdx.x * blockDim.x; i0 < n; i0 += (long long)gridDim.x * blockDim.x) {
            const long long i = i0 + threadIdx.x;
            bool claimed = false;
            unsigned pos = 0;
            if (i < n) {
                unsigned long long key[W];
#pragma unroll
                for (int w = 0; w < W; ++w) key[w] = src[i * S + w];
                claimed = merge_insert<W>(P, key, src[i * S + W], pos);
            }
            const long long slot = warp_append(&st->n_merged, claimed);
            if (claimed && slot < P.mt_cap) P.merged[slot] = pos;
        }
    }
}

// End of an iteration of a hash-partitioned run (one warp): the partitions' rows, the run's row (counters and
// estimators summed over partitions, numerators added in partition order), one shift update from the run's
// N_w applied to every partition, and each partition's list committed. An error in any partition stops the
// iteration in all of them before any list is committed.
__global__ void k_group_finish(const PartLink *links, int n_parts, GroupDev *g, fciqmc_row *ghist, long long ghist_cap,
                               long long target, int period, double c_shift) {
    int bad = g->status;
    for (int r = 0; r < n_parts && !bad; ++r) bad = links[r].st->status;
    if (bad) {
        if (threadIdx.x == 0) {
            g->status = bad;
            for (int r = 0; r < n_parts; ++r) atomicCAS(&links[r].st->status, 0, bad);
        }
        return;
    }
    double nums[MAXPARTS];
    for (int r = 0; r < n_parts; ++r) nums[r] = list_numerator(links[r].partial);
    if (threadIdx.x != 0) return;
    fciqmc_row tot = list_row(links[0].st, nums[0]);
    for (int r = 0; r < n_parts; ++r) {
        const fciqmc_row row = list_row(links[r].st, nums[r]);
        DevState *st = links[r].st;
        links[r].hist[st->hist_n % links[r].hist_cap] = row;
        st->hist_n++;
        if (r == 0) continue;
        tot.nw_in += row.nw_in;
        tot.nd_in += row.nd_in;
        tot.c0_in += row.c0_in;
        tot.num_in = __dadd_rn(tot.num_in, row.num_in);
        tot.nw_out += row.nw_out;
        tot.nd_out += row.nd_out;
        tot.attempts += row.attempts;
        tot.nulls += row.nulls;
        tot.spawn_events += row.spawn_events;
        tot.spawned_walkers += row.spawned_walkers;
        tot.death_walkers += row.death_walkers;
        tot.clone_walkers += row.clone_walkers;
        tot.merged_entries += row.merged_entries;
        tot.aborted_walkers += row.aborted_walkers;
        tot.inserted_dets += row.inserted_dets;
        tot.heavy_attempts += row.heavy_attempts;
    }
    ghist[g->hist_n % ghist_cap] = tot;
    g->hist_n++;
    for (int r = 0; r < n_parts; ++r) {
        DevState *st = links[r].st;
        shift_update(st, tot.nw_out, target, period, c_shift);  // the same state and input in every partition
        const long long nw_part = (long long)st->nw_in + (long long)st->d_nw;
        commit_list(st, (long long)st->nd_in + (long long)st->d_nd, links[r].cap, nw_part >> links[r].frac_bits,
                    links[r].heavy_warps, links[r].sweep_blocks);
    }
}

// ---------------------------------------------------------------------------- compaction and index
template <int W>
__global__ void k_compact_copy(Params P) {
    DevState *st = P.st;
    if (!st->compact_pending || st->status) return;
    const int lb = st->lb, pp = st->pp;
    const long long len = st->list_len;
    for (long long s0 = (long long)blockIdx.x * blockDim.x; s0 < len; s0 += (long long)gridDim.x * blockDim.x) {
        const long long s = s0 + threadIdx.x;
        int c = s < len ? P.pop[lb][pp][s] : 0;
        const long long ns = warp_append(&st->new_len, c != 0);
        if (c != 0) {
#pragma unroll
            for (int w = 0; w < W; ++w) P.det[lb ^ 1][ns * W + w] = P.det[lb][s * W + w];
            P.hd[lb ^ 1][ns] = P.hd[lb][s];
            P.hdf[lb ^ 1][ns] = P.hdf[lb][s];
            P.pop[lb ^ 1][pp][ns] = c;
            const ulonglong2 *ps = reinterpret_cast<const ulonglong2 *>(P.pre[lb] + s * PRE_WORDS);
            ulonglong2 *pd = reinterpret_cast<ulonglong2 *>(P.pre[lb ^ 1] + ns * PRE_WORDS);
            pd[0] = ps[0];
            pd[1] = ps[1];
            const unsigned *os = reinterpret_cast<const unsigned *>(P.occa[lb] + s * P.ostride);
            unsigned *od = reinterpret_cast<unsigned *>(P.occa[lb ^ 1] + ns * P.ostride);
            for (int k = 0; k < P.ostride / 4; ++k) od[k] = os[k];
        }
    }
}

// Whether a due compaction empties the old list's index entries one by one (a short list: len * 16 <=
// index capacity, positions held as int) rather than the whole index.
__device__ __forceinline__ bool sparse_index_clear(const Params &P, const DevState *st) {
    return st->list_len * 16 <= P.idx_cap && P.idx_cap <= (1LL << 31);
}

// Empties the whole index: forced (a rebuild, whatever the run's status), or for a due compaction whose
// list is too long for the sparse clear below.
__global__ void k_index_clear(Params P, int force) {
    DevState *st = P.st;
    if (!force && (st->status || !st->compact_pending || sparse_index_clear(P, st))) return;
    const long long nwords = P.idx_cap * (P.idx_stride);
    ulonglong2 *p = reinterpret_cast<ulonglong2 *>(P.idx);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nwords / 2; k += (long long)gridDim.x * blockDim.x)
        p[k] = make_ulonglong2(EMPTY, EMPTY);
}

// A due compaction with a short list (len * 16 <= index capacity): the old list's entries are emptied one
// by one instead of clearing the whole index. First every old slot's entry is located (into the old
// buffer's idle population array: no probe chain is cut before every key is found), then emptied.
template <int W>
__global__ void k_index_locate_old(Params P) {
    DevState *st = P.st;
    if (st->status || !st->compact_pending || !sparse_index_clear(P, st)) return;
    constexpr int S = Stride<W>::v;
    const int lb = st->lb;
    const long long n = st->list_len;
    int *pos = P.pop[lb][st->pp ^ 1];
    const unsigned long long imask = (unsigned long long)P.idx_cap - 1ull;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        unsigned long long key[W];
#pragma unroll
        for (int w = 0; w < W; ++w) key[w] = P.det[lb][s * W + w];
        unsigned long long h = table_hash<W>(key, kSaltIndex) >> (64 - P.idx_bits);
        int found = -1;
        for (long long probe = 0; probe < P.idx_cap; ++probe) {
            const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(P.idx + h * S);
            const bool match = x.x == key[0] && (W == 1 || x.y == key[W - 1]);
            const bool empty = x.x == EMPTY && (W == 1 || x.y == EMPTY);
            if (match) { found = (int)h; break; }
            if (empty) break;
            h = (h + 1ull) & imask;
        }
        pos[s] = found;
    }
}
template <int W>
__global__ void k_index_clear_old(Params P) {
    DevState *st = P.st;
    if (st->status || !st->compact_pending || !sparse_index_clear(P, st)) return;
    constexpr int S = Stride<W>::v;
    const long long n = st->list_len;
    const int *pos = P.pop[st->lb][st->pp ^ 1];
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int h = pos[s];
        if (h < 0) continue;
        ulonglong2 *e = reinterpret_cast<ulonglong2 *>(P.idx + (long long)h * S);
#pragma unroll
        for (int k = 0; k < S / 2; ++k) e[k] = make_ulonglong2(EMPTY, EMPTY);
    }
}

// Inserts slots [0, n) of a list buffer into the (cleared) index. force: rebuild the active list (at
// creation, or restoring it after a rejected set_walkers), whatever the run's status; otherwise the
// compacted list in the other buffer.
template <int W>
__global__ void k_index_fill(Params P, int force) {
    DevState *st = P.st;
    if (!force && (st->status || !st->compact_pending)) return;
    constexpr int S = Stride<W>::v;
    const int buf = force ? st->lb : (st->lb ^ 1);
    const long long n = force ? st->list_len : (long long)st->new_len;
    const unsigned long long imask = (unsigned long long)P.idx_cap - 1ull;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        unsigned long long key[W];
#pragma unroll
        for (int w = 0; w < W; ++w) key[w] = P.det[buf][s * W + w];
        unsigned long long h = table_hash<W>(key, kSaltIndex) >> (64 - P.idx_bits);
        bool done = false;
        for (long long probe = 0; probe < P.idx_cap; ++probe) {
            unsigned long long *x = P.idx + h * S;
            bool claimed;
            if (claim_key<W>(x, key, claimed)) {
                if (!claimed) set_status(st, FCIQMC_ERR_INVALID_ARG);  // duplicate determinant
                else x[W] = (unsigned long long)s;
                done = true;
                break;
            }
            h = (h + 1ull) & imask;
        }
        if (!done) set_status(st, FCIQMC_ERR_CAPACITY);
    }
}

// Inserts slots [lo, hi) of list buffer b (a list being loaded) into the index, the old list's entries
// already emptied: a key already present (a repeated determinant) sets check_bad to 2, a full table to 3.
template <int W>
__global__ void k_index_insert(Params P, int b, long long lo, long long hi) {
    constexpr int S = Stride<W>::v;
    const unsigned long long imask = (unsigned long long)P.idx_cap - 1ull;
    for (long long s = lo + (long long)blockIdx.x * blockDim.x + threadIdx.x; s < hi; s += (long long)gridDim.x * blockDim.x) {
        unsigned long long key[W];
#pragma unroll
        for (int w = 0; w < W; ++w) key[w] = P.det[b][s * W + w];
        unsigned long long h = table_hash<W>(key, kSaltIndex) >> (64 - P.idx_bits);
        bool done = false;
        for (long long probe = 0; probe < P.idx_cap; ++probe) {
            unsigned long long *x = P.idx + h * S;
            bool claimed;
            if (claim_key<W>(x, key, claimed)) {
                if (!claimed) atomicExch(&P.st->check_bad, 2);
                else x[W] = (unsigned long long)s;
                done = true;
                break;
            }
            h = (h + 1ull) & imask;
        }
        if (!done) atomicExch(&P.st->check_bad, 3);
    }
}

// Empties the spawn merge table (EMPTY keys, zero payloads).
__global__ void k_mt_clear(Params P, int W) {
    const int S = P.idx_stride;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < P.mt_cap; e += (long long)gridDim.x * blockDim.x) {
        for (int w = 0; w < W; ++w) P.mt[e * S + w] = EMPTY;
        P.mt[e * S + W] = 0ull;
    }
}

__global__ void k_compact_finish(Params P) {
    DevState *st = P.st;
    if (threadIdx.x != 0 || !st->compact_pending || st->status) return;
    st->lb ^= 1;
    st->list_len = (long long)st->new_len;
    st->claim = st->new_len;
    st->new_len = 0;
    st->compact_pending = 0;
    st->compactions++;
}

// ---------------------------------------------------------------------------- estimators, gather, setup
template <int W>
__global__ void __launch_bounds__(256) k_estimate(Params P) {
    __shared__ unsigned long long s_red[16];
    __shared__ double s_redf[8];
    DevState *st = P.st;
    const int lb = st->lb, pp = st->pp;
    const long long len = st->list_len;
    unsigned long long nw = 0, nd = 0;
    double num = 0.0;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < len; s += (long long)gridDim.x * blockDim.x) {
        const int c = P.pop[lb][pp][s];
        if (c == 0) continue;
        unsigned long long d[W];
#pragma unroll
        for (int w = 0; w < W; ++w) d[w] = P.det[lb][s * W + w];
        nw += (unsigned)(c < 0 ? -c : c);
        nd += 1;
        unsigned long long xd = 0;
        int diff = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) { xd |= d[w] ^ P.ref[w]; diff += __popcll(d[w] ^ P.ref[w]); }
        if (xd == 0) {
            st->est_c0 = c;
        } else if (diff == 2 || diff == 4) {
            double h0 = h0i<W>(P, d);
            if (P.hphf && n_open<W>(d) > 0) h0 = __dmul_rn(h0, kSqrt2);  // closed reference, open function
            num = __dadd_rn(num, __dmul_rn(h0, (double)c));
        }
    }
    unsigned long long accv[2] = {nw, nd};
    unsigned long long *const dst[2] = {&st->est_nw, &st->est_nd};
    flush_counters<256, 2>(accv, dst, s_red);
    double bs = block_sum_f64<256>(num, s_redf);
    if (threadIdx.x == 0) P.partial[blockIdx.x] = bs;
}

__global__ void k_estimate_finish(Params P, int nblocks) {
    if (threadIdx.x != 0) return;
    double num = 0.0;
    for (int b = 0; b < nblocks; ++b) num = __dadd_rn(num, P.partial[b]);
    P.st->est_num = num;
}

// Copies the occupied entries of the active list to od / op / oh (oh may be null; the idle list buffer for
// a read-back), count in new_len; entries past cap are counted but not written.
template <int W>
__global__ void k_gather(Params P, unsigned long long *od, int *op, double *oh, long long cap) {
    DevState *st = P.st;
    const int lb = st->lb, pp = st->pp;
    const long long len = st->list_len;
    for (long long s0 = (long long)blockIdx.x * blockDim.x; s0 < len; s0 += (long long)gridDim.x * blockDim.x) {
        const long long s = s0 + threadIdx.x;
        int c = s < len ? P.pop[lb][pp][s] : 0;
        const long long ns = warp_append(&st->new_len, c != 0);
        if (c != 0 && ns < cap) {
#pragma unroll
            for (int w = 0; w < W; ++w) od[ns * W + w] = P.det[lb][s * W + w];
            if (oh) oh[ns] = P.hd[lb][s];
            op[ns] = c;
        }
    }
}

// Checks slots [0, n) of list buffer b as loaded: n_elec occupied spin orbitals, none at or above n_so,
// inside the permitted space, owned by this partition, population neither 0 nor INT32_MIN. A failure sets
// st->check_bad. With convert, also the nearest float of each given diagonal element (the buffer is not
// the active one, so a failed check leaves nothing of the run changed).
template <int W>
__global__ void k_check_list(Params P, int b, long long n, int convert) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        int cnt = 0;
        bool ok = true;
        unsigned long long d[W];
#pragma unroll
        for (int w = 0; w < W; ++w) d[w] = P.det[b][s * W + w];
        if (P.space && !in_space<W>(P, d)) ok = false;
        if (P.hphf) {  // the stored (smaller) determinant of its spin-coupled pair, M_s = 0
            unsigned long long db[W];
            flip_spins<W>(d, db);
            int na = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) na += __popcll(d[w] & kEven);
            if (det_less<W>(db, d) || 2 * na != P.n_elec) ok = false;
        }
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const unsigned long long x = d[w];
            const int hi = P.n_so - 64 * w;
            if (hi < 64 && (hi <= 0 ? x != 0ull : (x >> hi) != 0ull)) ok = false;
            cnt += __popcll(x);
        }
        if (P.n_parts > 1 && fingerprint<W>(d, P.map1) % (unsigned long long)P.n_parts != (unsigned long long)P.part)
            ok = false;  // a determinant of another partition
        const int c = P.pop[b][0][s];
        if (!ok || cnt != P.n_elec || c == 0 || c == (-2147483647 - 1)) atomicExch(&P.st->check_bad, 1);
        if (convert) P.hdf[b][s] = __double2float_rn(P.hd[b][s]);
    }
}

// Index positions of the keys of slots [0, n) of list buffer b, into pos (-1 if absent). Lookups only:
// entries are emptied afterwards by k_index_clear_at, so no probe chain is cut before every key is found.
template <int W>
__global__ void k_index_locate(Params P, int b, long long n, int *pos) {
    constexpr int S = Stride<W>::v;
    const unsigned long long imask = (unsigned long long)P.idx_cap - 1ull;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        unsigned long long key[W];
#pragma unroll
        for (int w = 0; w < W; ++w) key[w] = P.det[b][s * W + w];
        unsigned long long h = table_hash<W>(key, kSaltIndex) >> (64 - P.idx_bits);
        int found = -1;
        for (long long probe = 0; probe < P.idx_cap; ++probe) {
            // the key words of an entry in one 16-byte load (entries are 16- or 32-byte aligned)
            const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(P.idx + h * S);
            const bool match = x.x == key[0] && (W == 1 || x.y == key[W - 1]);
            const bool empty = x.x == EMPTY && (W == 1 || x.y == EMPTY);
            if (match) { found = (int)h; break; }
            if (empty) break;
            h = (h + 1ull) & imask;
        }
        pos[s] = found;
    }
}

// Empties the index entries at pos[0, n) with 16-byte stores.
template <int W>
__global__ void k_index_clear_at(Params P, const int *pos, long long n) {
    constexpr int S = Stride<W>::v;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int h = pos[s];
        if (h < 0) continue;
        ulonglong2 *e = reinterpret_cast<ulonglong2 *>(P.idx + (long long)h * S);
#pragma unroll
        for (int k = 0; k < S / 2; ++k) e[k] = make_ulonglong2(EMPTY, EMPTY);
    }
}

// Slots [lo, n) of list buffer b as loaded: their derived words and occupied lists, and with compute their
// diagonal elements (H_ii - E0 and its nearest float; without, the float copies are made by the check).
template <int W>
__global__ void __launch_bounds__(256) k_prepare_list(Params P, int b, long long lo, long long n, int compute) {
    extern __shared__ double s_w[];
    __shared__ Tables T;
    load_tables(P, T);
    const int M = P.n_orb;
    if (compute) {
        for (int k = threadIdx.x; k < 2 * M * M; k += blockDim.x) s_w[k] = P.wpair[k];
        for (int k = threadIdx.x; k < M; k += blockDim.x) s_w[2 * M * M + k] = P.h[k * M + k];
    }
    __syncthreads();
    for (long long s = lo + (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        unsigned long long d[W];
#pragma unroll
        for (int w = 0; w < W; ++w) d[w] = P.det[b][s * W + w];
        store_derived<W>(P, T, b, s, d);
        if (compute) {
            const double v = __dsub_rn(P.hphf ? hphf_hdiag<W>(P, d, s_w, s_w + 2 * M * M) : hdiag<W>(P, d, s_w, s_w + 2 * M * M),
                                       P.E0);
            P.hd[b][s] = v;
            P.hdf[b][s] = __double2float_rn(v);
        }
    }
}

// Setup tables and reference facts: float integrals, pair terms, orbital map (Philox, key
// ("FCIQ", "MAP1"), counter (k, 0, 0, 0)), 1/L, E0 = H_00, and the reference's allowed single and
// double excitation counts (for P_double, Sec. VI). One block.
template <int W>
__global__ void __launch_bounds__(256) k_setup(Params P, long long n_eri, unsigned long long *map1_out, double *wpair_out,
                                               float *eri_f_out, double *recip_out, long long *facts, double *e0_out) {
    const int M = P.n_orb;
    for (long long k = threadIdx.x; k < n_eri; k += blockDim.x) eri_f_out[k] = __double2float_rn(P.eri[k]);
    for (int k = threadIdx.x; k < P.n_so; k += blockDim.x) {
        uint4 o = philox4x32_10(make_uint4((unsigned)k, 0u, 0u, 0u), make_uint2(0x46434951u, 0x4D415031u));
        map1_out[k] = (unsigned long long)o.x | ((unsigned long long)o.y << 32);
    }
    for (int k = threadIdx.x; k < M * M; k += blockDim.x) {
        int p = k / M, q = k % M;
        double jpq = eri_d(P, p, p, q, q);
        wpair_out[k] = jpq;
        wpair_out[M * M + k] = __dsub_rn(jpq, eri_d(P, p, q, q, p));
    }
    for (int k = threadIdx.x; k < 2 * MAXSO + 2; k += blockDim.x) recip_out[k] = k == 0 ? 0.0 : __ddiv_rn(1.0, (double)k);
    __syncthreads();
    // reference excitation counts by enumeration
    __shared__ unsigned long long s_ns, s_nd;
    if (threadIdx.x == 0) { s_ns = 0; s_nd = 0; }
    __syncthreads();
    unsigned long long ref[W];
#pragma unroll
    for (int w = 0; w < W; ++w) ref[w] = P.ref[w];
    const int N = P.n_elec, NS = P.n_so;
    unsigned long long ns = 0, nd = 0;
    for (int x = threadIdx.x; x < N; x += blockDim.x) {
        int i = P.ref_occ[x];
        for (int a = 0; a < NS; ++a)
            if (!bit_of<W>(ref, a) && (a & 1) == (i & 1) && P.irrep[a >> 1] == P.irrep[i >> 1]) ns++;
    }
    for (int pq = threadIdx.x; pq < N * N; pq += blockDim.x) {
        int x = pq / N, y = pq % N;
        if (y <= x) continue;
        int i = P.ref_occ[x], j = P.ref_occ[y];
        int gij = P.irrep[i >> 1] ^ P.irrep[j >> 1];
        for (int a = 0; a < NS; ++a) {
            if (bit_of<W>(ref, a)) continue;
            for (int b = a + 1; b < NS; ++b) {
                if (bit_of<W>(ref, b)) continue;
                if ((a & 1) + (b & 1) != (i & 1) + (j & 1)) continue;
                if ((P.irrep[a >> 1] ^ P.irrep[b >> 1]) != gij) continue;
                nd++;
            }
        }
    }
    atomicAdd(&s_ns, ns);
    atomicAdd(&s_nd, nd);
    __syncthreads();
    if (threadIdx.x == 0) {
        facts[0] = (long long)s_ns;
        facts[1] = (long long)s_nd;
    }
}

// The reference table: every double excitation the generator can select from the reference, in the
// order of attempt_begin (pair k1, the k2-th good a, the k3-th b of its class without a), with
// p = ((|H| (tau / P_double)) (npairs G M^(b|a) M^(a|b))) (1 / (M^(b|a) + M^(a|b))) as the exact path
// evaluates it, or for spin-coupled functions the target function and its p (hphf_exact's order); with a
// permitted space, excitations whose target lies outside it are marked as null excitations. One block.
// out = number of excitations, or -1 when they exceed cap or the packing.
template <int W>
__global__ void __launch_bounds__(256) k_ref_table(Params P, unsigned *pinfo, unsigned *off2, RefExc *ex,
                                                   long long cap, long long *out) {
    __shared__ Tables T;
    __shared__ DetView<W> v;
    __shared__ unsigned char occ[MAXN];
    __shared__ unsigned s_g[MAXPAIRS], s_go[MAXPAIRS], s_eo[MAXPAIRS];
    __shared__ int s_ok;
    load_tables(P, T);
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 0; w < W; ++w) v.d[w] = P.ref[w];
        prepare_det<W>(P, T, v, occ, 1);
    }
    __syncthreads();
    const int np = P.npairs;
    // G and the number of (a, b) choices of every pair
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        const unsigned short pr = T.pairs[k];
        const int i = occ[pr & 0xFF], j = occ[pr >> 8];
        const int si = i & 1, sj = j & 1, gij = T.irrep[i >> 1] ^ T.irrep[j >> 1];
        unsigned long long gm[W];
        const unsigned G = (unsigned)good_set<W>(P, v, si, sj, gij, gm);
        unsigned nx = 0;
        for (unsigned k2 = 0; k2 < G; ++k2) {
            const int ao = select_bit<W>(gm, (int)k2);
            const int ga = T.irrep[ao >> 1];
            const int ca = ga * 2 + (ao & 1), cb = (gij ^ ga) * 2 + (si + sj - (ao & 1));
            nx += (unsigned)v.cnt[cb] - (ca == cb ? 1u : 0u);
        }
        s_g[k] = G;
        s_eo[k] = nx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // exclusive prefix sums
        unsigned long long go = 0, eo = 0;
        for (int k = 0; k < np; ++k) {
            const unsigned g = s_g[k], e = s_eo[k];
            s_go[k] = (unsigned)go;
            s_eo[k] = (unsigned)eo;
            go += g;
            eo += e;
        }
        s_ok = (eo <= (unsigned long long)cap && eo < (1ull << 25) && go < (1ull << 24)) ? 1 : 0;
        *out = s_ok ? (long long)eo : -1;
    }
    __syncthreads();
    if (!s_ok) return;
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        const unsigned short pr = T.pairs[k];
        const int i = occ[pr & 0xFF], j = occ[pr >> 8];
        const int si = i & 1, sj = j & 1, gij = T.irrep[i >> 1] ^ T.irrep[j >> 1];
        unsigned long long gm[W];
        const unsigned G = (unsigned)good_set<W>(P, v, si, sj, gij, gm);
        pinfo[k] = (s_go[k] << 8) | G;
        unsigned e = s_eo[k];
        for (unsigned k2 = 0; k2 < G; ++k2) {
            const int ao = select_bit<W>(gm, (int)k2);
            const int ga = T.irrep[ao >> 1];
            const int ca = ga * 2 + (ao & 1), cb = (gij ^ ga) * 2 + (si + sj - (ao & 1));
            const unsigned same = ca == cb ? 1u : 0u;
            const unsigned m_ba = v.cnt[cb] - same, m_ab = v.cnt[ca] - same;
            off2[s_go[k] + k2] = (e << 7) | m_ba;
            unsigned long long bm[W];
#pragma unroll
            for (int w = 0; w < W; ++w) bm[w] = ~v.d[w] & T.mask[cb * MAXW + w];
            clear_bit<W>(bm, ao);
            for (unsigned k3 = 0; k3 < m_ba; ++k3, ++e) {
                const int bo = select_bit<W>(bm, (int)k3);
                const int A = min(ao, bo), B = max(ao, bo);
                double hd, p = 0.0;
                int fl = 0;  // 1: the target is stored on the flip of the generated determinant
                bool outside = false;  // a null excitation: the target lies outside the permitted space
                if (P.hphf) {
                    // spin-coupled functions (the reference is closed-shell): target stored on min(x, xbar),
                    // p = (tau |H_AB|) / (P(x) + P(xbar)) as the exact path evaluates it
                    unsigned long long x[W], xb[W], b[W];
#pragma unroll
                    for (int w = 0; w < W; ++w) x[w] = v.d[w];
                    flip<W>(x, i);
                    flip<W>(x, j);
                    flip<W>(x, ao);
                    flip<W>(x, bo);
                    flip_spins<W>(x, xb);
                    fl = det_less<W>(xb, x) ? 1 : 0;
#pragma unroll
                    for (int w = 0; w < W; ++w) b[w] = fl ? xb[w] : x[w];
                    outside = P.space && !in_space<W>(P, b);
                    hd = outside ? 0.0 : hphf_hij<W>(P, v, b);
                    if (hd != 0.0) {
                        double g = gen_prob<W>(P, v, x);
                        if (!det_same<W>(xb, x)) g = __dadd_rn(g, gen_prob<W>(P, v, xb));
                        p = __ddiv_rn(__dmul_rn(P.tau, fabs(hd)), g);
                    }
                } else {
                    if (P.space) {
                        unsigned long long x[W];
#pragma unroll
                        for (int w = 0; w < W; ++w) x[w] = v.d[w];
                        flip<W>(x, i);
                        flip<W>(x, j);
                        flip<W>(x, ao);
                        flip<W>(x, bo);
                        outside = !in_space<W>(P, x);
                    }
                    hd = outside ? 0.0 : hij_double<W>(P, v.d, i, j, A, B);
                    if (hd != 0.0) {
                        const long long K = (long long)P.npairs * (long long)G * (long long)m_ba * (long long)m_ab;
                        p = __dmul_rn(__dmul_rn(__dmul_rn(fabs(hd), P.cd), (double)K), P.recip[m_ba + m_ab]);
                    }
                }
                RefExc r;
                r.p_lo = outside ? -1.f : __double2float_rd(p);  // a negative bound marks a null excitation
                r.p_hi = outside ? -1.f : __double2float_ru(p);
                r.ps = hd > 0.0 ? p : -p;
                r.i = (unsigned char)(i ^ fl);  // the orbitals whose flips on the reference give the target
                r.j = (unsigned char)(j ^ fl);
                r.a = (unsigned char)(ao ^ fl);
                r.b = (unsigned char)(bo ^ fl);
                r.pad = 0;
                ex[e] = r;
            }
        }
    }
}

// E0 = H_00 of the reference (needs the pair table built by k_setup).
template <int W>
__global__ void k_reference_energy(Params P, double *e0_out) {
    extern __shared__ double s_w[];
    const int M = P.n_orb;
    for (int k = threadIdx.x; k < 2 * M * M; k += blockDim.x) s_w[k] = P.wpair[k];
    for (int k = threadIdx.x; k < M; k += blockDim.x) s_w[2 * M * M + k] = P.h[k * M + k];
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long ref[W];
#pragma unroll
        for (int w = 0; w < W; ++w) ref[w] = P.ref[w];
        *e0_out = hdiag<W>(P, ref, s_w, s_w + 2 * M * M);
    }
}

}  // namespace fq
