/*
 * Plain CPU oracle for the FCIQMC walker cycle (Booth, Smart, Alavi,
 * "Linear-scaling and parallelizable algorithms for stochastic quantum
 * chemistry").
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or
 * load this file; it exists so that tests, the smoke check and the CPU
 * baseline of the benchmark can compare the CUDA library against a slow,
 * obviously correct restatement of the method. It shares no code, header or
 * constant table with the CUDA side: every constant of the random-number
 * contract is written out again here.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no FMA contraction,
 * so every floating-point expression below is evaluated exactly as written).
 *
 * What is computed, per iteration (Sec. II, Eqs. 1, 3, 4; Sec. V; Sec. VI):
 *   1. for every walker on every occupied determinant D_i (populations taken
 *      at the start of the iteration, Sec. II "walkers spawned, cloned or
 *      killed within an iteration do not contribute"): draw an excitation
 *      D_j with normalised probability P_gen(j|i) (Sec. VI A/B), evaluate
 *      H_ij by the Slater-Condon rules, and spawn floor(p) + Bernoulli(frac p)
 *      walkers with p = tau |H_ij| / P_gen and sign -sign(C_i) sign(H_ij)
 *      (Eq. 3);
 *   2. death/cloning on every determinant with p_death = tau C_i (H_ii-E0-S)
 *      (Eq. 4);
 *   3. sort and compress the spawned list (Sec. V A), i.e. merge duplicate
 *      determinants, summing signed amounts and OR-ing initiator flags;
 *   4. annihilate the merged list against the post-death main list: add to
 *      occupied determinants, insert unoccupied ones only if the initiator
 *      flag is set (or the initiator approximation is off), computing the
 *      stored diagonal H_ii on insertion (Sec. V B);
 *   5. record the estimators (shift S, projected energy Eq. 2) and update S.
 *
 * Readings where the paper is silent (each one also fixed on the CUDA side):
 *   - random numbers: counter-based Philox4x32-10 (Salmon et al., SC'11) in
 *     place of the Mersenne twister, keyed by (seed, iteration) with counter
 *     (attempt, tag, fingerprint lo, fingerprint hi); fingerprint = Algorithm 1
 *     (p = 1099511628211, uint64 wraparound, no abs/mod) over the ascending
 *     occupied spin orbitals with a Philox-generated orbital map;
 *   - one Philox block (words r0, r1) per attempt: the top 53 bits of r0 make
 *     the type word, the other 75 bits R = r1 2^11 + (r0 mod 2^11) the choices;
 *   - random choices among n_1, n_2, ... options as the successive digits of R
 *     in mixed radix, k = floor(R n / 2^75) and then R <- R n mod 2^75,
 *     instead of redraw loops (the digits are uniform and independent within a
 *     relative bias of n_1 n_2 ... / 2^75, below 2^-51 for every supported size);
 *   - single/double choice: double iff (r0 >> 11) < floor(P_double 2^53), and
 *     P_double itself is the double/single ratio of the reference rounded to a
 *     multiple of 2^-53 so that the draw realises it exactly; the same word,
 *     uniform within the chosen type's sub-range, realises the Bernoulli part
 *     of the spawn;
 *   - initiator: |C_i| > threshold, or D_i is the reference;
 *   - shift: S <- S - zeta/(A tau) ln(N_w(n) / N_w(n-A)) every A iterations
 *     once N_w first reaches the target.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OQ_MAXW 2
#define OQ_MAXSO 128
#define OQ_CHUNK 4096   /* spawning attempts per parallel work unit */

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplications with the
 * published multipliers and Weyl key increments. */
void oq_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Two 64-bit words from one Philox block: (out0 | out1 << 32, out2 | out3 << 32). */
static void draw2(uint32_t a, uint32_t tag, uint64_t fp, uint32_t seed, uint32_t iter,
                  uint64_t *w0, uint64_t *w1)
{
    uint32_t ctr[4] = {a, tag, (uint32_t)fp, (uint32_t)(fp >> 32)};
    uint32_t key[2] = {seed, iter};
    uint32_t o[4];
    oq_philox(ctr, key, o);
    *w0 = (uint64_t)o[0] | ((uint64_t)o[1] << 32);
    *w1 = (uint64_t)o[2] | ((uint64_t)o[3] << 32);
}

/* Next digit of the 75-bit choice word R in mixed radix: k = floor(R n / 2^75), uniform in [0, n);
 * R keeps the remainder R n mod 2^75 for the next choice. */
static uint64_t next_digit(unsigned __int128 *R, uint64_t n)
{
    const unsigned __int128 x = *R * (unsigned __int128)n;
    *R = x & ((((unsigned __int128)1) << 75) - 1);
    return (uint64_t)(x >> 75);
}

/* The choice word of an attempt from its Philox words (r0, r1). */
static unsigned __int128 choice_word(uint64_t r0, uint64_t r1)
{
    return ((unsigned __int128)r1 << 11) | (unsigned __int128)(r0 & 0x7FFu);
}

/* Digits k[0..m) of the choice word of (r0, r1) for the radices n[0..m) (tests). */
void oq_digits(uint64_t r0, uint64_t r1, const uint64_t *n, int m, uint64_t *k)
{
    unsigned __int128 R = choice_word(r0, r1);
    for (int x = 0; x < m; ++x) k[x] = next_digit(&R, n[x]);
}

/* u = (r >> 11) * 2^-53, exactly representable, in [0, 1). */
static double unit53(uint64_t r)
{
    return (double)(r >> 11) * 0x1.0p-53;
}

/* ------------------------------------------------------------------------- */
/* Natural logarithm written from the mathematics (used by the shift update).
 * x = m 2^e with m in [sqrt(1/2), sqrt(2)); s = (m-1)/(m+1);
 * ln m = 2 atanh(s) = 2 s sum_{k>=0} s^{2k}/(2k+1), truncated after k = 11
 * (|s| <= 0.1716, so the first omitted term is below 1e-19 relative);
 * ln x = e*LN2_HI + (ln m + e*LN2_LO) with ln 2 split so that e*LN2_HI is exact. */
double oq_log(double x)
{
    const double LN2_HI = 0x1.62e42fe800000p-1;
    const double LN2_LO = 0x1.e8e7bcd5e4f1ep-31;
    const double SQRT2 = 0x1.6a09e667f3bcdp+0;
    if (!(x > 0.0)) return x == 0.0 ? -INFINITY : NAN;
    if (isinf(x)) return x;
    int e = 0;
    if (x < 0x1.0p-1022) { x = x * 0x1.0p54; e = -54; }
    uint64_t bits;
    memcpy(&bits, &x, 8);
    e += (int)((bits >> 52) & 0x7FF) - 1023;
    bits = (bits & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;
    double m;
    memcpy(&m, &bits, 8);
    if (m > SQRT2) { m = m * 0.5; e += 1; }
    double s = (m - 1.0) / (m + 1.0);
    double z = s * s;
    double poly = 1.0 / 23.0;
    for (int k = 10; k >= 0; --k) poly = poly * z + 1.0 / (double)(2 * k + 1);
    double t = s * poly;
    double lnm = t + t;
    double de = (double)e;
    double r = lnm + de * LN2_LO;
    return de * LN2_HI + r;
}

/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t iter;
    double shift;
    int64_t nw_in, nd_in, c0_in;
    double num_in;
    int64_t nw_out, nd_out;
    int64_t attempts, nulls, spawn_events, spawned_walkers;
    int64_t death_walkers, clone_walkers, merged_entries, aborted_walkers, inserted_dets;
} oq_row;

typedef struct {
    uint64_t d[OQ_MAXW];
    int64_t amt;
    int flag;
} spawn_t;

typedef struct {
    int n_orb, n_elec, n_so, W, n_alpha, n_beta;
    double *h, *eri, e_core;
    int64_t npair_sp;          /* spatial pairs M(M+1)/2 */
    int irrep[OQ_MAXSO / 2];
    int has_sym;
    uint64_t ref[OQ_MAXW];
    double E0;                 /* H_00 without e_core */
    double tau;
    int32_t init_thr;
    int64_t target;
    double zeta;
    int32_t period;
    double c_shift;            /* zeta / (A tau) */
    uint32_t seed;
    uint64_t map1[OQ_MAXSO];
    int64_t n_single_ref, n_double_ref;
    uint64_t d53;              /* double iff (r0 >> 11) < d53 */
    double p_double, p_single, cs, cd;
    /* state */
    int64_t n, cap;
    uint64_t *det;             /* n * W, sorted ascending (lexicographic on words) */
    int32_t *pop;
    double *hd;                /* H_ii - E0 */
    uint32_t iter;
    double shift;
    int vary;
    int64_t nw_prev;
    int n_since;
    int error;                 /* 0 ok, nonzero: numeric overflow */
    /* permitted space (Sec. VI: excitations outside it are returned as null excitations) */
    int space_flags;           /* bit 0: excitation level limit, bit 1: seniority limit */
    int max_exc, max_sen;
    uint64_t froz_occ[OQ_MAXW], froz_emp[OQ_MAXW];  /* spin orbitals that stay occupied / empty */
    int hphf;                  /* walkers live on spin-coupled functions (Sec. VI C) */
    /* real/integer hybrid walkers: populations are integers in units of 2^-frac_bits walkers */
    int frac_bits;
    int64_t occ_units;         /* occupation threshold in units (1: none) */
    double tau_s;              /* time step of the spawning probabilities, in units: tau 2^frac_bits */
} oq_t;

/* ---------------- bit-string helpers ---------------- */
static int det_bit(const oq_t *q, const uint64_t *d, int k) { (void)q; return (int)((d[k >> 6] >> (k & 63)) & 1u); }
static void det_flip(uint64_t *d, int k) { d[k >> 6] ^= (uint64_t)1 << (k & 63); }
static int det_eq(const oq_t *q, const uint64_t *a, const uint64_t *b)
{
    for (int w = 0; w < q->W; ++w) if (a[w] != b[w]) return 0;
    return 1;
}
static int det_cmp(int W, const uint64_t *a, const uint64_t *b)
{
    for (int w = W - 1; w >= 0; --w) {
        if (a[w] < b[w]) return -1;
        if (a[w] > b[w]) return 1;
    }
    return 0;
}
/* ascending occupied spin orbitals */
static int decode(const oq_t *q, const uint64_t *d, int *occ)
{
    int n = 0;
    for (int k = 0; k < q->n_so; ++k) if (det_bit(q, d, k)) occ[n++] = k;
    return n;
}
static int spin_of(int k) { return k & 1; }
static int spat_of(int k) { return k >> 1; }
static int class_of(const oq_t *q, int k) { return q->irrep[spat_of(k)] * 2 + spin_of(k); }
static int class_make(int irrep, int spin) { return irrep * 2 + spin; }

/* ---------------- integrals ---------------- */
static double h1(const oq_t *q, int p, int r) { return q->h[(int64_t)p * q->n_orb + r]; }
static int64_t pair_index(int64_t p, int64_t r) { return p >= r ? p * (p + 1) / 2 + r : r * (r + 1) / 2 + p; }
/* chemists' (pq|rs) over spatial orbitals, 8-fold packed */
static double eri4(const oq_t *q, int p, int r, int s, int t)
{
    int64_t a = pair_index(p, r), b = pair_index(s, t);
    return q->eri[pair_index(a, b)];
}

/* Algorithm 1 (Sec. V): hash = p*hash + map(det(i))*i over electrons i = 1..N. */
uint64_t oq_fingerprint(const oq_t *q, const uint64_t *d)
{
    int occ[OQ_MAXSO];
    int n = decode(q, d, occ);
    uint64_t hsh = 0;
    for (int i = 1; i <= n; ++i) hsh = 1099511628211ull * hsh + q->map1[occ[i - 1]] * (uint64_t)i;
    return hsh;
}

/* number of occupied spin orbitals strictly between k and l */
static int occ_between(const oq_t *q, const uint64_t *d, int k, int l)
{
    int lo = k < l ? k : l, hi = k < l ? l : k, c = 0;
    for (int m = lo + 1; m < hi; ++m) c += det_bit(q, d, m);
    return c;
}

/* ---------------- Slater-Condon rules (Sec. II) ---------------- */
/* Diagonal: sum_p h_pp + sum_{p<q} [(pp|qq) - delta_spin (pq|qp)], ascending order; each pair
 * term (Coulomb minus exchange) is formed first and then added to the running sum. */
double oq_hdiag(const oq_t *q, const uint64_t *d)
{
    int occ[OQ_MAXSO];
    int n = decode(q, d, occ);
    double v = 0.0;
    for (int x = 0; x < n; ++x) v = v + h1(q, spat_of(occ[x]), spat_of(occ[x]));
    for (int x = 0; x < n; ++x) {
        for (int y = x + 1; y < n; ++y) {
            int p = spat_of(occ[x]), r = spat_of(occ[y]);
            double t = eri4(q, p, p, r, r);
            if (spin_of(occ[x]) == spin_of(occ[y])) t = t - eri4(q, p, r, r, p);
            v = v + t;
        }
    }
    return v;
}

/* Single i -> a from source d: sign * [h_ia + sum_{j occ, j != i} ((ia|jj) - delta (ij|ja))]. */
static double hij_single(const oq_t *q, const uint64_t *d, int i, int a)
{
    int occ[OQ_MAXSO];
    int n = decode(q, d, occ);
    int I = spat_of(i), A = spat_of(a);
    double v = h1(q, I, A);
    for (int x = 0; x < n; ++x) {
        int j = occ[x];
        if (j == i) continue;
        int J = spat_of(j);
        v = v + eri4(q, I, A, J, J);
        if (spin_of(j) == spin_of(i)) v = v - eri4(q, I, J, J, A);
    }
    int par = occ_between(q, d, i, a) & 1;
    return par ? -v : v;
}

/* Double (i<j) -> (a<b) from source d. */
static double hij_double(const oq_t *q, const uint64_t *d, int i, int j, int a, int b)
{
    double v = 0.0;
    if (spin_of(i) == spin_of(a) && spin_of(j) == spin_of(b))
        v = v + eri4(q, spat_of(i), spat_of(a), spat_of(j), spat_of(b));
    if (spin_of(i) == spin_of(b) && spin_of(j) == spin_of(a))
        v = v - eri4(q, spat_of(i), spat_of(b), spat_of(j), spat_of(a));
    uint64_t t[OQ_MAXW];
    memcpy(t, d, sizeof(uint64_t) * q->W);
    int par = occ_between(q, t, i, a);
    det_flip(t, i);
    det_flip(t, a);
    par += occ_between(q, t, j, b);
    return (par & 1) ? -v : v;
}

/* Canonical matrix element <dst|H|src> evaluated from the source side (0 beyond doubles).
 * The diagonal case returns H_ii without e_core. */
double oq_hij(const oq_t *q, const uint64_t *src, const uint64_t *dst)
{
    int nd = 0;
    for (int w = 0; w < q->W; ++w) nd += __builtin_popcountll(src[w] ^ dst[w]);
    if (nd == 0) return oq_hdiag(q, src);
    if (nd != 2 && nd != 4) return 0.0;
    int holes[2], parts[2], nh = 0, np = 0;
    for (int k = 0; k < q->n_so; ++k) {
        int s = det_bit(q, src, k), t = det_bit(q, dst, k);
        if (s && !t) holes[nh++] = k;
        if (!s && t) parts[np++] = k;
    }
    if (nd == 2) return hij_single(q, src, holes[0], parts[0]);
    return hij_double(q, src, holes[0], holes[1], parts[0], parts[1]);
}

/* ---------------- excitation generator (Sec. VI) ---------------- */
static void unocc_counts(const oq_t *q, const uint64_t *d, int *cnt)
{
    for (int c = 0; c < 16; ++c) cnt[c] = 0;
    for (int k = 0; k < q->n_so; ++k) if (!det_bit(q, d, k)) cnt[class_of(q, k)]++;
}

/* Outcome of one excitation with explicit rank choices.
 * info[0] = kind (0 null, 1 single, 2 double)
 * info[1..3] = number of options at stage 1 (|E_ok| or N(N-1)/2), stage 2 (M_allow or
 *              M^a - delta_d, for the stage-1 choice) and stage 3 (M^(b|a), doubles)
 * info[4], info[5] = P_gen / P_type as the rational num/den
 * info[6..9] = orbitals i, j, a, b (j, b = -1 for singles; a < b for doubles). */
int oq_excite_ranks(const oq_t *q, const uint64_t *d, int type, uint64_t k1, uint64_t k2, uint64_t k3,
                    uint64_t *child, int64_t *info)
{
    int occ[OQ_MAXSO], cnt[16];
    int n = decode(q, d, occ);
    unocc_counts(q, d, cnt);
    for (int x = 0; x < 10; ++x) info[x] = 0;
    info[6] = info[7] = info[8] = info[9] = -1;
    memcpy(child, d, sizeof(uint64_t) * q->W);
    if (type == 1) {
        /* Sec. VI A: electrons with no symmetry-allowed a are removed from the choice
         * (delta_s renormalisation); i uniform over the rest, a uniform over M_allow. */
        int eok[OQ_MAXSO], nok = 0;
        for (int x = 0; x < n; ++x) if (cnt[class_of(q, occ[x])] > 0) eok[nok++] = occ[x];
        info[1] = nok;
        if (nok == 0 || k1 >= (uint64_t)nok) return 0;
        int i = eok[k1];
        int c = class_of(q, i);
        int mallow = cnt[c];
        info[2] = mallow;
        int seen = 0, a = -1;
        for (int k = 0; k < q->n_so; ++k) {
            if (!det_bit(q, d, k) && class_of(q, k) == c) {
                if ((uint64_t)seen == k2) { a = k; break; }
                seen++;
            }
        }
        if (a < 0) return 0;
        det_flip(child, i);
        det_flip(child, a);
        info[0] = 1;
        info[4] = 1;
        info[5] = (int64_t)mallow * (int64_t)nok;   /* M_allow (N - delta_s) */
        info[6] = i; info[8] = a;
        return 1;
    }
    /* Sec. VI B: unique pair {i,j} by inverse triangular index k = j(j-1)/2 + i. */
    int64_t npairs = (int64_t)n * (n - 1) / 2;
    info[1] = npairs;
    if (npairs == 0 || k1 >= (uint64_t)npairs) return 0;
    int ej = 1;
    while ((int64_t)ej * (ej + 1) / 2 <= (int64_t)k1) ej++;
    int ei = (int)((int64_t)k1 - (int64_t)ej * (ej - 1) / 2);
    int i = occ[ei], j = occ[ej];
    int si = spin_of(i), sj = spin_of(j);
    int gij = q->irrep[spat_of(i)] ^ q->irrep[spat_of(j)];
    /* a must carry an allowed spin and leave at least one symmetry/spin-allowed b */
    int good[OQ_MAXSO], ngood = 0;
    for (int k = 0; k < q->n_so; ++k) {
        if (det_bit(q, d, k)) continue;
        int sa = spin_of(k);
        if (si == sj && sa != si) continue;
        int ca = class_of(q, k);
        int cb = class_make(gij ^ q->irrep[spat_of(k)], si + sj - sa);
        int avail = cnt[cb] - (cb == ca ? 1 : 0);
        if (avail >= 1) good[ngood++] = k;
    }
    info[2] = ngood;
    if (ngood == 0 || k2 >= (uint64_t)ngood) return 0;
    int a = good[k2];
    int ca = class_of(q, a);
    int cb = class_make(gij ^ q->irrep[spat_of(a)], si + sj - spin_of(a));
    int cand[OQ_MAXSO], ncand = 0;
    for (int k = 0; k < q->n_so; ++k)
        if (!det_bit(q, d, k) && k != a && class_of(q, k) == cb) cand[ncand++] = k;
    info[3] = ncand;
    if (ncand == 0 || k3 >= (uint64_t)ncand) return 0;
    int b = cand[k3];
    int64_t m_ba = ncand;
    int64_t m_ab = cnt[ca] - (ca == cb ? 1 : 0);
    det_flip(child, i); det_flip(child, j); det_flip(child, a); det_flip(child, b);
    info[0] = 2;
    info[4] = m_ba + m_ab;
    info[5] = npairs * (int64_t)ngood * m_ba * m_ab;
    info[6] = i; info[7] = j;
    info[8] = a < b ? a : b;
    info[9] = a < b ? b : a;
    return 2;
}

/* ---------------- setup ---------------- */
static void count_ref_excitations(oq_t *q)
{
    int occ[OQ_MAXSO];
    int n = decode(q, q->ref, occ);
    int64_t ns = 0, ndb = 0;
    for (int x = 0; x < n; ++x)
        for (int a = 0; a < q->n_so; ++a)
            if (!det_bit(q, q->ref, a) && class_of(q, a) == class_of(q, occ[x])) ns++;
    for (int x = 0; x < n; ++x)
        for (int y = x + 1; y < n; ++y) {
            int i = occ[x], j = occ[y];
            int gij = q->irrep[spat_of(i)] ^ q->irrep[spat_of(j)];
            for (int a = 0; a < q->n_so; ++a) {
                if (det_bit(q, q->ref, a)) continue;
                for (int b = a + 1; b < q->n_so; ++b) {
                    if (det_bit(q, q->ref, b)) continue;
                    if (spin_of(a) + spin_of(b) != spin_of(i) + spin_of(j)) continue;
                    if ((q->irrep[spat_of(a)] ^ q->irrep[spat_of(b)]) != gij) continue;
                    ndb++;
                }
            }
        }
    q->n_single_ref = ns;
    q->n_double_ref = ndb;
}

void oq_destroy(oq_t *q)
{
    if (!q) return;
    free(q->h); free(q->eri); free(q->det); free(q->pop); free(q->hd);
    free(q);
}

static int ensure_cap(oq_t *q, int64_t need)
{
    if (need <= q->cap) return 0;
    int64_t nc = q->cap ? q->cap : 1024;
    while (nc < need) nc *= 2;
    uint64_t *d = realloc(q->det, sizeof(uint64_t) * q->W * nc);
    if (!d) return -1;
    q->det = d;
    int32_t *p = realloc(q->pop, sizeof(int32_t) * nc);
    if (!p) return -1;
    q->pop = p;
    double *hd = realloc(q->hd, sizeof(double) * nc);
    if (!hd) return -1;
    q->hd = hd;
    q->cap = nc;
    return 0;
}

oq_t *oq_create(const double *h, const double *eri_s8, double e_core, int n_elec, int n_orb, int ms2,
                const int32_t *orb_irrep, double tau, int32_t initiator_threshold, int64_t target_walkers,
                double shift_damping, int32_t shift_period, double initial_shift, int32_t initial_population,
                uint64_t seed, double p_double_override, const uint64_t *reference)
{
    if (n_orb < 1 || 2 * n_orb > OQ_MAXSO || n_elec < 1 || n_elec >= 2 * n_orb) return NULL;
    if ((n_elec + ms2) % 2 != 0 || ms2 < -n_elec || ms2 > n_elec) return NULL;
    oq_t *q = calloc(1, sizeof(oq_t));
    if (!q) return NULL;
    q->n_orb = n_orb; q->n_elec = n_elec; q->n_so = 2 * n_orb; q->W = (2 * n_orb + 63) / 64;
    q->n_alpha = (n_elec + ms2) / 2; q->n_beta = (n_elec - ms2) / 2;
    if (q->n_alpha > n_orb || q->n_beta > n_orb) { free(q); return NULL; }
    q->npair_sp = (int64_t)n_orb * (n_orb + 1) / 2;
    int64_t neri = q->npair_sp * (q->npair_sp + 1) / 2;
    q->h = malloc(sizeof(double) * n_orb * n_orb);
    q->eri = malloc(sizeof(double) * neri);
    memcpy(q->h, h, sizeof(double) * n_orb * n_orb);
    memcpy(q->eri, eri_s8, sizeof(double) * neri);
    q->e_core = e_core;
    q->has_sym = orb_irrep != NULL;
    for (int p = 0; p < n_orb; ++p) {
        q->irrep[p] = orb_irrep ? orb_irrep[p] : 0;
        if (q->irrep[p] < 0 || q->irrep[p] > 7) { oq_destroy(q); return NULL; }
    }
    if (reference) {
        memcpy(q->ref, reference, sizeof(uint64_t) * q->W);
    } else {
        memset(q->ref, 0, sizeof(q->ref));
        for (int p = 0; p < q->n_alpha; ++p) det_flip(q->ref, 2 * p);
        for (int p = 0; p < q->n_beta; ++p) det_flip(q->ref, 2 * p + 1);
    }
    q->tau = tau; q->init_thr = initiator_threshold; q->target = target_walkers;
    q->frac_bits = 0; q->occ_units = 1; q->tau_s = tau;
    q->zeta = shift_damping; q->period = shift_period;
    q->c_shift = shift_damping / ((double)shift_period * tau);
    q->seed = (uint32_t)seed;
    /* orbital map for Algorithm 1: Philox with key ("FCIQ", "MAP1"), counter (k, 0, 0, 0) */
    for (int k = 0; k < q->n_so; ++k) {
        uint32_t ctr[4] = {(uint32_t)k, 0u, 0u, 0u}, key[2] = {0x46434951u, 0x4D415031u}, o[4];
        oq_philox(ctr, key, o);
        q->map1[k] = (uint64_t)o[0] | ((uint64_t)o[1] << 32);
    }
    q->E0 = oq_hdiag(q, q->ref);
    count_ref_excitations(q);
    double pd = p_double_override > 0.0 ? p_double_override
              : (double)q->n_double_ref / (double)(q->n_single_ref + q->n_double_ref);
    if (pd > 1.0) pd = 1.0;
    q->d53 = (uint64_t)(pd * 0x1.0p53);
    q->p_double = (double)q->d53 * 0x1.0p-53;
    q->p_single = 1.0 - q->p_double;
    q->cs = tau / q->p_single;
    q->cd = tau / q->p_double;
    q->shift = initial_shift;
    if (ensure_cap(q, 1024)) { oq_destroy(q); return NULL; }
    q->n = 1;
    memcpy(q->det, q->ref, sizeof(uint64_t) * q->W);
    q->pop[0] = initial_population;
    q->hd[0] = 0.0;
    return q;
}

/* ---------------- generation probability of a given target (Sec. VI A, B) ---------------- */
/* Probability that one attempt from d generates the determinant x: the closed forms the generator
 * realises, 0 when x is not a single or double excitation it can produce.
 *   single i -> a (same class): P_single / (M_allow (N - delta_s))
 *   double {i,j} -> {a,b}: P_double (M^(b|a) + M^(a|b)) / (npairs G M^(b|a) M^(a|b)), the two orders
 *   of choosing a and b, G the number of good first virtuals of the pair. */
double oq_gen_prob(const oq_t *q, const uint64_t *d, const uint64_t *x)
{
    int holes[2], parts[2], nh = 0, np = 0;
    for (int k = 0; k < q->n_so; ++k) {
        int s = det_bit(q, d, k), t = det_bit(q, x, k);
        if (s && !t) { if (nh == 2) return 0.0; holes[nh++] = k; }
        if (!s && t) { if (np == 2) return 0.0; parts[np++] = k; }
    }
    if (nh != np || nh == 0) return 0.0;
    int occ[OQ_MAXSO], cnt[16];
    int n = decode(q, d, occ);
    unocc_counts(q, d, cnt);
    if (nh == 1) {
        if (class_of(q, holes[0]) != class_of(q, parts[0])) return 0.0;
        int nok = 0;
        for (int y = 0; y < n; ++y) if (cnt[class_of(q, occ[y])] > 0) nok++;
        int mallow = cnt[class_of(q, holes[0])];
        return q->p_single / (double)((int64_t)mallow * nok);
    }
    int i = holes[0], j = holes[1], a = parts[0], b = parts[1];
    int si = spin_of(i), sj = spin_of(j);
    if (spin_of(a) + spin_of(b) != si + sj) return 0.0;
    int gij = q->irrep[spat_of(i)] ^ q->irrep[spat_of(j)];
    if ((q->irrep[spat_of(a)] ^ q->irrep[spat_of(b)]) != gij) return 0.0;
    if (si == sj && (spin_of(a) != si || spin_of(b) != si)) return 0.0;
    int ngood = 0;   /* good first virtuals of the pair, as the generator counts them */
    for (int k = 0; k < q->n_so; ++k) {
        if (det_bit(q, d, k) || (si == sj && spin_of(k) != si)) continue;
        int cb = class_make(gij ^ q->irrep[spat_of(k)], si + sj - spin_of(k));
        if (cnt[cb] - (cb == class_of(q, k) ? 1 : 0) >= 1) ngood++;
    }
    int ca = class_of(q, a), cb = class_of(q, b);
    int64_t m_ba = cnt[cb] - (ca == cb ? 1 : 0);
    int64_t m_ab = cnt[ca] - (ca == cb ? 1 : 0);
    int64_t npairs = (int64_t)n * (n - 1) / 2;
    return (q->p_double * (double)(m_ba + m_ab)) / (double)(npairs * (int64_t)ngood * m_ba * m_ab);
}

/* ---------------- spin-coupled functions (Sec. VI C) ---------------- */
/* For M_s = 0 the spin flip F (alpha <-> beta for every electron) maps |D> to pi(D) |Dbar>: Dbar has
 * spin orbitals 2p and 2p + 1 exchanged, and pi(D) = (-1)^(doubly occupied spatial orbitals), since
 * the two creation operators of a doubly occupied orbital trade places while a lone electron keeps its
 * place among the others. F commutes with H. The functions are |D> for closed shells (Dbar = D) and
 * (|D> + sigma pi(D) |Dbar>) / sqrt(2) for open shells, sigma = pi(reference) = (-1)^(N/2) (the sector
 * of the closed-shell reference), stored on the smaller determinant of the pair. sigma pi(D) =
 * (-1)^(n_open / 2) with n_open singly occupied spatial orbitals. */
static const double SQRT2 = 0x1.6a09e667f3bcdp+0;   /* sqrt(2) rounded to nearest */

static void flip_spins(const oq_t *q, const uint64_t *d, uint64_t *out)
{
    memset(out, 0, sizeof(uint64_t) * OQ_MAXW);
    for (int k = 0; k < q->n_so; ++k) if (det_bit(q, d, k)) det_flip(out, k ^ 1);
}
static int n_open(const oq_t *q, const uint64_t *d)
{
    int c = 0;
    for (int p = 0; p < q->n_orb; ++p) c += det_bit(q, d, 2 * p) != det_bit(q, d, 2 * p + 1);
    return c;
}
static double pair_sign(const oq_t *q, const uint64_t *d) { return (n_open(q, d) / 2) % 2 ? -1.0 : 1.0; }

/* <Phi_a|H|Phi_b> for the functions stored on a != b. With <abar|H|bbar> = pi_a pi_b <a|H|b> and
 * <abar|H|b> = pi_a pi_b <a|H|bbar> the four determinant couplings fold into:
 *   both open: <a|H|b> + sigma pi_b <a|H|bbar>; one closed: sqrt(2) <a|H|b>; both closed: <a|H|b>. */
double oq_hphf_hij(const oq_t *q, const uint64_t *a, const uint64_t *b)
{
    uint64_t ab[OQ_MAXW], bb[OQ_MAXW];
    flip_spins(q, a, ab);
    flip_spins(q, b, bb);
    int a_open = !det_eq(q, a, ab), b_open = !det_eq(q, b, bb);
    double hab = oq_hij(q, a, b);
    if (a_open && b_open) return hab + pair_sign(q, b) * oq_hij(q, a, bb);
    if (a_open || b_open) return hab * SQRT2;
    return hab;
}

/* <Phi_a|H|Phi_a> = <a|H|a> + sigma pi_a <a|H|abar> (the second term only for two open shells). */
double oq_hphf_hdiag(const oq_t *q, const uint64_t *a)
{
    uint64_t ab[OQ_MAXW];
    flip_spins(q, a, ab);
    double v = oq_hdiag(q, a);
    if (!det_eq(q, a, ab)) v = v + pair_sign(q, a) * oq_hij(q, a, ab);
    return v;
}

/* H_ii (without e_core) of a stored walker: of the determinant, or of its spin-coupled function */
static double hdiag_of(const oq_t *q, const uint64_t *d) { return q->hphf ? oq_hphf_hdiag(q, d) : oq_hdiag(q, d); }

/* a determinant is stored as itself, or (spin-coupled functions) when it is the smaller of its pair */
static int stored_form(const oq_t *q, const uint64_t *d)
{
    if (!q->hphf) return 1;
    uint64_t db[OQ_MAXW];
    flip_spins(q, d, db);
    int na = 0;
    for (int p = 0; p < q->n_orb; ++p) na += det_bit(q, d, 2 * p);
    return na == q->n_alpha && det_cmp(q->W, d, db) <= 0;
}

/* Switches to spin-coupled functions; needs M_s = 0 and a closed-shell reference. */
/* Real/integer hybrid walkers (the multi-scale representation Sec. II mentions and defers): populations
 * become integers in units of 2^-bits walkers (the current list is rescaled); spawning probabilities are
 * formed with tau 2^bits, so the count drawn for a spawn is in units (Eq. 3 at resolution 2^-bits); death
 * (Eq. 4) is unchanged in units; a determinant's attempts are its walkers rounded stochastically; after
 * annihilation an amplitude below occ walkers is rounded stochastically to +-occ or removed. The initiator
 * threshold and the target stay in walkers (compared in units). Returns 0, or -1 for bits outside [0, 20], an
 * occupation threshold below one unit or above 2^31 units, a population or threshold that leaves int32, or
 * a second call. */
int oq_set_real(oq_t *q, int bits, double occ)
{
    if (bits < 0 || bits > 20 || q->frac_bits != 0) return -1;
    const double R = ldexp(1.0, bits);
    const double ou = nearbyint(occ * R);
    if (!(ou >= 1.0) || ou > 2147483647.0) return -1;
    for (int64_t x = 0; x < q->n; ++x)
        if (fabs((double)q->pop[x]) * R > 2147483647.0) return -1;
    if (q->init_thr >= 0 && (double)q->init_thr * R > 2147483647.0) return -1;
    for (int64_t x = 0; x < q->n; ++x) q->pop[x] = (int32_t)((int64_t)q->pop[x] << bits);
    if (q->init_thr >= 0) q->init_thr = (int32_t)((int64_t)q->init_thr << bits);
    q->target = q->target > (INT64_MAX >> bits) ? INT64_MAX : q->target << bits;
    q->frac_bits = bits;
    q->occ_units = (int64_t)ou;
    q->tau_s = q->tau * R;
    q->cs = q->tau_s / q->p_single;
    q->cd = q->tau_s / q->p_double;
    return 0;
}

int oq_set_hphf(oq_t *q, int on)
{
    if (on) {
        uint64_t rb[OQ_MAXW];
        flip_spins(q, q->ref, rb);
        if (q->n_alpha != q->n_beta || !det_eq(q, q->ref, rb)) return -1;
    }
    q->hphf = on ? 1 : 0;
    for (int64_t x = 0; x < q->n; ++x) q->hd[x] = hdiag_of(q, q->det + x * q->W) - q->E0;
    return 0;
}

/* ---------------- permitted space (Sec. VI) ---------------- */
/* A determinant lies in the permitted space when: at most max_exc of the reference's spin orbitals are
 * empty in it (excitation level, flag bit 0); at most max_sen spatial orbitals are singly occupied
 * (seniority, flag bit 1); every spin orbital of froz_occ is occupied and none of froz_emp is (an
 * active space: frozen core and deleted virtuals). */
static int in_space(const oq_t *q, const uint64_t *d)
{
    if (q->space_flags & 1) {
        int exc = 0;
        for (int k = 0; k < q->n_so; ++k)
            if (det_bit(q, q->ref, k) && !det_bit(q, d, k)) exc++;
        if (exc > q->max_exc) return 0;
    }
    if (q->space_flags & 2) {
        int sen = 0;
        for (int p = 0; p < q->n_orb; ++p)
            if (det_bit(q, d, 2 * p) != det_bit(q, d, 2 * p + 1)) sen++;
        if (sen > q->max_sen) return 0;
    }
    for (int k = 0; k < q->n_so; ++k) {
        if (det_bit(q, q->froz_occ, k) && !det_bit(q, d, k)) return 0;
        if (det_bit(q, q->froz_emp, k) && det_bit(q, d, k)) return 0;
    }
    return 1;
}

int oq_in_space(const oq_t *q, const uint64_t *d) { return in_space(q, d); }

/* Sets the permitted space (froz_occ / froz_emp: W words or NULL). Returns -1, leaving the space
 * unrestricted, when the reference lies outside it. */
int oq_set_space(oq_t *q, int flags, int max_exc, int max_sen, const uint64_t *froz_occ, const uint64_t *froz_emp)
{
    q->space_flags = flags & 3;
    q->max_exc = max_exc;
    q->max_sen = max_sen;
    memset(q->froz_occ, 0, sizeof(q->froz_occ));
    memset(q->froz_emp, 0, sizeof(q->froz_emp));
    if (froz_occ) memcpy(q->froz_occ, froz_occ, sizeof(uint64_t) * q->W);
    if (froz_emp) memcpy(q->froz_emp, froz_emp, sizeof(uint64_t) * q->W);
    if (!in_space(q, q->ref)) {
        q->space_flags = 0;
        memset(q->froz_occ, 0, sizeof(q->froz_occ));
        memset(q->froz_emp, 0, sizeof(q->froz_emp));
        return -1;
    }
    return 0;
}

/* ---------------- one spawning attempt and death (Eqs. 3, 4) ---------------- */
typedef struct {
    spawn_t *s;
    int64_t n, cap;
    int64_t nulls, events, walkers;
    int err;
    char pad[128];   /* keeps per-thread buffers on separate cache lines */
} sbuf_t;

static void sbuf_push(sbuf_t *b, int W, const uint64_t *d, int64_t amt, int flag)
{
    if (b->n == b->cap) {
        int64_t nc = b->cap ? 2 * b->cap : 1024;
        spawn_t *ns = realloc(b->s, sizeof(spawn_t) * nc);
        if (!ns) { b->err = 1; return; }
        b->s = ns; b->cap = nc;
    }
    memset(&b->s[b->n], 0, sizeof(spawn_t));
    memcpy(b->s[b->n].d, d, sizeof(uint64_t) * W);
    b->s[b->n].amt = amt;
    b->s[b->n].flag = flag;
    b->n++;
}

/* One spawning attempt a on determinant d (population c, fingerprint fp).
 * Returns the signed number of walkers spawned onto *child (0: none); *is_null = 1 when the
 * excitation generator returned a null excitation. Sets *err on a population overflow. */
static int64_t attempt_one(const oq_t *q, const uint64_t *d, int32_t c, uint64_t fp, uint32_t a,
                           uint64_t *child, int *is_null, int *err)
{
    uint64_t r0, r1;
    *is_null = 0;
    draw2(a, 0u, fp, q->seed, q->iter, &r0, &r1);
    unsigned __int128 R = choice_word(r0, r1);
    int type = (r0 >> 11) < q->d53 ? 2 : 1;
    int64_t info[10];
    /* stage option counts depend on the earlier choices, so the generator is queried stage by stage */
    oq_excite_ranks(q, d, type, 0, 0, 0, child, info);
    if (info[1] == 0) { *is_null = 1; return 0; }
    uint64_t k1 = next_digit(&R, (uint64_t)info[1]);
    oq_excite_ranks(q, d, type, k1, 0, 0, child, info);
    if (info[2] == 0) { *is_null = 1; return 0; }
    uint64_t k2 = next_digit(&R, (uint64_t)info[2]);
    uint64_t k3 = 0;
    if (type == 2) {
        oq_excite_ranks(q, d, type, k1, k2, 0, child, info);
        if (info[3] == 0) { *is_null = 1; return 0; }
        k3 = next_digit(&R, (uint64_t)info[3]);
    }
    int kind = oq_excite_ranks(q, d, type, k1, k2, k3, child, info);
    if (kind == 0) { *is_null = 1; return 0; }
    double hv, p;
    if (q->hphf) {
        /* Sec. VI C: from the stored determinant only; the target function holds child and its flip,
         * and its generation probability sums both: p = tau |H_AB| / (P(child) + P(flip)) */
        uint64_t xb[OQ_MAXW], b[OQ_MAXW];
        flip_spins(q, child, xb);
        memcpy(b, det_cmp(q->W, child, xb) <= 0 ? child : xb, sizeof(uint64_t) * OQ_MAXW);
        if (det_eq(q, b, d) || !in_space(q, b)) { *is_null = 1; return 0; }
        hv = oq_hphf_hij(q, d, b);
        if (hv == 0.0) return 0;
        double g = oq_gen_prob(q, d, child);
        if (!det_eq(q, xb, child)) g = g + oq_gen_prob(q, d, xb);
        p = (q->tau_s * fabs(hv)) / g;
        memcpy(child, b, sizeof(uint64_t) * q->W);
    } else {
        if (!in_space(q, child)) { *is_null = 1; return 0; }
        hv = kind == 1 ? hij_single(q, d, (int)info[6], (int)info[8])
                       : hij_double(q, d, (int)info[6], (int)info[7], (int)info[8], (int)info[9]);
        if (hv == 0.0) return 0;
        /* p = tau |H| / P_gen (Eq. 3), evaluated in the fixed order
         *   single: (|H| * (tau/P_single)) * (M_allow (N - delta_s))
         *   double: ((|H| * (tau/P_double)) * (npairs G M^(b|a) M^(a|b))) * (1 / (M^(b|a) + M^(a|b))) */
        if (kind == 1) p = (fabs(hv) * q->cs) * (double)info[5];
        else p = ((fabs(hv) * q->cd) * (double)info[5]) * (1.0 / (double)info[4]);
    }
    /* floor(p) walkers, plus one with probability p - floor(p). The Bernoulli draw reuses the type
     * word: given the type, t = r0 >> 11 is uniform on [0, d53) (double) or [d53, 2^53) (single), so
     * with the offset s and the range n of that interval, [t - s < (p - floor p) n] has probability
     * ceil((p - floor p) n) / n, within 1/n of p - floor p. */
    double fl = floor(p);
    if (fl >= 2147483647.0) { *err = 1; return 0; }
    uint64_t t = r0 >> 11;
    uint64_t off = kind == 2 ? 0 : q->d53;
    uint64_t range = kind == 2 ? q->d53 : ((uint64_t)1 << 53) - q->d53;
    int64_t nsp = (int64_t)fl + ((double)(t - off) < (p - fl) * (double)range ? 1 : 0);
    if (nsp == 0) return 0;
    int sgn_c = c > 0 ? 1 : -1, sgn_h = hv > 0.0 ? 1 : -1;
    return -(int64_t)sgn_c * sgn_h * nsp;
}

/* Spawning attempts of a determinant with population c: one per walker (Eq. 3). With populations in units
 * of 2^-b walkers the |c| 2^-b walkers are rounded stochastically, floor plus one with the probability of
 * the fraction, drawn with tag 4 (counter (0, 4, fingerprint), key (seed, iteration)). */
static int64_t attempts_of(const oq_t *q, const uint64_t *d, int32_t c)
{
    int64_t ac = c < 0 ? -(int64_t)c : c;
    if (q->frac_bits == 0) return ac;
    int64_t n = ac >> q->frac_bits, frac = ac & (((int64_t)1 << q->frac_bits) - 1);
    if (frac) {
        uint64_t u, unused;
        draw2(0u, 4u, oq_fingerprint(q, d), q->seed, q->iter, &u, &unused);
        if (unit53(u) < (double)frac * ldexp(1.0, -q->frac_bits)) n++;
    }
    return n;
}

/* Spawning attempts a0 <= a < a1 of determinant d (Eq. 3 once per walker). */
static void spawn_range(const oq_t *q, const uint64_t *d, int32_t c, uint64_t fp, int flag, uint32_t a0, uint32_t a1,
                        sbuf_t *b)
{
    for (uint32_t a = a0; a < a1; ++a) {
        uint64_t child[OQ_MAXW];
        int is_null = 0;
        int64_t amt = attempt_one(q, d, c, fp, a, child, &is_null, &b->err);
        if (is_null) b->nulls++;
        if (amt == 0) continue;
        sbuf_push(b, q->W, child, amt, flag);
        b->events++;
        b->walkers += amt < 0 ? -amt : amt;
    }
}

static int cmp_spawn_w1(const void *x, const void *y)
{
    const spawn_t *a = x, *b = y;
    return det_cmp(1, a->d, b->d);
}
static int cmp_spawn_w2(const void *x, const void *y)
{
    const spawn_t *a = x, *b = y;
    return det_cmp(2, a->d, b->d);
}

/* estimators of the current list: N_w, N_d, C_0 and sum_{i != 0} H_0i C_i (ascending det order) */
void oq_estimate(const oq_t *q, int64_t *nw, int64_t *nd, int64_t *c0, double *num)
{
    int64_t w = 0, dd = 0, cz = 0;
    double s = 0.0;
    for (int64_t x = 0; x < q->n; ++x) {
        const uint64_t *d = q->det + x * q->W;
        int32_t c = q->pop[x];
        if (c == 0) continue;
        w += c < 0 ? -(int64_t)c : c;
        dd++;
        if (det_eq(q, d, q->ref)) { cz = c; continue; }
        int nx = 0;
        for (int k = 0; k < q->W; ++k) nx += __builtin_popcountll(d[k] ^ q->ref[k]);
        if (nx == 2 || nx == 4) {
            double h0 = oq_hij(q, q->ref, d);
            if (q->hphf && n_open(q, d) > 0) h0 = h0 * SQRT2;  /* closed reference, open function */
            s = s + h0 * (double)c;
        }
    }
    *nw = w; *nd = dd; *c0 = cz; *num = s;
}

int oq_iterate(oq_t *q, int n_iter, oq_row *rows)
{
    const int W = q->W;
    for (int it = 0; it < n_iter; ++it) {
        oq_row *row = &rows[it];
        memset(row, 0, sizeof(*row));
        row->iter = q->iter;
        row->shift = q->shift;
        oq_estimate(q, &row->nw_in, &row->nd_in, &row->c0_in, &row->num_in);

        /* spawning from start-of-iteration populations (thread-local buffers, merged by sorting) */
        int nthreads = 1;
#ifdef _OPENMP
        nthreads = omp_get_max_threads();
#endif
        sbuf_t *bufs = calloc((size_t)nthreads, sizeof(sbuf_t));
        int32_t *newpop = malloc(sizeof(int32_t) * (q->n ? q->n : 1));
        int64_t death_w = 0, clone_w = 0;
        int numeric = 0;
        /* Work units: the attempts of each determinant in chunks of at most OQ_CHUNK (the attempt index is
         * a counter of the random numbers and the spawned list is sorted before it is merged, so how a
         * determinant's attempts are split across threads does not change the result); the first chunk of a
         * determinant also takes its death/cloning step. */
        int64_t *natt = malloc(sizeof(int64_t) * (q->n ? q->n : 1));
#pragma omp parallel for schedule(static)
        for (int64_t x = 0; x < q->n; ++x) natt[x] = attempts_of(q, q->det + x * W, q->pop[x]);
        int64_t n_units = 0;
        for (int64_t x = 0; x < q->n; ++x) {
            newpop[x] = q->pop[x];
            if (q->pop[x] == 0) continue;
            n_units += natt[x] > 0 ? (natt[x] + OQ_CHUNK - 1) / OQ_CHUNK : 1;  /* the first also takes the death step */
            row->attempts += natt[x];
        }
        int64_t *units = malloc(sizeof(int64_t) * 2 * (n_units ? n_units : 1));
        n_units = 0;
        for (int64_t x = 0; x < q->n; ++x) {
            if (q->pop[x] == 0) continue;
            int64_t a0 = 0;
            do {
                units[2 * n_units] = x;
                units[2 * n_units + 1] = a0;
                n_units++;
                a0 += OQ_CHUNK;
            } while (a0 < natt[x]);
        }
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : death_w, clone_w) reduction(| : numeric)
        for (int64_t u = 0; u < n_units; ++u) {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            const int64_t x = units[2 * u], a0 = units[2 * u + 1];
            const uint64_t *d = q->det + x * W;
            int32_t c = q->pop[x];
            uint64_t fp = oq_fingerprint(q, d);
            int64_t ac = c < 0 ? -(int64_t)c : c;
            int flag = q->init_thr < 0 || ac > q->init_thr || det_eq(q, d, q->ref);
            int64_t a1 = a0 + OQ_CHUNK < natt[x] ? a0 + OQ_CHUNK : natt[x];
            spawn_range(q, d, c, fp, flag, (uint32_t)a0, (uint32_t)a1, &bufs[tid]);
            if (a0 != 0) continue;
            /* death / cloning, Eq. 4: r = tau (H_ii - E0 - S) |C_i| */
            double r = (q->tau * (q->hd[x] - q->shift)) * (double)ac;
            double ar = fabs(r);
            double fl = floor(ar);
            if (fl >= 2147483647.0) { numeric = 1; continue; }
            uint64_t u, unused;
            draw2(0u, 3u, fp, q->seed, q->iter, &u, &unused);
            int64_t nd = (int64_t)fl + (unit53(u) < ar - fl ? 1 : 0);
            int64_t sc = c > 0 ? 1 : -1;
            int64_t nc;
            if (r >= 0.0) { nc = (int64_t)c - sc * nd; death_w += nd; }
            else { nc = (int64_t)c + sc * nd; clone_w += nd; }
            if (nc > 2147483647LL || nc < -2147483647LL) { numeric = 1; continue; }
            newpop[x] = (int32_t)nc;
        }
        free(units);
        free(natt);
        /* concatenate, sort and compress the spawned list (Sec. V A) */
        int64_t ns = 0;
        for (int t = 0; t < nthreads; ++t) {
            ns += bufs[t].n;
            row->nulls += bufs[t].nulls;
            row->spawn_events += bufs[t].events;
            row->spawned_walkers += bufs[t].walkers;
            if (bufs[t].err) numeric = 1;
        }
        spawn_t *sp = malloc(sizeof(spawn_t) * (ns ? ns : 1));
        int64_t off = 0;
        for (int t = 0; t < nthreads; ++t) {
            if (bufs[t].n) memcpy(sp + off, bufs[t].s, sizeof(spawn_t) * bufs[t].n);
            off += bufs[t].n;
            free(bufs[t].s);
        }
        free(bufs);
        qsort(sp, (size_t)ns, sizeof(spawn_t), W == 1 ? cmp_spawn_w1 : cmp_spawn_w2);
        int64_t nm = 0;
        for (int64_t x = 0; x < ns; ) {
            int64_t y = x;
            spawn_t m = sp[x];
            for (y = x + 1; y < ns && det_cmp(W, sp[y].d, m.d) == 0; ++y) {
                m.amt += sp[y].amt;
                m.flag |= sp[y].flag;
            }
            sp[nm++] = m;
            x = y;
        }
        row->death_walkers = death_w;
        row->clone_walkers = clone_w;
        row->merged_entries = nm;
        /* annihilation: merge the sorted merged list into the sorted post-death list */
        int64_t cap_new = q->n + nm;
        uint64_t *nd_det = malloc(sizeof(uint64_t) * W * (cap_new ? cap_new : 1));
        int32_t *nd_pop = malloc(sizeof(int32_t) * (cap_new ? cap_new : 1));
        double *nd_hd = malloc(sizeof(double) * (cap_new ? cap_new : 1));
        int64_t a = 0, bidx = 0, out = 0;
        while (a < q->n || bidx < nm) {
            int take;  /* 0: main only, 1: spawn only, 2: both */
            if (a >= q->n) take = 1;
            else if (bidx >= nm) take = 0;
            else {
                int cmp = det_cmp(W, q->det + a * W, sp[bidx].d);
                take = cmp < 0 ? 0 : (cmp > 0 ? 1 : 2);
            }
            if (take == 0) {
                if (newpop[a] != 0) {
                    memcpy(nd_det + out * W, q->det + a * W, sizeof(uint64_t) * W);
                    nd_pop[out] = newpop[a];
                    nd_hd[out] = q->hd[a];
                    out++;
                }
                a++;
            } else {
                const spawn_t *m = &sp[bidx];
                int occupied = take == 2 && newpop[a] != 0;
                if (occupied) {
                    int64_t v = (int64_t)newpop[a] + m->amt;
                    if (v > 2147483647LL || v < -2147483647LL) numeric = 1;
                    if (v != 0) {
                        memcpy(nd_det + out * W, q->det + a * W, sizeof(uint64_t) * W);
                        nd_pop[out] = (int32_t)v;
                        nd_hd[out] = q->hd[a];
                        out++;
                    }
                } else if (m->amt != 0) {
                    if (q->init_thr < 0 || m->flag) {
                        if (m->amt > 2147483647LL || m->amt < -2147483647LL) numeric = 1;
                        memcpy(nd_det + out * W, m->d, sizeof(uint64_t) * W);
                        nd_pop[out] = (int32_t)m->amt;
                        nd_hd[out] = hdiag_of(q, m->d) - q->E0;
                        out++;
                        row->inserted_dets++;
                    } else {
                        row->aborted_walkers += m->amt < 0 ? -m->amt : m->amt;
                    }
                }
                if (take == 2) a++;
                bidx++;
            }
        }
        free(sp);
        free(newpop);
        free(q->det); free(q->pop); free(q->hd);
        q->det = nd_det; q->pop = nd_pop; q->hd = nd_hd;
        q->n = out; q->cap = cap_new ? cap_new : 1;
        if (numeric) q->error = 1;
        /* occupation threshold of hybrid walkers: an amplitude below occ_units units is rounded stochastically
         * to +-occ_units (probability |C| / occ_units, draw tag 4 + 1) or removed; unbiased */
        if (q->occ_units > 1) {
            int64_t m = 0;
            for (int64_t x = 0; x < q->n; ++x) {
                int32_t c = q->pop[x];
                int64_t ac = c < 0 ? -(int64_t)c : c;
                if (ac < q->occ_units) {
                    uint64_t u, unused;
                    draw2(0u, 5u, oq_fingerprint(q, q->det + x * W), q->seed, q->iter, &u, &unused);
                    int keep = unit53(u) < (double)ac / (double)q->occ_units;
                    c = keep ? (int32_t)(c > 0 ? q->occ_units : -q->occ_units) : 0;
                }
                if (c == 0) continue;
                memmove(q->det + m * W, q->det + x * W, sizeof(uint64_t) * W);
                q->pop[m] = c;
                q->hd[m] = q->hd[x];
                m++;
            }
            q->n = m;
        }

        int64_t nw_out = 0;
        for (int64_t x = 0; x < q->n; ++x) nw_out += q->pop[x] < 0 ? -(int64_t)q->pop[x] : q->pop[x];
        row->nw_out = nw_out;
        row->nd_out = q->n;
        /* shift update (reading stated in the header) */
        if (!q->vary) {
            if (nw_out >= q->target) { q->vary = 1; q->nw_prev = nw_out; q->n_since = 0; }
        } else {
            q->n_since++;
            if (q->n_since == q->period) {
                double ratio = (double)nw_out / (double)q->nw_prev;
                q->shift = q->shift - q->c_shift * oq_log(ratio);
                q->nw_prev = nw_out;
                q->n_since = 0;
            }
        }
        q->iter++;
        if (q->error) return -1;
    }
    return 0;
}

/* ---------------- accessors ---------------- */
int64_t oq_n_dets(const oq_t *q) { return q->n; }
int oq_words(const oq_t *q) { return q->W; }

/* Threads of the parallel loops (the timing harness compares one thread with all cores); the results do
 * not depend on the count. */
void oq_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
int oq_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
void oq_get_walkers(const oq_t *q, uint64_t *dets, int32_t *pops, double *hd)
{
    memcpy(dets, q->det, sizeof(uint64_t) * q->W * q->n);
    memcpy(pops, q->pop, sizeof(int32_t) * q->n);
    if (hd) memcpy(hd, q->hd, sizeof(double) * q->n);
}
static const uint64_t *g_sort_base;
static int g_sort_w;
static int cmp_index(const void *x, const void *y)
{
    int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
    return det_cmp(g_sort_w, g_sort_base + a * g_sort_w, g_sort_base + b * g_sort_w);
}
/* Replace the walker list (any order, nonzero populations, distinct determinants) and the
 * dynamic state. H_ii is recomputed. Returns -1 on duplicates. */
int oq_set_walkers(oq_t *q, const uint64_t *dets, const int32_t *pops, int64_t n, uint32_t iter,
                   double shift, int vary, int64_t nw_prev, int n_since)
{
    for (int64_t x = 0; x < n; ++x) {
        if (pops[x] != 0 && !in_space(q, dets + x * q->W)) return -3;
        if (pops[x] != 0 && !stored_form(q, dets + x * q->W)) return -4;
    }
    int64_t *idx = malloc(sizeof(int64_t) * (n ? n : 1));
    for (int64_t x = 0; x < n; ++x) idx[x] = x;
    g_sort_base = dets; g_sort_w = q->W;
    qsort(idx, (size_t)n, sizeof(int64_t), cmp_index);
    free(q->det); free(q->pop); free(q->hd);
    q->det = NULL; q->pop = NULL; q->hd = NULL; q->cap = 0;
    if (ensure_cap(q, n ? n : 1)) { free(idx); return -2; }
    int64_t m = 0;
    for (int64_t x = 0; x < n; ++x) {
        const uint64_t *d = dets + idx[x] * q->W;
        if (pops[idx[x]] == 0) continue;
        if (m > 0 && det_cmp(q->W, q->det + (m - 1) * q->W, d) == 0) { free(idx); return -1; }
        memcpy(q->det + m * q->W, d, sizeof(uint64_t) * q->W);
        q->pop[m] = pops[idx[x]];
        q->hd[m] = hdiag_of(q, d) - q->E0;
        m++;
    }
    free(idx);
    q->n = m;
    q->iter = iter; q->shift = shift; q->vary = vary; q->nw_prev = nw_prev; q->n_since = n_since;
    return 0;
}
void oq_get_state(const oq_t *q, int64_t *iter, double *shift, int64_t *vary, int64_t *nw_prev, int64_t *n_since)
{
    *iter = q->iter; *shift = q->shift; *vary = q->vary; *nw_prev = q->nw_prev; *n_since = q->n_since;
}
/* scalar facts of the system: E0, P_double, n_single_ref, n_double_ref, d53 */
void oq_info(const oq_t *q, double *e0, double *pdouble, int64_t *ns, int64_t *nd, uint64_t *d53, uint64_t *ref)
{
    *e0 = q->E0; *pdouble = q->p_double; *ns = q->n_single_ref; *nd = q->n_double_ref; *d53 = q->d53;
    memcpy(ref, q->ref, sizeof(uint64_t) * q->W);
}
/* map1 table of the fingerprint */
void oq_map1(const oq_t *q, uint64_t *out) { memcpy(out, q->map1, sizeof(uint64_t) * q->n_so); }

/* H over an explicit determinant list: out[x*n+y] = <dets[y]|H|dets[x]> from source x (no e_core). */
void oq_hmatrix(const oq_t *q, const uint64_t *dets, int64_t n, double *out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t x = 0; x < n; ++x)
        for (int64_t y = 0; y < n; ++y)
            out[x * n + y] = oq_hij(q, dets + x * q->W, dets + y * q->W);
}

/* One full spawn attempt with the random-number contract, for tests: returns the signed
 * number of walkers spawned onto *child by attempt a of determinant d with population c
 * at the current iteration (0 when none; *is_null = 1 for a null excitation). */
int64_t oq_attempt(const oq_t *q, const uint64_t *d, int32_t c, uint32_t a, uint64_t *child, int *is_null)
{
    int err = 0;
    uint64_t fp = oq_fingerprint(q, d);
    memcpy(child, d, sizeof(uint64_t) * q->W);
    return attempt_one(q, d, c, fp, a, child, is_null, &err);
}

/* ------------------------------------------------------------------------- */
/* Energy functional E(h, V; c) = c^T H c / c^T c over an explicit determinant list and its gradient
 * with respect to h (full matrix, symmetric convention: dE = sum_pq grad_h[p][q] dh[p][q] for
 * symmetric dh) and to the packed ERIs (total derivative with respect to each stored element).
 * E uses the Slater-Condon elements above (over all ordered pairs, I and J ascending); the gradient
 * uses the density matrices obtained by applying the operators themselves:
 *   gamma_PQ   = sum_{I,J} c_J c_I <J| a+_{P s} a_{Q s} |I>                         (spin summed)
 *   Gamma_PQRS = sum_{I,J} c_J c_I <J| a+_{P s} a+_{R t} a_{S t} a_{Q s} |I>         (spin summed)
 * so that E = (sum h_PQ gamma_PQ + 1/2 sum (PQ|RS) Gamma_PQRS) / c^T c, grad_h = gamma / c^T c and
 * grad_eri[k] = 1/2 sum_{PQRS stored at k} Gamma_PQRS / c^T c. O(n^2) pairs: small lists only. */
static int occ_below(const uint64_t *d, int W, int k)
{
    int c = 0;
    for (int w = 0; w < W; ++w) {
        int lo = 64 * w;
        if (k <= lo) break;
        int nb = k - lo >= 64 ? 64 : k - lo;
        uint64_t m = nb >= 64 ? ~0ull : ((1ull << nb) - 1ull);
        c += __builtin_popcountll(d[w] & m);
    }
    return c;
}
/* apply a_k (annihilate) or a+_k (create) in place; returns the sign, 0 if the result vanishes */
static int apply_op(uint64_t *d, int W, int k, int create)
{
    int occ = (int)((d[k >> 6] >> (k & 63)) & 1u);
    if (create == occ) return 0;
    int s = (occ_below(d, W, k) & 1) ? -1 : 1;
    d[k >> 6] ^= (uint64_t)1 << (k & 63);
    return s;
}

int oq_rdm(const oq_t *q, const uint64_t *dets, const double *c, int64_t n, double *E_out, double *grad_h,
           double *grad_eri)
{
    const int W = q->W, M = q->n_orb, NS = q->n_so;
    double norm = 0.0;
    for (int64_t x = 0; x < n; ++x) norm = norm + c[x] * c[x];
    int64_t neri = q->npair_sp * (q->npair_sp + 1) / 2;
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    /* per-thread accumulators (rows I split statically), combined in thread order */
    double *t_num = calloc((size_t)nthreads, sizeof(double));
    double *t_h = calloc((size_t)nthreads * M * M, sizeof(double));
    double *t_e = calloc((size_t)nthreads * neri, sizeof(double));
    if (!t_num || !t_h || !t_e) { free(t_num); free(t_h); free(t_e); return -1; }
#pragma omp parallel for schedule(static)
    for (int64_t I = 0; I < n; ++I) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *gh = t_h + (size_t)tid * M * M, *ge = t_e + (size_t)tid * neri;
        const uint64_t *dI = dets + I * W;
        for (int64_t J = 0; J < n; ++J) {
            const uint64_t *dJ = dets + J * W;
            int nd = 0;
            for (int w = 0; w < W; ++w) nd += __builtin_popcountll(dI[w] ^ dJ[w]);
            if (nd > 4) continue;
            const double cc = c[J] * c[I];
            t_num[tid] = t_num[tid] + oq_hij(q, dI, dJ) * cc;
            /* one-body: a+_p a_qq |I> = |J> */
            for (int qq = 0; qq < NS; ++qq) {
                uint64_t K[OQ_MAXW];
                memcpy(K, dI, sizeof(uint64_t) * W);
                int s1 = apply_op(K, W, qq, 0);
                if (!s1) continue;
                for (int p = 0; p < NS; ++p) {
                    if ((p & 1) != (qq & 1)) continue;
                    uint64_t K2[OQ_MAXW];
                    memcpy(K2, K, sizeof(uint64_t) * W);
                    int s2 = apply_op(K2, W, p, 1);
                    if (!s2 || !det_eq(q, K2, dJ)) continue;
                    gh[(p >> 1) * M + (qq >> 1)] += cc * (double)(s1 * s2);
                }
            }
            /* two-body: a+_p a+_r a_s a_qq |I> = |J> */
            for (int qq = 0; qq < NS; ++qq) {
                uint64_t K1[OQ_MAXW];
                memcpy(K1, dI, sizeof(uint64_t) * W);
                int s1 = apply_op(K1, W, qq, 0);
                if (!s1) continue;
                for (int s = 0; s < NS; ++s) {
                    uint64_t K2[OQ_MAXW];
                    memcpy(K2, K1, sizeof(uint64_t) * W);
                    int s2 = apply_op(K2, W, s, 0);
                    if (!s2) continue;
                    /* the two created orbitals are J minus K2 */
                    int cre[2], nc = 0, bad = 0;
                    for (int k = 0; k < NS; ++k) {
                        int inJ = det_bit(q, dJ, k), inK = det_bit(q, K2, k);
                        if (inK && !inJ) bad = 1;
                        if (inJ && !inK) { if (nc < 2) cre[nc] = k; nc++; }
                    }
                    if (bad || nc != 2) continue;
                    for (int o = 0; o < 2; ++o) {
                        int r = cre[o], p = cre[1 - o];
                        if ((p & 1) != (qq & 1) || (r & 1) != (s & 1)) continue;
                        uint64_t K3[OQ_MAXW];
                        memcpy(K3, K2, sizeof(uint64_t) * W);
                        int s3 = apply_op(K3, W, r, 1);
                        int s4 = apply_op(K3, W, p, 1);
                        if (!s3 || !s4) continue;
                        ge[pair_index(pair_index(p >> 1, qq >> 1), pair_index(r >> 1, s >> 1))] +=
                            0.5 * cc * (double)(s1 * s2 * s3 * s4);
                    }
                }
            }
        }
    }
    double num = 0.0;
    memset(grad_h, 0, sizeof(double) * M * M);
    memset(grad_eri, 0, sizeof(double) * neri);
    for (int t = 0; t < nthreads; ++t) {
        num = num + t_num[t];
        for (int k = 0; k < M * M; ++k) grad_h[k] += t_h[(size_t)t * M * M + k];
        for (int64_t k = 0; k < neri; ++k) grad_eri[k] += t_e[(size_t)t * neri + k];
    }
    free(t_num); free(t_h); free(t_e);
    for (int k = 0; k < M * M; ++k) grad_h[k] = grad_h[k] / norm;
    for (int64_t k = 0; k < neri; ++k) grad_eri[k] = grad_eri[k] / norm;
    *E_out = num / norm;
    return 0;
}
