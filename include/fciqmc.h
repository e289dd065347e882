/*
 * fciqmc.h - C ABI of the GB300 FCIQMC walker cycle.
 *
 * The library advances a population of signed integer walkers on Slater
 * determinants by the FCIQMC master equation (Booth, Smart, Alavi,
 * "Linear-scaling and parallelizable algorithms for stochastic quantum
 * chemistry", Sec. II, Eq. 1):
 *
 *   C_i(n+1) = [1 - tau (H_ii - E0 - S)] C_i(n) - tau sum_{j != i} H_ij C_j(n)
 *
 * realised each iteration by spawning (Eq. 3) with a normalised random
 * excitation generator (Sec. VI), diagonal death/cloning (Eq. 4), and
 * annihilation of the spawned list into the main list with the initiator
 * filter (Sec. V, Sec. V B), followed by the shift and projected-energy
 * (Eq. 2) estimators. Every step runs in CUDA kernels for sm_103a.
 *
 * Conventions shared by all calls
 *   - Spin orbital k holds spatial orbital k >> 1 with spin k & 1 (0 = alpha).
 *     A determinant is W = ceil(2 n_orb / 64) uint64 words; bit k of word
 *     k >> 6 set means spin orbital k is occupied (Sec. III bit strings).
 *   - Integrals are real: h is n_orb x n_orb row-major and symmetric; ERIs are
 *     chemists' (pq|rs) packed 8-fold (Sec. II footnote): pair index
 *     pq = p(p+1)/2 + q for p >= q, element index pq(pq+1)/2 + rs for pq >= rs.
 *   - Orbital symmetry labels are 0..7 with the XOR direct product (abelian
 *     D2h-like groups, Sec. II); NULL means no spatial symmetry.
 *   - Limits: n_orb <= 64 (W <= 2), 1 <= n_elec <= 64, n_elec < 2 n_orb.
 *   - Every call returns an int status (0 = FCIQMC_OK, < 0 = error); no
 *     exception or abort crosses the ABI. fciqmc_strerror names a status.
 *   - Device memory comes only from the caller: fciqmc_workspace_bytes() says
 *     how much, and fciqmc_create() carves all device state out of that one
 *     buffer. The handle never allocates device memory and frees nothing the
 *     caller owns. Inputs are copied at creation; the caller keeps ownership
 *     of every array it passes.
 *   - One handle is driven from one host thread and one CUDA stream; there is
 *     no internal locking. Kernels are enqueued asynchronously on that stream;
 *     calls documented as synchronising wait for it.
 *   - Errors detected on the device (capacity, numeric overflow) stop the
 *     iteration in which they occur before it changes the committed walker
 *     list; later iterations already enqueued do nothing. The error stays set
 *     (sticky) until fciqmc_set_walkers; fciqmc_sync and fciqmc_estimators
 *     return it. The read-back calls (history, walkers, state, n_dets) still
 *     succeed and return the state of the last completed iteration, so a run
 *     can be restarted with larger capacities without changing its trajectory
 *     (the random numbers are keyed by iteration, not by history).
 */
#ifndef FCIQMC_H
#define FCIQMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    FCIQMC_OK = 0,
    FCIQMC_ERR_INVALID_ARG = -1,   /* bad argument or inconsistent input */
    FCIQMC_ERR_CAPACITY = -2,      /* main list, hash index or spawn table full */
    FCIQMC_ERR_NUMERIC = -3,       /* a population or spawn count left int32 */
    FCIQMC_ERR_TIMEOUT = -4,       /* a bounded device wait gave up */
    FCIQMC_ERR_CUDA = -5,          /* a CUDA runtime call failed */
    FCIQMC_ERR_UNSUPPORTED = -6,   /* size beyond the limits above */
    FCIQMC_ERR_WORKSPACE = -7,     /* workspace too small or misaligned (256 B) */
    FCIQMC_ERR_BOUNDS = -8         /* a device table index out of range; reported only by the debug build
                                      (compiled with -DFCIQMC_DEBUG), which checks every index the
                                      algorithm keeps in range by construction and skips the access */
};

typedef struct fciqmc_handle fciqmc_handle;

/* Limits of the permitted space (fciqmc_options.space_flags). */
enum {
    FCIQMC_SPACE_EXCITATION = 1,   /* at most max_excitation reference spin orbitals empty */
    FCIQMC_SPACE_SENIORITY = 2     /* at most max_seniority singly occupied spatial orbitals */
};

/* Run options. Zero-initialise and set what you need; fciqmc_default_options
 * fills the documented defaults. */
typedef struct {
    double shift_damping;        /* zeta of the shift update, default 0.05 */
    int32_t shift_period;        /* A: iterations between shift updates, default 10 */
    int32_t initial_population;  /* walkers placed on the reference, default 10 */
    double initial_shift;        /* S (relative to E0) until N_w first reaches target, default 0 */
    int64_t target_walkers;      /* vary-shift starts once N_w >= target, default 2^62 (never) */
    uint64_t seed;               /* low 32 bits key the random numbers, default 1 */
    double p_double;             /* > 0: fixed P_double; <= 0: from the reference (Sec. VI), default 0 */
    int64_t main_capacity;       /* determinant slots of the main list, default 1 << 20 */
    int64_t spawn_capacity;      /* entries of the spawn merge table (rounded up to a power of two),
                                    default main_capacity / 2 */
    int64_t history_capacity;    /* per-iteration estimator rows kept (ring), default 1 << 16 */
    const uint64_t *reference;   /* W words, NULL: aufbau (lowest orbitals of each spin filled) */
    int32_t grid_blocks;         /* blocks of the spawning and annihilation kernels; 0: enough to fill
                                    every SM at the kernels' occupancy. Never changes results. */
    double index_load;           /* largest load factor of the determinant hash index (its capacity is
                                    the next power of two >= main_capacity / index_load); 0: 0.5.
                                    Never changes results. */
    /* Permitted space (Sec. VI): an excitation generated outside it is a null excitation (no spawn;
     * the generation probabilities of the others are unchanged), so truncated CI, seniority-limited
     * and active-space calculations run unchanged otherwise. The reference and every loaded
     * determinant must lie in the space (else FCIQMC_ERR_INVALID_ARG). Default: unrestricted. */
    uint32_t space_flags;        /* FCIQMC_SPACE_* bits */
    int32_t max_excitation;      /* with FCIQMC_SPACE_EXCITATION */
    int32_t max_seniority;       /* with FCIQMC_SPACE_SENIORITY */
    const uint64_t *frozen_occupied;  /* W words or NULL: spin orbitals every determinant keeps occupied */
    const uint64_t *frozen_empty;     /* W words or NULL: spin orbitals no determinant occupies */
    /* Nonzero: walkers live on spin-coupled functions (Sec. VI C): |D> for closed shells and
     * (|D> + sigma pi(D) |Dbar>) / sqrt(2) otherwise, Dbar the spin-flipped determinant, pi(D) =
     * (-1)^(doubly occupied orbitals), sigma = pi(reference); each is stored on the smaller (as an
     * unsigned number, last word most significant) of D and Dbar. Needs ms2 = 0 and a closed-shell
     * reference (else FCIQMC_ERR_INVALID_ARG); loaded lists must hold stored determinants. */
    int32_t hphf;
    /* Hash-partitioned runs (Sec. V A, Algorithm 1): with n_partitions = P > 1 the handle holds partition
     * partition_index (0 <= index < P <= 64) of a run: the determinants whose Algorithm 1 fingerprint (the
     * one that keys the random numbers, see fciqmc_owner) is congruent to the index mod P. Its spawns onto
     * determinants of other partitions go to one outbox per destination of outbox_capacity entries (0: a
     * quarter of the spawn table); an overflowing outbox stops the iteration with FCIQMC_ERR_CAPACITY. A
     * partition is advanced only through fciqmc_group_* with the run's other partitions (fciqmc_step,
     * fciqmc_profile and fciqmc_batch_create refuse it); the reference's initial walkers are placed by its
     * own partition; loaded lists may hold only the partition's determinants. The random numbers do not
     * depend on the partitioning, so a run gives the same walkers for every P. 0 or 1: not partitioned. */
    int32_t n_partitions;
    int32_t partition_index;
    int64_t outbox_capacity;
    /* Real/integer hybrid walkers (the multi-scale representation Sec. II mentions and defers): with
     * walker_fraction_bits = b in [1, 20] populations are integers in units of 2^-b walkers (the int32 values
     * of fciqmc_get_walkers / fciqmc_set_walkers, the static estimator and the N_w and C_0 of the rows are in
     * units). A determinant makes |C| 2^-b spawning attempts rounded stochastically; a spawn's count is drawn
     * in units (Eq. 3 with tau 2^b); death (Eq. 4) acts on units; after annihilation an amplitude below
     * occupation_threshold walkers (<= 0: 1) is rounded stochastically to +-threshold or removed. Every step
     * keeps the expectation of Eq. 1. initial_population, target_walkers and the initiator threshold stay in
     * walkers. 0: integer walkers. */
    int32_t walker_fraction_bits;
    double occupation_threshold;
} fciqmc_options;

/* Per-iteration record. The estimators (nw_in .. num_in) describe the list at
 * the start of the iteration; nw_out / nd_out the list after it. */
typedef struct {
    int64_t iteration;        /* index of the iteration (0-based) */
    double shift;             /* S used in this iteration (relative to E0) */
    int64_t nw_in, nd_in;     /* sum |C_i|, number of occupied determinants */
    int64_t c0_in;            /* population of the reference determinant */
    double num_in;            /* sum_{i != 0} <D_i|H|D_0> C_i (Eq. 2 numerator) */
    int64_t nw_out, nd_out;
    int64_t attempts;         /* spawning attempts (= nw_in) */
    int64_t nulls;            /* attempts that drew a null excitation */
    int64_t spawn_events;     /* attempts that spawned at least one walker */
    int64_t spawned_walkers;  /* walkers spawned */
    int64_t death_walkers;    /* walkers removed by death */
    int64_t clone_walkers;    /* walkers added by cloning */
    int64_t merged_entries;   /* distinct determinants spawned onto */
    int64_t aborted_walkers;  /* spawned walkers discarded by the initiator rule */
    int64_t inserted_dets;    /* determinants newly occupied by spawning */
    int64_t heavy_attempts;   /* attempts from determinants with more than 256 walkers (32 for lists
                                 of few tiles), which the chunked spawning kernel (k_heavy) carries out */
} fciqmc_row;

/* Estimators of the current list (Sec. II, Eq. 2). Energies include e_core. */
typedef struct {
    int64_t iteration;        /* iterations completed */
    double shift;             /* S */
    double e_ref;             /* E0 + e_core, E0 = H_00 of the reference */
    double e_shift;           /* e_ref + S */
    double e_proj;            /* e_ref + proj_num / c0 (NaN if c0 == 0) */
    double proj_num;
    int64_t c0, n_walkers, n_dets;
    int32_t vary_shift;       /* 1 once the shift is being varied */
    int32_t status;           /* sticky device status (0 = OK) */
    int64_t list_slots;       /* slots in use in the main list (occupied + vacated) */
    int64_t compactions;      /* main-list compactions so far */
    int64_t exact_spawns;     /* spawn decisions taken by the exact FP64 path (diagnostic) */
    int64_t exact_deaths;     /* death decisions taken by the exact FP64 path (diagnostic) */
} fciqmc_estimates;

/* Dynamic state needed, together with the walker list, to resume a run. */
typedef struct {
    int64_t iteration;
    double shift;
    int32_t vary_shift;
    int32_t shift_counter;    /* iterations since the last shift update */
    int64_t nw_last_update;   /* N_w at the last shift update */
} fciqmc_state;

/* Facts fixed at creation. */
typedef struct {
    int32_t n_elec, n_orb, words;
    double e0;                /* H_00 without e_core */
    double e_core;
    double p_double;          /* as realised by the draw: d53 / 2^53 */
    uint64_t d53;             /* a spawn attempt is a double iff (r0 >> 11) < d53 */
    int64_t n_single_ref, n_double_ref;
    uint64_t reference[2];
    int64_t main_capacity, index_capacity, spawn_capacity, history_capacity;
    size_t workspace_bytes;
    int32_t grid_blocks;      /* persistent grid of the sweep kernels */
    int32_t num_sms;
    int64_t reference_excitations; /* double excitations of the reference tabulated with their spawning
                                      probability (on spin-coupled functions with their target
                                      function; with a permitted space those leaving it marked as
                                      null excitations); 0 when not tabulated: the reference's
                                      attempts read them */
} fciqmc_info;

/* Fills the defaults listed in fciqmc_options. */
void fciqmc_default_options(fciqmc_options *opt);

/* Device bytes fciqmc_create needs for this problem and these options
 * (opt may be NULL: defaults). Returns 0 for unsupported sizes. */
size_t fciqmc_workspace_bytes(int n_elec, int n_orb, const fciqmc_options *opt);

/* Creates a run (Sec. II problem statement).
 *   h, eri_s8       host arrays, layout above; copied.
 *   e_core          constant added to reported energies.
 *   n_elec, n_orb   electrons and spatial orbitals.
 *   ms2             2 S_z of the aufbau reference (ignored when opt->reference is set).
 *   orb_irrep       n_orb labels 0..7 (host), or NULL.
 *   tau             time step (> 0).
 *   initiator_threshold  < 0: plain FCIQMC; >= 0: a determinant is an initiator
 *                   iff |C_i| > threshold, the reference always (Sec. V B).
 *   opt             may be NULL.
 *   workspace       device pointer, 256-byte aligned, of workspace_bytes >=
 *                   fciqmc_workspace_bytes(); owned by the caller, must outlive the handle.
 *   cuda_stream     cudaStream_t (NULL: legacy default stream) all work is enqueued on.
 * Synchronising. On success *out receives the handle. */
int fciqmc_create(const double *h, const double *eri_s8, double e_core, int n_elec, int n_orb, int ms2,
                  const int32_t *orb_irrep, double tau, int32_t initiator_threshold,
                  const fciqmc_options *opt, void *workspace, size_t workspace_bytes, void *cuda_stream,
                  fciqmc_handle **out);

/* Enqueues n_iterations iterations on the stream. One iteration is the cycle of
 * Sec. II: for every walker a spawning attempt with the generator of Sec. VI
 * and the acceptance of Eq. 3, death/cloning of every determinant (Eq. 4), the
 * spawned walkers merged per determinant and annihilated into the main list
 * with the initiator filter (Sec. V A, V B), then the estimators (Eq. 2) and
 * the shift update. Asynchronous: device errors surface at the next
 * synchronising call. */
int fciqmc_step(fciqmc_handle *h, int32_t n_iterations);

/* Waits for the stream; returns the sticky device status. */
int fciqmc_sync(fciqmc_handle *h);

/* Synchronising: estimators of the current list into *out (host struct).
 * Returns the sticky device status (also in out->status). */
int fciqmc_estimators(fciqmc_handle *h, fciqmc_estimates *out);

/* Synchronising: copies up to max_rows of the most recent per-iteration rows,
 * oldest first, into rows (host); *n_rows receives the count. */
int fciqmc_history(fciqmc_handle *h, fciqmc_row *rows, int64_t max_rows, int64_t *n_rows);

/* Synchronising: number of occupied determinants of the current list. */
int fciqmc_n_dets(fciqmc_handle *h, int64_t *n_dets);

/* Synchronising: copies the main walker list (Sec. III: per occupied
 * determinant its bit string and signed walker count, with the stored
 * diagonal element) - the occupied determinants (W words each), their
 * populations and, if hdiag is not NULL, their stored H_ii - E0 - into host
 * arrays of capacity cap entries, in unspecified order (slot order of the
 * device list, not sorted: sort on the host if an order is needed); *n
 * receives the count.
 * Host arrays may be pinned or pageable. Returns FCIQMC_ERR_CAPACITY (with *n
 * set) if cap is too small. */
int fciqmc_get_walkers(fciqmc_handle *h, uint64_t *dets, int32_t *pops, double *hdiag, int64_t cap,
                       int64_t *n);

/* Synchronising: replaces the main walker list (Sec. III layout, as returned by
 * fciqmc_get_walkers) and, if st is not NULL, the dynamic state, so a run
 * resumes exactly (the random numbers are keyed by iteration and determinant,
 * not by history). dets: n x W words (host); pops: n nonzero populations;
 * hdiag: H_ii - E0 per determinant as returned by fciqmc_get_walkers, or NULL
 * to compute it. Determinants must be distinct and carry the run's electron
 * count. Clears the history and the device status. A rejected list (an
 * invalid entry or a repeated determinant: FCIQMC_ERR_INVALID_ARG) leaves the
 * run as it was. */
int fciqmc_set_walkers(fciqmc_handle *h, const uint64_t *dets, const int32_t *pops, const double *hdiag,
                       int64_t n, const fciqmc_state *st);

/* ---------------------------------------------------------------------------
 * Batched runs: several independent runs (any sizes, each with its own handle, workspace and seed)
 * advanced together by one CUDA graph whose independent branches are the runs' iteration sequences,
 * so their kernels execute concurrently. Results are those of advancing each run alone (the random
 * numbers are keyed per run and iteration). */
typedef struct fciqmc_batch fciqmc_batch;

/* Builds the graph for runs[0..n_runs) (same device; each run at most once), each advancing
 * iterations_per_launch iterations per launch. The batch does not own the runs; they must outlive
 * it. Synchronising. */
int fciqmc_batch_create(fciqmc_handle *const *runs, int n_runs, int32_t iterations_per_launch, fciqmc_batch **out);

/* Enqueues n_launches launches of the batch graph on cuda_stream, ordered after all work previously
 * enqueued on the runs' own streams; the runs' streams are made to wait for the batch, so later
 * calls on a run see its result. Asynchronous. */
int fciqmc_batch_step(fciqmc_batch *b, int32_t n_launches, void *cuda_stream);

/* Releases the graph and events (synchronising on the last batch stream). Accepts NULL. */
void fciqmc_batch_destroy(fciqmc_batch *b);

/* ---------------------------------------------------------------------------
 * Hash-partitioned runs (Sec. V A): the determinants of one run are divided among P partitions by
 * hash (Algorithm 1 fingerprint mod P), each partition a handle with its own main list, hash index, spawn
 * table and workspace (created with fciqmc_options.n_partitions = P and partition_index = r). An iteration
 * of the group is the paper's scheme: every partition spawns from its own determinants and routes each
 * spawn onto another partition's determinant into that partition's outbox (the spawned array ordered by
 * destination, Fig. 2); in the exchange each partition merges the entries bound for it; then every
 * partition annihilates its merged list against its own main list, and the run's N_w, C_0, numerator and
 * counters are summed over partitions for one row and one shift update, applied to all partitions. Here
 * the partitions share one GPU and the exchange reads the outboxes in device memory; the results are those
 * of the unpartitioned run (same random numbers), which the tests check against the oracle. */
typedef struct fciqmc_group fciqmc_group;

/* Device bytes fciqmc_group_create needs for n_partitions partitions and history_capacity rows (0: 2^16).
 * Returns 0 for n_partitions outside [2, 64]. */
size_t fciqmc_group_workspace_bytes(int32_t n_partitions, int64_t history_capacity);

/* Groups parts[0..n_partitions) (part r created with partition_index r, all with the same problem, time
 * step, initiator threshold and options, on the current device) into one run. workspace: device memory of
 * fciqmc_group_workspace_bytes(n_partitions, history_capacity) bytes, 256-byte aligned, owned by the caller.
 * cuda_stream: the stream the group's iterations are enqueued on. The group does not own the partitions;
 * they must outlive it. Synchronising. Returns FCIQMC_ERR_INVALID_ARG for mismatched partitions. */
int fciqmc_group_create(fciqmc_handle *const *parts, int32_t n_partitions, int64_t history_capacity, void *workspace,
                        size_t workspace_bytes, void *cuda_stream, fciqmc_group **out);

/* Enqueues n_iterations iterations of the partitioned run on the group's stream (ordered after work
 * previously enqueued on the partitions' streams, which are made to wait for it). Asynchronous. */
int fciqmc_group_step(fciqmc_group *g, int32_t n_iterations);

/* Waits for the group's stream; returns the group's sticky status (the first error of any partition, which
 * stops every partition before the failing iteration changes any committed list). */
int fciqmc_group_sync(fciqmc_group *g);

/* Synchronising: copies up to max_rows of the run's most recent rows (sums over the partitions; the
 * numerator added in partition order), oldest first, into rows (host); *n_rows receives the count. Each
 * partition's fciqmc_history holds its own list's rows. */
int fciqmc_group_history(fciqmc_group *g, fciqmc_row *rows, int64_t max_rows, int64_t *n_rows);

/* Releases the group's graph and events (synchronising). Accepts NULL. */
void fciqmc_group_destroy(fciqmc_group *g);

/* Host only, no GPU needed: the partition of each of n determinants (W = ceil(2 n_orb / 64) words each) in
 * a run of n_partitions partitions, owner[k] = fingerprint(D_k) mod n_partitions with the fingerprint of
 * Algorithm 1 (Sec. V): hash <- 1099511628211 hash + map(orbital_i) i over the occupied spin orbitals in
 * ascending order, i from 1, modulo 2^64, map(k) = the first two words of Philox4x32-10 with key
 * (0x46434951, 0x4D415031) and counter (k, 0, 0, 0). Returns FCIQMC_ERR_INVALID_ARG for a bad size,
 * partition count or NULL arrays. */
int fciqmc_owner(int n_orb, const uint64_t *dets, int64_t n, int32_t n_partitions, int32_t *owner);

/* Synchronising: dynamic state of the run. */
int fciqmc_get_state(fciqmc_handle *h, fciqmc_state *st);

/* Facts fixed at creation. Not synchronising. */
int fciqmc_get_info(const fciqmc_handle *h, fciqmc_info *info);

/* Kernels of one iteration, in launch order (indices into the kernel_ms array
 * of fciqmc_profile). */
#define FCIQMC_N_KERNELS 8
/* 0 compact_copy, 1 index_clear (three launches: the whole index, or the old
 * list's entries located then emptied), 2 index_fill, 3 compact_finish (no-ops unless
 * a compaction is due), 4 sweep (estimators, death, spawning), 5 heavy
 * (spawning from determinants with more than 256 walkers), 6 annihilate (with
 * the diagonal elements of the determinants it placed in new slots: two
 * launches), 7 finish (reductions, shift). */

/* Synchronising: runs n_iterations iterations exactly as fciqmc_step does, but
 * launching each kernel individually between CUDA events on the run's stream,
 * and adds each kernel's elapsed milliseconds, summed over the iterations,
 * into kernel_ms[FCIQMC_N_KERNELS] (host array, not cleared). */
int fciqmc_profile(fciqmc_handle *h, int32_t n_iterations, double *kernel_ms);

/* ---------------------------------------------------------------------------
 * Energy functional of a fixed amplitude vector and its density-matrix gradient.
 *
 * For n distinct determinants D_I (W words each) with real amplitudes c_I, and integrals h, (pq|rs)
 * in the layout of fciqmc_create,
 *   E(h, V) = sum_{I,J} c_I c_J <D_I|H|D_J> / sum_I c_I^2,
 * the variational energy of the vector (the Eq. 1 Hamiltonian restricted to it; a time-averaged
 * FCIQMC vector is the usual input). E is linear in h and V for fixed c; its gradient is the spin-
 * summed one-body density matrix gamma_PQ / c^T c with respect to h (symmetric convention: for a
 * symmetric change dh, dE = sum_PQ grad_h[P][Q] dh[P][Q]) and, with respect to each stored element
 * of the 8-fold packed ERIs, 1/2 the sum of the two-body density matrix Gamma_PQRS / c^T c over the
 * index orders stored there. The pairs that H connects are found once at creation (determinants
 * sharing a key D minus two electrons); the density matrices are computed at the first gradient
 * call and kept. All device memory comes from the caller's workspace. */
typedef struct fciqmc_rdm fciqmc_rdm;

/* Device bytes fciqmc_rdm_create needs (0 for unsupported sizes: n_orb <= 64, 2 <= n_elec <= 64,
 * n_elec < 2 n_orb, n_dets * n_elec (n_elec - 1) / 2 < 2^31). */
size_t fciqmc_rdm_workspace_bytes(int n_elec, int n_orb, int64_t n_dets);

/* Copies the determinants (device, n_dets x W, distinct, n_elec bits each) and amplitudes (device,
 * n_dets doubles) into the workspace and finds the connected pairs. Synchronising. */
int fciqmc_rdm_create(int n_elec, int n_orb, const uint64_t *dets_dev, const double *c_dev, int64_t n_dets,
                      void *workspace, size_t workspace_bytes, void *cuda_stream, fciqmc_rdm **out);

/* Enqueues E(h, V) for device integrals h_dev (n_orb^2) and eri_dev (packed) into e_dev (device,
 * one double). Asynchronous; the reduction order is fixed, so repeated calls give identical values. */
int fciqmc_rdm_energy(fciqmc_rdm *r, const double *h_dev, const double *eri_dev, double *e_dev);

/* Enqueues grad_h_dev (n_orb^2) = s dE/dh and grad_eri_dev (packed) = s dE/dV, with the scalar s
 * read from scale_dev (device, one double, e.g. the incoming gradient of a loss). Overwrites the
 * outputs. Asynchronous. */
int fciqmc_rdm_gradient(fciqmc_rdm *r, const double *scale_dev, double *grad_h_dev, double *grad_eri_dev);

/* Synchronising: counts[0..4] = key buckets, members of buckets with two or more determinants,
 * candidate pairs, connected single-excitation pairs and double-excitation pairs (the last two once
 * the gradient has been computed). Returns the construction status. */
int fciqmc_rdm_info(fciqmc_rdm *r, int64_t *counts);

/* Releases the host-side object (synchronising); the workspace stays the caller's. Accepts NULL. */
void fciqmc_rdm_destroy(fciqmc_rdm *r);

/* Largest walker list fciqmc_estimate_list_static accepts. Its scratch is one
 * static device array per device: FCIQMC_STATIC_MAX_DETS / 256 doubles (256 KiB)
 * and four 64-bit counters. */
#define FCIQMC_STATIC_MAX_DETS (1LL << 23)
/* fciqmc_estimate_list_static flag: the list holds spin-coupled functions (the
 * stored determinants of fciqmc_options.hphf runs). */
#define FCIQMC_STATIC_SPIN_COUPLED 1

/* The paper has no counterpart to this entry point: it is an allocation-free
 * form of fciqmc_estimators for callers that hold a walker list on the device
 * but cannot allocate device memory when they need its estimators. Examples
 * are a process that commits all device memory to a fixed pool up front, code
 * for which cudaMalloc's implicit device synchronisation is not acceptable,
 * and tools that only see device views of another program's list. It needs no
 * handle and no workspace.
 *
 * Computes, for the list (dets, pops) of n_dets entries (zero populations are
 * skipped): out[0] = sum |C_i|, out[1] = number of nonzero entries, out[2] =
 * C_0 (population of `reference`, 0 if absent), out[3] = sum_{i != 0}
 * <D_i|H|D_0> C_i, the projected-energy numerator, each term as in
 * fciqmc_estimators (with FCIQMC_STATIC_SPIN_COUPLED, sqrt(2) <D_i|H|D_0> for
 * open-shell functions), summed per 256-entry tile and then over tiles in
 * order, so the value agrees with fciqmc_estimators to rounding; out[4] = the
 * number of nonzero entries skipped as invalid (a bit at or beyond spin
 * orbital 2 n_orb, an electron count other than n_elec, a population of
 * INT32_MIN; with FCIQMC_STATIC_SPIN_COUPLED also M_s != 0 or a determinant
 * that is not the stored, smaller one of its spin-flip pair). Skipped entries
 * contribute to nothing and never index the integrals.
 *   h_dev, eri_dev  device arrays in the layout of fciqmc_create (n_orb^2 and
 *                   the 8-fold packed ERIs), read only.
 *   reference       host array of W words with n_elec bits set, none at or
 *                   beyond 2 n_orb (closed-shell with FCIQMC_STATIC_SPIN_COUPLED).
 *   dets_dev        device, n_dets x W words; pops_dev device, n_dets int32.
 *   flags           0 or FCIQMC_STATIC_SPIN_COUPLED.
 *   out_dev         device, 5 doubles, written by the last kernel.
 *   cuda_stream     stream the three kernels are enqueued on (asynchronous).
 * Returns FCIQMC_ERR_CAPACITY, before launching anything, if n_dets >
 * FCIQMC_STATIC_MAX_DETS; FCIQMC_ERR_UNSUPPORTED for sizes beyond the
 * library's limits; FCIQMC_ERR_INVALID_ARG for null pointers, unknown flags or
 * a reference that is not a determinant of the basis with n_elec electrons.
 * Scratch: the first call on each device looks up the device address of the
 * static array (cudaGetSymbolAddress, with that device current) and caches
 * it, so that first call should come before any stream capture. The array
 * stays resident on every device that loaded the library until the process
 * exits, is shared by all calls on that device and keeps the last call's
 * contents; each call clears its counters before use. Calls whose kernels
 * overlap on the GPU (different streams, no ordering) race on the array.
 * Allocates no memory: no cudaMalloc, no cudaFree, no allocating library call. */
int fciqmc_estimate_list_static(const double *h_dev, const double *eri_dev, int n_elec, int n_orb,
                                const uint64_t *reference, const uint64_t *dets_dev, const int32_t *pops_dev,
                                int64_t n_dets, int32_t flags, double *out_dev, void *cuda_stream);

/* Measurement utility (the paper has no counterpart): throughput of the random numbers every spawning
 * attempt draws, one Philox4x32-10 block keyed like an attempt's (the random-number contract of the
 * library: counter (attempt, tag, fingerprint), key (seed, iteration)). Evaluates about n_blocks blocks
 * over a grid that fills every SM of the current device (after a shorter warm-up launch), on cuda_stream,
 * timed with CUDA events, and writes blocks per second into *blocks_per_s (host). No spawning attempt can
 * take less than one block, so attempts/s of the walker cycle is at most this rate. Synchronising.
 * Returns FCIQMC_ERR_INVALID_ARG for n_blocks < 1 or a NULL output, FCIQMC_ERR_CUDA if a launch fails.
 * Allocates no device memory. */
int fciqmc_rng_throughput(int64_t n_blocks, void *cuda_stream, double *blocks_per_s);

/* Releases host-side resources (graphs, events). Synchronising. The
 * workspace stays the caller's. Accepts NULL. */
void fciqmc_destroy(fciqmc_handle *h);

/* Static text for a status code. */
const char *fciqmc_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* FCIQMC_H */
