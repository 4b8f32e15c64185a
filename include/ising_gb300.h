/*
 * ising_gb300.h -- C ABI of the GB300 (sm_103a) replica-parallel Metropolis
 * sweep with parallel tempering.
 *
 * Method: Dickson, Karimi & Hamze, "Importance of Explicit Vectorization for
 * CPU and GPU Software Performance" (arXiv:1004.0024).  The sampled model is
 * the Ising cost function of section 1,
 *     E(s) = -sum_i h_i s_i - sum_{edges (i,j)} J_ij s_i s_j ,   s_i = +-1,
 * (each undirected edge counted once), swept in the fixed sequential order of
 * Figure 1 with incrementally updated integer local fields
 * f_i = h_i + sum_j J_ij s_j (Figure 6: f_j -= 2 s_i J_ij after s_i flips),
 * under parallel tempering between adjacent inverse temperatures
 * (section 1, "use Parallel Tempering"; section 3.1).
 *
 * Conventions shared by every entry point
 *   - Every call returns int32_t: ISING_OK (0) or a negative ISING_ERR_*.
 *     ising_last_error() returns a thread-local message for the last failure.
 *   - The caller owns every array it passes; input arrays are copied before the
 *     call returns and may be freed afterwards.  The library owns all device
 *     state of a handle until ising_destroy().
 *   - Unless stated otherwise, pointers are HOST pointers.
 *   - Work is enqueued asynchronously on the handle's CUDA stream
 *     (ising_set_stream; default: the legacy default stream).  Calls that
 *     return data to host memory synchronise that stream.
 *   - A handle is not thread-safe: one host thread at a time per handle.
 *   - Spin index i = t*S + q for a graph declared as M identical slices of
 *     S = n/M spins (t = slice, q = site in the slice); M = 1 means "no slice
 *     structure declared".
 */
#ifndef ISING_GB300_H
#define ISING_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define ISING_OK 0
#define ISING_ERR_INVALID_ARG (-1)      /* bad size, pointer, ladder, mode   */
#define ISING_ERR_ASYMMETRIC_J (-2)     /* J_ij != J_ji or (i,j) w/o (j,i)   */
#define ISING_ERR_SELF_LOOP_OR_DUP (-3) /* i in row i, or a column repeated  */
#define ISING_ERR_FIELD_OVERFLOW (-4)   /* max_i |h_i|+sum_j|J_ij| too wide  */
#define ISING_ERR_NOT_INITIALISED (-5)  /* replicas_init not called yet      */
#define ISING_ERR_OOM (-6)              /* device allocation failed          */
#define ISING_ERR_CUDA (-7)             /* CUDA runtime error                */
#define ISING_ERR_TIMEOUT (-8)          /* a bounded device wait gave up     */
#define ISING_ERR_UNSUPPORTED (-9)      /* valid input outside kernel limits */

/* ---- random number generators ---- */
#define ISING_RNG_MT19937 0 /* one MT19937 per replica, init_genrand(seed + r);
                               PT swap stream init_genrand(seed + R)          */
#define ISING_RNG_PHILOX 1  /* Philox4x32-10, key (seed, r); see replicas_init */

typedef struct ising_s* ising_t;

/* Thread-local message describing the last non-OK status (never NULL). */
const char* ising_last_error(void);

/*
 * ising_create -- validate a sparse Ising model and upload its tables.
 *   n        number of spins (1 .. 2^24).
 *   row_ptr  [n+1] CSR offsets, row_ptr[0] = 0, non-decreasing.
 *   col      [row_ptr[n]] neighbour indices in [0, n); both directions of
 *            every edge are listed; no self loops, no repeats in a row.
 *   J        [row_ptr[n]] integer couplings, J of (i,j) equal to J of (j,i),
 *            |J| <= 32767.
 *   h        [n] integer biases.
 *   n_slices M >= 1: the graph is M identical slices of S = n/M spins in a
 *            Trotter ring (spin (q,t) coupled to (q,t+-1 mod M) with a
 *            per-site coupling; h and spatial couplings identical in every
 *            slice).  The declaration is verified; M = 1 accepts any graph.
 *   flags    reserved, pass 0.
 *   out      receives the handle.
 * Errors: INVALID_ARG (sizes, ranges, declared slice structure not found),
 * SELF_LOOP_OR_DUP, ASYMMETRIC_J, UNSUPPORTED (slice larger than the kernel's
 * shared-memory limits), OOM, CUDA.
 * Reference: the model of section 1; per-spin (target, J) records with the two
 * Trotter ("tau") edges kept apart from the spatial ones, section 2.2 and
 * Figure 6.
 */
int32_t ising_create(int32_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* J,
                     const int32_t* h, int32_t n_slices, uint32_t flags, ising_t* out);

/* Use `cuda_stream` (a cudaStream_t, NULL = legacy default stream) for all
 * later work of this handle. */
int32_t ising_set_stream(ising_t h, void* cuda_stream);

/*
 * ising_replicas_init -- allocate R replicas and draw their initial states.
 *   R          number of replicas = number of temperatures (1 .. 2^20).
 *   betas      [R] inverse temperatures, strictly ascending, > 0.  Slot r
 *              starts at temperature index r.
 *   seed       base seed.
 *   rng_mode   ISING_RNG_MT19937 or ISING_RNG_PHILOX.  MT19937: slot r owns
 *              init_genrand(seed + r); its first n outputs are the initial
 *              spins (s_i = +1 iff bit 31 is set) and sweep c consumes outputs
 *              n(1+c) .. n(2+c)-1, one per visited spin in index order.
 *              Philox4x32-10: key (seed, r), spin i = t*S + q of sweep c uses
 *              lane t&3 of counter ((t>>2)*S + q, c, instance, 0) and the
 *              initial spin lane t&3 of ((t>>2)*S + q, 0, instance, 3);
 *              instance is 0 for a handle made by ising_create.
 *   field_bits 16 or 32: width of the stored local fields.  16 requires
 *              max_i |h_i| + sum_j |J_ij| <= 32767.
 * Builds, in FP64 on the host, the flip thresholds
 * T_beta(k) = floor(2^32 exp(-2 beta k)) (flip iff k = s_i f_i <= 0 or
 * u < T_beta(k), Figure 1 with the Metropolis probability) and the swap
 * thresholds floor(2^32 exp(-(beta_{k+1}-beta_k) d)) up to their first zero.
 * When the swap tables would exceed 2^28 entries (a long, finely spaced
 * ladder) they are not built: sweeps work, and every call that would run a
 * PT pass returns UNSUPPORTED.
 * Re-initialising an initialised handle discards its replicas.
 * Errors: INVALID_ARG, FIELD_OVERFLOW, UNSUPPORTED, OOM, CUDA.
 */
/*
 * Acceptance mode of the flip thresholds (section 2.4 of the paper), used by
 * the next ising_replicas_init of the handle (a property of the handle, not
 * of checkpoints):
 *   ISING_ACCEPT_EXACT     T_beta(k) = floor(2^32 exp(-2 beta k)) in FP64 (default);
 *   ISING_ACCEPT_FAST      exp replaced by the paper's fast approximation:
 *                          2 ln^2 2 F(round(2^23 x log2 e) + 127 2^23), F(i) the
 *                          FP32 value with the bits of i (a linear interpolation
 *                          of 2^y between integer y, mean relative error 0),
 *                          0 below x = -126 ln 2;
 *   ISING_ACCEPT_ACCURATE  (2 ln^2 2 F(round(2^25 x log2 e) + 127 2^23))^(1/4),
 *                          relative error within (-0.01, 0.005), 0 below
 *                          x = -31.5 ln 2.
 * Both approximations are evaluated in FP32 steps (x = -2 beta k rounded
 * from FP64, round-half-even to the integer, the fourth root as two correctly
 * rounded square roots), then T = floor(2^32 min(1, e)), at most 2^32 - 1.
 * They bias the stationary distribution (by the approximation's error); the
 * swap thresholds stay exact.  Errors: INVALID_ARG (NULL handle, unknown mode).
 */
#define ISING_ACCEPT_EXACT 0
#define ISING_ACCEPT_FAST 1
#define ISING_ACCEPT_ACCURATE 2
int32_t ising_set_acceptance(ising_t h, int32_t mode);

int32_t ising_replicas_init(ising_t h, int32_t R, const double* betas, uint32_t seed,
                            int32_t rng_mode, int32_t field_bits);

/*
 * ising_sweep -- n sequential Metropolis sweeps (Figure 1) of every replica,
 * no PT pass in between.  Each sweep visits spins 0..n-1 of each replica in
 * index order (executed as a dependency-level wavefront that reproduces that
 * order exactly).  Asynchronous.  Errors: NOT_INITIALISED, INVALID_ARG, CUDA.
 */
int32_t ising_sweep(ising_t h, int64_t n);

/*
 * ising_pt_swap -- one parallel-tempering pass.  Pass p (0-based count of
 * passes so far) tries the pairs (k, k+1) with k = p mod 2 in ascending k and
 * swaps their temperature labels iff d = E(slot at k) - E(slot at k+1) <= 0 or
 * u < floor(2^32 exp(-(beta_{k+1}-beta_k) d)).  Words: MT19937 swap stream
 * init_genrand(seed + R), one per attempted pair in order; Philox: key
 * (seed, 0xFFFFFFFF), lane j&3 of counter (j>>2, p, instance, 1), j = k>>1.
 * Asynchronous.  Errors: NOT_INITIALISED, CUDA.
 */
int32_t ising_pt_swap(ising_t h);

/*
 * ising_run -- n sweeps with one PT pass after every swap_every-th sweep of
 * this call (swap_every <= 0: no PT).  The sequence is recorded once as a CUDA
 * graph per (n, swap_every) and replayed.  When all replicas fit on the GPU at
 * once the whole run is one persistent launch that keeps every replica in
 * shared memory and exchanges energies through a bounded grid barrier.
 * Asynchronous.  Errors: NOT_INITIALISED, INVALID_ARG, TIMEOUT (reported by a
 * later synchronising call), CUDA.
 */
int32_t ising_run(ising_t h, int64_t n, int32_t swap_every);

/*
 * ising_read_state -- copy the state to host buffers and synchronise.
 *   spins        [R*n] int8, slot-major (slot r, spin i at r*n + i), or NULL.
 *   fields       [R*n] int32 local fields f_i, slot-major, or NULL.
 *   energy       [R] int64 energies, by slot, or NULL.
 *   temp_of_slot [R] int32 temperature index held by each slot, or NULL.
 *   counters     [2] uint64 {sweeps done, PT passes done}, or NULL.
 * Errors: NOT_INITIALISED, TIMEOUT (a bounded device wait of an earlier
 * call gave up), CUDA.
 */
int32_t ising_read_state(ising_t h, int8_t* spins, int32_t* fields, int64_t* energy,
                         int32_t* temp_of_slot, uint64_t* counters);

/* accepted[R-1]: accepted swaps of pair (k, k+1) so far (host, synchronises). */
int32_t ising_read_swap_stats(ising_t h, uint64_t* accepted);

/*
 * ising_set_trotter -- split couplings.  The layered models of section 4 of
 * the paper come from a Trotter decomposition whose inter-slice coupling
 * depends on the temperature; the paper's original loop keeps the spatial
 * and Trotter parts of the field apart (sections 2.1 and 2.2, Figures 2 and
 * 3).  After this call the
 * state at temperature index k follows exp(-beta_k E_space - K[k] C):
 *   E_space  the cost function over the in-slice edges (h included),
 *   C        -sum over the Trotter (inter-slice) pairs of s s', every pair
 *            with unit weight (the graph's Trotter J values are ignored).
 * A flip of spin s has z = 2 (beta k_s + K k_tau), k_s = s f_space and
 * k_tau = s (s_{t-1} + s_{t+1}); a swap of the states at k, k+1 has
 * z = (beta_{k+1} - beta_k) dE + (K[k+1] - K[k]) dC, dE and dC the state at
 * k's E_space and C minus the state at k+1's.  Each product is rounded to
 * FP64 on its own; the threshold is T = min(floor(2^32 e^-z), 2^32 - 1), and
 * 2^32 - 1 for z <= 0; the move is taken iff T = 2^32 - 1 or the word u < T.
 * Flips look T up in a table built on the host with the C library's exp;
 * swaps evaluate e^-z on the device with a fixed FP64 exponential (Cody and
 * Waite's reduction, degree-13 Taylor polynomial, no fused operations).
 *   K  [R] host array by temperature index, finite (copied).
 * The current spins are kept; fields become the spatial ones and the
 * energies E_space (as ising_read_state reports them from then on), and C is
 * computed.  Words are drawn exactly as without split couplings.  Split
 * couplings last until the next ising_replicas_init.  Requires declared
 * slices with a Trotter ring (M >= 3) and the lean kernel (M in {4, 8, 16,
 * 32} or a multiple of 32 up to 1024, spatial degree <= 6, |J| <= 63, one
 * replica per block); not with learned passes or ising_run_noalloc.
 * Errors: INVALID_ARG (NULL argument, non-finite K, set twice),
 * NOT_INITIALISED, UNSUPPORTED (model or launch configuration without the
 * lean kernel, acceptance mode other than EXACT, a flip table above 8192
 * entries per temperature), OOM, CUDA.
 */
int32_t ising_set_trotter(ising_t h, const double* K);

/* C[R] (int64, by slot): -sum over Trotter pairs of s s' of each slot's
 * state under split couplings, zeros without them.  Synchronises.
 * Errors: INVALID_ARG, NOT_INITIALISED, TIMEOUT, CUDA. */
int32_t ising_read_trotter(ising_t h, int64_t* C);

/*
 * Host-side pieces of split couplings (no device needed; for tests and
 * tools):
 *   ising_split_flip_table  the flip tables ising_set_trotter builds: for
 *       temperature t (0 <= t < R) and k_s in [-ks, ks], k_tau in {-2, 0, 2},
 *       out[t * 3 (2 ks + 1) + (k_s + ks) * 3 + k_tau / 2 + 1] = T of
 *       z = 2 (betas[t] k_s + K[t] k_tau) (caller's buffer of R * 3 (2 ks + 1)
 *       uint32).  Errors: INVALID_ARG (R < 1, ks outside [0, 1364], NULL).
 *   ising_split_exp  the fixed FP64 exponential the device evaluates for
 *       swaps (the same source compiled for the host): e^x within about one
 *       ulp, 0 below -708.
 *   ising_split_swap_threshold  T of z = dbeta dE + dK dC as the device
 *       computes it (2^32 - 1 for z <= 0).
 */
int32_t ising_split_flip_table(int32_t R, const double* betas, const double* K, int32_t ks, uint32_t* out);

/*
 * ising_swap_thresholds -- the PT swap tables ising_replicas_init builds
 * (host only, for tests and tools): for pair k (0 <= k < R-1) and
 * 1 <= d < len[k], thr[off[k] + d] = floor(2^32 exp(-(betas[k+1]-betas[k]) d))
 * in FP64, len[k] the first d with a zero threshold or dmax (the energy
 * bound 2 (sum |h| + sum |J|) + 1 of the model); thr[off[k]] is unused.
 * *pt_ok = 0 when the tables would exceed 2^28 entries (PT is then refused).
 * off [R-1], len [R-1], pt_ok may be NULL; thr may be NULL to query
 * *n_entries, else it holds cap >= *n_entries values.  Errors: INVALID_ARG.
 */
int32_t ising_swap_thresholds(int32_t R, const double* betas, int64_t dmax, uint32_t* thr, int64_t cap,
                              int64_t* off, int32_t* len, int64_t* n_entries, int32_t* pt_ok);
double ising_split_exp(double x);
uint32_t ising_split_swap_threshold(double dbeta, double dK, int64_t dE, int64_t dC);

/* Energy and magnetisation m = sum_i s_i of the replica holding each
 * temperature index k (arrays [R], either may be NULL).  Synchronises. */
int32_t ising_read_observables(ising_t h, int64_t* energy_by_temp, int64_t* magnetisation_by_temp);


/*
 * ising_save / ising_load -- checkpoint blob of the full replica state (spins,
 * fields, energies, labels, MT19937 rings and positions, the generator key
 * {seed, instance}, counters, the count of learned passes; with split
 * couplings also K and the Trotter sums).  save: pass buf = NULL to query the
 * size in *size; otherwise cap >= *size.  load: the handle must be
 * initialised with the same n, R and modes (its seed may differ: the blob's
 * key replaces it); a blob with split couplings sets
 * them on a handle without them (ising_set_trotter) and needs the same K on a
 * handle with them; a blob without them is refused by a handle with them.
 * Running k sweeps, saving, loading into another handle and running m more
 * gives the same result as k + m straight sweeps.  Errors: NOT_INITIALISED,
 * INVALID_ARG, and those of ising_set_trotter.
 */
int32_t ising_save(ising_t h, void* buf, size_t cap, size_t* size);
int32_t ising_load(ising_t h, const void* buf, size_t size);

/* ising_set_seed -- continue the current state with other random numbers
 * (ISING_RNG_PHILOX only): the seed of every later Philox word (sweeps, PT
 * passes, learned passes) becomes `seed`; spins, fields, energies, labels
 * and counters are kept.  After ising_load this gives a second chain from a
 * checkpoint that is statistically independent of the saved chain's
 * continuation.  On a freshly initialised handle, the sweeps that follow are
 * those of a handle initialised with `seed` whose initial spins were set to
 * this handle's.  Errors: INVALID_ARG (NULL handle), NOT_INITIALISED,
 * UNSUPPORTED (MT19937 mode: its streams are seeded by ising_replicas_init). */
int32_t ising_set_seed(ising_t h, uint32_t seed);

/* Layout facts of a handle (for tests and tuning reports). */
typedef struct {
    int32_t n, slices, slice_size, levels, slice_depth, replicas;
    int32_t replicas_per_block, threads_per_block, blocks, smem_bytes;
    int32_t persistent_ok; /* 1 if ising_run fuses PT into one persistent launch */
    int32_t field_bits, rng_mode, kmax;
    int32_t fast_kernel;   /* 0 generic kernel, 1 register-resident kernel,
                              2 its lean variant (one replica per block,
                              M in {4,8,16,32} or a multiple of 32 up to
                              1024, degree <= 6, |J| <= 63; blocks of at
                              most 128 threads with two columns per thread
                              use a build for more resident blocks per SM),
                              3 the track-scheduled variant (lean's limits,
                              M <= 32, one thread per track of columns;
                              opt-in with ISING_LAUNCH_TRACK),
                              4 the packed variant (one replica per block of
                              one to eight warps, the columns' busy windows
                              packed into thread slots, fields gathered from
                              the neighbours' spins at each visit; M in
                              {8,16,32}, spatial degree <= 6, |J| <= 127,
                              plain couplings; the default where it applies) */
} ising_info_t;
int32_t ising_get_info(ising_t h, ising_info_t* out);

/* launch_flags of ising_set_launch */
#define ISING_LAUNCH_PERSISTENT 1 /* allow the persistent launch with fused PT */
#define ISING_LAUNCH_GENERIC 2    /* force the generic (shared-memory column) kernel */
#define ISING_LAUNCH_NO_LEAN 4    /* do not use the lean register-resident variant */
#define ISING_LAUNCH_TRACK 8      /* use the track-scheduled variant where it applies */
#define ISING_LAUNCH_NO_PACKED 16 /* do not use the packed variant (the lean one instead) */

/* Override the launch shape: replicas per block (0 = automatic, else a power
 * of two <= 32), threads per block (0 = automatic, else a multiple of 32 and
 * of the replicas per block, <= 1024) and launch_flags (ISING_LAUNCH_*; the
 * default of a new handle is ISING_LAUNCH_PERSISTENT).  Results are identical
 * for every accepted shape; only speed changes.  Errors: INVALID_ARG,
 * UNSUPPORTED (the shape does not fit the kernel's limits). */
int32_t ising_set_launch(ising_t h, int32_t replicas_per_block, int32_t threads_per_block,
                         int32_t launch_flags);

/* Launch statistics of a handle.  With profiling on, every sweep-kernel
 * launch is bracketed by CUDA events on its stream (graphs are bypassed) and
 * kernel_ms sums their elapsed times; ising_get_stats then synchronises. */
typedef struct {
    int64_t launches;       /* kernels this handle launched (all kinds)       */
    int64_t sweep_launches; /* of which sweep kernels                         */
    int64_t timed_launches; /* sweep launches bracketed by events             */
    double kernel_ms;       /* summed event time of the timed sweep launches  */
} ising_stats_t;
int32_t ising_set_profiling(ising_t h, int32_t on);
int32_t ising_get_stats(ising_t h, ising_stats_t* out);

/*
 * ising_run_noalloc -- ising_run for callers that cannot allocate device
 * memory when they run: code executing inside another framework's
 * allocation-free phase (a real-time loop, a region where device allocation
 * is forbidden) creates and initialises the handle beforehand, then advances
 * it with this call, which launches kernels and allocates nothing (no
 * cudaMalloc, cudaFree or allocating library routine).  The paper has no
 * counterpart; it is a deployment convenience.
 *   Same arguments and results as ising_run(h, n, swap_every), bit for bit.
 *   Requires ISING_RNG_PHILOX (MT19937 words are staged in a buffer that
 *   grows with replicas x spins), R <= 16384, and a handle whose replicas all
 *   fit on the GPU at once (ising_get_info(...).persistent_ok == 1).
 *   Scratch (grid-barrier and block counters, energies exchanged for the PT
 *   passes) is one file-scope device array of 128 KB that every GPU loading
 *   the library holds until the process exits.  ising_replicas_init resolves
 *   that array's device address (cudaGetSymbolAddress) on the handle's
 *   device, which also loads the device module holding it, so this call
 *   itself loads and allocates nothing; if the device current at this call
 *   has had no handle initialised on it, this call resolves the address
 *   first (and may then load the module): make such a first call before any
 *   stream capture and outside the allocation-free phase.  Every call shares
 *   the array and it keeps the last call's contents (the counters are
 *   cleared by each call), so calls whose kernels overlap on the GPU race:
 *   issue them on one stream, or otherwise order them.
 *   Each launch counts in ising_get_stats' launches and sweep_launches; no
 *   profiling events are recorded (their creation is not allocation-free).
 * Errors: NOT_INITIALISED, INVALID_ARG (n < 0, R > 16384, or swap_every >
 * 2^30 with n >= swap_every: one PT group would exceed a launch), UNSUPPORTED
 * (MT19937 mode, no persistent launch for this handle, split couplings set by
 * ising_set_trotter, or 0 < swap_every <= n on a ladder whose PT tables would
 * exceed 2^28 entries, the case ising_run refuses too), CUDA.
 */
int32_t ising_run_noalloc(ising_t h, int64_t n, int32_t swap_every);

/* ------------------------------------------------------------------------
 * Ragged batches: many independent instances (different models, sizes and
 * ladders) advanced together.  Not in the paper (its production runs sweep
 * "millions of systems", section 1, one CPU thread each); a batch lets one
 * GPU work on thousands of them at once.
 *
 * Each instance is described by ising_instance_t (host arrays, copied).
 * Instance b behaves exactly like a handle made with ising_create +
 * ising_replicas_init from the same arguments, except that its Philox
 * counters use instance = b (MT19937 streams depend only on its seed).
 * Execution: instances whose whole ladder fits one block ("resident") run all
 * sweeps of a call in one batched launch with the PT pass inside the block;
 * the others ("streamed") run one batched sweep launch per PT group followed
 * by one batched PT launch.  The sequence is recorded as one CUDA graph per
 * (n, swap_every) whose shape classes run as parallel branches.
 * ---------------------------------------------------------------------- */
typedef struct ising_batch_s* ising_batch_t;

typedef struct {
    int32_t n;              /* spins (see ising_create)                   */
    const int32_t* row_ptr; /* [n+1]                                      */
    const int32_t* col;     /* [row_ptr[n]]                               */
    const int32_t* J;       /* [row_ptr[n]]                               */
    const int32_t* h;       /* [n]                                        */
    int32_t n_slices;       /* M (see ising_create)                       */
    int32_t replicas;       /* R                                          */
    const double* betas;    /* [R] ascending, > 0                         */
    uint32_t seed;          /* base seed (see ising_replicas_init)        */
} ising_instance_t;

/* flags of ising_batch_create */
#define ISING_BATCH_PER_SWEEP 1 /* run with per-sweep batched launches, not persistent waves */

/* Create and initialise n_inst instances with one RNG mode and field width.
 * When every instance's model is one the packed kernel takes (layered, M in
 * {8, 16, 32}, spatial degree <= 6, |J| <= 127, at most 384 slots) and each
 * instance's ladder fits on the GPU at once, the batch runs as persistent
 * waves: whole instances grouped by block shape and level count, one
 * cooperative launch per wave and call that runs all the call's sweeps,
 * every instance's PT passes fused behind its own bounded barrier (flags:
 * ISING_BATCH_PER_SWEEP keeps the per-sweep launches).  Errors: as
 * ising_create / ising_replicas_init for the first failing instance (its
 * index is in ising_last_error()), INVALID_ARG (unknown flags). */
int32_t ising_batch_create(int32_t n_inst, const ising_instance_t* inst, int32_t rng_mode,
                           int32_t field_bits, uint32_t flags, ising_batch_t* out);
int32_t ising_batch_set_stream(ising_batch_t b, void* cuda_stream);

/* Autotuner: for every shape class (slice size, slices, replicas) time the
 * candidate launch shapes (resident vs streamed, replicas and threads per
 * block) on a representative instance and keep the cheapest in SM-time per
 * sweep.  flags reserved (0).  Results never change, only speed.  Runs
 * sweeps on scratch copies of the representatives, never on the batch.  A
 * batch of persistent waves has nothing to tune (returns OK). */
int32_t ising_batch_autotune(ising_batch_t b, uint32_t flags);

/* n sweeps of every instance with a PT pass after every swap_every-th sweep
 * of this call (swap_every <= 0: none).  Asynchronous. */
int32_t ising_batch_run(ising_batch_t b, int64_t n, int32_t swap_every);

/* State of instance `inst` (see ising_read_state; synchronises). */
int32_t ising_batch_read_state(ising_batch_t b, int32_t inst, int8_t* spins, int32_t* fields,
                               int64_t* energy, int32_t* temp_of_slot, uint64_t* counters);
int32_t ising_batch_read_swap_stats(ising_batch_t b, int32_t inst, uint64_t* accepted);

/* Launch facts of instance `inst`; resident = 1 if its whole ladder stays on
 * the GPU for a whole ising_batch_run call (one block per ladder, or the
 * persistent waves of a packed batch, fast_kernel 4). */
int32_t ising_batch_get_info(ising_batch_t b, int32_t inst, ising_info_t* out, int32_t* resident);
int32_t ising_batch_destroy(ising_batch_t b);

/*
 * ising_tc_gemm -- the bf16 tensor-core GEMM (tcgen05, FP32 accumulation in
 * tensor memory) used by the learned proposal's layers, exposed for tests.
 * All pointers are DEVICE pointers; work is enqueued on `stream`.
 *   C[m][n] = epi(sum_k A[m][k] B[n][k]), A [M][lda], B [N][ldb] bf16 row-major;
 *   epi: + bias[n] (bias may be NULL), ReLU if relu, zero where
 *   mask[m][ldm*...] <= 0 (mask bf16 [M][ldm] or NULL); C FP32 or bf16 (c_bf16).
 * Requires M % 128 == 0, K % 64 == 0, N in {32, 64, 128, 256}, leading
 * dimensions multiples of 8 and 16-byte aligned bases.  Errors: INVALID_ARG, CUDA.
 * The paper has no dense layers; this serves the learned proposal only.
 */
int32_t ising_tc_gemm(int32_t M, int32_t N, int32_t K, const void* A, int32_t lda, const void* B,
                      int32_t ldb, const float* bias, const void* mask, int32_t ldm, int32_t relu,
                      void* C, int32_t ldc, int32_t c_bf16, void* stream);

/*
 * Learned Trotter-column proposal (an addition; the paper samples with
 * single-spin Metropolis only).  For a handle declared as M <= 32 identical
 * slices, a "column" is the M spins (t*S + q, t = 0..M-1) of one site q.  Given
 * the rest of the replica, its conditional law is exp(-beta E_col(s)) with
 *     E_col(s) = -sum_t s_t phi_t - Jtau sum_t s_t s_{t+1 mod M}
 * (M = 2: one Trotter edge; M = 1: none), phi_t = h_q + sum over spatial
 * neighbours q' of J_qq' s_{q',t}: the share of the section 1 cost function
 * that involves the column.
 *
 * A network 33 -> 256 -> 256 -> 32 (ReLU hidden layers; inputs phi_t/8 for
 * t < M and beta at input M, logits of P(s'_t = +1) at outputs t < M) proposes
 * a whole column s' with independent bits; the move is accepted with the
 * exact Metropolis-Hastings probability
 *     min(1, exp(-beta (E_col(s') - E_col(s)) + log q(s) - log q(s'))),
 * so the chain keeps the Boltzmann law of every replica whatever the network.
 * Dense layers run on the tcgen05 GEMM (bf16 operands, FP32 accumulation);
 * training uses Adam (beta1 0.9, beta2 0.999, eps 1e-8) on FP32 master weights
 * with the mean Bernoulli negative log-likelihood of recorded columns.
 *
 * Parameter layout (float32, contiguous, ising_mlp_get/set_params):
 *   W1 [256][M+1], b1 [256], W2 [256][256], b2 [256], W3 [M][256], b3 [M];
 *   ising_mlp_n_params() gives the count.  Initial weights: uniform on
 *   +-1/sqrt(fan_in) from std::mt19937(seed), biases 0.
 * Pointers are HOST pointers; calls synchronise the network's stream (the
 * handle's stream for ising_mlp_collect / ising_learned_pass).
 */
typedef struct ising_mlp_s* ising_mlp_t;

/* Create a network for M slices (1..32) with room for `capacity` recorded
 * columns.  Errors: INVALID_ARG, OOM, CUDA. */
int32_t ising_mlp_create(int32_t n_slices, uint32_t seed, int64_t capacity, ising_mlp_t* out);
int32_t ising_mlp_set_stream(ising_mlp_t m, void* cuda_stream);
int64_t ising_mlp_n_params(ising_mlp_t m);
int32_t ising_mlp_get_params(ising_mlp_t m, float* out);
/* Replace the weights (layout above); resets the Adam moments. */
int32_t ising_mlp_set_params(ising_mlp_t m, const float* in);

/* Logits L [B][M] of inputs X [B][M+1] (rounded to bf16 like recorded
 * inputs).  B >= 1. */
int32_t ising_mlp_forward(ising_mlp_t m, int32_t B, const float* X, float* L);

/* Loss and gradient of one batch without changing the weights: X [B][M+1],
 * Y [B] bit t = 1 iff target s_t = +1; grad receives the gradient in the
 * parameter layout, *loss the mean negative log-likelihood.  B % 128 == 0. */
int32_t ising_mlp_grad(ising_mlp_t m, int32_t B, const float* X, const uint32_t* Y, float* grad,
                       float* loss);

/* Record the columns of every replica of handle h (R * S records:
 * X = (phi_t/8, beta), Y = the column's bits).  Requires h's M equal to the
 * network's M.  Errors: INVALID_ARG (capacity exceeded, slices differ),
 * NOT_INITIALISED. */
int32_t ising_mlp_collect(ising_mlp_t m, ising_t h);
/* As ising_mlp_collect; flags ISING_COLLECT_ORIENTED records each column in
 * the orientation its spatial field prefers: Y is the column if
 * sum_t s_t phi_t >= 0, else its complement (the training set of a network
 * meant for the flip-symmetric mixture proposal, which adds the other
 * orientation itself).  Errors as ising_mlp_collect, INVALID_ARG for
 * unknown flags. */
#define ISING_COLLECT_ORIENTED 1
int32_t ising_mlp_collect_flags(ising_mlp_t m, ising_t h, uint32_t flags);
int64_t ising_mlp_n_records(ising_mlp_t m);
int32_t ising_mlp_clear_records(ising_mlp_t m);
/* Copy records start .. start + n - 1 to the host: X [n][M + 1] (phi_t / 8 and
 * beta as stored, bf16 values widened to float), Y [n] (column bits).
 * Synchronous.  Errors: INVALID_ARG (NULL, range beyond the records). */
int32_t ising_mlp_get_records(ising_mlp_t m, int64_t start, int64_t n, float* X, uint32_t* Y);

/* `epochs` passes of Adam over the recorded columns in batches of `batch`
 * (a multiple of 128; records shuffled each epoch by std::mt19937_64(seed +
 * epoch), the last partial batch dropped) at learning rate lr.  *loss = mean
 * loss over the last epoch (may be NULL). */
int32_t ising_mlp_train(ising_mlp_t m, int32_t epochs, int32_t batch, float lr, float* loss);

/* Optional record of one learned pass, rows in visiting order (colour class,
 * then replica slot, then site within the class).  Arrays hold `capacity`
 * rows (>= R * S); NULL members are skipped. */
typedef struct {
    int64_t capacity;
    int32_t* replica;    /* [rows] replica slot                           */
    int32_t* site;       /* [rows] site q                                 */
    int32_t* phi;        /* [rows][32] phi_t, t < M                       */
    float* logits;       /* [rows][32] the network's logits, t < M        */
    uint32_t* old_bits;  /* [rows] column before the move (bit t: s_t=+1) */
    uint32_t* prop_bits; /* [rows] proposed column                        */
    uint8_t* accepted;   /* [rows]                                        */
} ising_learned_trace_t;

/* Counts of one learned pass. */
typedef struct {
    uint64_t proposed;        /* R * S                                        */
    uint64_t accepted;        /* accepted moves (including s' == s)           */
    uint64_t changed;         /* accepted moves with s' != s                  */
    uint64_t exact_decisions; /* decisions left to the FP64 product           */
} ising_learned_stats_t;

#define ISING_LEARNED_FP64_ONLY 1 /* decide every move by the FP64 product */
/* Flip-symmetric mixture proposal q_mix(s') = (q(s') + q(-s')) / 2: the sign
 * bit of word 33 (the second word of counter 2 + 4 * 8) takes q's draw or its
 * complement, and the Hastings ratio becomes q_mix(s) / q_mix(s') = q(s) /
 * q(s') * (1 + exp(-K(s))) / (1 + exp(-K(s'))), K(x) = sum_t x_t kappa_t,
 * kappa_t = log(c_t / (2^32 - c_t)) (FP32 screen with an error bound, FP64
 * otherwise, as for the plain ratio).  In this mode c_t is clamped to
 * [1, 2^32 - 256], so that every column has a positive probability.  A
 * column aligned along its Trotter ring then has its reversal as a likely
 * proposal. */
#define ISING_LEARNED_MIXTURE 2

/* One learned pass over handle h: every column of every replica once, the
 * colour classes of the slice graph (greedy colouring in site order; no two
 * sites of a class are spatial neighbours) in turn.  Random words:
 * Philox4x32-10 with key (seed, replica slot), counter (q, pass, instance,
 * 2 + 4j) giving words 4j..4j+3: word t < M draws s'_t = +1 iff
 * u_t < x_t = p_t 2^32 (p_t = sigmoid(logit_t) in FP32), an event of
 * probability exactly c_t 2^-32, c_t = ceil(x_t); q(s)/q(s') is the product of
 * those probabilities over the changed bits and log A is formed in FP64; word
 * 32 accepts iff log A >= 0 or log((u + 1/2) 2^-32) < log A.  The kernel
 * first evaluates both sides in FP32 with a proven error bound and falls back
 * to the FP64 product only when the bound cannot separate them, so every
 * decision equals the FP64 one (flags ISING_LEARNED_FP64_ONLY forces the
 * FP64 product for every move).  `pass` counts
 * the handle's learned passes since ising_replicas_init.  Energies are updated
 * by the exact integer dE and the local fields incrementally.  `stats`
 * (may be NULL) receives the counts of this pass.  With stats and trace both
 * NULL the pass is only enqueued on the handle's stream (no synchronisation);
 * a device-side error of such a pass is reported by the next call on the
 * network that synchronises.  Requires M <= 32, the network's M, R*S >= 1.
 * Errors: INVALID_ARG, NOT_INITIALISED, CUDA (including a GEMM timeout). */
int32_t ising_learned_pass(ising_t h, ising_mlp_t m, uint32_t flags, ising_learned_stats_t* stats,
                           const ising_learned_trace_t* trace);
/* Profiling of the fused network kernel inside learned passes: with it on,
 * each launch is bracketed by CUDA events on the handle's stream and the
 * totals (launches, real rows evaluated, milliseconds) accumulate. */
typedef struct {
    int64_t network_launches;
    int64_t network_rows;
    double network_ms;
} ising_mlp_stats_t;
int32_t ising_mlp_set_profiling(ising_mlp_t m, int32_t on);
int32_t ising_mlp_get_stats(ising_mlp_t m, ising_mlp_stats_t* out);
int32_t ising_mlp_destroy(ising_mlp_t m);

/*
 * Failure detection without a GPU fault (test support; the paper has no
 * counterpart).
 *   ising_set_alloc_cap(bytes): every later device allocation of the library
 *     larger than `bytes` fails with ISING_ERR_OOM before any CUDA call
 *     (0 removes the cap; process-wide).  An out-of-memory stand-in.
 *   ising_selftest_wait(kind, stream): launches a kernel whose bounded wait is
 *     made to run out -- kind 0 a grid barrier that one block never reaches,
 *     kind 1 an mbarrier phase that nothing completes -- and returns
 *     ISING_ERR_TIMEOUT when the kernel reported it (the normal outcome);
 *     the context stays usable.  Synchronises `stream` (a cudaStream_t).
 */
int32_t ising_set_alloc_cap(uint64_t bytes);
int32_t ising_selftest_wait(int32_t kind, void* stream);

/*
 * ising_measure_latencies -- the latencies, in SM clock cycles per
 * operation, of the operations on the critical path of one sweep level,
 * measured on the current device: cycles[0] a shared-memory load whose
 * address depends on the previous one, cycles[1] a dependent 32-bit integer
 * multiply-add, cycles[2] a dependent warp shuffle, cycles[3] a barrier of
 * one block's 8 warps (chains of 4096 operations in one 256-thread block,
 * clock64).  Not in the paper: it gives the latency floor of a sweep (levels
 * x the dependent chain of one level) that bench.py reports next to the
 * issue-rate roofline.  Synchronises the device.  Errors: INVALID_ARG (NULL
 * cycles), OOM, CUDA.
 */
int32_t ising_measure_latencies(double* cycles);

/* Release all device memory of the handle (NULL is ignored).  MT19937 word
 * buffers of 256 MB or more are not returned to the driver: up to two of
 * them are kept (after a device synchronisation) for the next handle whose
 * buffer fits, which then skips the allocation. */
int32_t ising_destroy(ising_t h);

/* Frees the word buffers kept by ising_destroy and the host copies of the
 * swap-threshold tables kept for the last two ladders (at most 2^24 entries
 * each; ising_replicas_init reuses them for a ladder with the same betas and
 * energy bound instead of evaluating its exponentials again).  Process-wide;
 * always ISING_OK.  An allocation that fails frees the word buffers and
 * retries by itself. */
int32_t ising_release_cached_memory(void);

#ifdef __cplusplus
}
#endif
#endif /* ISING_GB300_H */
