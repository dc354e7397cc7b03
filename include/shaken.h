/*
 * shaken.h -- C ABI of the GB300 shaken-dynamics library (libshaken.so).
 *
 * The shaken dynamics (D'Autilia, Andrianaivo, Troiani, arXiv:1908.07341,
 * Section 2) is a probabilistic cellular automaton on two L x L periodic
 * sublattices: sigma on Lambda_1 and tau on Lambda_2.  One full step is two
 * synchronous half-steps in which every spin of one sublattice is redrawn
 * independently given the other (Eq. "fact"):
 *
 *   half-step A (Eq. "leftTrans"):  P(tau_x = +1 | sigma) = e^{h}/(2 cosh h),
 *        h = <-h_x(sigma) = J (sigma_{x down} + sigma_{x left}) + q sigma_x
 *   half-step B (Eq. "rightTrans"): P(sigma_x = +1 | tau) = e^{h}/(2 cosh h),
 *        h = ->h_x(tau)   = J (tau_{x up} + tau_{x right}) + q tau_x
 *
 * with x = (i, j), x^up = (i, j+1), x^right = (i+1, j), x^down = (i, j-1),
 * x^left = (i-1, j) on the torus (Section 2) and (q, J) already multiplied by
 * beta (Section 2, "rescaling the interactions").
 *
 * Conventions fixed by this library (identical in the CPU oracle):
 *   - site index u = j*L + i (row j, column i);
 *   - SHK_INT8 planes: one int8 per site, +1 or -1, at byte u;
 *   - SHK_BITPACK planes: uint32 word w = u >> 5 holds sites 32w..32w+31,
 *     bit p = u & 31 (least significant bit = smallest u), bit set iff +1;
 *     requires L % 32 == 0 so that every row is a whole number of words;
 *   - step t (0-based) is half-step A with half-step index hs = 2t followed
 *     by half-step B with hs = 2t + 1 (the order of Eqs. leftTrans/rightTrans);
 *   - the draw is "+1 iff r < T[k]" with a 32-bit uniform r per site and the
 *     integer threshold table of shk_thresholds(); the uniform of site u is
 *     built from Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit seed,
 *     counter (hs, u >> 5, lattice_id, c), c = 0..7: the 32 output words
 *     R[0..31] of the 32-site block form a 32 x 32 bit matrix and
 *     r(u) = sum_b bit_{u & 31}(R[b]) 2^(31-b).  Trajectories are therefore a
 *     pure function of (initial state, q, J, seed, lattice_id, t).
 *   - observables of step t are exact int64 sums on the pair (sigma_t, tau_t)
 *     at the end of the step (Section 3.1 magnetisation; Eq. "gs_ham2"):
 *       [0] M_sigma = sum sigma_x            [1] M_tau = sum tau_x
 *       [2] S_q     = sum sigma_x tau_x
 *       [3] S_J     = sum sigma_x (tau_{x up} + tau_{x right})
 *       [4] C_nn    = sum sigma_x (sigma_{x up} + sigma_{x right})
 *     so m = M_sigma / L^2 and H(sigma_t, tau_t) = -(J S_J + q S_q).
 *
 * Memory and threads: device memory is always owned by the caller (for
 * example PyTorch tensors); the library never allocates or frees device
 * memory.  Host buffers are caller-owned.  Work is enqueued asynchronously on
 * the caller's CUDA stream (passed as void*, NULL = legacy default stream);
 * only the shk_read_* / shk_write_* calls synchronise that stream.  A handle
 * must not be used from two host threads at once.  No C++ exception and no
 * abort crosses this interface: every function returns a status code and
 * leaves a message for shk_last_error().
 */
#ifndef SHAKEN_H
#define SHAKEN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define SHK_OK          0
#define SHK_EINVAL    (-1)  /* an argument is out of range (message says which) */
#define SHK_ENOMEM    (-2)  /* a caller buffer is smaller than required          */
#define SHK_ECUDA     (-3)  /* a CUDA runtime call or kernel launch failed        */
#define SHK_ESTATE    (-4)  /* the handle is not ready (e.g. q, J never set)      */
#define SHK_EBUSY     (-5)  /* no free capacity; retry later (never blocks)       */
#define SHK_ETIMEOUT  (-6)  /* a bounded wait gave up                             */
#define SHK_ECANCELLED (-7) /* the job was cancelled                              */

/* ------------------------------------------------------------ enumerations */
#define SHK_BITPACK 1
#define SHK_INT8    2

#define SHK_INIT_ALL_UP   0
#define SHK_INIT_ALL_DOWN 1
#define SHK_INIT_RANDOM   2   /* each spin +1 with probability 1/2 */

#define SHK_HALF_A 0          /* sigma -> tau, left field (Eq. leftTrans)  */
#define SHK_HALF_B 1          /* tau -> sigma, right field (Eq. rightTrans) */

#define SHK_NOBS 5
#define SHK_OBS_M_SIGMA 0
#define SHK_OBS_M_TAU   1
#define SHK_OBS_S_Q     2
#define SHK_OBS_S_J     3
#define SHK_OBS_C_NN    4

#define SHK_MAX_L 262144      /* largest side accepted (2^18)                  */
#define SHK_MAX_STEP 0x80000000ull  /* step indices t must stay below 2^31     */

/* ------------------------------------------------------------ diagnostics */

/* Static English text for a status code. */
const char* shk_strerror(int status);

/* Message of the last failing call on this handle, or, for handle == NULL,
 * of the last failing handle-free call made by this host thread.  The string
 * is owned by the library and valid until the next call on the same handle
 * (or thread). */
const char* shk_last_error(const void* handle);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int shk_version(void);

/* Bounds checks of the debug build (libshaken built with -DSHK_DEBUG_BOUNDS,
 * build.py --debug-bounds): every global-memory access of the kernels checks
 * its index against its buffer; the first access out of range is recorded and
 * redirected to the buffer's first element, so no kernel faults.  *first_site
 * receives that access's site, translation unit << 16 | source line (units:
 * 1 sweeps, 2 batch and serving, 3 Section 3 kernels), or 0 if none, and the
 * record is cleared.  Synchronises the device.  SHK_ESTATE in the normal
 * build (*first_site = 0). */
int shk_debug_bounds(uint32_t* first_site);

/* ------------------------------------------------------------ thresholds */

/* The six integer thresholds of the per-site draw (Algorithm 3: the site
 * becomes +1 when its uniform is below e^h / (2 cosh h)), indexed k = 3*[s = +1] + n, where s is the
 * spin of the site itself and n in {0, 1, 2} the number of +1 neighbours in
 * the field, so that h = q*s + J*(2n - 2).  For h > 0,
 * T = min(2^32 - 1, floor(2^32 / (1 + e^{-2h}))) in IEEE double; for h < 0,
 * T(h) = 2^32 - T(-h); T(0) = 2^31.  Hence T[k] + T[5-k] = 2^32 whenever the
 * field is non-zero, and P(+1) = T[k] / 2^32 exactly.
 * Host-only (no GPU needed).  Returns SHK_EINVAL for non-finite q or J or a
 * NULL out. */
int shk_thresholds(double q, double J, uint32_t out[6]);

/* ------------------------------------------------------------ stateless hot path */

/* Bytes of one spin plane of side L in the given layout (0 if invalid). */
size_t shk_plane_bytes(int L, int layout);

/* One synchronous half-step over a whole L x L plane (Eq. leftTrans for
 * half = SHK_HALF_A, Eq. rightTrans for half = SHK_HALF_B; the sites are
 * independent given src, Eq. "fact").
 *   src, dst   device pointers to distinct planes of shk_plane_bytes(L, layout)
 *              bytes, 16-byte aligned (SHK_EINVAL otherwise): for A src = sigma,
 *              dst = tau; for B src = tau, dst = sigma.
 *   T          host array of six thresholds satisfying T[k] + T[5-k] = 2^32
 *              (as produced by shk_thresholds; SHK_EINVAL otherwise).
 *   seed, lattice_id, hs   key and counter words of the random numbers
 *              (hs = 2t for A of step t, 2t + 1 for B).
 *   obs_accum  nullable device array of SHK_NOBS int64 to which the fused
 *              reductions are ADDED (the caller zeroes it): A adds M_tau of dst
 *              to [1] and sum src_x (src_{x down} + src_{x left}), which equals
 *              C_nn of src, to [4]; B adds M_sigma of dst to [0], S_q to [2],
 *              S_J to [3].
 *   stream     cudaStream_t as void*.
 * Asynchronous.  Layout SHK_BITPACK requires L % 32 == 0; SHK_INT8 accepts
 * any 2 <= L <= SHK_MAX_L. */
int shk_halfstep(int layout, int half, const void* src, void* dst, int L,
                 const uint32_t T[6], uint64_t seed, uint32_t lattice_id,
                 uint32_t hs, int64_t* obs_accum, void* stream);

/* Launch-shape variants of the half-step sweep kernels (bit-packed, and int8
 * with L % 32 == 0): blocks drawn per thread, load prefetching, block size and
 * resident blocks per SM.  The choice does not change any result -- every
 * variant draws the same spins -- only the speed.  The setting is
 * process-wide and applies to launches enqueued after the call; the autotuner
 * (paper_1908_07341_gb300.tune) times the variants and sets the fastest.
 * A variant whose shape does not fit the lattice (rows of fewer blocks than
 * it walks or loads at once, or, for the vector variants, fewer blocks than
 * one full wave of threads needs) falls back to the one-block-per-thread
 * queue sweep for that launch.
 * The paper has no counterpart (it is a property of this implementation).
 * shk_sweep_variant_name returns NULL for an unknown (layout, variant);
 * shk_set_sweep_variant returns SHK_EINVAL for one. */
int shk_sweep_variant_count(int layout);
const char* shk_sweep_variant_name(int layout, int variant);
int shk_get_sweep_variant(int layout);
int shk_set_sweep_variant(int layout, int variant);

/* Fills a device plane with an initial state: all +1, all -1 or random
 * (+1 iff the site uniform of counter (plane_index, u >> 5, lattice_id,
 * 256 + c) under key init_seed is below 2^31).  plane: 16-byte aligned
 * (SHK_EINVAL otherwise).  Asynchronous. */
int shk_init_plane(int layout, void* plane, int L, int kind, uint64_t init_seed,
                   uint32_t lattice_id, uint32_t plane_index, void* stream);

/* Diagonal spin-spin sums of one bit-packed plane (Section 3.3, Table 1):
 *   out[k]          += sum_x s_x s_{x + (l_k, l_k)}     (SW-NE: (0,0) with (l,l))
 *   out[n_lags + k] += sum_x s_x s_{x + (l_k, -l_k)}    (NW-SE: (0,l) with (l,0))
 * over all x = (i, j) of the torus (translation average times L^2).
 * plane: device bit-packed plane (L % 32 == 0, 16-byte aligned); lags: host array of n_lags
 * (1..8) lags in [0, L); out: device int64[2 n_lags], ADDED to (caller
 * zeroes it).  Asynchronous. */
int shk_diag_correlations(const void* plane, int L, const int* lags, int n_lags, int64_t* out, void* stream);

/* The comparison dynamics of Section 3.2 for the square-lattice Ising model
 * H_G(s) = -J sum_x s_x (s_{x up} + s_{x right}) (the paper's parallel heat
 * bath on odd and even sites, whose stationary law is the Gibbs measure):
 * step t redraws the sites with i + j even (half-step index 2t), then those
 * with i + j odd (2t + 1), each +1 with probability e^h / (2 cosh h),
 * h = J (2n - 4), n the number of + among its four neighbours.  Thresholds
 * T[n] by the rule of shk_thresholds.  Only the redrawn sites consume
 * uniforms: numbered row by row, a = j (L/2) + floor(i/2), site a takes column
 * a & 31 of the block construction of this header with counter
 * (hs, a >> 5, lattice_id, 512 + c).  plane: device bit-packed sigma
 * (L % 32 == 0, 16-byte aligned), updated in place; dev_obs (nullable): n_steps rows of
 * (M, C_nn) int64, C_nn = sum_x s_x (s_{x up} + s_{x right}), H_G = -J C_nn.
 * Errors: SHK_EINVAL for a bad L, a NULL or misaligned plane, a non-finite J
 * or steps past 2^31.  Asynchronous. */
int shk_checkerboard_thresholds(double J, uint32_t out[5]);
int shk_checkerboard_run(void* plane, int L, double J, uint64_t seed, uint32_t lattice_id, uint64_t t0,
                         uint64_t n_steps, int64_t* dev_obs, void* stream);

/* Dynamics selectors of the coalescence and coupling-from-the-past calls:
 * the shaken dynamics (parameters q, J) and the checkerboard heat bath above
 * (parameter J; q ignored, may be NULL). */
#define SHK_DYN_SHAKEN 0
#define SHK_DYN_CHECKERBOARD 1
#define SHK_CFTP_MAX_K 20

/* Coalescence times (Section 3.2): for each pair, two copies of the chain
 * on an L x L torus (32 <= L <= 256, L % 32 == 0), one from all +1 and one
 * from all -1, driven by the same random numbers (seed, lattice id, steps).
 * Both dynamics preserve the order for J, q >= 0, so the two copies sandwich
 * every other start, and once the sigma planes agree they agree forever.
 * host_T[i] receives the first n <= max_steps with
 * sigma_top(n) == sigma_bottom(n), or max_steps + 1 if they never met.
 * dev_scratch: shk_coalescence_scratch_bytes(n_pairs) device bytes owned by
 * the caller.  Synchronous (waits for the result). */
size_t shk_coalescence_scratch_bytes(int n_pairs);
int shk_coalescence_times(int dynamics, int n_pairs, const int* L, const double* q, const double* J,
                          const uint64_t* seed, const uint32_t* lattice_id, uint64_t max_steps, void* dev_scratch,
                          size_t bytes, uint64_t* host_T, void* stream);

/* Perfect samples by coupling from the past (Propp-Wilson, Section 3.2), for
 * the same pairs as shk_coalescence_times.  The step from time -s to -s + 1
 * (s >= 1) uses the random numbers of forward step index s - 1, whatever the
 * starting time.  Attempt k = 0, 1, ..., k_max runs the all +1 and all -1
 * chains from time -2^k to 0; the first attempt after which their sigma planes
 * agree gives the sample.  host_k[i] receives that k, or -1 when no attempt
 * up to k_max (<= SHK_CFTP_MAX_K) coalesced.  dev_samples: device buffer of
 * n_pairs samples, sample_stride_bytes apart (a multiple of 4, at least
 * L^2 / 8 for the largest L, 4-byte aligned); sample i receives the
 * bit-packed sigma at time 0 (zero when host_k[i] is -1).  dev_scratch:
 * shk_cftp_scratch_bytes(n_pairs) device bytes.  Synchronous.  Exact draws
 * from the stationary law need J, q >= 0 (the monotone case). */
size_t shk_cftp_scratch_bytes(int n_pairs);
int shk_cftp(int dynamics, int n_pairs, const int* L, const double* q, const double* J, const uint64_t* seed,
             const uint32_t* lattice_id, int k_max, void* dev_samples, size_t sample_stride_bytes,
             void* dev_scratch, size_t bytes, int32_t* host_k, void* stream);

/* Measurement helper (no counterpart in the paper): blocks x 256 threads
 * each run iters Philox4x32-10 calls of the half-step's generator with no
 * memory traffic and XOR their outputs into *dev_out (device uint32).  The
 * caller times the launch on its stream; blocks * 256 * iters / seconds is
 * the measured Philox ceiling of the bit-packed draw.  Asynchronous. */
int shk_philox_peak(int blocks, uint32_t iters, uint32_t* dev_out, void* stream);

/* Bounded waits (no counterpart in the paper).  The int8 sweep variants that
 * move rows with bulk asynchronous copies (strip-bulk*) wait for each copy on
 * an mbarrier for at most about two seconds; a wait that gives up sets a
 * device fault word, lets the launch finish without the rest of its rows and
 * leaves the output incomplete.  shk_sweep_status synchronises `stream` and
 * returns SHK_ETIMEOUT (and clears the word) if that happened since the last
 * check; shk_read_observables and shk_read_spins check it as well.
 * shk_bulk_wait_timeout_test launches one warp that waits, at most
 * limit_cycles SM clock cycles (1..2^30), for a barrier no copy will complete,
 * and reports in *timed_out whether the wait gave up and set the word (it
 * should): the failure path, exercised without a fault.  Synchronous. */
int shk_sweep_status(void* stream);
int shk_bulk_wait_timeout_test(uint32_t limit_cycles, int* timed_out, void* stream);

/* Run-time specialisation of the half-step sweeps (no counterpart in the
 * paper).  The draw of Eqs. leftTrans / rightTrans compares the random bit
 * planes with the bits of the three class thresholds of (q, J); compiled with
 * those thresholds as constants, the masks fold into the logic and the sweep
 * runs faster.  A bit-packed or int8 half-step whose sweep variant has a
 * specialised form asks for it at each launch; the first request for a
 * (variant, thresholds, device) queues a compile with NVRTC for sm_103a
 * (about a second of host time), kept for the life of the process.  Until
 * that kernel is ready, and wherever NVRTC cannot be loaded or the compile
 * fails, the generic kernel runs: the spins and sums are identical either way.
 * shk_set_specialize(mode), process-wide: 0 off; 1 (default) compile on a
 * background thread, launches do not wait for it (at most 2 tables queued,
 * 512 per process; requests beyond these run generic), except for the
 * process's first compile, which runs on the calling thread; 2 compile at
 * first use and wait for it (at most two minutes, then the generic kernel
 * runs).  SHK_EINVAL for another mode; shk_get_specialize returns
 * the current one.  A compiled kernel is loaded at its first launch on a
 * stream that is not being captured into a CUDA graph (launches under capture
 * run generic until then).  shk_specialize_status
 * reports the entries compiled, failed and still queued and the host seconds
 * spent compiling (all entries), and copies the last
 * failure's log (truncated, NUL-terminated) into log when log_bytes > 0; any
 * pointer may be NULL.  The bounds-checked build never specialises. */
int shk_set_specialize(int mode);
int shk_get_specialize(void);
int shk_specialize_status(int* compiled, int* failed, int* queued, double* compile_seconds, char* log,
                          size_t log_bytes);
/* Queues the compile of the specialised form of sweep variant `variant` of
 * `layout` for the thresholds of (q, J), without launching anything and
 * without a GPU (the first launch on a device loads it); with wait != 0 it
 * also waits for the compile.  SHK_EINVAL for non-finite q or J, an unknown
 * variant or one without a specialised form; SHK_ESTATE when specialisation
 * is off, NVRTC cannot be loaded, the compile failed (wait != 0) or in the
 * bounds-checked build; SHK_ETIMEOUT when wait != 0 and the compile took
 * longer than two minutes.  For callers that know their tables ahead of time. */
int shk_specialize_prepare(int layout, int variant, double q, double J, int wait);
/* Stops the background compiler: waits for the compile in flight, if any,
 * and queues no more (tables not yet compiled then run generic).  Idempotent.
 * A process should call it before it exits while compiles may be running;
 * the library also does so from an exit handler, and the Python binding from
 * its interpreter-exit hook, which runs before any C exit handler. */
int shk_specialize_shutdown(void);

/* ------------------------------------------------------------ lattice handle */

typedef struct shk_lattice shk_lattice;

/* Device bytes a lattice of side L needs: both planes plus 512 bytes of
 * observable ring (256 of them reserved).  0 if (L, layout) is invalid. */
size_t shk_lattice_bytes(int L, int layout);

/* Creates a handle over caller-owned device memory dev_mem (at least
 * shk_lattice_bytes(L, layout) bytes, 256-byte aligned, kept alive by the
 * caller until shk_lattice_destroy).  The planes start undefined: call
 * shk_lattice_init or shk_write_spins.  Errors: SHK_EINVAL (bad L, layout,
 * alignment or NULL), SHK_ENOMEM (bytes too small). */
int shk_lattice_create(int L, int layout, void* dev_mem, size_t bytes, void* stream,
                       shk_lattice** out);

/* Releases the host-side handle; the device memory stays the caller's. */
void shk_lattice_destroy(shk_lattice* lat);

/* Sets sigma and tau to an initial state (see shk_init_plane; plane 0 is
 * sigma, plane 1 is tau) and the step counter to 0.  Only sigma matters for
 * the dynamics: half-step A overwrites tau without reading it. */
int shk_lattice_init(shk_lattice* lat, int kind, uint64_t init_seed);

/* Sets (q, J) (already rescaled by beta) and rebuilds the threshold table.
 * Non-finite values give SHK_EINVAL. */
int shk_set_params(shk_lattice* lat, double q, double J);

/* Sets the Philox key (seed) and the lattice id (third counter word). */
int shk_set_seed(shk_lattice* lat, uint64_t seed, uint32_t lattice_id);

/* Step counter t of the next step to run (checkpoint / resume: the state
 * after step t-1 plus (q, J, seed, lattice_id, t) determines the future). */
int shk_set_step(shk_lattice* lat, uint64_t step);
int shk_get_step(const shk_lattice* lat, uint64_t* step);

/* Runs n_steps full steps t, t+1, ..., t+n_steps-1 and advances the step
 * counter.  dev_obs, if not NULL, is a device array of n_steps * SHK_NOBS
 * int64 that receives the observables of every step (row s = step t+s).
 * Asynchronous on the handle's stream.  Errors: SHK_ESTATE if q, J were never
 * set, SHK_EINVAL if the step counter would reach SHK_MAX_STEP. */
int shk_run(shk_lattice* lat, uint64_t n_steps, int64_t* dev_obs);

/* Copies the observables of the last completed step to host_out (synchronises
 * the stream).  SHK_ESTATE if no step has run since the last init/write. */
int shk_read_observables(shk_lattice* lat, int64_t host_out[SHK_NOBS]);

/* Host <-> device spin transfer as int8 +/-1 arrays of L*L entries (u = j*L+i),
 * whatever the device layout; plane 0 = sigma, 1 = tau.  Synchronous. */
int shk_read_spins(shk_lattice* lat, int plane, int8_t* host_out);
int shk_write_spins(shk_lattice* lat, int plane, const int8_t* host_in);

/* Raw transfer of one plane in its device layout (shk_plane_bytes bytes),
 * host buffer caller-owned (pinned memory makes it asynchronous).  Enqueued on
 * the handle's stream; does not synchronise. */
int shk_upload_plane(shk_lattice* lat, int plane, const void* host_raw, size_t bytes);
int shk_download_plane(shk_lattice* lat, int plane, void* host_raw, size_t bytes);

/* Device pointer of plane 0 (sigma) or 1 (tau) inside the handle's memory. */
void* shk_plane_ptr(shk_lattice* lat, int plane);

/* ------------------------------------------------------------ batched lattices */

/* Many independent bit-packed lattices of uneven side L (32 <= L <= 65536,
 * L % 32 == 0), each with its own (q, J), seed and lattice id (for example one
 * lattice per cell of a (q, J) phase-diagram grid, as in Section 3.1 of the
 * paper, which ran one (q, J) point per CPU thread).  One persistent kernel
 * advances every lattice by steps_per_launch full steps per launch: each
 * lattice is cut into tiles of whole rows (about tile_sites sites each); a CTA
 * takes a tile and its halo rows into shared memory and steps it there.  A
 * run (shk_batch_run) is one launch of a CUDA graph whose while node repeats
 * the kernel n_steps / steps_per_launch times (the kernel counts the launches
 * down on the device; a one-thread kernel before the graph sets the count).
 * Every lattice follows
 * exactly the trajectory shk_run would give it (same random numbers), and its
 * five sums of every step t >= burn_in are folded into SHK_NSTATS exact int64
 * statistics:
 *   [0] sum M_sigma  [1] sum M_sigma^2  [2] sum |M_sigma|  [3] sum S_J
 *   [4] sum S_q      [5] sum S_J^2      [6] sum S_q^2      [7] sum S_J*S_q
 *   [8] sum C_nn     [9] sum C_nn^2    [10] number of steps added
 * from which <m>, <|m|>, the susceptibility N(<m^2> - <m>^2) and the moments
 * of H = -(J S_J + q S_q) follow exactly.  Device memory (shk_batch_bytes) is
 * the caller's; the handle must not be used from two host threads at once. */
#define SHK_NSTATS 11
typedef struct shk_batch shk_batch;

size_t shk_batch_bytes(int n, const int* L);
int shk_batch_create(int n, const int* L, const double* q, const double* J, const uint64_t* seed,
                     const uint32_t* lattice_id, void* dev_mem, size_t bytes, void* stream,
                     shk_batch** out);
void shk_batch_destroy(shk_batch* b);
const char* shk_batch_last_error(const shk_batch* b);
/* steps_per_launch in 1..32, block_threads in {128, 256, 512}, tile_sites >=
 * 1024 (rows per tile = max(1, min(L, tile_sites / L))).  Defaults 8, 256,
 * 2^18.  SHK_EINVAL if a tile would not fit in shared memory. */
int shk_batch_configure(shk_batch* b, int steps_per_launch, int block_threads, int tile_sites);
/* Initial state of every lattice (shk_init_plane with its lattice id); resets
 * the step counter and the statistics. */
int shk_batch_init(shk_batch* b, int kind, uint64_t init_seed);
/* n_steps (a multiple of steps_per_launch) more steps of every lattice;
 * asynchronous on the batch's stream. */
int shk_batch_run(shk_batch* b, uint64_t n_steps, uint64_t burn_in);
int shk_batch_get_step(shk_batch* b, uint64_t* step);
/* n x SHK_NSTATS statistics, n x SHK_NOBS sums of the last step, spins of one
 * lattice (int8 +/-1, plane 0 = sigma, 1 = tau).  Synchronous. */
int shk_batch_read_stats(shk_batch* b, int64_t* host_stats);
int shk_batch_read_observables(shk_batch* b, int64_t* host_obs);
int shk_batch_read_spins(shk_batch* b, int idx, int plane, int8_t* host_out);

/* ------------------------------------------------------------ serving */

/* A simulation request: one bit-packed lattice pair of side L (32 <= L <=
 * 8192, L % 32 == 0) run for n_steps full steps from an initial state, with
 * the statistics of the steps t >= burn_in (as in shk_batch).  deadline_ticks
 * (0 = none): a job not finished within that many scheduler ticks of its
 * submission is retired with status SHK_ETIMEOUT at the end of the tick that
 * reaches the deadline, queued or running; a running one reports the steps it
 * completed, their statistics and the hash of its sigma at that point. */
typedef struct {
    int L;
    double q, J;
    uint64_t seed;
    uint32_t lattice_id;
    int init_kind;          /* SHK_INIT_* */
    uint64_t init_seed;
    uint64_t n_steps;
    uint64_t burn_in;
    uint64_t deadline_ticks;
} shk_job;

/* A finished, cancelled or expired job.  sigma_hash is the 64-bit FNV-1a hash
 * of the final sigma plane's bytes (bit-packed layout; 0 for a job that never
 * ran or was cancelled); ticks count scheduler ticks. */
typedef struct {
    uint64_t job_id;
    int status;             /* SHK_OK, SHK_ECANCELLED or SHK_ETIMEOUT */
    uint64_t steps_done;
    int64_t stats[SHK_NSTATS];
    int64_t last_obs[SHK_NOBS];
    uint64_t sigma_hash;
    uint64_t submit_tick, admit_tick, done_tick;
} shk_result;

/* Continuous batching of jobs (no counterpart in the paper, which ran a fixed
 * grid of (q, J) points).  Queued jobs are admitted oldest first at each tick
 * while a slot is free and the job's device memory (three planes and a small
 * scratch) fits both the caller's arena and hbm_budget; every active job is
 * then advanced by min(steps_per_tick, remaining) steps in one launch of the
 * batched kernel, its lattice, step counter and random-number key resident on
 * the device; finished jobs are retired with exact statistics.  A job's result
 * is independent of the other jobs in the mix.  shk_server_tick is
 * synchronous (it waits for the tick's launch); shk_server_submit never
 * blocks (SHK_EBUSY when max_pending jobs already wait). */
typedef struct shk_server shk_server;
size_t shk_server_bytes(int max_slots, size_t arena_bytes);
int shk_server_create(int max_slots, size_t hbm_budget, void* dev_mem, size_t bytes, void* stream,
                      shk_server** out);
void shk_server_destroy(shk_server* s);
const char* shk_server_last_error(const shk_server* s);
/* A tick enqueues launches_per_tick launches of steps_per_launch steps each
 * (a job finishing part-way skips the rest) and waits for them.  Tiles hold
 * at most tile_sites sites, fewer while little work is active.  Defaults: 2
 * steps per launch, 16 launches per tick, 256 threads, 2^18 sites per tile,
 * 2^20 queued jobs. */
int shk_server_configure(shk_server* s, int steps_per_launch, int launches_per_tick, int block_threads,
                         int tile_sites, size_t max_pending);
int shk_server_submit(shk_server* s, const shk_job* job, uint64_t* job_id);
int shk_server_cancel(shk_server* s, uint64_t job_id);
/* One scheduler tick: admission, the tick's launches, retirement of finished
 * jobs, then expiry of jobs whose deadline tick has been reached.  Every call
 * advances the tick counter by one, with or without work. */
int shk_server_tick(shk_server* s, int* n_active, int* n_pending);
int shk_server_poll(shk_server* s, shk_result* out, int max, int* n_out);
int shk_server_stats(shk_server* s, uint64_t* tick, size_t* used_bytes);
/* Spins of a job that is running (admitted, not yet retired), between ticks:
 * plane 0 = sigma, 1 = tau as int8 +/-1 into host_out (L*L bytes, row-major;
 * bytes is the buffer's size), and in *steps_done the full steps it has
 * completed (the state is the one after that step, Eqs. leftTrans /
 * rightTrans).  No counterpart in the paper; it lets a caller inspect or
 * check a job in flight.  Synchronises the server's stream.  Errors:
 * SHK_EINVAL for a NULL argument, a bad plane, or a job id that is not
 * running; SHK_ENOMEM if bytes < L*L (nothing written). */
int shk_server_read_job(shk_server* s, uint64_t job_id, int plane, int8_t* host_out, size_t bytes,
                        uint64_t* steps_done);

/* ------------------------------------------------------------ allocation-free run */

/* Largest tau plane the library's own scratch array holds (8 MiB): bit-packed
 * L <= 8192, int8 L <= 2896. */
#define SHK_STATIC_SCRATCH_PLANE_BYTES (8u << 20)

/* The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory.  Examples are a plug-in inside a host
 * application that owns all device memory through its own pool, or a
 * latency-critical loop in which cudaMalloc's implicit synchronisation is not
 * acceptable.  It runs n_steps full steps t0 .. t0+n_steps-1 of the shaken
 * chain (the sigma-marginal of the alternate dynamics) in place on the
 * caller's sigma plane, and gives the same spins and sums as shk_run on a
 * handle holding that sigma.
 *   sigma     device plane of shk_plane_bytes(L, layout) bytes (input and
 *             output), 16-byte aligned (the sweeps use 16-byte vector loads).
 *   last_obs  nullable device array of SHK_NOBS int64, 8-byte aligned: the
 *             five sums of the last step (sigma, tau at its end).
 *   stream    cudaStream_t as void*; the device that is current at the call
 *             is the one used.
 * The call allocates nothing and calls no allocating routine.  The transient
 * tau plane and the observable accumulators live in a file-scope static device
 * array of 8 MiB + 256 B.  Every GPU that loads the library holds that array
 * until the process exits.  The array keeps the last call's contents;
 * accumulators are cleared at the start of every call.  Calls whose GPU work
 * overlaps (different streams or host threads) share the array and race.
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress); make the first call on a device before any stream
 * capture.  The call never compiles or loads a run-time specialised sweep
 * (loading a module allocates): it uses one only if an earlier call of the
 * library already loaded it on this device, and the generic sweep otherwise,
 * with the same spins and sums.
 * Errors: SHK_EINVAL for sizes beyond the scratch (message says the limit),
 * bad L/layout, a NULL or misaligned sigma, a misaligned last_obs, non-finite
 * q or J, or a step index reaching SHK_MAX_STEP (all before any launch);
 * SHK_ECUDA if a launch fails.  Messages via shk_last_error(NULL). */
int shk_shaken_run_static(int layout, void* sigma, int L, double q, double J, uint64_t seed,
                          uint32_t lattice_id, uint64_t t0, uint64_t n_steps, int64_t* last_obs,
                          void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SHAKEN_H */
