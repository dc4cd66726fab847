/*
 * mt.h -- C ABI of libmt, a GB300 (sm_103a) implementation of the particle
 * mass-transfer step of Engdahl, Schmidt & Benson, "Accelerating and
 * parallelizing Lagrangian simulations of mixing-limited reactive transport"
 * (arXiv 1811.05474), with the random-walk move before it and the A + B -> E
 * reaction after it.
 *
 * One time step (mt_step) is, in the paper's order:
 *   1. move      Eq. 2 with alpha_L = 0: x <- x + v dt + sqrt(2 D_rw dt) xi,
 *                xi standard normal per particle and axis; particles leaving
 *                [0, L] are mirrored back (Sec. 3).
 *   2. search    every pair within the cutoff s_max (Sec. 2.1), by a
 *                uniform-grid cell list built with a counting sort over cell
 *                keys (MT_SEARCH_CELL), or by testing all pairs
 *                (MT_SEARCH_BRUTE), or all pairs without a cutoff, the
 *                paper's full-matrix reference (MT_SEARCH_FULL, Sec. 1.1).
 *   3. weights   Eq. 3: nu_ij proportional to exp(-s_ij^2 / (8 D_mt dt)),
 *                normalised per row, P_ij = nu_ij / sum_j nu_ij (Sec. 1.1,
 *                MT_NORM_ROW), or symmetrically (P_ij + P_ji)/2, which
 *                conserves each species' total mass (MT_NORM_SYM, default).
 *   4. exchange  Eq. 4 and Eq. 7: dM_i = 1/2 sum_j P_ij (M_j - M_i),
 *                M <- M + dM for species A and B, from start-of-step masses
 *                ("matrix explicit", Sec. 1.1).
 *   5. react     A + B -> E, irreversible and at equilibrium, per particle
 *                after the transfer (Sec. 3, Sec. 7): m = min(A, B);
 *                A -= m; B -= m.
 *
 * Number formats.  Positions are fixed point: x = X * 2^-k with X a 64-bit
 * integer (k = frac_bits).  Drift and random-walk displacement are rounded to
 * that grid; the cutoff is s_max rounded down to it (Smax = floor(s_max 2^k)
 * ticks) and the pair test is exact integer arithmetic.  MT_FP64 computes
 * weights, normalisation, exchange and reaction in IEEE binary64.  MT_MIXED
 * computes the weights (exponentials), their row sums and the normalised
 * weights in binary32, and everything that touches a mass in binary64: the
 * masses are stored as binary64, and each flux term P_ij (M_j - M_i), its sum
 * over j, the update and the reaction are binary64 operations.
 * MT_MIXED_DF32 (not part of the paper's arithmetic; a faster variant) keeps
 * binary32 weights and stores each mass as an unevaluated sum of two binary32
 * numbers (about 48 significant bits), with binary32 flux terms summed with
 * compensation and compensated additions for the update and the reaction.
 *
 * Conventions.
 *   - Every function returns mt_status (0 = MT_OK, < 0 error) and never
 *     aborts the process; mt_last_error() describes the last failure on the
 *     calling thread.
 *   - Device memory: the library allocates none.  The caller allocates one
 *     device buffer of mt_workspace_bytes() bytes (256-byte aligned) and
 *     passes it to mt_create; the handle owns its contents until mt_destroy.
 *   - Work is enqueued on the stream given to mt_create (NULL: a stream the
 *     handle creates).  mt_step / mt_run return before the GPU finishes;
 *     mt_read_* and mt_sync wait for the stream and report device-side
 *     errors.
 *   - Arrays are axis-major (all x, then all y) and in the caller's particle
 *     order; the library reorders particles internally and always reads back
 *     in the order of mt_upload.
 *   - A handle is used by one host thread at a time.  Several handles may
 *     share a GPU on different streams.
 */
#ifndef MT_H
#define MT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MT_OK = 0,
  MT_ERR_INVALID = -1,    /* bad argument or parameter */
  MT_ERR_WORKSPACE = -2,  /* workspace NULL, too small or misaligned */
  MT_ERR_CUDA = -3,       /* a CUDA runtime call failed */
  MT_ERR_DEVICE = -4,     /* a device-side check failed (index out of range) */
  MT_ERR_TIMEOUT = -5,    /* a bounded device-side wait gave up */
  MT_ERR_STATE = -6       /* call out of order (e.g. step before upload) */
} mt_status;

enum { MT_SEARCH_CELL = 0, MT_SEARCH_BRUTE = 1, MT_SEARCH_FULL = 2 };
enum { MT_FP64 = 0, MT_MIXED = 1, MT_MIXED_DF32 = 2 };
enum { MT_NORM_SYM = 0, MT_NORM_ROW = 1 };
enum { MT_MEM_HOST = 0, MT_MEM_DEVICE = 1 };
enum { MT_WALLS_REFLECT = 0, MT_WALLS_PERIODIC = 1 };

typedef struct mt_params {
  int32_t dim;          /* 1 or 2 */
  int32_t frac_bits;    /* k of x = X 2^-k; 0 = choose (largest k with
                           s_max 2^k < 2^30 and L 2^k < 2^61) */
  int64_t n;            /* number of particles, 0 <= n < 2^31 */
  double L[2];          /* domain [0, L0] (x [0, L1]); L > 0 */
  double v[2];          /* constant advection velocity (Eq. 2) */
  double D_mt;          /* diffusion coefficient of the transfer (Eq. 3), > 0 */
  double D_rw;          /* diffusion coefficient of the random walk, >= 0 */
  double dt;            /* time step, > 0 */
  double cutoff;        /* s_max; <= 0 selects 3 sqrt(4 D_mt dt) */
  int32_t search;       /* MT_SEARCH_* */
  int32_t precision;    /* MT_FP64, MT_MIXED or MT_MIXED_DF32 */
  int32_t norm;         /* MT_NORM_* */
  int32_t react;        /* 1: apply A + B -> E after the transfer */
  uint64_t seed;        /* key of the Philox4x32-10 random-walk generator */
  uint64_t realisation; /* counter word separating independent realisations */
  int32_t observe_cap;  /* steps kept in the observables ring; 0 = off */
  int32_t cell_shift;   /* log2 of the cell width in ticks; 0 = choose */
  int32_t seg_target;   /* 1-d cell search: particles per segment of the
                           one-kernel step, in [16, 1024]; 0 = choose (the
                           largest that fits the staging, lowered so the
                           segments fill whole waves of the step's resident
                           CTAs on the current device) */
  int32_t walls;        /* MT_WALLS_REFLECT (Sec. 3, default) or
                           MT_WALLS_PERIODIC: the domain wraps, positions
                           live in [0, L) and pairs take the minimum-image
                           separation; needs s_max < L/2 per axis (any
                           value with MT_SEARCH_FULL); in a batch, each
                           realisation wraps on its own domain */
  int32_t species;      /* chemical species each particle carries: 0 or 2 =
                           A and B; 3 .. MT_MAX_SPECIES adds species 2, 3,
                           ... moved by the same transfer (Sec. 1.1: one
                           system of Eq. 4 per species, all with the same
                           weights; cost linear in the species count).  Only
                           A and B react; the others are conservative.
                           More than 2: the step runs as the multi-kernel
                           pipeline */
  int32_t stored_p;     /* 0: weights computed where they are used (two
                           passes, each pair's weight evaluated in both).
                           1 or more: the SPaM form (Sec. 6: the sparse
                           transfer matrix is stored and applied by sparse
                           matrix-vector products): each step stores nu_ij
                           once per unordered pair, in a band of b entries
                           per particle (its right neighbours in sorted
                           order), and both passes read it; 1 chooses b from
                           the mean density with headroom, b >= 2 sets it.
                           Entries past the band are recomputed, so any b is
                           correct.  1-d MT_SEARCH_CELL */
} mt_params;

#define MT_MAX_SPECIES 8

/* A batch: count independent 1-d realisations (the ensembles of repeated
 * simulations behind the paper's averaged results, Sec. 3 and Sec. 6.1)
 * advanced together, each step in one pass over all of them.  Realisation r
 * has n[r] >= 1 particles on its own domain [0, L[r]] with its own walls,
 * and its random walk uses the counter word realisation[r] (NULL:
 * p->realisation + r); everything else is shared.  Each realisation's result
 * is the one a single handle with the same parameters, n = n[r], L = L[r]
 * and realisation = realisation[r] would compute (up to the summation order
 * of ties and of a step the general pipeline redoes). */
typedef struct mt_batch {
  int32_t count;                /* realisations, >= 1 */
  int32_t reserved;             /* 0 */
  const int64_t* n;             /* host array [count] */
  const double* L;              /* host array [count] */
  const uint64_t* realisation;  /* host array [count] or NULL */
} mt_batch;

typedef struct mt_handle mt_handle;

/* Fill p with defaults: dim 1, n 0, L 1000, v 0, D_mt = D_rw = 0.1, dt 1,
 * cutoff 3 sqrt(4 D_mt dt), cell search, FP64, SYM, react on, seed 0,
 * observe_cap 0. */
mt_status mt_params_init(mt_params* p);

/* Copy p to out with every "choose" field resolved (frac_bits, cutoff,
 * cell_shift), exactly as mt_create will use them.  Validates p. */
mt_status mt_resolve(const mt_params* p, mt_params* out);

/* Device bytes the handle needs for p (validates p). */
mt_status mt_workspace_bytes(const mt_params* p, size_t* bytes);

/* Create a handle.  workspace: device pointer to >= mt_workspace_bytes
 * bytes, 256-byte aligned, owned by the caller and used by the handle until
 * mt_destroy.  stream: a cudaStream_t, or NULL for a stream the handle
 * creates and destroys.  The state is empty until mt_upload. */
mt_status mt_create(const mt_params* p, void* workspace, size_t workspace_bytes,
                    void* stream, mt_handle** out);

/* Batch versions of mt_resolve, mt_workspace_bytes and mt_create.  p gives
 * the shared parameters: dim must be 1 and search MT_SEARCH_CELL; p->n and
 * p->L[0] are ignored (the resolved p has n = sum of n[r] and L[0] = the
 * length of the axis the realisations share, side by side).  The default
 * frac_bits follows the largest L[r].  The handle then works like any
 * other, with the realisations' arrays concatenated in order (realisation 0's
 * particles first, each in its own coordinates [0, L[r]]); observables rows
 * hold 4 doubles per realisation and pairs never join two realisations.
 * The batch arrays are read during the call only. */
mt_status mt_batch_resolve(const mt_params* p, const mt_batch* b, mt_params* out);
mt_status mt_batch_workspace_bytes(const mt_params* p, const mt_batch* b, size_t* bytes);
mt_status mt_batch_create(const mt_params* p, const mt_batch* b, void* workspace,
                          size_t workspace_bytes, void* stream, mt_handle** out);

/* Autotuner for the 1-d cell path: times `steps` steps (after `warmup`
 * steps, the first of which captures the CUDA graph) of each candidate cell
 * width (cell_shift c - 1 .. c + 2 around the resolver's choice c) and
 * segment size (seg_target: the resolver's choice, 256, 512, 1024) on the
 * inputs x, A, B (as mt_upload takes them) and returns in *best the resolved
 * parameters of the fastest, and its time per step in *best_ms (may be
 * NULL).  b may be NULL (one system).  The candidates run one after another
 * on workspace (device, >= mt_autotune_workspace_bytes to try them all;
 * candidates that do not fit are skipped) and stream; the caller's arrays
 * are only read, and the workspace holds no usable state afterwards.  Other
 * parameter sets (2-d, brute force) have a single candidate.  Not part of
 * the paper: the cell list replaces its KD-tree, and this picks the list's
 * cell width and the kernel's tiling. */
mt_status mt_autotune_workspace_bytes(const mt_params* p, const mt_batch* b, size_t* bytes);
mt_status mt_autotune(const mt_params* p, const mt_batch* b, const double* x, const double* A,
                      const double* B, int32_t mem, void* workspace, size_t workspace_bytes,
                      void* stream, int32_t warmup, int32_t steps, mt_params* best,
                      float* best_ms);

/* ---- Serving ----------------------------------------------------------
 * A request server: simulations of different sizes and dimensions are
 * submitted over time (host arrays, copied at submission) and each is
 * admitted when a slot and room in the device pool are free (its footprint
 * is its workspace size).  Resident requests keep their state on the device
 * and are advanced in chunks of graph-replayed steps, each on its own
 * stream, so their work overlaps on the device; finished requests free
 * their slot and memory for the next.  Each request computes exactly what
 * a single handle with its parameters computes.  Not part of the paper. */
typedef struct mt_server mt_server;

enum { MT_REQ_QUEUED = 0, MT_REQ_RUNNING = 1, MT_REQ_DONE = 2, MT_REQ_FAILED = 3 };

typedef struct mt_server_config {
  int32_t max_active;   /* requests resident at once (streams), 1 .. 1024 */
  int32_t chunk_steps;  /* steps a resident request runs per round, >= 1 */
  int32_t backfill;     /* 1: admit a later request while the oldest waits
                           for memory; 0: strict arrival order */
  int32_t reserved;     /* 0 */
} mt_server_config;

typedef struct mt_request_info {
  int32_t state;        /* MT_REQ_* */
  int32_t status;       /* mt_status of a failed request */
  int64_t steps_done;
  double t_submit;      /* seconds since mt_server_create */
  double t_admit;
  double t_done;
  double gpu_ms;        /* sum of its chunks' times (CUDA events) */
  size_t footprint;     /* device bytes it holds while resident */
} mt_request_info;

typedef struct mt_server_summary {
  int64_t queued, running, done, failed;
  size_t pool_used;     /* device bytes held now */
  size_t pool_peak;     /* most device bytes held at once */
  int64_t step_samples; /* finished chunks (one step-latency sample each) */
} mt_server_summary;

/* Device bytes a request with params p holds while resident. */
mt_status mt_server_footprint(const mt_params* p, size_t* bytes);

/* pool: device memory (256-byte aligned) of pool_bytes, the HBM budget for
 * resident requests; owned by the caller, used until mt_server_destroy. */
mt_status mt_server_create(const mt_server_config* cfg, void* pool, size_t pool_bytes,
                           mt_server** out);

/* Queue a request: params p, host arrays x (dim*n), A, B (n), steps to run.
 * *id receives its identifier.  A request whose footprint exceeds the whole
 * pool is refused (MT_ERR_WORKSPACE); one with more than two species needs
 * mt_server_submit_species (MT_ERR_INVALID here). */
mt_status mt_server_submit(mt_server* s, const mt_params* p, const double* x, const double* A,
                           const double* B, int64_t steps, int64_t* id);

/* The same for any species count: M holds species*n doubles (species 0 is
 * A, 1 is B, then species 2, ...), each in the caller's particle order. */
mt_status mt_server_submit_species(mt_server* s, const mt_params* p, const double* x,
                                   const double* M, int64_t steps, int64_t* id);

/* One scheduling round (retire finished chunks, enqueue next chunks, admit
 * queued requests); does not wait for running work.  *queued and *running
 * (may be NULL) receive the counts after the round. */
mt_status mt_server_poll(mt_server* s, int32_t* queued, int32_t* running);

mt_status mt_server_info(const mt_server* s, int64_t id, mt_request_info* info);

/* Results of a finished request: masses (n each, the caller's order, host)
 * and up to cap observables rows (4 doubles each, the last ones; may be NULL
 * when cap = 0); *rows (may be NULL) receives the rows written. */
mt_status mt_server_result(const mt_server* s, int64_t id, double* A, double* B,
                           double* observables, int64_t cap, int64_t* rows);

/* Species sp (0 = A, 1 = B, ...) of a finished request: n doubles in the
 * caller's order into host memory out. */
mt_status mt_server_result_species(const mt_server* s, int64_t id, int32_t sp, double* out);

/* Forget a finished or failed request (frees its host copy). */
mt_status mt_server_release(mt_server* s, int64_t id);

/* Counters, and the first cap per-step latencies (ms; one per finished
 * chunk: its event time divided by its steps) into step_ms (host). */
mt_status mt_server_stats(const mt_server* s, mt_server_summary* out, float* step_ms,
                          int64_t cap);

/* Waits for the slots' streams, destroys resident handles and the server. */
void mt_server_destroy(mt_server* s);

/* Load the state: x (dim*n doubles, axis-major, each in [0, L_d]), A and B
 * (n doubles each).  mem says whether the three pointers are host or device
 * memory.  Positions are rounded to the grid (X = rint(x 2^k)).  Resets the
 * step counter and the observables.  Asynchronous for device pointers; host
 * arrays are copied before the call returns. */
mt_status mt_upload(mt_handle* h, const double* x, const double* A,
                    const double* B, int32_t mem);

/* Species s of a state with p->species > 2 (any s in [0, species); 0 is A
 * and 1 is B): set it from n doubles in the caller's particle order (host or
 * device memory, per mem), or read it back the same way.  mt_upload sets
 * A and B and zeroes species 2 and up; call mt_set_species after it and
 * between steps.  Both wait for the stream when mem is MT_MEM_HOST.  Errors:
 * MT_ERR_INVALID for s out of range or a NULL array, MT_ERR_STATE before
 * mt_upload. */
mt_status mt_set_species(mt_handle* h, int32_t s, const double* M, int32_t mem);
mt_status mt_read_species(mt_handle* h, int32_t s, double* M, int32_t mem);

/* Checkpoint and resume.  mt_save writes the handle's whole device state
 * (positions, ids, masses, step counter, observables, the step's internal
 * tables) and its resolved parameters to the file at path; it waits for the
 * stream.  mt_checkpoint_params reads the parameters back from such a file,
 * to create a handle for it (same parameters: mt_create, or mt_batch_create
 * with the same batch).  mt_load restores the state into such a handle; the
 * handle then continues exactly as the saved one would have (the
 * counter-based random walk is keyed by the step counter, which the state
 * holds), bit for bit on the same device kind.  The handle's own noise
 * source (mt_set_noise) replaces the saved one.  Errors: MT_ERR_STATE
 * (mt_save before mt_upload); MT_ERR_INVALID (unreadable or foreign file, or
 * a handle with other resolved parameters or realisations; the device state
 * is then unchanged). */
mt_status mt_save(mt_handle* h, const char* path);
mt_status mt_checkpoint_params(const char* path, mt_params* p);
mt_status mt_load(mt_handle* h, const char* path);

/* Random-walk noise for the following steps: a device pointer to dim*n
 * floats, axis-major and indexed by the caller's particle order, read by
 * every mt_step until it is replaced; NULL returns to the built-in
 * Philox4x32-10 / Box-Muller generator keyed by (seed, realisation, step,
 * particle).  The caller keeps the buffer alive and unchanged until the
 * steps that read it have run. */
mt_status mt_set_noise(mt_handle* h, const float* xi_device);

/* Enqueue one time step (move, search, transfer, react). */
mt_status mt_step(mt_handle* h);

/* Enqueue nsteps time steps.  With the built-in generator the steps are
 * replayed from a CUDA graph captured on the first call. */
mt_status mt_run(mt_handle* h, int64_t nsteps);

/* Wait for the handle's stream and report device-side errors. */
mt_status mt_sync(mt_handle* h);

/* Current masses (n doubles each) in the caller's particle order, into host
 * or device memory.  Waits for the stream. */
mt_status mt_read_masses(mt_handle* h, double* A, double* B, int32_t mem);

/* Current positions as doubles (dim*n, axis-major, caller's order). */
mt_status mt_read_positions(mt_handle* h, double* x, int32_t mem);

/* Current positions as exact grid ticks X (dim*n int64). */
mt_status mt_read_ticks(mt_handle* h, int64_t* X, int32_t mem);

/* Observables of the last min(steps, cap, observe_cap) steps, oldest first,
 * 4 doubles each: sum A, sum B, sum (A - B), mean A after the step (a batch
 * handle: 4 per realisation, realisation 0 first).  The sums are taken after
 * every step over fixed chunks of the state in a fixed order, in the
 * precision's arithmetic (binary64, or double-binary32 in MT_MIXED_DF32), so they are
 * bitwise reproducible.  out: host memory for 4*cap doubles (4*count*cap for
 * a batch).  *count receives the rows written. */
mt_status mt_read_observables(mt_handle* h, double* out, int64_t cap,
                              int64_t* count);

/* The observables of the last rows steps enqueued (1 <= rows <= min(steps
 * enqueued, observe_cap)), oldest first, in mt_read_observables' layout,
 * copied to out (host or device memory) by copies enqueued on the handle's
 * stream behind those steps; the call does not wait (with page-locked host
 * memory the copies are asynchronous too).  out holds the rows once the
 * stream has reached the copies (mt_sync, or an event recorded after the
 * call).  The copies run in stream order, so no later step overwrites a
 * row before it is copied. */
mt_status mt_copy_observables_async(mt_handle* h, double* out, int64_t rows);

/* The observables row of step number `step` (1 <= step <= steps enqueued,
 * and one of the last observe_cap), copied to out (host or device memory,
 * 4 doubles per realisation) by a copy enqueued on the handle's stream; the
 * call does not wait.  On the one-kernel path a step's observables are
 * computed beside the next step, so a pipelined reader asks for the row of
 * the step before the one it just enqueued (no extra work is enqueued); the
 * row of the last step enqueued is computed by this call first.  Errors:
 * MT_ERR_INVALID (step out of range, out NULL). */
mt_status mt_copy_observables_row_async(mt_handle* h, double* out, int64_t step);

/* Pairs {i, j} (caller's particle indices, i < j) within the cutoff at the
 * current positions, as the handle's search finds them.  pi, pj: device
 * pointers with room for cap entries (may be NULL when cap = 0); *count
 * receives the total number of pairs, which may exceed cap (then only cap
 * are written).  Pair order is unspecified.  Not for MT_SEARCH_FULL. */
mt_status mt_read_pairs(mt_handle* h, int32_t* pi, int32_t* pj, int64_t cap,
                        int64_t* count);

/* Steps taken since mt_upload. */
mt_status mt_steps_done(const mt_handle* h, int64_t* steps);

/* Test hook for the generator: out[4*i .. 4*i+3] = Philox4x32-10 of counter
 * (c0 + i, c1, c2, c3) under key (k0, k1), for i < n; out is a device
 * pointer.  Enqueued on the handle's stream. */
mt_status mt_philox(mt_handle* h, uint32_t c0, uint32_t c1, uint32_t c2,
                    uint32_t c3, uint32_t k0, uint32_t k1, int64_t n,
                    uint32_t* out);

/* Test hook for failure detection (not part of the paper).  With hold = 1
 * the first tile of the cell-list scan (the multi-kernel pipeline's
 * decoupled look-back prefix sum) stops publishing its status word, so every
 * later tile's wait for it runs out after spin_limit polls (0: the built-in
 * bound) and the step reports MT_ERR_TIMEOUT at the next mt_sync or
 * mt_read_* instead of hanging; the state of that step is then undefined.
 * hold = 0 restores normal operation; mt_upload clears both settings.
 * Errors: MT_ERR_STATE before mt_upload, MT_ERR_INVALID for hold not 0/1
 * or spin_limit < 0.  Waits for the stream. */
mt_status mt_test_hold_scan(mt_handle* h, int32_t hold, int64_t spin_limit);

/* The built-in random walk's standard normals (Eq. 2's xi) for particles
 * given by their index gid in a system (its caller order), at step `step`:
 * the values a single handle with p's seed and realisation draws for those
 * particles at that step (Philox4x32-10 keyed by the seed, counter (gid,
 * step, realisation); Box-Muller).  gid: device array of n indices (< 2^32);
 * out: device array of dim*n floats, axis-major, in the order of gid.  For
 * the domain decomposition (Sec. 2.2, Sec. 6): a slab's particles take the
 * same walk as in the undivided system (pass them to mt_set_noise).
 * Enqueued on stream (NULL: the default stream).  Errors: MT_ERR_INVALID
 * (dim, n < 0, NULL arrays). */
mt_status mt_walk_normals(const mt_params* p, const int64_t* gid, int64_t n, uint64_t step,
                          float* out, void* stream);

/* Per-kernel timing: with on = 1 every following step records a CUDA event
 * on the handle's stream before each of its kernels and one after the last
 * (graph replays included; turning it on or off drops a captured graph).
 * Not part of the paper; instrumentation for roofline measurements. */
mt_status mt_set_profiling(mt_handle* h, int32_t on);

/* Durations in milliseconds of the kernels of the last profiled step, in
 * launch order (waits for that step).  Where a step without a graph waits
 * for the host to read device state between two kernels, that idle time is
 * counted in neither.  ms: host array of cap floats; *count receives the
 * number of kernels in a step (may exceed cap). */
mt_status mt_read_profile(mt_handle* h, float* ms, int32_t cap, int32_t* count);

/* Name of kernel idx of the last profiled step ("" if out of range). */
const char* mt_profile_name(const mt_handle* h, int32_t idx);

/* Mass transfer (Eq. 3, 4, 7) plus, if react = 1, the A + B -> E reaction,
 * for n particles on a line, in binary64, with no device allocation.  The
 * paper has no counterpart: this is for callers that cannot call cudaMalloc
 * (their allocator belongs to a host application or another runtime, or
 * allocation is forbidden while their pipeline runs) and so cannot provide a
 * workspace.  They pass device arrays: x (n positions in [0, L], sorted
 * ascending), A and B (n masses) in, A_out and B_out (n masses, not aliasing
 * the inputs) out.  D_mt, dt, cutoff (<= 0: 3 sqrt(4 D_mt dt)) and norm
 * (MT_NORM_*) mean what they mean in mt_params; positions are rounded to
 * the grid that mt_resolve would choose for this L and cutoff.
 * Intermediates live in a fixed device array inside libmt, held by every GPU
 * that loads the library until exit: n may not exceed 1048576 (larger n is
 * rejected with MT_ERR_INVALID).  The first call on a device looks up that
 * array's address (cudaGetSymbolAddress).  All calls share the array:
 * calls that overlap on the GPU race and give wrong results.
 * Runs on stream (NULL: the default stream) and waits for it before
 * returning; MT_ERR_INVALID if a position is outside [0, L], NaN or out of
 * ascending order, and A_out and B_out are then undefined (they may have
 * been written). */
mt_status mt_transfer_1d_noalloc(const double* x, const double* A, const double* B,
                                 double* A_out, double* B_out, int64_t n, double L,
                                 double D_mt, double dt, double cutoff, int32_t norm,
                                 int32_t react, void* stream);

/* Device throughput probe (not part of the paper; it measures the peaks
 * that the binary64 and all-pairs passes are compared against).  which:
 * 0 binary64 fused multiply-adds, 1 binary32 fused multiply-adds, 2 binary32
 * fast exponentials (__expf), 3 binary64 exponentials (the library's exp),
 * 4 the binary64 exp(-t) the MT_FP64 weights (Eq. 3) use.  Runs
 * independent chains of that operation on 8 CTAs of 256 threads per
 * multiprocessor of the current device (about 10 ms per launch), times the
 * fastest of three launches with CUDA events on stream (NULL: the default
 * stream) and stores operations per second in *ops_per_s.  scratch: device
 * memory of at least 8 bytes per CTA (64 KiB covers 1024 SMs), overwritten.
 * Errors: MT_ERR_INVALID (which), MT_ERR_WORKSPACE (scratch), MT_ERR_CUDA. */
mt_status mt_probe_rate(int32_t which, void* scratch, size_t scratch_bytes, void* stream,
                        double* ops_per_s);

/* Test hook: the binary64 exp(-t) that the MT_FP64 weights (Eq. 3) use,
 * out[i] = exp(-t[i]) for t[i] >= 0 (Tang's table-driven method; about one
 * unit in the last place), so that tests can check it against the exact
 * exponential.  t, out: device arrays of n doubles.  Enqueued on stream
 * (NULL: the default stream).  Errors: MT_ERR_INVALID (n < 0, NULL arrays),
 * MT_ERR_CUDA. */
mt_status mt_test_exp_neg(const double* t, double* out, int64_t n, void* stream);

/* Description of the last error on this thread (static storage). */
const char* mt_last_error(void);

/* Release the handle (not the workspace).  Waits for its stream. */
void mt_destroy(mt_handle* h);

#ifdef __cplusplus
}
#endif
#endif
