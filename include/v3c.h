/*
 * v3c: polynomial commitment of trace columns on a GB300 (sm_103a).
 *
 * What it computes (V3DB, arXiv 2603.03065).  The paper's prover is built on
 * Plonky2 with its default field and FRI setup (Sec. 5, evaluation
 * environment).  It spends its time in FFT-based polynomial arithmetic over
 * a padded power-of-two domain G_B = 2^ceil(log2 G) (Sec. 2.1, "binning
 * effect"; Sec. 5.2, Metrics).  It commits with Poseidon (Sec. 4.3) in
 * balanced Merkle trees whose openings follow the bits of the leaf index
 * (Sec. 4.3; Sec. 4.4, MerkleOpen).  The paper fixes no numeric parameters.
 * This library implements the following readings:
 *
 *   field   F_p, p = 2^64 - 2^32 + 1, generator g = 7; every value passed
 *           in or out is a canonical uint64 in [0, p).
 *   LDE     for each column: a = iNTT_n(col); b_i = a_i * 7^i for i < n and
 *           0 for n <= i < N = n * 2^rate_bits; E = NTT_N(b), so that
 *           E_j = P(7 * w_N^j).  The LDE matrix is row-major [N][ld].  Row t
 *           holds E_{bitrev_{log N}(t)} of every column.  Columns c..ld-1
 *           are written as zero.
 *   hash    Poseidon, width 12, rate 8, capacity 4, S-box x^7, rounds 4 full
 *           + 22 partial + 4 full.  Each round does ARC, then the S-box, then
 *           the MDS.  The round constants come from SplitMix64 seeded with
 *           "V3DBPOS1".  The MDS is the first small-entry circulant drawn
 *           whose every square minor is nonzero.
 *   leaf    sponge in overwrite mode over the first `width` entries of a row
 *           (chunks of 8, no padding).  The digest is lanes 0..3.  Rows of
 *           width <= 4 are zero-padded to 4 instead of hashed.
 *   tree    node = Perm(left || right || 0^4)[0..4), with the left child at
 *           the even index, cut at a cap of 2^cap_height digests.
 *           Storage is level-major: level 0 (N leaf digests), level 1
 *           (N/2 digests), ..., level logN-h-1.  That is
 *           (2N - 2^(h+1)) * 4 uint64 in all.  The cap (level logN-h) is
 *           stored separately as [2^h][4].
 *
 * Conventions.  Every call returns a v3c_status.  No C++ exception crosses
 * the ABI and nothing aborts.  The caller owns every pointer it passes in.
 * "d_" pointers are device pointers of the context's device; "h_" pointers
 * are host pointers.  A cudaStream_t is passed as void*; NULL is the legacy
 * default stream.  A call that takes a stream only enqueues work on it.  The
 * results are valid once that stream reaches the point of the call.  Input
 * canonicity (< p) is a precondition.  V3C_FLAG_VALIDATE makes v3c_commit
 * and the serving loop check it and return V3C_EINVAL.
 */
#ifndef V3C_H
#define V3C_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    V3C_OK = 0,
    V3C_EINVAL = 1,     /* bad argument, shape or non-canonical input */
    V3C_ENOMEM = 2,     /* device memory or HBM budget exhausted */
    V3C_ECUDA = 3,      /* a CUDA runtime call failed; see v3c_last_error_detail */
    V3C_EAGAIN = 4,     /* not finished yet, or submit queue full */
    V3C_ETIMEDOUT = 5,  /* a bounded wait gave up */
    V3C_ENOTFOUND = 6,  /* unknown commit id or ticket */
    V3C_ECANCELED = 7   /* request cancelled or serving stopped */
} v3c_status;

typedef struct v3c_ctx v3c_ctx;
typedef uint64_t v3c_commit_id;

/* Limits of this build. */
#define V3C_MAX_LOG_N 22        /* input rows n = 2^log_n (log_n + rate_bits <= 25) */
#define V3C_MAX_LOG_LDE 25      /* N = 2^(log_n + rate_bits) */
#define V3C_MAX_RATE_BITS 4

#define V3C_FLAG_VALIDATE 0x1u  /* check that inputs are canonical */
#define V3C_FLAG_NO_GRAPH 0x4u  /* v3c_commit: launch stages directly instead of replaying a CUDA graph */

typedef struct {
    uint64_t hbm_budget_bytes;  /* resident commit objects + scratch; 0 = 90% of free memory */
    uint32_t max_inflight;      /* serving: concurrent batches on the device (0 = 4) */
    uint32_t flags;             /* V3C_FLAG_* applied to every call */
    uint32_t autotune;          /* 1 = v3c_commit times tile variants (NTT radix cap, stage tiles,
                                   leaf-hash CTA size) once per (log_n, rate_bits) shape on a
                                   synthetic problem and keeps the fastest; 0 = built-in defaults */
    uint32_t timeout_ms;        /* bounded host waits (0 = 60000) */
} v3c_config;

/* Returns a static English description of a status code. */
const char* v3c_strerror(v3c_status s);

/* Detail of the last failure on this context (thread-local copy, never NULL). */
const char* v3c_last_error_detail(v3c_ctx* ctx);

/* Library log messages (no counterpart in the paper).  level 0: a call
 * failed (the text of v3c_last_error_detail); 1: resources and choices
 * (plan tables built, scratch arena grown, autotuned tiles, serving started
 * or stopped); 2: detail (CUDA graphs captured, the FRI combination's load
 * path).  Messages up to max_level go to fn(user, level, text).  fn may be
 * called from any thread that calls the library and from the serving
 * thread, sometimes with the context's lock held: it must return quickly
 * and must not call into the library.  fn = NULL (the default) keeps the
 * library silent.  Errors: EINVAL (ctx NULL). */
typedef void (*v3c_log_fn)(void* user, int level, const char* text);
v3c_status v3c_set_log(v3c_ctx* ctx, v3c_log_fn fn, void* user, int max_level);

/* Creates a context on CUDA device `device`.  cfg may be NULL (defaults).
 * The first call on a device derives the Poseidon parameters and allocates
 * nothing else.  *out receives the context; v3c_destroy frees it.  Errors:
 * EINVAL (bad device or out NULL), ECUDA, ENOMEM. */
v3c_status v3c_create(int device, const v3c_config* cfg, v3c_ctx** out);

/* Stops serving, waits for in-flight work and frees every resident object,
 * plan table and scratch buffer of the context. */
v3c_status v3c_destroy(v3c_ctx* ctx);

/* Coset low-degree extension of c columns (the LDE reading above).
 *   d_cols   device, column-major [c][n] (column j at d_cols + j*n), n = 2^log_n
 *   d_lde    device, row-major [N][ld], N = n * 2^rate_bits; ld >= c.  Columns
 *            c..ld-1 are zero-filled.  A 16-byte aligned d_lde with even ld
 *            takes the vector-store path.
 * Scratch (about (n + N) * c * 8 bytes) is taken from the context's arena and
 * kept for reuse.  Limits: log_n <= V3C_MAX_LOG_N, rate_bits <= V3C_MAX_RATE_BITS,
 * log_n + rate_bits <= V3C_MAX_LOG_LDE.  Errors: EINVAL (shape, NULL),
 * ENOMEM (arena), ECUDA. */
v3c_status v3c_lde(v3c_ctx* ctx, const uint64_t* d_cols, uint32_t c, uint32_t log_n,
                   uint32_t rate_bits, uint64_t* d_lde, uint32_t ld, void* stream);

/* Merkle tree over 2^log_rows rows (the leaf and tree readings above).
 *   d_rows   device, row-major, stride ld (uint64), the first `width` entries hashed
 *   d_tree   device, (2N - 2^(h+1)) * 4 uint64, level-major (may be NULL iff h == log_rows)
 *   d_cap    device, 2^h * 4 uint64
 * d_tree and d_cap are 16-byte aligned (digests are stored as 16-byte pairs).
 * Uses no scratch.  Errors: EINVAL (h > log_rows, width > ld, NULL, a
 * misaligned d_tree or d_cap), ECUDA. */
v3c_status v3c_merkle(v3c_ctx* ctx, const uint64_t* d_rows, uint32_t ld, uint32_t width,
                      uint32_t log_rows, uint32_t cap_height, uint64_t* d_tree, uint64_t* d_cap,
                      void* stream);

/* Where a request's input lives (v3c_commit_desc.on_device). */
#define V3C_INPUT_HOST_COPY 0   /* host memory; the serving loop copies it at submit */
#define V3C_INPUT_DEVICE 1      /* device memory, kept alive by the caller until DONE */
#define V3C_INPUT_HOST_BORROW 2 /* host memory (pinned for an asynchronous copy), kept alive by the
                                   caller until DONE; copied to the device at admission */

/* One commit request: LDE of `cols` followed by the Merkle tree of its rows. */
typedef struct {
    const uint64_t* cols;  /* [c][n] column-major; see on_device */
    int32_t on_device;     /* V3C_INPUT_*; v3c_commit treats both host kinds alike (copied in the call) */
    uint32_t c;
    uint32_t log_n;
    uint32_t rate_bits;
    uint32_t cap_height;
} v3c_commit_desc;

/* Batched commit (many uneven shapes in one launch per stage).  For each desc
 * it allocates a resident object that holds the LDE [N][ld] (ld = c rounded
 * up to even) and the tree, and enqueues every stage on `stream`.  The stages
 * run as one persistent launch each over all descs.  A batch signature
 * (shapes, tiles) seen a second time is captured, stage launches and the
 * copy of the job table together, into a CUDA graph; later calls with that
 * signature rewrite the job table and replay the graph.  V3C_FLAG_NO_GRAPH,
 * V3C_FLAG_TIMING and large host inputs select direct launches.  ids[i]
 * receives the object id.  Host inputs are copied to the device inside the
 * call; large ones (at least 16 columns and 2^22 words) in column chunks on a
 * copy stream into a buffer of their own, each chunk's first two stages
 * starting when it lands; those copies do not wait for earlier work on
 * `stream`, so they overlap the previous commit's kernels.  The
 * objects stay resident until v3c_release.  Errors: EINVAL, ENOMEM (the HBM
 * budget would be exceeded; nothing is allocated), ECUDA. */
v3c_status v3c_commit(v3c_ctx* ctx, const v3c_commit_desc* descs, uint32_t nb, v3c_commit_id* ids,
                      void* stream);

/* ---------------- a commit split over several GPUs ----------------
 *
 * In bit-reversed row order, LDE rows [q N/G, (q+1) N/G) (G = 2^log_parts,
 * q < G) are the evaluations on the coset 7 w_N^kappa <w_{N/G}>, with
 * kappa = bitrev_{log G}(q), again in bit-reversed order: the LDE of rate
 * rate_bits - log_parts on a shifted coset, and a whole subtree of the
 * commit's Merkle tree.  With cap_height >= log_parts its top level is the
 * part's slice [q 2^h / G, (q+1) 2^h / G) of the cap, so G devices commit
 * one request with a single exchange: the coefficients (each device computes
 * those of its share of the columns with v3c_coeffs, then all gather them),
 * after which each device commits its part with v3c_commit_part and the cap
 * is the concatenation of the parts' caps in order of q.  (Scope: the
 * multi-GPU split of the LDE + Merkle commit; the paper's prover is one CPU
 * process, Sec. 5, evaluation environment.) */

/* Coefficients of the interpolant of each column, a = iNTT_n(col), natural
 * order, n^-1 applied: the first half of the LDE (the inverse transform)
 * without the coset shift.
 *   d_cols    device, column-major [c][n], n = 2^log_n
 *   d_coeffs  device, column-major [c][n]
 * Scratch c * n words from the context's arena when n > 2^10.  Errors:
 * EINVAL (shape, NULL), ENOMEM (arena), ECUDA. */
v3c_status v3c_coeffs(v3c_ctx* ctx, const uint64_t* d_cols, uint32_t c, uint32_t log_n, uint64_t* d_coeffs,
                      void* stream);

typedef struct {
    const uint64_t* coeffs;  /* device [c][n]: v3c_coeffs of all c columns (kept alive until the
                                call's work is done) */
    uint32_t c, log_n, rate_bits, cap_height;  /* the whole commit's shape */
    uint32_t log_parts;      /* G = 2^log_parts parts; log_parts <= min(rate_bits, cap_height) */
    uint32_t part;           /* q < G */
} v3c_part_desc;

/* Commits part q of the split above as a resident object: its N/G LDE rows
 * [N/G][ld] (object row t' is the commit's row q N/G + t'), its subtree
 * levels and its cap slice [2^(h - log_parts)][4]; v3c_commit_buffers
 * reports log_rows = log N - log_parts and cap_height = h - log_parts, and
 * v3c_open takes object row numbers.  Scratch c * N/G words from the arena.
 * Errors: EINVAL (shape, part, log_parts), ENOMEM (budget or arena), ECUDA. */
v3c_status v3c_commit_part(v3c_ctx* ctx, const v3c_part_desc* desc, v3c_commit_id* id, void* stream);

/* Device pointers and shape of a resident object (valid until release).
 * Any output pointer may be NULL. */
v3c_status v3c_commit_buffers(v3c_ctx* ctx, v3c_commit_id id, uint64_t** d_lde, uint32_t* ld,
                              uint64_t** d_tree, uint64_t** d_cap, uint32_t* log_rows,
                              uint32_t* cap_height);

/* Copies the cap ([2^h][4]) of a resident object to h_cap.  Waits for the
 * object's own work only (its completion event), not for later work on the
 * producing stream, so a caller may enqueue the next commit before reading
 * this one's cap.  Errors: ENOTFOUND, ECUDA. */
v3c_status v3c_commit_cap(v3c_ctx* ctx, v3c_commit_id id, uint64_t* h_cap);

/* Opening of leaf `leaf` (MerkleOpen, Sec. 4.4).  h_row receives the c
 * committed values of LDE row `leaf`.  h_path receives (logN - h) sibling
 * digests [k][4] for k = 0 .. logN-h-1: the sibling at level k is
 * level_k[(leaf >> k) ^ 1].  The path ends at cap entry leaf >> (logN - h).
 * Errors: ENOTFOUND, EINVAL (leaf >= N), ECUDA. */
v3c_status v3c_open(v3c_ctx* ctx, v3c_commit_id id, uint64_t leaf, uint64_t* h_row,
                    uint64_t* h_path);

/* Frees a resident object (after its work has completed). */
v3c_status v3c_release(v3c_ctx* ctx, v3c_commit_id id);

/* Bytes of HBM a resident commit of this shape occupies (LDE + tree + cap). */
uint64_t v3c_commit_footprint(uint32_t c, uint32_t log_n, uint32_t rate_bits, uint32_t cap_height);

/* ---------------- serving (continuous batching) ---------------- */

typedef struct {
    uint32_t queue_capacity;    /* pending submissions (0 = 4096) */
    uint32_t max_batch;         /* requests fused into one batched launch (0 = 32) */
    uint32_t max_inflight;      /* batches in flight on separate streams (0 = ctx setting) */
    uint32_t flags;             /* V3C_FLAG_VALIDATE */
    uint64_t slot_scratch_bytes; /* LDE scratch + staged inputs one pass may take (0 = 16 GiB);
                                    a pass always takes at least one request */
    uint64_t batch_elems;        /* LDE elements (c * 2^(log_n + rate_bits)) one batched launch may
                                    take (0 = 2^28; ~45 ms of work on one GB300), so a large
                                    request is not made to wait for a whole batch of its class;
                                    a pass always takes at least one request */
} v3c_serve_cfg;

typedef enum {
    V3C_REQ_QUEUED = 0,
    V3C_REQ_ADMITTED = 1,  /* memory reserved, inputs staged */
    V3C_REQ_RUNNING = 2,   /* part of a batch launched on the device */
    V3C_REQ_DONE = 3,      /* cap ready; object resident until release */
    V3C_REQ_FAILED = 4
} v3c_req_state;

typedef struct {
    double t_submit, t_admit, t_start, t_done;  /* seconds, steady clock of the context */
} v3c_req_times;

/* Starts the scheduler thread.  Requests are grouped by size class (LDE
 * elements c * 2^(log_n + rate_bits): up to 2^24, up to 2^27, above) and
 * admitted in arrival order within a class while their footprint fits the
 * HBM budget minus what is resident.  Each scheduler pass fuses the queued
 * requests of one class (the class whose oldest request arrived first) into
 * one batched launch on a free slot; up to max_inflight batches run at once
 * on separate streams, the small class's streams at the highest priority.
 * The last free slot goes to the class that has waited longest, and a
 * request that has waited more than 0.25 s for memory holds back newer
 * requests of the other classes.  A request that arrives while others are on
 * the device joins the next pass of its class. */
v3c_status v3c_serve_start(v3c_ctx* ctx, const v3c_serve_cfg* cfg);

/* Non-blocking submit.  desc->on_device says where desc->cols lives:
 * V3C_INPUT_HOST_COPY copies the host input into library memory before the
 * call returns.  V3C_INPUT_HOST_BORROW (pinned host memory) and
 * V3C_INPUT_DEVICE borrow the caller's buffer, which must stay alive until
 * the state reaches DONE.  *ticket receives the id, which is also the commit
 * id for v3c_open and v3c_release.  Errors: EAGAIN (queue full), EINVAL,
 * ENOMEM (the footprint exceeds the whole budget), ECANCELED (not
 * serving). */
v3c_status v3c_serve_submit(v3c_ctx* ctx, const v3c_commit_desc* desc, uint64_t* ticket);

/* Non-blocking poll.  Returns OK when DONE: h_cap (if not NULL) receives the
 * cap.  Returns EAGAIN while queued or running, or the failure status.
 * state and times may be NULL. */
v3c_status v3c_serve_poll(v3c_ctx* ctx, uint64_t ticket, v3c_req_state* state, uint64_t* h_cap,
                          v3c_req_times* times);

/* Stops the scheduler after the in-flight batches complete.  Queued
 * requests resolve to FAILED with ECANCELED. */
v3c_status v3c_serve_stop(v3c_ctx* ctx);

/* Host-side failure injection for tests of the serving loop (no counterpart
 * in the paper).  The scheduler thread raises an exception at the start of
 * its pass number `after_passes` from now (0: the next pass).  As after any
 * failure of that thread, batches already on the device complete (their
 * requests become DONE), queued and admitted requests resolve to FAILED with
 * ECANCELED, later submits return ECANCELED, and v3c_serve_stop still
 * releases the loop; the context stays usable for v3c_commit.  Errors:
 * EINVAL (not serving), ECANCELED (already stopped or failed). */
v3c_status v3c_serve_inject_failure(v3c_ctx* ctx, uint32_t after_passes);

/* ---------------- introspection ---------------- */

/* Number of this library's kernel launches enqueued by the context so far. */
uint64_t v3c_kernel_launches(v3c_ctx* ctx);

/* Number of v3c_commit calls served by replaying a captured CUDA graph. */
uint64_t v3c_graph_replays(v3c_ctx* ctx);

/* The autotuner's tile choices as text (no counterpart in the paper), so
 * that a later process on the same kind of GPU can skip the timing runs:
 *   {"sm_count": 152, "entries": [{"log_n": 20, "rate_bits": 3, "a_cols": 8,
 *     "c_q": 8, "c_qc": 2, "kcap": 4, "h_threads": 128}, ...]}
 * One entry per (log_n, rate_bits): the choices depend on the per-CTA shape,
 * not on the column count.  v3c_tune_export writes the text, NUL-terminated,
 * into buf (cap bytes) and its length into *len; with cap too small it
 * returns EINVAL with *len set, so a caller can retry.  v3c_tune_import
 * reads such text and replaces the context's choices for its shapes; with
 * v3c_config.autotune set, an imported shape is not timed again.  It refuses
 * (EINVAL, context unchanged) text for another SM count, malformed text and
 * out-of-range values (tiles powers of two up to 16384, c_qc <= c_q, kcap
 * 1..4, h_threads 64 or 128). */
v3c_status v3c_tune_export(v3c_ctx* ctx, char* buf, size_t cap, size_t* len);
v3c_status v3c_tune_import(v3c_ctx* ctx, const char* text);

/* Device memory accounting, for leak checks and budgeting:
 *   out[0]  bytes of resident objects (commit objects, FRI states, snapshots)
 *           the context counts against its HBM budget;
 *   out[1]  bytes currently allocated from the device's default
 *           stream-ordered pool by this process (every context and any other
 *           user of that pool; memory whose stream-ordered free has not yet
 *           executed still counts, so synchronise first);
 *   out[2]  bytes of the context's scratch arena (kept for reuse).
 * Errors: EINVAL (NULL), ECUDA. */
v3c_status v3c_mem_stats(v3c_ctx* ctx, uint64_t* out);

/* Per-stage timing.  With V3C_FLAG_TIMING in the context's flags, every
 * stage launch is bracketed by two CUDA events recorded on the stream it is
 * launched on.  v3c_stage_stats waits for the pending events and returns
 * the accumulated device time and launch count of each stage since the last
 * reset.  Stages: 0 = LDE stage A (inverse column DFTs), 1 = stage B (inverse
 * + coset + forward DFT), 2 = stage C (forward DFTs and row writes), 3 =
 * leaf hash, 4 = Merkle levels, 5 = FRI batch combination, 6 = FRI folds and
 * final coefficients, 7 = opening gathers (v3c_fri_query, v3c_open_batch,
 * v3c_snapshot_open_lists), 8 = SetEq grand products (the scan and the
 * zeroing launch as one stage), 9 = snapshot slot digests, 10 = snapshot
 * codebook digest.  Each stage launch also opens an NVTX range named after
 * its stage, with or without V3C_FLAG_TIMING. */
#define V3C_FLAG_TIMING 0x2u
#define V3C_NUM_STAGES 11
typedef struct {
    double ms[V3C_NUM_STAGES];
    uint64_t launches[V3C_NUM_STAGES];
} v3c_stage_stats_t;
v3c_status v3c_stage_stats(v3c_ctx* ctx, v3c_stage_stats_t* out, int reset);

/* Microbenchmarks of the integer multiply pipe (the denominator of the
 * integer roofline: the measured rate of 32x32->64 wide multiplies).
 * Independent chains of multiply-adds on every SM, `reps` timed runs after
 * one warm-up.  kind 0: 32x32->64 wide multiply-adds (mad.wide.u32);
 * kind 1: 32-bit multiply-adds (mad.lo.u32, one IMAD lane each).  *rate
 * receives operations per second (best run); *mhz (may be NULL) the SM clock
 * of that run, from the kernel's clock64() span over its event time.
 * Synchronous.  Errors: EINVAL (kind), ECUDA. */
v3c_status v3c_int_pipe_rate(v3c_ctx* ctx, uint32_t kind, uint32_t reps, double* rate, double* mhz);

/* v3c_int_pipe_rate with kind 0. */
v3c_status v3c_int_peak(v3c_ctx* ctx, uint32_t reps, double* rate, double* mhz);

/* Self-test of the library's bounded device waits (no counterpart in the
 * paper).  The kernels that wait on the GPU (the SetEq look-back, the copy
 * pipeline of the FRI combination) give every wait a time or poll limit,
 * after which they record an error word that the host turns into
 * V3C_ETIMEDOUT, and the context stays usable.  This call runs one
 * single-thread kernel whose wait can never be satisfied and that gives up
 * after `limit_us` microseconds of the GPU's global timer:
 *   kind 0: a shared-memory barrier (mbarrier) phase that expects two
 *           arrivals and gets one, waited on with the same bounded wait as
 *           the FRI copy pipeline;
 *   kind 1: a device word that nothing sets, polled with short sleeps.
 * Synchronous on `stream`.  Returns V3C_ETIMEDOUT when the wait gave up (the
 * expected outcome).  Errors: EINVAL (kind > 1, limit_us of 0 or above
 * 2000000), ECUDA. */
v3c_status v3c_wait_selftest(v3c_ctx* ctx, uint32_t kind, uint32_t limit_us, void* stream);

/* ---------------- allocation-free LDE ---------------- */

/* No counterpart in the paper: this entry point serves callers that cannot
 * allocate device memory.  One example is a process that shares the GPU
 * with a server whose caching allocator already owns the HBM.  Another is a
 * latency-critical path that must not take the device-wide synchronisation
 * that cudaMalloc/cudaFree may imply.  It computes exactly what v3c_lde
 * computes, with the same arguments, on the CURRENT CUDA device and with no
 * context.  It calls no cudaMalloc, no cudaFree and no other allocating
 * routine.
 *
 * Its work space is one file-scope device array of V3C_NOALLOC_SCRATCH_BYTES.
 * The library's modules load lazily, so the array is reserved on a device by
 * the first call of this entry point there, and held until the process
 * exits.
 * It needs 8 * (64 + T + c * (n + N)) bytes.  T is the shape's table size,
 * at most 2n + 2^14 words.  The c * (n + N) term is 0 when
 * n <= 2^(13 - rate_bits).
 * A larger shape returns V3C_EINVAL before anything is enqueued; for example
 * 135 x 2^14 rows at rate 3 is too large.  The caller still passes and owns
 * the input and output buffers.
 *
 * The first call on a device loads the module (reserving the array and the
 * stage kernels' code) and looks up the array's device address with that
 * device current.  Make that first call before any stream capture and
 * before another allocator takes the device's free memory; a first call
 * that finds no room for the array returns ENOMEM.  The address is cached
 * per device ordinal for the device's primary context: it is not valid
 * across cudaDeviceReset or in another context on the same device.  All
 * calls share the array, which keeps the last call's contents.  Every word
 * is rewritten before it is read, so nothing is cleared.  Calls whose work
 * overlaps on the GPU (different streams, no ordering) race on the array,
 * so order them.  Errors: EINVAL (shape, NULL, or over the limit), ENOMEM
 * (first call: no room for the array), ECUDA. */
#define V3C_NOALLOC_SCRATCH_BYTES (32u << 20)
v3c_status v3c_lde_noalloc(const uint64_t* d_cols, uint32_t c, uint32_t log_n, uint32_t rate_bits,
                           uint64_t* d_lde, uint32_t ld, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* V3C_H */
