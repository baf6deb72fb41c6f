/*
 * bm.h — C ABI of the GB300 threshold / symmetric-function query library.
 *
 * What is computed (Kaser and Lemire, "Threshold and Symmetric Functions over
 * Bitmaps", Sec. 1 "Formulation", Sec. 2.2 and 2.3): given N bitmaps
 * B_1..B_N of r bits and a threshold theta, the output bitmap has bit i set
 * iff c_i = |{k : bit i of B_k is set}| >= theta (the threshold function
 * T(theta, .)); for a symmetric function f given by its truth table over the
 * counts 0..N, bit i is set iff f(c_i) = 1.  The cardinality is the number of
 * ones of the output bitmap.
 *
 * Conventions shared by every entry point:
 *  - Bit layout (Sec. 2.1, "Uncompressed Bitmaps"): row i is bit (i mod 64)
 *    of 64-bit word i / 64, least significant bit first; a bitmap of r rows
 *    has ceil(r / 64) words.  Output bits at rows >= r are always written 0;
 *    input bits at rows >= r are ignored.
 *  - A repeated id counts once per repeat (integer weights by replication,
 *    Sec. 2.3).  theta = 0 selects every row; theta > N selects none; theta = 1
 *    is the union (wide OR) and theta = N the intersection (wide AND).
 *  - Streams: every query entry point is asynchronous on `stream` (a
 *    cudaStream_t passed as void*; NULL is the legacy default stream).
 *    Host arrays (ids, truth tables, query descriptors) are copied before the
 *    call returns and may be reused at once.  Device outputs are valid once
 *    the stream reaches the point of the call.
 *  - Ownership: the pool owns its device bitmaps; the caller owns output
 *    buffers (device memory it allocated, e.g. a torch tensor).
 *  - Errors: 0 is success; negative values are the BM_E* codes below and
 *    leave outputs untouched unless stated.  Device-side bounded waits that
 *    expire are reported by bm_pool_status().
 *  - Thread safety: calls on one pool are serialised by an internal mutex.
 */
#ifndef BM_H
#define BM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BM_OK 0
#define BM_EINVAL (-1)    /* bad argument: NULL pointer, n = 0, n > BM_N_MAX, bad kind ... */
#define BM_ERANGE (-2)    /* id >= capacity, id not loaded, position >= r or unsorted */
#define BM_ENOMEM (-3)    /* device or pinned allocation failed, or the pool budget is exceeded */
#define BM_ECUDA (-4)     /* a CUDA runtime call failed */
#define BM_ETIMEOUT (-5)  /* a bounded device-side wait expired */
#define BM_EBUSY (-6)     /* admission refused (server memory budget or slot table full) */
#define BM_ENOTREADY (-7) /* a result is not complete yet */

/* Largest number of inputs of one query (counts then fit 16 bits). */
#define BM_N_MAX 65535u

typedef struct bm_pool bm_pool;

/* ------------------------------------------------------------------------
 * Bitmap pool: a device-resident set of `capacity` bitmaps of r rows.
 * ---------------------------------------------------------------------- */

/*
 * Create a pool on CUDA device `device` for `capacity` bitmaps of `r_bits`
 * rows (1 <= r_bits <= 2^32).  Dense storage is one device allocation with
 * each bitmap padded to a multiple of 32 words (256 bytes), zero-filled.
 * `mem_budget` bounds the pool's total device bytes (dense storage, position
 * lists, their tile index and staging); 0 means no bound.  The paper keeps
 * the N bitmaps of a query in memory (Sec. 1, after the complexity tables);
 * the pool is that memory, resident in HBM.
 * Returns BM_ENOMEM if the dense storage alone exceeds the budget or cannot
 * be allocated.  *out receives the pool.
 */
int bm_pool_create(int device, uint64_t r_bits, uint32_t capacity, uint64_t mem_budget,
                   bm_pool** out);

/* Free every device and pinned allocation of the pool.  NULL is accepted. */
int bm_pool_destroy(bm_pool* pool);

/*
 * Load `count` dense bitmaps into ids first_id .. first_id + count - 1.
 * Bitmap j is read from words + j * src_stride_words (ceil(r/64) words);
 * `words` is a device pointer if words_on_device != 0, else host memory.
 * Input bits at rows >= r are cleared in the pool copy.  The per-bitmap
 * cardinality is computed on the device and kept on the host for the
 * selector's density features.  Synchronous.
 * Errors: BM_ERANGE if the id range exceeds capacity.
 */
int bm_pool_put_dense(bm_pool* pool, uint32_t first_id, uint32_t count, const uint64_t* words,
                      uint64_t src_stride_words, int words_on_device);

/*
 * Load sorted position lists (the "sorted integer list" form of a set,
 * Sec. 1 and 4.2) for ids first_id .. first_id + count - 1.  List j is
 * positions[offsets[j] .. offsets[j+1]) (offsets are host uint64, count + 1
 * entries, relative to `positions`); `positions` is device memory if
 * positions_on_device != 0, else host memory.  Lists must be strictly
 * increasing and every position < r (checked on the host for host input,
 * by a device check kernel for device input; BM_ERANGE otherwise).  A
 * per-list tile index (first list entry at each multiple of 8192 rows) is
 * built on the device.  In the pool each list starts 16-byte aligned and is
 * padded to a multiple of four entries (at most three extra entries per
 * list), which the sparse kernels read as whole 16-byte vectors.  Host input
 * passes through a temporary device copy of `count` lists' entries.
 * Synchronous.  A list loaded for an id replaces any earlier list of that id
 * (the earlier list's arena space is not reused).
 * Errors: BM_ENOMEM when the arena would pass 2^32 entries or the memory
 * budget.
 */
int bm_pool_put_positions(bm_pool* pool, uint32_t first_id, uint32_t count,
                          const uint32_t* positions, const uint64_t* offsets,
                          int positions_on_device);

/*
 * As bm_pool_put_positions, but list j holds the rows where bitmap j is 0
 * (the complement's positions): the sparse path can then take a dense input
 * through its few zeros.  By the complement identity (Sec. 2.3: NOT T(theta,
 * b) = T(N - theta + 1, NOT b), read input by input), a query with D such
 * inputs starts every ScanCount counter at D and subtracts one per listed
 * zero, so each counter still ends at the number of inputs holding its row;
 * results are identical on every path.  A bitmap without a dense copy gets
 * cardinality r - (list length).  Same arguments and errors as
 * bm_pool_put_positions.
 */
int bm_pool_put_complement_positions(bm_pool* pool, uint32_t first_id, uint32_t count,
                                     const uint32_t* positions, const uint64_t* offsets,
                                     int positions_on_device);

/*
 * Build the run-length form of ids first_id .. first_id + count - 1 from their
 * dense copies (which must be loaded; BM_ERANGE otherwise): the word-aligned
 * form of a compressed bitmap (Sec. 2.1, EWAH), in which every 64-bit word is
 * clean-0 (all zeros), clean-1 (all ones) or literal, kept per 256-word tile:
 * a tile that one clean run covers is only its class in a summary word; any
 * other tile is a container of two masks per 32-word slice (literal words,
 * clean-1 words), the literal ranks of the slices and the tile's literal
 * words.  Queries on BM_PATH_RLE read only the summaries of their inputs and
 * the containers of the tiles where an input mixes kinds.  Synchronous (the
 * words pass through host memory once).  Rebuilding an id appends a new form;
 * the earlier one's space is not reused.  Errors: BM_ENOMEM over the memory
 * budget.
 */
int bm_pool_put_rle(bm_pool* pool, uint32_t first_id, uint32_t count);

/* Statistics of id's run-length form: maximal runs of words of one kind
 * (clean-0, clean-1, literal), literal words, and the device bytes of its
 * form (containers and one 4-byte summary per tile).  Any pointer may be
 * NULL.  BM_ERANGE if the id has none. */
int bm_pool_rle_info(const bm_pool* pool, uint32_t id, uint64_t* runs, uint64_t* literal_words,
                     uint64_t* device_bytes);

typedef struct bm_pool_info_t {
    uint64_t r_bits;           /* rows per bitmap */
    uint64_t words;            /* ceil(r / 64) */
    uint64_t stride_words;     /* words between consecutive bitmaps in dense storage */
    uint32_t capacity;         /* number of ids */
    uint32_t dense_loaded;     /* ids holding a dense bitmap */
    uint32_t lists_loaded;     /* ids holding a position list */
    uint32_t sm_count;         /* streaming multiprocessors of the pool's device */
    uint64_t device_bytes;     /* device bytes held by the pool */
    const uint64_t* dense_base;/* device address of id 0's dense words */
    uint32_t rle_loaded;       /* ids holding a run-length form */
    uint32_t reserved;
} bm_pool_info_t;

/* Fill *out with the pool's shape. */
int bm_pool_info(const bm_pool* pool, bm_pool_info_t* out);

/*
 * Host-side cardinality of bitmap `id` (from its dense load, else its
 * position list length).  BM_ERANGE if the id holds neither.
 */
int bm_pool_bitmap_cardinality(const bm_pool* pool, uint32_t id, uint64_t* out);

/*
 * Synchronise the pool's device and report device-side failures since the
 * previous call: BM_ETIMEOUT if a kernel's bounded wait expired (its outputs
 * are then undefined), else BM_OK.  Clears the flag, and after an expired
 * wait also resets the per-call cardinality accumulators a kernel that gave up
 * may have left unfinished, so later calls start clean.
 */
int bm_pool_status(bm_pool* pool);

/*
 * Shape of the pool's dense kernel (results are identical for every choice;
 * bm_pool_autotune picks one by measurement).
 *   variant 0: direct streaming loads, 256 threads per CTA; `threads` and
 *              `stages` ignored.
 *   variant 1: bulk-copy (TMA) pipeline through shared memory with
 *              `threads` consumer threads per CTA (64, 128 or 256) and
 *              `stages` pipeline stages (2..8, fewer if shared memory is
 *              short) of 16 bitmaps each.
 * ctas_per_sm (1..8) caps the persistent grid at ctas_per_sm x SM count.
 * adder: layout of the adder tree (Sec. 4.3 "Sideways Sum"): 0 = blocks of
 *   16 inputs through 15 full adders, 1 = blocks of 8 inputs through 7
 *   (fewer live registers, one more carry ripple per 8 inputs), 2 = blocks
 *   of 32 inputs (two 16-input trees joined by one more full adder: half
 *   the carry ripples; needs words_per_thread 2); variant 0.
 * words_per_thread: 64-bit words of each input a thread owns, 2 (16-byte
 *   loads) or 1 (8-byte loads, twice the threads per row range); variant 0.
 * BM_EINVAL for values outside these ranges.
 */
typedef struct bm_dense_config_t {
    int32_t variant, threads, stages, ctas_per_sm, adder, words_per_thread;
} bm_dense_config_t;
int bm_pool_set_dense_config(bm_pool* pool, const bm_dense_config_t* cfg);
int bm_pool_get_dense_config(bm_pool* pool, bm_dense_config_t* cfg);

/*
 * Shape of the sparse (ScanCount) kernel: tile_rows rows of 16-bit counters
 * per CTA (a multiple of 8192, at most 65536; a query of at most 255 inputs
 * counts in 8 bits over twice the rows, at most 65536, in the same shared
 * memory), `threads` per CTA (64..512, a
 * multiple of 32), ctas_per_sm (1..8), unroll = 32-vector pieces in each
 * of the two load batches a warp keeps in flight (2 or 4).  BM_EINVAL
 * outside these ranges.
 */
typedef struct bm_sparse_config_t {
    uint32_t tile_rows;
    int32_t threads, ctas_per_sm, unroll;
} bm_sparse_config_t;
int bm_pool_set_sparse_config(bm_pool* pool, const bm_sparse_config_t* cfg);
int bm_pool_get_sparse_config(bm_pool* pool, bm_sparse_config_t* cfg);

/*
 * Shape of the batch kernel: dense persistent CTAs per SM (1 to 3; 3 only
 * resides with words_per_thread 1), adder
 * layout (0, 1 or 2) and words per thread (as for the dense kernel; here the
 * 32-input blocks also take one word per thread).
 */
typedef struct bm_batch_config_t {
    int32_t ctas_per_sm, adder, words_per_thread;
} bm_batch_config_t;
int bm_pool_set_batch_config(bm_pool* pool, const bm_batch_config_t* cfg);
int bm_pool_get_batch_config(bm_pool* pool, bm_batch_config_t* cfg);

/*
 * Looped recurrence for small thresholds (Sec. 4.4, Algorithm "Looped"):
 * with max_t in 1..3, a single dense query whose predicate is a plain
 * threshold "count >= T" (or its negation "count < T", 1 <= T <= N) with
 * t = min(T, N - T + 1) <= max_t runs t running ORs per input instead of the
 * counter planes; the form with N - T + 1 goes through the complement
 * identity, corrected (Sec. 2.3: NOT theta(T, b) = theta(N - T + 1, NOT b)).
 * max_t = 0 (the default) turns it off.  Results are identical either way.
 * Applies to bm_threshold, bm_symmetric and bm_query_run on the dense path;
 * not to batches, weighted queries or bm_threshold_noalloc.
 * BM_EINVAL if max_t > 3 or an argument is NULL.
 */
int bm_pool_set_looped(bm_pool* pool, uint32_t max_t);
int bm_pool_get_looped(bm_pool* pool, uint32_t* max_t);

/*
 * Autotuner: time candidate shapes of the dense, sparse (if lists are
 * loaded) and batch kernels on queries over the pool's own bitmaps (CUDA
 * events, median of repeats) and install the fastest of each.  With a
 * cache_path, a result stored there for the same GPU model and pool shape
 * is reused instead of measuring, and new results are appended.  report
 * (may be NULL) receives a one-line text summary, truncated to report_len.
 * Needs at least one loaded dense bitmap.  Synchronous.
 */
int bm_pool_autotune(bm_pool* pool, const char* cache_path, char* report, uint64_t report_len);

/* ------------------------------------------------------------------------
 * Single queries
 * ---------------------------------------------------------------------- */

/*
 * Threshold query T(theta, {B_ids[0], ..., B_ids[n-1]}) (Sec. 2.3).
 * ids: host array of n pool ids (1 <= n <= BM_N_MAX, repeats allowed).
 * out_words: device, ceil(r/64) words, written in full.
 * out_card: device uint64, receives the output's cardinality (may be NULL).
 * Runs the dense bit-sliced carry-save counter over the pool's dense words.
 * Errors: BM_EINVAL (NULL ids/out_words, n = 0 or > BM_N_MAX), BM_ERANGE (an
 * id >= capacity or without a dense bitmap), BM_ECUDA (launch failure).
 */
int bm_threshold(bm_pool* pool, const uint32_t* ids, uint32_t n, uint32_t theta,
                 uint64_t* out_words, uint64_t* out_card, void* stream);

/*
 * Symmetric-function query (Sec. 2.2; counter-based form in Sec. 4.2):
 * output bit i = f(c_i) with f given by `table`, a host array of
 * ceil((n + 1) / 64) uint64 words whose bit c (word c / 64, bit c mod 64) is
 * f(c) for c = 0..n; bits above n are ignored.  Other arguments and errors
 * as bm_threshold.
 */
int bm_symmetric(bm_pool* pool, const uint32_t* ids, uint32_t n, const uint64_t* table,
                 uint64_t* out_words, uint64_t* out_card, void* stream);

/* Query kinds of bm_query. */
#define BM_KIND_THRESHOLD 0u /* count >= theta */
#define BM_KIND_INTERVAL 1u  /* lo <= count <= hi (T_lo AND NOT T_{hi+1}, Sec. 4.3) */
#define BM_KIND_TABLE 2u     /* f(count) from a truth table */

/* Kernel paths of bm_query.  Results are identical on every path. */
#define BM_PATH_AUTO 0   /* the pool's selector chooses (learned model, else a density rule) */
#define BM_PATH_DENSE 1  /* bit-sliced carry-save counter over the dense words */
#define BM_PATH_SPARSE 2 /* ScanCount over the position lists (every id needs a list) */
#define BM_PATH_RLE 3    /* run-length form with clean-run pruning (every id needs one).
                            BM_PATH_AUTO takes it in place of the dense counter when
                            every id has one and its runs, literal words and tile
                            summaries are estimated faster to read than the dense
                            words */

typedef struct bm_query {
    const uint32_t* ids;    /* host array of n pool ids (repeats allowed) */
    uint32_t n;             /* 1 .. BM_N_MAX */
    uint32_t kind;          /* BM_KIND_* */
    uint32_t theta;         /* BM_KIND_THRESHOLD */
    uint32_t lo, hi;        /* BM_KIND_INTERVAL (hi is clamped to n) */
    const uint64_t* table;  /* BM_KIND_TABLE: host, ceil((n+1)/64) words, bit c = f(c) */
    uint64_t* out_words;    /* device, ceil(r/64) words, written in full */
    int32_t path;           /* BM_PATH_* */
    uint32_t reserved;      /* must be 0 */
} bm_query;

/*
 * Run one query on the path it names.  out_card: device uint64 or NULL.
 * *chosen_path (may be NULL) receives the path that ran.  Errors as
 * bm_threshold, plus BM_EINVAL for a bad kind/path and BM_ERANGE when the
 * sparse (run-length) path is asked for an id without a position list
 * (run-length form).
 */
int bm_query_run(bm_pool* pool, const bm_query* q, uint64_t* out_card, int32_t* chosen_path,
                 void* stream);

/*
 * Batched queries (not in the paper, which runs one query at a time): run
 * the nq queries q[0..nq) as one replay of a CUDA graph holding two
 * persistent kernels.  Dense queries are cut into (slab, query) items, a
 * slab being 32768 rows (16384 with one word per thread), taken slab-major, so each slab of the pool is read from HBM once
 * and served from L2 to every query of the batch that reads it; sparse
 * queries into (query, row tile) ScanCount items; run-length queries run
 * after the graph, one launch of the run-length kernel each, on the same
 * stream.  BM_PATH_AUTO queries are
 * routed by the learned selector when one is installed (its network runs on
 * the device for the whole batch), else by the density rule.
 * out_cards: device, nq uint64, receives each query's cardinality.
 * chosen_paths: host, nq entries (may be NULL), receives each query's path.
 * Every result equals that of the same query run alone.  Host arrays are
 * copied before the call returns; up to three batches may be in flight.
 * Errors as bm_query_run, for the first failing query (nothing is launched).
 */
int bm_threshold_batch(bm_pool* pool, const bm_query* q, uint32_t nq, uint64_t* out_cards,
                       int32_t* chosen_paths, void* stream);

/*
 * Weighted threshold with an optional combining step (Sec. 2.3: a weight is
 * a number of copies of an input; the result of a threshold is again a
 * bitmap, Sec. 1).  Row i of the output is selected iff
 *     sum over k of weights[k] * (bit i of bitmap ids[k])  >=  theta,
 * and is then combined with the pool bitmap post_id: unchanged
 * (BM_POST_NONE), AND, OR or AND NOT (result AND NOT bitmap), in the same
 * pass.  theta = 0 selects every row; theta above the sum of the weights
 * selects none.  Each input is read once whatever its weight (dense path).
 * weights[k] <= BM_WEIGHT_MAX, sum of the weights < 2^32; weight 0 drops an
 * input.  out_card: device uint64 or NULL.  Errors: BM_EINVAL (null pointer,
 * n > BM_N_MAX, a weight or sum out of range, bad post_op, reserved != 0),
 * BM_ERANGE (an id or post_id without a dense bitmap), BM_ECUDA.
 */
#define BM_POST_NONE 0u
#define BM_POST_AND 1u
#define BM_POST_OR 2u
#define BM_POST_ANDNOT 3u
#define BM_WEIGHT_MAX 16777215u /* 2^24 - 1 */

typedef struct bm_weighted_query {
    const uint32_t* ids;      /* host, n pool ids (repeats allowed) */
    const uint32_t* weights;  /* host, n weights */
    uint32_t n;               /* 0 .. BM_N_MAX */
    uint32_t post_op;         /* BM_POST_* */
    uint64_t theta;
    uint32_t post_id;         /* the combined bitmap (post_op != BM_POST_NONE) */
    uint32_t reserved;        /* must be 0 */
    uint64_t* out_words;      /* device, ceil(r/64) words, written in full */
} bm_weighted_query;

int bm_weighted_threshold(bm_pool* pool, const bm_weighted_query* q, uint64_t* out_card,
                          void* stream);

/*
 * Number of ones among the first r_bits rows of a device bitmap `words`
 * (ceil(r/64) words), written to the device uint64 *out_card (Sec. 2.1: the
 * cardinality of the set a bitmap stores).  Asynchronous on `stream`.
 */
int bm_cardinality(const uint64_t* words, uint64_t r_bits, uint64_t* out_card, void* stream);

/*
 * Failure-path self-test: launch a one-warp kernel that waits on a device
 * barrier phase nothing completes, with a bound of limit_us microseconds
 * (1 .. 2,000,000).  The wait expires, the kernel sets the pool's error word
 * and returns; the next bm_pool_status() reports BM_ETIMEOUT.  The GPU
 * context stays usable.  Every bounded wait of the library reports this way.
 */
int bm_pool_selftest_wait(bm_pool* pool, uint32_t limit_us, void* stream);

/* ------------------------------------------------------------------------
 * Serving loop (not in the paper): continuous batching over a resident pool
 * ---------------------------------------------------------------------- */

typedef struct bm_server bm_server;

typedef struct bm_server_config {
    uint64_t mem_budget;      /* device bytes for result bitmaps of admitted requests */
    uint32_t max_batch;       /* most requests per batch launch */
    uint32_t max_inflight;    /* batches in flight at once, on as many streams (1..4) */
    uint32_t max_queue;       /* most requests waiting for admission; more: BM_EBUSY */
    uint32_t batch_window_us; /* pause before forming a batch, to let it grow (0: none) */
    uint32_t slo_us;          /* latency objective (0: none), see bm_server_create */
    uint32_t reserved;        /* must be 0 */
} bm_server_config;

typedef struct bm_server_stats_t {
    uint64_t submitted, completed, refused, batches, batched_queries;
    uint32_t waiting;         /* requests not yet admitted */
    uint32_t free_slots, total_slots;
    uint32_t max_batch_seen;
    int32_t last_error;       /* last launch error (BM_OK if none) */
    uint64_t cancelled;       /* removed by bm_server_cancel before admission */
    uint64_t expired;         /* deadline passed before admission */
} bm_server_stats_t;

/*
 * Start a serving loop over `pool`: a scheduler thread forms batches of
 * waiting requests whenever one of max_inflight streams is free and runs
 * each with bm_threshold_batch.  Admission is by device memory: the server
 * allocates mem_budget bytes once and a request is admitted only when an
 * output slot (one bitmap, ceil(r/64) words rounded to 256 bytes) is free;
 * slots come back when results are released.  BM_ENOMEM if the budget holds
 * no slot or cannot be allocated.
 *
 * Load shedding (slo_us > 0): the scheduler keeps running estimates of a
 * batch's fixed time and of its time per input id (a request's work grows
 * with its number of inputs), from the batches it ran.
 * A submission is refused (BM_EBUSY) when the requests ahead of it, waiting
 * and in flight, would not drain within slo_us by those estimates; every
 * batch is bounded so that its oldest request can still complete within
 * slo_us of its submission; a waiting request that could not complete in
 * time even in a batch of its own is dropped before it runs and completes as
 * expired (BM_ETIMEOUT), as with a deadline.  Admitted requests therefore
 * finish near or within the objective under overload instead of queueing
 * without bound.  slo_us = 0 keeps batches of up to max_batch.
 */
int bm_server_create(bm_pool* pool, const bm_server_config* cfg, bm_server** out);

/* Stop the scheduler, wait for batches in flight, free everything. */
int bm_server_destroy(bm_server* server);

/*
 * Submit a query (its out_words is ignored: the result lives in a server
 * slot) on any path bm_threshold_batch takes.  The query is copied; ids are
 * validated at once for its path (BM_EINVAL, BM_ERANGE).  BM_EBUSY when
 * max_queue requests already wait, or when the latency objective refuses it
 * (see bm_server_create).  *ticket identifies the request.
 */
int bm_server_submit(bm_server* server, const bm_query* q, uint64_t* ticket);

/*
 * As bm_server_submit, with a deadline: if the request is still waiting for
 * admission deadline_us microseconds after submission, it completes without
 * running and bm_server_wait / bm_server_result report BM_ETIMEOUT for it
 * (release it as any other).  deadline_us = 0: no deadline.
 */
int bm_server_submit_deadline(bm_server* server, const bm_query* q, uint64_t deadline_us,
                              uint64_t* ticket);

/*
 * Withdraw a request that is still waiting for admission (its ticket is
 * forgotten).  BM_EBUSY if it was already admitted (it then runs to
 * completion and must be collected or released), BM_ERANGE for an unknown
 * ticket.
 */
int bm_server_cancel(bm_server* server, uint64_t ticket);

/* Wait up to timeout_ms for a request: BM_OK, BM_ETIMEOUT, or its launch error. */
int bm_server_wait(bm_server* server, uint64_t ticket, uint32_t timeout_ms);

/*
 * Result of a completed request: the output bitmap copied to host_words
 * (ceil(r/64) words; may be NULL), its cardinality, the latency from submit
 * to batch completion and the part spent waiting before launch (both in
 * microseconds), and the path it ran on.  BM_ENOTREADY if not complete.
 * Any output pointer may be NULL.
 */
int bm_server_result(bm_server* server, uint64_t ticket, uint64_t* host_words, uint64_t* card,
                     double* latency_us, double* queue_us, int32_t* path);

/* Forget a completed request and return its output slot. */
int bm_server_release(bm_server* server, uint64_t ticket);

/*
 * Load generator for the serving loop: submit qs[i] at arrival_s[i] seconds
 * after the call starts (open loop, e.g. Poisson arrivals), collect every
 * result in order and release it.  Per request (host arrays of n entries,
 * each may be NULL): latency_us and queue_us as in bm_server_result, cards,
 * and status (BM_OK, BM_EBUSY when refused by admission, BM_ETIMEOUT when
 * dropped by its deadline or the latency objective, or an error).
 * *wall_s: time from the first submission to the last collection.
 */
int bm_server_replay(bm_server* server, const bm_query* qs, uint32_t n, const double* arrival_s,
                     double* latency_us, double* queue_us, uint64_t* cards, int32_t* status,
                     double* wall_s);

/* Counters of the serving loop. */
int bm_server_stats(bm_server* server, bm_server_stats_t* out);

/* ------------------------------------------------------------------------
 * Learned kernel selector (not in the paper: the paper compares its
 * algorithms by measured time per query and reports each one's
 * "suboptimality", the extra time over the best, App. C; here a small
 * network predicts that time so the fastest kernel can be picked)
 * ---------------------------------------------------------------------- */

/* Number of selector features and candidates (the network's in/outputs). */
#define BM_SELECTOR_FEATURES 6u
#define BM_SELECTOR_HIDDEN 64u
#define BM_SELECTOR_CANDIDATES 6u
/*
 * Candidate c runs: 0 = dense counter in the pool's shape; 1, 2, 3 = ScanCount
 * with tiles of 16384, 32768, 65536 rows; 4 = dense counter with one 64-bit
 * word per thread (direct loads, twice the threads: for queries whose rows
 * leave the pool's shape short of parallelism); 5 = the run-length path.  In
 * a batch, candidates 0 and 4 both run in the batch's dense kernel, and the
 * run-length candidate, which runs as a launch of its own, is taken over a
 * dense pick only if its predicted time beats the dense one divided by the
 * batch's measured gain (2.5): a query left in the dense kernel shares the
 * pool's reads with the others.
 */

/*
 * Features of a query (6 floats, host): log2 n; the first count where f
 * changes, divided by n (theta / n for a threshold); log10 of the mean and of
 * the largest input density (cardinality / r, floored at 1e-9); log2 r; log2
 * of the bytes of the inputs' run-length forms (summaries and containers)
 * over their dense bytes, or 0 when an input has no run-length form.
 */
int bm_query_features(const bm_pool* pool, const bm_query* q, float* out);

/*
 * Install a trained selector: params (host fp32, the layout of
 * bm_mlp_forward with F = 6, H = 64, C = 6) predicts each candidate's log
 * time from the standardised features (x - mean) / std.  Queries with
 * path BM_PATH_AUTO then run the candidate with the smallest prediction
 * among those whose inputs are loaded (lists for ScanCount, run-length forms
 * for candidate 5).  params = NULL removes it (the fixed density rule
 * applies, with the run-length cost model).  Results never depend on the
 * choice.
 */
int bm_pool_set_selector(bm_pool* pool, const float* params, uint64_t nparams, const float* mean,
                         const float* stdev, uint32_t n_out);

/* The path that BM_PATH_AUTO would pick for q as a single query
   (bm_query_run); *tile_rows (may be NULL) receives, for BM_PATH_SPARSE, the
   tile rows; for BM_PATH_DENSE, 1 when the one-word-per-thread shape
   (candidate 4) is picked, else 0; for BM_PATH_RLE, 0. */
int bm_query_select(const bm_pool* pool, const bm_query* q, int32_t* path, uint32_t* tile_rows);

/*
 * Network F -> H -> H -> C with ReLU after the two hidden layers, fp32,
 * device buffers.  params: W1[F][H], b1[H], W2[H][H], b2[H], W3[H][C], b3[C]
 * (weights [in][out], row-major).  x: [batch][F]; h1, h2: [batch][H]
 * (written, kept for the backward pass); y: [batch][C].
 */
int bm_mlp_forward(const float* params, uint32_t F, uint32_t H, uint32_t C, const float* x,
                   uint32_t batch, float* h1, float* h2, float* y, void* stream);

/*
 * Gradients of L = sum((y - target)^2) / (batch * C) with respect to every
 * parameter, written to `grads` (the layout of params), from the forward
 * pass's x, h1, h2, y.  workspace: device, batch * (C + 2H) floats.
 * loss: device float receiving L, or NULL.
 */
int bm_mlp_backward(const float* params, uint32_t F, uint32_t H, uint32_t C, const float* x,
                    const float* h1, const float* h2, const float* y, const float* target,
                    uint32_t batch, float* grads, float* workspace, float* loss, void* stream);

/*
 * One Adam step (Kingma and Ba 2015, bias-corrected; step is 1-based) over
 * `count` parameters, updating params, m and v in place on the device.
 */
int bm_mlp_adam(float* params, const float* grads, float* m, float* v, uint64_t count,
                uint32_t step, float lr, float beta1, float beta2, float eps, void* stream);

/* ------------------------------------------------------------------------
 * Threshold query that allocates nothing (no counterpart in the paper)
 * ---------------------------------------------------------------------- */

/* Largest n accepted by bm_threshold_noalloc (size of its fixed scratch). */
#define BM_NOALLOC_MAX_N 16384u

/*
 * For callers that cannot call cudaMalloc: for example a plugin inside a host
 * program that owns every device allocation, or a service that must not
 * allocate (and so must not risk an allocation's implicit synchronisation or
 * failure) once it is running.  The paper has no counterpart: it is an
 * interface choice of this library.
 *
 * Same result as bm_threshold, computed by the same dense kernel, but on the
 * caller's own bitmaps and with no pool: bitmap j (0 <= j < n_bitmaps) is
 * words + j * stride_words, ceil(r_bits / 64) words.  `words` must be
 * 16-byte aligned, stride_words even and >= ceil(r_bits / 64) rounded up to
 * even, and every bitmap readable up to that rounded length.  ids is a host
 * array of n ids; out_words (device, ceil(r_bits / 64) words) and out_card
 * (device uint64, may be NULL) are written as by bm_threshold.
 *
 * Scratch: the ids are copied into one fixed device array of
 * BM_NOALLOC_MAX_N uint32 declared in the library; every GPU that loads the
 * library holds it until the process exits.  n > BM_NOALLOC_MAX_N is
 * rejected with BM_EINVAL.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  Every call shares the array and it
 * keeps the previous call's ids, so calls whose work overlaps on the GPU
 * (different streams, no ordering between them) race on it: order them.
 * No cudaMalloc, cudaFree or other allocating routine is called.
 * Errors: BM_EINVAL (NULL pointer, n = 0 or too large, bad alignment or
 * stride, r_bits = 0 or > 2^32), BM_ERANGE (an id >= n_bitmaps), BM_ECUDA.
 */
int bm_threshold_noalloc(const uint64_t* words, uint64_t stride_words, uint32_t n_bitmaps,
                         uint64_t r_bits, const uint32_t* ids, uint32_t n, uint32_t theta,
                         uint64_t* out_words, uint64_t* out_card, void* stream);

/* Static text for a status code. */
const char* bm_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* BM_H */
