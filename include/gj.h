/*
 * gj.h -- C ABI of the GB300 join / grouped-aggregation library (libgj.so).
 *
 * Operators (paper: "Efficiently Processing Joins and Grouped Aggregations on
 * GPUs", PACMMOD 2025):
 *   - inner equi-join T(key, r1.., s1..) of R(key, r1..) and S(key, s1..), R.key a
 *     primary key and S.key a foreign key                       -- Sec. 2.2
 *   - group-by R(k, r1..rn) -> A(k, a1..an) with reducible aggregates, the group
 *     count g unknown in advance                                  -- Sec. 2.2, Alg. 1
 *   - the radix-partition primitive: stable, partitions stored contiguously,
 *     on bits [i, j) of the key                                   -- Sec. 2.3
 *
 * Conventions for every entry point
 *   - Column data, outputs and counters are DEVICE pointers owned by the caller
 *     and must stay valid until the work queued on `stream` has finished. The
 *     descriptor structs themselves (gj_table, gj_options, arrays of ops) are
 *     HOST memory and are read before the call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream). Work is enqueued asynchronously; result counts are written to
 *     device int64 words so that no call needs a host synchronisation.
 *   - Scratch memory comes from the allocator set with gj_set_allocator, or from
 *     cudaMallocAsync/cudaFreeAsync on `stream` when none is set. Scratch is
 *     released (stream-ordered) before the call returns.
 *   - Return value: argument errors are reported synchronously. Errors found by
 *     the kernels (duplicate primary key, output capacity, a bounded wait that
 *     ran out) are written to a device status word; with options.sync = 1 the
 *     call synchronises `stream` and returns that status, otherwise read it with
 *     gj_get_device_status. Kernels never trap.
 *   - Row counts are limited to 2^30 - 1 per input (GJ_ERR_UNSUPPORTED above).
 *   - Output row order is unspecified. PHJ-TR, PHJ-UR, SMJ-TR, SMJ-UR, SGB-TR
 *     and SGB-UR produce the same order on every run (stable partitioning, no
 *     atomics deciding positions); NPHJ, the many-to-many joins, HGB, PGB and
 *     SGB-DE assign positions or codes through hash tables filled concurrently,
 *     so their row order may differ between runs while the result multiset does
 *     not.
 */
#ifndef GJ_H_
#define GJ_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GJ_MAX_COLS 8
#define GJ_MAX_AGGS 32

typedef enum {
  GJ_OK = 0,
  GJ_ERR_INVALID_ARG = 1,   /* bad pointer, type, count or option */
  GJ_ERR_UNSUPPORTED = 2,   /* valid request outside what is implemented */
  GJ_ERR_OOM = 3,           /* scratch allocation failed */
  GJ_ERR_CAPACITY = 4,      /* result larger than the caller's capacity (rows past it are dropped) */
  GJ_ERR_DUPLICATE_KEY = 5, /* R.key is not unique in gj_join (primary-key assumption, Sec. 2.2) */
  GJ_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
  GJ_ERR_CUDA = 7           /* a CUDA runtime call failed */
} gj_status;

typedef enum { GJ_I32 = 0, GJ_I64 = 1 } gj_dtype;

/* A columnar relation: one key column and up to GJ_MAX_COLS payload/value
 * columns, each an array of n elements of its type (Sec. 3: relations are stored
 * as columns, every column an array). */
typedef struct {
  int32_t key_type;               /* gj_dtype */
  int32_t ncols;                  /* 0..GJ_MAX_COLS */
  int64_t n;                      /* rows */
  void* key;                      /* device, n elements */
  int32_t col_type[GJ_MAX_COLS];  /* gj_dtype of each column */
  void* cols[GJ_MAX_COLS];        /* device, n elements each */
} gj_table;

typedef enum { GJ_AGG_SUM = 0, GJ_AGG_COUNT = 1, GJ_AGG_MIN = 2, GJ_AGG_MAX = 3 } gj_agg;

typedef enum {
  GJ_JOIN_AUTO = 0,
  GJ_JOIN_PHJ_TR = 1, /* radix-partitioned hash join, payloads partitioned with the keys (GFTR, Sec. 4.1.4) */
  GJ_JOIN_PHJ_UR = 2, /* same partitioning of (key, tuple id), payloads gathered by id (GFUR, Sec. 3.1.2, 4.1.4) */
  GJ_JOIN_NPHJ = 3,   /* non-partitioned hash join: global table on R, S probed in order (Sec. 3.1.3) */
  GJ_JOIN_NPHJ_MN = 4, /* many-to-many (R.key need not be unique, Sec. 5.1.9): global table on R with a chain
                         of equal keys; every (r, s) pair is written, |T| = sum over S of its matches.
                         gj_join only; never chosen by AUTO */
  GJ_JOIN_SMJ_TR = 5, /* sort-merge join: both sides radix-sorted on the whole key with their payloads,
                         tiles of S merged against their range of R (merge path), Sec. 3.1.1 */
  GJ_JOIN_SMJ_UR = 6, /* the same with (key, tuple id) sorted and payloads gathered by id (GFUR) */
  GJ_JOIN_PHJ_MN = 7  /* many-to-many with GFTR: R and S radix-partitioned with their payloads, a global
                         table whose slots cluster each partition's keys, key chains inside partitions
                         (Sec. 5.1.9); gj_join only; never chosen by AUTO */
} gj_join_variant;

typedef enum {
  GJ_GB_AUTO = 0,
  GJ_GB_HGB = 1, /* hash-based, dense group ids then shared-memory aggregation (Sec. 4.2, Alg. 1); its
                    dictionary table holds 2 x groups_hint entries when a hint is set (a larger group
                    count gives GJ_ERR_CAPACITY), else 2 x n. With 1 <= groups_hint <= 32 and only COUNT
                    and aggregates over 4-byte columns (at most three distinct), a single pass without
                    dictionary runs first (up to 16: tiles sorted by group in shared memory; 17 to 32:
                    lane-held aggregates); when the data holds more keys than that pass takes, it gives
                    way to the dictionary path, with the same result */
  GJ_GB_SGB = 2, /* sort-based with the values sorted alongside the key (SGB-TR, Sec. 4.1.3), on the key
                    bits that vary only; synchronises the stream once to read the key range */
  GJ_GB_PGB = 3, /* partition-based with per-partition shared-memory tables (PGB-TR, Sec. 4.3); a partition
                    with far more rows than the others (few groups, skew) is cut into slices aggregated by
                    several blocks into partial rows, then merged (Sec. 4.3's remedy for overly large
                    partitions); scratch for partial rows of up to the sliced partitions' rows, sized by
                    one stream synchronisation when n x (key bytes + 8 x aggregates) exceeds 256 MB */
  GJ_GB_SGB_UR = 4, /* SGB with (key, tuple id) sorted and values gathered through the ids (GFUR, Sec. 4.1.2) */
  GJ_GB_PGB_UR = 5, /* PGB with (key, tuple id) partitioned and values gathered through the ids (GFUR) */
  GJ_GB_SGB_DE = 6  /* SGB on dictionary codes: dense group ids (HGB stage 1) sorted on ceil(log2 g) bits
                       with the values, keys decoded from the dictionary (Sec. 4.4); synchronises the
                       stream once to read g */
} gj_groupby_variant;

/* How AUTO picks a variant: the paper's rules (Sec. 7, Fig. groupby-dt), the
 * trained network (Sec. 6's learned selection; the cost model while no network
 * is installed), or the GB300-calibrated cost model (gj_cost_estimate). */
typedef enum { GJ_SELECT_HEURISTIC = 0, GJ_SELECT_MLP = 1, GJ_SELECT_COST = 2 } gj_selector_mode;

typedef struct {
  int32_t join_variant;     /* gj_join_variant */
  int32_t groupby_variant;  /* gj_groupby_variant */
  int32_t selector;         /* gj_selector_mode used when a variant is AUTO */
  int32_t radix_bits;       /* total partition bits for PHJ / PGB; 0 = choose from sizes */
  int32_t bits_per_pass;    /* 1..8; 0 = balanced passes of at most 8 bits */
  int32_t tile;             /* reserved for the tuner; 0 = default */
  int32_t sync;             /* 1 = synchronise `stream` and return device-detected errors */
  int32_t reserved;
  float zipf_hint;          /* selector features (negative = unknown) */
  float match_ratio_hint;
  int64_t groups_hint;      /* expected group count, 0 = unknown; sizes HGB's and SGB-DE's dictionary and
                               PGB's partition count, and is a selector feature */
} gj_options;

/* Fills *opt with the defaults (AUTO variants, the cost-model selector, sync = 0). */
void gj_options_default(gj_options* opt);

/* Human-readable name of a status code; never NULL. */
const char* gj_status_string(gj_status s);

/* Scratch allocator hooks. alloc(bytes, stream, ctx) returns device memory or
 * NULL (-> GJ_ERR_OOM); free(ptr, stream, ctx) releases it stream-ordered.
 * Passing NULL for both restores cudaMallocAsync/cudaFreeAsync. Not thread-safe
 * against concurrent calls of the other entry points. */
gj_status gj_set_allocator(void* (*alloc)(size_t bytes, void* stream, void* ctx),
                           void (*free_fn)(void* ptr, void* stream, void* ctx), void* ctx);

/* Synchronises `stream`, returns the first error recorded by a kernel of this
 * library on the current device since the last call, and clears it. */
gj_status gj_get_device_status(void* stream);

/* radix-partition (Sec. 2.3). Partitions the rows of `in` (key and every column)
 * stably on bits [bit_lo, bit_hi) of d(key), where d is the key's own binary
 * representation (key_transform 0), the key with its sign bit flipped so that
 * digit order is signed order (1), or the MurmurHash3 fmix32/fmix64 finaliser of
 * the key (2). bit_hi - bit_lo is 1..32 for 4-byte and 1..64 for 8-byte keys;
 * digits of at most 8 bits are handled per pass, least significant first, so a
 * full-width range is an LSD radix sort. `out` has the same types and ncols as
 * `in`, with out->n >= in->n; its buffers must not overlap the input's.
 * d_offsets (device, optional) receives 2^(bit_hi-bit_lo)+1 int64 partition
 * bounds (partition p occupies rows [d_offsets[p], d_offsets[p+1])); it must be
 * NULL when bit_hi - bit_lo > 24. */
gj_status gj_radix_partition(const gj_table* in, int32_t bit_lo, int32_t bit_hi, int32_t key_transform,
                             gj_table* out, int64_t* d_offsets, const gj_options* opt, void* stream);

/* radix-partition without any device allocation. For callers that must not
 * allocate device memory: code that runs while another component owns the
 * device's memory budget (a framework that reserved it all in its own pool),
 * code called from inside an allocator or a memory-pressure handler, and
 * latency-bound paths that cannot afford the implicit device synchronisation
 * and pool growth that cudaMalloc/cudaFree can cause. Every other entry point
 * takes scratch from cudaMallocAsync or the gj_set_allocator hook; this one
 * takes it from a fixed array inside the library. The paper has no counterpart:
 * the result is exactly gj_radix_partition's for one pass.
 * Limits: bit_hi - bit_lo <= 8 (a single pass) and in->n <= 2^21 rows, else
 * GJ_ERR_UNSUPPORTED; arguments as for gj_radix_partition otherwise.
 * Memory: the array is about 0.5 MB (per-tile digit offsets for 2^21 rows in
 * tiles of 4096) and is resident on every device that loads the library until
 * the process exits. The call makes no cudaMalloc, cudaFree
 * or allocator-hook call. Its first call on a device looks up the array's
 * device address with that device current; make that first call before any
 * stream capture. All calls share the one array, which keeps what the last call
 * left in it (each call clears the part it uses): calls whose work can overlap
 * on the GPU -- unordered streams or concurrent host threads -- race on it, so
 * the caller must order them. sync = 1 synchronises `stream` and returns the
 * errors its kernels recorded (an empty input included); with sync = 0 they are
 * kept for the next sync = 1 call of this entry point. */
gj_status gj_radix_partition_noalloc(const gj_table* in, int32_t bit_lo, int32_t bit_hi, int32_t key_transform,
                                     gj_table* out, int64_t* d_offsets, int32_t sync, void* stream);

/* gather (Sec. 2.3): out[i] = in[map[i]] for i < n; in holds n_in elements of
 * elem_bytes (4 or 8) bytes, map n int32 indices, out n elements (all device
 * memory, not overlapping). A clustered map (indices in order, or nearly) reads
 * in sequentially; an unclustered one (a random permutation) reads it at
 * random. An index outside [0, n_in) is recorded as GJ_ERR_INVALID_ARG on the
 * device (returned with opt->sync = 1) and its out[i] is left unwritten. */
gj_status gj_gather(const void* in, int64_t n_in, int32_t elem_bytes, const int32_t* map, int64_t n, void* out,
                    const gj_options* opt, void* stream);

/* Inner equi-join (Sec. 2.2): T(key, R.cols.., S.cols..) = { (r.key, r.., s..) :
 * r in R, s in S, r.key = s.key }. For the primary-key variants (PHJ_TR, PHJ_UR,
 * NPHJ, SMJ_TR, SMJ_UR and AUTO) R.key must be unique; a repeated key yields
 * GJ_ERR_DUPLICATE_KEY. NPHJ_MN and PHJ_MN join any R and S (many-to-many,
 * Sec. 5.1) and write every matching pair. R and S keys have the same type.
 * T has key_type = R.key_type, ncols = R.ncols + S.ncols (at most GJ_MAX_COLS,
 * else GJ_ERR_INVALID_ARG) with the R columns first, column types as in the inputs. Rows beyond T_capacity are dropped with
 * GJ_ERR_CAPACITY; T_capacity >= S.n always suffices for a primary-key join.
 * *d_T_count (device int64) receives |T| (also when rows were dropped). */
gj_status gj_join(const gj_table* R, const gj_table* S, const gj_options* opt, gj_table* T,
                  int64_t T_capacity, int64_t* d_T_count, void* stream);

/* GROUP BY in.key with aggregate j = ops[j] over value column op_col[j]
 * (COUNT ignores its column) -- Sec. 2.2, Alg. 1. Aggregates are int64; SUM
 * wraps in two's complement. out_keys (device, in.key_type) and out_aggs[j]
 * (device int64 each; the array of nagg pointers is host memory) receive one
 * row per group; capacity >= number of groups (in.n always suffices), overflow
 * -> GJ_ERR_CAPACITY. *d_ngroups (device int64) receives g. 1 <= nagg <= GJ_MAX_AGGS. */
gj_status gj_groupby(const gj_table* in, int32_t nagg, const int32_t* ops, const int32_t* op_col,
                     const gj_options* opt, void* out_keys, int64_t* const* out_aggs, int64_t capacity,
                     int64_t* d_ngroups, void* stream);

/* A column of the join result: side 0 = R, 1 = S; col = payload index on that
 * side, or -1 for the join key. modulus > 0 applies C '%' (truncating) to the
 * value, which is read as int64. */
typedef struct {
  int32_t side;
  int32_t col;
  int64_t modulus;
} gj_colref;

/* GROUP BY group_key over R join S with aggregate j = ops[j] over agg_cols[j]
 * of the matching rows, without materialising the join result (the group-by
 * that follows a join, Sec. 1). Group keys and aggregates are int64; out_keys
 * (device int64) and out_aggs[j] (device int64) receive one row per group,
 * capacity >= number of groups; *d_ngroups (device int64) receives g. R.key
 * must be unique as in gj_join. */
gj_status gj_join_groupby(const gj_table* R, const gj_table* S, gj_colref group_key, int32_t nagg,
                          const int32_t* ops, const gj_colref* agg_cols, const gj_options* opt,
                          int64_t* out_keys, int64_t* const* out_aggs, int64_t capacity, int64_t* d_ngroups,
                          void* stream);

/* ---- Batched execution ----------------------------------------------------
 * Many join -> group-by queries (each as in gj_join_groupby) run in ONE
 * persistent kernel launch that drains a device-side task queue: per query,
 * tasks that clear its tables, build a hash table on R, probe S and aggregate
 * each match into dense group slots, and write the groups out. Tasks are
 * ordered so that every task's dependencies sit earlier in the queue; a task
 * waits for them with a bounded spin (GJ_ERR_TIMEOUT if it gives up). The
 * launch is captured once in a CUDA graph and replayed. The paper has no
 * batched mode; each query computes exactly what gj_join_groupby computes.
 *
 * Restrictions of the persistent kernel: int32 keys; group_key.modulus in
 * [1, 2^20] (groups are the residues, read as dense slots); at most
 * GJ_BATCH_MAX_AGGS aggregates per query (a limit of every query). Column and output pointers are
 * device memory that must stay valid and at the same address for the life of
 * the plan; every launch recomputes all outputs from the current input
 * contents. */
#define GJ_BATCH_MAX_AGGS 8

typedef struct {
  gj_table R;
  gj_table S;
  gj_colref group_key;
  int32_t nagg;
  int32_t ops[GJ_BATCH_MAX_AGGS];
  gj_colref agg_cols[GJ_BATCH_MAX_AGGS];
  int64_t* out_keys;                       /* device int64, capacity rows */
  int64_t* out_aggs[GJ_BATCH_MAX_AGGS];    /* device int64 each */
  int64_t capacity;
  int64_t* d_ngroups;                      /* device int64 */
} gj_query;

typedef struct gj_batch_plan gj_batch_plan;

/* Tuning knobs of a batch plan; zero fields mean "let the autotuner choose".
 * build_rows / probe_rows: rows per build / probe task; lookahead: how many
 * queries ahead their clear+build tasks are queued before a query's probe
 * tasks; blocks_per_sm: resident CTAs of the persistent kernel per SM. */
typedef struct {
  int32_t build_rows;
  int32_t probe_rows;
  int32_t lookahead;
  int32_t blocks_per_sm;
} gj_batch_config;

/* Validates the queries and chooses each one's join variant: opt->join_variant
 * for all of them, or with AUTO the choice opt->selector makes for that query
 * as gj_join_groupby would (PHJ-TR, PHJ-UR or NPHJ; opt's hints apply to every
 * query; opt NULL = defaults). Queries that run NPHJ within the restrictions
 * above go to the persistent kernel; the others (another variant, int64 keys,
 * a modulus outside [1, 2^20]) run one at a time after it through the
 * gj_join_groupby path. Then uploads the task queue, allocates the workspace,
 * runs the autotuner for the zero fields of *cfg (cfg may be NULL: all
 * tuned; the tuner times each candidate on this batch and keeps the fastest;
 * results are cached per device and batch shape), and captures the chosen
 * configuration in a CUDA graph. `stream` is used for tuning and set-up. */
gj_status gj_batch_create(const gj_query* queries, int32_t nq, const gj_batch_config* cfg, const gj_options* opt,
                          gj_batch_plan** plan, void* stream);
/* Replays the captured graph on `stream`, then runs the queries that run alone:
 * all nq queries, asynchronously (the one-at-a-time queries allocate and free
 * their scratch through the allocator as gj_join_groupby does). */
gj_status gj_batch_launch(gj_batch_plan* plan, void* stream);
/* variants[nq]: the gj_join_variant each query of the plan runs. */
gj_status gj_batch_get_variants(const gj_batch_plan* plan, int32_t* variants);
/* The configuration the plan runs with. */
gj_status gj_batch_get_config(const gj_batch_plan* plan, gj_batch_config* cfg);
/* Frees the plan, its graph and workspace (synchronises the device). */
gj_status gj_batch_destroy(gj_batch_plan* plan);

/* ---- Learned variant selector ---------------------------------------------
 * A multi-layer perceptron x(12) -> 64 -> ReLU -> 64 -> ReLU -> y(11), FP32,
 * predicting log run time of the join variants PHJ-TR, PHJ-UR, NPHJ, SMJ-TR,
 * SMJ-UR (y0..y4) and the group-by variants HGB, SGB, PGB, SGB-UR, PGB-UR,
 * SGB-DE (y5..y10). The paper chooses variants with cost models and heuristics
 * (Sec. 4.1.3, 4.1.4, 4.4, 5.1.10, Fig. groupby-dt); the network has no
 * counterpart there and those rules remain the fallback. Parameters are one
 * float array of GJ_MLP_PARAMS values, row-major [out][in] weights each followed
 * by its bias: w1[64][12] b1[64] w2[64][64] b2[64] w3[11][64] b3[11]. All
 * pointers below are device memory; all calls are asynchronous on `stream`. */
#define GJ_MLP_IN 12
#define GJ_MLP_HIDDEN 64
#define GJ_MLP_OUT 11
#define GJ_MLP_JOIN_OUT 5
#define GJ_MLP_PARAMS 5707

/* y[batch][11] = f(theta, x[batch][12]). */
gj_status gj_mlp_forward(const float* theta, const float* x, int32_t batch, float* y, void* stream);
/* loss = (1/batch) sum_b sum_o mask[b][o] (y[b][o] - t[b][o])^2 and its gradient
 * grad[GJ_MLP_PARAMS] (overwritten). Reductions run in a fixed order, so the
 * result is identical on every run. batch >= 1. */
gj_status gj_mlp_loss_grad(const float* theta, const float* x, const float* t, const float* mask, int32_t batch,
                           float* grad, float* loss, void* stream);
/* Adam (Kingma & Ba) with bias correction; step counts from 1; m, v are state
 * arrays of GJ_MLP_PARAMS floats, zero before the first step. */
gj_status gj_mlp_adam_step(float* theta, const float* grad, float* m, float* v, int32_t step, float lr, float beta1,
                           float beta2, float eps, void* stream);
/* theta -= lr * grad. */
gj_status gj_mlp_sgd_step(float* theta, const float* grad, float lr, void* stream);
/* For each of n feature rows (already normalised), the argmin of y0..y4 as a
 * gj_join_variant (PHJ_TR, PHJ_UR, NPHJ, SMJ_TR, SMJ_UR) and of y5..y10 as a
 * gj_groupby_variant (1 + index - 5). */
gj_status gj_mlp_select(const float* theta, const float* x, int32_t n, int32_t* join_variant, int32_t* gb_variant,
                        void* stream);

/* Selector used by gj_join / gj_groupby / gj_join_groupby when a variant is
 * AUTO and options.selector = GJ_SELECT_MLP (gj_join_groupby, which runs
 * PHJ-TR, PHJ-UR and NPHJ only, takes the argmin of y0..y2). host_theta: GJ_MLP_PARAMS floats (host);
 * mean / stdev: GJ_MLP_IN floats (host) normalising the raw features
 * (x - mean) / stdev. Passing NULL theta removes the network, and AUTO falls
 * back to the cost model (gj_cost_estimate). The raw features of a query are
 *   0 log2(|R|+1)  1 log2(|S|+1)  2 key bytes  3 R payload columns
 *   4 S payload columns  5 Zipf factor  6 match ratio  7 log2(groups+1)
 *   8 aggregates  9 log2((|R|+1)/(|S|+1))  10 payload bytes per S row
 *   11 log2(groups+1) / log2(|S|+2)
 * with options' hints standing in for unknown skew, match ratio and groups.
 * Features a call knows nothing about take the training mean (0 after
 * normalisation): 7, 8 and 11 for gj_join, 0, 3, 6 and 9 for gj_groupby. */
gj_status gj_selector_set(const float* host_theta, const float* mean, const float* stdev);
/* The variants AUTO would run under the paper's rules (GJ_SELECT_HEURISTIC):
 * for the join, Sec. 7 (GFTR partitioned join if the match ratio is >= 25 %,
 * the foreign keys are skewed or keys are 8 bytes, else the GFUR partitioned
 * join); for the group-by, Fig. groupby-dt without a mandated sort (HGB when
 * the expected groups' aggregates fit in shared memory, else the sort-based
 * variant under high skew, else PGB-TR). Only sizes, types and options are read:
 * the column pointers of R and S may be NULL. `S` is the group-by input. */
gj_status gj_heuristic_choose(const gj_table* R, const gj_table* S, int32_t nagg, const gj_options* opt,
                              int32_t* join_variant, int32_t* gb_variant);
/* The variants an AUTO request would run (host only, no device work): for the
 * join of R and S as gj_join runs it (fused = 0) or as gj_join_groupby runs it
 * with nagg aggregates (fused = 1; it implements PHJ-TR, PHJ-UR and NPHJ); for
 * the group-by of S with nagg aggregates ops[] (ops may be NULL: 8-byte slots) as
 * gj_groupby runs it. Explicit variants in *opt are returned unchanged; AUTO
 * follows opt->selector as the operators do. Either output pointer may be NULL. */
gj_status gj_auto_variants(const gj_table* R, const gj_table* S, int32_t nagg, const int32_t* ops,
                           const gj_options* opt, int32_t fused, int32_t* join_variant, int32_t* gb_variant);
/* ---- Cost-model selection (Sec. 4.1.1, 4.1.3, 4.1.4, 4.4) ------------------
 * The paper's bandwidth models carried over to every variant of this library:
 * a variant's cost is the bytes it moves in units of sequential global-memory
 * bytes (cost / B_G is a time). Unclustered accesses count B_G / B_R times their
 * bytes (M1; B_R measured with the clustered-vs-unclustered gather of Table
 * gather-profile, gj_gather), or B_G / B_L2 times when the structure they go to
 * fits in l2_bytes; every kernel launch and host synchronisation adds a fixed
 * cost; the partition-based group-by pays for the contention on its hottest
 * partition (share 1 / H(g, z) of the rows under Zipf factor z), counted as if
 * one SM took those rows. Fields <= 0 that
 * name device figures (l2_bytes, smem_bytes, num_sms) are read from the current
 * device, or take GB300's when there is none. */
typedef struct {
  double bg_over_br;    /* B_G / B_R: unclustered-access slowdown beyond L2 (>= 1) */
  double bg_over_bl2;   /* B_G / B_L2: unclustered-access slowdown inside l2_bytes (>= 1) */
  double l2_bytes;      /* footprint that counts as L2-resident; 0 = half the device's L2 */
  double smem_bytes;    /* shared memory per block for HGB's aggregates; 0 = the device's opt-in maximum */
  double launch_bytes;  /* fixed cost of one kernel launch, in bytes at B_G */
  double sync_bytes;    /* fixed cost of one host synchronisation inside a call */
  double hot_row_bytes; /* bytes of work per row of the hottest PGB partition (as if on one SM) */
  int32_t num_sms;      /* 0 = the device's */
  int32_t reserved;
} gj_cost_params;

/* GB300 defaults: B_G / B_R = 27.5 (measured: unclustered gathers 9.82x slower
 * than clustered ones over 2^27 int32, and the paper's reading of that gap,
 * B_G / B_R = 3 x gap - 2), B_G / B_L2 = 27.5 / 4.5 (the paper's B_L2 = 4.5 B_G),
 * launch 2e7 and synchronisation 6e7 bytes (about 3 and 9 us at 6.8 TB/s),
 * 10 bytes per hot-partition row. */
void gj_cost_params_default(gj_cost_params* p);
/* Installs the parameters used by GJ_SELECT_COST (and by GJ_SELECT_MLP without
 * a network) in this process; NULL restores the defaults. Ratios below 1 or
 * negative sizes give GJ_ERR_INVALID_ARG. */
gj_status gj_set_cost_params(const gj_cost_params* p);
/* The model's costs (bytes at B_G) under the installed parameters, host only:
 * join_cost[5] for PHJ-TR, PHJ-UR, NPHJ, SMJ-TR, SMJ-UR of R join S (R needed),
 * gb_cost[6] for HGB, SGB, PGB, SGB-UR, PGB-UR, SGB-DE of a group-by of S with
 * nagg aggregates ops[] (ops NULL: SUMs) over all of S's columns. Hints in *opt
 * stand in for the match ratio (unknown: 1), Zipf factor (unknown: 0) and group
 * count (unknown: |S|). Either output may be NULL; column pointers are not read.
 * GJ_SELECT_COST picks the argmin (of the first three for gj_join_groupby). */
gj_status gj_cost_estimate(const gj_table* R, const gj_table* S, int32_t nagg, const int32_t* ops,
                           const gj_options* opt, double* join_cost, double* gb_cost);

/* Writes the 12 raw features of a query into out[12] (host). Either table may be
 * NULL when only one operator is chosen. */
gj_status gj_query_features(const gj_table* R, const gj_table* S, int32_t nagg, const gj_options* opt, float* out);

/* ---- Bounded waits (no counterpart in the paper) ---------------------------
 * Kernels that wait on other blocks (look-backs over tiles, bulk-copy
 * mbarriers, the batched mode's task dependencies) give up once a wait has
 * lasted longer than the current device's wait limit, record GJ_ERR_TIMEOUT and
 * finish, so no launch of this library can hang its GPU.
 *
 * gj_set_wait_limit sets the limit of the waits on other blocks, in
 * nanoseconds of the GPU's global timer, for launches made on the current device
 * after it returns; 0 restores the default of 2 s. A short limit makes
 * legitimate waits fail too (the results are then wrong, but every write stays
 * inside the caller's buffers): it is meant for testing the failure path. A
 * block's wait for its own bulk copies keeps the 2 s limit whatever is set.
 *
 * gj_check_bounded_wait runs one of those waits on a flag that nothing ever
 * sets -- kind 0: the warp-wide look-back over a predecessor tile that never
 * publishes; 1: an mbarrier that nothing arrives at; 2: a task counter that
 * never reaches its target -- synchronises `stream` and returns (and clears) the
 * device status, GJ_ERR_TIMEOUT when the wait gave up as it should. */
gj_status gj_set_wait_limit(uint64_t ns);
gj_status gj_check_bounded_wait(int32_t kind, void* stream);

/* ---- Measurement support (no counterpart in the paper) -------------------
 * gj_profile_enable(1) makes every kernel launch of the library record a CUDA
 * event before and after itself on its stream; gj_profile_read synchronises the
 * device, adds the elapsed times per kernel kind into ms[kind] and the launch
 * counts into launches[kind] for kind < max_kinds (host arrays), clears the
 * records and returns the number of kinds. gj_kernel_name(kind) names a kind.
 * gj_kernel_launches() is the number of kernels launched by the library since
 * load, counted whether or not timing is enabled. */
void gj_profile_enable(int32_t on);
int32_t gj_profile_read(double* ms, int64_t* launches, int32_t max_kinds);
const char* gj_kernel_name(int32_t kind);
int64_t gj_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* GJ_H_ */
