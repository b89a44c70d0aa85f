/*
 * scl.h -- C ABI of the GB300 SparkCL per-partition offload library (libscl).
 *
 * SparkCL (Segal et al., 2015) runs a user kernel over the primitive arrays of
 * one RDD partition on an accelerator: mapParameters() turns the partition
 * into device buffers and sets the range (Sec. 3.1.1.1), run() executes once
 * per element (Sec. 3.1.1.2), mapReturnValue() hands back a value or an array
 * (Sec. 3.1.1.3); MapCL / MapCLPartition / ReduceCL apply that to an RDD and
 * fold the partition results with a tree reduce (Sec. 3.1.3).  This library
 * is that path on one GB300: load a partition (scl_load_partition*), run a
 * map (scl_map), run a map fused with a reduce (scl_map_reduce,
 * scl_keyed_reduce), return the value or array, and fold results across
 * partitions (scl_combine*).  The user kernels are a fixed catalogue of
 * hand-written sm_103a kernels (mix32, poly3, identity; sum / sum-min-max /
 * keyed count+sum).  Around it: many partitions in one persistent launch
 * (scl_batch_*), a continuous-batching server (scl_server_*), a
 * device-polling server (scl_devserver_*), a launch-shape autotuner
 * (scl_autotune) and an allocation-free single call
 * (scl_map_reduce_noalloc).
 *
 * Conventions
 *   - Every call returns an int status: SCL_OK (0) or an SCL_E_* code.  No
 *     call aborts, exits or throws across the ABI.  scl_last_error() gives a
 *     message for the calling thread's most recent failure.
 *   - Device memory: the caller hands scl_create an arena (any device buffer,
 *     e.g. a torch uint8 tensor) that it owns and keeps alive until
 *     scl_destroy.  The library sub-allocates partitions, outputs and its
 *     scratch from that arena; it calls no cudaMalloc.  It does allocate
 *     pinned host memory (cudaHostAlloc) for result staging: a few bytes at
 *     scl_create, and the servers' rings and staging when they start.
 *   - Streams: a `void* stream` is a cudaStream_t owned by the caller (0 =
 *     legacy default stream).  Calls named *_async only enqueue work; the
 *     others synchronise that stream before returning.
 *   - Host input pointers are read only during the call (the copy is
 *     finished before an _async call returns unless the memory is pinned, in
 *     which case it must stay untouched until the stream reaches the copy).
 *   - Thread safety: calls on one context are serialised by a context lock
 *     (the servers' submit and wait calls may come from any thread).  Work
 *     enqueued by single-partition *_async calls uses a scratch area per
 *     stream, so calls on different streams may overlap on the device; a
 *     batch has its own scratch (one launch of a batch at a time);
 *     scl_map_reduce_noalloc shares one fixed scratch (see there).
 */
#ifndef SCL_H
#define SCL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SCL_ABI_VERSION 1

/* ------------------------------------------------------------ status codes */
#define SCL_OK            0
#define SCL_E_INVALID     1  /* bad handle, argument, dtype/kernel mismatch  */
#define SCL_E_NOMEM       2  /* the arena has no free block large enough     */
#define SCL_E_BUDGET      3  /* admission would exceed the HBM budget        */
#define SCL_E_KEY_RANGE   4  /* a key outside [0, num_keys) was seen (pair skipped) */
#define SCL_E_TIMEOUT     5  /* a bounded wait gave up                        */
#define SCL_E_PENDING     6  /* server task not finished yet                  */
#define SCL_E_CUDA        7  /* a CUDA runtime call failed (message has text) */
#define SCL_E_STATE       8  /* call not valid in the current state           */
#define SCL_E_UNSUPPORTED 9  /* combination not in the kernel catalogue      */

/* --------------------------------------------------------------- the types */
typedef struct scl_ctx scl_ctx;      /* one library context on one device     */
typedef struct scl_batch scl_batch;  /* a planned batch of partition tasks    */
typedef uint64_t scl_part;           /* opaque partition handle (0 = none)    */

/* Element type of a partition's primitive arrays (Sec. 3.1.1.1: partitions
 * are turned into arrays of primitive types before the kernel runs). */
typedef enum {
    SCL_U32 = 0,          /* uint32_t[n]                                  */
    SCL_I32 = 1,          /* int32_t[n] (same 32-bit patterns as SCL_U32) */
    SCL_F32 = 2,          /* float[n]                                     */
    SCL_KV_I32_F32 = 3    /* int32_t keys[n] + float vals[n], two arrays  */
} scl_dtype;

/* The catalogue of map kernels (the run() body, Sec. 3.1.1.2). */
typedef enum {
    SCL_K_IDENT = 0,      /* y = x                                          */
    SCL_K_MIX32 = 1,      /* 32-bit x: x^=x>>16; x*=0x7feb352d; x^=x>>15;
                             x*=0x846ca68b; x^=x>>16 (mod 2^32)             */
    SCL_K_POLY3 = 2       /* fp32 x: t = fma(c0, x*x, c1); y = fma(t, x, c2),
                             x*x rounded once; default c = {0.5, -1.25, 0.1} */
} scl_map_kernel;

/* The catalogue of reductions (ReduceCL, Sec. 3.1.3 item 3; the reduce-by-key
 * of the WordCount demo, Sec. 3.2.3). */
typedef enum {
    SCL_R_NONE = 0,             /* map only (scl_map)                        */
    SCL_R_SUM = 1,              /* U32/I32: uint64 sum (mod 2^64) of y as
                                   unsigned; F32: sum                         */
    SCL_R_SUM_MIN_MAX = 2,      /* F32: sum, min, max of y                   */
    SCL_R_KEYED_COUNT_SUM = 3   /* KV: per key count (uint32) and sum        */
} scl_reduce;

/* Context configuration. */
typedef struct {
    int32_t device;              /* CUDA device ordinal                        */
    int32_t reserved0;
    void* arena;                 /* device buffer the library sub-allocates;
                                    caller-owned, 256-byte aligned             */
    uint64_t arena_bytes;        /* its size                                   */
    uint64_t hbm_budget_bytes;   /* server admission budget; 0 = arena_bytes   */
    int32_t inflight_batches;    /* server: batches in flight at once (1..16)  */
    int32_t reserved1;
    const char* tune_cache_path; /* autotune cache file; NULL = none           */
} scl_config;

/* Result of one partition's map+reduce (the value mapReturnValue returns,
 * Sec. 3.1.1.3).  48 bytes, same layout on host and device.
 *   SUM on U32/I32:       u64_sum
 *   SUM / SUM_MIN_MAX on F32: f64_sum (fp64 fold of the partial sums),
 *                         f32_sum (f64_sum rounded), f32_min, f32_max
 *                         (NaN ignored; empty: +inf / -inf)
 *   KEYED_COUNT_SUM:      u64_sum = pairs counted, f64_sum = their value sum
 *   n:                    elements (pairs) in the partition
 *   status:               SCL_OK or SCL_E_KEY_RANGE (the large-key reduce
 *                         also: SCL_E_STATE, its keys changed;
 *                         SCL_E_TIMEOUT, a bounded device wait ran out)     */
typedef struct {
    uint64_t u64_sum;
    double f64_sum;
    float f32_sum;
    float f32_min;
    float f32_max;
    int32_t status;
    uint64_t n;
    uint32_t kind;       /* internal kernel id that produced it */
    uint32_t reserved;
} scl_result;

/* One partition task of a batch or of the server. 64 bytes.
 * Keyed tasks write their tables to device arrays the caller owns:
 * counts_out[num_keys] (uint32), sums_out[num_keys] (float) and, if not NULL,
 * sums64_out[num_keys] (double, the fp64 fold before rounding).            */
typedef struct {
    scl_part part;
    int32_t kernel;      /* scl_map_kernel                                  */
    int32_t reduce;      /* scl_reduce                                      */
    uint32_t num_keys;   /* keyed: 1..4096                                  */
    float coef[3];       /* poly3 coefficients                              */
    uint32_t* counts_out;
    float* sums_out;
    double* sums64_out;
    uint64_t reserved;
} scl_task;

/* ------------------------------------------------------------- errors, info */

/* Static text for a status code. Never NULL. */
const char* scl_strerror(int status);

/* Message of the calling thread's last failed call ("" if none).  The pointer
 * stays valid until that thread's next call into the library. */
const char* scl_last_error(void);

/* ABI version (SCL_ABI_VERSION of the built library). */
int scl_abi_version(void);

/* Total kernel launches this library has made in the process (a graph
 * replay counts each kernel node), for launch accounting. */
int scl_kernel_launches_total(uint64_t* out);

/* ---------------------------------------------------------------- contexts */

/* Create a context on cfg->device over the caller's arena.  Queries the
 * device (SM count, L2 size), carves the scratch region from the arena and
 * loads autotuned launch shapes from cfg->tune_cache_path if it exists.
 * Errors: SCL_E_INVALID (NULL args, misaligned or too small arena),
 * SCL_E_CUDA. */
int scl_create(const scl_config* cfg, scl_ctx** out);

/* Destroy a context: stops the servers if running, frees host staging.
 * The arena is not touched (the caller frees it). NULL is a no-op. */
int scl_destroy(scl_ctx* ctx);

/* Bytes of the arena still free / the largest free block. */
int scl_arena_stats(scl_ctx* ctx, uint64_t* free_bytes, uint64_t* largest_block);

/* ------------------------------------------------------------- partitions */

/* mapParameters, data side (Sec. 3.1.1.1): copy one host primitive array of
 * n elements into a new arena-resident partition.  `host` may be pageable or
 * pinned; the copy is enqueued on `stream` and, for pageable memory, finished
 * before return.  n = 0 is allowed (an empty partition).
 * Errors: SCL_E_INVALID (dtype is KV, NULL host with n>0), SCL_E_NOMEM. */
int scl_load_partition(scl_ctx* ctx, const void* host, scl_dtype dtype,
                       uint64_t n, void* stream, scl_part* out);

/* Same for a keyed partition: keys[n] int32 and vals[n] float (SoA). */
int scl_load_partition_kv(scl_ctx* ctx, const int32_t* keys, const float* vals,
                          uint64_t n, void* stream, scl_part* out);

/* mapParameters for data produced on the device (Sec. 3.1.1.1): a new
 * arena-resident partition of n elements of `dtype` (keyed: keys then values)
 * whose contents are undefined until the caller writes them through the
 * device pointers scl_partition_info returns.  Nothing is copied or enqueued.
 * Like a loaded partition it is library-owned and counts as resident data in
 * the servers' HBM budget.  Errors: SCL_E_INVALID (bad dtype), SCL_E_NOMEM. */
int scl_alloc_partition(scl_ctx* ctx, scl_dtype dtype, uint64_t n, scl_part* out);

/* Wrap caller-owned device arrays as a partition without copying (e.g. a
 * torch tensor's data_ptr).  dev1 is the value array for SCL_KV_I32_F32 and
 * must be NULL otherwise.  The arrays must outlive the handle.  4-byte
 * alignment is required (16-byte aligned arrays take the vector path).  Any
 * address the GPU can load from works, including pinned host memory: kernels
 * then stream the partition straight from host memory over the host link
 * (no staging copy). */
int scl_wrap_device(scl_ctx* ctx, void* dev0, void* dev1, scl_dtype dtype,
                    uint64_t n, scl_part* out);

/* Refresh a resident partition with new host data of the same length (the
 * data side of mapParameters for the next task on the same buffers,
 * Sec. 3.1.1.1): host0[n] (and host1[n] for keyed) are copied into the
 * partition's device arrays on `stream`; nothing is allocated.  With pinned
 * host memory the copy is asynchronous: keep the host arrays unchanged until
 * the stream reaches it.  Works for library-owned and wrapped partitions. */
int scl_reload_partition(scl_ctx* ctx, scl_part part, const void* host0,
                         const void* host1, void* stream);

/* Release a partition (returns its arena block if the library owns it). */
int scl_free_partition(scl_ctx* ctx, scl_part part);

/* Describe a partition: dtype, length and device pointers (dev1 NULL unless
 * keyed).  Any output pointer may be NULL. */
int scl_partition_info(scl_ctx* ctx, scl_part part, scl_dtype* dtype,
                       uint64_t* n, void** dev0, void** dev1);

/* Copy a partition's array(s) back to host memory (mapReturnValue returning
 * an array, Sec. 3.1.1.3).  host0 receives n elements; host1 the values of a
 * keyed partition (may be NULL otherwise).  Synchronous on `stream`. */
int scl_read_partition(scl_ctx* ctx, scl_part part, void* host0, void* host1,
                       void* stream);

/* ------------------------------------------------------------ map / reduce */

/* MapCL with an output array (Sec. 3.1.3 item 1; Fig. 3's c[gid] = f(a[gid])):
 * allocate a partition of the same dtype and length and write y = map(x) to
 * it.  Kernels: MIX32 on U32/I32, POLY3 on F32, IDENT on U32/I32/F32 (copy).
 * `coef` is read for POLY3 (NULL = default).  Enqueued on `stream`; the
 * handle is usable for stream-ordered work at once.
 * Errors: SCL_E_UNSUPPORTED, SCL_E_NOMEM, SCL_E_INVALID. */
int scl_map(scl_ctx* ctx, scl_part in, scl_map_kernel kernel,
            const float coef[3], void* stream, scl_part* out);

/* The same map written into an existing partition of the same length and a
 * 32-bit dtype (allocates nothing; out may equal in for an in-place map). */
int scl_map_into(scl_ctx* ctx, scl_part in, scl_map_kernel kernel,
                 const float coef[3], scl_part out, void* stream);

/* MapCLPartition + ReduceCL over one partition, fused into one pass
 * (Sec. 3.1.3 items 2-3): y = map(x) for every element, folded by `reduce`.
 * Valid (kernel, reduce, dtype): {IDENT, MIX32} x SUM on U32/I32;
 * {IDENT, POLY3} x {SUM, SUM_MIN_MAX} on F32.  (Keyed partitions: see
 * scl_keyed_reduce / scl_keyed_reduce_hashed.)  Writes *out (host) and
 * synchronises `stream`.  Integer sums are exact; fp32 sums are fp32 only
 * within each thread's 4 x items_per_thread elements of a chunk and fp64
 * after (across chunks, threads, segments), folded in a fixed order, so a
 * result is bitwise reproducible and identical whether the partition runs
 * alone or in a batch of the same context.  Empty partition: sums 0,
 * min +inf, max -inf. */
int scl_map_reduce(scl_ctx* ctx, scl_part part, scl_map_kernel kernel,
                   const float coef[3], scl_reduce reduce, void* stream,
                   scl_result* out);

/* The same, enqueue-only: the result is written to device memory `dev_out`
 * (one scl_result) when the stream reaches it.  Each stream has its own
 * scratch, so calls on different streams may overlap on the device; calls on
 * one stream run in order.  (A destroyed stream's handle must not be reused
 * for a new stream while its calls are still running.) */
int scl_map_reduce_async(scl_ctx* ctx, scl_part part, scl_map_kernel kernel,
                         const float coef[3], scl_reduce reduce, void* stream,
                         scl_result* dev_out);

/* Keyed reduce of one KV partition (the reduce-by-key of Sec. 3.2.3):
 * counts_out[k] = number of pairs with key k (exact), sums_out[k] = their
 * value sum (fp32 accumulation per block, fp64 across blocks, rounded), and
 * sums64_out[k] the fp64 value (NULL to skip).  All outputs are HOST arrays
 * of num_keys (1..4096) entries.  Pairs with a key outside [0, num_keys)
 * are skipped and the call returns SCL_E_KEY_RANGE after writing the tables
 * of the valid pairs.  `result` (may be NULL) receives the totals. */
int scl_keyed_reduce(scl_ctx* ctx, scl_part part, uint32_t num_keys,
                     void* stream, uint32_t* counts_out, float* sums_out,
                     double* sums64_out, scl_result* result);

/* The keyed reduce after hashing each key into a bucket (WordCount's hash
 * into buckets before counting, Sec. 3.2.3): pair (key, value) is counted in
 * bucket (mix32(key) * num_keys) >> 32 (64-bit product), so every 32-bit key
 * is valid and no pair is skipped.  Outputs and errors as scl_keyed_reduce.
 * In a batch or server task the same reduce is kernel SCL_K_MIX32 with
 * reduce SCL_R_KEYED_COUNT_SUM on a keyed partition. */
int scl_keyed_reduce_hashed(scl_ctx* ctx, scl_part part, uint32_t num_keys,
                            void* stream, uint32_t* counts_out, float* sums_out,
                            double* sums64_out, scl_result* result);

/* Largest key space of scl_keyed_reduce_large (2^24 keys). */
#define SCL_MAX_LARGE_KEYS 16777216u

/* The keyed reduce for key spaces larger than 4096 (a WordCount-size
 * vocabulary, Sec. 3.2.3).  num_keys in [1, SCL_MAX_LARGE_KEYS].  Three paths
 * (scl_set_large_path chooses; by default packed from 2^17 to 2^22 keys,
 * else bucket-partitioned, else direct):
 *   - packed direct, for up to 2^22 keys: ids below 4096 go to a per-block
 *     shared-memory table; every other pair whose value is non-negative and
 *     inside a window [B/256, B) -- B the power of two above the largest value
 *     among the partition's first 65,536 -- takes one 64-bit integer add in
 *     L2 to a packed word per id (count in bits 40..63, round(v * 2^F) in
 *     bits 0..39, rounding error at most 2^-18 of v); other values take the
 *     direct path's two atomics.  If a packed word overflowed (an id with more
 *     than 32,768 packed pairs or 2^24 pairs), the call redoes itself on the
 *     device without packing (the result is the same; it takes longer).  Needs
 *     8 B per key from the arena;
 *   - bucket-partitioned, for partitions of 2^20 to 2^31 - 1 pairs whose key
 *     and value arrays are 16-byte aligned, over more than 4096 keys: the
 *     pairs are grouped by bucket (4096 to 16384 consecutive ids) in a
 *     temporary copy, then every bucket is counted in a per-block
 *     shared-memory table; when ids below 1024 hold at least 1/8 of the
 *     pairs (a vocabulary numbered by frequency) they are counted as the
 *     pairs are read instead of being copied.  Needs 8 B per pair plus a
 *     few bytes per chunk and bucket from the arena;
 *   - direct, otherwise or when the arena has no room for that copy: keys
 *     below 4096 (the frequent ids when words are numbered by frequency) go
 *     to a per-block shared-memory table, every other key straight to global
 *     atomics.
 * All yield the same tables.  HOST outputs of num_keys entries; sums_out is
 * the fp64 sum rounded to fp32.  Counts are exact; sums are fp32 partial sums
 * of at most 131,072 pairs per block and key added in fp64, within 1e-5 of an
 * fp64 fold (atomic order varies between runs).  Uses temporary device
 * tables from the arena (16 B per key), released before returning.  Returns
 * SCL_E_KEY_RANGE after writing the valid pairs' tables if a key was outside
 * [0, num_keys); SCL_E_STATE if the keys changed while the call read them
 * (the partitioned path reads them twice); SCL_E_TIMEOUT if one of the
 * partitioned path's bounded waits for its bulk copies ran out. */
int scl_keyed_reduce_large(scl_ctx* ctx, scl_part part, uint32_t num_keys, void* stream,
                           uint32_t* counts_out, float* sums_out, double* sums64_out,
                           scl_result* result);

/* Path of the large-key reduce.  A path that cannot run (partitioned: an
 * unaligned or short partition, or no arena room; packed: more than 2^22
 * keys, or no arena room) falls back to the direct kernel. */
typedef enum {
    SCL_LARGE_AUTO = 0,          /* packed for 2^17 to 2^22 keys, else partitioned */
    SCL_LARGE_PACKED = 1,
    SCL_LARGE_PARTITIONED = 2,
    SCL_LARGE_DIRECT = 3         /* the direct kernel without packing */
} scl_large_path;

/* Choose the path of this context's later large-key calls.
 * Errors: SCL_E_INVALID (unknown path). */
int scl_set_large_path(scl_ctx* ctx, scl_large_path path);

/* Enqueue-only form on DEVICE tables the caller owns: counts_dev (uint32),
 * sums_dev (float) and sums64_dev (double, required: it is the accumulator),
 * num_keys entries each, and dev_result (one scl_result).  All are zeroed or
 * overwritten on `stream` before use.  The partitioned path's temporary copy
 * is kept per stream (reused by later calls on that stream, returned by
 * scl_destroy); growing it synchronises the device. */
int scl_keyed_reduce_large_async(scl_ctx* ctx, scl_part part, uint32_t num_keys,
                                 void* stream, uint32_t* counts_dev, float* sums_dev,
                                 double* sums64_dev, scl_result* dev_result);

/* Enqueue-only keyed reduce; outputs are DEVICE arrays (sums64 may be NULL),
 * dev_result (device, may be NULL) gets the totals and status. */
int scl_keyed_reduce_async(scl_ctx* ctx, scl_part part, uint32_t num_keys,
                           void* stream, uint32_t* counts_out, float* sums_out,
                           double* sums64_out, scl_result* dev_result);

/* ------------------------------------- ReduceCL over partition arrays (Fig. 3) */

/* Largest number of arrays scl_reduce_arrays folds in one call. */
#define SCL_MAX_REDUCE_ARRAYS 1024

/* The paper's worked example (Fig. 3, Sec. 3.2.2 VectorAdd): the binary
 * kernel c[gid] = a[gid] + b[gid] used by ReduceCL, which folds the arrays of
 * an RDD's elements with a tree reduce.  scl_reduce_arrays folds k
 * equal-length partition arrays in one pass: out[i] = the tree sum of
 * parts[0][i] .. parts[k-1][i].  The tree is the binary-counter tree: arrays
 * are taken in order; whenever the two newest subtrees hold the same number
 * of arrays they are combined (older + newer); the leftover subtrees are
 * combined newest first, each older one on the left (the balanced pairwise
 * tree when k is a power of two).  F32: fp32 adds in that order, so results
 * are bitwise reproducible; U32/I32: addition mod 2^32.
 *
 * All partitions must have the same length and dtype class (F32, or 32-bit
 * integers); 1 <= k <= SCL_MAX_REDUCE_ARRAYS.  Enqueued on `stream`.
 * scl_reduce_arrays allocates the output partition (dtype of parts[0]);
 * scl_reduce_arrays_into writes an existing partition of the same length and
 * allocates nothing.  Errors: SCL_E_INVALID, SCL_E_UNSUPPORTED (keyed),
 * SCL_E_NOMEM. */
int scl_reduce_arrays(scl_ctx* ctx, const scl_part* parts, uint32_t k, void* stream,
                      scl_part* out);
int scl_reduce_arrays_into(scl_ctx* ctx, const scl_part* parts, uint32_t k,
                           scl_part out, void* stream);

/* One step of Fig. 3 itself: c = a + b elementwise (scl_reduce_arrays with
 * k = 2). */
int scl_vector_add(scl_ctx* ctx, scl_part a, scl_part b, void* stream, scl_part* out);

/* ----------------------------------------------- ReduceCL across partitions */

/* Host tree-combine of k per-partition results (ReduceCL's treeReduce,
 * Sec. 3.1.3 item 3 and Sec. 3.2.2): sums add (uint64 mod 2^64; fp64 by a
 * pairwise tree), min of mins, max of maxes, n adds; status is the first
 * non-OK status.  k = 0 gives the empty result. Pure host code. */
int scl_combine(const scl_result* parts, uint32_t k, scl_result* out);

/* Host merge of k keyed tables, row-major [k][num_keys]: counts add, fp64
 * sums add by a pairwise tree.  sums64 may be NULL (then only counts). */
int scl_combine_keyed(const uint32_t* counts, const double* sums64, uint32_t k,
                      uint32_t num_keys, uint32_t* counts_out,
                      double* sums64_out);

/* ------------------------------------------------------------ launch shapes */

/* Kernel families, each with its own launch shape. */
#define SCL_FAMILY_U32   0   /* uint32 partitions: mix32 / identity + uint64 sum     */
#define SCL_FAMILY_F32   1   /* fp32 partitions: poly3 / identity + sum / min / max  */
#define SCL_FAMILY_KEYED 2   /* keyed count + sum                                     */
#define SCL_FAMILY_MIXED 3   /* batches mixing families (uses the F32 block and
                                items per thread, its own CTAs per SM)                */

/* Launch shape of one kernel family: what the autotuner chooses.  A chunk is
 * block * items_per_thread * 4 elements; streaming partitions are cut into
 * segments of 1..4 chunks, so (block, items_per_thread) also fixes how fp32
 * sums are grouped -- results are bitwise stable for a fixed shape.  path 1
 * (TMA bulk-copy pipeline, one extra producer warp) exists for the U32 and
 * F32 families and gives bit-identical results to path 0 of the same
 * (block, items_per_thread). */
typedef struct {
    int32_t block;             /* data threads per CTA: 256 or 512               */
    int32_t items_per_thread;  /* 128-bit vectors per thread per chunk: 2, 4, 8  */
    int32_t ctas_per_sm;       /* resident CTAs per SM; 0 = as many as fit       */
    int32_t path;              /* 0 = vector loads, 1 = TMA bulk-copy pipeline,
                                  2 = keyed 512x2 capped at 48 registers        */
    int32_t stages;            /* TMA ring depth; 0 = the shape's default        */
    int32_t reserved;
} scl_shape;

/* Read / set a family's launch shape.  scl_set_shape returns
 * SCL_E_UNSUPPORTED for a shape that is not compiled into the library.  A
 * batch keeps the shape it was created with. */
int scl_get_shape(scl_ctx* ctx, int family, scl_shape* out);
int scl_set_shape(scl_ctx* ctx, int family, const scl_shape* shape);

/* Autotuner configuration; every field may be 0 for its default. */
typedef struct {
    uint64_t probe_bytes;   /* bytes read by each probe batch (512 MiB)          */
    uint32_t reps;          /* timed launches per candidate (10)                 */
    uint32_t families;      /* bit (1 << SCL_FAMILY_*) per family to tune (all)  */
} scl_autotune_config;

typedef struct {
    scl_shape chosen[4];    /* per family, the shape now in effect               */
    double best_ms[4];      /* its probe time (large + small batch), ms          */
    uint32_t candidates[4]; /* candidates timed                                  */
} scl_autotune_report;

/* Choose each family's launch shape by measurement: block size, items per
 * thread, CTAs per SM, load path and TMA ring depth.  Two probe batches are
 * filled on the device in the arena -- four large partitions, and uneven
 * partitions with log-normal sizes (median 16,384, sigma 1.5) -- each reading
 * probe_bytes (larger than the L2 by default); every compiled candidate is
 * timed with CUDA events on `stream` (best of three rounds of `reps`
 * launches) and the candidate with the smallest sum of (time / best time)
 * over the probes is kept.  The FP32 family is tuned first and its candidates
 * are also scored on a mixed batch, because MIXED inherits its block and
 * items per thread; MIXED then tunes CTAs per SM.  If the context has a tune
 * cache path, the result is written there and loaded by later contexts on a
 * GPU with the same SM count.  cfg and report may be NULL.  Takes a few
 * seconds; the arena needs about 8 x probe_bytes free (the probe shrinks to
 * fit, down to 16 MiB).  Errors: SCL_E_NOMEM, SCL_E_CUDA, SCL_E_TIMEOUT. */
int scl_autotune(scl_ctx* ctx, const scl_autotune_config* cfg, void* stream,
                 scl_autotune_report* report);

/* ---------------------------------------------------------------- batches */

/* Plan many partition tasks as ONE persistent launch (thousands of uneven
 * partitions; the paper's "enough data" concern, Sec. 3 item 2, and kernel
 * caching per worker, Sec. 3.1.1.2).  Streaming tasks are cut into segments
 * that CTAs pull from a queue; keyed tasks into even shares of the keyed work
 * (pairs plus a fixed cost per piece) over the CTAs that take keyed pieces.
 * A batch whose tasks mix families (uint32, fp32, keyed) launches, with
 * splitting on (the default, scl_set_batch_split), one persistent kernel per
 * family, concurrently: the keyed-only kernel first on `stream` (512-thread
 * CTAs capped at 48 registers, two per SM, so that two streaming CTAs stay
 * resident beside them on every SM), the others on two side streams the
 * batch owns, forked from `stream` and joined back into it.  With splitting off it is one launch of the mixed kernel, a
 * cost-weighted share of whose CTAs take the keyed pieces while the rest
 * stream.  The plan, task table and scratch are placed in the arena; nothing
 * runs yet.
 * Tasks keep referencing their partitions: those must stay alive while the
 * batch exists.  Errors: SCL_E_INVALID, SCL_E_UNSUPPORTED, SCL_E_NOMEM. */
int scl_batch_create(scl_ctx* ctx, const scl_task* tasks, uint32_t ntasks,
                     scl_batch** out);

/* Enqueue the batch on `stream` (its CUDA graph if one was captured, else a
 * direct launch).  Results land in device memory; read them with
 * scl_batch_results.  Launches of one batch must not overlap (use one
 * stream or order them). */
int scl_batch_launch(scl_batch* batch, void* stream);

/* Capture the batch's launch into a CUDA graph on `stream` (which must not
 * be capturing already); later scl_batch_launch calls replay it. */
int scl_batch_capture(scl_batch* batch, void* stream);

/* Copy the last launch's results to host results[ntasks] after synchronising
 * `stream`.  Returns SCL_E_KEY_RANGE if any task saw a bad key, and
 * SCL_E_TIMEOUT / SCL_E_STATE if the launch set its device error word (the
 * batch's scratch is then reset, so the next launch starts clean). */
int scl_batch_results(scl_batch* batch, void* stream, scl_result* results);

/* Whether later scl_batch_create calls of this context split a batch that
 * mixes families into concurrent per-family launches (on = 1, the default;
 * off = 0: one mixed-kernel launch).  Results are the same either way except
 * the fp32 keyed sums, which are rounded in a different order.
 * Errors: SCL_E_INVALID (on not 0 or 1). */
int scl_set_batch_split(scl_ctx* ctx, int on);

/* Kernel launches that one launch of this batch makes (for accounting). */
int scl_batch_kernel_launches(scl_batch* batch, uint32_t* count);

/* Free the batch (its graph and arena blocks). NULL is a no-op. */
int scl_batch_destroy(scl_batch* batch);

/* One-shot: create, launch, read results, destroy. */
int scl_batch_run(scl_ctx* ctx, const scl_task* tasks, uint32_t ntasks,
                  void* stream, scl_result* results);

/* ------------------------------------------------- allocation-free variant */

/* Largest partition scl_map_reduce_noalloc accepts (2^26 elements). */
#define SCL_NOALLOC_MAX_ELEMENTS 67108864ull

/* Map + reduce of one partition without allocating anything: no context, no
 * arena, no cudaMalloc/cudaFree, no pinned staging, no allocating library
 * call.  The paper has no counterpart; this exists for callers that cannot
 * allocate device memory at the moment they need a result -- plug-ins inside
 * an application whose own pool already holds all of the GPU's memory, and
 * latency-critical paths that cannot take the device synchronisation of
 * cudaMalloc/cudaFree.
 *
 * dev_in: device array of n elements of `dtype` (U32, I32 or F32; 4-byte
 * aligned, 16-byte aligned takes the vector path).  kernel / coef / reduce:
 * as scl_map_reduce (no keyed reduce).  dev_out: one device scl_result,
 * written when `stream` reaches the launch.  Enqueue-only: nothing is
 * synchronised.
 *
 * Scratch: a fixed device array inside the library, 96 B of counters plus
 * 4096 segment partials of 32 B (128 KB in all); every GPU that loads the
 * library holds it until the process exits.  Partitions larger than
 * SCL_NOALLOC_MAX_ELEMENTS are rejected with SCL_E_INVALID before anything is
 * enqueued.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) and the launch limits, with that device current,
 * and keeps them for that device ordinal for the life of the process (a
 * cudaDeviceReset is not followed); make that first call before any stream
 * capture.  Each call clears the 96 B of counters on `stream` before its
 * launch.  All calls share the one
 * array: calls whose work can overlap on the GPU (different streams, or
 * different host threads) race and give wrong results -- order them, e.g. on
 * one stream.  Errors: SCL_E_INVALID, SCL_E_UNSUPPORTED, SCL_E_CUDA. */
int scl_map_reduce_noalloc(const void* dev_in, scl_dtype dtype, uint64_t n,
                           scl_map_kernel kernel, const float coef[3],
                           scl_reduce reduce, void* stream, scl_result* dev_out);

/* ----------------------------------------------------------------- server */

/* The continuous-batching server.  The paper serialises acceleration tasks
 * per device by giving each accelerator worker one core (Sec. 3.1.5) and asks
 * for enough data per offload (Sec. 3 items 1-2); here tasks that arrive
 * while others run are admitted as HBM budget frees, packed into the next
 * persistent launch, and overlap on the device with batches already running.
 *
 * Admission: a task is charged an estimate of its device working set (plan
 * entry, segment partials, keyed tables, and its input if it brings new data);
 * it enters the GPU queue when partitions resident in the arena + working sets
 * of admitted tasks + its own fit hbm_budget_bytes, otherwise it waits FIFO.
 * A task that can never fit is rejected with SCL_E_BUDGET.  A task that brings
 * new data is copied at admission and joins a launch once its copy has
 * landed; tasks admitted after it do not wait for that copy. */
typedef struct {
    int32_t inflight_batches;   /* launches on the GPU at once, one stream each
                                   (1..16; 0 = 4)                                  */
    uint32_t max_batch_tasks;   /* tasks per launch (1..65536; 0 = 4096);
                                   1 = unbatched: one launch per task             */
    uint64_t hbm_budget_bytes;  /* 0 = scl_config's budget, else the arena size    */
    uint64_t reserved[2];
} scl_server_config;

typedef struct {
    uint64_t submitted, completed, rejected;
    uint64_t batches, max_batch, kernel_launches;
    uint64_t admission_waits;    /* tasks that waited for budget                   */
    uint64_t budget_bytes, resident_bytes, bytes_in_use, peak_bytes_in_use;
} scl_server_stats;

/* Start the server threads (batcher + completion) on this context.  Only one
 * server per context.  Partitions referenced by tasks must stay alive until
 * their tasks complete.  Errors: SCL_E_STATE (already running). */
int scl_server_start(scl_ctx* ctx, const scl_server_config* cfg);

/* Submit one task on a resident partition; returns at once with a ticket.
 * Keyed tasks write their tables to the task's device arrays.  Thread-safe.
 * Errors: SCL_E_INVALID, SCL_E_UNSUPPORTED, SCL_E_BUDGET, SCL_E_STATE. */
int scl_server_submit(scl_ctx* ctx, const scl_task* task, uint64_t* ticket);

/* Submit a task that brings new data (mapParameters' copy, Sec. 3.1.1.1):
 * host0[n] (and host1[n] for keyed) are copied to a transient partition when
 * the task is admitted, and freed when it completes; the copy counts in the
 * task's latency.  The host arrays must stay valid until the task completes
 * (pinned memory copies asynchronously).  task->part is ignored. */
int scl_server_submit_load(scl_ctx* ctx, const void* host0, const void* host1,
                           scl_dtype dtype, uint64_t n, const scl_task* task,
                           uint64_t* ticket);

/* SCL_OK and the result once the task is done (the ticket is then retired),
 * SCL_E_PENDING before.  A failed task has its status in out->status. */
int scl_server_poll(scl_ctx* ctx, uint64_t ticket, scl_result* out);

/* Block until the task is done or timeout_ms passes (SCL_E_TIMEOUT). */
int scl_server_wait(scl_ctx* ctx, uint64_t ticket, uint32_t timeout_ms,
                    scl_result* out);

int scl_server_get_stats(scl_ctx* ctx, scl_server_stats* out);

/* Drain admitted work, stop the threads, release the server.  No-op if not
 * running.  Called by scl_destroy. */
int scl_server_stop(scl_ctx* ctx);

/* Open-loop trace driver: submit tasks[i] at arrival_s[i] seconds after the
 * start (scheduled, not when the previous task finished), then wait for all.
 * latency_ns[i] = completion time - scheduled arrival (may be NULL);
 * results[i] the result (may be NULL).  Runs on the calling thread. */
int scl_server_replay(scl_ctx* ctx, const scl_task* tasks, const double* arrival_s,
                      uint32_t n, int64_t* latency_ns, scl_result* results);

/* Data of one task of a replayed trace that brings new data
 * (scl_server_replay_load): host0[n] (keys for SCL_KV_I32_F32) and host1[n]
 * (values, keyed only) are copied to the device at admission, as
 * scl_server_submit_load does.  host0 == NULL: the task runs on its resident
 * partition tasks[i].part. */
typedef struct {
    const void* host0;
    const void* host1;
    uint64_t n;
    int32_t dtype;       /* scl_dtype */
    uint32_t reserved;
} scl_task_data;

/* scl_server_replay where some tasks bring new data (data[i].host0 != NULL):
 * their host-to-device copy is part of their latency.  Results are collected
 * while the trace is still being submitted. */
int scl_server_replay_load(scl_ctx* ctx, const scl_task* tasks, const scl_task_data* data,
                           const double* arrival_s, uint32_t n, int64_t* latency_ns,
                           scl_result* results);

/* ------------------------------------------------------ device-polling server */

/* The device-polling server: the same offload of partition tasks as the
 * continuous-batching server, with no kernel launch per batch.  One kernel
 * stays resident on the GPU; scl_devserver_submit writes the task as a job
 * into pinned host memory the kernel reads through its mapped address and
 * then advances a published-work count (the doorbell); the kernel's CTAs
 * claim the job's work units (streaming segments, keyed pieces) from a
 * device counter, run them and write the result and a done word into pinned
 * host memory, where a driver thread hands it out.  The paper runs each
 * partition task through its worker's accelerator, one at a time per device
 * (Sec. 3.1.1-3.1.5); it has no device-resident dispatcher.
 *
 * Results: uint32 and fp32 tasks give bitwise the result scl_map_reduce gives
 * with the fp32 family's (block, items per thread) -- the same segment code;
 * keyed tasks give exact counts and fp64-accumulated sums (float atomics make
 * their last bits depend on timing, as in the batch kernels).
 *
 * Waits are bounded.  The host ends the kernel after idle_stop_ns without
 * work (and launches it again with the next job).  In the kernel, a CTA
 * waiting for the doorbell gives up after wait_limit_ns (or an iteration
 * limit if the GPU timer stalls), sets an error word in host memory and
 * returns; a job descriptor that fails the kernel's bounds checks does the
 * same.  The driver then ends the kernel, fails the jobs in flight with
 * status SCL_E_TIMEOUT, zeroes the device state and carries on
 * (device_errors counts these).
 *
 * While the kernel is resident it holds the SMs: other launches on the
 * device start as its CTAs leave, i.e. idle_stop_ns after its last job or at
 * scl_devserver_stop.  Partitions and keyed output arrays referenced by jobs
 * must stay alive until the jobs complete. */
typedef struct {
    uint32_t job_ring;        /* jobs in flight (0 = 16384)                      */
    uint32_t unit_ring;       /* work units in flight, also streaming partial
                                 slots (0 = 1048576)                             */
    uint32_t keyed_slots;     /* multi-piece keyed jobs in flight (0 = 256)      */
    int32_t ctas_per_sm;      /* resident CTAs per SM (0 = as many as fit)       */
    uint64_t idle_stop_ns;    /* end the kernel after this long without work
                                 (0 = 2 ms; UINT64_MAX = never: the device wait
                                 limit then ends it, as an error)                */
    uint64_t wait_limit_ns;   /* longest device wait for the doorbell (0 = 1 s)  */
    uint64_t reserved[2];
} scl_devserver_config;

typedef struct {
    uint64_t submitted, completed, failed;
    uint64_t kernel_launches;  /* resident-kernel instances started             */
    uint64_t idle_stops;       /* instances ended by the host after idling      */
    uint64_t device_errors;    /* instances ended by a device wait limit or a
                                  failed descriptor check                       */
    uint64_t units;            /* work units published                          */
    uint64_t ring_waits;       /* jobs that waited for ring space               */
    uint64_t max_inflight;     /* most jobs in flight at once                   */
    uint32_t grid, block;      /* launch shape of the resident kernel           */
    uint32_t items_per_thread, reserved0;
    uint64_t reserved[3];
} scl_devserver_stats;

/* Start the device-polling server on this context (the kernel is launched
 * with the first job).  Takes unit_ring x 32 + keyed_slots x 48 Ki +
 * job_ring x 140 bytes of the arena (47 MB at the defaults) and job_ring x 180
 * + unit_ring x 8 bytes of pinned host memory (11 MB).
 * Errors: SCL_E_STATE (already running), SCL_E_INVALID, SCL_E_NOMEM,
 * SCL_E_UNSUPPORTED (no compiled kernel for the fp32 family's shape). */
int scl_devserver_start(scl_ctx* ctx, const scl_devserver_config* cfg);

/* Submit one task on a resident partition; returns at once with a ticket.
 * Thread-safe.  Errors: SCL_E_INVALID, SCL_E_UNSUPPORTED, SCL_E_BUDGET (more
 * work units than the rings hold), SCL_E_STATE (not running), SCL_E_CUDA
 * (the server met a CUDA error and stopped taking work). */
int scl_devserver_submit(scl_ctx* ctx, const scl_task* task, uint64_t* ticket);

/* SCL_OK and the result once done (the ticket is then retired), SCL_E_PENDING
 * before.  A failed job has its status in out->status. */
int scl_devserver_poll(scl_ctx* ctx, uint64_t ticket, scl_result* out);

/* Block until the job is done or timeout_ms passes (SCL_E_TIMEOUT). */
int scl_devserver_wait(scl_ctx* ctx, uint64_t ticket, uint32_t timeout_ms,
                       scl_result* out);

int scl_devserver_get_stats(scl_ctx* ctx, scl_devserver_stats* out);

/* Finish the jobs in flight, end the kernel, release the server.  No-op if
 * not running.  Called by scl_destroy. */
int scl_devserver_stop(scl_ctx* ctx);

/* Open-loop trace driver, as scl_server_replay: submit tasks[i] at
 * arrival_s[i] seconds after the start, then wait for all (each wait bounded
 * by 60 s, else SCL_E_TIMEOUT).  latency_ns[i] = completion seen by the host
 * - scheduled arrival (may be NULL); results[i] (may be NULL). */
int scl_devserver_replay(scl_ctx* ctx, const scl_task* tasks, const double* arrival_s,
                         uint32_t n, int64_t* latency_ns, scl_result* results);

#ifdef __cplusplus
}
#endif

#endif /* SCL_H */
