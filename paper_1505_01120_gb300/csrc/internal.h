// internal.h -- structures shared by the sm_103a kernels and the host runtime
// of libscl.  Not part of the ABI (include/scl.h is).
//
// Execution model.  A launch runs a set of partition tasks.  Each task is one
// partition with one catalogue kernel (SparkCL's per-partition kernel run,
// Sec. 3.1.1-3.1.3).  Two kinds of work units exist:
//   * streaming segments: a task of a streaming kind (uint32 sum, fp32
//     sum/min/max) is cut into fixed segments whose length depends only on the
//     partition length and the launch shape; CTAs of a persistent grid pull
//     segments from one global counter; every segment leaves one partial in
//     its own slot, and the CTA that finishes a task's last segment folds the
//     slots in slot order (one atomic ticket per task).
//   * keyed pieces: keyed tasks are split by the host planner into contiguous
//     pieces, an even share of the keyed work per CTA; each CTA accumulates
//     its piece into a shared-memory table and writes the table to its slot;
//     a second, small kernel folds the slots of multi-piece tasks.
#pragma once

#include <stdint.h>

#include "scl.h"

#if !defined(__CUDACC__)   // plain C++ (the host tests): the geometry helpers below
#ifndef __host__
#define __host__
#endif
#ifndef __device__
#define __device__
#endif
#endif

namespace scl {

constexpr uint32_t kMaxKeys = 4096;                 // shared-memory table entries
constexpr uint32_t kKeyedTableWords = 2 * kMaxKeys; // count[kMaxKeys] then sum[kMaxKeys]
// Fp32 sums of the first kKeyedHead ids of a table (the frequent words when a
// vocabulary is numbered by frequency) go to a private copy per warp and lane
// class, folded into the table after accumulating: shared-memory float
// atomics contending for one address serialise (on GB300, Zipf(1.2) keys made
// the table 7x slower than uniform keys; with the copies, 1.2x).
constexpr uint32_t kKeyedHead = 32;
constexpr uint32_t kKeyedHeadClasses = 4;
constexpr uint32_t kKeyedHeadStride = kKeyedHead + 1;   // copies start on different banks
__host__ __device__ constexpr uint32_t kKeyedHeadWords(uint32_t block) {
    return block / 32 * kKeyedHeadClasses * kKeyedHeadStride;
}
// Shared memory of a keyed CTA (blocks of up to 512 threads): table, copies.
constexpr uint32_t kKeyedSmemBytes = (kKeyedTableWords + kKeyedHeadWords(512)) * 4;
// Fixed-point windows of the keyed-only kernel (Sec. 3.2.3's reduce-by-key
// with integer table adds).  Shared-memory integer adds cost about half of
// fp32 adds under random-key bank conflicts on GB300, so a piece's values in
// [B * 2^-kFixTinyBits, B) -- B the power of two just above the largest value
// of its first chunk -- are added as int32 multiples of 2^-F, F chosen so that
// fewer than 2^kFixCountBits such adds to one key cannot overflow.  The int32
// sums are folded into the fp32 table every kFixWindow pairs; a window in
// which a key took 2^kFixCountBits pairs or more makes the piece run again on
// the fp32 table alone.  Each value's rounding error is below
// 2^(kFixCountBits + kFixTinyBits - 32) = 2^-18 of its magnitude.  Values
// whose magnitude is outside the window (smaller, larger, non-finite) take
// fp32 adds; the sign does not matter; zeros add nothing.
constexpr uint32_t kFixCountBits = 9;   // also keeps |round(v * 2^F)| <= 2^22 (exact FMA rounding)
constexpr uint32_t kFixTinyBits = 5;
constexpr uint64_t kFixWindow = 65536;        // pairs per window, a multiple of every chunk
constexpr uint64_t kFixMinPairs = 16384;      // shorter pieces use the fp32 table only
constexpr uint32_t kFixMinKeys = 1024;        // smaller key spaces use the fp32 table only
constexpr uint32_t kFixSumOffset = kKeyedSmemBytes;              // int32 window sums
constexpr uint32_t kFixSnapOffset = kFixSumOffset + kMaxKeys * 4; // counts at the window's start
constexpr uint32_t kFixMaxOffset = kFixSnapOffset + kMaxKeys * 4; // per-warp maxima
constexpr uint32_t kKeyedFastSmemBytes = kFixMaxOffset + 16 * 4;
constexpr uint64_t kKeyedPieceAlign = 64;           // piece boundaries, in pairs
constexpr uint64_t kKeyedMinPiece = 32768;          // pairs; keeps table flushes cheap
constexpr uint64_t kKeyedMinFragment = 8192;        // pairs; shorter end pieces join a neighbour
constexpr uint64_t kKeyedTaskOverhead = 4096;       // pair-equivalents per keyed task (default)
constexpr uint64_t kKeyedPieceOverheadFast = 32;    // per thread of a keyed-only CTA
constexpr uint64_t kKeyedPieceOverheadMixed = 16;   // per thread of a mixed-kernel CTA
constexpr uint32_t kMaxSegChunks = 4;               // a streaming segment is 1..4 chunks
constexpr uint32_t kTargetSegsPerTask = 256;
constexpr uint32_t kFoldBlock = 256;                // keyed fold kernel block size
// A keyed task of at most this many pieces is folded by the CTA that writes
// its last piece table; one of more pieces by k_keyed_fold, whose CTAs split
// the ids (a task of many pieces ends with all of them, at the kernel's end).
constexpr uint32_t kFoldInKernelMaxPieces = 8;

// Work kinds: (map kernel, reduce) combinations of the catalogue.
enum Kind : uint32_t {
    K_U32_IDENT = 0,   // uint64 sum of raw uint32
    K_U32_MIX32 = 1,   // uint64 sum of mix32(x)
    K_F32_IDENT = 2,   // sum / min / max of raw fp32
    K_F32_POLY3 = 3,   // sum / min / max of poly3(x)
    K_KEYED = 4,       // per-key count / sum
    K_KEYED_MIX = 5,   // per-bucket count / sum, bucket = (mix32(key) * num_keys) >> 32
    K_NUM = 6
};

__host__ __device__ constexpr bool is_keyed(uint32_t k) { return k == K_KEYED || k == K_KEYED_MIX; }

// Which kinds a compiled persistent kernel contains.
enum Mask : uint32_t { M_U32 = 0, M_F32 = 1, M_KEYED = 2, M_ALL = 3, M_NUM = 4 };

__host__ __device__ constexpr bool mask_has_u32(int m) { return m == M_U32 || m == M_ALL; }
__host__ __device__ constexpr bool mask_has_f32(int m) { return m == M_F32 || m == M_ALL; }
__host__ __device__ constexpr bool mask_has_keyed(int m) { return m == M_KEYED || m == M_ALL; }
__host__ __device__ constexpr bool mask_has_stream(int m) { return m != M_KEYED; }

enum TaskFlags : uint32_t { TF_ALIGNED = 1u };  // in0 (and in1) 16-byte aligned

struct alignas(16) DevTask {
    const void* in0;        // values, or keys for K_KEYED
    const void* in1;        // values for K_KEYED
    scl_result* result;     // device result slot
    uint32_t* counts_out;   // keyed outputs (device)
    float* sums_out;
    double* sums64_out;     // may be null
    uint64_t n;             // elements / pairs
    uint32_t kind;
    uint32_t num_keys;
    uint32_t nseg;          // streaming segments or keyed pieces of this task
    uint32_t slot0;         // first partial slot of this task
    uint32_t seg_elems;     // streaming segment length (elements)
    uint32_t flags;
    float coef[3];
    uint32_t seg_base;      // first global streaming segment of this task
};
static_assert(sizeof(DevTask) == 96, "DevTask layout");

struct KPiece {             // one keyed piece: pairs [begin, end) of a task
    uint64_t begin, end;
    uint32_t task, slot;
};
static_assert(sizeof(KPiece) == 24, "KPiece layout");

struct alignas(16) StreamPartial {  // one streaming segment's partial
    float shi, slo; // sum (fp32 kinds) as a float-float pair: shi + slo
    uint64_t u;     // uint64 sum (uint32 kinds)
    float mn, mx;
    uint32_t pad[2];
};
static_assert(sizeof(StreamPartial) == 32, "StreamPartial layout");

// Header words of a launch's scratch.
enum HdrWord : uint32_t {
    H_QUEUE = 0, H_EXIT = 1, H_ERROR = 2, H_FOLD_EXIT = 3,
    H_LARGE_TICKET = 8, H_LARGE_BAD = 9,   // the large-key reduce's finishing ticket and key flag
    H_RADIX_TICKET = 10,                   // the large-key reduce's bucket-scan ticket
    H_WORDS = 16
};

struct KernelArgs {
    const DevTask* tasks;       // null: single-task mode, the task is `single`
    const uint32_t* seg_task;   // global streaming segment -> task (batch mode)
    const uint32_t* kp_first;   // [grid + 1] first keyed piece of each CTA (batch mode)
    const KPiece* kpieces;
    const uint32_t* fold_tasks; // keyed tasks with more than one piece (batch mode)
    StreamPartial* spart;       // streaming partial slots
    uint32_t* kpart;            // keyed partial tables, kKeyedTableWords words per slot
    StreamPartial* fpart;       // keyed fold: one partial per (fold task, key block)
    uint32_t* tickets;          // per task; zero between launches
    uint32_t* task_flags;       // per task; bit 0 = a key was out of range
    uint32_t* hdr;              // H_WORDS words
    uint32_t nseg_stream;       // total streaming segments
    uint32_t nkeyed_ctas;       // single-task keyed mode: number of pieces
    uint32_t nfold;             // entries of fold_tasks (batch mode)
    uint32_t pad;
    uint32_t* err_out;          // if set, the last CTA to exit copies H_ERROR here
    DevTask single;
};

// Geometry of a streaming task's segments, shared by host planning and tests.
__host__ __device__ constexpr uint32_t stream_seg_elems(uint64_t n, uint32_t chunk) {
    uint64_t per = (uint64_t)chunk * kTargetSegsPerTask;
    uint64_t c = (n + per - 1) / per;
    if (c < 1) c = 1;
    if (c > kMaxSegChunks) c = kMaxSegChunks;
    return (uint32_t)(c * chunk);
}

__host__ __device__ constexpr uint32_t stream_nseg(uint64_t n, uint32_t seg_elems) {
    uint64_t s = (n + seg_elems - 1) / seg_elems;
    return s < 1 ? 1u : (uint32_t)s;
}

// Single-task keyed pieces: piece c of G covers [B(c), B(c+1)).
__host__ __device__ inline uint64_t keyed_single_bound(uint64_t n, uint32_t c, uint32_t G) {
    if (c == 0) return 0;
    if (c >= G) return n;
    uint64_t b = (uint64_t)c * n / G;   // c < 2^20, n < 2^43 in practice: no overflow
    return b / kKeyedPieceAlign * kKeyedPieceAlign;
}

__host__ __device__ inline uint32_t keyed_single_pieces(uint64_t n, uint32_t grid) {
    uint64_t g = (n + kKeyedMinPiece - 1) / kKeyedMinPiece;
    if (g < 1) g = 1;
    if (g > grid) g = grid;
    return (uint32_t)g;
}

// ReduceCL over k equal-length partition arrays (the vector-add kernel of
// Fig. 3 folded by a tree reduce, Sec. 3.2.2).
constexpr uint32_t kMaxTreeArrays = 1024;
constexpr int kTreeLevels = 11;                     // 2^10 leaves need 11 levels

struct TreeArgs {
    const char* in[kMaxTreeArrays];   // device addresses of the k input arrays
    char* out;
    uint64_t n;                       // elements per array
    uint32_t k;
    uint32_t pad;
};

// Keyed reduce over key spaces larger than the shared table: keys below
// kMaxKeys are accumulated in a per-CTA shared-memory table (the hot ids of a
// frequency-ordered dictionary) and flushed every kLargePiece pairs; the rest
// go straight to global count / fp64 sum atomics.
constexpr uint32_t kMaxLargeKeys = 1u << 24;
constexpr uint64_t kLargePiece = 131072;
// Pairs per piece of the direct kernel (64 Mi pairs over 2^20 uniform keys,
// packed: 0.479 ms at 131,072, 0.454 at 32,768 -- more CTAs keep more L2 adds
// in flight -- 0.448 at 16,384, where skewed keys lose to table flushes).
constexpr uint64_t kDirectPiece = 32768;

// Packed L2 accumulators of the direct path (num_keys up to kMaxPackedKeys):
// one 64-bit word per id, count in bits 40..63 and a fixed-point sum in bits
// 0..39, so an id takes one 64-bit integer add per pair in L2 instead of a
// count add and an fp64 add (the L2 atomic units take either add at about the
// same rate).  Non-negative values in [B/256, B), B the power of two above the
// largest value of the partition's first kPackedScaleSample values, are added
// as round(v * 2^F) <= 2^25 (rounding error at most 2^-18 of the value); other
// pairs take the count / fp64 adds.  If a sum field overflowed into its count
// or a count wrapped, the decoded counts differ from the number of packed adds:
// the finishing pass then sets kLargeRepair and guarded kernels redo the call
// without packing.
constexpr uint32_t kMaxPackedKeys = 1u << 22;
// Smallest key space the automatic choice packs: below it a uniform key set
// puts many adds on each packed word and the partitioned path is faster
// (2^14 uniform keys: 0.67 against 0.51 ms; skewed keys prefer the direct
// kernel at any size).
constexpr uint32_t kMinPackedKeys = 1u << 17;
constexpr uint32_t kPackedScaleSample = 65536;
constexpr uint32_t kPackedCountShift = 40;
constexpr uint32_t kLargeRepair = 8u;     // bit of *bad: redo the call without packing

struct LargeFix {
    float scale, inv;         // 2^F, 2^-F
    uint32_t lo, span;        // value bit patterns packed: [lo, lo + span)
    uint32_t on;              // 0: no window; every pair takes the count / fp64 adds
    uint32_t pad;
    unsigned long long npacked;   // pairs added to the packed words
    unsigned long long ndecoded;  // counts decoded from them (finishing pass)
};

struct LargeKeyedArgs {
    const char* keys;
    const char* vals;
    uint64_t n;
    uint32_t num_keys;
    uint32_t aligned;
    uint32_t* counts;         // [num_keys], zeroed before the launch
    double* sums64;           // [num_keys], zeroed before the launch
    float* sums32;            // [num_keys] written by the finishing pass
    scl_result* result;       // zeroed before the launch
    uint32_t* ticket;         // zero between launches (finishing pass)
    uint32_t* bad;            // zeroed before the launch
    unsigned long long* packed;   // [num_keys] packed words, zeroed before; null: no packing
    LargeFix* fix;            // the window (set by the scale pass) and its counters
    uint32_t guard;           // 1: the kernel runs only if *bad has kLargeRepair
    uint32_t pad;
};

// Device-polling server.  The host publishes jobs in pinned host memory that
// the device reads through its mapped address; a resident kernel claims work
// units (streaming segments or keyed pieces) from a device counter.  Jobs are
// published in order: job p sits in ring slot p % job_ring, its units follow
// those of job p - 1, and the host's doorbell is the count of jobs published.
// One CTA at a time reads the doorbell and expands new jobs into device
// memory (descriptor copy, unit -> slot map) before it raises the device's
// count of available units; every other CTA reads only device memory.
constexpr uint64_t kDbKeyedPiece = 65536;     // pairs per keyed piece (at least)
constexpr uint32_t kDbMaxKeyedPieces = 4096;
constexpr uint32_t kDbAccWords = kMaxKeys * 3; // keyed accumulator: u32 count, f64 sum
constexpr uint32_t kDbMaxExpand = 64;          // jobs expanded per doorbell read

enum DbErr : uint32_t { DB_ERR_WAIT = 1u, DB_ERR_DESC = 2u };

struct alignas(16) DbJob {     // 128 bytes, host memory (and its device copy)
    DevTask t;                 // result: mapped host slot; slot0: partial range or accumulator
    uint64_t unit0;            // first unit of the job in this kernel instance's numbering
    uint32_t seq;              // written to done[ring] once the result is in place
    uint32_t ring;             // p % job_ring (tickets, flags, results, done)
    uint32_t pad[4];
};
static_assert(sizeof(DbJob) == 128, "DbJob layout");

struct alignas(128) DbHost {   // pinned host memory, mapped
    unsigned long long jobs;   // jobs published (host writes, release): the doorbell
    uint32_t pad0[30];
    uint32_t stop;             // host: stop once no published unit is left
    uint32_t pad1[31];
    uint32_t err;              // device: DbErr bits
    uint32_t pad2[31];
};

struct alignas(128) DbState {  // device memory, zero at every kernel start
    unsigned long long next;   // claim counter
    uint32_t pad0[30];
    unsigned long long tail;   // units expanded (available to claim)
    uint32_t stop;             // device mirror of DbHost::stop
    uint32_t pad1[29];
    uint32_t lock;             // held by the CTA reading the doorbell
    uint32_t pad2;
    unsigned long long jobs_seen;   // jobs expanded (lock holder only)
    uint32_t pad3[28];
};

struct DbArgs {
    KernelArgs ka;              // spart, tickets, task_flags of the job ring
    DbHost* host;               // device address of the mapped header
    const DbJob* jobs;          // [job_ring], mapped
    uint32_t* done;             // [job_ring], mapped
    DbState* state;
    DbJob* djobs;               // [job_ring] device copies of the descriptors
    uint32_t* dunit;            // [unit_ring] unit -> ring slot of its job
    uint32_t* kacc;             // [kacc_slots][kDbAccWords]: count[kMaxKeys] u32, sum[kMaxKeys] f64
    unsigned long long wait_limit_ns;
    unsigned long long max_polls;
    uint32_t job_ring, unit_ring, spart_cap, kacc_slots;
};

// Keyed pieces of a device-polled keyed job of n pairs.
__host__ __device__ inline uint32_t db_keyed_pieces(uint64_t n) {
    uint64_t g = (n + kDbKeyedPiece - 1) / kDbKeyedPiece;
    if (g < 1) g = 1;
    if (g > kDbMaxKeyedPieces) g = kDbMaxKeyedPieces;
    return (uint32_t)g;
}

// Host-side launch entry of one compiled persistent-kernel instantiation.
struct KernelEntry {
    int mask, block, ipt;              // block = threads that touch data (consumers)
    const void* fn;                    // __global__ function pointer
    size_t dyn_smem;                   // dynamic shared memory per CTA
    int path;                          // PATH_LDG or PATH_TMA
    int stages;                        // TMA ring stages (0 for LDG)
};

// PATH_LEAN: the keyed-only kernel capped at kKeyedLeanRegs registers.
enum Path : int { PATH_LDG = 0, PATH_TMA = 1, PATH_LEAN = 2 };
constexpr int kKeyedLeanRegs = 48;
constexpr int kLeanKeyedBlock = 512, kLeanKeyedIpt = 2;   // its one compiled shape

// Threads launched per CTA: TMA kernels add one producer warp.
inline int launch_threads(const KernelEntry& e) { return e.block + (e.path == PATH_TMA ? 32 : 0); }

// Provided by the kernel translation units.
extern const void* fold_kernel_fn();
extern const void* map_kernel_fn(int kind, int aligned);
extern int map_kernel_block();
extern int map_kernel_ipt();
extern const void* tree_add_kernel_fn(int f32, int aligned, uint32_t k);
extern const void* large_keyed_kernel_fn(int aligned);
extern const void* large_keyed_finish_fn();
extern const void* large_scale_fn();
extern const void* large_repair_zero_fn();
extern const void* doorbell_kernel_fn(int block, int ipt);

}  // namespace scl
