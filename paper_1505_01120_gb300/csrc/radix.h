// radix.h -- the bucket-partitioned keyed reduce for large key spaces
// (WordCount-size vocabularies, Sec. 3.2.3): geometry and kernel arguments,
// shared by the kernels (kernels_radix.cuh) and the host runtime.
//
// Keys are grouped by bucket b = key >> log_t, so that every bucket's 2^log_t
// ids fit the shared-memory table of one CTA.  log_t is the smallest of 12,
// 13, 14 (4096 to 16384 ids) that keeps the buckets within
// kRadixPreferredBuckets, so that a tile of the scatter writes runs of
// several pairs per bucket (on GB300 the scatter took 288 / 401 / 600 us for
// 64 Mi pairs into 256 / 512 / 1024 buckets, more than a wider table costs
// the reduce; the whole call over 2^20 uniform keys took 506 / 481 / 486 us
// preferring 256 / 128 / 64 buckets); above 2^21 keys, 16384-id buckets (up
// to 1024).
// Ids below kRadixHotIds -- the frequent words when a vocabulary is numbered
// by frequency -- are counted apart by the histogram; when they hold at
// least 1/8 of the pairs they are not partitioned: the scatter counts them in
// its own shared table as it reads them, so under skew most pairs are read
// once.  Both scatter forms are launched and the scan's choice runs.
//   1. k_radix_hist: each chunk of the partition counts its other pairs per
//      bucket (hist[b][c]); keys outside [0, num_keys) set the range flag
//      and are dropped.
//   2. k_radix_scan: each bucket's row of chunk counts becomes exclusive
//      offsets within the bucket (one warp per row); the last CTA turns the
//      bucket totals into bucket starts (bstart[0..nb], bstart[nb] = pairs
//      kept) and cost starts (bcost[0..nb]).
//   3. k_radix_scatter: each chunk writes its pairs to its range of every
//      bucket, bstart[b] + hist[b][c] onwards, as {key % 2^log_t, value}; a
//      tile is first grouped by bucket in shared memory so that runs go out
//      as contiguous stores.  Pairs of hot ids go to the CTA's hot table,
//      flushed to the outputs with global atomics every kLargePiece pairs.
//   4. k_radix_reduce: the kept pairs are split over a persistent grid in
//      even shares of cost, a bucket costing its pairs plus a fixed
//      radix_bucket_cost() for its table's flush (so the many small buckets
//      of a skewed key set do not land on a few CTAs); a CTA accumulates each
//      bucket segment of its share in the shared table and writes it out
//      (plain stores when it holds the whole bucket, global atomics
//      otherwise).
// A finishing pass (the one of the direct path) rounds the fp64 sums to fp32
// and forms the totals.
#pragma once

#include <stdint.h>

#include "internal.h"

namespace scl {

constexpr uint32_t kRadixBlock = 512;
constexpr uint32_t kRadixHistTile = kRadixBlock * 16;    // keys per pass-1 tile
constexpr uint32_t kRadixTile = kRadixBlock * 8;         // pairs per pass-2 tile
constexpr uint32_t kRadixChunkAlign = kRadixHistTile;    // chunk lengths, in pairs
constexpr uint64_t kRadixMinPairs = 1u << 20;            // smaller partitions: direct path
constexpr uint64_t kRadixMaxPairs = (1ull << 31) - 1;    // offsets are uint32
constexpr uint32_t kRadixBadKey = 1u;                    // flag bit: key out of range
constexpr uint32_t kRadixBadPlace = 2u;                  // flag bit: pass 3 saw other counts
constexpr uint32_t kRadixBadWait = 4u;                   // flag bit: a bounded wait ran out
constexpr uint32_t kRadixScanBlock = 256;                // 8 bucket rows per CTA
constexpr uint32_t kRadixMaxBuckets = 2 * kRadixBlock;   // two per scatter thread
constexpr uint32_t kRadixPreferredBuckets = 128;         // runs of 32 pairs per tile
constexpr uint32_t kRadixHotIds = 1024;                  // ids kept out of the partition
constexpr uint32_t kRadixHotFlushTiles = 32;             // kLargePiece pairs
constexpr uint32_t kRadixMinLogT = 12;                   // 4096 ids per bucket
constexpr uint32_t kRadixMaxLogT = 14;                   // 16384: 2^24 keys in 1024 buckets

struct RadixGeometry {
    uint32_t log_t = 0;     // ids per bucket: 2^log_t
    uint32_t nb = 0;        // buckets: ceil(num_keys / 2^log_t)
    uint32_t chunk = 0;     // pairs per chunk (a multiple of kRadixChunkAlign)
    uint32_t nchunks = 0;   // ceil(n / chunk)
};

// The narrowest buckets that keep their number within kRadixPreferredBuckets
// (at most kRadixMaxLogT); about two chunks per resident CTA of the scatter
// kernel (`slots`), each a whole number of pass-1 tiles.
__host__ __device__ inline RadixGeometry radix_geometry(uint64_t n, uint32_t num_keys,
                                                        uint32_t slots) {
    RadixGeometry g;
    g.log_t = kRadixMinLogT;
    while (g.log_t < kRadixMaxLogT &&
           ((uint64_t)num_keys + (1u << g.log_t) - 1) >> g.log_t > kRadixPreferredBuckets)
        ++g.log_t;
    g.nb = (uint32_t)(((uint64_t)num_keys + (1u << g.log_t) - 1) >> g.log_t);
    const uint64_t want = 2ull * (slots ? slots : 1);
    uint64_t chunk = (n + want - 1) / want;
    chunk = (chunk + kRadixChunkAlign - 1) / kRadixChunkAlign * kRadixChunkAlign;
    if (chunk == 0) chunk = kRadixChunkAlign;
    g.chunk = (uint32_t)chunk;
    g.nchunks = (uint32_t)((n + chunk - 1) / chunk);
    return g;
}

// Bytes of each temporary table, in the order they are laid out (each start
// rounded up to 256 bytes).  bk's padding keeps the 16-byte loads of pass 4,
// two pairs each, inside the block when n is odd.
struct RadixLayout {
    uint64_t bk = 0, hist = 0, tot = 0, bstart = 0, bcost = 0, mode = 0, total = 0;
};

// Cost of a non-empty bucket's table work (flush, barriers, its loads'
// latency) in pairs: as many as it has ids.  Measured on GB300 with Zipf(1.2)
// keys over 2^24 ids (1023 buckets of ~650 pairs beside one of 60 Mi): a
// quarter of the ids left the last CTAs with the small buckets (972 us), the
// full count balanced them (771 us), twice it over-corrected (820 us).
__host__ __device__ constexpr uint32_t radix_bucket_cost(uint32_t log_t) { return 1u << log_t; }

__host__ __device__ inline uint64_t radix_up256(uint64_t x) { return (x + 255) / 256 * 256; }

__host__ __device__ inline RadixLayout radix_layout(uint64_t n, const RadixGeometry& g) {
    RadixLayout l;
    l.bk = 0;
    l.hist = radix_up256(n * 8);
    l.tot = l.hist + radix_up256(((uint64_t)g.nb + 1) * g.nchunks * 4);   // + the hot row
    l.bstart = l.tot + radix_up256(((uint64_t)g.nb + 1) * 4);
    l.bcost = l.bstart + radix_up256(((uint64_t)g.nb + 1) * 4);
    l.mode = l.bcost + radix_up256(((uint64_t)g.nb + 1) * 4);
    l.total = l.mode + 256;
    return l;
}

// Dynamic shared memory of the scatter kernel, in words: (TMA) the input
// tile -- keys, values -- and its mbarrier, the stage tile, (HOT) the hot
// table -- counts, fp32 sums, head copies --, then count / tile offset /
// shift / cursor words per bucket, then one word per warp and the tile total.
__host__ __device__ constexpr uint32_t radix_scatter_in_words(bool tma) {
    return tma ? 2 * kRadixTile + 4 : 0u;
}
__host__ __device__ constexpr uint32_t radix_scatter_hot_words(bool hot) {
    return hot ? 2 * kRadixHotIds + kKeyedHeadWords(kRadixBlock) : 0u;
}
// Whether a form stages its input with TMA: the plain one.  (Measured on
// GB300, 64 Mi pairs: the plain form 5-6% faster with it at 3 CTAs per SM;
// the hot-id form, at 2 CTAs per SM with it, 2-3% slower.)
__host__ __device__ constexpr bool radix_scatter_tma(bool hot) { return !hot; }
__host__ __device__ constexpr uint32_t radix_scatter_smem(uint32_t nb, bool hot) {
    return (radix_scatter_in_words(radix_scatter_tma(hot)) + 2 * kRadixTile +
            radix_scatter_hot_words(hot) + 4 * nb + kRadixBlock / 32 + 4) * 4;
}

// Dynamic shared memory of the histogram kernel: a count per bucket and the
// hot row.
__host__ __device__ inline uint32_t radix_hist_smem(uint32_t nb) { return (nb + 1) * 4; }

// The reduce kernel per bucket width: threads per CTA and dynamic shared
// memory (count and fp32 sum per id, then the head copies).
// (8192 ids: 2 CTAs of 1024 threads per SM beat 3 of 512 by 3% on GB300.)
__host__ __device__ constexpr uint32_t radix_reduce_block(uint32_t log_t) {
    return log_t >= 13 ? 1024u : 512u;
}
__host__ __device__ constexpr uint32_t radix_reduce_smem(uint32_t log_t) {
    return ((2u << log_t) + kKeyedHeadWords(radix_reduce_block(log_t))) * 4;
}

// Limits the kernels rely on: cost starts fit 32 bits at the largest
// partition and bucket count, and every form's shared memory fits a CTA.
static_assert((uint64_t)kRadixMaxPairs +
                      (uint64_t)kRadixMaxBuckets * radix_bucket_cost(kRadixMaxLogT) <
                  (1ull << 32),
              "cost starts overflow");
static_assert(radix_scatter_smem(kRadixMaxBuckets, false) <= 227 * 1024 &&
                  radix_scatter_smem(kRadixMaxBuckets, true) <= 227 * 1024,
              "scatter shared memory");
static_assert(radix_reduce_smem(kRadixMaxLogT) <= 227 * 1024, "reduce shared memory");

struct RadixArgs {
    const char* keys;         // int32 keys, 16-byte aligned
    const char* vals;         // float values, 16-byte aligned
    uint64_t n;               // pairs in the partition (< 2^31)
    uint32_t num_keys;
    uint32_t nb;
    uint32_t chunk;
    uint32_t nchunks;
    uint32_t log_t;
    uint32_t fixed;           // radix_bucket_cost(log_t)
    uint32_t* hist;           // [nb + 1][nchunks]: counts, then offsets within the row
                              // (row nb: pairs of hot ids)
    uint32_t* tot;            // [nb + 1] pairs per row
    uint32_t* bstart;         // [nb + 1] bucket starts in bk
    uint32_t* bcost;          // [nb + 1] bucket starts in cost (< 2^32: n + nb * fixed)
    uint32_t* mode;           // 1: hot ids bypass the partition (set by the scan)
    uint32_t* bk;             // [2n] pairs {key % 2^log_t, value bits}, grouped by bucket
    uint32_t* counts;         // [num_keys], zeroed by pass 1
    double* sums64;           // [num_keys], zeroed by pass 1
    uint32_t* ticket;         // zero between launches (scan's last CTA)
    uint32_t* bad;            // kRadixBadKey | kRadixBadPlace, zeroed before pass 1
};

// The kernels (kern_radix.cu).
const void* radix_hist_fn();
const void* radix_scan_fn();
const void* radix_scatter_fn(uint32_t log_t, bool hot);
const void* radix_reduce_fn(uint32_t log_t);

}  // namespace scl
