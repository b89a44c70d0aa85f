// radix.h -- the bucket-partitioned keyed reduce for large key spaces
// (WordCount-size vocabularies, Sec. 3.2.3): geometry and kernel arguments,
// shared by the kernels (kernels_radix.cuh) and the host runtime.
//
// Keys are grouped by bucket b = key / kMaxKeys, so that every bucket's keys
// fit the kMaxKeys-entry shared-memory table of one CTA:
//   1. k_radix_hist: each chunk of the partition counts its pairs per bucket
//      (hist[b][c]); keys outside [0, num_keys) set the range flag and are
//      dropped.
//   2. k_radix_scan: each bucket's row of chunk counts becomes exclusive
//      offsets within the bucket (one warp per row); the last CTA turns the
//      bucket totals into bucket starts (bstart[0..nb], bstart[nb] = pairs
//      kept).
//   3. k_radix_scatter: each chunk writes its pairs to its range of every
//      bucket, bstart[b] + hist[b][c] onwards, as {key % kMaxKeys, value}.
//      Up to kRadixStagedMaxBuckets buckets a tile is first grouped by bucket
//      in shared memory so that runs go out as contiguous stores; with more
//      buckets a tile holds about one pair per bucket and pairs go straight
//      to their slots.
//   4. k_radix_reduce: the kept pairs are split evenly over a persistent
//      grid; a CTA accumulates each bucket segment of its share in the shared
//      table and writes it out (plain stores when it holds the whole bucket,
//      global atomics otherwise).
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
constexpr uint32_t kRadixBadPlace = 2u;                  // flag bit: pass 2 saw other counts
constexpr uint32_t kRadixScanBlock = 256;                // 8 bucket rows per CTA
constexpr uint32_t kRadixStagedMaxBuckets = 512;

struct RadixGeometry {
    uint32_t nb = 0;        // buckets: ceil(num_keys / kMaxKeys)
    uint32_t chunk = 0;     // pairs per chunk (a multiple of kRadixChunkAlign)
    uint32_t nchunks = 0;   // ceil(n / chunk)
};

// About two chunks per resident CTA of the scatter kernel (`slots`), each a
// whole number of pass-1 tiles.
__host__ __device__ inline RadixGeometry radix_geometry(uint64_t n, uint32_t num_keys,
                                                        uint32_t slots) {
    RadixGeometry g;
    g.nb = (num_keys + kMaxKeys - 1) / kMaxKeys;
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
    uint64_t bk = 0, hist = 0, tot = 0, bstart = 0, total = 0;
};

__host__ __device__ inline uint64_t radix_up256(uint64_t x) { return (x + 255) / 256 * 256; }

__host__ __device__ inline RadixLayout radix_layout(uint64_t n, const RadixGeometry& g) {
    RadixLayout l;
    l.bk = 0;
    l.hist = radix_up256(n * 8);
    l.tot = l.hist + radix_up256((uint64_t)g.nb * g.nchunks * 4);
    l.bstart = l.tot + radix_up256((uint64_t)g.nb * 4);
    l.total = l.bstart + radix_up256(((uint64_t)g.nb + 1) * 4);
    return l;
}

// Dynamic shared memory of the scatter kernel.  Staged: the tile, then
// count / tile offset / shift / cursor words per bucket, then one word per
// warp and the tile total.  Unstaged: a cursor per bucket.
__host__ __device__ inline bool radix_staged(uint32_t nb) { return nb <= kRadixStagedMaxBuckets; }

__host__ __device__ inline uint32_t radix_scatter_smem(uint32_t nb) {
    return radix_staged(nb) ? kRadixTile * 8 + 4 * nb * 4 + (kRadixBlock / 32) * 4 + 16
                            : nb * 4 + 16;
}

struct RadixArgs {
    const char* keys;         // int32 keys, 16-byte aligned
    const char* vals;         // float values, 16-byte aligned
    uint64_t n;               // pairs in the partition (< 2^31)
    uint32_t num_keys;
    uint32_t nb;
    uint32_t chunk;
    uint32_t nchunks;
    uint32_t* hist;           // [nb][nchunks]: counts, then offsets within the bucket
    uint32_t* tot;            // [nb] pairs per bucket
    uint32_t* bstart;         // [nb + 1] bucket starts in bk
    uint32_t* bk;             // [2n] pairs {key % kMaxKeys, value bits}, grouped by bucket
    uint32_t* counts;         // [num_keys], zeroed before pass 4
    double* sums64;           // [num_keys], zeroed before pass 4
    uint32_t* ticket;         // zero between launches (scan's last CTA)
    uint32_t* bad;            // kRadixBadKey | kRadixBadPlace, zeroed before pass 1
};

// The kernels (kern_radix.cu).
const void* radix_hist_fn();
const void* radix_scan_fn();
const void* radix_scatter_fn(bool staged);
const void* radix_reduce_fn();

}  // namespace scl
