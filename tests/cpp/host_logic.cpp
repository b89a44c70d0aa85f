// host_logic.cpp -- checks of the library's host-side geometry and
// allocation logic, compiled with plain g++ (no GPU):
//   * streaming segments cover a partition exactly, 1..4 chunks each;
//   * single-task keyed pieces cover [0, n) in 64-pair-aligned cuts;
//   * the batch planner's keyed pieces cover every keyed task exactly once,
//     in task order with non-decreasing CTAs, small tasks whole, no short end
//     fragments, CTAs in range;
//   * the range allocator against a reference bitmap under random use;
//   * the bucket-partitioned large-key reduce: its geometry and table layout,
//     and, replaying the four passes' offset arithmetic on random keys, that
//     every partitioned pair is written once inside its bucket and read once
//     by the reduce's cost shares (hot ids counted apart), with no index
//     outside the tables and no share far above its cost;
//   * the scatter's TMA form: every bulk copy it issues is waited on exactly
//     once, in order, with never two outstanding.
// Prints "ok" and exits 0, or names the first failed check and exits 1.
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <random>
#include <vector>

#include "internal.h"
#include "plan_keyed.h"
#include "radix.h"
#include "range_alloc.h"

using namespace scl;

static int g_fail = 0;
#define CHECK(cond, ...)                                   \
    do {                                                   \
        if (!(cond)) {                                     \
            fprintf(stderr, "FAIL %s:%d: ", __FILE__, __LINE__); \
            fprintf(stderr, __VA_ARGS__);                  \
            fprintf(stderr, "\n");                         \
            g_fail = 1;                                    \
            return;                                        \
        }                                                  \
    } while (0)

static void check_stream_segments() {
    const uint32_t chunks[] = {256 * 2 * 4, 256 * 8 * 4, 512 * 8 * 4};
    std::mt19937_64 rng(1);
    for (uint32_t chunk : chunks) {
        for (int it = 0; it < 20000; ++it) {
            uint64_t n = it < 100 ? (uint64_t)it : rng() % (1ull << (rng() % 36));
            const uint32_t se = stream_seg_elems(n, chunk);
            const uint32_t ns = stream_nseg(n, se);
            CHECK(se % chunk == 0 && se >= chunk && se <= kMaxSegChunks * chunk, "seg %u n %llu", se,
                  (unsigned long long)n);
            CHECK(ns >= 1, "nseg 0");
            CHECK((uint64_t)(ns - 1) * se < n || (n == 0 && ns == 1), "last segment empty n %llu",
                  (unsigned long long)n);
            CHECK((uint64_t)ns * se >= n, "segments short n %llu", (unsigned long long)n);
            // the length depends only on n and the chunk: more elements never
            // give shorter segments
            CHECK(stream_seg_elems(n + 1, chunk) >= se, "not monotone at %llu", (unsigned long long)n);
        }
    }
}

static void check_keyed_single() {
    std::mt19937_64 rng(2);
    for (int it = 0; it < 5000; ++it) {
        const uint64_t n = it < 50 ? (uint64_t)it * 17 : rng() % (1ull << (rng() % 34));
        const uint32_t grid = 1 + (uint32_t)(rng() % 2000);
        const uint32_t G = keyed_single_pieces(n, grid);
        CHECK(G >= 1 && G <= grid, "G %u", G);
        uint64_t prev = 0;
        for (uint32_t c = 0; c < G; ++c) {
            const uint64_t b = keyed_single_bound(n, c, G), e = keyed_single_bound(n, c + 1, G);
            CHECK(b == prev && b <= e, "gap or overlap at piece %u", c);
            CHECK(c == 0 || b % kKeyedPieceAlign == 0, "unaligned cut");
            prev = e;
        }
        CHECK(prev == n, "pieces end at %llu of %llu", (unsigned long long)prev,
              (unsigned long long)n);
    }
}

static void check_keyed_plan() {
    std::mt19937_64 rng(3);
    std::lognormal_distribution<double> ln(std::log(16384.0), 1.5);
    for (int it = 0; it < 400; ++it) {
        const uint32_t ntasks = 1 + (uint32_t)(rng() % 3000);
        std::vector<std::pair<uint32_t, uint64_t>> keyed;
        for (uint32_t i = 0; i < ntasks; ++i) {
            uint64_t n = (uint64_t)std::min(ln(rng), 8388608.0);
            if (rng() % 50 == 0) n = rng() % 300;   // tiny and empty tasks
            keyed.emplace_back(i * 3 + (uint32_t)(rng() % 3), n);
        }
        std::sort(keyed.begin(), keyed.end());
        keyed.erase(std::unique(keyed.begin(), keyed.end(),
                                [](const auto& a, const auto& b) { return a.first == b.first; }),
                    keyed.end());
        const uint32_t Gk = 1 + (uint32_t)(rng() % 1216);
        // the per-piece cost the batch planner charges: the default, and 16 or
        // 32 pair-equivalents per thread of a 256- or 512-thread CTA
        const uint64_t overheads[] = {kKeyedTaskOverhead, 4096, 8192, 16384};
        const uint64_t overhead = overheads[rng() % 4];
        std::vector<KeyedPlanPiece> out;
        plan_keyed_pieces(keyed, Gk, &out, overhead);
        size_t k = 0;
        uint32_t last_cta = 0;
        for (const auto& t : keyed) {
            CHECK(k < out.size() && out[k].task == t.first, "task %u has no piece", t.first);
            uint64_t pos = 0;
            uint32_t slot = 0;
            size_t first = k;
            while (k < out.size() && out[k].task == t.first) {
                const KeyedPlanPiece& p = out[k];
                CHECK(p.e0 == pos && p.e0 <= p.e1, "task %u piece %u: gap or overlap", t.first, slot);
                CHECK(p.slot == slot, "slot order");
                CHECK(p.cta < Gk, "cta %u out of range %u", p.cta, Gk);
                CHECK(p.cta >= last_cta, "CTAs not non-decreasing");
                last_cta = p.cta;
                pos = p.e1;
                ++slot;
                ++k;
            }
            CHECK(pos == t.second, "task %u covered to %llu of %llu", t.first,
                  (unsigned long long)pos, (unsigned long long)t.second);
            const size_t np = k - first;
            CHECK(t.second > kKeyedMinPiece || np == 1, "small task %u split in %zu", t.first, np);
            if (np > 1) {
                CHECK(out[first].e1 - out[first].e0 >= kKeyedMinFragment, "short first piece");
                CHECK(out[k - 1].e1 - out[k - 1].e0 >= kKeyedMinFragment, "short last piece");
            }
        }
        CHECK(k == out.size(), "extra pieces");
    }
}

static void check_range_alloc() {
    std::mt19937_64 rng(4);
    for (int round = 0; round < 50; ++round) {
        const uint32_t cap = 1 + (uint32_t)(rng() % 5000);
        RangeAlloc ra;
        ra.init(cap);
        std::vector<char> used(cap, 0);
        std::vector<std::pair<uint32_t, uint32_t>> live;
        for (int op = 0; op < 4000; ++op) {
            if (live.empty() || rng() % 2) {
                const uint32_t n = 1 + (uint32_t)(rng() % 64);
                uint32_t off = 0;
                // the reference: is there any free run of n?
                bool exists = false;
                for (uint32_t i = 0, run = 0; i < cap && !exists; ++i) {
                    run = used[i] ? 0 : run + 1;
                    exists = run >= n;
                }
                const bool ok = ra.alloc(n, &off);
                CHECK(ok == exists, "alloc(%u) %d but a free run %s", n, (int)ok,
                      exists ? "exists" : "does not exist");
                if (ok) {
                    CHECK(off + n <= cap, "range beyond cap");
                    for (uint32_t i = off; i < off + n; ++i) {
                        CHECK(!used[i], "overlapping ranges at %u", i);
                        used[i] = 1;
                    }
                    live.emplace_back(off, n);
                }
            } else {
                const size_t j = rng() % live.size();
                const auto r = live[j];
                live[j] = live.back();
                live.pop_back();
                ra.release(r.first, r.second);
                for (uint32_t i = r.first; i < r.first + r.second; ++i) used[i] = 0;
            }
        }
        for (const auto& r : live) ra.release(r.first, r.second);
        CHECK(ra.free_ranges() == 1, "free list not coalesced: %zu ranges", ra.free_ranges());
        uint32_t off = 7;
        CHECK(ra.alloc(cap, &off) && off == 0, "whole range not free after releasing all");
    }
}

static void check_radix() {
    std::mt19937_64 rng(5);
    // geometry and layout over a wide range of sizes
    for (int it = 0; it < 20000; ++it) {
        const uint64_t n = kRadixMinPairs + rng() % (kRadixMaxPairs - kRadixMinPairs + 1);
        const uint32_t nk = kMaxKeys + 1 + (uint32_t)(rng() % (kMaxLargeKeys - kMaxKeys));
        const uint32_t slots = 1 + (uint32_t)(rng() % 4096);
        const RadixGeometry g = radix_geometry(n, nk, slots);
        CHECK(g.chunk % kRadixChunkAlign == 0 && g.chunk >= kRadixChunkAlign, "chunk %u", g.chunk);
        CHECK((uint64_t)g.nchunks * g.chunk >= n && (uint64_t)(g.nchunks - 1) * g.chunk < n,
              "chunks do not cover n %llu", (unsigned long long)n);
        CHECK(g.log_t >= kRadixMinLogT && g.log_t <= kRadixMaxLogT, "log_t %u", g.log_t);
        CHECK(g.nb >= 2 && g.nb <= kRadixMaxBuckets && ((uint64_t)g.nb << g.log_t) >= nk &&
                  ((uint64_t)(g.nb - 1) << g.log_t) < nk,
              "buckets %u of 2^%u for %u keys", g.nb, g.log_t, nk);
        CHECK(g.log_t == kRadixMinLogT ||
                  (((uint64_t)nk + (1u << (g.log_t - 1)) - 1) >> (g.log_t - 1)) >
                      kRadixPreferredBuckets,
              "buckets wider than needed: 2^%u for %u keys", g.log_t, nk);
        CHECK(g.nb <= kRadixPreferredBuckets || g.log_t == kRadixMaxLogT,
              "%u buckets of 2^%u", g.nb, g.log_t);
        CHECK(radix_reduce_smem(g.log_t) <= 227 * 1024, "reduce shared memory %u",
              radix_reduce_smem(g.log_t));
        CHECK(g.nchunks <= 2ull * slots + 1 || g.chunk == kRadixChunkAlign, "too many chunks");
        const RadixLayout l = radix_layout(n, g);
        CHECK(l.hist >= n * 8 + 8 || (n % 2 == 0 && l.hist >= n * 8),
              "no room for the last 16-byte load");
        CHECK(l.hist % 256 == 0 && l.tot % 256 == 0 && l.bstart % 256 == 0, "unaligned table");
        CHECK(l.tot >= l.hist + (uint64_t)g.nb * g.nchunks * 4 && l.bstart >= l.tot + g.nb * 4ull &&
                  l.total >= l.bstart + (g.nb + 1ull) * 4,
              "tables overlap");
        for (int hot = 0; hot < 2; ++hot)
            CHECK(radix_scatter_smem(g.nb, hot != 0) <= 227 * 1024,
                  "scatter shared memory %u", radix_scatter_smem(g.nb, hot != 0));
    }
    // replay of the passes' offsets (scaled-down sizes, same formulas)
    for (int it = 0; it < 48; ++it) {
        const uint64_t n = kRadixMinPairs + rng() % (3 * kRadixMinPairs);
        const uint32_t shape = it % 4;
        const uint32_t space = (it / 4) % 4;
        const uint32_t nk = space == 0 ? kMaxKeys + 1 + (uint32_t)(rng() % 10)
                            : space == 1 ? kMaxLargeKeys - (uint32_t)(rng() % 5000)   // 2^14 ids
                            : space == 2 ? (1u << 22) + 1 + (uint32_t)(rng() % 1000)  // 2^13 ids
                                         : kMaxKeys * (2 + (uint32_t)(rng() % 300)) - (uint32_t)(rng() % 7);
        const uint32_t slots = 64 + (uint32_t)(rng() % 800), grid4 = 64 + (uint32_t)(rng() % 800);
        const RadixGeometry g = radix_geometry(n, nk, slots);
        std::vector<uint32_t> keys(n);
        for (auto& k : keys) {
            k = shape == 1 ? (uint32_t)(rng() % 3)                  // one bucket
                : shape == 2 ? nk - 1 - (uint32_t)(rng() % 2)      // the last bucket
                             : (uint32_t)(rng() % (nk + nk / 50)); // some out of range
        }
        if (shape == 3) std::sort(keys.begin(), keys.end());
        // pass 1 (row nb: hot ids) + scan, and the scan's choice of form
        std::vector<uint32_t> hist((size_t)(g.nb + 1) * g.nchunks, 0), tot(g.nb + 1, 0),
            bstart(g.nb + 1, 0);
        for (uint32_t c = 0; c < g.nchunks; ++c)
            for (uint64_t i = (uint64_t)c * g.chunk; i < std::min<uint64_t>(n, (uint64_t)(c + 1) * g.chunk); ++i)
                if (keys[i] < nk)
                    ++hist[(size_t)(keys[i] < kRadixHotIds ? g.nb : keys[i] >> g.log_t) * g.nchunks + c];
        for (uint32_t b = 0; b <= g.nb; ++b) {
            uint32_t run = 0;
            for (uint32_t c = 0; c < g.nchunks; ++c) {
                const uint32_t v = hist[(size_t)b * g.nchunks + c];
                hist[(size_t)b * g.nchunks + c] = run;
                run += v;
            }
            tot[b] = run;
        }
        uint64_t kept = 0;
        for (uint32_t b = 0; b < g.nb; ++b) kept += tot[b];
        const bool hot_on = tot[g.nb] != 0 && (uint64_t)tot[g.nb] * 8 >= kept + tot[g.nb];
        if (it == 5) CHECK(hot_on, "one-bucket keys 0..2 should bypass the partition");
        for (uint32_t b = 0; b < g.nb; ++b)
            bstart[b + 1] = bstart[b] + tot[b] + (b == 0 && !hot_on ? tot[g.nb] : 0u);
        const uint64_t nv = bstart[g.nb];
        // pass 3: each chunk's tiles advance per-bucket cursors
        std::vector<uint32_t> owner(nv, UINT32_MAX);
        for (uint32_t c = 0; c < g.nchunks; ++c) {
            std::vector<uint32_t> cur(g.nb);
            for (uint32_t b = 0; b < g.nb; ++b)
                cur[b] = bstart[b] + hist[(size_t)b * g.nchunks + c] +
                         (b == 0 && !hot_on ? hist[(size_t)g.nb * g.nchunks + c] : 0u);
            const uint64_t e0 = std::min<uint64_t>(n, (uint64_t)(c + 1) * g.chunk);
            for (uint64_t t0 = (uint64_t)c * g.chunk; t0 < e0; t0 += kRadixTile) {
                uint32_t tn = 0;
                for (uint64_t i = t0; i < std::min<uint64_t>(e0, t0 + kRadixTile); ++i) {
                    if (keys[i] >= nk || (hot_on && keys[i] < kRadixHotIds)) continue;   // hot table
                    ++tn;
                    const uint32_t b = keys[i] >> g.log_t;
                    const uint64_t pos = cur[b]++;
                    CHECK(pos >= bstart[b] && pos < bstart[b + 1], "pair %llu outside its bucket",
                          (unsigned long long)i);
                    CHECK(owner[pos] == UINT32_MAX, "position %llu written twice",
                          (unsigned long long)pos);
                    owner[pos] = keys[i];
                }
                CHECK(tn <= kRadixTile, "tile overflow");
            }
        }
        for (uint64_t q = 0; q < nv; ++q) CHECK(owner[q] != UINT32_MAX, "position %llu unwritten",
                                                (unsigned long long)q);
        // cost starts as the scan's last CTA forms them
        const uint32_t fixed = radix_bucket_cost(g.log_t);
        std::vector<uint64_t> bcost(g.nb + 1, 0);
        for (uint32_t b = 0, ne = 0; b <= g.nb; ++b) {
            bcost[b] = bstart[b] + (uint64_t)ne * fixed;
            if (b < g.nb && bstart[b + 1] > bstart[b]) ++ne;
        }
        CHECK(bcost[g.nb] < (1ull << 32), "cost overflows 32 bits");
        // pass 4: even shares of cost, bucket search, pieces of at most kLargePiece
        std::vector<uint32_t> cnt(nk, 0), seen(nv, 0);
        if (hot_on)
            for (uint32_t k : keys)   // the scatter's hot table
                if (k < kRadixHotIds) ++cnt[k];
        const uint64_t ctot = bcost[g.nb];
        uint64_t most = 0;
        for (uint32_t blk = 0; blk < grid4; ++blk) {
            const uint64_t clo = ctot * blk / grid4, chi = ctot * (blk + 1) / grid4;
            if (clo >= chi) continue;
            uint32_t bl = 0, bh = g.nb - 1;
            while (bl < bh) {
                const uint32_t mid = (bl + bh + 1) / 2;
                if (bcost[mid] <= clo) bl = mid;
                else bh = mid - 1;
            }
            CHECK(bcost[bl] <= clo, "search overshot cost %llu", (unsigned long long)clo);
            uint64_t work = 0;
            for (uint32_t b = bl; b < g.nb && bcost[b] < chi; ++b) {
                const uint64_t nbk = bstart[b + 1] - bstart[b];
                if (!nbk) continue;
                const uint64_t first = bcost[b] + fixed;
                const uint64_t j0 = clo > first ? std::min(clo - first, nbk) : 0;
                const uint64_t j1 = chi > first ? std::min(chi - first, nbk) : 0;
                if (j0 >= j1) continue;
                work += j1 - j0 + fixed;
                const uint64_t s = bstart[b] + j0, se = bstart[b] + j1;
                const uint32_t T = 1u << g.log_t;
                const uint32_t hot = std::min(T, nk - b * T);
                for (uint64_t p0 = s; p0 < se; p0 += kLargePiece) {
                    const uint64_t p1 = std::min(p0 + kLargePiece, se);
                    // 16-byte loads of two pairs: words [4 q, 4 q + 4)
                    const uint64_t q0 = p0 >> 1, q1 = (p1 + 1) >> 1;
                    CHECK((q1 - 1) * 16 + 16 <= radix_layout(n, g).hist, "load past bk");
                    for (uint64_t i = p0; i < p1; ++i) {
                        const uint32_t k = owner[i];
                        CHECK((k >> g.log_t) == b && (k & (T - 1)) < hot, "pair %llu in bucket %u",
                              (unsigned long long)i, b);
                        ++seen[i];
                        ++cnt[k];
                    }
                    (void)q0;
                }
            }
            most = std::max(most, work);
        }
        // no CTA gets much more than its share of the cost (one bucket's table at most)
        CHECK(most <= ctot / grid4 + 2ull * fixed + 2, "CTA work %llu, share %llu",
              (unsigned long long)most, (unsigned long long)(ctot / grid4));
        for (uint64_t q = 0; q < nv; ++q) CHECK(seen[q] == 1, "pair %llu reduced %u times",
                                                (unsigned long long)q, seen[q]);
        std::vector<uint32_t> ref(nk, 0);
        for (uint32_t k : keys)
            if (k < nk) ++ref[k];
        CHECK(cnt == ref, "counts differ");
    }
}

// The large-key scatter's TMA form (plain form): one input buffer, one
// mbarrier.  Replays a CTA's issue / wait sequence over its chunks: the first
// whole tile of a chunk is issued at the chunk's start, the next whole tile
// right after a tile's ranks; a whole tile waits on the barrier, a ragged
// last tile loads by registers.  Every issued copy must be waited on exactly
// once, in order (phase parity alternating), and no copy may be issued while
// another is outstanding (the buffer is single).
static void check_radix_tma_protocol() {
    std::mt19937_64 rng(6);
    for (int it = 0; it < 20000; ++it) {
        const uint32_t nchunks = 1 + (uint32_t)(rng() % 5);
        uint32_t issued = 0, waited = 0, phase = 0;
        bool outstanding = false;
        for (uint32_t c = 0; c < nchunks; ++c) {
            const uint32_t len = it < 64 ? (uint32_t)(it * 1024)
                                         : (uint32_t)(rng() % (12 * kRadixTile + 3));
            if (kRadixTile <= len) {   // chunk start
                CHECK(!outstanding, "issue while a copy is outstanding (chunk start)");
                outstanding = true;
                ++issued;
            }
            for (uint32_t t0 = 0; t0 < len; t0 += kRadixTile) {
                if (t0 + kRadixTile <= len) {   // whole tile: wait on the barrier
                    CHECK(outstanding, "wait with no copy issued (len %u, t0 %u)", len, t0);
                    outstanding = false;
                    ++waited;
                    phase ^= 1u;
                }
                // after the ranks: the next whole tile
                if (t0 + 2 * kRadixTile <= len) {
                    CHECK(!outstanding, "issue while a copy is outstanding (len %u)", len);
                    outstanding = true;
                    ++issued;
                }
            }
        }
        CHECK(!outstanding && issued == waited, "copies issued %u, waited %u", issued, waited);
        CHECK(phase == (waited & 1u), "phase parity");
    }
}

int main() {
    check_stream_segments();
    if (!g_fail) check_keyed_single();
    if (!g_fail) check_keyed_plan();
    if (!g_fail) check_range_alloc();
    if (!g_fail) check_radix();
    if (!g_fail) check_radix_tma_protocol();
    if (g_fail) return 1;
    printf("ok\n");
    return 0;
}
