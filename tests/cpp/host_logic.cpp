// host_logic.cpp -- checks of the library's host-side geometry and
// allocation logic, compiled with plain g++ (no GPU):
//   * streaming segments cover a partition exactly, 1..4 chunks each;
//   * single-task keyed pieces cover [0, n) in 64-pair-aligned cuts;
//   * the batch planner's keyed pieces cover every keyed task exactly once,
//     in task order with non-decreasing CTAs, small tasks whole, no short end
//     fragments, CTAs in range;
//   * the range allocator against a reference bitmap under random use.
// Prints "ok" and exits 0, or names the first failed check and exits 1.
#include <stdio.h>
#include <stdlib.h>

#include <random>
#include <vector>

#include "internal.h"
#include "plan_keyed.h"
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
        std::vector<KeyedPlanPiece> out;
        plan_keyed_pieces(keyed, Gk, &out);
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

int main() {
    check_stream_segments();
    if (!g_fail) check_keyed_single();
    if (!g_fail) check_keyed_plan();
    if (!g_fail) check_range_alloc();
    if (g_fail) return 1;
    printf("ok\n");
    return 0;
}
