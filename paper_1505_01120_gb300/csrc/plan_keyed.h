// plan_keyed.h -- the keyed part of the batch planner, as a pure function of
// the keyed tasks' lengths and the number of CTAs that take keyed pieces
// (kept free of CUDA so the host tests can run it).
#pragma once

#include <stdint.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "internal.h"

namespace scl {

struct KeyedPlanPiece {
    uint64_t e0, e1;   // pairs [e0, e1) of the task
    uint32_t task;     // the task's index in the batch
    uint32_t slot;     // piece number within the task
    uint32_t cta;      // the CTA that runs it
};

// Keyed work of a batch over Gk CTAs (Gk >= 1).  `keyed` lists the keyed
// tasks in batch order as (task index, pairs).  Each task costs
// pairs + overhead; CTA c takes the even share [W*c/Gk, W*(c+1)/Gk)
// of the total W, so a task is cut where the shares meet, at multiples of
// kKeyedPieceAlign pairs.  A task of at most kKeyedMinPiece pairs stays whole,
// on the CTA holding most of it; in a larger task, end pieces shorter than
// kKeyedMinFragment join their neighbour.  Every task gets at least one
// (possibly empty) piece; pieces come out in task order with non-decreasing
// CTAs, and together cover each task's [0, pairs) exactly once.
inline void plan_keyed_pieces(const std::vector<std::pair<uint32_t, uint64_t>>& keyed,
                              uint32_t Gk, std::vector<KeyedPlanPiece>* out,
                              uint64_t overhead = kKeyedTaskOverhead) {
    out->clear();
    uint64_t W = 0;
    for (const auto& k : keyed) W += k.second + overhead;
    if (keyed.empty() || Gk == 0) return;
    auto R = [&](uint64_t cta) -> uint64_t { return (uint64_t)((unsigned __int128)cta * W / Gk); };
    struct Frag {
        uint64_t e0, e1;
        uint32_t cta;
    };
    std::vector<Frag> frag;
    uint64_t A = 0;
    for (const auto& k : keyed) {
        const uint64_t n = k.second, cost = n + overhead, B = A + cost;
        uint32_t c0 = (uint32_t)((unsigned __int128)A * Gk / W);
        while (c0 + 1 < Gk && R(c0 + 1) <= A) ++c0;
        while (c0 > 0 && R(c0) > A) --c0;
        auto emap = [&](uint64_t w) -> uint64_t {
            if (w >= B) return n;
            const uint64_t e = (uint64_t)((unsigned __int128)(w - A) * n / cost);
            return e / kKeyedPieceAlign * kKeyedPieceAlign;
        };
        // the task's share of each CTA it spans
        frag.clear();
        for (uint32_t cta = c0; cta < Gk && R(cta) < B; ++cta) {
            const uint64_t lo = std::max(A, R(cta));
            const uint64_t hi = std::min(B, cta + 1 == Gk ? W : R(cta + 1));
            if (lo >= hi) continue;
            const uint64_t e0 = emap(lo), e1 = emap(hi);
            if (e0 >= e1) continue;
            frag.push_back(Frag{e0, e1, cta});
        }
        if (frag.empty()) frag.push_back(Frag{0, n, c0});   // empty or tiny task
        if (frag.size() > 1 && n <= kKeyedMinPiece) {
            const Frag* big = &frag[0];
            for (const Frag& f : frag)
                if (f.e1 - f.e0 > big->e1 - big->e0) big = &f;
            frag = {Frag{0, n, big->cta}};
        }
        while (frag.size() > 1 && frag.front().e1 - frag.front().e0 < kKeyedMinFragment) {
            frag[1].e0 = frag.front().e0;
            frag.erase(frag.begin());
        }
        while (frag.size() > 1 && frag.back().e1 - frag.back().e0 < kKeyedMinFragment) {
            frag[frag.size() - 2].e1 = frag.back().e1;
            frag.pop_back();
        }
        uint32_t slot = 0;
        for (const Frag& f : frag) out->push_back(KeyedPlanPiece{f.e0, f.e1, k.first, slot++, f.cta});
        A = B;
    }
}

}  // namespace scl
