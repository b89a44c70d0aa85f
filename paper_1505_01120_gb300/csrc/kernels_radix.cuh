// kernels_radix.cuh -- sm_103a kernels of the bucket-partitioned keyed
// reduce (large key spaces, Sec. 3.2.3); the passes are described in radix.h.
//
// Shared-memory atomics measured on GB300 decide the shapes below: integer
// adds whose result is unused stay fast when many lanes hit one address, so
// the histogram counts with plain atomics; integer adds that return the old
// value, and float adds, serialise on a contended address, so ranks are taken
// per warp group and the hot ids' float sums are spread over private copies.
#pragma once

#include "kernels.cuh"
#include "kernels_tma.cuh"
#include "radix.h"

namespace scl {
namespace dev {

constexpr uint32_t kAllLanes = 0xffffffffu;

constexpr uint32_t kNoBucket = 0xffffffffu;
constexpr int kGroupMin = 4;   // lanes sharing lane 0's bucket before they reserve together

// Rank of this lane's pair within bucket b (cnt[b] before it); b is
// kNoBucket for lanes without a pair.  When at least kGroupMin lanes share
// lane 0's bucket -- under skew, most of the warp -- one atomic reserves
// their slots; every other lane reserves its own.
__device__ __forceinline__ uint32_t warp_rank(uint32_t* cnt, uint32_t b, uint32_t lane) {
    const uint32_t b0 = __shfl_sync(kAllLanes, b, 0);
    const uint32_t peers = __ballot_sync(kAllLanes, b == b0);
    if (b0 != kNoBucket && __popc(peers) >= kGroupMin) {   // warp-uniform
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&cnt[b0], (uint32_t)__popc(peers));
        base = __shfl_sync(kAllLanes, base, 0);
        if ((peers >> lane) & 1u) return base + __popc(peers & ((1u << lane) - 1u));
    }
    return b != kNoBucket ? atomicAdd(&cnt[b], 1u) : 0u;
}

// Loads 4 consecutive words starting at element i of [.., e): one 16-byte
// load when the four are inside, else element loads; `in` gets one bit per
// element that exists.
template <typename I>
__device__ __forceinline__ uint4 radix_load4(const char* base, I i, I e, uint32_t* in) {
    if (i + 4 <= e) {
        *in = 0xfu;
        return ld_stream_v4(base + i * 4);
    }
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    uint32_t m = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (i + q < e) {
            w[q] = ld_stream_b32(base + (i + q) * 4);
            m |= 1u << q;
        }
    *in = m;
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// Pass 1: per chunk, pairs per bucket, pairs of hot ids (below kRadixHotIds)
// counted apart in row nb (bucket-major rows of hist); zeroes the outputs.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_radix_hist(const __grid_constant__ RadixArgs a) {
    extern __shared__ uint32_t hist[];   // [nb + 1]
    const uint32_t rows = a.nb + 1;
    uint32_t bad = 0;
    // the output tables start at zero (read first by pass 3's hot flushes)
    for (uint32_t i = blockIdx.x * BLOCK + threadIdx.x; i < a.num_keys; i += gridDim.x * BLOCK) {
        a.counts[i] = 0u;
        a.sums64[i] = 0.0;
    }
    for (uint32_t c = blockIdx.x; c < a.nchunks; c += gridDim.x) {
        for (uint32_t i = threadIdx.x; i < rows; i += BLOCK) hist[i] = 0u;
        __syncthreads();
        const uint64_t b0 = (uint64_t)c * a.chunk;
        const uint32_t len = (uint32_t)(min(b0 + a.chunk, a.n) - b0);
        const char* kp = a.keys + b0 * 4;
        for (uint32_t t0 = 0; t0 < len; t0 += (uint32_t)BLOCK * 16) {
            uint4 k[4];
            uint32_t in[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                k[j] = radix_load4(kp, t0 + ((uint32_t)j * BLOCK + threadIdx.x) * 4, len, &in[j]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t kk[4] = {k[j].x, k[j].y, k[j].z, k[j].w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (!((in[j] >> q) & 1u)) continue;
                    if (kk[q] >= a.num_keys) bad = kRadixBadKey;
                    else atomicAdd(&hist[kk[q] < kRadixHotIds ? a.nb : kk[q] >> a.log_t], 1u);
                }
            }
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < rows; i += BLOCK)
            a.hist[(size_t)i * a.nchunks + c] = hist[i];
        __syncthreads();   // hist is zeroed again for the next chunk
    }
    if (bad) atomicOr(a.bad, bad);
}

// Exclusive scan of one row by one warp, in place; returns the row total.
__device__ __forceinline__ uint32_t warp_exclusive_scan(uint32_t* row, uint32_t n,
                                                        uint32_t lane) {
    const uint32_t per = (n + 31) / 32;
    const uint32_t i0 = min(lane * per, n), i1 = min(i0 + per, n);
    uint32_t s = 0;
    for (uint32_t i = i0; i < i1; ++i) s += row[i];
    uint32_t x = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kAllLanes, x, d);
        if ((int)lane >= d) x += y;
    }
    const uint32_t total = __shfl_sync(kAllLanes, x, 31);
    uint32_t base = x - s;
    for (uint32_t i = i0; i < i1; ++i) {
        const uint32_t v = row[i];
        row[i] = base;
        base += v;
    }
    return total;
}

// Block-wide exclusive scan of f(i) for i in [0, n), each thread a run of
// consecutive i; calls out(i, prefix) in order and returns the total.  Uses
// wsum[BLOCK / 32] with barriers around it.
template <int BLOCK, typename F, typename O>
__device__ __forceinline__ uint32_t block_scan_runs(uint32_t n, uint32_t* wsum, F f, O out) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t per = (n + BLOCK - 1) / BLOCK;
    const uint32_t i0 = min(threadIdx.x * per, n), i1 = min(i0 + per, n);
    uint32_t s = 0;
    for (uint32_t i = i0; i < i1; ++i) s += f(i);
    uint32_t x = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kAllLanes, x, d);
        if ((int)lane >= d) x += y;
    }
    __syncthreads();
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t total = 0, before = 0;
    for (uint32_t w = 0; w < (uint32_t)BLOCK / 32; ++w) {
        before += w < warp ? wsum[w] : 0u;
        total += wsum[w];
    }
    uint32_t base = before + x - s;
    for (uint32_t i = i0; i < i1; ++i) {
        out(i, base);
        base += f(i);
    }
    return total;
}

// Pass 2: one warp per row (nb bucket rows and the hot row): chunk counts ->
// offsets within the row.  The last CTA decides whether the hot ids bypass
// the partition (at least 1/8 of the kept pairs) -- if not, bucket 0 also
// holds them, its chunk offsets being the sum of the two rows' -- and forms
// the bucket starts and cost starts.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_radix_scan(const __grid_constant__ RadixArgs a) {
    constexpr int W = BLOCK / 32;
    __shared__ uint32_t wsum[W];
    __shared__ uint32_t last, hot_on;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t b = blockIdx.x * W + warp;
    if (b <= a.nb) {
        const uint32_t tot = warp_exclusive_scan(a.hist + (size_t)b * a.nchunks, a.nchunks, lane);
        if (lane == 0) a.tot[b] = tot;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // every CTA's totals, read through L2
    const uint32_t nhot = __ldcg(&a.tot[a.nb]);
    const uint32_t kept = block_scan_runs<BLOCK>(
        a.nb, wsum, [&](uint32_t i) { return __ldcg(&a.tot[i]); }, [&](uint32_t, uint32_t) {});
    if (threadIdx.x == 0) {
        hot_on = nhot != 0u && (uint64_t)nhot * 8 >= (uint64_t)kept + nhot;
        *a.mode = hot_on;
    }
    __syncthreads();
    const uint32_t extra0 = hot_on ? 0u : nhot;   // bucket 0 takes the hot pairs
    auto pairs = [&](uint32_t i) { return __ldcg(&a.tot[i]) + (i == 0 ? extra0 : 0u); };
    const uint32_t total = block_scan_runs<BLOCK>(
        a.nb, wsum, pairs, [&](uint32_t i, uint32_t pre) { a.bstart[i] = pre; });
    // cost starts: each non-empty bucket adds its pairs plus a.fixed
    const uint32_t ne = block_scan_runs<BLOCK>(
        a.nb, wsum, [&](uint32_t i) { return pairs(i) ? 1u : 0u; },
        [&](uint32_t i, uint32_t pre) { a.bcost[i] = a.bstart[i] + pre * a.fixed; });
    if (threadIdx.x == 0) {
        a.bstart[a.nb] = total;
        a.bcost[a.nb] = total + ne * a.fixed;
        *a.ticket = 0u;
    }
}

// Pass 3: per tile, (HOT) pairs of hot ids into the CTA's hot table, and for
// the others ranks within buckets, tile offsets, the pairs grouped in shared
// memory, then written out as runs.  Offsets inside a chunk are 32-bit
// (n < 2^31).  The next tile's keys and values are fetched while this one
// is ranked, grouped and written: with TMA, by two bulk copies into a shared
// input buffer issued as soon as the ranks are taken (its mbarrier wait is
// bounded; a wait that runs out sets kRadixBadWait and the CTA stops after
// waiting, bounded, for its copies); otherwise by register loads issued
// before the write-out.  Three CTAs per SM (at most 40 registers) where the
// shared memory allows.
template <int BLOCK, int LOG_T, bool HOT, bool TMA>
__global__ void __launch_bounds__(BLOCK, 3) k_radix_scatter(const __grid_constant__ RadixArgs a) {
    // both forms are launched; the scan's choice runs, the other returns
    if (__ldcg(a.mode) != (HOT ? 1u : 0u)) return;
    static_assert(BLOCK * 8 == (int)kRadixTile && 2 * BLOCK == (int)kRadixMaxBuckets, "tile");
    static_assert(TMA == radix_scatter_tma(HOT), "the form's layout is radix_scatter_smem's");
    constexpr int W = BLOCK / 32;
    constexpr uint32_t IN_W = radix_scatter_in_words(TMA);
    constexpr uint32_t HOT_W = radix_scatter_hot_words(HOT);
    extern __shared__ __align__(16) uint32_t rsmem[];
    uint32_t* smem = rsmem;
    const uint32_t* in_k = smem;                       // TMA: [kRadixTile] keys
    const uint32_t* in_v = smem + kRadixTile;          // TMA: [kRadixTile] values
    const uint32_t bar = smem_u32(smem + 2 * kRadixTile);   // TMA: the input mbarrier
    uint2* stage = reinterpret_cast<uint2*>(smem + IN_W);   // [kRadixTile]
    uint32_t* hcnt = smem + IN_W + 2 * kRadixTile;     // HOT: [kRadixHotIds] hot counts
    float* hsum = reinterpret_cast<float*>(hcnt + kRadixHotIds);   // [kRadixHotIds]
    float* heads = hsum + kRadixHotIds;                // head copies of ids < kKeyedHead
    float* myhead = heads + ((threadIdx.x >> 5) * kKeyedHeadClasses +
                             (threadIdx.x & (kKeyedHeadClasses - 1))) * kKeyedHeadStride;
    uint32_t* tcnt = smem + IN_W + 2 * kRadixTile + HOT_W;   // [nb] pairs of the tile
    uint32_t* toff = tcnt + a.nb;                    // [nb] their first slot in the tile
    uint32_t* shift = toff + a.nb;                   // [nb] bk position - tile slot
    uint32_t* gcur = shift + a.nb;                   // [nb] next position in bk
    uint32_t* wsum = gcur + a.nb;                    // [W], then the tile total
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr uint32_t lt = LOG_T, idmask = (1u << LOG_T) - 1u;
    const uint32_t cap = (uint32_t)a.n, nb = a.nb, nk = a.num_keys;
    uint2* bk = reinterpret_cast<uint2*>(a.bk);
    uint32_t bad = 0;
    if (HOT)
        for (uint32_t i = threadIdx.x; i < HOT_W; i += BLOCK)
            hcnt[i] = 0u;   // hot counts, sums and head copies
    uint32_t phase = 0;   // TMA: parity of the input mbarrier's next phase
    if (TMA && threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // TMA, thread 0: the whole tile at t0 of the chunk into the input buffer
    auto issue = [&](const char* kp, const char* vp, uint32_t t0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_tx(bar, 2 * kRadixTile * 4);
        bulk_g2s(smem_u32(in_k), kp + (size_t)t0 * 4, kRadixTile * 4, bar);
        bulk_g2s(smem_u32(in_v), vp + (size_t)t0 * 4, kRadixTile * 4, bar);
    };
    // hot table -> outputs (global atomics), cleared; between barriers
    auto flush_hot = [&]() {
        fold_head_copies(heads, hsum, kKeyedHead);
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < kRadixHotIds; i += BLOCK) {
            const uint32_t hc = hcnt[i];
            if (hc) {
                atomicAdd(&a.counts[i], hc);
                atomicAdd(&a.sums64[i], (double)hsum[i]);
                hcnt[i] = 0u;
                hsum[i] = 0.f;
            }
        }
        __syncthreads();
    };
    uint32_t tiles = 0;   // since the hot table's last flush
    bool stopped = false;
    for (uint32_t c = blockIdx.x; c < a.nchunks && !stopped; c += gridDim.x) {
        for (uint32_t i = threadIdx.x; i < nb; i += BLOCK) {
            // without the bypass bucket 0 holds the hot ids too (row nb)
            gcur[i] = a.bstart[i] + a.hist[(size_t)i * a.nchunks + c] +
                      (!HOT && i == 0 ? a.hist[(size_t)nb * a.nchunks + c] : 0u);
            tcnt[i] = 0u;
        }
        const uint64_t b0 = (uint64_t)c * a.chunk;
        const uint32_t len = (uint32_t)(min(b0 + a.chunk, a.n) - b0);
        const char* kp = a.keys + b0 * 4;
        const char* vp = a.vals + b0 * 4;
        uint4 kk[2], vv[2];
        uint32_t in[2];
        // register loads of the tile at t0 (every tile without TMA, the ragged
        // last tile with it)
        auto load = [&](uint32_t t0) {
            if (t0 + kRadixTile <= len) {   // CTA-uniform: a whole tile
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const uint32_t i = t0 + ((uint32_t)j * BLOCK + threadIdx.x) * 4;
                    kk[j] = ld_stream_v4(kp + (size_t)i * 4);
                    vv[j] = ld_stream_v4(vp + (size_t)i * 4);
                    in[j] = 0xfu;
                }
            } else {
                uint32_t vin;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const uint32_t i = t0 + ((uint32_t)j * BLOCK + threadIdx.x) * 4;
                    kk[j] = radix_load4(kp, i, len, &in[j]);
                    vv[j] = radix_load4(vp, i, len, &vin);
                }
            }
        };
        if (TMA) {
            if (threadIdx.x == 0 && kRadixTile <= len) issue(kp, vp, 0);
        } else {
            load(0);
        }
        __syncthreads();
        for (uint32_t t0 = 0; t0 < len; t0 += kRadixTile) {
            bool ok = true;
            if (TMA) {
                if (t0 + kRadixTile <= len) {   // CTA-uniform: the bulk-copied tile
                    ok = mbar_wait(bar, phase, a.bad);
                    phase ^= 1u;
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const uint32_t i = ((uint32_t)j * BLOCK + threadIdx.x) * 4;
                        kk[j] = ok ? *reinterpret_cast<const uint4*>(in_k + i) : make_uint4(0, 0, 0, 0);
                        vv[j] = ok ? *reinterpret_cast<const uint4*>(in_v + i) : make_uint4(0, 0, 0, 0);
                        in[j] = ok ? 0xfu : 0u;   // after a failed wait: no pairs
                    }
                } else {
                    load(t0);
                }
            }
            const uint32_t k[8] = {kk[0].x, kk[0].y, kk[0].z, kk[0].w,
                                   kk[1].x, kk[1].y, kk[1].z, kk[1].w};
            const uint32_t v[8] = {vv[0].x, vv[0].y, vv[0].z, vv[0].w,
                                   vv[1].x, vv[1].y, vv[1].z, vv[1].w};
            uint32_t rank2[4] = {0u, 0u, 0u, 0u};   // ranks (< kRadixTile), two per word
            uint32_t valid = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const bool in_range = ((in[q >> 2] >> (q & 3)) & 1u) && k[q] < nk;
                if (HOT && in_range && k[q] < kRadixHotIds) {   // the CTA's hot table
                    atomicAdd(&hcnt[k[q]], 1u);
                    atomicAdd(k[q] < kKeyedHead ? &myhead[k[q]] : &hsum[k[q]],
                              __uint_as_float(v[q]));
                }
                const bool cold = in_range && (!HOT || k[q] >= kRadixHotIds);
                valid |= cold ? 1u << q : 0u;
                const uint32_t r = warp_rank(tcnt, cold ? k[q] >> lt : kNoBucket, lane);
                rank2[q >> 1] |= (r & 0xffffu) << (16 * (q & 1));
            }
            if (TMA) {
                if (__syncthreads_or(!ok)) {   // a wait ran out: stop this CTA
                    if (threadIdx.x == 0) {
                        mbar_wait(bar, phase ^ 1u, a.bad);   // its copy, bounded
                        atomicOr(a.bad, kRadixBadWait);
                    }
                    stopped = true;
                    break;
                }
                // the input buffer is read: fetch the next whole tile into it
                if (threadIdx.x == 0 && t0 + 2 * kRadixTile <= len) issue(kp, vp, t0 + kRadixTile);
            } else {
                __syncthreads();
            }
            // tile offsets: buckets 2t and 2t + 1 in thread t (nb <= 2 * BLOCK)
            const uint32_t b2 = 2 * threadIdx.x;
            uint32_t x = (b2 < nb ? tcnt[b2] : 0u) + (b2 + 1 < nb ? tcnt[b2 + 1] : 0u);
            const uint32_t own = x;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(kAllLanes, x, d);
                if ((int)lane >= d) x += y;
            }
            if (lane == 31) wsum[warp] = x;
            __syncthreads();
            uint32_t before = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) before += (uint32_t)w < warp ? wsum[w] : 0u;
            const uint32_t off0 = before + x - own;
            const uint32_t c0 = b2 < nb ? tcnt[b2] : 0u;   // unchanged since the scan
            const uint32_t c1 = b2 + 1 < nb ? tcnt[b2 + 1] : 0u;
            if (b2 < nb) {
                toff[b2] = off0;
                shift[b2] = gcur[b2] - off0;
                gcur[b2] += c0;
                tcnt[b2] = 0u;
            }
            if (b2 + 1 < nb) {
                toff[b2 + 1] = off0 + c0;
                shift[b2 + 1] = gcur[b2 + 1] - (off0 + c0);
                gcur[b2 + 1] += c1;
                tcnt[b2 + 1] = 0u;
            }
            if (threadIdx.x == BLOCK - 1) wsum[W] = before + x;
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if ((valid >> q) & 1u) {
                    const uint32_t s =
                        toff[k[q] >> lt] + ((rank2[q >> 1] >> (16 * (q & 1))) & 0xffffu);
                    if (s < kRadixTile) stage[s] = make_uint2(k[q], v[q]);
                }
            const uint32_t tn = min(wsum[W], kRadixTile);
            __syncthreads();
            if (!TMA && t0 + kRadixTile < len) load(t0 + kRadixTile);
            for (uint32_t i = threadIdx.x; i < tn; i += BLOCK) {
                const uint2 p = stage[i];
                const uint32_t pb = p.x >> lt;
                const uint32_t pos = pb < nb ? shift[pb] + i : cap;
                if (pos < cap) bk[pos] = make_uint2(p.x & idmask, p.y);
                else bad = kRadixBadPlace;
            }
            // No barrier here: the next tile rewrites stage, toff, shift and
            // wsum only after the barrier that follows its ranks, which every
            // thread reaches after this write-out.
            if (HOT && ++tiles == kRadixHotFlushTiles) {   // fp32 partial sums stay short
                flush_hot();
                tiles = 0;
            }
        }
        __syncthreads();   // gcur and tcnt are reset for the next chunk
    }
    if (HOT && tiles && !stopped) flush_hot();
    if (bad) atomicOr(a.bad, bad);
}

// Pass 4: the grouped pairs split over the grid in even shares of cost
// (radix.h); each bucket segment of a CTA's share is accumulated in the
// shared table of 2^LOG_T ids, with the head copies of its first ids (flushed
// every kLargePiece pairs so fp32 partial sums stay short), and written out.
// The table is zeroed once; each flush clears the entries it writes out and
// the head copies it folds.
template <int BLOCK, int LOG_T>
__global__ void __launch_bounds__(BLOCK) k_radix_reduce(const __grid_constant__ RadixArgs a) {
    constexpr uint32_t T = 1u << LOG_T;
    constexpr uint32_t HP = kKeyedHeadStride;
    extern __shared__ __align__(16) uint32_t rsmem[];
    uint32_t* smem = rsmem;
    uint32_t* hc = smem;                                   // [T] counts
    float* hs = reinterpret_cast<float*>(smem + T);        // [T] fp32 sums
    float* head = hs + T;                                  // [BLOCK / 32 * classes][HP]
    float* my = head + ((threadIdx.x >> 5) * kKeyedHeadClasses +
                        (threadIdx.x & (kKeyedHeadClasses - 1))) * HP;
    const uint64_t ctot = __ldg(&a.bcost[a.nb]);
    const uint64_t clo = ctot * blockIdx.x / gridDim.x;
    const uint64_t chi = ctot * (blockIdx.x + 1) / gridDim.x;
    if (clo >= chi) return;
    for (uint32_t i = threadIdx.x; i < 2 * T + kKeyedHeadWords(BLOCK); i += BLOCK) smem[i] = 0u;
    __syncthreads();
    // the bucket holding cost position clo: the last b with bcost[b] <= clo
    uint32_t bl = 0, bh = a.nb - 1;
    while (bl < bh) {
        const uint32_t mid = (bl + bh + 1) / 2;
        if (__ldg(&a.bcost[mid]) <= clo) bl = mid;
        else bh = mid - 1;
    }
    const uint64_t cap = a.n;
    for (uint32_t b = bl; b < a.nb; ++b) {
        const uint64_t c0 = __ldg(&a.bcost[b]);
        if (c0 >= chi) break;
        const uint64_t bbeg = __ldg(&a.bstart[b]);
        const uint64_t nbk = min((uint64_t)__ldg(&a.bstart[b + 1]), cap) - min(bbeg, cap);
        if (nbk == 0) continue;
        // pair j of the bucket sits at cost position c0 + fixed + j
        const uint64_t first = c0 + a.fixed;
        const uint64_t j0 = clo > first ? min(clo - first, nbk) : 0;
        const uint64_t j1 = chi > first ? min(chi - first, nbk) : 0;
        if (j0 >= j1) continue;
        const bool single = j0 == 0 && j1 == nbk && nbk <= kLargePiece;
        const uint32_t hot = min(T, a.num_keys - b * T);
        for (uint64_t p0 = bbeg + j0; p0 < bbeg + j1; p0 += kLargePiece) {
            const uint64_t p1 = min(p0 + kLargePiece, bbeg + j1);
            // pairs [p0, p1) as 16-byte loads of two pairs each
            const uint64_t q0 = p0 >> 1, q1 = (p1 + 1) >> 1;
            for (uint64_t q = q0 + threadIdx.x; q < q1; q += (uint64_t)BLOCK * 4) {
                uint4 w[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint64_t qq = q + (uint64_t)j * BLOCK;
                    w[j] = qq < q1 ? ld_stream_v4(a.bk + qq * 4) : make_uint4(0u, 0u, 0u, 0u);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint64_t qq = q + (uint64_t)j * BLOCK;
                    if (qq < q1) {
                        if (2 * qq >= p0) {
                            const uint32_t kk = w[j].x & (T - 1);
                            atomicAdd(&hc[kk], 1u);
                            atomicAdd(kk < kKeyedHead ? &my[kk] : &hs[kk], __uint_as_float(w[j].y));
                        }
                        if (2 * qq + 1 < p1) {
                            const uint32_t kk = w[j].z & (T - 1);
                            atomicAdd(&hc[kk], 1u);
                            atomicAdd(kk < kKeyedHead ? &my[kk] : &hs[kk], __uint_as_float(w[j].w));
                        }
                    }
                }
            }
            __syncthreads();
            fold_head_copies(head, hs, min(hot, kKeyedHead));
            __syncthreads();
            uint32_t* cnt = a.counts + (size_t)b * T;
            double* sum = a.sums64 + (size_t)b * T;
            for (uint32_t i = threadIdx.x; i < hot; i += BLOCK) {
                const uint32_t c = hc[i];
                if (c) {
                    const float t = hs[i];
                    if (single) {
                        cnt[i] = c;
                        sum[i] = (double)t;
                    } else {
                        atomicAdd(&cnt[i], c);
                        atomicAdd(&sum[i], (double)t);
                    }
                    hc[i] = 0u;
                    hs[i] = 0.f;
                }
            }
            __syncthreads();   // the table is clean for the next piece
        }
    }
}

}  // namespace dev
}  // namespace scl
