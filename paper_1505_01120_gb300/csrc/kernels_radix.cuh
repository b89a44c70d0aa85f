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

// Pass 1: per chunk, pairs per bucket (bucket-major rows of hist).
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_radix_hist(const __grid_constant__ RadixArgs a) {
    extern __shared__ uint32_t hist[];   // [nb]
    uint32_t bad = 0;
    for (uint32_t c = blockIdx.x; c < a.nchunks; c += gridDim.x) {
        for (uint32_t i = threadIdx.x; i < a.nb; i += BLOCK) hist[i] = 0u;
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
                    if (kk[q] < a.num_keys) atomicAdd(&hist[kk[q] / kMaxKeys], 1u);
                    else bad = kRadixBadKey;
                }
            }
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < a.nb; i += BLOCK)
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

// Pass 2: one warp per bucket row: chunk counts -> offsets within the bucket;
// the last CTA scans the bucket totals into bucket starts.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_radix_scan(const __grid_constant__ RadixArgs a) {
    constexpr int W = BLOCK / 32;
    __shared__ uint32_t wsum[W];
    __shared__ uint32_t last;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t b = blockIdx.x * W + warp;
    if (b < a.nb) {
        const uint32_t tot = warp_exclusive_scan(a.hist + (size_t)b * a.nchunks, a.nchunks, lane);
        if (lane == 0) a.tot[b] = tot;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // every CTA's totals, read through L2; per-thread runs, then warp and block
    const uint32_t per = (a.nb + BLOCK - 1) / BLOCK;
    const uint32_t i0 = min(threadIdx.x * per, a.nb), i1 = min(i0 + per, a.nb);
    uint32_t s = 0;
    for (uint32_t i = i0; i < i1; ++i) s += __ldcg(&a.tot[i]);
    uint32_t x = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kAllLanes, x, d);
        if ((int)lane >= d) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t before = 0;
    for (uint32_t w = 0; w < warp; ++w) before += wsum[w];
    uint32_t base = before + x - s;
    for (uint32_t i = i0; i < i1; ++i) {
        a.bstart[i] = base;
        base += __ldcg(&a.tot[i]);
    }
    if (threadIdx.x == BLOCK - 1) {
        a.bstart[a.nb] = base;
        *a.ticket = 0u;
    }
}

// Pass 3, up to kRadixStagedMaxBuckets buckets: per tile, ranks within
// buckets, tile offsets, the pairs grouped in shared memory, then written
// out as runs.  The next tile's loads are issued before the write-out.
// Offsets inside a chunk are 32-bit (n < 2^31).
template <int BLOCK>
__device__ __forceinline__ void scatter_staged(const RadixArgs& a, uint32_t* smem, uint32_t& bad) {
    static_assert(BLOCK * 8 == (int)kRadixTile, "tile");
    constexpr int W = BLOCK / 32;
    uint2* stage = reinterpret_cast<uint2*>(smem);   // [kRadixTile]
    uint32_t* tcnt = smem + 2 * kRadixTile;          // [nb] pairs of the tile
    uint32_t* toff = tcnt + a.nb;                    // [nb] their first slot in the tile
    uint32_t* shift = toff + a.nb;                   // [nb] bk position - tile slot
    uint32_t* gcur = shift + a.nb;                   // [nb] next position in bk
    uint32_t* wsum = gcur + a.nb;                    // [W], then the tile total
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t cap = (uint32_t)a.n, nb = a.nb, nk = a.num_keys;
    uint2* bk = reinterpret_cast<uint2*>(a.bk);
    for (uint32_t c = blockIdx.x; c < a.nchunks; c += gridDim.x) {
        for (uint32_t i = threadIdx.x; i < nb; i += BLOCK) {
            gcur[i] = a.bstart[i] + a.hist[(size_t)i * a.nchunks + c];
            tcnt[i] = 0u;
        }
        const uint64_t b0 = (uint64_t)c * a.chunk;
        const uint32_t len = (uint32_t)(min(b0 + a.chunk, a.n) - b0);
        const char* kp = a.keys + b0 * 4;
        const char* vp = a.vals + b0 * 4;
        uint4 kk[2], vv[2];
        uint32_t in[2];
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
        load(0);
        __syncthreads();
        for (uint32_t t0 = 0; t0 < len; t0 += kRadixTile) {
            const uint32_t k[8] = {kk[0].x, kk[0].y, kk[0].z, kk[0].w,
                                   kk[1].x, kk[1].y, kk[1].z, kk[1].w};
            const uint32_t v[8] = {vv[0].x, vv[0].y, vv[0].z, vv[0].w,
                                   vv[1].x, vv[1].y, vv[1].z, vv[1].w};
            uint32_t rank[8], valid = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const bool ok = ((in[q >> 2] >> (q & 3)) & 1u) && k[q] < nk;
                valid |= ok ? 1u << q : 0u;
                rank[q] = warp_rank(tcnt, ok ? k[q] / kMaxKeys : kNoBucket, lane);
            }
            __syncthreads();
            // tile offsets: one bucket per thread (nb <= BLOCK)
            const uint32_t b = threadIdx.x;
            const uint32_t cnt = b < nb ? tcnt[b] : 0u;
            uint32_t x = cnt;
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
            if (b < nb) {
                const uint32_t off = before + x - cnt;
                toff[b] = off;
                shift[b] = gcur[b] - off;
                gcur[b] += cnt;
                tcnt[b] = 0u;
            }
            if (threadIdx.x == BLOCK - 1) wsum[W] = before + x;
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if ((valid >> q) & 1u) {
                    const uint32_t s = toff[k[q] / kMaxKeys] + rank[q];
                    if (s < kRadixTile) stage[s] = make_uint2(k[q], v[q]);
                }
            const uint32_t tn = min(wsum[W], kRadixTile);
            __syncthreads();
            if (t0 + kRadixTile < len) load(t0 + kRadixTile);
            for (uint32_t i = threadIdx.x; i < tn; i += BLOCK) {
                const uint2 p = stage[i];
                const uint32_t pb = p.x / kMaxKeys;
                const uint32_t pos = pb < nb ? shift[pb] + i : cap;
                if (pos < cap) bk[pos] = make_uint2(p.x % kMaxKeys, p.y);
                else bad = kRadixBadPlace;
            }
            // No barrier here: the next tile rewrites stage, toff, shift and
            // wsum only after the barrier that follows its ranks, which every
            // thread reaches after this write-out.
        }
        __syncthreads();   // gcur and tcnt are reset for the next chunk
    }
}

// Pass 3, more buckets: each valid pair takes the next slot of its bucket.
template <int BLOCK>
__device__ __forceinline__ void scatter_direct(const RadixArgs& a, uint32_t* gcur, uint32_t& bad) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t cap = (uint32_t)a.n, nb = a.nb, nk = a.num_keys;
    uint2* bk = reinterpret_cast<uint2*>(a.bk);
    for (uint32_t c = blockIdx.x; c < a.nchunks; c += gridDim.x) {
        for (uint32_t i = threadIdx.x; i < nb; i += BLOCK)
            gcur[i] = a.bstart[i] + a.hist[(size_t)i * a.nchunks + c];
        __syncthreads();
        const uint64_t b0 = (uint64_t)c * a.chunk;
        const uint32_t len = (uint32_t)(min(b0 + a.chunk, a.n) - b0);
        const char* kp = a.keys + b0 * 4;
        const char* vp = a.vals + b0 * 4;
        for (uint32_t t0 = 0; t0 < len; t0 += (uint32_t)BLOCK * 8) {
            uint4 kk[2], vv[2];
            uint32_t in[2], vin;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const uint32_t i = t0 + ((uint32_t)j * BLOCK + threadIdx.x) * 4;
                kk[j] = radix_load4(kp, i, len, &in[j]);
                vv[j] = radix_load4(vp, i, len, &vin);
            }
            const uint32_t k[8] = {kk[0].x, kk[0].y, kk[0].z, kk[0].w,
                                   kk[1].x, kk[1].y, kk[1].z, kk[1].w};
            const uint32_t v[8] = {vv[0].x, vv[0].y, vv[0].z, vv[0].w,
                                   vv[1].x, vv[1].y, vv[1].z, vv[1].w};
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const bool ok = ((in[q >> 2] >> (q & 3)) & 1u) && k[q] < nk;
                const uint32_t pos = warp_rank(gcur, ok ? k[q] / kMaxKeys : kNoBucket, lane);
                if (ok) {
                    if (pos < cap) bk[pos] = make_uint2(k[q] % kMaxKeys, v[q]);
                    else bad = kRadixBadPlace;
                }
            }
        }
        __syncthreads();   // gcur is reloaded for the next chunk
    }
}

// Three CTAs per SM (at most 40 registers) keep loads in flight across the
// barriers of the staged tiles.
template <int BLOCK, bool STAGED>
__global__ void __launch_bounds__(BLOCK, 3) k_radix_scatter(const __grid_constant__ RadixArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t bad = 0;
    if constexpr (STAGED) scatter_staged<BLOCK>(a, smem, bad);
    else scatter_direct<BLOCK>(a, smem, bad);
    if (bad) atomicOr(a.bad, bad);
}

// Pass 4: an even share of the grouped pairs per CTA; each bucket segment
// of the share is accumulated in the shared table, with the head copies of
// its first ids (flushed every kLargePiece pairs so fp32 partial sums stay
// short), and written out.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_radix_reduce(const __grid_constant__ RadixArgs a) {
    constexpr uint32_t HP = kKeyedHeadStride;
    constexpr uint32_t NCOPY = BLOCK / 32 * kKeyedHeadClasses;
    __shared__ uint32_t hc[kMaxKeys];
    __shared__ float hs[kMaxKeys];
    __shared__ float head[kKeyedHeadWords(BLOCK)];
    float* my = head + ((threadIdx.x >> 5) * kKeyedHeadClasses +
                        (threadIdx.x & (kKeyedHeadClasses - 1))) * HP;
    const uint64_t nv = min((uint64_t)__ldg(&a.bstart[a.nb]), a.n);
    const uint64_t lo = nv * blockIdx.x / gridDim.x;
    const uint64_t hi = nv * (blockIdx.x + 1) / gridDim.x;
    if (lo >= hi) return;
    // bucket holding pair lo: the last b with bstart[b] <= lo
    uint32_t bl = 0, bh = a.nb - 1;
    while (bl < bh) {
        const uint32_t mid = (bl + bh + 1) / 2;
        if (__ldg(&a.bstart[mid]) <= lo) bl = mid;
        else bh = mid - 1;
    }
    uint32_t b = bl;
    uint64_t s = lo;
    while (s < hi && b < a.nb) {
        const uint64_t bbeg = __ldg(&a.bstart[b]);
        const uint64_t bend = min((uint64_t)__ldg(&a.bstart[b + 1]), nv);
        if (bend <= s) {   // empty bucket
            ++b;
            continue;
        }
        const uint64_t se = min(hi, bend);
        const bool single = s == bbeg && se == bend && se - s <= kLargePiece;
        const uint32_t hot = min(kMaxKeys, a.num_keys - b * kMaxKeys);
        for (uint64_t p0 = s; p0 < se; p0 += kLargePiece) {
            const uint64_t p1 = min(p0 + kLargePiece, se);
            for (uint32_t i = threadIdx.x; i < hot; i += BLOCK) {
                hc[i] = 0u;
                hs[i] = 0.f;
            }
            for (uint32_t i = threadIdx.x; i < kKeyedHeadWords(BLOCK); i += BLOCK) head[i] = 0.f;
            __syncthreads();
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
                            const uint32_t kk = w[j].x % kMaxKeys;
                            atomicAdd(&hc[kk], 1u);
                            atomicAdd(kk < kKeyedHead ? &my[kk] : &hs[kk], __uint_as_float(w[j].y));
                        }
                        if (2 * qq + 1 < p1) {
                            const uint32_t kk = w[j].z % kMaxKeys;
                            atomicAdd(&hc[kk], 1u);
                            atomicAdd(kk < kKeyedHead ? &my[kk] : &hs[kk], __uint_as_float(w[j].w));
                        }
                    }
                }
            }
            __syncthreads();
            uint32_t* cnt = a.counts + (size_t)b * kMaxKeys;
            double* sum = a.sums64 + (size_t)b * kMaxKeys;
            for (uint32_t i = threadIdx.x; i < hot; i += BLOCK) {
                const uint32_t c = hc[i];
                if (c) {
                    float t = hs[i];
                    if (i < kKeyedHead)
                        for (uint32_t r = 0; r < NCOPY; ++r) t += head[r * HP + i];
                    if (single) {
                        cnt[i] = c;
                        sum[i] = (double)t;
                    } else {
                        atomicAdd(&cnt[i], c);
                        atomicAdd(&sum[i], (double)t);
                    }
                }
            }
            __syncthreads();   // the tables are zeroed again by the next piece
        }
        s = se;
        ++b;
    }
}

}  // namespace dev
}  // namespace scl
