// kernels.cuh -- sm_103a kernels of the SparkCL per-partition path.
//
//   k_persistent<BLOCK, IPT, MASK>  MapCLPartition + ReduceCL fused (Sec. 3.1.3
//                                   items 2-3): every element of a partition is
//                                   mapped by the catalogue kernel (the run()
//                                   body of Sec. 3.1.1.2) and folded, in one
//                                   HBM pass, by a persistent grid.
//   k_keyed_lean<BLOCK, IPT>        the keyed-only persistent kernel capped at 48
//                                   registers, for keyed tasks that share the SMs
//                                   with a concurrent streaming launch.
//   k_keyed_fold                    second pass of the keyed reduce (Sec. 3.2.3):
//                                   folds the per-piece tables of keyed tasks cut
//                                   into more than 8 pieces (fewer: the CTA that
//                                   writes the last piece folds them).
//   k_map<BLOCK, IPT, KIND, ALIGNED> MapCL with a materialised output array
//                                   (Sec. 3.1.3 item 1; Fig. 3's c[gid] = f(a[gid])).
//
// Data path: 128-bit vector loads (ld.global.nc, no L1 allocation, 256-byte L2
// prefetch) of IPT independent vectors per thread before any use, so a CTA
// has BLOCK*IPT*16 bytes in flight; streaming sums are fp32 per thread per
// chunk, float-float pairs across chunks (the fp32 pipe, not GB300's slow
// fp64 pipe), a fixed-order warp-butterfly and block tree, one partial per
// segment and one atomic ticket per task; the last CTA of a task folds the
// segment partials in slot order (deterministic).
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "internal.h"

namespace scl {
namespace dev {

// ----------------------------------------------------------------- loads

__device__ __forceinline__ uint4 ld_stream_v4(const void* p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ uint32_t ld_stream_b32(const void* p) {
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Asks L2 for the 128-byte line holding p (no register result, no fault
// semantics beyond those of a load of p; p must lie inside an allocation).
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void st_stream_v4(void* p, uint4 v) {
    asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};"
                 :: "l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
}

// ------------------------------------------------------- catalogue maps

// mix32: xorshift-multiply finaliser on 32-bit words (all steps mod 2^32).
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// poly3: t = fma(a, x*x, b); y = fma(t, x, c); the product x*x rounded once.
// Explicit _rn intrinsics so that no contraction can change the roundings.
__device__ __forceinline__ float poly3(float x, float a, float b, float c) {
    const float x2 = __fmul_rn(x, x);
    const float t = __fmaf_rn(a, x2, b);
    return __fmaf_rn(t, x, c);
}

template <int KIND>
__device__ __forceinline__ uint32_t map_u32(uint32_t x) {
    if constexpr (KIND == K_U32_MIX32) return mix32(x);
    else return x;
}

template <int KIND>
__device__ __forceinline__ float map_f32(float x, float a, float b, float c) {
    if constexpr (KIND == K_F32_POLY3) return poly3(x, a, b, c);
    else return x;
}

// --------------------------------------------------- float-float sums

// Sums past one thread's chunk are carried as float-float pairs (hi + lo, two
// fp32 words, about 44 bits of precision) on the fp32 pipe: GB300 runs fp64
// adds at a small fraction of its fp32 rate, and fp64 block trees saturated
// its fp64 pipe on batches of small partitions.  two_sum is exact (hi + lo
// equals a + b) and its result does not depend on the operand order, so a
// xor-butterfly leaves the same pair in every lane.  A non-finite hi keeps lo
// at zero, so inf and NaN propagate as in fp64.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float ap = __fsub_rn(s, bp);
    const float e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
    return ff{s, isfinite(s) ? e : 0.f};
}

// a + b with |a| >= |b| (or a zero).
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return ff{s, isfinite(s) ? e : 0.f};
}

__device__ __forceinline__ ff ff_add(ff x, ff y) {
    const ff s = ff_two_sum(x.hi, y.hi);
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ ff ff_add_f(ff x, float y) {
    const ff s = ff_two_sum(x.hi, y);
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}

// The pair of a double: hi its fp32 rounding, lo the rounding of the rest.
__device__ __forceinline__ ff ff_of_double(double d) {
    const float hi = (float)d;
    return ff{hi, isfinite(hi) ? (float)(d - (double)hi) : 0.f};
}

__device__ __forceinline__ double ff_to_double(ff x) { return (double)x.hi + (double)x.lo; }

__device__ __forceinline__ ff ff_shfl_xor(ff x, int o) {
    return ff{__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
}

// ------------------------------------------------------ block reductions

struct RedSmem {
    float shi[32], slo[32];
    unsigned long long u[32];
    float mn[32];
    float mx[32];
    uint32_t q;      // next streaming segment (prefetched by thread 0)
    uint32_t flag;   // broadcast: this CTA folds the task
};

// Every thread returns the block total.  Fixed association order:
// a xor-butterfly within each warp, then the same butterfly over the warp
// totals.  Ends with a barrier so the smem can be reused at once.
template <int BLOCK>
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, RedSmem& sm) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sm.u[w] = v;
    __syncthreads();
    v = (l < BLOCK / 32) ? sm.u[l] : 0ull;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    return v;
}

template <int BLOCK>
__device__ __forceinline__ void block_reduce_ff(ff& s, float& mn, float& mx, RedSmem& sm) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s = ff_add(s, ff_shfl_xor(s, o));
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sm.shi[w] = s.hi;
        sm.slo[w] = s.lo;
        sm.mn[w] = mn;
        sm.mx[w] = mx;
    }
    __syncthreads();
    const bool in = l < BLOCK / 32;
    s = in ? ff{sm.shi[l], sm.slo[l]} : ff{0.f, 0.f};
    mn = in ? sm.mn[l] : CUDART_INF_F;
    mx = in ? sm.mx[l] : -CUDART_INF_F;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s = ff_add(s, ff_shfl_xor(s, o));
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    __syncthreads();
}

// block_reduce_ff of a sum and block_sum_u64 of a count in one exchange (same
// association orders, so the same totals), for the keyed write-out.
template <int BLOCK>
__device__ __forceinline__ void block_reduce_ff_u64(ff& s, unsigned long long& u, RedSmem& sm) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s = ff_add(s, ff_shfl_xor(s, o));
        u += __shfl_xor_sync(0xffffffffu, u, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sm.shi[w] = s.hi;
        sm.slo[w] = s.lo;
        sm.u[w] = u;
    }
    __syncthreads();
    const bool in = l < BLOCK / 32;
    s = in ? ff{sm.shi[l], sm.slo[l]} : ff{0.f, 0.f};
    u = in ? sm.u[l] : 0ull;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s = ff_add(s, ff_shfl_xor(s, o));
        u += __shfl_xor_sync(0xffffffffu, u, o);
    }
    __syncthreads();
}

__device__ __forceinline__ void write_result(scl_result* r, uint64_t u, double s, float mn,
                                             float mx, int32_t status, uint64_t n,
                                             uint32_t kind) {
    scl_result o;
    o.u64_sum = u;
    o.f64_sum = s;
    o.f32_sum = (float)s;
    o.f32_min = mn;
    o.f32_max = mx;
    o.status = status;
    o.n = n;
    o.kind = kind;
    o.reserved = 0;
    *r = o;
}

// ------------------------------------------------- streaming segment

// One segment [b, e) of a streaming task.  Thread t of the CTA handles, in
// each chunk of BLOCK*IPT*4 elements starting at c, the four elements
// c + 4*(j*BLOCK + t) + {0..3} for j < IPT -- the same mapping in the vector
// path and in the masked scalar path (ragged tail, or an unaligned
// partition), so the fp32 grouping of a chunk never depends on the path.
// Returns true in thread 0 of the CTA that wrote the task's final result.
template <int BLOCK, int IPT, int KIND>
__device__ __forceinline__ bool stream_segment(const KernelArgs& a, const DevTask& t,
                                               uint32_t task, uint32_t local, RedSmem& sm) {
    constexpr bool F32 = (KIND == K_F32_IDENT || KIND == K_F32_POLY3);
    constexpr uint32_t CH = BLOCK * IPT * 4;
    const uint64_t b = (uint64_t)local * t.seg_elems;
    const uint64_t e = min(b + (uint64_t)t.seg_elems, t.n);
    const char* base = static_cast<const char*>(t.in0);
    const float ca = t.coef[0], cb = t.coef[1], cc = t.coef[2];

    unsigned long long usum = 0;
    ff fsum{0.f, 0.f};
    float mn = CUDART_INF_F, mx = -CUDART_INF_F;

    uint64_t i = b;
    if (t.flags & TF_ALIGNED) {
        for (; i + CH <= e; i += CH) {
            uint4 v[IPT];
            const char* p = base + (i + (uint64_t)threadIdx.x * 4) * 4;
#pragma unroll
            for (int j = 0; j < IPT; ++j) v[j] = ld_stream_v4(p + (size_t)j * BLOCK * 16);
            if constexpr (F32) {
                float cs = 0.f;
#pragma unroll
                for (int j = 0; j < IPT; ++j) {
                    const float y0 = map_f32<KIND>(__uint_as_float(v[j].x), ca, cb, cc);
                    const float y1 = map_f32<KIND>(__uint_as_float(v[j].y), ca, cb, cc);
                    const float y2 = map_f32<KIND>(__uint_as_float(v[j].z), ca, cb, cc);
                    const float y3 = map_f32<KIND>(__uint_as_float(v[j].w), ca, cb, cc);
                    cs += __fadd_rn(__fadd_rn(y0, y1), __fadd_rn(y2, y3));
                    mn = fminf(mn, fminf(fminf(y0, y1), fminf(y2, y3)));
                    mx = fmaxf(mx, fmaxf(fmaxf(y0, y1), fmaxf(y2, y3)));
                }
                fsum = ff_add_f(fsum, cs);
            } else {
#pragma unroll
                for (int j = 0; j < IPT; ++j) {
                    usum += (unsigned long long)map_u32<KIND>(v[j].x) +
                            (unsigned long long)map_u32<KIND>(v[j].y) +
                            (unsigned long long)map_u32<KIND>(v[j].z) +
                            (unsigned long long)map_u32<KIND>(v[j].w);
                }
            }
        }
    }
    // masked scalar path: the ragged tail of the segment, or every chunk of an
    // unaligned partition
    for (; i < e; i += CH) {
        float cs = 0.f;
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const uint64_t g = i + ((uint64_t)j * BLOCK + threadIdx.x) * 4;
            uint32_t w[4];
            bool ok[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ok[q] = g + q < e;
                w[q] = ok[q] ? ld_stream_b32(base + (g + q) * 4) : 0u;
            }
            if constexpr (F32) {
                float y[4], ys[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    y[q] = map_f32<KIND>(__uint_as_float(w[q]), ca, cb, cc);
                    ys[q] = ok[q] ? y[q] : 0.f;
                    if (ok[q]) {
                        mn = fminf(mn, y[q]);
                        mx = fmaxf(mx, y[q]);
                    }
                }
                cs += __fadd_rn(__fadd_rn(ys[0], ys[1]), __fadd_rn(ys[2], ys[3]));
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (ok[q]) usum += (unsigned long long)map_u32<KIND>(w[q]);
            }
        }
        if constexpr (F32) fsum = ff_add_f(fsum, cs);
    }

    if constexpr (F32) block_reduce_ff<BLOCK>(fsum, mn, mx, sm);
    else usum = block_sum_u64<BLOCK>(usum, sm);

    if (t.nseg == 1) {
        if (threadIdx.x == 0)
            write_result(t.result, usum, F32 ? ff_to_double(fsum) : (double)usum,
                         F32 ? mn : 0.f, F32 ? mx : 0.f, SCL_OK, t.n, t.kind);
        return threadIdx.x == 0;
    }
    if (threadIdx.x == 0) {
        StreamPartial* sp = a.spart + t.slot0 + local;
        sp->shi = fsum.hi;
        sp->slo = fsum.lo;
        sp->u = usum;
        sp->mn = mn;
        sp->mx = mx;
        __threadfence();
        const uint32_t prev = atomicAdd(&a.tickets[task], 1u);
        sm.flag = (prev == t.nseg - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (sm.flag == 0) return false;   // uniform across the CTA
    __threadfence();

    // This CTA finished the task's last segment: fold the partials in slot order.
    ff fs{0.f, 0.f};
    unsigned long long fu = 0;
    float fmn = CUDART_INF_F, fmx = -CUDART_INF_F;
    for (uint32_t s = threadIdx.x; s < t.nseg; s += BLOCK) {
        const StreamPartial* sp = a.spart + t.slot0 + s;
        if constexpr (F32) {
            fs = ff_add(fs, ff{__ldcg(&sp->shi), __ldcg(&sp->slo)});
            fmn = fminf(fmn, __ldcg(&sp->mn));
            fmx = fmaxf(fmx, __ldcg(&sp->mx));
        } else {
            fu += __ldcg(reinterpret_cast<const unsigned long long*>(&sp->u));
        }
    }
    if constexpr (F32) block_reduce_ff<BLOCK>(fs, fmn, fmx, sm);
    else fu = block_sum_u64<BLOCK>(fu, sm);
    if (threadIdx.x == 0) {
        write_result(t.result, fu, F32 ? ff_to_double(fs) : (double)fu, F32 ? fmn : 0.f,
                     F32 ? fmx : 0.f, SCL_OK, t.n, t.kind);
        a.tickets[task] = 0u;   // ready for the next launch
    }
    return threadIdx.x == 0;
}

// ------------------------------------------------------------ keyed piece

// Adds the head copies of ids [0, nhead) into the table's fp32 sums and
// clears them.  Warp w owns copies w * kKeyedHeadClasses onwards; lane l sums
// its warp's copies of id l and adds them with one atomic, so the warps fold
// in parallel.  Call between barriers.
__device__ __forceinline__ void fold_head_copies(float* heads, float* sum, uint32_t nhead) {
    const uint32_t lane = threadIdx.x & 31;
    float* own = heads + (threadIdx.x >> 5) * kKeyedHeadClasses * kKeyedHeadStride;
    float t = 0.f;
#pragma unroll
    for (uint32_t r = 0; r < kKeyedHeadClasses; ++r) {
        t += own[r * kKeyedHeadStride + lane];
        own[r * kKeyedHeadStride + lane] = 0.f;
    }
    if (t != 0.f && lane < nhead) atomicAdd(&sum[lane], t);
}

// Counts go straight to the table (integer adds to one address do not
// serialise); fp32 sums of ids below kKeyedHead go to this thread's head copy
// (`head`), the rest to the table.  Hashed ids spread the frequent keys, so
// the hashed form uses the table only.
template <bool HASHED>
__device__ __forceinline__ void keyed_add(uint32_t k, uint32_t v, uint32_t nk, uint32_t* cnt,
                                          float* sum, float* head, uint32_t& bad) {
    if constexpr (HASHED) k = __umulhi(mix32(k), nk);   // (mix32(key) * nk) >> 32, always < nk
    if (k < nk) {           // a negative int32 key is a huge uint32: rejected here
        atomicAdd(&cnt[k], 1u);
        atomicAdd(!HASHED && k < kKeyedHead ? &head[k] : &sum[k], __uint_as_float(v));
    } else {
        bad = 1u;
    }
}

// The fixed-point window of one piece: magnitudes with bit patterns in
// [lo, lo + span) are added to the int32 sums as round(v * scale), scale =
// 2^F; inv = 2^-F folds them back.
struct FixWin {
    float scale, inv;
    uint32_t lo, span;
};

// round(v * scale) for |v * scale| <= 2^22 (scale a power of two, so the
// product is exact): adding 1.5 * 2^23 in the same rounding step leaves the
// integer, rounded to nearest even, in the low mantissa bits.  One fp32 FMA
// instead of a conversion on the slower XU pipe.
__device__ __forceinline__ int32_t fix_round(float v, float scale) {
    return __float_as_int(__fmaf_rn(v, scale, 12582912.0f)) - 0x4B400000;
}

// As keyed_add, with values inside the window added to the int32 sums.
template <bool HASHED>
__device__ __forceinline__ void keyed_add_fix(uint32_t k, uint32_t v, uint32_t nk, uint32_t* cnt,
                                              float* sum, float* head, int32_t* isum,
                                              const FixWin& w, uint32_t& bad) {
    if constexpr (HASHED) k = __umulhi(mix32(k), nk);
    if (k < nk) {
        atomicAdd(&cnt[k], 1u);
        const uint32_t ab = v & 0x7fffffffu;
        if (!HASHED && k < kKeyedHead)
            atomicAdd(&head[k], __uint_as_float(v));
        else if (ab - w.lo < w.span)
            atomicAdd(&isum[k], fix_round(__uint_as_float(v), w.scale));
        else if (ab != 0u)   // a zero of either sign adds nothing
            atomicAdd(&sum[k], __uint_as_float(v));
    } else {
        bad = 1u;
    }
}

// Folds the window's int32 sums into the fp32 table and starts a new window;
// returns nonzero in a thread if one of its keys took 2^kFixCountBits pairs
// or more in the window (its int32 sum may have wrapped).  Call between
// barriers.
template <int BLOCK, bool HASHED>
__device__ __forceinline__ uint32_t fix_fold(uint32_t nk, const uint32_t* cnt, float* sum,
                                             int32_t* isum, uint32_t* snap, float inv) {
    uint32_t over = 0;
    for (uint32_t k = threadIdx.x; k < nk; k += BLOCK) {
        const uint32_t c = cnt[k];
        if (HASHED || k >= kKeyedHead) over |= (uint32_t)(c - snap[k] >= (1u << kFixCountBits));
        const int32_t q = isum[k];
        if (q != 0) {
            sum[k] += (float)q * inv;
            isum[k] = 0;
        }
        snap[k] = c;
    }
    return over;
}

// Asks L2 for pairs [c, min(c + BLOCK*IPT*4, e)) of a key array and a value
// array: one prefetch per 128 bytes, spread over the CTA, every address
// inside the range.
template <int BLOCK, int IPT>
__device__ __forceinline__ void prefetch_chunk_l2(const char* kb, const char* vb, uint64_t c,
                                                  uint64_t e) {
    constexpr uint64_t CH = (uint64_t)BLOCK * IPT * 4;
    const uint64_t len = c < e ? min(e - c, CH) : 0ull;
    const uint32_t lines = (uint32_t)((len + 31) / 32);   // 32 pairs = 128 bytes per array
    for (uint32_t l = threadIdx.x; l < 2 * lines; l += BLOCK) {
        const bool key = l < lines;
        const uint64_t el = c + (uint64_t)(key ? l : l - lines) * 32;   // < c + len <= e
        prefetch_l2((key ? kb : vb) + el * 4);
    }
}

// One pass over pairs [b, e): 128-bit loads of IPT vectors of keys and of
// values per thread, then the table adds; while a chunk's adds run, the next
// chunk is on its way into L2, so a warp's next loads wait on L2 rather than
// DRAM.  FIX: through the fixed-point
// window, folded every kFixWindow pairs and at the end; returns nonzero in
// every thread if a window overflowed.
template <int BLOCK, int IPT, bool HASHED, bool FIX>
__device__ __forceinline__ uint32_t keyed_pass(const DevTask& t, uint64_t b, uint64_t e,
                                               uint32_t* tab, float* head, const FixWin& w,
                                               uint32_t& bad) {
    constexpr uint32_t CH = BLOCK * IPT * 4;
    static_assert(kFixWindow % CH == 0, "windows hold whole chunks");
    uint32_t* cnt = tab;
    float* sum = reinterpret_cast<float*>(tab + kMaxKeys);
    int32_t* isum = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(tab) + kFixSumOffset);
    uint32_t* snap = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(tab) + kFixSnapOffset);
    const uint32_t nk = t.num_keys;
    const char* kb = static_cast<const char*>(t.in0);
    const char* vb = static_cast<const char*>(t.in1);
    uint32_t over = 0;
    uint64_t next_fold = b + kFixWindow;
    auto add = [&](uint32_t k, uint32_t v) {
        if constexpr (FIX) keyed_add_fix<HASHED>(k, v, nk, cnt, sum, head, isum, w, bad);
        else keyed_add<HASHED>(k, v, nk, cnt, sum, head, bad);
    };
    auto window = [&](uint64_t i) {   // CTA-uniform
        if constexpr (FIX) {
            if (i >= next_fold) {
                __syncthreads();
                over |= fix_fold<BLOCK, HASHED>(nk, cnt, sum, isum, snap, w.inv);
                __syncthreads();
                next_fold += kFixWindow;
            }
        }
    };
    uint64_t i = b;
    if (t.flags & TF_ALIGNED) {
        for (; i + CH <= e; i += CH) {
            window(i);
            uint4 kv[IPT], vv[IPT];
            const uint64_t off = (i + (uint64_t)threadIdx.x * 4) * 4;
#pragma unroll
            for (int j = 0; j < IPT; ++j) kv[j] = ld_stream_v4(kb + off + (size_t)j * BLOCK * 16);
#pragma unroll
            for (int j = 0; j < IPT; ++j) vv[j] = ld_stream_v4(vb + off + (size_t)j * BLOCK * 16);
            prefetch_chunk_l2<BLOCK, IPT>(kb, vb, i + CH, e);
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                add(kv[j].x, vv[j].x);
                add(kv[j].y, vv[j].y);
                add(kv[j].z, vv[j].z);
                add(kv[j].w, vv[j].w);
            }
        }
    }
    // The last, partial chunk of aligned arrays: its whole vectors by 128-bit
    // loads issued together (a thread past the end re-reads the chunk's first
    // vector and drops it), then the at most 3 pairs after the last whole
    // vector.  (i is a multiple of 4: pieces start at multiples of 64 pairs.)
    if ((t.flags & TF_ALIGNED) && i < e) {
        window(i);
        const uint64_t ev = e & ~(uint64_t)3;
        if (i + 4 <= ev) {
            uint4 kv[IPT], vv[IPT];
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                const uint64_t g = i + ((uint64_t)j * BLOCK + threadIdx.x) * 4;
                const uint64_t gc = g + 4 <= ev ? g : i;
                kv[j] = ld_stream_v4(kb + gc * 4);
                vv[j] = ld_stream_v4(vb + gc * 4);
            }
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                const uint64_t g = i + ((uint64_t)j * BLOCK + threadIdx.x) * 4;
                if (g + 4 <= ev) {
                    add(kv[j].x, vv[j].x);
                    add(kv[j].y, vv[j].y);
                    add(kv[j].z, vv[j].z);
                    add(kv[j].w, vv[j].w);
                }
            }
        }
        if (threadIdx.x < e - ev)
            add(ld_stream_b32(kb + (ev + threadIdx.x) * 4), ld_stream_b32(vb + (ev + threadIdx.x) * 4));
        i = e;
    }
    for (; i < e; i += CH) {
        window(i);
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const uint64_t g = i + ((uint64_t)j * BLOCK + threadIdx.x) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (g + q < e) add(ld_stream_b32(kb + (g + q) * 4), ld_stream_b32(vb + (g + q) * 4));
        }
    }
    if constexpr (FIX) {
        __syncthreads();
        over |= fix_fold<BLOCK, HASHED>(nk, cnt, sum, isum, snap, w.inv);
        return (uint32_t)__syncthreads_or((int)over);
    }
    return 0u;
}

// Zeroes words [0, n) of a shared array, 16 bytes per store where it can.
template <int BLOCK>
__device__ __forceinline__ void smem_zero(uint32_t* p, uint32_t n) {
    const uint32_t n4 = n / 4;
    for (uint32_t i = threadIdx.x; i < n4; i += BLOCK)
        reinterpret_cast<uint4*>(p)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (uint32_t i = n4 * 4 + threadIdx.x; i < n; i += BLOCK) p[i] = 0u;
}

// Zeroes the count and fp32 sum of ids [0, nk) and the head copies (and, with
// FIX, the int32 sums and count snapshots).  Call between barriers.
template <int BLOCK, bool HASHED, bool FIX>
__device__ __forceinline__ void keyed_zero(uint32_t* tab, uint32_t nk) {
    smem_zero<BLOCK>(tab, nk);
    smem_zero<BLOCK>(tab + kMaxKeys, nk);
    if constexpr (FIX) {
        smem_zero<BLOCK>(reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(tab) + kFixSumOffset), nk);
        smem_zero<BLOCK>(reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(tab) + kFixSnapOffset), nk);
    }
    if (!HASHED) smem_zero<BLOCK>(tab + kKeyedTableWords, kKeyedHeadWords(BLOCK));
}

// Largest finite |v| (as a bit pattern) over this thread's pairs of the first
// chunk of [b, e); the chunk's values are read again from L2 by the pass.
// Aligned arrays and a whole first chunk (every FAST piece: it holds at least
// kFixMinPairs >= BLOCK*IPT*4 pairs) take IPT unconditional 128-bit loads,
// all in flight at once; otherwise one guarded 32-bit load per pair.
__device__ __forceinline__ uint32_t finite_abs_max4(uint32_t m, uint4 v) {
    const uint32_t a[4] = {v.x & 0x7fffffffu, v.y & 0x7fffffffu, v.z & 0x7fffffffu,
                           v.w & 0x7fffffffu};
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (a[q] < 0x7f800000u) m = max(m, a[q]);
    return m;
}

template <int BLOCK, int IPT>
__device__ __forceinline__ uint32_t first_chunk_max(const DevTask& t, uint64_t b, uint64_t e) {
    const char* vb = static_cast<const char*>(t.in1);
    uint32_t m = 0;
    constexpr uint64_t CH = (uint64_t)BLOCK * IPT * 4;
    if ((t.flags & TF_ALIGNED) && e - b >= CH) {
        uint4 v[IPT];
#pragma unroll
        for (int j = 0; j < IPT; ++j)
            v[j] = ld_stream_v4(vb + (b + ((uint64_t)j * BLOCK + threadIdx.x) * 4) * 4);
#pragma unroll
        for (int j = 0; j < IPT; ++j) m = finite_abs_max4(m, v[j]);
        return m;
    }
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const uint64_t g = b + ((uint64_t)j * BLOCK + threadIdx.x) * 4;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (g + q < e) {
                const uint32_t ab = ld_stream_b32(vb + (g + q) * 4) & 0x7fffffffu;
                if (ab < 0x7f800000u) m = max(m, ab);
            }
    }
    return m;
}

// The window of a piece whose first chunk's largest finite magnitude has the
// bit pattern m: B = 2^(E+1) for m in [2^E, 2^(E+1)), F = 31 - kFixCountBits
// - (E+1), so |round(v * 2^F)| <= 2^(31 - kFixCountBits) for |v| < B.  False
// if m is zero or outside [2^-90, 2^90) (the pass then uses fp32 adds only).
__device__ __forceinline__ bool fix_window(uint32_t m, FixWin* w) {
    if (m < 0x12800000u || m >= 0x6c800000u) return false;   // [2^-90, 2^90)
    const int e1 = (int)(m >> 23) - 127 + 1;                    // B = 2^e1
    const int F = 31 - (int)kFixCountBits - e1;
    w->scale = __uint_as_float((uint32_t)(F + 127) << 23);
    w->inv = __uint_as_float((uint32_t)(127 - F) << 23);
    w->lo = (uint32_t)(e1 - (int)kFixTinyBits + 127) << 23;
    w->span = ((uint32_t)(e1 + 127) << 23) - w->lo;
    return true;
}

// Pairs [b, e) of a keyed task accumulated into the CTA's shared-memory table
// (count[kMaxKeys] then fp32 sum[kMaxKeys], then the head copies), zeroed
// first; the head copies are folded into the table at the end.  FAST (the
// keyed-only kernel, whose CTAs have kKeyedFastSmemBytes of shared memory):
// long pieces over large key spaces go through the fixed-point window, and a
// piece whose window overflowed runs again on the fp32 table alone.  Returns,
// in every thread, whether any key was out of range.  Ends with a barrier.
template <int BLOCK, int IPT, bool HASHED, bool FAST = false>
__device__ __forceinline__ int keyed_accumulate(const DevTask& t, uint64_t b, uint64_t e,
                                                uint32_t* tab) {
    static_assert(kKeyedHeadWords(BLOCK) * 4 + kKeyedTableWords * 4 <= kKeyedSmemBytes, "smem");
    static_assert(BLOCK / 32 <= 16, "per-warp maxima");
    float* sum = reinterpret_cast<float*>(tab + kMaxKeys);
    float* heads = reinterpret_cast<float*>(tab + kKeyedTableWords);
    float* head = heads + ((threadIdx.x >> 5) * kKeyedHeadClasses +
                           (threadIdx.x & (kKeyedHeadClasses - 1))) * kKeyedHeadStride;
    const uint32_t nk = t.num_keys;
    FixWin w{0.f, 0.f, 0u, 0u};
    uint32_t bad = 0;
    bool done = false;
    if constexpr (FAST) {
        if (nk >= kFixMinKeys && e - b >= kFixMinPairs) {
            uint32_t* wmax =
                reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(tab) + kFixMaxOffset);
            const uint32_t m = __reduce_max_sync(0xffffffffu, first_chunk_max<BLOCK, IPT>(t, b, e));
            if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
            keyed_zero<BLOCK, HASHED, true>(tab, nk);
            __syncthreads();
            uint32_t mm = 0;
#pragma unroll
            for (int q = 0; q < BLOCK / 32; ++q) mm = max(mm, wmax[q]);
            if (!fix_window(mm, &w)) {
                keyed_pass<BLOCK, IPT, HASHED, false>(t, b, e, tab, head, w, bad);
            } else if (keyed_pass<BLOCK, IPT, HASHED, true>(t, b, e, tab, head, w, bad)) {
                // a window overflowed: run the piece again on the fp32 table
                keyed_zero<BLOCK, HASHED, false>(tab, nk);
                __syncthreads();
                bad = 0;
                keyed_pass<BLOCK, IPT, HASHED, false>(t, b, e, tab, head, w, bad);
            }
            done = true;
        }
    }
    if (!done) {
        keyed_zero<BLOCK, HASHED, false>(tab, nk);
        __syncthreads();
        keyed_pass<BLOCK, IPT, HASHED, false>(t, b, e, tab, head, w, bad);
    }
    const int any_bad = __syncthreads_or((int)bad);
    if (!HASHED) {
        fold_head_copies(heads, sum, min(nk, kKeyedHead));
        __syncthreads();
    }
    return any_bad;
}

// The fold of a keyed task cut into t.nseg pieces, by the CTA that wrote its
// last piece table: per id, the counts (exact, uint32) and the fp32 sums (a
// float-float pair) over the tables in piece order; then the outputs, and the
// result with the totals.  Four consecutive ids per thread are read as 16-byte
// vectors, four pieces' loads in flight at a time.  Call between barriers.
template <int BLOCK>
__device__ __forceinline__ void keyed_fold_task(const KernelArgs& a, const DevTask& t,
                                                uint32_t task, RedSmem& sm) {
    const uint32_t nk = t.num_keys, np = t.nseg;
    const uint32_t* base = a.kpart + (size_t)t.slot0 * kKeyedTableWords;
    unsigned long long ctot = 0;
    ff stot{0.f, 0.f};
    auto put = [&](uint32_t k, uint32_t c, ff s) {
        const double sd = ff_to_double(s);
        t.counts_out[k] = c;
        t.sums_out[k] = (float)sd;
        if (t.sums64_out) t.sums64_out[k] = sd;
        ctot += c;
        stot = ff_add(stot, s);
    };
    for (uint32_t q = threadIdx.x; q < nk / 4; q += BLOCK) {
        uint4 c{0u, 0u, 0u, 0u};
        ff s[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        uint32_t p = 0;
        for (; p + 4 <= np; p += 4) {
            uint4 cc[4], sv[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const uint32_t* tb = base + (size_t)(p + r) * kKeyedTableWords;
                cc[r] = __ldcg(reinterpret_cast<const uint4*>(tb) + q);
                sv[r] = __ldcg(reinterpret_cast<const uint4*>(tb + kMaxKeys) + q);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                c.x += cc[r].x; c.y += cc[r].y; c.z += cc[r].z; c.w += cc[r].w;
                s[0] = ff_add_f(s[0], __uint_as_float(sv[r].x));
                s[1] = ff_add_f(s[1], __uint_as_float(sv[r].y));
                s[2] = ff_add_f(s[2], __uint_as_float(sv[r].z));
                s[3] = ff_add_f(s[3], __uint_as_float(sv[r].w));
            }
        }
        for (; p < np; ++p) {
            const uint32_t* tb = base + (size_t)p * kKeyedTableWords;
            const uint4 cc = __ldcg(reinterpret_cast<const uint4*>(tb) + q);
            const uint4 sv = __ldcg(reinterpret_cast<const uint4*>(tb + kMaxKeys) + q);
            c.x += cc.x; c.y += cc.y; c.z += cc.z; c.w += cc.w;
            s[0] = ff_add_f(s[0], __uint_as_float(sv.x));
            s[1] = ff_add_f(s[1], __uint_as_float(sv.y));
            s[2] = ff_add_f(s[2], __uint_as_float(sv.z));
            s[3] = ff_add_f(s[3], __uint_as_float(sv.w));
        }
        put(4 * q, c.x, s[0]);
        put(4 * q + 1, c.y, s[1]);
        put(4 * q + 2, c.z, s[2]);
        put(4 * q + 3, c.w, s[3]);
    }
    for (uint32_t k = nk / 4 * 4 + threadIdx.x; k < nk; k += BLOCK) {
        uint32_t c = 0;
        ff s{0.f, 0.f};
        for (uint32_t p = 0; p < np; ++p) {
            const uint32_t* tb = base + (size_t)p * kKeyedTableWords;
            c += __ldcg(tb + k);
            s = ff_add_f(s, __uint_as_float(__ldcg(tb + kMaxKeys + k)));
        }
        put(k, c, s);
    }
    block_reduce_ff_u64<BLOCK>(stot, ctot, sm);
    if (threadIdx.x == 0) {
        const uint32_t fl = atomicExch(&a.task_flags[task], 0u);
        write_result(t.result, ctot, ff_to_double(stot), CUDART_INF_F, -CUDART_INF_F,
                     fl ? SCL_E_KEY_RANGE : SCL_OK, t.n, t.kind);
        a.tickets[task] = 0u;
    }
}

// One keyed piece: pairs [b, e) of task `task`, accumulated into the CTA's
// shared-memory table (count, fp32 sum) and written to the outputs (single
// piece) or to partial slot slot0 + slot; the last writer of a task of at
// most kFoldInKernelMaxPieces pieces folds it.  Returns true in thread 0 if
// it wrote the task's result.
template <int BLOCK, int IPT, bool HASHED, bool FAST>
__device__ __forceinline__ bool keyed_piece(const KernelArgs& a, const DevTask& t, uint32_t task,
                                            uint32_t slot, uint64_t b, uint64_t e,
                                            uint32_t* tab, RedSmem& sm) {
    const int any_bad = keyed_accumulate<BLOCK, IPT, HASHED, FAST>(t, b, e, tab);
    const uint32_t* cnt = tab;
    const float* sum = reinterpret_cast<const float*>(tab + kMaxKeys);
    const uint32_t nk = t.num_keys;
    bool wrote = false;
    if (t.nseg == 1) {
        unsigned long long ctot = 0;
        ff stot{0.f, 0.f};
        // 16 bytes per access where the outputs allow it (uniform branch)
        const bool vec = ((reinterpret_cast<uintptr_t>(t.counts_out) |
                           reinterpret_cast<uintptr_t>(t.sums_out) |
                           reinterpret_cast<uintptr_t>(t.sums64_out)) & 15u) == 0;
        const uint32_t nv = vec ? nk / 4 : 0u;
        for (uint32_t q = threadIdx.x; q < nv; q += BLOCK) {
            const uint4 c = reinterpret_cast<const uint4*>(cnt)[q];
            const float4 s = reinterpret_cast<const float4*>(sum)[q];
            reinterpret_cast<uint4*>(t.counts_out)[q] = c;
            reinterpret_cast<float4*>(t.sums_out)[q] = s;
            if (t.sums64_out) {
                reinterpret_cast<double2*>(t.sums64_out)[2 * q] = make_double2(s.x, s.y);
                reinterpret_cast<double2*>(t.sums64_out)[2 * q + 1] = make_double2(s.z, s.w);
            }
            ctot += (unsigned long long)c.x + c.y + c.z + c.w;
            stot = ff_add_f(ff_add_f(ff_add_f(ff_add_f(stot, s.x), s.y), s.z), s.w);
        }
        for (uint32_t k = nv * 4 + threadIdx.x; k < nk; k += BLOCK) {
            const uint32_t c = cnt[k];
            const float s = sum[k];
            t.counts_out[k] = c;
            t.sums_out[k] = s;
            if (t.sums64_out) t.sums64_out[k] = (double)s;
            ctot += c;
            stot = ff_add_f(stot, s);
        }
        block_reduce_ff_u64<BLOCK>(stot, ctot, sm);
        if (threadIdx.x == 0) {
            write_result(t.result, ctot, ff_to_double(stot), CUDART_INF_F, -CUDART_INF_F,
                         any_bad ? SCL_E_KEY_RANGE : SCL_OK, t.n, t.kind);
            wrote = true;
        }
    } else {
        uint32_t* dst = a.kpart + (size_t)(t.slot0 + slot) * kKeyedTableWords;
        const uint32_t nv = nk / 4;
        for (uint32_t q = threadIdx.x; q < nv; q += BLOCK) {
            __stcg(reinterpret_cast<uint4*>(dst) + q, reinterpret_cast<const uint4*>(cnt)[q]);
            __stcg(reinterpret_cast<uint4*>(dst + kMaxKeys) + q,
                   reinterpret_cast<const uint4*>(sum)[q]);
        }
        for (uint32_t k = nv * 4 + threadIdx.x; k < nk; k += BLOCK) {
            __stcg(dst + k, cnt[k]);
            __stcg(dst + kMaxKeys + k, __float_as_uint(sum[k]));
        }
        if (any_bad && threadIdx.x == 0) atomicOr(&a.task_flags[task], 1u);
        // a task of few pieces: one ticket per written piece table; the CTA
        // that writes the last one folds the task (more pieces: k_keyed_fold)
        if (t.nseg <= kFoldInKernelMaxPieces) {
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) sm.flag = atomicAdd(&a.tickets[task], 1u) == t.nseg - 1;
            __syncthreads();
        }
        if (t.nseg <= kFoldInKernelMaxPieces && sm.flag) {
            __threadfence();
            keyed_fold_task<BLOCK>(a, t, task, sm);
            wrote = threadIdx.x == 0;
        }
    }
    __syncthreads();   // the table is re-zeroed by the next piece
    return wrote;
}

// ------------------------------------------------------- persistent kernel

// Residency targets, as register caps: the streaming-only kernels get a full
// SM of threads (32 registers; the uint32 kernel's 64-bit accumulators would
// otherwise take 40 and cost two CTAs per SM of loads in flight), the mixed
// kernel half of it (64 registers; its table allows 5 CTAs, and without a
// target ptxas takes up to 168 registers), the keyed-only kernel three
// 256-thread CTAs (its fixed-point window's shared memory allows no more).
// At 2 items per thread the 32-register cap would spill; those shapes get 42.
template <int MASK, int BLOCK, int IPT>
constexpr int persistent_min_blocks() {
    return (MASK == M_U32 || MASK == M_F32) ? (IPT >= 4 ? 2048 : 1536) / BLOCK
           : MASK == M_KEYED                ? (BLOCK == 256 ? 3 : 2)
                                            : 1024 / BLOCK;
}

template <int BLOCK, int IPT, int MASK>
__device__ __forceinline__ void persistent_body(const KernelArgs& a) {
    __shared__ RedSmem sm;
    extern __shared__ uint4 dyn_smem[];

    if constexpr (mask_has_keyed(MASK)) {
        // In the mixed kernel the keyed pieces load at most 4 vectors per thread
        // per array: at the streaming shape's 8 they would hold 64 registers of
        // loads and cap the kernel at 2 CTAs per SM.  Keyed results do not
        // depend on the shape (exact counts; sums from shared-memory atomics).
        constexpr int KIPT = (MASK == M_ALL && IPT > 4) ? 4 : IPT;
        // The keyed-only kernel has the shared memory of the fixed-point window.
        constexpr bool FAST = MASK == M_KEYED;
        uint32_t* tab = reinterpret_cast<uint32_t*>(dyn_smem);
        if (a.tasks == nullptr) {
            if (is_keyed(a.single.kind) && blockIdx.x < a.nkeyed_ctas) {
                const uint32_t G = a.nkeyed_ctas;
                const uint64_t b = keyed_single_bound(a.single.n, blockIdx.x, G);
                const uint64_t e = keyed_single_bound(a.single.n, blockIdx.x + 1, G);
                if (a.single.kind == K_KEYED_MIX)
                    keyed_piece<BLOCK, KIPT, true, FAST>(a, a.single, 0u, blockIdx.x, b, e, tab, sm);
                else
                    keyed_piece<BLOCK, KIPT, false, FAST>(a, a.single, 0u, blockIdx.x, b, e, tab, sm);
            }
        } else {
            const uint32_t p0 = a.kp_first[blockIdx.x], p1 = a.kp_first[blockIdx.x + 1];
            for (uint32_t p = p0; p < p1; ++p) {
                const KPiece kp = a.kpieces[p];
                const DevTask t = a.tasks[kp.task];
                if (t.kind == K_KEYED_MIX)
                    keyed_piece<BLOCK, KIPT, true, FAST>(a, t, kp.task, kp.slot, kp.begin, kp.end,
                                                         tab, sm);
                else
                    keyed_piece<BLOCK, KIPT, false, FAST>(a, t, kp.task, kp.slot, kp.begin, kp.end,
                                                          tab, sm);
            }
        }
    }

    if constexpr (mask_has_stream(MASK)) {
        if (a.nseg_stream > 0) {
            if (threadIdx.x == 0) sm.q = atomicAdd(&a.hdr[H_QUEUE], 1u);
            __syncthreads();
            uint32_t q = sm.q;
            while (q < a.nseg_stream) {
                __syncthreads();   // everyone has read sm.q
                if (threadIdx.x == 0) sm.q = atomicAdd(&a.hdr[H_QUEUE], 1u);
                const uint32_t task = a.tasks ? a.seg_task[q] : 0u;
                const DevTask t = a.tasks ? a.tasks[task] : a.single;
                const uint32_t local = q - t.seg_base;
                bool done = false;
                if constexpr (mask_has_u32(MASK)) {
                    if (t.kind == K_U32_IDENT) {
                        stream_segment<BLOCK, IPT, K_U32_IDENT>(a, t, task, local, sm);
                        done = true;
                    } else if (t.kind == K_U32_MIX32) {
                        stream_segment<BLOCK, IPT, K_U32_MIX32>(a, t, task, local, sm);
                        done = true;
                    }
                }
                if constexpr (mask_has_f32(MASK)) {
                    if (!done && t.kind == K_F32_IDENT) {
                        stream_segment<BLOCK, IPT, K_F32_IDENT>(a, t, task, local, sm);
                        done = true;
                    } else if (!done && t.kind == K_F32_POLY3) {
                        stream_segment<BLOCK, IPT, K_F32_POLY3>(a, t, task, local, sm);
                        done = true;
                    }
                }
                if (!done) {   // a kind this instantiation does not contain: host bug
                    if (threadIdx.x == 0) atomicOr(&a.hdr[H_ERROR], 1u);
                    __syncthreads();
                }
                q = sm.q;   // written by thread 0 before the segment's barriers
            }
        }
    }

    // Last CTA out rewinds the segment counter for the next launch.
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t done = atomicAdd(&a.hdr[H_EXIT], 1u);
        if (done == gridDim.x - 1) {
            atomicExch(&a.hdr[H_QUEUE], 0u);
            atomicExch(&a.hdr[H_EXIT], 0u);
            if (a.err_out) *a.err_out = atomicOr(&a.hdr[H_ERROR], 0u);
        }
    }
}

template <int BLOCK, int IPT, int MASK>
__global__ void __launch_bounds__(BLOCK, (persistent_min_blocks<MASK, BLOCK, IPT>()))
    k_persistent(const __grid_constant__ KernelArgs a) {
    persistent_body<BLOCK, IPT, MASK>(a);
}

// The keyed-only kernel held to kKeyedLeanRegs registers per thread, for a
// batch whose streaming tasks run concurrently in kernels of their own: two
// 512-thread CTAs of it take 48 Ki of an SM's 64 Ki registers, so two
// 256-thread streaming CTAs (32 registers) stay resident beside them and
// stream from DRAM while the keyed CTAs are bound by shared-memory atomics.
template <int BLOCK, int IPT>
__global__ void __maxnreg__(kKeyedLeanRegs) k_keyed_lean(const __grid_constant__ KernelArgs a) {
    persistent_body<BLOCK, IPT, M_KEYED>(a);
}

// --------------------------------------------------------- keyed fold pass

// grid (key blocks, fold tasks).  Each thread folds one key over the task's
// piece tables in piece order: count exact in uint32, sum in fp64.
template <int FB>
__global__ void __launch_bounds__(FB) k_keyed_fold(const __grid_constant__ KernelArgs a) {
    static_assert(FB == kFoldBlock, "fold block");
    __shared__ RedSmem sm;
    const uint32_t fi = blockIdx.y;
    const uint32_t task = a.tasks ? a.fold_tasks[fi] : 0u;
    const DevTask t = a.tasks ? a.tasks[task] : a.single;
    const uint32_t nk = t.num_keys;
    const uint32_t nkb = (nk + kFoldBlock - 1) / kFoldBlock;
    if (blockIdx.x >= nkb) return;   // uniform: this task has fewer key blocks

    const uint32_t k = blockIdx.x * kFoldBlock + threadIdx.x;
    unsigned long long ctot = 0;
    ff stot{0.f, 0.f};
    if (k < nk) {
        const uint32_t* src = a.kpart + (size_t)t.slot0 * kKeyedTableWords + k;
        const uint32_t np = t.nseg;
        uint32_t c = 0;
        ff s{0.f, 0.f};
        uint32_t p = 0;
        for (; p + 4 <= np; p += 4) {
            uint32_t cc[4], sv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                cc[q] = __ldcg(src + (size_t)(p + q) * kKeyedTableWords);
                sv[q] = __ldcg(src + (size_t)(p + q) * kKeyedTableWords + kMaxKeys);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                c += cc[q];
                s = ff_add_f(s, __uint_as_float(sv[q]));
            }
        }
        for (; p < np; ++p) {
            c += __ldcg(src + (size_t)p * kKeyedTableWords);
            s = ff_add_f(s, __uint_as_float(__ldcg(src + (size_t)p * kKeyedTableWords + kMaxKeys)));
        }
        const double sd = ff_to_double(s);
        t.counts_out[k] = c;
        t.sums_out[k] = (float)sd;
        if (t.sums64_out) t.sums64_out[k] = sd;
        ctot = c;
        stot = s;
    }
    block_reduce_ff_u64<kFoldBlock>(stot, ctot, sm);
    if (threadIdx.x == 0) {
        StreamPartial* fp = a.fpart + (size_t)fi * (kMaxKeys / kFoldBlock) + blockIdx.x;
        fp->shi = stot.hi;
        fp->slo = stot.lo;
        fp->u = ctot;
        __threadfence();
        const uint32_t prev = atomicAdd(&a.tickets[task], 1u);
        if (prev == nkb - 1) {
            __threadfence();
            ff s{0.f, 0.f};
            unsigned long long c = 0;
            for (uint32_t kb = 0; kb < nkb; ++kb) {
                const StreamPartial* q = a.fpart + (size_t)fi * (kMaxKeys / kFoldBlock) + kb;
                s = ff_add(s, ff{__ldcg(&q->shi), __ldcg(&q->slo)});
                c += __ldcg(reinterpret_cast<const unsigned long long*>(&q->u));
            }
            const uint32_t fl = atomicExch(&a.task_flags[task], 0u);
            write_result(t.result, c, ff_to_double(s), CUDART_INF_F, -CUDART_INF_F,
                         fl ? SCL_E_KEY_RANGE : SCL_OK, t.n, t.kind);
            a.tickets[task] = 0u;
        }
    }
}

// ------------------------------------------------------------- map kernel

template <int BLOCK, int IPT, int KIND, bool ALIGNED>
__global__ void __launch_bounds__(BLOCK) k_map(const void* in, void* out, uint64_t n, float ca,
                                               float cb, float cc) {
    constexpr uint32_t CH = BLOCK * IPT * 4;
    const char* ib = static_cast<const char*>(in);
    char* ob = static_cast<char*>(out);
    const uint64_t nch = ALIGNED ? n / CH : 0;
    for (uint64_t c = blockIdx.x; c < nch; c += gridDim.x) {
        const uint64_t off = (c * CH + (uint64_t)threadIdx.x * 4) * 4;
        uint4 v[IPT];
#pragma unroll
        for (int j = 0; j < IPT; ++j) v[j] = ld_stream_v4(ib + off + (size_t)j * BLOCK * 16);
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            uint4 r;
            if constexpr (KIND == K_F32_POLY3) {
                r.x = __float_as_uint(poly3(__uint_as_float(v[j].x), ca, cb, cc));
                r.y = __float_as_uint(poly3(__uint_as_float(v[j].y), ca, cb, cc));
                r.z = __float_as_uint(poly3(__uint_as_float(v[j].z), ca, cb, cc));
                r.w = __float_as_uint(poly3(__uint_as_float(v[j].w), ca, cb, cc));
            } else {
                r.x = map_u32<KIND>(v[j].x);
                r.y = map_u32<KIND>(v[j].y);
                r.z = map_u32<KIND>(v[j].z);
                r.w = map_u32<KIND>(v[j].w);
            }
            st_stream_v4(ob + off + (size_t)j * BLOCK * 16, r);
        }
    }
    const uint64_t stride = (uint64_t)gridDim.x * BLOCK;
    for (uint64_t i = nch * CH + (uint64_t)blockIdx.x * BLOCK + threadIdx.x; i < n; i += stride) {
        const uint32_t w = ld_stream_b32(ib + i * 4);
        uint32_t r;
        if constexpr (KIND == K_F32_POLY3) r = __float_as_uint(poly3(__uint_as_float(w), ca, cb, cc));
        else r = map_u32<KIND>(w);
        reinterpret_cast<uint32_t*>(ob)[i] = r;
    }
}

// ------------------------------------------------- tree add of k arrays

template <bool F32>
__device__ __forceinline__ uint32_t add1(uint32_t a, uint32_t b) {
    if constexpr (F32) return __float_as_uint(__fadd_rn(__uint_as_float(a), __uint_as_float(b)));
    else return a + b;
}

template <bool F32>
__device__ __forceinline__ uint4 add4(uint4 a, uint4 b) {
    return make_uint4(add1<F32>(a.x, b.x), add1<F32>(a.y, b.y), add1<F32>(a.z, b.z),
                      add1<F32>(a.w, b.w));
}

// Binary-counter tree: level L holds a complete subtree of 2^L leaves exactly
// when bit L of the leaf count is set.  Pushing a leaf carries it upward,
// combining (older level value) + (newer carry), like an increment.
template <bool F32, int LV, typename V>
__device__ __forceinline__ void tree_push(V (&st)[LV], uint32_t& cnt, V x) {
    bool carry = true;   // no early exit: every st[L] index stays a constant
#pragma unroll
    for (int L = 0; L < LV; ++L) {
        const bool occupied = (cnt >> L) & 1u;
        if (carry && occupied) {
            if constexpr (sizeof(V) == 16) x = add4<F32>(st[L], x);
            else x = add1<F32>(st[L], x);
        } else if (carry) {
            st[L] = x;
            carry = false;
        }
    }
    ++cnt;
}

// Leftover subtrees are combined newest (lowest level) first, each older one
// on the left.
template <bool F32, int LV, typename V>
__device__ __forceinline__ V tree_finish(const V (&st)[LV], uint32_t cnt) {
    V acc{};
    bool have = false;
#pragma unroll
    for (int L = 0; L < LV; ++L) {
        if (cnt & (1u << L)) {
            if (!have) {
                acc = st[L];
                have = true;
            } else if constexpr (sizeof(V) == 16) {
                acc = add4<F32>(st[L], acc);
            } else {
                acc = add1<F32>(st[L], acc);
            }
        }
    }
    return acc;
}

// out[i] = tree sum over j < k of in[j][i].  Grid-stride over 128-bit vectors
// (ALIGNED: every array 16-byte aligned), then over the scalar remainder.
// LV stack levels hold up to 2^LV - 1 arrays.
template <bool F32, bool ALIGNED, int LV>
__global__ void __launch_bounds__(256) k_tree_add(const __grid_constant__ TreeArgs a) {
    const uint64_t nv = ALIGNED ? a.n / 4 : 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint32_t k = a.k;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
        uint4 st[LV];
        uint32_t cnt = 0;
        uint32_t j = 0;
        for (; j + 4 <= k; j += 4) {
            uint4 x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = ld_stream_v4(a.in[j + q] + v * 16);
#pragma unroll
            for (int q = 0; q < 4; ++q) tree_push<F32, LV>(st, cnt, x[q]);
        }
        for (; j < k; ++j) tree_push<F32, LV>(st, cnt, ld_stream_v4(a.in[j] + v * 16));
        st_stream_v4(a.out + v * 16, tree_finish<F32, LV>(st, cnt));
    }
    for (uint64_t i = nv * 4 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
         i += stride) {
        uint32_t st[LV];
        uint32_t cnt = 0;
        for (uint32_t j = 0; j < k; ++j)
            tree_push<F32, LV>(st, cnt, ld_stream_b32(a.in[j] + i * 4));
        reinterpret_cast<uint32_t*>(a.out)[i] = tree_finish<F32, LV>(st, cnt);
    }
}

// ------------------------------------------------- large key spaces

// One pair of the direct path: ids below kMaxKeys to the CTA's shared table;
// the others to their packed word (a non-negative value inside the window w)
// or to the count / fp64 adds.
__device__ __forceinline__ void large_add(uint32_t k, uint32_t vbits, const LargeKeyedArgs& a,
                                          const LargeFix& w, uint32_t* hc, float* hs,
                                          float* head, uint32_t& bad, uint32_t& npk) {
    const float v = __uint_as_float(vbits);
    if (k >= a.num_keys) {
        bad = 1u;
    } else if (k < kMaxKeys) {
        atomicAdd(&hc[k], 1u);
        atomicAdd(k < kKeyedHead ? &head[k] : &hs[k], v);
    } else if (w.on && vbits - w.lo < w.span) {   // a negative value's bits are never inside
        atomicAdd(&a.packed[k], (1ull << kPackedCountShift) +
                                    (unsigned long long)__float2uint_rn(v * w.scale));
        ++npk;
    } else {
        atomicAdd(&a.counts[k], 1u);
        atomicAdd(&a.sums64[k], (double)v);
    }
}

// Whether a guarded kernel of the repair chain has nothing to do.
__device__ __forceinline__ bool large_skip(const LargeKeyedArgs& a) {
    return a.guard && !(__ldcg(a.bad) & kLargeRepair);
}

// The packed window of a partition (one CTA): B is the power of two above the
// largest finite non-negative value among the first kPackedScaleSample
// values, F = 25 - log2 B, packed values lie in [B/256, B).  No window (on =
// 0) when that value is 0 or outside [2^-90, 2^90).
template <int FB>
__global__ void __launch_bounds__(FB) k_large_scale(const __grid_constant__ LargeKeyedArgs a) {
    __shared__ uint32_t wm[FB / 32];
    const uint64_t ns = min(a.n, (uint64_t)kPackedScaleSample);
    uint32_t m = 0;
    for (uint64_t i = threadIdx.x; i < ns; i += FB) {
        const uint32_t b = ld_stream_b32(a.vals + i * 4);
        if (b < 0x7f800000u) m = max(m, b);   // finite and not negative
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < FB / 32; ++q) m = max(m, wm[q]);
        LargeFix f;
        f.scale = f.inv = 0.f;
        f.lo = f.span = 0u;
        f.on = m >= 0x12800000u && m < 0x6c800000u;   // [2^-90, 2^90)
        if (f.on) {
            const int e1 = (int)(m >> 23) - 127 + 1;   // B = 2^e1
            const int F = 25 - e1;
            f.scale = __uint_as_float((uint32_t)(F + 127) << 23);
            f.inv = __uint_as_float((uint32_t)(127 - F) << 23);
            f.lo = (uint32_t)(e1 - 8 + 127) << 23;
            f.span = ((uint32_t)(e1 + 127) << 23) - f.lo;
        }
        f.pad = 0u;
        f.npacked = 0ull;
        f.ndecoded = 0ull;
        *a.fix = f;
    }
}

// First kernel of the repair chain: the outputs and the result back to zero
// (the guarded direct pass and finishing pass follow, without packing).
template <int FB>
__global__ void __launch_bounds__(FB) k_large_repair_zero(const __grid_constant__ LargeKeyedArgs a) {
    if (large_skip(a)) return;
    for (uint64_t k = (uint64_t)blockIdx.x * FB + threadIdx.x; k < a.num_keys;
         k += (uint64_t)gridDim.x * FB) {
        a.counts[k] = 0u;
        a.sums64[k] = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x < sizeof(scl_result) / 4)
        reinterpret_cast<uint32_t*>(a.result)[threadIdx.x] = 0u;
}

// Grid-stride over pieces of kDirectPiece pairs; each piece zeroes the shared
// hot table (and the head copies of its first ids), accumulates, and flushes
// its non-zero entries to global memory.
template <bool ALIGNED>
__global__ void __launch_bounds__(256) k_keyed_large(const __grid_constant__ LargeKeyedArgs a) {
    __shared__ uint32_t hc[kMaxKeys];
    __shared__ float hs[kMaxKeys];
    __shared__ float heads[kKeyedHeadWords(256)];
    if (large_skip(a)) return;
    LargeFix w;
    w.on = 0u;
    w.lo = w.span = 0u;
    w.scale = 0.f;
    if (a.packed) w = *a.fix;
    uint32_t npk = 0;
    float* head = heads + ((threadIdx.x >> 5) * kKeyedHeadClasses +
                           (threadIdx.x & (kKeyedHeadClasses - 1))) * kKeyedHeadStride;
    const uint32_t hot = min(a.num_keys, kMaxKeys);
    const uint64_t npieces = (a.n + kDirectPiece - 1) / kDirectPiece;
    uint32_t bad = 0;
    for (uint64_t pc = blockIdx.x; pc < npieces; pc += gridDim.x) {
        for (uint32_t i = threadIdx.x; i < hot; i += blockDim.x) {
            hc[i] = 0u;
            hs[i] = 0.f;
        }
        for (uint32_t i = threadIdx.x; i < kKeyedHeadWords(256); i += blockDim.x) heads[i] = 0.f;
        __syncthreads();
        const uint64_t b = pc * kDirectPiece;
        const uint64_t e = min(b + kDirectPiece, a.n);
        uint64_t i = b;
        if constexpr (ALIGNED) {
            constexpr uint32_t CH = 256 * 4 * 4;
            for (; i + CH <= e; i += CH) {
                uint4 kv[4], vv[4];
                const uint64_t off = (i + (uint64_t)threadIdx.x * 4) * 4;
#pragma unroll
                for (int j = 0; j < 4; ++j) kv[j] = ld_stream_v4(a.keys + off + (size_t)j * 4096);
#pragma unroll
                for (int j = 0; j < 4; ++j) vv[j] = ld_stream_v4(a.vals + off + (size_t)j * 4096);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    large_add(kv[j].x, vv[j].x, a, w, hc, hs, head, bad, npk);
                    large_add(kv[j].y, vv[j].y, a, w, hc, hs, head, bad, npk);
                    large_add(kv[j].z, vv[j].z, a, w, hc, hs, head, bad, npk);
                    large_add(kv[j].w, vv[j].w, a, w, hc, hs, head, bad, npk);
                }
            }
        }
        for (uint64_t g = i + threadIdx.x; g < e; g += blockDim.x)
            large_add(ld_stream_b32(a.keys + g * 4), ld_stream_b32(a.vals + g * 4), a, w, hc, hs,
                      head, bad, npk);
        __syncthreads();
        fold_head_copies(heads, hs, min(hot, kKeyedHead));
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < hot; k += blockDim.x) {
            const uint32_t c = hc[k];
            if (c) {
                atomicAdd(&a.counts[k], c);
                atomicAdd(&a.sums64[k], (double)hs[k]);
            }
        }
        __syncthreads();   // the table is zeroed again by the next piece
    }
    if (bad) atomicOr(a.bad, 1u);
    if (a.packed) {
        const uint32_t wn = __reduce_add_sync(0xffffffffu, npk);
        if ((threadIdx.x & 31) == 0 && wn) atomicAdd(&a.fix->npacked, (unsigned long long)wn);
    }
}

// Finishing pass: the packed words decoded into the count / fp64 tables (if
// any), fp32 sums, totals (count exact, value sum fp64) and status.  The last
// CTA writes f32_sum, checks that the decoded counts add up to the packed adds
// (else kLargeRepair: the guarded repair chain follows) and resets the ticket.
template <int FB>
__global__ void __launch_bounds__(FB) k_keyed_large_finish(const __grid_constant__ LargeKeyedArgs a) {
    static_assert(FB == 256, "finish block");
    __shared__ RedSmem sm;
    if (large_skip(a)) return;
    const double inv = a.packed ? (double)a.fix->inv : 0.0;
    unsigned long long c = 0, cp = 0;
    ff s{0.f, 0.f};
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.num_keys;
         k += (uint64_t)gridDim.x * blockDim.x) {
        double v = a.sums64[k];
        uint32_t ck = a.counts[k];
        if (a.packed) {
            const unsigned long long w = a.packed[k];
            if (w) {
                const uint32_t pc = (uint32_t)(w >> kPackedCountShift);
                const unsigned long long q = w & ((1ull << kPackedCountShift) - 1);
                cp += pc;
                ck += pc;
                v += (double)q * inv;
                a.counts[k] = ck;
                a.sums64[k] = v;
            }
        }
        a.sums32[k] = (float)v;
        c += ck;
        s = ff_add(s, ff_of_double(v));
    }
    float d0 = CUDART_INF_F, d1 = -CUDART_INF_F;
    block_reduce_ff<256>(s, d0, d1, sm);
    c = block_sum_u64<256>(c, sm);
    if (a.packed) cp = block_sum_u64<256>(cp, sm);
    if (threadIdx.x == 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.result->u64_sum), c);
        atomicAdd(&a.result->f64_sum, ff_to_double(s));
        if (a.packed && cp) atomicAdd(&a.fix->ndecoded, cp);
        __threadfence();
        if (atomicAdd(a.ticket, 1u) == gridDim.x - 1) {
            __threadfence();
            if (a.packed && __ldcg(&a.fix->ndecoded) != __ldcg(&a.fix->npacked))
                atomicOr(a.bad, kLargeRepair);
            scl_result* r = a.result;
            const double tot = __ldcg(&r->f64_sum);
            r->f32_sum = (float)tot;
            r->f32_min = CUDART_INF_F;
            r->f32_max = -CUDART_INF_F;
            // bit 0: a key out of range; bit 1: the bucket-partitioned path
            // counted the keys differently in its two reads (they changed);
            // bit 2: one of its bounded waits ran out
            const uint32_t bad = __ldcg(a.bad) & 7u;
            r->status = (bad & 4u) ? SCL_E_TIMEOUT
                        : (bad & 2u) ? SCL_E_STATE : bad ? SCL_E_KEY_RANGE : SCL_OK;
            r->n = a.n;
            r->kind = K_KEYED;
            *a.ticket = 0u;
        }
    }
}

}  // namespace dev
}  // namespace scl

// Instantiate the persistent kernel for one mask over the tuned shapes and
// define kernel_table_<name>().
#define SCL_DYN(M)                                             \
    ((M) == scl::M_KEYED          ? scl::kKeyedFastSmemBytes     \
     : scl::mask_has_keyed(M)     ? scl::kKeyedSmemBytes         \
                                  : 0)
#define SCL_SHAPE(M, B, I) {M, B, I, (const void*)&scl::dev::k_persistent<B, I, M>, SCL_DYN(M), 0, 0}
#define SCL_LEAN_SHAPE(B, I)                                                         \
    {scl::M_KEYED, B, I, (const void*)&scl::dev::k_keyed_lean<B, I>, scl::kKeyedFastSmemBytes, \
     scl::PATH_LEAN, 0}
#define SCL_DEFINE_TABLE(NAME, M)                                                   \
    namespace scl {                                                                 \
    const KernelEntry* kernel_table_##NAME(int* count) {                            \
        static const KernelEntry tab[] = {SCL_SHAPE(M, 256, 2), SCL_SHAPE(M, 256, 4), \
                                          SCL_SHAPE(M, 256, 8), SCL_SHAPE(M, 512, 2), \
                                          SCL_SHAPE(M, 512, 4), SCL_SHAPE(M, 512, 8)}; \
        *count = (int)(sizeof(tab) / sizeof(tab[0]));                               \
        return tab;                                                                 \
    }                                                                               \
    }
