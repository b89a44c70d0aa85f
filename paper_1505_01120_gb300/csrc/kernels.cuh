// kernels.cuh -- sm_103a kernels of the SparkCL per-partition path.
//
//   k_persistent<BLOCK, IPT, MASK>  MapCLPartition + ReduceCL fused (Sec. 3.1.3
//                                   items 2-3): every element of a partition is
//                                   mapped by the catalogue kernel (the run()
//                                   body of Sec. 3.1.1.2) and folded, in one
//                                   HBM pass, by a persistent grid.
//   k_keyed_fold                    second pass of the keyed reduce (Sec. 3.2.3):
//                                   folds the per-piece tables of keyed tasks.
//   k_map<BLOCK, IPT, KIND, ALIGNED> MapCL with a materialised output array
//                                   (Sec. 3.1.3 item 1; Fig. 3's c[gid] = f(a[gid])).
//
// Data path: 128-bit vector loads (ld.global.nc, no L1 allocation, 256-byte L2
// prefetch) of IPT independent vectors per thread before any use, so a CTA
// has BLOCK*IPT*16 bytes in flight; streaming sums are fp32 per thread per
// chunk, fp64 across chunks, a fixed-order warp-butterfly and block tree, one
// partial per segment and one atomic ticket per task; the last CTA of a task
// folds the segment partials in slot order (deterministic).
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

// ------------------------------------------------------ block reductions

struct RedSmem {
    double d[32];
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
__device__ __forceinline__ void block_reduce_f(double& s, float& mn, float& mx, RedSmem& sm) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sm.d[w] = s;
        sm.mn[w] = mn;
        sm.mx[w] = mx;
    }
    __syncthreads();
    const bool in = l < BLOCK / 32;
    s = in ? sm.d[l] : 0.0;
    mn = in ? sm.mn[l] : CUDART_INF_F;
    mx = in ? sm.mx[l] : -CUDART_INF_F;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
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
    double dsum = 0.0;
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
                dsum += (double)cs;
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
        if constexpr (F32) dsum += (double)cs;
    }

    if constexpr (F32) block_reduce_f<BLOCK>(dsum, mn, mx, sm);
    else usum = block_sum_u64<BLOCK>(usum, sm);
    if constexpr (!F32) dsum = (double)usum;

    if (t.nseg == 1) {
        if (threadIdx.x == 0)
            write_result(t.result, usum, dsum, F32 ? mn : 0.f, F32 ? mx : 0.f, SCL_OK, t.n, t.kind);
        return threadIdx.x == 0;
    }
    if (threadIdx.x == 0) {
        StreamPartial* sp = a.spart + t.slot0 + local;
        sp->s = dsum;
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
    double fs = 0.0;
    unsigned long long fu = 0;
    float fmn = CUDART_INF_F, fmx = -CUDART_INF_F;
    for (uint32_t s = threadIdx.x; s < t.nseg; s += BLOCK) {
        const StreamPartial* sp = a.spart + t.slot0 + s;
        if constexpr (F32) {
            fs += __ldcg(&sp->s);
            fmn = fminf(fmn, __ldcg(&sp->mn));
            fmx = fmaxf(fmx, __ldcg(&sp->mx));
        } else {
            fu += __ldcg(reinterpret_cast<const unsigned long long*>(&sp->u));
        }
    }
    if constexpr (F32) block_reduce_f<BLOCK>(fs, fmn, fmx, sm);
    else {
        fu = block_sum_u64<BLOCK>(fu, sm);
        fs = (double)fu;
    }
    if (threadIdx.x == 0) {
        write_result(t.result, fu, fs, F32 ? fmn : 0.f, F32 ? fmx : 0.f, SCL_OK, t.n, t.kind);
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

// Pairs [b, e) of a keyed task accumulated into the CTA's shared-memory table
// (count[kMaxKeys] then fp32 sum[kMaxKeys], then the head copies), zeroed
// first; the head copies are folded into the table at the end.  Returns, in
// every thread, whether any key was out of range.  Ends with a barrier.
template <int BLOCK, int IPT, bool HASHED>
__device__ __forceinline__ int keyed_accumulate(const DevTask& t, uint64_t b, uint64_t e,
                                                uint32_t* tab) {
    constexpr uint32_t CH = BLOCK * IPT * 4;
    static_assert(kKeyedHeadWords(BLOCK) * 4 + kKeyedTableWords * 4 <= kKeyedSmemBytes, "smem");
    uint32_t* cnt = tab;
    float* sum = reinterpret_cast<float*>(tab + kMaxKeys);
    float* heads = reinterpret_cast<float*>(tab + kKeyedTableWords);
    float* head = heads + ((threadIdx.x >> 5) * kKeyedHeadClasses +
                           (threadIdx.x & (kKeyedHeadClasses - 1))) * kKeyedHeadStride;
    const uint32_t nk = t.num_keys;
    for (uint32_t k = threadIdx.x; k < nk; k += BLOCK) {
        cnt[k] = 0u;
        sum[k] = 0.f;
    }
    if (!HASHED)
        for (uint32_t i = threadIdx.x; i < kKeyedHeadWords(BLOCK); i += BLOCK) heads[i] = 0.f;
    __syncthreads();

    const char* kb = static_cast<const char*>(t.in0);
    const char* vb = static_cast<const char*>(t.in1);
    uint32_t bad = 0;
    uint64_t i = b;
    if (t.flags & TF_ALIGNED) {
        for (; i + CH <= e; i += CH) {
            uint4 kv[IPT], vv[IPT];
            const uint64_t off = (i + (uint64_t)threadIdx.x * 4) * 4;
#pragma unroll
            for (int j = 0; j < IPT; ++j) kv[j] = ld_stream_v4(kb + off + (size_t)j * BLOCK * 16);
#pragma unroll
            for (int j = 0; j < IPT; ++j) vv[j] = ld_stream_v4(vb + off + (size_t)j * BLOCK * 16);
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                keyed_add<HASHED>(kv[j].x, vv[j].x, nk, cnt, sum, head, bad);
                keyed_add<HASHED>(kv[j].y, vv[j].y, nk, cnt, sum, head, bad);
                keyed_add<HASHED>(kv[j].z, vv[j].z, nk, cnt, sum, head, bad);
                keyed_add<HASHED>(kv[j].w, vv[j].w, nk, cnt, sum, head, bad);
            }
        }
    }
    for (; i < e; i += CH) {
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const uint64_t g = i + ((uint64_t)j * BLOCK + threadIdx.x) * 4;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (g + q < e)
                    keyed_add<HASHED>(ld_stream_b32(kb + (g + q) * 4),
                                      ld_stream_b32(vb + (g + q) * 4), nk, cnt, sum, head, bad);
        }
    }
    const int any_bad = __syncthreads_or((int)bad);
    if (!HASHED) {
        fold_head_copies(heads, sum, min(nk, kKeyedHead));
        __syncthreads();
    }
    return any_bad;
}

// One keyed piece: pairs [b, e) of task `task`, accumulated into the CTA's
// shared-memory table (count, fp32 sum) and written to the outputs (single
// piece) or to partial slot slot0 + slot.  Returns true in thread 0 if it
// wrote the task's result (single piece).
template <int BLOCK, int IPT, bool HASHED>
__device__ __forceinline__ bool keyed_piece(const KernelArgs& a, const DevTask& t, uint32_t task,
                                            uint32_t slot, uint64_t b, uint64_t e,
                                            uint32_t* tab, RedSmem& sm) {
    const int any_bad = keyed_accumulate<BLOCK, IPT, HASHED>(t, b, e, tab);
    const uint32_t* cnt = tab;
    const float* sum = reinterpret_cast<const float*>(tab + kMaxKeys);
    const uint32_t nk = t.num_keys;
    bool wrote = false;
    if (t.nseg == 1) {
        unsigned long long ctot = 0;
        double stot = 0.0;
        for (uint32_t k = threadIdx.x; k < nk; k += BLOCK) {
            const uint32_t c = cnt[k];
            const float s = sum[k];
            t.counts_out[k] = c;
            t.sums_out[k] = s;
            if (t.sums64_out) t.sums64_out[k] = (double)s;
            ctot += c;
            stot += (double)s;
        }
        float dummy0 = CUDART_INF_F, dummy1 = -CUDART_INF_F;
        block_reduce_f<BLOCK>(stot, dummy0, dummy1, sm);
        ctot = block_sum_u64<BLOCK>(ctot, sm);
        if (threadIdx.x == 0) {
            write_result(t.result, ctot, stot, CUDART_INF_F, -CUDART_INF_F,
                         any_bad ? SCL_E_KEY_RANGE : SCL_OK, t.n, t.kind);
            wrote = true;
        }
    } else {
        uint32_t* dst = a.kpart + (size_t)(t.slot0 + slot) * kKeyedTableWords;
        for (uint32_t k = threadIdx.x; k < nk; k += BLOCK) {
            __stcg(dst + k, cnt[k]);
            __stcg(dst + kMaxKeys + k, __float_as_uint(sum[k]));
        }
        if (any_bad && threadIdx.x == 0) atomicOr(&a.task_flags[task], 1u);
    }
    __syncthreads();   // the table is re-zeroed by the next piece
    return wrote;
}

// ------------------------------------------------------- persistent kernel

// Residency targets, as register caps: the streaming-only kernels get a full
// SM of threads (32 registers; the uint32 kernel's 64-bit accumulators would
// otherwise take 40 and cost two CTAs per SM of loads in flight), kernels
// with a keyed table half of it (64 registers; the table allows 6 CTAs, and
// without a target ptxas takes up to 168 registers for the mixed kernel).
// At 2 items per thread the 32-register cap would spill; those shapes get 42.
template <int MASK, int BLOCK, int IPT>
constexpr int persistent_min_blocks() {
    return (MASK == M_U32 || MASK == M_F32) ? (IPT >= 4 ? 2048 : 1536) / BLOCK : 1024 / BLOCK;
}

template <int BLOCK, int IPT, int MASK>
__global__ void __launch_bounds__(BLOCK, (persistent_min_blocks<MASK, BLOCK, IPT>()))
    k_persistent(const __grid_constant__ KernelArgs a) {
    __shared__ RedSmem sm;
    extern __shared__ uint4 dyn_smem[];

    if constexpr (mask_has_keyed(MASK)) {
        // In the mixed kernel the keyed pieces load at most 4 vectors per thread
        // per array: at the streaming shape's 8 they would hold 64 registers of
        // loads and cap the kernel at 2 CTAs per SM.  Keyed results do not
        // depend on the shape (exact counts; sums from shared-memory atomics).
        constexpr int KIPT = (MASK == M_ALL && IPT > 4) ? 4 : IPT;
        uint32_t* tab = reinterpret_cast<uint32_t*>(dyn_smem);
        if (a.tasks == nullptr) {
            if (is_keyed(a.single.kind) && blockIdx.x < a.nkeyed_ctas) {
                const uint32_t G = a.nkeyed_ctas;
                const uint64_t b = keyed_single_bound(a.single.n, blockIdx.x, G);
                const uint64_t e = keyed_single_bound(a.single.n, blockIdx.x + 1, G);
                if (a.single.kind == K_KEYED_MIX)
                    keyed_piece<BLOCK, KIPT, true>(a, a.single, 0u, blockIdx.x, b, e, tab, sm);
                else
                    keyed_piece<BLOCK, KIPT, false>(a, a.single, 0u, blockIdx.x, b, e, tab, sm);
            }
        } else {
            const uint32_t p0 = a.kp_first[blockIdx.x], p1 = a.kp_first[blockIdx.x + 1];
            for (uint32_t p = p0; p < p1; ++p) {
                const KPiece kp = a.kpieces[p];
                const DevTask t = a.tasks[kp.task];
                if (t.kind == K_KEYED_MIX)
                    keyed_piece<BLOCK, KIPT, true>(a, t, kp.task, kp.slot, kp.begin, kp.end, tab, sm);
                else
                    keyed_piece<BLOCK, KIPT, false>(a, t, kp.task, kp.slot, kp.begin, kp.end, tab, sm);
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
    double stot = 0.0;
    if (k < nk) {
        const uint32_t* src = a.kpart + (size_t)t.slot0 * kKeyedTableWords + k;
        const uint32_t np = t.nseg;
        uint32_t c = 0;
        double s = 0.0;
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
                s += (double)__uint_as_float(sv[q]);
            }
        }
        for (; p < np; ++p) {
            c += __ldcg(src + (size_t)p * kKeyedTableWords);
            s += (double)__uint_as_float(__ldcg(src + (size_t)p * kKeyedTableWords + kMaxKeys));
        }
        t.counts_out[k] = c;
        t.sums_out[k] = (float)s;
        if (t.sums64_out) t.sums64_out[k] = s;
        ctot = c;
        stot = s;
    }
    float d0 = CUDART_INF_F, d1 = -CUDART_INF_F;
    block_reduce_f<kFoldBlock>(stot, d0, d1, sm);
    ctot = block_sum_u64<kFoldBlock>(ctot, sm);
    if (threadIdx.x == 0) {
        StreamPartial* fp = a.fpart + (size_t)fi * (kMaxKeys / kFoldBlock) + blockIdx.x;
        fp->s = stot;
        fp->u = ctot;
        __threadfence();
        const uint32_t prev = atomicAdd(&a.tickets[task], 1u);
        if (prev == nkb - 1) {
            __threadfence();
            double s = 0.0;
            unsigned long long c = 0;
            for (uint32_t kb = 0; kb < nkb; ++kb) {
                const StreamPartial* q = a.fpart + (size_t)fi * (kMaxKeys / kFoldBlock) + kb;
                s += __ldcg(&q->s);
                c += __ldcg(reinterpret_cast<const unsigned long long*>(&q->u));
            }
            const uint32_t fl = atomicExch(&a.task_flags[task], 0u);
            write_result(t.result, c, s, CUDART_INF_F, -CUDART_INF_F,
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

__device__ __forceinline__ void large_add(uint32_t k, uint32_t vbits, const LargeKeyedArgs& a,
                                          uint32_t* hc, float* hs, float* head, uint32_t& bad) {
    const float v = __uint_as_float(vbits);
    if (k >= a.num_keys) {
        bad = 1u;
    } else if (k < kMaxKeys) {
        atomicAdd(&hc[k], 1u);
        atomicAdd(k < kKeyedHead ? &head[k] : &hs[k], v);
    } else {
        atomicAdd(&a.counts[k], 1u);
        atomicAdd(&a.sums64[k], (double)v);
    }
}

// Grid-stride over pieces of kLargePiece pairs; each piece zeroes the shared
// hot table (and the head copies of its first ids), accumulates, and flushes
// its non-zero entries to global memory.
template <bool ALIGNED>
__global__ void __launch_bounds__(256) k_keyed_large(const __grid_constant__ LargeKeyedArgs a) {
    __shared__ uint32_t hc[kMaxKeys];
    __shared__ float hs[kMaxKeys];
    __shared__ float heads[kKeyedHeadWords(256)];
    float* head = heads + ((threadIdx.x >> 5) * kKeyedHeadClasses +
                           (threadIdx.x & (kKeyedHeadClasses - 1))) * kKeyedHeadStride;
    const uint32_t hot = min(a.num_keys, kMaxKeys);
    const uint64_t npieces = (a.n + kLargePiece - 1) / kLargePiece;
    uint32_t bad = 0;
    for (uint64_t pc = blockIdx.x; pc < npieces; pc += gridDim.x) {
        for (uint32_t i = threadIdx.x; i < hot; i += blockDim.x) {
            hc[i] = 0u;
            hs[i] = 0.f;
        }
        for (uint32_t i = threadIdx.x; i < kKeyedHeadWords(256); i += blockDim.x) heads[i] = 0.f;
        __syncthreads();
        const uint64_t b = pc * kLargePiece;
        const uint64_t e = min(b + kLargePiece, a.n);
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
                    large_add(kv[j].x, vv[j].x, a, hc, hs, head, bad);
                    large_add(kv[j].y, vv[j].y, a, hc, hs, head, bad);
                    large_add(kv[j].z, vv[j].z, a, hc, hs, head, bad);
                    large_add(kv[j].w, vv[j].w, a, hc, hs, head, bad);
                }
            }
        }
        for (uint64_t g = i + threadIdx.x; g < e; g += blockDim.x)
            large_add(ld_stream_b32(a.keys + g * 4), ld_stream_b32(a.vals + g * 4), a, hc, hs,
                      head, bad);
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
}

// Finishing pass: fp32 sums, totals (count exact, value sum fp64) and status.
// The last CTA writes f32_sum and resets the ticket.
template <int FB>
__global__ void __launch_bounds__(FB) k_keyed_large_finish(const __grid_constant__ LargeKeyedArgs a) {
    static_assert(FB == 256, "finish block");
    __shared__ RedSmem sm;
    unsigned long long c = 0;
    double s = 0.0;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.num_keys;
         k += (uint64_t)gridDim.x * blockDim.x) {
        const double v = a.sums64[k];
        a.sums32[k] = (float)v;
        c += a.counts[k];
        s += v;
    }
    float d0 = CUDART_INF_F, d1 = -CUDART_INF_F;
    block_reduce_f<256>(s, d0, d1, sm);
    c = block_sum_u64<256>(c, sm);
    if (threadIdx.x == 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.result->u64_sum), c);
        atomicAdd(&a.result->f64_sum, s);
        __threadfence();
        if (atomicAdd(a.ticket, 1u) == gridDim.x - 1) {
            __threadfence();
            scl_result* r = a.result;
            const double tot = __ldcg(&r->f64_sum);
            r->f32_sum = (float)tot;
            r->f32_min = CUDART_INF_F;
            r->f32_max = -CUDART_INF_F;
            // bit 0: a key out of range; bit 1: the bucket-partitioned path
            // counted the keys differently in its two reads (they changed);
            // bit 2: one of its bounded waits ran out
            const uint32_t bad = __ldcg(a.bad);
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
#define SCL_DYN(M) (scl::mask_has_keyed(M) ? scl::kKeyedSmemBytes : 0)
#define SCL_SHAPE(M, B, I) {M, B, I, (const void*)&scl::dev::k_persistent<B, I, M>, SCL_DYN(M), 0, 0}
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
