// kernels_tma.cuh -- the streaming map/reduce as a TMA bulk-copy pipeline.
//
// k_stream_tma<CB, IPT, STAGES, MASK>: warp 0 is the producer, warps
// 1..CB/32 are consumers (CB consumer threads).  One producer lane pulls
// segments from the global counter, reads the task descriptor, and for every
// chunk of CB*IPT*4 elements waits for a free ring stage, writes the stage's
// metadata and issues one cp.async.bulk global->shared copy that completes on
// the stage's "full" mbarrier.  Consumers wait on "full", map and accumulate
// from shared memory with the same per-thread element mapping and the same
// fp32/fp64 association as k_persistent<CB, IPT>, release the stage on its
// "empty" mbarrier, and at a segment's last chunk reduce among themselves
// (named barrier 1) into the segment's slot; the last segment's CTA folds the
// task.  Results are bit-identical to the LDG kernel of the same (CB, IPT).
//
// Ragged last chunks and unaligned partitions go "direct": the producer
// only signals the stage and consumers read global memory with masked loads.
//
// Every mbarrier wait is bounded (about one second of clock64 cycles); on
// expiry the thread sets H_ERROR bit 2 and stops, after waiting (bounded) for
// the copies it issued.  The host reports that as SCL_E_TIMEOUT.
#pragma once

#include "kernels.cuh"

namespace scl {
namespace dev {

constexpr long long kWaitCycles = 2000000000ll;   // ~1 s at 2 GHz
constexpr uint32_t kErrTimeout = 4u;
constexpr uint32_t kRun = 4;   // segments per producer grab

enum StageFlags : uint32_t { SF_LAST = 1u, SF_DIRECT = 2u, SF_END = 4u };

struct alignas(16) StageMeta {
    const char* gptr;       // global address of the chunk's first element
    scl_result* result;
    uint64_t n;             // task length
    uint32_t task, local, nvalid, flags;
    uint32_t kind, nseg, slot0;
    float coef[3];
};
static_assert(sizeof(StageMeta) == 64, "StageMeta layout");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t* err) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) {
            atomicOr(err, kErrTimeout);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

template <int NT>
__device__ __forceinline__ void named_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

// Block reductions over the CB consumer threads (tid = consumer index), the
// same butterfly-then-warp-totals order as block_sum_u64 / block_reduce_ff.
template <int CB>
__device__ __forceinline__ unsigned long long csum_u64(unsigned long long v, uint32_t tid,
                                                       RedSmem& sm) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = tid >> 5, l = tid & 31;
    if (l == 0) sm.u[w] = v;
    named_sync<CB>();
    v = (l < CB / 32) ? sm.u[l] : 0ull;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    named_sync<CB>();
    return v;
}

template <int CB>
__device__ __forceinline__ void creduce_ff(ff& s, float& mn, float& mx, uint32_t tid,
                                           RedSmem& sm) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s = ff_add(s, ff_shfl_xor(s, o));
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const int w = tid >> 5, l = tid & 31;
    if (l == 0) {
        sm.shi[w] = s.hi;
        sm.slo[w] = s.lo;
        sm.mn[w] = mn;
        sm.mx[w] = mx;
    }
    named_sync<CB>();
    const bool in = l < CB / 32;
    s = in ? ff{sm.shi[l], sm.slo[l]} : ff{0.f, 0.f};
    mn = in ? sm.mn[l] : CUDART_INF_F;
    mx = in ? sm.mx[l] : -CUDART_INF_F;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s = ff_add(s, ff_shfl_xor(s, o));
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    named_sync<CB>();
}

template <int CB, int IPT, int STAGES>
struct TmaLayout {
    static constexpr uint32_t kChunk = CB * IPT * 4;            // elements per stage
    static constexpr uint32_t kStageBytes = kChunk * 4;
    static constexpr uint32_t kData = 0;
    static constexpr uint32_t kMeta = kStageBytes * STAGES;
    static constexpr uint32_t kFull = kMeta + sizeof(StageMeta) * STAGES;
    static constexpr uint32_t kEmpty = kFull + 8 * STAGES;
    static constexpr uint32_t kBytes = kEmpty + 8 * STAGES;
};

// Accumulate one chunk (stage) into the consumer's running sums.
template <int CB, int IPT, int KIND>
__device__ __forceinline__ void consume_chunk(const StageMeta& m, const char* stage,
                                              uint32_t tid, unsigned long long& usum,
                                              ff& fsum, float& mn, float& mx) {
    constexpr bool F32 = (KIND == K_F32_IDENT || KIND == K_F32_POLY3);
    const float ca = m.coef[0], cb = m.coef[1], cc = m.coef[2];
    if (!(m.flags & SF_DIRECT)) {
        uint4 v[IPT];
#pragma unroll
        for (int j = 0; j < IPT; ++j)
            v[j] = *reinterpret_cast<const uint4*>(stage + ((size_t)j * CB + tid) * 16);
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
            for (int j = 0; j < IPT; ++j)
                usum += (unsigned long long)map_u32<KIND>(v[j].x) +
                        (unsigned long long)map_u32<KIND>(v[j].y) +
                        (unsigned long long)map_u32<KIND>(v[j].z) +
                        (unsigned long long)map_u32<KIND>(v[j].w);
        }
        return;
    }
    // direct: masked global loads, same element mapping
    const uint32_t nv = m.nvalid;
    float cs = 0.f;
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const uint32_t g = ((uint32_t)j * CB + tid) * 4;
        uint32_t w[4];
        bool ok[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            ok[q] = g + q < nv;
            w[q] = ok[q] ? ld_stream_b32(m.gptr + (size_t)(g + q) * 4) : 0u;
        }
        if constexpr (F32) {
            float ys[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float y = map_f32<KIND>(__uint_as_float(w[q]), ca, cb, cc);
                ys[q] = ok[q] ? y : 0.f;
                if (ok[q]) {
                    mn = fminf(mn, y);
                    mx = fmaxf(mx, y);
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

// Segment end: reduce among consumers, write the slot or the result, take the
// task's ticket, fold if last.  Same order as stream_segment's epilogue.
template <int CB, bool F32>
__device__ __forceinline__ void segment_end(const KernelArgs& a, const StageMeta& m,
                                            uint32_t tid, unsigned long long usum, ff fsum,
                                            float mn, float mx, RedSmem& sm) {
    if constexpr (F32) creduce_ff<CB>(fsum, mn, mx, tid, sm);
    else usum = csum_u64<CB>(usum, tid, sm);
    if (m.nseg == 1) {
        if (tid == 0)
            write_result(m.result, usum, F32 ? ff_to_double(fsum) : (double)usum,
                         F32 ? mn : 0.f, F32 ? mx : 0.f, SCL_OK, m.n, m.kind);
        return;
    }
    if (tid == 0) {
        StreamPartial* sp = a.spart + m.slot0 + m.local;
        sp->shi = fsum.hi;
        sp->slo = fsum.lo;
        sp->u = usum;
        sp->mn = mn;
        sp->mx = mx;
        __threadfence();
        const uint32_t prev = atomicAdd(&a.tickets[m.task], 1u);
        sm.flag = (prev == m.nseg - 1) ? 1u : 0u;
    }
    named_sync<CB>();
    const uint32_t last = sm.flag;
    named_sync<CB>();   // sm.flag may be rewritten by the next segment
    if (!last) return;
    __threadfence();
    ff fs{0.f, 0.f};
    unsigned long long fu = 0;
    float fmn = CUDART_INF_F, fmx = -CUDART_INF_F;
    for (uint32_t s = tid; s < m.nseg; s += CB) {
        const StreamPartial* sp = a.spart + m.slot0 + s;
        if constexpr (F32) {
            fs = ff_add(fs, ff{__ldcg(&sp->shi), __ldcg(&sp->slo)});
            fmn = fminf(fmn, __ldcg(&sp->mn));
            fmx = fmaxf(fmx, __ldcg(&sp->mx));
        } else {
            fu += __ldcg(reinterpret_cast<const unsigned long long*>(&sp->u));
        }
    }
    if constexpr (F32) creduce_ff<CB>(fs, fmn, fmx, tid, sm);
    else fu = csum_u64<CB>(fu, tid, sm);
    if (tid == 0) {
        write_result(m.result, fu, F32 ? ff_to_double(fs) : (double)fu, F32 ? fmn : 0.f,
                     F32 ? fmx : 0.f, SCL_OK, m.n, m.kind);
        a.tickets[m.task] = 0u;
    }
}

template <int CB, int IPT, int STAGES, int MASK>
__global__ void __launch_bounds__(CB + 32) k_stream_tma(const __grid_constant__ KernelArgs a) {
    using L = TmaLayout<CB, IPT, STAGES>;
    static_assert(mask_has_stream(MASK) && !mask_has_keyed(MASK), "streaming kinds only");
    extern __shared__ __align__(128) char smem[];
    __shared__ RedSmem sm;
    StageMeta* meta = reinterpret_cast<StageMeta*>(smem + L::kMeta);
    const uint32_t full0 = smem_u32(smem + L::kFull);
    const uint32_t empty0 = smem_u32(smem + L::kEmpty);
    uint32_t* err = &a.hdr[H_ERROR];

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, CB / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (threadIdx.x < 32) {
        // ------------------------------------------------------ producer
        if (threadIdx.x == 0 && a.nseg_stream > 0) {
            uint32_t s = 0, ph = 0;
            bool ok = true;
            uint32_t armed = 0;     // stages whose bulk copy may still be in flight
            uint32_t arm_par = 0;   // parity of the full-barrier phase each completes
            const uint32_t N = a.nseg_stream;
            uint32_t cur_task = 0xffffffffu;
            DevTask t = a.single;
            // Grab runs of kRun consecutive segments: one counter atomic per run,
            // the next run's atomic in flight while this run's copies go out, and
            // the task descriptor re-read only when the task changes.
            uint32_t q = atomicAdd(&a.hdr[H_QUEUE], kRun);
            while (ok && q < N) {
                const uint32_t qn = atomicAdd(&a.hdr[H_QUEUE], kRun);
                const uint32_t qe = min(q + kRun, N);
                for (; ok && q < qe; ++q) {
                    const uint32_t task = a.tasks ? a.seg_task[q] : 0u;
                    if (task != cur_task) {
                        t = a.tasks ? a.tasks[task] : a.single;
                        cur_task = task;
                    }
                    const uint32_t local = q - t.seg_base;
                    const uint64_t b = (uint64_t)local * t.seg_elems;
                    const uint64_t e = min(b + (uint64_t)t.seg_elems, t.n);
                    const bool aligned = (t.flags & TF_ALIGNED) != 0;
                    uint64_t c = b;
                    do {
                        if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, err)) {
                            ok = false;
                            break;
                        }
                        armed &= ~(1u << s);
                        const uint64_t nv64 = min((uint64_t)L::kChunk, e - c);
                        const uint32_t nv = (uint32_t)nv64;
                        const bool direct = !aligned || nv != L::kChunk;
                        StageMeta m;
                        m.gptr = static_cast<const char*>(t.in0) + c * 4;
                        m.result = t.result;
                        m.n = t.n;
                        m.task = task;
                        m.local = local;
                        m.nvalid = nv;
                        m.flags = (c + nv64 >= e ? SF_LAST : 0u) | (direct ? SF_DIRECT : 0u);
                        m.kind = t.kind;
                        m.nseg = t.nseg;
                        m.slot0 = t.slot0;
                        m.coef[0] = t.coef[0];
                        m.coef[1] = t.coef[1];
                        m.coef[2] = t.coef[2];
                        meta[s] = m;
                        const uint32_t fb = full0 + 8 * s;
                        if (direct) {
                            mbar_arrive(fb);
                        } else {
                            mbar_arrive_tx(fb, L::kStageBytes);
                            bulk_g2s(smem_u32(smem + L::kData + (size_t)s * L::kStageBytes),
                                     m.gptr, L::kStageBytes, fb);
                            armed |= 1u << s;
                            arm_par = (arm_par & ~(1u << s)) | (ph << s);
                        }
                        c += nv64;
                        if (++s == STAGES) {
                            s = 0;
                            ph ^= 1u;
                        }
                    } while (c < e);
                }
                q = qn;
            }
            if (ok && mbar_wait(empty0 + 8 * s, ph ^ 1u, err)) {
                meta[s].flags = SF_END;
                mbar_arrive(full0 + 8 * s);
                armed = 0;   // consumers are alive and will drain every stage
            }
            // Gave up: wait (bounded) until each copy still in flight has landed.
            for (uint32_t k = 0; k < (uint32_t)STAGES; ++k) {
                if (!(armed & (1u << k))) continue;
                const uint32_t par = (arm_par >> k) & 1u;
                const long long t0 = clock64();
                while (!mbar_try(full0 + 8 * k, par) && clock64() - t0 < kWaitCycles) {
                }
            }
        }
    } else if (a.nseg_stream > 0) {
        // ------------------------------------------------------ consumers
        const uint32_t tid = threadIdx.x - 32;
        const uint32_t lane = tid & 31;
        uint32_t s = 0, ph = 0;
        unsigned long long usum = 0;
        ff fsum{0.f, 0.f};
        float mn = CUDART_INF_F, mx = -CUDART_INF_F;
        for (;;) {
            if (!mbar_wait(full0 + 8 * s, ph, err)) break;
            const StageMeta m = meta[s];
            if (m.flags & SF_END) break;
            const char* stage = smem + L::kData + (size_t)s * L::kStageBytes;
            bool f32 = false;
            if constexpr (mask_has_u32(MASK)) {
                if (m.kind == K_U32_IDENT)
                    consume_chunk<CB, IPT, K_U32_IDENT>(m, stage, tid, usum, fsum, mn, mx);
                else if (m.kind == K_U32_MIX32)
                    consume_chunk<CB, IPT, K_U32_MIX32>(m, stage, tid, usum, fsum, mn, mx);
            }
            if constexpr (mask_has_f32(MASK)) {
                if (m.kind == K_F32_IDENT) {
                    consume_chunk<CB, IPT, K_F32_IDENT>(m, stage, tid, usum, fsum, mn, mx);
                    f32 = true;
                } else if (m.kind == K_F32_POLY3) {
                    consume_chunk<CB, IPT, K_F32_POLY3>(m, stage, tid, usum, fsum, mn, mx);
                    f32 = true;
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty0 + 8 * s);
            if (m.flags & SF_LAST) {
                if (f32) segment_end<CB, true>(a, m, tid, usum, fsum, mn, mx, sm);
                else segment_end<CB, false>(a, m, tid, usum, fsum, mn, mx, sm);
                usum = 0;
                fsum = ff{0.f, 0.f};
                mn = CUDART_INF_F;
                mx = -CUDART_INF_F;
            }
            if (++s == STAGES) {
                s = 0;
                ph ^= 1u;
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

}  // namespace dev
}  // namespace scl

#define SCL_TMA_SHAPE(M, B, I, S)                                                      \
    {M, B, I, (const void*)&scl::dev::k_stream_tma<B, I, S, M>,                        \
     scl::dev::TmaLayout<B, I, S>::kBytes, 1, S}
