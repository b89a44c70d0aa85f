// kernels_db.cuh -- k_doorbell: the resident kernel of the device-polling
// server (continuous offload of partition tasks without a launch per batch).
//
// SparkCL offloads each partition task through its worker's accelerator
// (Sec. 3.1.1-3.1.3) and serialises them per device (Sec. 3.1.5).  Here one
// kernel stays resident.  The host writes job p (one partition task) into
// ring slot p % job_ring of pinned host memory and then raises the count of
// published jobs (the doorbell).  Jobs are cut into work units (streaming
// segments or keyed pieces) numbered in publication order.  Every CTA claims
// units from a device counter, one ahead, and waits until the units it holds
// are available, then runs them:
//   * a streaming segment, with the batch kernel's own segment code
//     (stream_segment): same segment geometry, same reduction order, so a
//     task's result is bitwise the one scl_map_reduce gives with the same
//     (block, items per thread);
//   * a keyed piece: the shared-memory table of keyed_accumulate, flushed
//     into the job's count / fp64 accumulator with L2 atomics; the CTA that
//     takes the job's last ticket writes the outputs and re-zeroes the slot.
// The CTA that completes a job writes its result into mapped host memory and
// then, with a system-scope release, the job's sequence number into done[].
//
// Reads of host memory through the mapped address are slow and do not
// overlap well across the GPU, so only one CTA at a time reads the doorbell
// (a try-lock that nobody waits on).  When it finds new jobs it copies their
// descriptors into device memory, writes the unit -> slot map of their units
// with the whole CTA, and only then raises the device's count of available
// units (release).  Every other CTA reads only device memory (acquire).
//
// Every wait ends: when the host asks the kernel to stop (a claim not yet
// available is dropped), or after wait_limit_ns of global-timer time or
// max_polls iterations, whichever comes first; the CTA then sets DB_ERR_WAIT
// in the host's error word and returns.  A descriptor that fails a check
// sets DB_ERR_DESC and ends the CTA without touching memory through it.
#pragma once

#include "kernels.cuh"

namespace scl {
namespace dev {

__device__ __forceinline__ unsigned long long ld_acquire_sys_u64(const void* p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu_u64(const void* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_volatile_u32(const void* p) {
    uint32_t v;
    asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint4 ld_volatile_v4(const void* p) {
    uint4 v;
    asm volatile("ld.volatile.global.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p)
                 : "memory");
    return v;
}

__device__ __forceinline__ void st_release_sys_u32(void* p, uint32_t v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Any nonzero value is an error; a plain store, so no host-memory atomics.
__device__ __forceinline__ void db_set_err(const DbArgs& a, uint32_t bit) {
    st_release_sys_u32(&a.host->err, bit);
}

enum DbAction : uint32_t { DBA_READY = 0, DBA_STOP = 1, DBA_ERROR = 2, DBA_NAP = 3, DBA_EXPAND = 4 };

struct DbSmem {
    DbJob cur;                 // descriptor of the unit being run
    unsigned long long mine;   // unit this CTA holds
    unsigned long long x0, x1; // jobs being expanded
    unsigned long long xend;   // units available once they are
    uint32_t local;            // unit index within its job
    uint32_t action;           // db_wait's decision (thread 0 writes)
    uint32_t fetched;          // db_fetch's verdict (thread 0 writes)
    uint32_t xok;
};

// Whole CTA, lock held: copy jobs [x0, x1) into device memory, map their
// units, then release the units and the lock.  False (uniform): a
// descriptor failed the continuity checks; DB_ERR_DESC is set.
template <int BLOCK>
__device__ __noinline__ bool db_expand(const DbArgs& a, DbSmem& db, uint32_t* scratch) {
    DbState* ds = a.state;
    const unsigned long long x0 = db.x0;
    const uint32_t nj = (uint32_t)(db.x1 - x0);
    uint4* sj = reinterpret_cast<uint4*>(scratch);   // nj * 128 bytes <= 8 KB
    for (uint32_t i = threadIdx.x; i < nj * 8; i += BLOCK) {
        const uint32_t slot = (uint32_t)((x0 + i / 8) % a.job_ring);
        const uint4 v = ld_volatile_v4(reinterpret_cast<const uint4*>(a.jobs + slot) + (i % 8));
        sj[i] = v;
        __stcg(reinterpret_cast<uint4*>(a.djobs + slot) + (i % 8), v);
    }
    __syncthreads();
    const DbJob* J = reinterpret_cast<const DbJob*>(scratch);
    if (threadIdx.x == 0) {
        unsigned long long u = __ldcg(&ds->tail);   // changes only under the lock
        uint32_t ok = 1;
        for (uint32_t i = 0; i < nj; ++i) {
            if (J[i].ring != (uint32_t)((x0 + i) % a.job_ring) || J[i].unit0 != u ||
                J[i].t.nseg == 0 || J[i].t.nseg > a.unit_ring)
                ok = 0;
            u += J[i].t.nseg;
        }
        db.xok = ok;
        db.xend = u;
    }
    __syncthreads();
    if (!db.xok) {
        if (threadIdx.x == 0) {
            db_set_err(a, DB_ERR_DESC);
            __threadfence();
            atomicExch(&ds->lock, 0u);
        }
        return false;
    }
    for (uint32_t i = 0; i < nj; ++i) {
        const uint32_t slot = J[i].ring;
        const unsigned long long u0 = J[i].unit0;
        for (uint32_t k = threadIdx.x; k < J[i].t.nseg; k += BLOCK)
            __stcg(a.dunit + (u0 + k) % a.unit_ring, slot);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        __stcg(&ds->jobs_seen, db.x1);
        __threadfence();   // release: descriptors and unit map before the units
        atomicMax(&ds->tail, db.xend);
        __threadfence();
        atomicExch(&ds->lock, 0u);
    }
    return true;
}

// Whole CTA: wait until unit db.mine is available.  Returns DBA_READY,
// DBA_STOP or DBA_ERROR (uniform).  Bounded (see the file comment).
template <int BLOCK>
__device__ __forceinline__ uint32_t db_wait(const DbArgs& a, DbSmem& db, uint32_t* scratch) {
    DbState* ds = a.state;
    unsigned long long t0 = 0;
    uint32_t nap = 32;
    if (threadIdx.x == 0) t0 = global_ns();
    for (unsigned long long it = 0;; ++it) {
        if (threadIdx.x == 0) {
            uint32_t act = DBA_NAP;
            if (db.mine < ld_acquire_gpu_u64(&ds->tail)) {
                act = DBA_READY;
            } else if (ld_volatile_u32(&ds->stop)) {
                act = DBA_STOP;
            } else if (atomicCAS(&ds->lock, 0u, 1u) == 0u) {
                const unsigned long long hj = ld_acquire_sys_u64(&a.host->jobs);
                const uint32_t hs = ld_volatile_u32(&a.host->stop);
                const unsigned long long seen = __ldcg(&ds->jobs_seen);
                if (hj > seen) {
                    db.x0 = seen;
                    db.x1 = hj - seen > kDbMaxExpand ? seen + kDbMaxExpand : hj;
                    act = DBA_EXPAND;   // the lock stays held until db_expand ends
                } else {
                    if (hs) atomicExch(&ds->stop, 1u);
                    __threadfence();
                    atomicExch(&ds->lock, 0u);
                    if (hs) act = DBA_STOP;
                }
            }
            if (act == DBA_NAP && (it >= a.max_polls || global_ns() - t0 > a.wait_limit_ns)) {
                db_set_err(a, DB_ERR_WAIT);
                act = DBA_ERROR;
            }
            db.action = act;
        }
        __syncthreads();
        const uint32_t act = db.action;
        if (act == DBA_READY || act == DBA_STOP || act == DBA_ERROR) return act;
        if (act == DBA_EXPAND) {
            if (!db_expand<BLOCK>(a, db, scratch)) return DBA_ERROR;
        } else if (threadIdx.x == 0) {
            __nanosleep(nap);
            if (nap < 512) nap <<= 1;
        }
        __syncthreads();   // db.action read by all before thread 0 writes it again
    }
}

// Thread 0: the descriptor of available unit u (device memory only) into
// `cur`, checked.  False: a bad descriptor.
__device__ __forceinline__ static bool db_fetch(const DbArgs& a, unsigned long long u, DbJob& cur,
                                                uint32_t& local) {
    const uint32_t j = __ldcg(a.dunit + u % a.unit_ring);
    if (j >= a.job_ring) return false;
    const uint4* src = reinterpret_cast<const uint4*>(a.djobs + j);
    uint4 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __ldcg(src + q);
    uint4* dst = reinterpret_cast<uint4*>(&cur);
#pragma unroll
    for (int q = 0; q < 8; ++q) dst[q] = v[q];
    const DevTask& t = cur.t;
    if (cur.ring != j || u < cur.unit0 || u - cur.unit0 >= t.nseg || t.kind >= K_NUM) return false;
    local = (uint32_t)(u - cur.unit0);
    if (is_keyed(t.kind)) {
        if (t.num_keys < 1 || t.num_keys > kMaxKeys) return false;
        if (t.nseg > 1 && t.slot0 >= a.kacc_slots) return false;
    } else if (t.nseg > 1 && (uint64_t)t.slot0 + t.nseg > a.spart_cap) {
        return false;
    }
    return true;
}

// One keyed piece of a device-polled job.  Returns true in thread 0 of the
// CTA that wrote the job's result.
// Keyed pieces load at most 4 vectors per thread per array (keys and values
// double the registers a chunk holds); their sums do not depend on the shape.
template <int BLOCK, int IPT_STREAM>
__device__ __forceinline__ bool db_keyed_unit(const DbArgs& a, const DevTask& t, uint32_t j,
                                              uint32_t local, uint32_t* tab, RedSmem& sm) {
    constexpr int IPT = IPT_STREAM > 4 ? 4 : IPT_STREAM;
    if (t.nseg == 1) {
        if (t.kind == K_KEYED_MIX)
            return keyed_piece<BLOCK, IPT, true, false>(a.ka, t, j, 0u, 0ull, t.n, tab, sm);
        return keyed_piece<BLOCK, IPT, false, false>(a.ka, t, j, 0u, 0ull, t.n, tab, sm);
    }
    const uint64_t b = keyed_single_bound(t.n, local, t.nseg);
    const uint64_t e = keyed_single_bound(t.n, local + 1, t.nseg);
    const int any_bad = t.kind == K_KEYED_MIX ? keyed_accumulate<BLOCK, IPT, true>(t, b, e, tab)
                                              : keyed_accumulate<BLOCK, IPT, false>(t, b, e, tab);
    const uint32_t nk = t.num_keys;
    uint32_t* acnt = a.kacc + (size_t)t.slot0 * kDbAccWords;
    double* asum = reinterpret_cast<double*>(acnt + kMaxKeys);
    const uint32_t* cnt = tab;
    const float* sum = reinterpret_cast<const float*>(tab + kMaxKeys);
    for (uint32_t k = threadIdx.x; k < nk; k += BLOCK) {
        const uint32_t c = cnt[k];
        if (c) {
            atomicAdd(&acnt[k], c);
            atomicAdd(&asum[k], (double)sum[k]);
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        if (any_bad) atomicOr(&a.ka.task_flags[j], 1u);
        __threadfence();
        const uint32_t prev = atomicAdd(&a.ka.tickets[j], 1u);
        sm.flag = (prev == t.nseg - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (sm.flag == 0) return false;   // uniform across the CTA
    __threadfence();

    // Last piece: the outputs, then the accumulator back to zero.
    unsigned long long ctot = 0;
    ff stot{0.f, 0.f};
    for (uint32_t k = threadIdx.x; k < nk; k += BLOCK) {
        const uint32_t c = __ldcg(&acnt[k]);
        const double s = __ldcg(&asum[k]);
        t.counts_out[k] = c;
        t.sums_out[k] = (float)s;
        if (t.sums64_out) t.sums64_out[k] = s;
        acnt[k] = 0u;
        asum[k] = 0.0;
        ctot += c;
        stot = ff_add(stot, ff_of_double(s));
    }
    float d0 = CUDART_INF_F, d1 = -CUDART_INF_F;
    block_reduce_ff<BLOCK>(stot, d0, d1, sm);
    ctot = block_sum_u64<BLOCK>(ctot, sm);
    if (threadIdx.x == 0) {
        const uint32_t fl = atomicExch(&a.ka.task_flags[j], 0u);
        write_result(t.result, ctot, ff_to_double(stot), CUDART_INF_F, -CUDART_INF_F,
                     fl ? SCL_E_KEY_RANGE : SCL_OK, t.n, t.kind);
        a.ka.tickets[j] = 0u;
    }
    return threadIdx.x == 0;
}

template <int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK) k_doorbell(const __grid_constant__ DbArgs a) {
    __shared__ RedSmem sm;
    __shared__ DbSmem db;
    extern __shared__ uint4 dyn_smem[];
    uint32_t* tab = reinterpret_cast<uint32_t*>(dyn_smem);

    unsigned long long ahead = 0;
    if (threadIdx.x == 0) db.mine = atomicAdd(&a.state->next, 1ull);
    for (;;) {
        __syncthreads();   // db.mine
        if (db_wait<BLOCK>(a, db, tab) != DBA_READY) break;   // uniform
        if (threadIdx.x == 0) {
            db.fetched = db_fetch(a, db.mine, db.cur, db.local) ? 1u : 0u;
            if (db.fetched) ahead = atomicAdd(&a.state->next, 1ull);
            else db_set_err(a, DB_ERR_DESC);
        }
        __syncthreads();
        if (!db.fetched) break;   // uniform
        const DevTask t = db.cur.t;
        const uint32_t j = db.cur.ring, local = db.local;
        bool wrote;
        switch (t.kind) {
            case K_U32_IDENT:
                wrote = stream_segment<BLOCK, IPT, K_U32_IDENT>(a.ka, t, j, local, sm);
                break;
            case K_U32_MIX32:
                wrote = stream_segment<BLOCK, IPT, K_U32_MIX32>(a.ka, t, j, local, sm);
                break;
            case K_F32_IDENT:
                wrote = stream_segment<BLOCK, IPT, K_F32_IDENT>(a.ka, t, j, local, sm);
                break;
            case K_F32_POLY3:
                wrote = stream_segment<BLOCK, IPT, K_F32_POLY3>(a.ka, t, j, local, sm);
                break;
            default:
                wrote = db_keyed_unit<BLOCK, IPT>(a, t, j, local, tab, sm);
                break;
        }
        if (wrote)   // thread 0 of the CTA that completed the job; the release
                     // orders the result (this thread) and the CTA's outputs
                     // (before the last barrier) before the done word
            st_release_sys_u32(a.done + j, db.cur.seq);
        __syncthreads();   // db.cur, sm and tab are free again
        if (threadIdx.x == 0) db.mine = ahead;
    }
}

}  // namespace dev
}  // namespace scl

#define SCL_DB_ENTRY(B, I) \
    if (ipt == I) return (const void*)&scl::dev::k_doorbell<B, I>;
