// kernels_db.cuh -- k_doorbell: the resident kernel of the device-polling
// server (continuous offload of partition tasks without a launch per batch).
//
// SparkCL offloads each partition task through its worker's accelerator
// (Sec. 3.1.1-3.1.3) and serialises them per device (Sec. 3.1.5).  Here one
// kernel stays resident: the host writes a job (one partition task) and the
// unit -> job entries of its work units into pinned host memory and then
// advances a published-unit count (the doorbell).  Every CTA claims units in
// order from a device counter, one ahead, waits until the doorbell covers its
// claim, reads the job through the mapped address and runs the unit:
//   * a streaming segment, with the batch kernel's own segment code
//     (stream_segment): same segment geometry, same reduction order, so a
//     task's result is bitwise the one scl_map_reduce gives with the same
//     (block, items per thread);
//   * a keyed piece: the shared-memory table of keyed_accumulate, flushed
//     into the job's count / fp64 accumulator with L2 atomics; the CTA that
//     takes the job's last ticket writes the outputs and re-zeroes the slot.
// The CTA that completes a job writes its result into mapped host memory and
// then, after a system-scope fence, the job's sequence number into done[].
//
// Waiting: only thread 0 of a CTA waits, only for the host's doorbell, never
// for another CTA.  One CTA at a time (a try-lock, never waited on) reads
// the host words and mirrors them in device memory; the others read the
// mirror and back off with __nanosleep.  Every wait ends: when the host asks
// the kernel to stop (its claim is then unpublished and dropped), or after
// wait_limit_ns of global-timer time or max_polls iterations, whichever comes
// first; the CTA then sets DB_ERR_WAIT in the host's error word and returns.
// A job descriptor that fails the bounds checks sets DB_ERR_DESC and ends the
// CTA without touching memory through it.
#pragma once

#include "kernels.cuh"

namespace scl {
namespace dev {

__device__ __forceinline__ unsigned long long ld_acquire_sys_u64(const void* p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
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

enum DbWait : uint32_t { DBW_READY = 0, DBW_STOP = 1, DBW_ERROR = 2 };

// Thread 0: wait until unit u is published.  Bounded (see the file comment).
__device__ __noinline__ static uint32_t db_wait(const DbArgs& a, unsigned long long u) {
    DbState* ds = a.state;
    volatile unsigned long long* vtail = &ds->tail;
    volatile uint32_t* vstop = &ds->stop;
    const unsigned long long t0 = global_ns();
    uint32_t nap = 32;
    for (unsigned long long it = 0; it < a.max_polls; ++it) {
        if (u < *vtail) {
            __threadfence_system();
            return DBW_READY;
        }
        if (*vstop) return DBW_STOP;
        if (atomicCAS(&ds->lock, 0u, 1u) == 0u) {
            const unsigned long long ht = ld_acquire_sys_u64(&a.host->tail);
            const uint32_t hs = ld_volatile_u32(&a.host->stop);
            __threadfence();
            if (ht > *vtail) atomicMax(&ds->tail, ht);
            if (hs) atomicExch(&ds->stop, 1u);
            __threadfence();
            atomicExch(&ds->lock, 0u);
            if (u < ht) {
                __threadfence_system();
                return DBW_READY;
            }
            if (hs) return DBW_STOP;
        }
        if (global_ns() - t0 > a.wait_limit_ns) break;
        __nanosleep(nap);
        if (nap < 1024) nap <<= 1;
    }
    db_set_err(a, DB_ERR_WAIT);
    return DBW_ERROR;
}

// Thread 0: read and check the job of unit u into `cur`.  False: bad descriptor.
__device__ __forceinline__ static bool db_fetch(const DbArgs& a, unsigned long long u, DbJob& cur, uint32_t& local) {
    const uint32_t j = ld_volatile_u32(a.unit_job + (u % a.unit_ring));
    if (j >= a.job_ring) return false;
    const uint4* src = reinterpret_cast<const uint4*>(a.jobs + j);
    uint4 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = ld_volatile_v4(src + q);
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
            return keyed_piece<BLOCK, IPT, true>(a.ka, t, j, 0u, 0ull, t.n, tab, sm);
        return keyed_piece<BLOCK, IPT, false>(a.ka, t, j, 0u, 0ull, t.n, tab, sm);
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
    double stot = 0.0;
    for (uint32_t k = threadIdx.x; k < nk; k += BLOCK) {
        const uint32_t c = __ldcg(&acnt[k]);
        const double s = __ldcg(&asum[k]);
        t.counts_out[k] = c;
        t.sums_out[k] = (float)s;
        if (t.sums64_out) t.sums64_out[k] = s;
        acnt[k] = 0u;
        asum[k] = 0.0;
        ctot += c;
        stot += s;
    }
    float d0 = CUDART_INF_F, d1 = -CUDART_INF_F;
    block_reduce_f<BLOCK>(stot, d0, d1, sm);
    ctot = block_sum_u64<BLOCK>(ctot, sm);
    if (threadIdx.x == 0) {
        const uint32_t fl = atomicExch(&a.ka.task_flags[j], 0u);
        write_result(t.result, ctot, stot, CUDART_INF_F, -CUDART_INF_F,
                     fl ? SCL_E_KEY_RANGE : SCL_OK, t.n, t.kind);
        a.ka.tickets[j] = 0u;
    }
    return threadIdx.x == 0;
}

struct DbSmem {
    DbJob cur;
    uint32_t local;
    uint32_t status;
};

template <int BLOCK, int IPT>
__global__ void __launch_bounds__(BLOCK) k_doorbell(const __grid_constant__ DbArgs a) {
    __shared__ RedSmem sm;
    __shared__ DbSmem db;
    extern __shared__ uint4 dyn_smem[];
    uint32_t* tab = reinterpret_cast<uint32_t*>(dyn_smem);

    unsigned long long mine = 0, ahead = 0;
    if (threadIdx.x == 0) mine = atomicAdd(&a.state->next, 1ull);
    for (;;) {
        if (threadIdx.x == 0) {
            uint32_t st = db_wait(a, mine);
            if (st == DBW_READY && !db_fetch(a, mine, db.cur, db.local)) {
                db_set_err(a, DB_ERR_DESC);
                st = DBW_ERROR;
            }
            db.status = st;
        }
        __syncthreads();
        if (db.status != DBW_READY) break;   // uniform
        if (threadIdx.x == 0) ahead = atomicAdd(&a.state->next, 1ull);
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
        if (wrote) {   // thread 0 of the CTA that completed the job
            __threadfence_system();
            st_release_sys_u32(a.done + j, db.cur.seq);
        }
        __syncthreads();   // db.cur and sm are free again
        if (threadIdx.x == 0) mine = ahead;
    }
}

}  // namespace dev
}  // namespace scl

#define SCL_DB_ENTRY(B, I) \
    if (ipt == I) return (const void*)&scl::dev::k_doorbell<B, I>;
