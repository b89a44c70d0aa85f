// capi.cu -- the extern "C" entry points declared in include/scl.h.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "runtime.h"
#include "devserver.h"
#include "radix.h"
#include "server.h"

namespace scl {
const char* last_error();
uint64_t launches_total();
}  // namespace scl

using namespace scl;

namespace {

struct DeviceGuard {
    explicit DeviceGuard(int dev) { cudaSetDevice(dev); }
};

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

#define CTX_ENTER(ctx)                                                     \
    if (!(ctx)) return fail(SCL_E_INVALID, "null context");               \
    clear_error();                                                         \
    std::lock_guard<std::recursive_mutex> lock_((ctx)->mu);               \
    DeviceGuard dg_((ctx)->device)

size_t dtype_words(scl_dtype dt) { return dt == SCL_KV_I32_F32 ? 2 : 1; }

double pairwise_sum(const scl_result* r, uint32_t lo, uint32_t hi) {
    if (hi - lo == 1) return r[lo].f64_sum;
    const uint32_t mid = lo + (hi - lo) / 2;
    return pairwise_sum(r, lo, mid) + pairwise_sum(r, mid, hi);
}

}  // namespace

// A batch is one launch group or, when its tasks mix families and splitting is
// on, one group per family (keyed, uint32, fp32) launched concurrently on forked
// streams: the keyed-only kernel (fixed-point window, two 512-thread CTAs per
// SM) next to the streaming kernels (eight CTAs per SM), in place of the mixed
// kernel whose CTAs hold the fp32 keyed table at four per SM.  Every group
// writes into one scratch block: results, tickets and flags at the positions
// of `order`, a header per group.
struct scl_batch {
    struct Group {
        Plan plan;
        PlanImage img;
        KernelArgs args;
        uint32_t first = 0, count = 0;   // positions [first, first + count) of `order`
    };
    Ctx* ctx = nullptr;
    std::vector<Group> groups;
    std::vector<uint32_t> order;          // position -> the caller's task index
    void* scratch = nullptr;              // results, tickets, flags, headers (zeroed)
    size_t scratch_bytes = 0;
    scl_result* results = nullptr;        // in `order`
    uint32_t* hdr = nullptr;              // H_WORDS per group
    cudaStream_t side[2] = {nullptr, nullptr};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[2] = {nullptr, nullptr};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t ntasks = 0;
    uint32_t kernels = 0;                 // kernel launches per scl_batch_launch
    std::vector<scl_result> staged;
};

namespace {

// Frees what a batch holds on the device (after a device synchronisation).
void batch_release(scl_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto& g : b->groups)
        if (g.img.block) b->ctx->arena.release(g.img.block);
    if (b->scratch) b->ctx->arena.release(b->scratch);
    for (int i = 0; i < 2; ++i) {
        if (b->side[i]) cudaStreamDestroy(b->side[i]);
        if (b->join[i]) cudaEventDestroy(b->join[i]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
}

// The groups' launches on `st`: the first group on `st` itself, the others on
// the batch's side streams, forked from `st` before and joined into it after.
// Stream capture records the same fork and join.
int batch_launch_groups(scl_batch* b, cudaStream_t st) {
    if (b->groups.size() == 1) return launch_plan(b->ctx, b->groups[0].plan, b->groups[0].args, st);
    SCL_CUDA(cudaEventRecord(b->fork, st));
    for (size_t g = 1; g < b->groups.size(); ++g)
        SCL_CUDA(cudaStreamWaitEvent(b->side[g - 1], b->fork, 0));
    for (size_t g = 0; g < b->groups.size(); ++g) {
        const scl_batch::Group& G = b->groups[g];
        SCL_TRY(launch_plan(b->ctx, G.plan, G.args, g ? b->side[g - 1] : st));
    }
    for (size_t g = 1; g < b->groups.size(); ++g) {
        SCL_CUDA(cudaEventRecord(b->join[g - 1], b->side[g - 1]));
        SCL_CUDA(cudaStreamWaitEvent(st, b->join[g - 1], 0));
    }
    return SCL_OK;
}

}  // namespace

extern "C" {

const char* scl_strerror(int status) {
    switch (status) {
        case SCL_OK: return "ok";
        case SCL_E_INVALID: return "invalid argument";
        case SCL_E_NOMEM: return "arena out of memory";
        case SCL_E_BUDGET: return "HBM admission budget exceeded";
        case SCL_E_KEY_RANGE: return "key out of range";
        case SCL_E_TIMEOUT: return "timed out";
        case SCL_E_PENDING: return "pending";
        case SCL_E_CUDA: return "CUDA error";
        case SCL_E_STATE: return "invalid state";
        case SCL_E_UNSUPPORTED: return "unsupported combination";
        default: return "unknown status";
    }
}

const char* scl_last_error(void) { return last_error(); }

int scl_abi_version(void) { return SCL_ABI_VERSION; }

int scl_kernel_launches_total(uint64_t* out) {
    if (!out) return fail(SCL_E_INVALID, "null output");
    *out = launches_total();
    return SCL_OK;
}

// ---------------------------------------------------------------- contexts

int scl_create(const scl_config* cfg, scl_ctx** out) {
    clear_error();
    if (!cfg || !out) return fail(SCL_E_INVALID, "null argument");
    *out = nullptr;
    if (!cfg->arena || cfg->arena_bytes < (1u << 20))
        return fail(SCL_E_INVALID, "arena must be a device buffer of at least 1 MiB");
    if ((uintptr_t)cfg->arena % kAlign)
        return fail(SCL_E_INVALID, "arena must be 256-byte aligned");
    int ndev = 0;
    SCL_CUDA(cudaGetDeviceCount(&ndev));
    if (cfg->device < 0 || cfg->device >= ndev)
        return fail(SCL_E_INVALID, "device %d not present (%d devices)", cfg->device, ndev);
    SCL_CUDA(cudaSetDevice(cfg->device));
    cudaPointerAttributes pa;
    SCL_CUDA(cudaPointerGetAttributes(&pa, cfg->arena));
    if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)
        return fail(SCL_E_INVALID, "arena is not device memory");

    scl_ctx* c = new (std::nothrow) scl_ctx();
    if (!c) return fail(SCL_E_NOMEM, "host allocation failed");
    c->device = cfg->device;
    c->arena_bytes = cfg->arena_bytes;
    c->hbm_budget = cfg->hbm_budget_bytes;
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    cudaDeviceGetAttribute(&c->l2_bytes, cudaDevAttrL2CacheSize, c->device);
    c->arena.init((char*)cfg->arena, cfg->arena_bytes);
    c->d_result = (scl_result*)c->arena.alloc(sizeof(scl_result));
    c->d_kout = (uint32_t*)c->arena.alloc((size_t)kMaxKeys * 16);
    int st = SCL_OK;
    if (!c->d_result || !c->d_kout) st = fail(SCL_E_NOMEM, "arena too small");
    if (st == SCL_OK && (cudaHostAlloc((void**)&c->h_result, 2 * sizeof(scl_result),
                                       cudaHostAllocMapped) != cudaSuccess ||
                         cudaHostGetDevicePointer((void**)&c->dh_result, c->h_result, 0) !=
                             cudaSuccess))
        st = fail(SCL_E_CUDA, "cudaHostAlloc failed");
    if (st == SCL_OK && cfg->tune_cache_path) {
        c->tune_path = cfg->tune_cache_path;
        st = load_tuning(c, cfg->tune_cache_path);
    }
    if (st != SCL_OK) {
        if (c->h_result) cudaFreeHost(c->h_result);
        delete c;
        return st;
    }
    *out = c;
    return SCL_OK;
}

int scl_server_stop(scl_ctx* ctx);
int scl_devserver_stop(scl_ctx* ctx);

int scl_destroy(scl_ctx* ctx) {
    if (!ctx) return SCL_OK;
    scl_server_stop(ctx);
    scl_devserver_stop(ctx);
    {
        std::lock_guard<std::recursive_mutex> g(ctx->mu);
        cudaSetDevice(ctx->device);
        if (ctx->h_result) cudaFreeHost(ctx->h_result);
    }
    delete ctx;
    return SCL_OK;
}

int scl_arena_stats(scl_ctx* ctx, uint64_t* free_bytes, uint64_t* largest_block) {
    if (!ctx) return fail(SCL_E_INVALID, "null context");
    if (free_bytes) *free_bytes = ctx->arena.free_bytes();
    if (largest_block) *largest_block = ctx->arena.largest_free();
    return SCL_OK;
}

// -------------------------------------------------------------- partitions

static int new_partition(scl_ctx* c, scl_dtype dt, uint64_t n, Partition* p) {
    const size_t bytes = align_up(n * 4);
    void* b = c->arena.alloc(bytes * dtype_words(dt));
    if (!b) return fail(SCL_E_NOMEM, "arena: no block for a partition of %llu elements",
                        (unsigned long long)n);
    p->dtype = dt;
    p->n = n;
    p->block = b;
    p->d0 = b;
    p->d1 = dt == SCL_KV_I32_F32 ? (char*)b + bytes : nullptr;
    return SCL_OK;
}

static scl_part register_partition(scl_ctx* c, const Partition& p) {
    const scl_part h = c->next_part++;
    c->parts[h] = p;
    if (p.block) c->resident_bytes += align_up(p.n * 4) * dtype_words(p.dtype);
    return h;
}

int scl_load_partition(scl_ctx* ctx, const void* host, scl_dtype dtype, uint64_t n,
                       void* stream, scl_part* out) {
    CTX_ENTER(ctx);
    if (!out) return fail(SCL_E_INVALID, "null output");
    if (dtype != SCL_U32 && dtype != SCL_I32 && dtype != SCL_F32)
        return fail(SCL_E_INVALID, "scl_load_partition takes U32, I32 or F32 (use _kv for keyed)");
    if (n && !host) return fail(SCL_E_INVALID, "null host pointer");
    Partition p;
    SCL_TRY(new_partition(ctx, dtype, n, &p));
    if (n) {
        cudaError_t e = cudaMemcpyAsync(p.d0, host, n * 4, cudaMemcpyHostToDevice, S(stream));
        if (e != cudaSuccess) {
            ctx->arena.release(p.block);
            return fail(SCL_E_CUDA, "H2D copy failed: %s", cudaGetErrorString(e));
        }
    }
    *out = register_partition(ctx, p);
    return SCL_OK;
}

int scl_load_partition_kv(scl_ctx* ctx, const int32_t* keys, const float* vals, uint64_t n,
                          void* stream, scl_part* out) {
    CTX_ENTER(ctx);
    if (!out) return fail(SCL_E_INVALID, "null output");
    if (n && (!keys || !vals)) return fail(SCL_E_INVALID, "null host pointer");
    Partition p;
    SCL_TRY(new_partition(ctx, SCL_KV_I32_F32, n, &p));
    if (n) {
        cudaError_t e = cudaMemcpyAsync(p.d0, keys, n * 4, cudaMemcpyHostToDevice, S(stream));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p.d1, vals, n * 4, cudaMemcpyHostToDevice, S(stream));
        if (e != cudaSuccess) {
            ctx->arena.release(p.block);
            return fail(SCL_E_CUDA, "H2D copy failed: %s", cudaGetErrorString(e));
        }
    }
    *out = register_partition(ctx, p);
    return SCL_OK;
}

int scl_alloc_partition(scl_ctx* ctx, scl_dtype dtype, uint64_t n, scl_part* out) {
    CTX_ENTER(ctx);
    if (!out) return fail(SCL_E_INVALID, "null output");
    if ((int)dtype < 0 || dtype > SCL_KV_I32_F32) return fail(SCL_E_INVALID, "bad dtype");
    Partition p;
    SCL_TRY(new_partition(ctx, dtype, n, &p));
    *out = register_partition(ctx, p);
    return SCL_OK;
}

int scl_wrap_device(scl_ctx* ctx, void* dev0, void* dev1, scl_dtype dtype, uint64_t n,
                    scl_part* out) {
    CTX_ENTER(ctx);
    if (!out) return fail(SCL_E_INVALID, "null output");
    if ((int)dtype < 0 || dtype > SCL_KV_I32_F32) return fail(SCL_E_INVALID, "bad dtype");
    if (n && !dev0) return fail(SCL_E_INVALID, "null device pointer");
    if (dtype == SCL_KV_I32_F32 && n && !dev1)
        return fail(SCL_E_INVALID, "keyed partition needs a value array");
    if (dtype != SCL_KV_I32_F32 && dev1)
        return fail(SCL_E_INVALID, "dev1 must be NULL for non-keyed partitions");
    if (((uintptr_t)dev0 | (uintptr_t)dev1) % 4)
        return fail(SCL_E_INVALID, "arrays must be 4-byte aligned");
    Partition p{dtype, n, dev0, dev1, nullptr};
    *out = register_partition(ctx, p);
    return SCL_OK;
}

int scl_reload_partition(scl_ctx* ctx, scl_part part, const void* host0, const void* host1,
                         void* stream) {
    CTX_ENTER(ctx);
    const Partition* p = ctx->part(part);
    if (!p) return fail(SCL_E_INVALID, "unknown partition handle");
    if (!p->n) return SCL_OK;
    if (!host0 || (p->d1 && !host1)) return fail(SCL_E_INVALID, "null host array");
    SCL_CUDA(cudaMemcpyAsync(p->d0, host0, p->n * 4, cudaMemcpyHostToDevice, S(stream)));
    if (p->d1)
        SCL_CUDA(cudaMemcpyAsync(p->d1, host1, p->n * 4, cudaMemcpyHostToDevice, S(stream)));
    return SCL_OK;
}

int scl_free_partition(scl_ctx* ctx, scl_part part) {
    CTX_ENTER(ctx);
    auto it = ctx->parts.find(part);
    if (it == ctx->parts.end()) return fail(SCL_E_INVALID, "unknown partition handle");
    if (it->second.block) {
        // stream-ordered work may still read it
        SCL_CUDA(cudaDeviceSynchronize());
        ctx->arena.release(it->second.block);
        ctx->resident_bytes -= align_up(it->second.n * 4) * dtype_words(it->second.dtype);
    }
    ctx->parts.erase(it);
    return SCL_OK;
}

int scl_partition_info(scl_ctx* ctx, scl_part part, scl_dtype* dtype, uint64_t* n, void** dev0,
                       void** dev1) {
    CTX_ENTER(ctx);
    const Partition* p = ctx->part(part);
    if (!p) return fail(SCL_E_INVALID, "unknown partition handle");
    if (dtype) *dtype = p->dtype;
    if (n) *n = p->n;
    if (dev0) *dev0 = p->d0;
    if (dev1) *dev1 = p->d1;
    return SCL_OK;
}

int scl_read_partition(scl_ctx* ctx, scl_part part, void* host0, void* host1, void* stream) {
    CTX_ENTER(ctx);
    const Partition* p = ctx->part(part);
    if (!p) return fail(SCL_E_INVALID, "unknown partition handle");
    if (p->n && !host0) return fail(SCL_E_INVALID, "null host pointer");
    if (p->n) {
        SCL_CUDA(cudaMemcpyAsync(host0, p->d0, p->n * 4, cudaMemcpyDeviceToHost, S(stream)));
        if (p->d1 && host1)
            SCL_CUDA(cudaMemcpyAsync(host1, p->d1, p->n * 4, cudaMemcpyDeviceToHost, S(stream)));
    }
    SCL_CUDA(cudaStreamSynchronize(S(stream)));
    return SCL_OK;
}

// ------------------------------------------------------------ map / reduce

static int map_kind(const Partition& p, scl_map_kernel kernel, uint32_t* kind) {
    if (p.dtype == SCL_KV_I32_F32) return fail(SCL_E_UNSUPPORTED, "maps take a 1-array partition");
    if (kernel == SCL_K_IDENT) *kind = K_U32_IDENT;
    else if (kernel == SCL_K_MIX32 && p.dtype != SCL_F32) *kind = K_U32_MIX32;
    else if (kernel == SCL_K_POLY3 && p.dtype == SCL_F32) *kind = K_F32_POLY3;
    else return fail(SCL_E_UNSUPPORTED, "map kernel %d does not apply to dtype %d", (int)kernel,
                     (int)p.dtype);
    return SCL_OK;
}

static int launch_map(scl_ctx* ctx, const Partition& src, uint32_t kind, const float coef[3],
                      void* dst, cudaStream_t st) {
    if (!src.n) return SCL_OK;
    static const float kDef[3] = {0.5f, -1.25f, 0.1f};
    const float* cf = coef ? coef : kDef;
    const int aligned = ((uintptr_t)src.d0 % 16) == 0 && ((uintptr_t)dst % 16) == 0;
    const void* fn = map_kernel_fn((int)kind, aligned);
    const int blk = map_kernel_block();
    const uint64_t chunk = (uint64_t)blk * map_kernel_ipt() * 4;
    const uint64_t want = aligned ? (src.n + chunk - 1) / chunk : (src.n + blk - 1) / blk;
    const uint32_t grid =
        (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)ctx->sms * 8));
    const void* sp = src.d0;
    uint64_t n = src.n;
    float a = cf[0], b = cf[1], cc = cf[2];
    void* params[] = {(void*)&sp, (void*)&dst, (void*)&n, &a, &b, &cc};
    SCL_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(blk), params, 0, st));
    count_launches(1);
    return SCL_OK;
}

int scl_map(scl_ctx* ctx, scl_part in, scl_map_kernel kernel, const float coef[3], void* stream,
            scl_part* out) {
    CTX_ENTER(ctx);
    if (!out) return fail(SCL_E_INVALID, "null output");
    const Partition* p = ctx->part(in);
    if (!p) return fail(SCL_E_INVALID, "unknown partition handle");
    uint32_t kind;
    SCL_TRY(map_kind(*p, kernel, &kind));
    const Partition src = *p;
    Partition o;
    SCL_TRY(new_partition(ctx, src.dtype, src.n, &o));
    const int st = launch_map(ctx, src, kind, coef, o.d0, S(stream));
    if (st != SCL_OK) {
        ctx->arena.release(o.block);
        return st;
    }
    *out = register_partition(ctx, o);
    return SCL_OK;
}

int scl_map_into(scl_ctx* ctx, scl_part in, scl_map_kernel kernel, const float coef[3],
                 scl_part out, void* stream) {
    CTX_ENTER(ctx);
    const Partition* p = ctx->part(in);
    const Partition* o = ctx->part(out);
    if (!p || !o) return fail(SCL_E_INVALID, "unknown partition handle");
    uint32_t kind;
    SCL_TRY(map_kind(*p, kernel, &kind));
    if (o->n != p->n || o->dtype == SCL_KV_I32_F32)
        return fail(SCL_E_INVALID, "output partition must be a 32-bit array of the same length");
    return launch_map(ctx, *p, kind, coef, o->d0, S(stream));
}

static int map_reduce_common(scl_ctx* ctx, scl_part part, scl_map_kernel kernel,
                             const float coef[3], scl_reduce reduce, void* stream,
                             scl_result* dev_out, uint32_t* err_out = nullptr) {
    const Partition* p = ctx->part(part);
    if (!p) return fail(SCL_E_INVALID, "unknown partition handle");
    uint32_t kind;
    if (reduce == SCL_R_KEYED_COUNT_SUM)
        return fail(SCL_E_UNSUPPORTED, "use scl_keyed_reduce for keyed partitions");
    SCL_TRY(resolve_kind(p->dtype, kernel, reduce, &kind));
    return run_single(ctx, *p, kind, coef, 0, nullptr, nullptr, nullptr, dev_out, S(stream),
                      err_out);
}

// After a synchronous single call: a non-zero device error word means a
// bounded wait expired (or an unknown work kind was met); report it and reset
// the single-call scratch so the next launch starts clean.
static int check_single_error(scl_ctx* ctx, cudaStream_t st) {
    const uint32_t err = *reinterpret_cast<uint32_t*>(ctx->h_result + 1);
    if (!err) return SCL_OK;
    Scratch& sc = ctx->single_for(st);
    SCL_CUDA(cudaMemset(sc.hdr, 0, H_WORDS * 4));
    SCL_CUDA(cudaMemset(sc.tickets, 0, sc.task_cap * 4));
    SCL_CUDA(cudaDeviceSynchronize());
    return fail((err & 4u) ? SCL_E_TIMEOUT : SCL_E_STATE,
                "device error word 0x%x after the launch", err);
}

static int fetch_single(scl_ctx* ctx, cudaStream_t st) {
    SCL_CUDA(cudaMemcpyAsync(ctx->h_result, ctx->d_result, sizeof(scl_result),
                             cudaMemcpyDeviceToHost, st));
    SCL_CUDA(cudaMemcpyAsync(ctx->h_result + 1, ctx->single_for(st).hdr + H_ERROR, 4,
                             cudaMemcpyDeviceToHost, st));
    SCL_CUDA(cudaStreamSynchronize(st));
    return check_single_error(ctx, st);
}

int scl_map_reduce(scl_ctx* ctx, scl_part part, scl_map_kernel kernel, const float coef[3],
                   scl_reduce reduce, void* stream, scl_result* out) {
    CTX_ENTER(ctx);
    if (!out) return fail(SCL_E_INVALID, "null output");
    // The kernel writes the result and the error word straight into pinned
    // host memory (its mapped address): no copies, one synchronisation.
    SCL_TRY(map_reduce_common(ctx, part, kernel, coef, reduce, stream, ctx->dh_result,
                              reinterpret_cast<uint32_t*>(ctx->dh_result + 1)));
    SCL_CUDA(cudaStreamSynchronize(S(stream)));
    SCL_TRY(check_single_error(ctx, S(stream)));
    *out = *ctx->h_result;
    return SCL_OK;
}

int scl_map_reduce_async(scl_ctx* ctx, scl_part part, scl_map_kernel kernel, const float coef[3],
                         scl_reduce reduce, void* stream, scl_result* dev_out) {
    CTX_ENTER(ctx);
    if (!dev_out) return fail(SCL_E_INVALID, "null device result pointer");
    return map_reduce_common(ctx, part, kernel, coef, reduce, stream, dev_out);
}

static int keyed_common(scl_ctx* ctx, scl_part part, uint32_t num_keys, void* stream,
                        uint32_t* counts, float* sums, double* sums64, scl_result* dres,
                        uint32_t kind = K_KEYED) {
    const Partition* p = ctx->part(part);
    if (!p) return fail(SCL_E_INVALID, "unknown partition handle");
    if (p->dtype != SCL_KV_I32_F32) return fail(SCL_E_UNSUPPORTED, "partition is not keyed");
    if (num_keys < 1 || num_keys > kMaxKeys)
        return fail(SCL_E_INVALID, "num_keys %u not in [1, %u]", num_keys, kMaxKeys);
    return run_single(ctx, *p, kind, nullptr, num_keys, counts, sums, sums64, dres, S(stream));
}

int scl_keyed_reduce(scl_ctx* ctx, scl_part part, uint32_t num_keys, void* stream,
                     uint32_t* counts_out, float* sums_out, double* sums64_out,
                     scl_result* result) {
    CTX_ENTER(ctx);
    if (!counts_out || !sums_out) return fail(SCL_E_INVALID, "null output table");
    uint32_t* dc = ctx->d_kout;
    float* ds = (float*)(ctx->d_kout + kMaxKeys);
    double* d64 = (double*)(ctx->d_kout + 2 * kMaxKeys);
    SCL_TRY(keyed_common(ctx, part, num_keys, stream, dc, ds, d64, ctx->d_result));
    SCL_CUDA(cudaMemcpyAsync(counts_out, dc, num_keys * 4, cudaMemcpyDeviceToHost, S(stream)));
    SCL_CUDA(cudaMemcpyAsync(sums_out, ds, num_keys * 4, cudaMemcpyDeviceToHost, S(stream)));
    if (sums64_out)
        SCL_CUDA(cudaMemcpyAsync(sums64_out, d64, num_keys * 8, cudaMemcpyDeviceToHost, S(stream)));
    SCL_TRY(fetch_single(ctx, S(stream)));
    if (result) *result = *ctx->h_result;
    if (ctx->h_result->status == SCL_E_KEY_RANGE)
        return fail(SCL_E_KEY_RANGE, "a key outside [0, %u) was skipped", num_keys);
    return SCL_OK;
}

int scl_keyed_reduce_hashed(scl_ctx* ctx, scl_part part, uint32_t num_keys, void* stream,
                            uint32_t* counts_out, float* sums_out, double* sums64_out,
                            scl_result* result) {
    CTX_ENTER(ctx);
    if (!counts_out || !sums_out) return fail(SCL_E_INVALID, "null output table");
    uint32_t* dc = ctx->d_kout;
    float* ds = (float*)(ctx->d_kout + kMaxKeys);
    double* d64 = (double*)(ctx->d_kout + 2 * kMaxKeys);
    SCL_TRY(keyed_common(ctx, part, num_keys, stream, dc, ds, d64, ctx->d_result, K_KEYED_MIX));
    SCL_CUDA(cudaMemcpyAsync(counts_out, dc, num_keys * 4, cudaMemcpyDeviceToHost, S(stream)));
    SCL_CUDA(cudaMemcpyAsync(sums_out, ds, num_keys * 4, cudaMemcpyDeviceToHost, S(stream)));
    if (sums64_out)
        SCL_CUDA(cudaMemcpyAsync(sums64_out, d64, num_keys * 8, cudaMemcpyDeviceToHost, S(stream)));
    SCL_TRY(fetch_single(ctx, S(stream)));
    if (result) *result = *ctx->h_result;
    return SCL_OK;
}

// Bucket tables of the partitioned path: per call (stored in *call_tmp; the
// caller releases it after synchronising) or kept per stream and grown on
// demand.  Null when the arena has no room.
static void* radix_tables(Ctx* c, Scratch& sc, size_t bytes, void** call_tmp) {
    if (call_tmp) return *call_tmp = c->arena.alloc(bytes);
    if (sc.radix && sc.radix_cap >= bytes) return sc.radix;
    if (cudaDeviceSynchronize() != cudaSuccess) return nullptr;   // earlier calls may read it
    if (sc.radix) {
        sc.blocks.erase(std::remove(sc.blocks.begin(), sc.blocks.end(), sc.radix), sc.blocks.end());
        c->arena.release(sc.radix);
        sc.radix = nullptr;
        sc.radix_cap = 0;
    }
    size_t cap = align_up(bytes + bytes / 8);
    void* q = c->arena.alloc(cap);
    if (!q) q = c->arena.alloc(cap = bytes);
    if (!q) return nullptr;
    sc.radix = q;
    sc.radix_cap = cap;
    sc.blocks.push_back(q);
    return q;
}

// The scatter and the wider reduce tables need more than 48 KB of dynamic
// shared memory: allow each variant its size once per device.
static int prepare_radix() {
    static std::mutex mu;
    static std::vector<int> ready;
    int dev = 0;
    SCL_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> g(mu);
    if (std::find(ready.begin(), ready.end(), dev) != ready.end()) return SCL_OK;
    for (uint32_t lt = kRadixMinLogT; lt <= kRadixMaxLogT; ++lt) {
        for (int hot = 0; hot < 2; ++hot)
            SCL_CUDA(cudaFuncSetAttribute(radix_scatter_fn(lt, hot != 0),
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)radix_scatter_smem(kRadixMaxBuckets, hot != 0)));
        SCL_CUDA(cudaFuncSetAttribute(radix_reduce_fn(lt),
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)radix_reduce_smem(lt)));
    }
    ready.push_back(dev);
    return SCL_OK;
}

// Histogram, scan, scatter and per-bucket reduce (radix.h).  *launched is
// false, with nothing enqueued, when the arena has no room for the tables.
static int launch_radix(Ctx* c, Scratch& sc, const Partition& p, uint32_t nk, uint32_t* counts,
                        double* sums64, uint32_t* bad, cudaStream_t st, void** call_tmp,
                        bool* launched) {
    *launched = false;
    SCL_TRY(prepare_radix());
    // the bucket width depends only on num_keys; the chunking on the scatter's residency
    const RadixGeometry g0 = radix_geometry(p.n, nk, 1);
    const void* scatter = radix_scatter_fn(g0.log_t, false);
    const void* scatter_hot = radix_scatter_fn(g0.log_t, true);
    const void* reduce = radix_reduce_fn(g0.log_t);
    const uint32_t rblock = radix_reduce_block(g0.log_t);
    const size_t hist_smem = radix_hist_smem(g0.nb);
    const size_t scat_smem = radix_scatter_smem(g0.nb, false);
    const size_t scat_hot_smem = radix_scatter_smem(g0.nb, true);
    const size_t red_smem = radix_reduce_smem(g0.log_t);
    int occ_h = 0, occ_s = 0, occ_sh = 0, occ_r = 0;
    SCL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_h, radix_hist_fn(), kRadixBlock,
                                                           hist_smem));
    SCL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_s, scatter, kRadixBlock,
                                                           scat_smem));
    SCL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_sh, scatter_hot, kRadixBlock,
                                                           scat_hot_smem));
    SCL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_r, reduce, rblock, red_smem));
    const uint32_t slots_h = (uint32_t)c->sms * std::max(occ_h, 1);
    const uint32_t slots_s = (uint32_t)c->sms * std::max(occ_s, 1);
    const uint32_t slots_sh = (uint32_t)c->sms * std::max(occ_sh, 1);
    const uint32_t slots_r = (uint32_t)c->sms * std::max(occ_r, 1);
    const RadixGeometry g = radix_geometry(p.n, nk, slots_s);
    const RadixLayout l = radix_layout(p.n, g);
    char* t = static_cast<char*>(radix_tables(c, sc, l.total, call_tmp));
    if (!t) return SCL_OK;
    RadixArgs r;
    memset(&r, 0, sizeof r);
    r.keys = static_cast<const char*>(p.d0);
    r.vals = static_cast<const char*>(p.d1);
    r.n = p.n;
    r.num_keys = nk;
    r.nb = g.nb;
    r.chunk = g.chunk;
    r.nchunks = g.nchunks;
    r.log_t = g.log_t;
    r.fixed = radix_bucket_cost(g.log_t);
    r.bk = reinterpret_cast<uint32_t*>(t + l.bk);
    r.hist = reinterpret_cast<uint32_t*>(t + l.hist);
    r.tot = reinterpret_cast<uint32_t*>(t + l.tot);
    r.bstart = reinterpret_cast<uint32_t*>(t + l.bstart);
    r.bcost = reinterpret_cast<uint32_t*>(t + l.bcost);
    r.mode = reinterpret_cast<uint32_t*>(t + l.mode);
    r.counts = counts;
    r.sums64 = sums64;
    r.ticket = sc.hdr + H_RADIX_TICKET;   // reset to zero by the scan's last CTA
    r.bad = bad;
    void* params[] = {&r};
    SCL_CUDA(cudaLaunchKernel(radix_hist_fn(), dim3(std::min(g.nchunks, slots_h)),
                              dim3(kRadixBlock), params, hist_smem, st));
    const uint32_t rows = kRadixScanBlock / 32;   // one warp per bucket row
    SCL_CUDA(cudaLaunchKernel(radix_scan_fn(), dim3((g.nb + 1 + rows - 1) / rows),
                              dim3(kRadixScanBlock), params, 0, st));
    // the scan chose one form (hot ids bypassing the partition or not); the
    // other returns at once
    SCL_CUDA(cudaLaunchKernel(scatter, dim3(std::min(g.nchunks, slots_s)), dim3(kRadixBlock),
                              params, scat_smem, st));
    SCL_CUDA(cudaLaunchKernel(scatter_hot, dim3(std::min(g.nchunks, slots_sh)), dim3(kRadixBlock),
                              params, scat_hot_smem, st));
    SCL_CUDA(cudaLaunchKernel(reduce, dim3(slots_r), dim3(rblock), params, red_smem, st));
    count_launches(5);
    *launched = true;
    return SCL_OK;
}

// Large key spaces: kMinPackedKeys to kMaxPackedKeys keys, the direct kernel with packed
// L2 words (shared table for ids below kMaxKeys, one 64-bit add per other
// pair, count / fp64 adds for values outside the window) and its repair
// chain; above, the bucket-partitioned path for partitions of at least
// kRadixMinPairs aligned pairs when its tables fit the arena; otherwise the
// direct kernel without packing.  Then the finishing pass.
static int launch_large_keyed(scl_ctx* ctx, const Partition& p, uint32_t nk, uint32_t* counts,
                              float* sums, double* sums64, scl_result* res, cudaStream_t st,
                              void** call_tmp) {
    Scratch& sc = ctx->single_for(st);   // per stream: calls on different streams may overlap
    SCL_TRY(ensure_scratch(ctx, &sc, 1, 0, 0, 0));
    LargeKeyedArgs a;
    memset(&a, 0, sizeof a);
    a.keys = static_cast<const char*>(p.d0);
    a.vals = static_cast<const char*>(p.d1);
    a.n = p.n;
    a.num_keys = nk;
    a.aligned = ((uintptr_t)p.d0 % 16) == 0 && ((uintptr_t)p.d1 % 16) == 0;
    a.counts = counts;
    a.sums64 = sums64;
    a.sums32 = sums;
    a.result = res;
    a.ticket = sc.hdr + H_LARGE_TICKET;   // reset to zero by the finishing pass
    a.bad = sc.hdr + H_LARGE_BAD;
    SCL_CUDA(cudaMemsetAsync(res, 0, sizeof(scl_result), st));
    SCL_CUDA(cudaMemsetAsync(a.bad, 0, 4, st));
    void* params[] = {&a};
    bool done = false;   // the partitioned path zeroes the output tables in its first kernel
    // Key spaces of kMinPackedKeys to kMaxPackedKeys: the direct kernel with
    // packed L2 words (one 64-bit add per pair); others: the bucket-
    // partitioned path when its tables fit the arena.
    const int path = ctx->large_path;
    const bool packed = nk > kMaxKeys && nk <= kMaxPackedKeys && p.n &&
                        ((path == SCL_LARGE_AUTO && nk >= kMinPackedKeys) ||
                         path == SCL_LARGE_PACKED);
    if (!packed && (path == SCL_LARGE_AUTO || path == SCL_LARGE_PARTITIONED) && a.aligned &&
        nk > kMaxKeys && p.n >= kRadixMinPairs && p.n <= kRadixMaxPairs)
        SCL_TRY(launch_radix(ctx, sc, p, nk, counts, sums64, a.bad, st, call_tmp, &done));
    if (!done) {
        SCL_CUDA(cudaMemsetAsync(counts, 0, (size_t)nk * 4, st));
        SCL_CUDA(cudaMemsetAsync(sums64, 0, (size_t)nk * 8, st));
    }
    if (packed) {
        char* t = static_cast<char*>(radix_tables(ctx, sc, align_up((size_t)nk * 8) + 256,
                                                  call_tmp));
        if (t) {   // else the direct kernel without packing
            a.packed = reinterpret_cast<unsigned long long*>(t);
            a.fix = reinterpret_cast<LargeFix*>(t + align_up((size_t)nk * 8));
            SCL_CUDA(cudaMemsetAsync(a.packed, 0, (size_t)nk * 8, st));
            SCL_CUDA(cudaLaunchKernel(large_scale_fn(), dim3(1), dim3(256), params, 0, st));
            count_launches(1);
        }
    }
    const void* fn = large_keyed_kernel_fn(a.aligned);
    int nb = 0;
    SCL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 256, 0));
    const uint64_t pieces = (p.n + kDirectPiece - 1) / kDirectPiece;
    const uint32_t grid = (uint32_t)std::max<uint64_t>(
        1, std::min<uint64_t>(pieces, (uint64_t)ctx->sms * std::max(nb, 1)));
    if (p.n && !done) {
        SCL_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(256), params, 0, st));
        count_launches(1);
    }
    // two CTAs per SM: each CTA adds its totals with three atomics on the same
    // three words, so fewer CTAs wait less on them
    const uint32_t fgrid = (uint32_t)std::max<uint64_t>(
        1, std::min<uint64_t>(((uint64_t)nk + 255) / 256, (uint64_t)ctx->sms * 2));
    SCL_CUDA(cudaLaunchKernel(large_keyed_finish_fn(), dim3(fgrid), dim3(256), params, 0, st));
    count_launches(1);
    if (a.packed) {
        // The repair chain: each kernel returns at once unless the finishing
        // pass found that a packed word overflowed; then the outputs are
        // zeroed and the call is done again without packing.
        LargeKeyedArgs r = a;
        r.packed = nullptr;
        r.guard = 1u;
        void* rparams[] = {&r};
        const uint32_t zgrid = (uint32_t)std::max<uint64_t>(
            1, std::min<uint64_t>(((uint64_t)nk + 255) / 256, (uint64_t)ctx->sms * 4));
        SCL_CUDA(cudaLaunchKernel(large_repair_zero_fn(), dim3(zgrid), dim3(256), rparams, 0, st));
        SCL_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(256), rparams, 0, st));
        SCL_CUDA(cudaLaunchKernel(large_keyed_finish_fn(), dim3(fgrid), dim3(256), rparams, 0, st));
        count_launches(3);
    }
    return SCL_OK;
}

int scl_set_large_path(scl_ctx* ctx, scl_large_path path) {
    CTX_ENTER(ctx);
    if ((int)path < SCL_LARGE_AUTO || (int)path > SCL_LARGE_DIRECT)
        return fail(SCL_E_INVALID, "unknown large-key path %d", (int)path);
    ctx->large_path = (int)path;
    return SCL_OK;
}

static int large_part(scl_ctx* ctx, scl_part part, uint32_t nk, const Partition** out) {
    const Partition* p = ctx->part(part);
    if (!p) return fail(SCL_E_INVALID, "unknown partition handle");
    if (p->dtype != SCL_KV_I32_F32) return fail(SCL_E_UNSUPPORTED, "partition is not keyed");
    if (nk < 1 || nk > kMaxLargeKeys)
        return fail(SCL_E_INVALID, "num_keys %u not in [1, %u]", nk, kMaxLargeKeys);
    *out = p;
    return SCL_OK;
}

int scl_keyed_reduce_large_async(scl_ctx* ctx, scl_part part, uint32_t num_keys, void* stream,
                                 uint32_t* counts_dev, float* sums_dev, double* sums64_dev,
                                 scl_result* dev_result) {
    CTX_ENTER(ctx);
    const Partition* p = nullptr;
    SCL_TRY(large_part(ctx, part, num_keys, &p));
    if (!counts_dev || !sums_dev || !sums64_dev || !dev_result)
        return fail(SCL_E_INVALID, "all device tables and the result are required");
    return launch_large_keyed(ctx, *p, num_keys, counts_dev, sums_dev, sums64_dev, dev_result,
                              S(stream), nullptr);
}

int scl_keyed_reduce_large(scl_ctx* ctx, scl_part part, uint32_t num_keys, void* stream,
                           uint32_t* counts_out, float* sums_out, double* sums64_out,
                           scl_result* result) {
    CTX_ENTER(ctx);
    const Partition* p = nullptr;
    SCL_TRY(large_part(ctx, part, num_keys, &p));
    if (!counts_out || !sums_out) return fail(SCL_E_INVALID, "null output table");
    const size_t nk = num_keys;
    char* buf = (char*)ctx->arena.alloc(nk * 16 + kAlign);
    if (!buf) return fail(SCL_E_NOMEM, "arena: no room for %u-key tables", num_keys);
    double* d64 = (double*)buf;
    uint32_t* dc = (uint32_t*)(buf + nk * 8);
    float* ds = (float*)(buf + nk * 12);
    scl_result* dr = (scl_result*)(buf + align_up(nk * 16));
    void* tmp = nullptr;   // bucket tables of the partitioned path, if it runs
    int st = launch_large_keyed(ctx, *p, num_keys, dc, ds, d64, dr, S(stream), &tmp);
    if (st == SCL_OK) {
        cudaStream_t s = S(stream);
        if (cudaMemcpyAsync(counts_out, dc, nk * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(sums_out, ds, nk * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            (sums64_out &&
             cudaMemcpyAsync(sums64_out, d64, nk * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
            cudaMemcpyAsync(ctx->h_result, dr, sizeof(scl_result), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = fail(SCL_E_CUDA, "large keyed reduce: copy back failed");
    }
    cudaStreamSynchronize(S(stream));
    ctx->arena.release(buf);
    if (tmp) ctx->arena.release(tmp);
    if (st != SCL_OK) return st;
    if (result) *result = *ctx->h_result;
    if (ctx->h_result->status == SCL_E_TIMEOUT)
        return fail(SCL_E_TIMEOUT, "a bounded device wait gave up");
    if (ctx->h_result->status == SCL_E_STATE)
        return fail(SCL_E_STATE, "the keys changed while the call read them");
    if (ctx->h_result->status == SCL_E_KEY_RANGE)
        return fail(SCL_E_KEY_RANGE, "a key outside [0, %u) was skipped", num_keys);
    return SCL_OK;
}

int scl_keyed_reduce_async(scl_ctx* ctx, scl_part part, uint32_t num_keys, void* stream,
                           uint32_t* counts_out, float* sums_out, double* sums64_out,
                           scl_result* dev_result) {
    CTX_ENTER(ctx);
    if (!counts_out || !sums_out) return fail(SCL_E_INVALID, "null output table");
    return keyed_common(ctx, part, num_keys, stream, counts_out, sums_out, sums64_out,
                        dev_result ? dev_result : ctx->d_result);
}

// ------------------------------------------------ ReduceCL over arrays

static bool int_class(scl_dtype d) { return d == SCL_U32 || d == SCL_I32; }

static int check_arrays(scl_ctx* ctx, const scl_part* parts, uint32_t k,
                        std::vector<Partition>* ps) {
    if (!parts || k < 1 || k > kMaxTreeArrays)
        return fail(SCL_E_INVALID, "need 1..%u partitions", kMaxTreeArrays);
    ps->resize(k);
    for (uint32_t j = 0; j < k; ++j) {
        const Partition* p = ctx->part(parts[j]);
        if (!p) return fail(SCL_E_INVALID, "partition %u: unknown handle", j);
        if (p->dtype == SCL_KV_I32_F32)
            return fail(SCL_E_UNSUPPORTED, "keyed partitions cannot be added elementwise");
        (*ps)[j] = *p;
        if (p->n != (*ps)[0].n) return fail(SCL_E_INVALID, "partition %u differs in length", j);
        if (int_class(p->dtype) != int_class((*ps)[0].dtype))
            return fail(SCL_E_INVALID, "partition %u differs in dtype class", j);
    }
    return SCL_OK;
}

static int launch_tree_add(scl_ctx* ctx, const std::vector<Partition>& ps, void* out,
                           cudaStream_t st) {
    const uint64_t n = ps[0].n;
    if (!n) return SCL_OK;
    TreeArgs a;
    memset(&a, 0, sizeof a);
    bool aligned = ((uintptr_t)out % 16) == 0;
    for (size_t j = 0; j < ps.size(); ++j) {
        a.in[j] = static_cast<const char*>(ps[j].d0);
        aligned = aligned && ((uintptr_t)ps[j].d0 % 16) == 0;
    }
    a.out = static_cast<char*>(out);
    a.n = n;
    a.k = (uint32_t)ps.size();
    const int f32 = ps[0].dtype == SCL_F32;
    const void* fn = tree_add_kernel_fn(f32, aligned, a.k);
    int nb = 0;
    SCL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 256, 0));
    const uint64_t work = aligned ? (n + 3) / 4 : n;
    const uint64_t want = (work + 255) / 256;
    const uint32_t grid = (uint32_t)std::max<uint64_t>(
        1, std::min<uint64_t>(want, (uint64_t)ctx->sms * std::max(nb, 1)));
    void* params[] = {&a};
    SCL_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(256), params, 0, st));
    count_launches(1);
    return SCL_OK;
}

int scl_reduce_arrays_into(scl_ctx* ctx, const scl_part* parts, uint32_t k, scl_part out,
                           void* stream) {
    CTX_ENTER(ctx);
    std::vector<Partition> ps;
    SCL_TRY(check_arrays(ctx, parts, k, &ps));
    const Partition* o = ctx->part(out);
    if (!o) return fail(SCL_E_INVALID, "unknown output partition");
    if (o->n != ps[0].n || o->dtype == SCL_KV_I32_F32 ||
        int_class(o->dtype) != int_class(ps[0].dtype))
        return fail(SCL_E_INVALID, "output partition must match the inputs' length and dtype");
    return launch_tree_add(ctx, ps, o->d0, S(stream));
}

int scl_reduce_arrays(scl_ctx* ctx, const scl_part* parts, uint32_t k, void* stream,
                      scl_part* out) {
    CTX_ENTER(ctx);
    if (!out) return fail(SCL_E_INVALID, "null output");
    std::vector<Partition> ps;
    SCL_TRY(check_arrays(ctx, parts, k, &ps));
    Partition o;
    SCL_TRY(new_partition(ctx, ps[0].dtype, ps[0].n, &o));
    const int st = launch_tree_add(ctx, ps, o.d0, S(stream));
    if (st != SCL_OK) {
        ctx->arena.release(o.block);
        return st;
    }
    *out = register_partition(ctx, o);
    return SCL_OK;
}

int scl_vector_add(scl_ctx* ctx, scl_part a, scl_part b, void* stream, scl_part* out) {
    const scl_part parts[2] = {a, b};
    return scl_reduce_arrays(ctx, parts, 2, stream, out);
}

// ----------------------------------------------------------------- combine

int scl_combine(const scl_result* parts, uint32_t k, scl_result* out) {
    clear_error();
    if (!out || (k && !parts)) return fail(SCL_E_INVALID, "null argument");
    scl_result r;
    memset(&r, 0, sizeof r);
    r.f32_min = INFINITY;
    r.f32_max = -INFINITY;
    r.status = SCL_OK;
    for (uint32_t i = 0; i < k; ++i) {
        r.u64_sum += parts[i].u64_sum;
        r.n += parts[i].n;
        if (parts[i].f32_min == parts[i].f32_min && parts[i].f32_min < r.f32_min)
            r.f32_min = parts[i].f32_min;
        if (parts[i].f32_max == parts[i].f32_max && parts[i].f32_max > r.f32_max)
            r.f32_max = parts[i].f32_max;
        if (r.status == SCL_OK && parts[i].status != SCL_OK) r.status = parts[i].status;
    }
    if (k) {
        r.f64_sum = pairwise_sum(parts, 0, k);
        r.kind = parts[0].kind;
    }
    r.f32_sum = (float)r.f64_sum;
    *out = r;
    return SCL_OK;
}

int scl_combine_keyed(const uint32_t* counts, const double* sums64, uint32_t k, uint32_t num_keys,
                      uint32_t* counts_out, double* sums64_out) {
    clear_error();
    if (!counts_out || (k && !counts) || (sums64 && !sums64_out))
        return fail(SCL_E_INVALID, "null argument");
    std::vector<double> col(k);
    for (uint32_t j = 0; j < num_keys; ++j) {
        uint32_t c = 0;
        for (uint32_t i = 0; i < k; ++i) c += counts[(size_t)i * num_keys + j];
        counts_out[j] = c;
        if (sums64) {
            // pairwise tree over the k partitions
            for (uint32_t i = 0; i < k; ++i) col[i] = sums64[(size_t)i * num_keys + j];
            uint32_t m = k;
            while (m > 1) {
                uint32_t h = (m + 1) / 2;
                for (uint32_t i = 0; i + h < m; ++i) col[i] += col[i + h];
                m = h;
            }
            sums64_out[j] = k ? col[0] : 0.0;
        }
    }
    return SCL_OK;
}

// ------------------------------------------------------------ launch shapes

int scl_get_shape(scl_ctx* ctx, int family, scl_shape* out) {
    CTX_ENTER(ctx);
    if (!out || family < 0 || family >= M_NUM) return fail(SCL_E_INVALID, "bad family or output");
    const Shape s = ctx->shape_for(family);
    out->block = s.block;
    out->items_per_thread = s.ipt;
    out->ctas_per_sm = s.ctas_per_sm;
    out->path = s.path;
    out->stages = find_entry(family, s) ? find_entry(family, s)->stages : s.stages;
    out->reserved = 0;
    return SCL_OK;
}

int scl_set_shape(scl_ctx* ctx, int family, const scl_shape* in) {
    CTX_ENTER(ctx);
    if (!in || family < 0 || family >= M_NUM) return fail(SCL_E_INVALID, "bad family or shape");
    Shape s{in->block, in->items_per_thread, in->ctas_per_sm, in->path, in->stages};
    if (in->ctas_per_sm < 0) return fail(SCL_E_INVALID, "ctas_per_sm must be >= 0");
    if (family == M_ALL) {   // block / items per thread follow the F32 family
        s.block = ctx->shape[M_F32].block;
        s.ipt = ctx->shape[M_F32].ipt;
        if (in->path != PATH_LDG) return fail(SCL_E_UNSUPPORTED, "mixed batches use path 0");
    }
    if (!find_entry(family, s))
        return fail(SCL_E_UNSUPPORTED, "shape %d x %d path %d stages %d is not compiled",
                    s.block, s.ipt, s.path, s.stages);
    ctx->shape[family] = s;
    return SCL_OK;
}

int scl_autotune(scl_ctx* ctx, const scl_autotune_config* cfg, void* stream,
                 scl_autotune_report* report) {
    CTX_ENTER(ctx);
    return autotune(ctx, cfg, S(stream), report);
}

// ----------------------------------------------------------------- batches

int scl_batch_create(scl_ctx* ctx, const scl_task* tasks, uint32_t ntasks, scl_batch** out) {
    CTX_ENTER(ctx);
    if (!out || (ntasks && !tasks)) return fail(SCL_E_INVALID, "null argument");
    *out = nullptr;
    scl_batch* b = new (std::nothrow) scl_batch();
    if (!b) return fail(SCL_E_NOMEM, "host allocation failed");
    b->ctx = ctx;
    b->ntasks = ntasks;
    int st = SCL_OK;
    auto bail = [&](int code) {
        cudaDeviceSynchronize();
        batch_release(b);
        delete b;
        return code;
    };
    if (ntasks == 0) {
        *out = b;
        return SCL_OK;
    }
    // One plan over every task validates them and resolves their kinds.
    Plan all;
    st = plan_tasks(ctx, tasks, ntasks, &all);
    if (st != SCL_OK) return bail(st);
    std::vector<std::vector<uint32_t>> fam;
    if (ctx->batch_split && all.mask == M_ALL) {
        fam.resize(3);   // launch order: keyed (the longest), uint32, fp32
        for (uint32_t i = 0; i < ntasks; ++i) {
            const int m = mask_of_kind(all.tasks[i].kind);
            fam[m == M_KEYED ? 0 : m == M_U32 ? 1 : 2].push_back(i);
        }
        fam.erase(std::remove_if(fam.begin(), fam.end(),
                                 [](const std::vector<uint32_t>& v) { return v.empty(); }),
                  fam.end());
    } else {
        fam.emplace_back(ntasks);
        for (uint32_t i = 0; i < ntasks; ++i) fam[0][i] = i;
    }
    const size_t ng = fam.size();
    const size_t o_tk = align_up(ntasks * sizeof(scl_result));
    const size_t o_fl = o_tk + align_up(ntasks * 4ull);
    const size_t o_hdr = o_fl + align_up(ntasks * 4ull);
    b->scratch_bytes = o_hdr + ng * align_up(H_WORDS * 4);
    b->scratch = ctx->arena.alloc(b->scratch_bytes);
    if (!b->scratch)
        return bail(fail(SCL_E_NOMEM, "arena: no block of %zu bytes for the batch", b->scratch_bytes));
    char* z = static_cast<char*>(b->scratch);
    b->results = reinterpret_cast<scl_result*>(z);
    b->hdr = reinterpret_cast<uint32_t*>(z + o_hdr);
    if (cudaMemset(z, 0, b->scratch_bytes) != cudaSuccess)
        return bail(fail(SCL_E_CUDA, "zeroing the batch scratch failed"));
    std::vector<scl_task> sub;
    for (size_t g = 0; g < ng; ++g) {
        scl_batch::Group& G = b->groups.emplace_back();
        G.first = (uint32_t)b->order.size();
        G.count = (uint32_t)fam[g].size();
        sub.clear();
        for (uint32_t i : fam[g]) {
            b->order.push_back(i);
            sub.push_back(tasks[i]);
        }
        // keyed tasks beside streaming groups: the register-capped keyed kernel
        const Shape lean{kLeanKeyedBlock, kLeanKeyedIpt, 2, PATH_LEAN, 0};
        const bool beside = ng > 1 && fam[g].size() && is_keyed(all.tasks[fam[g][0]].kind);
        st = plan_tasks(ctx, sub.data(), G.count, &G.plan, beside ? &lean : nullptr);
        if (st != SCL_OK) return bail(st);
        ExternalScratch ext;
        ext.results = b->results + G.first;
        ext.tickets = reinterpret_cast<uint32_t*>(z + o_tk) + G.first;
        ext.flags = reinterpret_cast<uint32_t*>(z + o_fl) + G.first;
        ext.hdr = b->hdr + g * (align_up(H_WORDS * 4) / 4);
        ext.task_cap = G.count;
        std::vector<char> host;
        st = build_image(ctx, G.plan, &G.img, &host, &G.args, &ext);
        if (st != SCL_OK) return bail(st);
        if (cudaMemcpy(G.img.block, host.data(), G.img.plan_bytes, cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return bail(fail(SCL_E_CUDA, "uploading the batch plan failed"));
        b->kernels += 1u + (G.plan.fold_tasks.empty() ? 0u : 1u);
    }
    for (size_t g = 1; g < ng; ++g)
        if (cudaStreamCreateWithFlags(&b->side[g - 1], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->join[g - 1], cudaEventDisableTiming) != cudaSuccess)
            return bail(fail(SCL_E_CUDA, "creating the batch's side streams failed"));
    if (ng > 1 && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(SCL_E_CUDA, "creating the batch's fork event failed"));
    if (cudaDeviceSynchronize() != cudaSuccess)   // order before launches on any stream
        return bail(fail(SCL_E_CUDA, "uploading the batch plan failed"));
    b->staged.resize(ntasks);
    *out = b;
    return SCL_OK;
}

int scl_batch_launch(scl_batch* b, void* stream) {
    if (!b) return fail(SCL_E_INVALID, "null batch");
    CTX_ENTER(b->ctx);
    if (b->exec) {
        SCL_CUDA(cudaGraphLaunch(b->exec, S(stream)));
        count_launches(b->kernels);
        return SCL_OK;
    }
    if (b->groups.empty()) return SCL_OK;
    return batch_launch_groups(b, S(stream));
}

int scl_batch_capture(scl_batch* b, void* stream) {
    if (!b) return fail(SCL_E_INVALID, "null batch");
    CTX_ENTER(b->ctx);
    if (b->exec || b->groups.empty()) return SCL_OK;
    SCL_CUDA(cudaStreamBeginCapture(S(stream), cudaStreamCaptureModeThreadLocal));
    const uint64_t before = launches_total();
    int st = batch_launch_groups(b, S(stream));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(S(stream), &g);
    count_launches(0 - (launches_total() - before));   // capture launched nothing
    if (st != SCL_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(SCL_E_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(SCL_E_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    }
    b->graph = g;
    b->exec = x;
    return SCL_OK;
}

int scl_batch_results(scl_batch* b, void* stream, scl_result* results) {
    if (!b) return fail(SCL_E_INVALID, "null batch");
    CTX_ENTER(b->ctx);
    if (b->ntasks && !results) return fail(SCL_E_INVALID, "null results");
    if (!b->ntasks) return SCL_OK;
    const size_t hw = align_up(H_WORDS * 4) / 4;
    std::vector<uint32_t> hdr(b->groups.size() * hw);
    SCL_CUDA(cudaMemcpyAsync(b->staged.data(), b->results, b->ntasks * sizeof(scl_result),
                             cudaMemcpyDeviceToHost, S(stream)));
    SCL_CUDA(cudaMemcpyAsync(hdr.data(), b->hdr, hdr.size() * 4, cudaMemcpyDeviceToHost, S(stream)));
    SCL_CUDA(cudaStreamSynchronize(S(stream)));
    uint32_t err = 0;
    for (size_t g = 0; g < b->groups.size(); ++g) err |= hdr[g * hw + H_ERROR];
    if (err) {
        SCL_CUDA(cudaMemset(b->scratch, 0, b->scratch_bytes));
        SCL_CUDA(cudaDeviceSynchronize());
        return fail((err & 4u) ? SCL_E_TIMEOUT : SCL_E_STATE,
                    "device error word 0x%x after the batch", err);
    }
    for (uint32_t p = 0; p < b->ntasks; ++p) results[b->order[p]] = b->staged[p];
    for (uint32_t i = 0; i < b->ntasks; ++i)
        if (results[i].status == SCL_E_KEY_RANGE)
            return fail(SCL_E_KEY_RANGE, "task %u saw a key out of range", i);
    return SCL_OK;
}

int scl_set_batch_split(scl_ctx* ctx, int on) {
    CTX_ENTER(ctx);
    if (on != 0 && on != 1) return fail(SCL_E_INVALID, "batch split must be 0 or 1, not %d", on);
    ctx->batch_split = on;
    return SCL_OK;
}

int scl_batch_kernel_launches(scl_batch* b, uint32_t* count) {
    if (!b || !count) return fail(SCL_E_INVALID, "null argument");
    *count = b->kernels;
    return SCL_OK;
}

int scl_batch_destroy(scl_batch* b) {
    if (!b) return SCL_OK;
    {
        std::lock_guard<std::recursive_mutex> g(b->ctx->mu);
        cudaSetDevice(b->ctx->device);
        cudaDeviceSynchronize();
        batch_release(b);
    }
    delete b;
    return SCL_OK;
}

int scl_batch_run(scl_ctx* ctx, const scl_task* tasks, uint32_t ntasks, void* stream,
                  scl_result* results) {
    scl_batch* b = nullptr;
    SCL_TRY(scl_batch_create(ctx, tasks, ntasks, &b));
    int st = scl_batch_launch(b, stream);
    if (st == SCL_OK) st = scl_batch_results(b, stream, results);
    std::string keep = last_error();
    scl_batch_destroy(b);
    if (st != SCL_OK) return fail(st, "%s", keep.c_str());
    return SCL_OK;
}

}  // extern "C"
