// runtime.cu -- host runtime of libscl: errors, arena, kernel lookup, the
// single-partition launch and the batch planner.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>

#include "plan_keyed.h"
#include "runtime.h"

namespace scl {

const KernelEntry* kernel_table_u32(int* count);
const KernelEntry* kernel_table_f32(int* count);
const KernelEntry* kernel_table_keyed(int* count);
const KernelEntry* kernel_table_keyed_lean(int* count);
const KernelEntry* kernel_table_all(int* count);
const KernelEntry* kernel_table_tma_u32(int* count);
const KernelEntry* kernel_table_tma_f32(int* count);

// ------------------------------------------------------------------ errors

static thread_local std::string t_err;

int fail(int code, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return code;
}

void clear_error() { t_err.clear(); }
const char* last_error() { return t_err.c_str(); }

static std::atomic<uint64_t> g_launches{0};
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
uint64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }

// ------------------------------------------------------------------- arena

void Arena::init(char* base, size_t size) {
    std::lock_guard<std::mutex> g(mu_);
    base_ = base;
    size_ = size / kAlign * kAlign;
    free_.clear();
    used_.clear();
    if (size_) free_[0] = size_;
}

void* Arena::alloc(size_t bytes) {
    bytes = align_up(bytes ? bytes : 1);
    std::lock_guard<std::mutex> g(mu_);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
        if (it->second < bytes) continue;
        const size_t off = it->first, sz = it->second;
        free_.erase(it);
        if (sz > bytes) free_[off + bytes] = sz - bytes;
        used_[off] = bytes;
        return base_ + off;
    }
    return nullptr;
}

void Arena::release(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> g(mu_);
    const size_t off = (size_t)((char*)p - base_);
    auto u = used_.find(off);
    if (u == used_.end()) return;
    size_t start = off, sz = u->second;
    used_.erase(u);
    auto nx = free_.lower_bound(start);
    if (nx != free_.end() && nx->first == start + sz) {
        sz += nx->second;
        nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {
        auto pv = std::prev(nx);
        if (pv->first + pv->second == start) {
            start = pv->first;
            sz += pv->second;
            free_.erase(pv);
        }
    }
    free_[start] = sz;
}

size_t Arena::free_bytes() {
    std::lock_guard<std::mutex> g(mu_);
    size_t s = 0;
    for (auto& kv : free_) s += kv.second;
    return s;
}

size_t Arena::largest_free() {
    std::lock_guard<std::mutex> g(mu_);
    size_t s = 0;
    for (auto& kv : free_) s = std::max(s, kv.second);
    return s;
}

// ----------------------------------------------------------- kernel lookup

static const KernelEntry* table(int mask, int* count) {
    switch (mask) {
        case M_U32: return kernel_table_u32(count);
        case M_F32: return kernel_table_f32(count);
        case M_KEYED: return kernel_table_keyed(count);
        default: return kernel_table_all(count);
    }
}

const KernelEntry* find_entry(int mask, int block, int ipt, int path, int stages) {
    int n = 0;
    const KernelEntry* t = nullptr;
    if (path == PATH_TMA) {
        if (mask == M_U32) t = kernel_table_tma_u32(&n);
        else if (mask == M_F32) t = kernel_table_tma_f32(&n);
        else return nullptr;
    } else if (path == PATH_LEAN) {
        if (mask != M_KEYED) return nullptr;
        t = kernel_table_keyed_lean(&n);
    } else {
        t = table(mask, &n);
    }
    for (int i = 0; i < n; ++i)
        if (t[i].block == block && t[i].ipt == ipt && (stages == 0 || t[i].stages == stages))
            return &t[i];
    return nullptr;
}

int prepare_entry(const KernelEntry* e) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, bool> done;
    int dev = 0;
    SCL_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_pair(e->fn, dev);
    if (done.count(key)) return SCL_OK;
    if (e->dyn_smem > 48 * 1024)
        SCL_CUDA(cudaFuncSetAttribute(e->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)e->dyn_smem));
    done[key] = true;
    return SCL_OK;
}

int mask_of_kind(uint32_t kind) {
    switch (kind) {
        case K_U32_IDENT:
        case K_U32_MIX32: return M_U32;
        case K_F32_IDENT:
        case K_F32_POLY3: return M_F32;
        default: return M_KEYED;
    }
}

int resolve_kind(scl_dtype dt, int kernel, int reduce, uint32_t* kind) {
    switch (dt) {
        case SCL_U32:
        case SCL_I32:
            if (reduce != SCL_R_SUM) break;
            if (kernel == SCL_K_IDENT) { *kind = K_U32_IDENT; return SCL_OK; }
            if (kernel == SCL_K_MIX32) { *kind = K_U32_MIX32; return SCL_OK; }
            break;
        case SCL_F32:
            if (reduce != SCL_R_SUM && reduce != SCL_R_SUM_MIN_MAX) break;
            if (kernel == SCL_K_IDENT) { *kind = K_F32_IDENT; return SCL_OK; }
            if (kernel == SCL_K_POLY3) { *kind = K_F32_POLY3; return SCL_OK; }
            break;
        case SCL_KV_I32_F32:
            if (reduce == SCL_R_KEYED_COUNT_SUM && kernel == SCL_K_IDENT) {
                *kind = K_KEYED;
                return SCL_OK;
            }
            if (reduce == SCL_R_KEYED_COUNT_SUM && kernel == SCL_K_MIX32) {
                *kind = K_KEYED_MIX;
                return SCL_OK;
            }
            break;
        default:
            return fail(SCL_E_INVALID, "unknown dtype %d", (int)dt);
    }
    return fail(SCL_E_UNSUPPORTED, "no catalogue kernel for dtype %d, map %d, reduce %d",
                (int)dt, kernel, reduce);
}

// ------------------------------------------------------------ launch shape

// F32 tasks must see the same (block, items-per-thread) whether they run
// alone or inside a mixed batch, so the mixed kernel borrows the fp32 shape.
Shape Ctx::shape_for(int mask) const {
    Shape s = shape[mask];
    if (mask == M_ALL) {
        s.block = shape[M_F32].block;
        s.ipt = shape[M_F32].ipt;
        s.path = PATH_LDG;
        s.stages = 0;
    }
    return s;
}

uint32_t Ctx::grid_max(int mask, const Shape& sh) {
    const KernelEntry* e = find_entry(mask, sh);
    if (!e) return 1;
    int nb = 0;
    auto it = occ_cache.find(e->fn);
    if (it != occ_cache.end()) {
        nb = it->second;
    } else {
        if (prepare_entry(e) != SCL_OK ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, e->fn, launch_threads(*e),
                                                          e->dyn_smem) != cudaSuccess)
            nb = 1;
        if (nb < 1) nb = 1;
        occ_cache[e->fn] = nb;
    }
    const int per = sh.ctas_per_sm > 0 ? std::min(sh.ctas_per_sm, nb) : nb;
    return (uint32_t)(sms * per);
}

// ----------------------------------------------------------------- scratch

static int grow(Ctx* c, void** p, size_t* cap, size_t need, size_t elem, bool zero,
                std::vector<void*>& blocks) {
    if (*cap >= need && *p) return SCL_OK;
    size_t n = std::max<size_t>(need, 64);
    size_t pow2 = 64;
    while (pow2 < n) pow2 <<= 1;
    // Work already enqueued may still read the old block.
    SCL_CUDA(cudaDeviceSynchronize());
    if (*p) {
        blocks.erase(std::remove(blocks.begin(), blocks.end(), *p), blocks.end());
        c->arena.release(*p);
        *p = nullptr;
        *cap = 0;
    }
    void* q = c->arena.alloc(pow2 * elem);
    if (!q) return fail(SCL_E_NOMEM, "arena: no block of %zu bytes for scratch", pow2 * elem);
    if (zero) {
        // cudaMemset runs on the legacy stream, which does not order against
        // non-blocking streams: finish it before any launch can see the block
        SCL_CUDA(cudaMemset(q, 0, pow2 * elem));
        SCL_CUDA(cudaDeviceSynchronize());
    }
    blocks.push_back(q);
    *p = q;
    *cap = pow2;
    return SCL_OK;
}

int ensure_scratch(Ctx* c, Scratch* s, size_t tasks, size_t sslots, size_t kslots,
                   size_t fparts) {
    if (!s->hdr) {
        void* h = c->arena.alloc(H_WORDS * 4);
        if (!h) return fail(SCL_E_NOMEM, "arena: no room for scratch header");
        SCL_CUDA(cudaMemset(h, 0, H_WORDS * 4));
        SCL_CUDA(cudaDeviceSynchronize());
        s->hdr = (uint32_t*)h;
        s->blocks.push_back(h);
    }
    if (s->task_cap < tasks || !s->tickets) {
        size_t cap = s->task_cap;
        void* t = s->tickets;
        SCL_TRY(grow(c, &t, &cap, tasks, 4, true, s->blocks));
        size_t cap2 = s->task_cap;
        void* f = s->flags;
        SCL_TRY(grow(c, &f, &cap2, tasks, 4, true, s->blocks));
        s->tickets = (uint32_t*)t;
        s->flags = (uint32_t*)f;
        s->task_cap = std::min(cap, cap2);
    }
    if (sslots) {
        void* p = s->spart;
        SCL_TRY(grow(c, &p, &s->spart_cap, sslots, sizeof(StreamPartial), false, s->blocks));
        s->spart = (StreamPartial*)p;
    }
    if (kslots) {
        void* p = s->kpart;
        SCL_TRY(grow(c, &p, &s->kpart_cap, kslots, (size_t)kKeyedTableWords * 4, false, s->blocks));
        s->kpart = (uint32_t*)p;
    }
    if (fparts) {
        void* p = s->fpart;
        SCL_TRY(grow(c, &p, &s->fpart_cap, fparts, sizeof(StreamPartial), false, s->blocks));
        s->fpart = (StreamPartial*)p;
    }
    return SCL_OK;
}

void fill_task(DevTask* t, const Partition& p, uint32_t kind, const float* coef, uint32_t nk) {
    memset(t, 0, sizeof *t);
    t->in0 = p.d0;
    t->in1 = p.d1;
    t->n = p.n;
    t->kind = kind;
    t->num_keys = nk;
    static const float kDef[3] = {0.5f, -1.25f, 0.1f};
    const float* cf = coef ? coef : kDef;
    t->coef[0] = cf[0];
    t->coef[1] = cf[1];
    t->coef[2] = cf[2];
    const bool al = ((uintptr_t)p.d0 % 16 == 0) && (!p.d1 || (uintptr_t)p.d1 % 16 == 0);
    t->flags = al ? TF_ALIGNED : 0u;
}

// --------------------------------------------------------- single launches

static int launch_entry(const KernelEntry* e, uint32_t grid, const KernelArgs& args,
                        cudaStream_t st) {
    SCL_TRY(prepare_entry(e));
    void* params[] = {const_cast<KernelArgs*>(&args)};
    SCL_CUDA(cudaLaunchKernel(e->fn, dim3(grid), dim3(launch_threads(*e)), params, e->dyn_smem, st));
    count_launches(1);
    return SCL_OK;
}

int run_single(Ctx* c, const Partition& p, uint32_t kind, const float* coef, uint32_t nk,
               uint32_t* counts, float* sums, double* sums64, scl_result* dres,
               cudaStream_t st, uint32_t* err_out) {
    const int mask = mask_of_kind(kind);
    const Shape sh = c->shape_for(mask);
    const KernelEntry* e = find_entry(mask, sh);
    if (!e) return fail(SCL_E_STATE, "no kernel for shape %d x %d", sh.block, sh.ipt);
    const uint32_t gmax = c->grid_max(mask, sh);

    KernelArgs a;
    memset(&a, 0, sizeof a);
    fill_task(&a.single, p, kind, coef, nk);
    DevTask& t = a.single;
    t.result = dres;
    t.counts_out = counts;
    t.sums_out = sums;
    t.sums64_out = sums64;
    uint32_t grid;
    Scratch& sc = c->single_for(st);
    if (is_keyed(kind)) {
        const uint32_t G = keyed_single_pieces(p.n, gmax);
        t.nseg = G;
        a.nkeyed_ctas = G;
        grid = G;
        SCL_TRY(ensure_scratch(c, &sc, 1, 0, G > 1 ? G : 0, kMaxKeys / kFoldBlock));
    } else {
        const uint32_t chunk = (uint32_t)(sh.block * sh.ipt * 4);
        t.seg_elems = stream_seg_elems(p.n, chunk);
        t.nseg = stream_nseg(p.n, t.seg_elems);
        a.nseg_stream = t.nseg;
        grid = std::min(gmax, t.nseg);
        SCL_TRY(ensure_scratch(c, &sc, 1, t.nseg, 0, 0));
    }
    a.spart = sc.spart;
    a.kpart = sc.kpart;
    a.fpart = sc.fpart;
    a.tickets = sc.tickets;
    a.task_flags = sc.flags;
    a.hdr = sc.hdr;
    a.err_out = err_out;
    SCL_TRY(launch_entry(e, grid, a, st));
    if (is_keyed(kind) && t.nseg > kFoldInKernelMaxPieces) {   // else its last piece folds it
        const uint32_t nkb = (nk + kFoldBlock - 1) / kFoldBlock;
        void* params[] = {&a};
        SCL_CUDA(cudaLaunchKernel(fold_kernel_fn(), dim3(nkb, 1), dim3(kFoldBlock), params, 0, st));
        count_launches(1);
    }
    return SCL_OK;
}

// ----------------------------------------------------------------- planner

// The fixed cost of a keyed piece in pair-equivalents: zeroing the table,
// the window scan, the first loads, the end-of-piece barriers and the
// write-out, at the rate a CTA adds pairs.  Measured on the 10,000-task
// batch's 3,374 keyed tasks (log-normal lengths, median 16 Ki pairs): the
// keyed-only kernel (fixed-point window) balances best at 32 pairs per
// thread of the CTA, the mixed kernel (fp32 table) at 16.
static uint64_t keyed_piece_overhead(int mask, const Shape& s) {
    return (uint64_t)s.block * (mask == M_KEYED ? kKeyedPieceOverheadFast : kKeyedPieceOverheadMixed);
}

int plan_tasks(Ctx* c, const scl_task* in, uint32_t nt, Plan* P, const Shape* shape) {
    P->tasks.assign(nt, DevTask{});
    bool has_u32 = false, has_f32 = false, has_keyed = false;
    std::vector<uint32_t> kind(nt);
    for (uint32_t i = 0; i < nt; ++i) {
        const Partition* p = c->part(in[i].part);
        if (!p) return fail(SCL_E_INVALID, "task %u: unknown partition handle %llu", i,
                            (unsigned long long)in[i].part);
        SCL_TRY(resolve_kind(p->dtype, in[i].kernel, in[i].reduce, &kind[i]));
        uint32_t nk = 0;
        if (is_keyed(kind[i])) {
            nk = in[i].num_keys;
            if (nk < 1 || nk > kMaxKeys)
                return fail(SCL_E_INVALID, "task %u: num_keys %u not in [1, %u]", i, nk, kMaxKeys);
            if (!in[i].counts_out || !in[i].sums_out)
                return fail(SCL_E_INVALID, "task %u: keyed task needs counts_out and sums_out", i);
        }
        fill_task(&P->tasks[i], *p, kind[i], in[i].coef, nk);
        DevTask& t = P->tasks[i];
        t.counts_out = in[i].counts_out;
        t.sums_out = in[i].sums_out;
        t.sums64_out = in[i].sums64_out;
        has_u32 |= mask_of_kind(kind[i]) == M_U32;
        has_f32 |= mask_of_kind(kind[i]) == M_F32;
        has_keyed |= is_keyed(kind[i]);
    }
    const int ntypes = (int)has_u32 + (int)has_f32 + (int)has_keyed;
    P->mask = ntypes > 1 ? M_ALL : has_keyed ? M_KEYED : has_f32 ? M_F32 : M_U32;
    P->shape = shape ? *shape : c->shape_for(P->mask);
    if (!find_entry(P->mask, P->shape))
        return fail(SCL_E_STATE, "no kernel for shape %d x %d", P->shape.block, P->shape.ipt);
    const uint32_t gmax = c->grid_max(P->mask, P->shape);
    const uint32_t chunk = (uint32_t)(P->shape.block * P->shape.ipt * 4);

    // streaming segments: task-relative, length fixed by n and the shape
    P->seg_task.clear();
    P->nseg_stream = 0;
    P->sslots = 0;
    uint64_t W = 0;   // keyed cost
    const uint64_t kov = keyed_piece_overhead(P->mask, P->shape);
    for (uint32_t i = 0; i < nt; ++i) {
        DevTask& t = P->tasks[i];
        if (is_keyed(kind[i])) {
            W += t.n + kov;
            continue;
        }
        t.seg_elems = stream_seg_elems(t.n, chunk);
        t.nseg = stream_nseg(t.n, t.seg_elems);
        t.slot0 = P->sslots;
        t.seg_base = P->nseg_stream;
        P->sslots += t.nseg;
        P->nseg_stream += t.nseg;
        P->seg_task.insert(P->seg_task.end(), t.nseg, i);
    }

    // keyed pieces: an even share of the keyed cost per CTA, cut at 64-pair
    // boundaries, in CTA order
    uint32_t Gk = 0;
    if (has_keyed) {
        uint64_t g = (W + kKeyedMinPiece - 1) / kKeyedMinPiece;
        Gk = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(g, gmax));
        // In a mixed batch only a share of the CTAs take keyed pieces, in
        // proportion to the keyed work's cost, and the others stream from the
        // start: keyed pieces are bound by shared-memory atomics and streaming
        // segments by DRAM, so the two overlap on every SM instead of running
        // one after the other.  (A keyed pair costs about 3.2x a streamed
        // element: 8 bytes at ~0.6 of the HBM rate against 4 bytes at ~0.96.)
        if (P->nseg_stream > 0) {
            uint64_t ws = 0;
            for (uint32_t i = 0; i < nt; ++i)
                if (!is_keyed(kind[i])) ws += P->tasks[i].n;
            const double wk = 3.2 * (double)W, share = wk / (wk + (double)ws);
            const uint64_t gs = (uint64_t)std::ceil(share * gmax);
            Gk = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(Gk, gs));
        }
    }
    uint32_t grid = std::max<uint32_t>(Gk, std::min<uint32_t>(gmax, P->nseg_stream));
    P->grid = std::max<uint32_t>(grid, 1);
    P->kp_first.assign(P->grid + 1, 0);
    P->kpieces.clear();
    P->fold_tasks.clear();
    P->kslots = 0;
    if (has_keyed) {
        std::vector<std::pair<uint32_t, uint64_t>> keyed;
        for (uint32_t i = 0; i < nt; ++i)
            if (is_keyed(kind[i])) keyed.emplace_back(i, P->tasks[i].n);
        std::vector<KeyedPlanPiece> pieces;
        plan_keyed_pieces(keyed, Gk, &pieces, kov);
        for (size_t k = 0; k < pieces.size();) {
            const uint32_t i = pieces[k].task;
            size_t e = k;
            while (e < pieces.size() && pieces[e].task == i) {
                P->kpieces.push_back(KPiece{pieces[e].e0, pieces[e].e1, i, pieces[e].slot});
                P->kp_first[pieces[e].cta + 1]++;
                ++e;
            }
            DevTask& t = P->tasks[i];
            t.nseg = (uint32_t)(e - k);
            t.slot0 = P->kslots;
            if (t.nseg > 1) {
                P->kslots += t.nseg;
                if (t.nseg > kFoldInKernelMaxPieces) P->fold_tasks.push_back(i);
            }
            k = e;
        }
        // pieces come in non-decreasing CTA order: counts -> first piece per CTA
        for (uint32_t g = 0; g < P->grid; ++g) P->kp_first[g + 1] += P->kp_first[g];
    }
    P->fold_gridx = P->fold_tasks.empty() ? 0 : (kMaxKeys + kFoldBlock - 1) / kFoldBlock;
    return SCL_OK;
}

template <typename T>
static T* carve(char* base, size_t* off, size_t count) {
    T* p = reinterpret_cast<T*>(base + *off);
    *off = align_up(*off + count * sizeof(T));
    return p;
}

int build_image(Ctx* c, Plan& p, PlanImage* img, std::vector<char>* host, KernelArgs* args,
                const ExternalScratch* ext) {
    const size_t nt = p.tasks.size();
    if (ext && nt > ext->task_cap)
        return fail(SCL_E_INVALID, "batch of %zu tasks exceeds the scratch capacity %zu", nt,
                    ext->task_cap);
    const size_t own = ext ? 0 : nt;   // results / counters carried in the block
    // sizes (offsets relative to the block)
    size_t off = 0;
    char* nil = nullptr;
    auto o_tasks = off; carve<DevTask>(nil, &off, nt);
    auto o_seg = off; carve<uint32_t>(nil, &off, p.seg_task.size());
    auto o_kpf = off; carve<uint32_t>(nil, &off, p.kp_first.size());
    auto o_kp = off; carve<KPiece>(nil, &off, p.kpieces.size());
    auto o_fold = off; carve<uint32_t>(nil, &off, p.fold_tasks.size());
    const size_t plan_bytes = off;
    auto o_res = off; carve<scl_result>(nil, &off, own);
    const size_t zero_off = off;
    auto o_hdr = off; carve<uint32_t>(nil, &off, ext ? 0 : H_WORDS);
    auto o_tk = off; carve<uint32_t>(nil, &off, own);
    auto o_fl = off; carve<uint32_t>(nil, &off, own);
    const size_t zero_bytes = off - zero_off;
    auto o_sp = off; carve<StreamPartial>(nil, &off, p.sslots);
    auto o_fp = off; carve<StreamPartial>(nil, &off, p.fold_tasks.size() * (kMaxKeys / kFoldBlock));
    auto o_kt = off; carve<uint32_t>(nil, &off, (size_t)p.kslots * kKeyedTableWords);
    const size_t bytes = off;

    char* b = (char*)c->arena.alloc(bytes);
    if (!b) return fail(SCL_E_NOMEM, "arena: no block of %zu bytes for the batch", bytes);
    img->block = b;
    img->bytes = bytes;
    img->tasks = (DevTask*)(b + o_tasks);
    img->seg_task = (uint32_t*)(b + o_seg);
    img->kp_first = (uint32_t*)(b + o_kpf);
    img->kpieces = (KPiece*)(b + o_kp);
    img->fold_tasks = (uint32_t*)(b + o_fold);
    img->results = ext ? ext->results : (scl_result*)(b + o_res);
    img->hdr = ext ? ext->hdr : (uint32_t*)(b + o_hdr);
    img->tickets = ext ? ext->tickets : (uint32_t*)(b + o_tk);
    img->flags = ext ? ext->flags : (uint32_t*)(b + o_fl);
    img->spart = (StreamPartial*)(b + o_sp);
    img->fpart = (StreamPartial*)(b + o_fp);
    img->kpart = (uint32_t*)(b + o_kt);
    img->plan_bytes = plan_bytes;
    img->zero_off = zero_off;
    img->zero_bytes = zero_bytes;

    for (size_t i = 0; i < nt; ++i) p.tasks[i].result = img->results + i;
    host->assign(plan_bytes, 0);
    char* h = host->data();
    if (nt) memcpy(h + o_tasks, p.tasks.data(), nt * sizeof(DevTask));
    if (!p.seg_task.empty()) memcpy(h + o_seg, p.seg_task.data(), p.seg_task.size() * 4);
    if (!p.kp_first.empty()) memcpy(h + o_kpf, p.kp_first.data(), p.kp_first.size() * 4);
    if (!p.kpieces.empty()) memcpy(h + o_kp, p.kpieces.data(), p.kpieces.size() * sizeof(KPiece));
    if (!p.fold_tasks.empty()) memcpy(h + o_fold, p.fold_tasks.data(), p.fold_tasks.size() * 4);

    memset(args, 0, sizeof *args);
    args->tasks = img->tasks;
    args->seg_task = img->seg_task;
    args->kp_first = img->kp_first;
    args->kpieces = img->kpieces;
    args->fold_tasks = img->fold_tasks;
    args->spart = img->spart;
    args->kpart = img->kpart;
    args->fpart = img->fpart;
    args->tickets = img->tickets;
    args->task_flags = img->flags;
    args->hdr = img->hdr;
    args->nseg_stream = p.nseg_stream;
    args->nfold = (uint32_t)p.fold_tasks.size();
    args->err_out = ext ? ext->err_out : nullptr;
    return SCL_OK;
}

int launch_plan(Ctx* c, const Plan& p, const KernelArgs& args, cudaStream_t st) {
    (void)c;
    if (p.tasks.empty()) return SCL_OK;
    const KernelEntry* e = find_entry(p.mask, p.shape);
    if (!e) return fail(SCL_E_STATE, "no kernel for the plan's shape");
    SCL_TRY(launch_entry(e, p.grid, args, st));
    if (!p.fold_tasks.empty()) {   // keyed tasks of many pieces; the others fold in the kernel
        void* params[] = {const_cast<KernelArgs*>(&args)};
        SCL_CUDA(cudaLaunchKernel(fold_kernel_fn(), dim3(p.fold_gridx, (uint32_t)p.fold_tasks.size()),
                                  dim3(kFoldBlock), params, 0, st));
        count_launches(1);
    }
    return SCL_OK;
}

// ------------------------------------------------------------ tuning cache

static const char* kMaskNames[M_NUM] = {"u32", "f32", "keyed", "all"};

int load_tuning(Ctx* c, const char* path) {
    std::ifstream f(path);
    if (!f) return SCL_OK;   // no cache yet
    std::string line;
    while (std::getline(f, line)) {
        std::istringstream is(line);
        std::string name;
        int sms = 0, b = 0, ipt = 0, cps = 0, path = 0, stages = 0;
        if (!(is >> name >> sms >> b >> ipt >> cps >> path >> stages)) continue;
        if (sms != c->sms) continue;
        for (int m = 0; m < M_NUM; ++m)
            if (name == kMaskNames[m] && find_entry(m, b, ipt, path, stages))
                c->shape[m] = Shape{b, ipt, cps, path, stages};
    }
    return SCL_OK;
}

int save_tuning(Ctx* c, const char* path) {
    std::ofstream f(path);
    if (!f) return fail(SCL_E_INVALID, "cannot write tune cache %s", path);
    f << "# mask sms block items_per_thread ctas_per_sm path stages\n";
    for (int m = 0; m < M_NUM; ++m)
        f << kMaskNames[m] << " " << c->sms << " " << c->shape[m].block << " " << c->shape[m].ipt
          << " " << c->shape[m].ctas_per_sm << " " << c->shape[m].path << " "
          << c->shape[m].stages << "\n";
    return SCL_OK;
}

}  // namespace scl
