// server.cu -- continuous-batching server over the persistent batch launch.
#include <string.h>

#include <algorithm>

#include "server.h"

namespace scl {

constexpr size_t kPlanStaging = 4u << 20;   // pinned plan staging per slot

uint64_t task_working_set(Ctx* c, const scl_task& t, const Partition& p, bool load) {
    uint64_t ws = 4096;   // plan entry, result, header share
    if (p.dtype == SCL_KV_I32_F32) {
        const uint64_t pieces = std::min<uint64_t>(c->sms * 8ull, p.n / kKeyedMinPiece + 1);
        ws += (uint64_t)kMaxKeys * 16 + pieces * kKeyedTableWords * 4;
    } else {
        ws += 32ull * (p.n / 4096 + 1);
    }
    if (load) ws += align_up(p.n * 4) * (p.dtype == SCL_KV_I32_F32 ? 2 : 1);
    (void)t;
    return ws;
}

Server::~Server() { stop(); }

int Server::start(Ctx* c, const scl_server_config* in) {
    ctx = c;
    if (in) cfg = *in;
    if (cfg.inflight_batches <= 0) cfg.inflight_batches = 4;
    if (cfg.inflight_batches > 16) return fail(SCL_E_INVALID, "inflight_batches must be 1..16");
    if (cfg.max_batch_tasks == 0) cfg.max_batch_tasks = 4096;
    if (cfg.max_batch_tasks > 65536) return fail(SCL_E_INVALID, "max_batch_tasks must be <= 65536");
    budget = cfg.hbm_budget_bytes ? cfg.hbm_budget_bytes
                                  : (c->hbm_budget ? c->hbm_budget : c->arena_bytes);
    SCL_CUDA(cudaSetDevice(c->device));
    SCL_CUDA(cudaStreamCreateWithFlags(&copy_stream, cudaStreamNonBlocking));
    slots.resize(cfg.inflight_batches);
    const size_t cap = cfg.max_batch_tasks;
    for (auto& s : slots) {
        SCL_CUDA(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
        SCL_CUDA(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
        SCL_CUDA(cudaHostAlloc((void**)&s.h_res, (cap + 1) * sizeof(scl_result),
                               cudaHostAllocMapped));
        // Pinned staging for plan uploads, allocated here and never resized
        // while serving: page-locking memory can take milliseconds (and freeing
        // pinned memory synchronises the device), which would stall the batcher
        // in the middle of a trace.
        s.h_plan_cap = kPlanStaging;
        SCL_CUDA(cudaHostAlloc((void**)&s.h_plan, s.h_plan_cap, cudaHostAllocDefault));
        SCL_CUDA(cudaHostGetDevicePointer((void**)&s.d_res, s.h_res, 0));
        const size_t zb = align_up(H_WORDS * 4) + 2 * align_up(cap * 4);
        s.zero = c->arena.alloc(zb);
        if (!s.zero) return fail(SCL_E_NOMEM, "arena: no room for the server's scratch");
        SCL_CUDA(cudaMemset(s.zero, 0, zb));
        char* z = static_cast<char*>(s.zero);
        s.ext.hdr = reinterpret_cast<uint32_t*>(z);
        s.ext.tickets = reinterpret_cast<uint32_t*>(z + align_up(H_WORDS * 4));
        s.ext.flags = reinterpret_cast<uint32_t*>(z + align_up(H_WORDS * 4) + align_up(cap * 4));
        s.ext.task_cap = cap;
        s.ext.results = s.d_res;
        s.ext.err_out = reinterpret_cast<uint32_t*>(s.d_res + cap);
    }
    SCL_CUDA(cudaDeviceSynchronize());
    memset(&stats, 0, sizeof stats);
    stats.budget_bytes = budget;
    done.reserve(1u << 17);   // results wait here until collected: no rehash mid-trace
    stopping = false;
    batcher_exited = false;
    batcher = std::thread([this] { batcher_loop(); });
    completer = std::thread([this] { completer_loop(); });
    return SCL_OK;
}

void Server::stop() {
    {
        std::lock_guard<std::mutex> g(mu);
        if (!batcher.joinable() && !completer.joinable()) return;
        stopping = true;
    }
    cv_work.notify_all();
    if (batcher.joinable()) batcher.join();
    if (completer.joinable()) completer.join();
    cudaSetDevice(ctx->device);
    for (auto& s : slots) {
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.done) cudaEventDestroy(s.done);
        if (s.h_plan) cudaFreeHost(s.h_plan);
        if (s.h_res) cudaFreeHost(s.h_res);
        if (s.zero) ctx->arena.release(s.zero);
        s = Slot();
    }
    if (copy_stream) cudaStreamDestroy(copy_stream);
    copy_stream = nullptr;
    // tasks never launched: free their staged inputs
    for (auto* q : {&waiting, &admitted})
        for (auto& t : *q) {
            if (t.ready) cudaEventDestroy(t.ready);
            if (t.block) ctx->arena.release(t.block);
        }
    waiting.clear();
    admitted.clear();
}

int Server::stage_load(SrvTask& t) {
    const size_t bytes = align_up(t.n * 4);
    const bool kv = t.dtype == SCL_KV_I32_F32;
    void* b = ctx->arena.alloc(bytes * (kv ? 2 : 1));
    if (!b) return fail(SCL_E_NOMEM, "arena full while staging a task's input");
    t.block = b;
    if (t.n) {
        SCL_CUDA(cudaMemcpyAsync(b, t.host0, t.n * 4, cudaMemcpyHostToDevice, copy_stream));
        if (kv)
            SCL_CUDA(cudaMemcpyAsync((char*)b + bytes, t.host1, t.n * 4, cudaMemcpyHostToDevice,
                                     copy_stream));
    }
    SCL_CUDA(cudaEventCreateWithFlags(&t.ready, cudaEventDisableTiming));
    SCL_CUDA(cudaEventRecord(t.ready, copy_stream));
    std::lock_guard<std::recursive_mutex> g(ctx->mu);
    t.task.part = ctx->next_part++;
    ctx->parts[t.task.part] = Partition{t.dtype, t.n, b, kv ? (char*)b + bytes : nullptr, nullptr};
    return SCL_OK;
}

// Move waiting tasks to the GPU queue while they fit the budget (FIFO: the
// head blocks the rest, so a large task is not starved by small ones).
void Server::admit_locked() {
    while (!waiting.empty()) {
        SrvTask& t = waiting.front();
        const uint64_t resident = ctx->resident_bytes.load();
        if (resident + inflight_bytes + t.ws_bytes > budget) {
            if (inflight_bytes > 0) break;   // wait for running work to return budget
            // nothing in flight and it still does not fit (resident data grew
            // since it was accepted): it never will
            Done d;
            memset(&d.r, 0, sizeof d.r);
            d.r.status = SCL_E_BUDGET;
            d.t_submit = t.t_submit;
            d.t_done = now_ns();
            done[t.ticket] = d;
            stats.rejected++;
            waiting.pop_front();
            cv_done.notify_all();
            continue;
        }
        inflight_bytes += t.ws_bytes;
        stats.peak_bytes_in_use = std::max(stats.peak_bytes_in_use, resident + inflight_bytes);
        if (t.load && stage_load(t) != SCL_OK) {
            inflight_bytes -= t.ws_bytes;
            Done d;
            memset(&d.r, 0, sizeof d.r);
            d.r.status = SCL_E_NOMEM;
            d.t_submit = t.t_submit;
            d.t_done = now_ns();
            done[t.ticket] = d;
            stats.completed++;
            waiting.pop_front();
            cv_done.notify_all();
            continue;
        }
        admitted.push_back(std::move(t));
        waiting.pop_front();
    }
    admitted_n.store(admitted.size(), std::memory_order_release);
}

int Server::submit(SrvTask&& t, uint64_t* ticket) {
    std::lock_guard<std::mutex> g(mu);
    if (stopping) return fail(SCL_E_STATE, "server is stopping");
    if (t.ws_bytes + ctx->resident_bytes.load() > budget) {
        stats.rejected++;
        return fail(SCL_E_BUDGET, "task needs %llu bytes; budget %llu, resident %llu",
                    (unsigned long long)t.ws_bytes, (unsigned long long)budget,
                    (unsigned long long)ctx->resident_bytes.load());
    }
    t.ticket = next_ticket++;
    *ticket = t.ticket;
    stats.submitted++;
    const uint64_t tk = t.ticket;
    waiting.push_back(std::move(t));
    admit_locked();
    if (!waiting.empty() && waiting.back().ticket == tk) stats.admission_waits++;
    cv_work.notify_one();
    return SCL_OK;
}

void Server::batcher_loop() {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        // Spin up to 1 ms for new work before sleeping: a condition-variable
        // wake-up costs more than most batches take on the GPU (at 2,000
        // tasks/s a 100 us spin left p50 10 us higher than at 10,000).
        if (admitted.empty() && !stopping) {
            lk.unlock();
            const int64_t t0 = now_ns();
            while (admitted_n.load(std::memory_order_acquire) == 0 && now_ns() - t0 < 1000000) {
            }
            lk.lock();
        }
        Slot* free_slot = nullptr;
        cv_work.wait(lk, [&] {
            free_slot = nullptr;
            for (auto& s : slots)
                if (!s.busy) {
                    free_slot = &s;
                    break;
                }
            return (stopping && admitted.empty() && waiting.empty()) ||
                   (!admitted.empty() && free_slot);
        });
        if (admitted.empty()) break;   // stopping, nothing left to launch
        Slot& s = *free_slot;
        // Take, in admission order, the tasks whose input is on the device: a
        // task that brings new data joins a launch once its copy has landed,
        // so a large copy does not hold back the tasks admitted after it.
        // Only a bounded prefix is looked at, so a long backlog costs nothing.
        s.tasks.clear();
        std::vector<SrvTask> pending;
        size_t scanned = 0;
        while (!admitted.empty() && s.tasks.size() < cfg.max_batch_tasks &&
               scanned < (size_t)cfg.max_batch_tasks + 256) {
            SrvTask& t = admitted.front();
            if (!t.ready || cudaEventQuery(t.ready) != cudaErrorNotReady)
                s.tasks.push_back(std::move(t));
            else
                pending.push_back(std::move(t));
            admitted.pop_front();
            ++scanned;
        }
        for (auto it = pending.rbegin(); it != pending.rend(); ++it)
            admitted.push_front(std::move(*it));
        admitted_n.store(admitted.size(), std::memory_order_release);
        if (s.tasks.empty()) {   // only copies in flight: look again shortly
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(5));
            lk.lock();
            continue;
        }
        s.busy = true;
        lk.unlock();
        const int st = launch_slot(s);
        lk.lock();
        if (st == SCL_OK) {
            stats.batches++;
            stats.max_batch = std::max<uint64_t>(stats.max_batch, s.tasks.size());
            s.launched = true;   // the completer may now poll its event
        } else {
            lk.unlock();
            finish_slot(s, st);
            lk.lock();
        }
    }
    batcher_exited = true;
}

int Server::launch_slot(Slot& s) {
    const uint32_t n = (uint32_t)s.tasks.size();
    std::vector<scl_task> tv(n);
    for (uint32_t i = 0; i < n; ++i) tv[i] = s.tasks[i].task;
    std::vector<char> host;
    {
        std::lock_guard<std::recursive_mutex> g(ctx->mu);
        s.plan = Plan();
        s.img = PlanImage();
        SCL_TRY(plan_tasks(ctx, tv.data(), n, &s.plan));
        SCL_TRY(build_image(ctx, s.plan, &s.img, &host, &s.args, &s.ext));
    }
    // one upload; counters are already zero, results come back by themselves.
    // A plan larger than the pinned staging goes up from pageable memory
    // (the call returns once the bytes are staged; no device-wide sync).
    if (host.size() <= s.h_plan_cap) {
        memcpy(s.h_plan, host.data(), host.size());
        SCL_CUDA(cudaMemcpyAsync(s.img.block, s.h_plan, s.img.plan_bytes,
                                 cudaMemcpyHostToDevice, s.stream));
    } else {
        SCL_CUDA(cudaMemcpyAsync(s.img.block, host.data(), s.img.plan_bytes,
                                 cudaMemcpyHostToDevice, s.stream));
        SCL_CUDA(cudaStreamSynchronize(s.stream));   // `host` is freed on return
    }
    for (auto& t : s.tasks)
        if (t.ready) SCL_CUDA(cudaStreamWaitEvent(s.stream, t.ready, 0));
    s.t_launch = now_ns();
    SCL_TRY(launch_plan(ctx, s.plan, s.args, s.stream));
    SCL_CUDA(cudaEventRecord(s.done, s.stream));
    {
        std::lock_guard<std::mutex> g(mu);
        stats.kernel_launches += 1 + (s.plan.fold_tasks.empty() ? 0 : 1);
    }
    return SCL_OK;
}

void Server::finish_slot(Slot& s, int status) {
    const int64_t t = now_ns();
    const uint32_t n = (uint32_t)s.tasks.size();
    uint32_t err = 0;
    if (status == SCL_OK) memcpy(&err, s.h_res + s.ext.task_cap, 4);
    if (err || status != SCL_OK) {
        // a failed launch may have left counters set: clear them before reuse
        const size_t zb = align_up(H_WORDS * 4) + 2 * align_up(s.ext.task_cap * 4);
        cudaMemset(s.zero, 0, zb);
        cudaDeviceSynchronize();
    }
    std::vector<Done> ds(n);
    for (uint32_t i = 0; i < n; ++i) {
        Done& d = ds[i];
        if (status == SCL_OK) {
            d.r = s.h_res[i];
            if (err) d.r.status = (err & 4u) ? SCL_E_TIMEOUT : SCL_E_STATE;
        } else {
            memset(&d.r, 0, sizeof d.r);
            d.r.status = status;
        }
        d.t_submit = s.tasks[i].t_submit;
        d.t_done = t;
    }
    {
        std::lock_guard<std::recursive_mutex> g(ctx->mu);
        for (auto& tk : s.tasks)
            if (tk.load) {
                ctx->parts.erase(tk.task.part);
                ctx->arena.release(tk.block);
                if (tk.ready) cudaEventDestroy(tk.ready);
            }
        if (s.img.block) ctx->arena.release(s.img.block);
        s.img = PlanImage();
    }
    {
        std::lock_guard<std::mutex> g(mu);
        for (uint32_t i = 0; i < n; ++i) {
            done[s.tasks[i].ticket] = ds[i];
            inflight_bytes -= s.tasks[i].ws_bytes;
        }
        stats.completed += n;
        s.tasks.clear();
        s.launched = false;
        s.busy = false;
        admit_locked();
    }
    cv_work.notify_one();
    cv_done.notify_all();
}

void Server::completer_loop() {
    cudaSetDevice(ctx->device);
    for (;;) {
        bool any_busy = false, progressed = false;
        for (auto& s : slots) {
            bool launched;
            {
                std::lock_guard<std::mutex> g(mu);
                launched = s.launched;
                any_busy |= s.busy;
            }
            if (!launched) continue;
            const cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaErrorNotReady) continue;
            finish_slot(s, q == cudaSuccess ? SCL_OK : SCL_E_CUDA);
            progressed = true;
        }
        if (!any_busy) {
            std::unique_lock<std::mutex> lk(mu);
            bool idle = true;
            for (auto& s : slots) idle &= !s.busy;
            if (stopping && batcher_exited && idle && admitted.empty() && waiting.empty()) break;
        }
        if (!progressed) std::this_thread::yield();
    }
}

}  // namespace scl

using namespace scl;

namespace {

int srv_of(scl_ctx* ctx, Server** s) {
    if (!ctx) return fail(SCL_E_INVALID, "null context");
    if (!ctx->server) return fail(SCL_E_STATE, "server not started");
    *s = ctx->server.get();
    return SCL_OK;
}

}  // namespace

extern "C" {

int scl_server_start(scl_ctx* ctx, const scl_server_config* cfg) {
    if (!ctx) return fail(SCL_E_INVALID, "null context");
    clear_error();
    std::lock_guard<std::recursive_mutex> g(ctx->mu);
    if (ctx->server) return fail(SCL_E_STATE, "server already running");
    std::unique_ptr<Server> s(new Server());
    const int st = s->start(ctx, cfg);
    if (st != SCL_OK) return st;
    ctx->server = std::move(s);
    return SCL_OK;
}

static int submit_common(scl_ctx* ctx, SrvTask&& t, const Partition& p, uint64_t* ticket) {
    Server* s = nullptr;
    SCL_TRY(srv_of(ctx, &s));
    uint32_t kind;
    SCL_TRY(resolve_kind(p.dtype, t.task.kernel, t.task.reduce, &kind));
    if (is_keyed(kind)) {
        if (t.task.num_keys < 1 || t.task.num_keys > kMaxKeys)
            return fail(SCL_E_INVALID, "num_keys %u not in [1, %u]", t.task.num_keys, kMaxKeys);
        if (!t.task.counts_out || !t.task.sums_out)
            return fail(SCL_E_INVALID, "keyed task needs counts_out and sums_out");
    }
    t.ws_bytes = task_working_set(ctx, t.task, p, t.load);
    if (!t.t_submit) t.t_submit = now_ns();
    return s->submit(std::move(t), ticket);
}

int scl_server_submit(scl_ctx* ctx, const scl_task* task, uint64_t* ticket) {
    if (!ctx || !task || !ticket) return fail(SCL_E_INVALID, "null argument");
    clear_error();
    Partition p;
    {
        std::lock_guard<std::recursive_mutex> g(ctx->mu);
        const Partition* q = ctx->part(task->part);
        if (!q) return fail(SCL_E_INVALID, "unknown partition handle");
        p = *q;
    }
    SrvTask t;
    t.task = *task;
    return submit_common(ctx, std::move(t), p, ticket);
}

int scl_server_submit_load(scl_ctx* ctx, const void* host0, const void* host1, scl_dtype dtype,
                           uint64_t n, const scl_task* task, uint64_t* ticket) {
    if (!ctx || !task || !ticket) return fail(SCL_E_INVALID, "null argument");
    clear_error();
    if ((int)dtype < 0 || dtype > SCL_KV_I32_F32) return fail(SCL_E_INVALID, "bad dtype");
    if (n && (!host0 || (dtype == SCL_KV_I32_F32 && !host1)))
        return fail(SCL_E_INVALID, "null host array");
    SrvTask t;
    t.task = *task;
    t.task.part = 0;
    t.load = true;
    t.host0 = host0;
    t.host1 = host1;
    t.dtype = dtype;
    t.n = n;
    Partition p{dtype, n, nullptr, nullptr, nullptr};
    return submit_common(ctx, std::move(t), p, ticket);
}

int scl_server_poll(scl_ctx* ctx, uint64_t ticket, scl_result* out) {
    Server* s = nullptr;
    SCL_TRY(srv_of(ctx, &s));
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->done.find(ticket);
    if (it == s->done.end()) {
        if (ticket == 0 || ticket >= s->next_ticket)
            return fail(SCL_E_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
        return SCL_E_PENDING;
    }
    if (out) *out = it->second.r;
    s->done.erase(it);
    return SCL_OK;
}

int scl_server_wait(scl_ctx* ctx, uint64_t ticket, uint32_t timeout_ms, scl_result* out) {
    Server* s = nullptr;
    SCL_TRY(srv_of(ctx, &s));
    std::unique_lock<std::mutex> lk(s->mu);
    if (ticket == 0 || ticket >= s->next_ticket)
        return fail(SCL_E_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                        [&] { return s->done.count(ticket) > 0; });
    if (!ok) return fail(SCL_E_TIMEOUT, "ticket %llu not done after %u ms",
                         (unsigned long long)ticket, timeout_ms);
    auto it = s->done.find(ticket);
    if (out) *out = it->second.r;
    s->done.erase(it);
    return SCL_OK;
}

int scl_server_get_stats(scl_ctx* ctx, scl_server_stats* out) {
    Server* s = nullptr;
    SCL_TRY(srv_of(ctx, &s));
    if (!out) return fail(SCL_E_INVALID, "null output");
    std::lock_guard<std::mutex> g(s->mu);
    *out = s->stats;
    out->resident_bytes = ctx->resident_bytes.load();
    out->bytes_in_use = ctx->resident_bytes.load() + s->inflight_bytes;
    return SCL_OK;
}

int scl_server_stop(scl_ctx* ctx) {
    if (!ctx) return SCL_OK;
    std::unique_ptr<Server> s;
    {
        std::lock_guard<std::recursive_mutex> g(ctx->mu);
        s = std::move(ctx->server);
    }
    if (s) s->stop();
    return SCL_OK;
}

// Open-loop replay: submits task i at its scheduled arrival on this thread
// while a collector thread takes each result as soon as it is done, so the
// map of finished results stays small however long the trace is.
static int replay(scl_ctx* ctx, const scl_task* tasks, const scl_task_data* data,
                  const double* arrival_s, uint32_t n, int64_t* latency_ns, scl_result* results) {
    Server* s = nullptr;
    SCL_TRY(srv_of(ctx, &s));
    if (n && (!tasks || !arrival_s)) return fail(SCL_E_INVALID, "null argument");
    std::vector<uint64_t> tickets(n, 0);
    std::vector<int64_t> sched(n);
    std::vector<int> sub_status(n, SCL_OK);
    std::atomic<uint32_t> published{0};
    std::thread collector([&] {
        for (uint32_t i = 0; i < n; ++i) {
            while (published.load(std::memory_order_acquire) <= i) std::this_thread::yield();
            if (sub_status[i] != SCL_OK) continue;
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_done.wait(lk, [&] { return s->done.count(tickets[i]) > 0; });
            auto it = s->done.find(tickets[i]);
            if (latency_ns) latency_ns[i] = it->second.t_done - sched[i];
            if (results) results[i] = it->second.r;
            s->done.erase(it);
        }
    });
    const int64_t t0 = now_ns() + 1000000;   // start 1 ms from now
    for (uint32_t i = 0; i < n; ++i) {
        sched[i] = t0 + (int64_t)(arrival_s[i] * 1e9);
        int64_t now = now_ns();
        while (now < sched[i]) {
            if (sched[i] - now > 200000) std::this_thread::sleep_for(std::chrono::microseconds(100));
            else std::this_thread::yield();
            now = now_ns();
        }
        SrvTask t;
        t.task = tasks[i];
        t.t_submit = sched[i];   // open loop: latency counts from the scheduled arrival
        Partition p;
        const scl_task_data* d = data ? &data[i] : nullptr;
        if (d && d->host0) {
            const scl_dtype dt = (scl_dtype)d->dtype;
            if ((int)dt < 0 || dt > SCL_KV_I32_F32 || (dt == SCL_KV_I32_F32 && d->n && !d->host1)) {
                sub_status[i] = fail(SCL_E_INVALID, "task %u: bad data description", i);
            } else {
                t.task.part = 0;
                t.load = true;
                t.host0 = d->host0;
                t.host1 = d->host1;
                t.dtype = dt;
                t.n = d->n;
                p = Partition{dt, d->n, nullptr, nullptr, nullptr};
            }
        } else {
            std::lock_guard<std::recursive_mutex> g(ctx->mu);
            const Partition* q = ctx->part(tasks[i].part);
            if (!q) sub_status[i] = fail(SCL_E_INVALID, "task %u: unknown partition", i);
            else p = *q;
        }
        if (sub_status[i] == SCL_OK) sub_status[i] = submit_common(ctx, std::move(t), p, &tickets[i]);
        published.store(i + 1, std::memory_order_release);
    }
    collector.join();
    int worst = SCL_OK;
    for (uint32_t i = 0; i < n; ++i) {
        if (sub_status[i] == SCL_OK) continue;
        if (latency_ns) latency_ns[i] = -1;
        if (results) {
            memset(&results[i], 0, sizeof results[i]);
            results[i].status = sub_status[i];
        }
        if (worst == SCL_OK) worst = sub_status[i];
    }
    if (worst != SCL_OK) return fail(worst, "some tasks were not submitted");
    return SCL_OK;
}

int scl_server_replay(scl_ctx* ctx, const scl_task* tasks, const double* arrival_s, uint32_t n,
                      int64_t* latency_ns, scl_result* results) {
    return replay(ctx, tasks, nullptr, arrival_s, n, latency_ns, results);
}

int scl_server_replay_load(scl_ctx* ctx, const scl_task* tasks, const scl_task_data* data,
                           const double* arrival_s, uint32_t n, int64_t* latency_ns,
                           scl_result* results) {
    return replay(ctx, tasks, data, arrival_s, n, latency_ns, results);
}

}  // extern "C"
