// devserver.cu -- the device-polling server: host driver of k_doorbell.
#include <string.h>

#include <algorithm>

#include "devserver.h"

static_assert(sizeof(scl_devserver_config) == 48, "scl_devserver_config layout");
static_assert(sizeof(scl_devserver_stats) == 112, "scl_devserver_stats layout");

namespace scl {

static_assert(sizeof(DbState) == 384 && sizeof(DbHost) == 384, "doorbell header layout");

const void* doorbell_kernel_256(int ipt);
const void* doorbell_kernel_512(int ipt);

const void* doorbell_kernel_fn(int block, int ipt) {
    if (block == 256) return doorbell_kernel_256(ipt);
    if (block == 512) return doorbell_kernel_512(ipt);
    return nullptr;
}

template <class T>
static inline void store_release(T* p, T v) {
    __atomic_store_n(p, v, __ATOMIC_RELEASE);
}
template <class T>
static inline T load_acquire(const T* p) {
    return __atomic_load_n(p, __ATOMIC_ACQUIRE);
}

// ------------------------------------------------------------ DevServer

DevServer::~DevServer() { stop(); }

int DevServer::start(Ctx* c, const scl_devserver_config* in) {
    ctx = c;
    if (in) cfg = *in;
    if (!cfg.job_ring) cfg.job_ring = 16384;
    if (!cfg.unit_ring) cfg.unit_ring = 1u << 20;
    if (!cfg.keyed_slots) cfg.keyed_slots = 256;
    if (!cfg.idle_stop_ns) cfg.idle_stop_ns = 2000000;
    if (!cfg.wait_limit_ns) cfg.wait_limit_ns = 1000000000;
    if (cfg.job_ring > (1u << 20) || cfg.unit_ring > (1u << 26) || cfg.keyed_slots > 65536)
        return fail(SCL_E_INVALID, "devserver rings: job_ring <= 2^20, unit_ring <= 2^26, "
                                   "keyed_slots <= 65536");
    if (cfg.wait_limit_ns > 60000000000ull)
        return fail(SCL_E_INVALID, "wait_limit_ns must be at most 60 s");
    const Shape sh = c->shape_for(M_F32);
    block = sh.block;
    ipt = sh.ipt;
    fn = doorbell_kernel_fn(block, ipt);
    if (!fn) return fail(SCL_E_UNSUPPORTED, "no device-polling kernel for shape %d x %d", block, ipt);
    SCL_CUDA(cudaSetDevice(c->device));
    int occ = 0;
    SCL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, block, kKeyedSmemBytes));
    if (occ < 1) return fail(SCL_E_STATE, "the device-polling kernel does not fit an SM");
    const int per = cfg.ctas_per_sm > 0 ? std::min<int>(cfg.ctas_per_sm, occ) : occ;
    grid = (uint32_t)(c->sms * per);
    SCL_CUDA(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));

    // pinned host block: header | jobs | results | done
    const size_t o_jobs = sizeof(DbHost);
    const size_t o_res = align_up(o_jobs + (size_t)cfg.job_ring * sizeof(DbJob), 128);
    const size_t o_done = align_up(o_res + (size_t)cfg.job_ring * sizeof(scl_result), 128);
    const size_t hbytes = o_done + (size_t)cfg.job_ring * 4;
    SCL_CUDA(cudaHostAlloc((void**)&hblock, hbytes, cudaHostAllocMapped));
    memset(hblock, 0, hbytes);
    char* dh = nullptr;
    SCL_CUDA(cudaHostGetDevicePointer((void**)&dh, hblock, 0));
    hh = reinterpret_cast<DbHost*>(hblock);
    hjobs = reinterpret_cast<DbJob*>(hblock + o_jobs);
    hres = reinterpret_cast<scl_result*>(hblock + o_res);
    hdone = reinterpret_cast<uint32_t*>(hblock + o_done);
    dres = reinterpret_cast<scl_result*>(dh + o_res);

    // arena block: state | tickets | flags | keyed accumulators | job copies |
    // unit map | partials
    const size_t d_tick = align_up(sizeof(DbState));
    const size_t d_flag = d_tick + align_up((size_t)cfg.job_ring * 4);
    const size_t d_kacc = d_flag + align_up((size_t)cfg.job_ring * 4);
    const size_t d_djobs = d_kacc + align_up((size_t)cfg.keyed_slots * kDbAccWords * 4);
    const size_t d_dunit = d_djobs + align_up((size_t)cfg.job_ring * sizeof(DbJob));
    const size_t d_spart = d_dunit + align_up((size_t)cfg.unit_ring * 4);
    const size_t dbytes = d_spart + (size_t)cfg.unit_ring * sizeof(StreamPartial);
    dblock = c->arena.alloc(dbytes);
    if (!dblock)
        return fail(SCL_E_NOMEM, "arena: no room for the device-polling server (%zu bytes)", dbytes);
    zero_small = sizeof(DbState);
    zero_all = d_djobs;   // the job copies and unit map are written before they are read
    SCL_CUDA(cudaMemsetAsync(dblock, 0, zero_all, stream));
    SCL_CUDA(cudaStreamSynchronize(stream));
    char* db = static_cast<char*>(dblock);
    memset(&args, 0, sizeof args);
    args.ka.spart = reinterpret_cast<StreamPartial*>(db + d_spart);
    args.ka.tickets = reinterpret_cast<uint32_t*>(db + d_tick);
    args.ka.task_flags = reinterpret_cast<uint32_t*>(db + d_flag);
    args.host = reinterpret_cast<DbHost*>(dh);
    args.jobs = reinterpret_cast<const DbJob*>(dh + o_jobs);
    args.done = reinterpret_cast<uint32_t*>(dh + o_done);
    args.state = reinterpret_cast<DbState*>(db);
    args.kacc = reinterpret_cast<uint32_t*>(db + d_kacc);
    args.djobs = reinterpret_cast<DbJob*>(db + d_djobs);
    args.dunit = reinterpret_cast<uint32_t*>(db + d_dunit);
    args.wait_limit_ns = cfg.wait_limit_ns;
    args.max_polls = cfg.wait_limit_ns / 16 + 4096;   // a backstop if the GPU timer stalls
    args.job_ring = cfg.job_ring;
    args.unit_ring = cfg.unit_ring;
    args.spart_cap = cfg.unit_ring;
    args.kacc_slots = cfg.keyed_slots;

    ring.assign(cfg.job_ring, DbInflight{});
    free_kslots.clear();
    for (uint32_t k = cfg.keyed_slots; k-- > 0;) free_kslots.push_back(k);
    spart.init(cfg.unit_ring);
    memset(&stats, 0, sizeof stats);
    done.reserve(1u << 17);   // results wait here until collected: no rehash mid-trace
    stats.grid = grid;
    stats.block = (uint32_t)block;
    stats.items_per_thread = (uint32_t)ipt;
    last_activity = last_progress = now_ns();
    driver = std::thread([this] { driver_loop(); });
    return SCL_OK;
}

int DevServer::submit(const scl_task& task, const Partition& p, int64_t t_submit,
                      uint64_t* ticket) {
    uint32_t kind = 0;
    SCL_TRY(resolve_kind(p.dtype, task.kernel, task.reduce, &kind));
    uint32_t nk = 0;
    if (is_keyed(kind)) {
        nk = task.num_keys;
        if (nk < 1 || nk > kMaxKeys)
            return fail(SCL_E_INVALID, "num_keys %u not in [1, %u]", nk, kMaxKeys);
        if (!task.counts_out || !task.sums_out)
            return fail(SCL_E_INVALID, "keyed task needs counts_out and sums_out");
    }
    DbPending q;
    fill_task(&q.t, p, kind, task.coef, nk);
    q.t.counts_out = task.counts_out;
    q.t.sums_out = task.sums_out;
    q.t.sums64_out = task.sums64_out;
    if (is_keyed(kind)) {
        q.t.nseg = db_keyed_pieces(p.n);
    } else {
        q.t.seg_elems = stream_seg_elems(p.n, (uint32_t)(block * ipt * 4));
        q.t.nseg = stream_nseg(p.n, q.t.seg_elems);
    }
    if (q.t.nseg > cfg.unit_ring)
        return fail(SCL_E_BUDGET, "task has %u work units, the ring holds %u", q.t.nseg,
                    cfg.unit_ring);
    q.t_submit = t_submit ? t_submit : now_ns();
    {
        std::lock_guard<std::mutex> g(mu);
        if (broken) return fail(SCL_E_CUDA, "the device-polling server stopped after an error");
        if (quitting) return fail(SCL_E_STATE, "the device-polling server is stopping");
        q.ticket = next_ticket++;
        *ticket = q.ticket;
        stats.submitted++;
        if (!queue.empty() || !publish_locked(q)) {
            queue.push_back(q);
            stats.ring_waits++;
        } else if (!running) {
            launch_locked();   // on failure the job is failed with SCL_E_CUDA
        }
    }
    cv_work.notify_one();
    return SCL_OK;
}

// Write job `pubs` into its ring slot, then ring the doorbell.
bool DevServer::publish_locked(DbPending& q) {
    const uint32_t nseg = q.t.nseg;
    const bool keyed = is_keyed(q.t.kind);
    if (!inflight_pubs.empty()) {
        // the slot of job pubs - job_ring must be free, and the unit map
        // entries of jobs in flight must not be overwritten
        const auto& oldest = *inflight_pubs.begin();
        if (pubs - oldest.first >= cfg.job_ring) return false;
        if (units + nseg - oldest.second > cfg.unit_ring) return false;
    }
    uint32_t sp = UINT32_MAX, ks = UINT32_MAX;
    if (nseg > 1) {
        if (keyed) {
            if (free_kslots.empty()) return false;
            ks = free_kslots.back();
            free_kslots.pop_back();
        } else if (!spart.alloc(nseg, &sp)) {
            return false;
        }
    }
    const uint32_t j = (uint32_t)(pubs % cfg.job_ring);
    const uint32_t seq = next_seq++;
    if (next_seq == 0) next_seq = 1;

    DbJob job;
    memset(&job, 0, sizeof job);
    job.t = q.t;
    job.t.result = dres + j;
    job.t.slot0 = nseg > 1 ? (keyed ? ks : sp) : 0u;
    job.unit0 = units;
    job.seq = seq;
    job.ring = j;
    hjobs[j] = job;
    hdone[j] = 0;
    DbInflight& f = ring[j];
    f.ticket = q.ticket;
    f.seq = seq;
    f.nseg = nseg;
    f.unit0 = units;
    f.pub = pubs;
    f.spart0 = sp;
    f.kslot = ks;
    f.n = q.t.n;
    f.kind = q.t.kind;
    f.t_submit = q.t_submit;
    inflight_pubs[pubs] = units;
    units += nseg;
    ++pubs;
    store_release(&hh->jobs, (unsigned long long)pubs);   // the doorbell
    pub_gen.fetch_add(1, std::memory_order_release);

    inflight.push_back(j);
    stats.units += nseg;
    stats.max_inflight = std::max<uint64_t>(stats.max_inflight, inflight.size());
    last_activity = now_ns();
    return true;
}

int DevServer::launch_locked() {
    void* params[] = {&args};
    const cudaError_t e =
        cudaLaunchKernel(fn, dim3(grid), dim3(block), params, kKeyedSmemBytes, stream);
    if (e != cudaSuccess) {
        broken = true;
        fail(SCL_E_CUDA, "device-polling kernel launch: %s", cudaGetErrorString(e));
        recover_locked(SCL_E_CUDA);
        return SCL_E_CUDA;
    }
    running = true;
    stats.kernel_launches++;
    count_launches(1);
    last_progress = now_ns();
    return SCL_OK;
}

// Ask the kernel to stop, wait (bounded) until it has ended, zero the state.
int DevServer::end_kernel_locked(bool zero_all_state) {
    if (running) {
        store_release(&hh->stop, 1u);
        const int64_t deadline =
            now_ns() + (int64_t)cfg.wait_limit_ns + 5000000000ll;
        cudaError_t q;
        while ((q = cudaStreamQuery(stream)) == cudaErrorNotReady) {
            if (now_ns() > deadline) {
                broken = true;
                return fail(SCL_E_TIMEOUT, "the device-polling kernel did not end");
            }
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        running = false;
        if (q != cudaSuccess) {
            broken = true;
            return fail(SCL_E_CUDA, "device-polling kernel: %s", cudaGetErrorString(q));
        }
    }
    if (cudaMemsetAsync(dblock, 0, zero_all_state ? zero_all : zero_small, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
        broken = true;
        return fail(SCL_E_CUDA, "device-polling server: state reset failed");
    }
    store_release(&hh->jobs, 0ull);
    store_release(&hh->stop, 0u);
    store_release(&hh->err, 0u);
    units = 0;
    pubs = 0;
    return SCL_OK;
}

void DevServer::complete_locked(uint32_t j, const scl_result& r, int64_t now) {
    DbInflight& f = ring[j];
    Done d;
    d.r = r;
    d.t_submit = f.t_submit;
    d.t_done = now;
    done[f.ticket] = d;
    if (f.spart0 != UINT32_MAX) spart.release(f.spart0, f.nseg);
    if (f.kslot != UINT32_MAX) free_kslots.push_back(f.kslot);
    inflight_pubs.erase(f.pub);
    f = DbInflight{};
    last_activity = now;
    done_gen.fetch_add(1, std::memory_order_release);
}

bool DevServer::wait_done(uint64_t ticket, int64_t spin_ns, int64_t timeout_ns, Done* out) {
    const int64_t t0 = now_ns();
    std::unique_lock<std::mutex> lk(mu);
    uint64_t seen = done_gen.load(std::memory_order_acquire);
    for (;;) {
        auto it = done.find(ticket);
        if (it != done.end()) {
            *out = it->second;
            done.erase(it);
            return true;
        }
        const int64_t now = now_ns();
        if (now - t0 >= timeout_ns) return false;
        if (now - t0 < spin_ns) {
            // spin without the lock until some job completes
            lk.unlock();
            while (done_gen.load(std::memory_order_acquire) == seen && now_ns() - t0 < spin_ns) {
            }
            lk.lock();
            seen = done_gen.load(std::memory_order_acquire);
            continue;
        }
        cv_done.wait_for(lk, std::chrono::nanoseconds(std::min<int64_t>(timeout_ns - (now - t0),
                                                                      1000000)));
        seen = done_gen.load(std::memory_order_acquire);
    }
}

// End the kernel after a device error (or a CUDA error), hand out what
// finished, fail the rest.
void DevServer::recover_locked(int status) {
    if (status != SCL_E_CUDA) stats.device_errors++;
    end_kernel_locked(true);
    const int64_t now = now_ns();
    for (uint32_t j : inflight) {
        if (load_acquire(&hdone[j]) == ring[j].seq) {
            complete_locked(j, hres[j], now);
            stats.completed++;
            continue;
        }
        scl_result r;
        memset(&r, 0, sizeof r);
        r.status = broken ? SCL_E_CUDA : status;
        r.n = ring[j].n;
        r.kind = ring[j].kind;
        complete_locked(j, r, now);
        stats.failed++;
    }
    inflight.clear();
    inflight_pubs.clear();
    spart.init(cfg.unit_ring);
    free_kslots.clear();
    for (uint32_t k = cfg.keyed_slots; k-- > 0;) free_kslots.push_back(k);
    if (broken) {
        for (auto& q : queue) {
            Done d;
            memset(&d.r, 0, sizeof d.r);
            d.r.status = SCL_E_CUDA;
            d.t_submit = q.t_submit;
            d.t_done = now;
            done[q.ticket] = d;
            stats.failed++;
        }
        queue.clear();
    }
    cv_done.notify_all();
}

void DevServer::driver_loop() {
    std::vector<std::pair<uint32_t, uint32_t>> watch;   // (ring index, seq) in flight
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        bool progress = false;
        int64_t now = now_ns();
        for (size_t i = 0; i < inflight.size();) {
            const uint32_t j = inflight[i];
            if (load_acquire(&hdone[j]) == ring[j].seq) {
                complete_locked(j, hres[j], now);
                stats.completed++;
                inflight[i] = inflight.back();
                inflight.pop_back();
                progress = true;
            } else {
                ++i;
            }
        }
        if (progress) {
            last_progress = now;
            cv_done.notify_all();
        }
        if (running && load_acquire(&hh->err) != 0u) {
            recover_locked(SCL_E_TIMEOUT);
            progress = true;
        } else if (running && !inflight.empty() && now - last_progress > 200000000ll) {
            // watchdog: nothing finished for 200 ms; did the kernel end?
            const cudaError_t q = cudaStreamQuery(stream);
            if (q != cudaErrorNotReady) {
                if (q != cudaSuccess) broken = true;
                recover_locked(q == cudaSuccess ? SCL_E_TIMEOUT : SCL_E_CUDA);
                progress = true;
            }
            last_progress = now;
        }
        while (!broken && !queue.empty() && publish_locked(queue.front())) {
            queue.pop_front();
            progress = true;
        }
        if (!broken && !running && !inflight.empty()) launch_locked();
        now = now_ns();
        if (running && inflight.empty() && queue.empty() && cfg.idle_stop_ns != UINT64_MAX &&
            now - last_activity > (int64_t)cfg.idle_stop_ns) {
            if (end_kernel_locked(false) == SCL_OK) stats.idle_stops++;
        }
        if (quitting && ((inflight.empty() && queue.empty()) || broken)) {
            if (running) end_kernel_locked(false);
            break;
        }
        if (progress) continue;
        if (!inflight.empty()) {
            // watch the done words of the jobs in flight without the lock, until
            // one completes, a job is published, the device reports an error,
            // or 50 us pass (the other checks above run again)
            watch.clear();
            for (uint32_t j : inflight) watch.emplace_back(j, ring[j].seq);
            const uint64_t gen = pub_gen.load(std::memory_order_acquire);
            lk.unlock();
            const int64_t until = now_ns() + 50000;
            for (bool hit = false; !hit;) {
                for (const auto& w : watch)
                    if (load_acquire(&hdone[w.first]) == w.second) {
                        hit = true;
                        break;
                    }
                if (pub_gen.load(std::memory_order_acquire) != gen ||
                    load_acquire(&hh->err) != 0u || now_ns() > until)
                    break;
            }
            lk.lock();
        } else if (running) {
            cv_work.wait_for(lk, std::chrono::microseconds(50));
        } else {
            cv_work.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
}

void DevServer::stop() {
    {
        std::lock_guard<std::mutex> g(mu);
        quitting = true;
    }
    cv_work.notify_all();
    if (driver.joinable()) driver.join();
    std::lock_guard<std::mutex> g(mu);
    if (running) end_kernel_locked(false);
    if (!inflight.empty() || !queue.empty()) {
        broken = true;
        recover_locked(SCL_E_CUDA);
    }
    if (ctx) cudaSetDevice(ctx->device);
    if (stream) cudaStreamDestroy(stream);
    stream = nullptr;
    if (hblock) cudaFreeHost(hblock);
    hblock = nullptr;
    if (dblock) ctx->arena.release(dblock);
    dblock = nullptr;
}

}  // namespace scl

using namespace scl;

static int dsrv_of(scl_ctx* ctx, DevServer** out) {
    if (!ctx) return fail(SCL_E_INVALID, "null context");
    clear_error();
    std::lock_guard<std::recursive_mutex> g(ctx->mu);
    if (!ctx->devserver) return fail(SCL_E_STATE, "device-polling server not running");
    *out = ctx->devserver.get();
    return SCL_OK;
}

static int dsrv_submit(scl_ctx* ctx, DevServer* s, const scl_task& task, int64_t t_submit,
                       uint64_t* ticket) {
    Partition p;
    {
        std::lock_guard<std::recursive_mutex> g(ctx->mu);
        const Partition* q = ctx->part(task.part);
        if (!q) return fail(SCL_E_INVALID, "unknown partition handle");
        p = *q;
    }
    return s->submit(task, p, t_submit, ticket);
}

extern "C" {

int scl_devserver_start(scl_ctx* ctx, const scl_devserver_config* cfg) {
    if (!ctx) return fail(SCL_E_INVALID, "null context");
    clear_error();
    std::lock_guard<std::recursive_mutex> g(ctx->mu);
    if (ctx->devserver) return fail(SCL_E_STATE, "device-polling server already running");
    std::unique_ptr<DevServer> s(new DevServer());
    const int st = s->start(ctx, cfg);
    if (st != SCL_OK) {
        std::string msg = scl_last_error();
        s.reset();   // releases what start() took
        return fail(st, "%s", msg.c_str());
    }
    ctx->devserver = std::move(s);
    return SCL_OK;
}

int scl_devserver_submit(scl_ctx* ctx, const scl_task* task, uint64_t* ticket) {
    if (!task || !ticket) return fail(SCL_E_INVALID, "null argument");
    DevServer* s = nullptr;
    SCL_TRY(dsrv_of(ctx, &s));
    return dsrv_submit(ctx, s, *task, 0, ticket);
}

int scl_devserver_poll(scl_ctx* ctx, uint64_t ticket, scl_result* out) {
    DevServer* s = nullptr;
    SCL_TRY(dsrv_of(ctx, &s));
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

int scl_devserver_wait(scl_ctx* ctx, uint64_t ticket, uint32_t timeout_ms, scl_result* out) {
    DevServer* s = nullptr;
    SCL_TRY(dsrv_of(ctx, &s));
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (ticket == 0 || ticket >= s->next_ticket)
            return fail(SCL_E_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    }
    Done d;
    if (!s->wait_done(ticket, 200000, (int64_t)timeout_ms * 1000000, &d))
        return fail(SCL_E_TIMEOUT, "ticket %llu not done after %u ms",
                    (unsigned long long)ticket, timeout_ms);
    if (out) *out = d.r;
    return SCL_OK;
}

int scl_devserver_get_stats(scl_ctx* ctx, scl_devserver_stats* out) {
    DevServer* s = nullptr;
    SCL_TRY(dsrv_of(ctx, &s));
    if (!out) return fail(SCL_E_INVALID, "null output");
    std::lock_guard<std::mutex> g(s->mu);
    *out = s->stats;
    return SCL_OK;
}

int scl_devserver_stop(scl_ctx* ctx) {
    if (!ctx) return SCL_OK;
    std::unique_ptr<DevServer> s;
    {
        std::lock_guard<std::recursive_mutex> g(ctx->mu);
        s = std::move(ctx->devserver);
    }
    if (s) s->stop();
    return SCL_OK;
}

int scl_devserver_replay(scl_ctx* ctx, const scl_task* tasks, const double* arrival_s,
                         uint32_t n, int64_t* latency_ns, scl_result* results) {
    DevServer* s = nullptr;
    SCL_TRY(dsrv_of(ctx, &s));
    if (n && (!tasks || !arrival_s)) return fail(SCL_E_INVALID, "null argument");
    std::vector<uint64_t> tickets(n, 0);
    std::vector<int64_t> sched(n);
    std::vector<int> sub_status(n, SCL_OK);
    std::vector<int> wait_status(n, SCL_OK);
    // A collector thread takes each result as soon as it is done, so the map
    // of finished results stays small however long the trace is.
    std::atomic<uint32_t> published{0};
    std::thread collector([&] {
        for (uint32_t i = 0; i < n; ++i) {
            while (published.load(std::memory_order_acquire) <= i) std::this_thread::yield();
            if (sub_status[i] != SCL_OK) continue;
            Done d;
            if (!s->wait_done(tickets[i], 0, 60000000000ll, &d)) {
                wait_status[i] = SCL_E_TIMEOUT;
                continue;
            }
            if (latency_ns) latency_ns[i] = d.t_done - sched[i];
            if (results) results[i] = d.r;
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
        // open loop: latency counts from the scheduled arrival
        sub_status[i] = dsrv_submit(ctx, s, tasks[i], sched[i], &tickets[i]);
        published.store(i + 1, std::memory_order_release);
    }
    collector.join();
    int worst = SCL_OK;
    for (uint32_t i = 0; i < n; ++i) {
        int st = sub_status[i] != SCL_OK ? sub_status[i] : wait_status[i];
        if (st == SCL_OK) continue;
        if (st == SCL_E_TIMEOUT && sub_status[i] == SCL_OK)
            st = fail(SCL_E_TIMEOUT, "task %u not done after 60 s", i);
        if (latency_ns) latency_ns[i] = -1;
        if (results) {
            memset(&results[i], 0, sizeof results[i]);
            results[i].status = st;
        }
        if (worst == SCL_OK) worst = st;
    }
    if (worst != SCL_OK) return fail(worst, "some tasks were not submitted or not done");
    return SCL_OK;
}

}  // extern "C"
