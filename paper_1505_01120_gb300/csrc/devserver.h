// devserver.h -- host side of the device-polling server (k_doorbell).
//
// Jobs are published, not launched: submit() writes job p's descriptor into
// ring slot p % job_ring of pinned host memory and raises the count of
// published jobs (the doorbell); the resident kernel picks the job up.  A driver thread watches the done
// words, hands out results, publishes jobs that waited for ring space, ends
// the kernel after idle_stop_ns without work, and recovers when the device
// reports an error (its wait limit ran out, or a descriptor failed a check):
// it stops the kernel, fails the jobs still in flight with SCL_E_TIMEOUT,
// zeroes the device state and carries on.  A kernel instance is launched
// whenever work is published and none is running.
#pragma once

#include <map>

#include "range_alloc.h"
#include "server.h"

namespace scl {

struct DbInflight {
    uint64_t ticket = 0;
    uint32_t seq = 0;
    uint32_t nseg = 0;
    uint64_t unit0 = 0;
    uint64_t pub = 0;               // publication index
    uint32_t spart0 = UINT32_MAX;   // partial range (streaming, nseg > 1)
    uint32_t kslot = UINT32_MAX;    // keyed accumulator (keyed, nseg > 1)
    uint64_t n = 0;
    uint32_t kind = 0;
    int64_t t_submit = 0;
};

struct DbPending {
    uint64_t ticket = 0;
    DevTask t{};
    int64_t t_submit = 0;
};

struct DevServer {
    Ctx* ctx = nullptr;
    scl_devserver_config cfg{};
    const void* fn = nullptr;
    int block = 0, ipt = 0;
    uint32_t grid = 0;
    cudaStream_t stream = nullptr;

    // pinned host memory, mapped: header | jobs | results | done
    char* hblock = nullptr;
    DbHost* hh = nullptr;
    DbJob* hjobs = nullptr;
    scl_result* hres = nullptr;
    uint32_t* hdone = nullptr;
    scl_result* dres = nullptr;   // device address of hres
    // arena block: state | tickets | flags | keyed accumulators | partials
    void* dblock = nullptr;
    size_t zero_small = 0;        // state + tickets + flags
    size_t zero_all = 0;          // ... + keyed accumulators
    DbArgs args{};

    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::deque<DbPending> queue;             // waiting for ring space
    std::vector<DbInflight> ring;            // by job ring slot (publication index % job_ring)
    std::vector<uint32_t> free_kslots, inflight;
    std::map<uint64_t, uint64_t> inflight_pubs;   // publication index -> first unit
    RangeAlloc spart;
    uint64_t pubs = 0;                       // jobs published in this kernel instance
    uint64_t units = 0;                      // their units
    uint32_t next_seq = 1;
    bool running = false, broken = false, quitting = false;
    int64_t last_activity = 0, last_progress = 0;
    std::unordered_map<uint64_t, Done> done;
    uint64_t next_ticket = 1;
    std::atomic<uint64_t> pub_gen{0};    // bumped by every publish
    std::atomic<uint64_t> done_gen{0};   // bumped by every completion
    scl_devserver_stats stats{};
    std::thread driver;

    ~DevServer();
    int start(Ctx* c, const scl_devserver_config* cfg);
    int submit(const scl_task& task, const Partition& p, int64_t t_submit, uint64_t* ticket);
    // Wait for a ticket: spin (lock released) up to spin_ns, then block.
    // True with the result taken out; false on timeout.
    bool wait_done(uint64_t ticket, int64_t spin_ns, int64_t timeout_ns, Done* out);
    void stop();

  private:
    bool publish_locked(DbPending& p);
    int launch_locked();
    int end_kernel_locked(bool zero_all_state);
    void complete_locked(uint32_t j, const scl_result& r, int64_t now);
    void recover_locked(int status);
    void driver_loop();
};

}  // namespace scl
