// server.h -- continuous-batching server over the persistent batch launch.
//
// Tasks arrive at any time (scl_server_submit / scl_server_submit_load).
// Admission: a task enters the GPU queue only when the resident partitions
// plus the working sets of admitted tasks plus its own fit the HBM budget;
// otherwise it waits, FIFO.  A batcher thread packs every admitted task (up
// to max_batch_tasks) into one persistent launch as soon as one of K
// in-flight slots is free, so work arriving while other batches run joins
// the next launch and overlaps with them on the device; a task that brings
// new data joins a launch once its host-to-device copy has landed (launch
// order is admission order among the tasks whose input is on the device).
// A completion thread
// polls each slot's event, stamps completion times, publishes results,
// returns budget and admits waiting tasks.  With max_batch_tasks = 1 and one
// slot it is the unbatched baseline: one launch per task, FIFO.
#pragma once

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>

#include "runtime.h"

namespace scl {

inline int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct SrvTask {
    uint64_t ticket = 0;
    scl_task task{};
    uint64_t ws_bytes = 0;      // device bytes charged to the budget
    int64_t t_submit = 0;
    // tasks that bring new data: host arrays copied at admission
    bool load = false;
    const void* host0 = nullptr;
    const void* host1 = nullptr;
    scl_dtype dtype = SCL_U32;
    uint64_t n = 0;
    void* block = nullptr;      // arena block of the loaded partition
    cudaEvent_t ready = nullptr;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;         // owned by a batch (set and cleared under Server::mu)
    bool launched = false;     // its work and event are enqueued (under Server::mu)
    std::vector<SrvTask> tasks;
    Plan plan;
    PlanImage img;
    KernelArgs args;
    char* h_plan = nullptr;     // pinned staging for the plan upload
    size_t h_plan_cap = 0;
    // Results land here straight from the kernel: pinned host memory the
    // device writes through its mapped address; entry [cap] holds the error
    // word.  Counters, tickets and flags stay in `zero`, which the kernels
    // return to zero after every launch, so a launch needs no memset.
    scl_result* h_res = nullptr;
    scl_result* d_res = nullptr;   // device address of h_res
    void* zero = nullptr;          // arena block: hdr | tickets | flags
    ExternalScratch ext;
    int64_t t_launch = 0;
};

struct Done {
    scl_result r;
    int64_t t_submit, t_done;
};

struct Server {
    Ctx* ctx = nullptr;
    scl_server_config cfg{};
    uint64_t budget = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<SrvTask> waiting;    // not admitted yet
    std::deque<SrvTask> admitted;   // admitted, not launched
    std::atomic<size_t> admitted_n{0};   // admitted.size(), readable without the lock
    std::vector<Slot> slots;
    std::unordered_map<uint64_t, Done> done;
    uint64_t next_ticket = 1;
    uint64_t inflight_bytes = 0;
    cudaStream_t copy_stream = nullptr;
    bool stopping = false;
    bool batcher_exited = false;
    std::thread batcher, completer;
    scl_server_stats stats{};

    ~Server();
    int start(Ctx* c, const scl_server_config* cfg);
    int submit(SrvTask&& t, uint64_t* ticket);
    void stop();

  private:
    void batcher_loop();
    void completer_loop();
    int launch_slot(Slot& s);
    void finish_slot(Slot& s, int status);
    void admit_locked();
    int stage_load(SrvTask& t);
};

// Working-set estimate a task is charged at admission.
uint64_t task_working_set(Ctx* c, const scl_task& t, const Partition& p, bool load);

}  // namespace scl
