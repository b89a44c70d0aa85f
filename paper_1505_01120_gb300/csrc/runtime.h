// runtime.h -- host-side context of libscl: arena sub-allocator, partition
// registry, launch shapes, scratch, and the planner that turns partition
// tasks into one persistent launch.  Internal; the ABI is include/scl.h.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "scl.h"

namespace scl {

// ------------------------------------------------------------------ errors

int fail(int code, const char* fmt, ...);
void clear_error();

#define SCL_CUDA(expr)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return ::scl::fail(SCL_E_CUDA, "%s failed: %s (%s:%d)", #expr,                   \
                               cudaGetErrorString(e_), __FILE__, __LINE__);                  \
    } while (0)

#define SCL_TRY(expr)                \
    do {                             \
        int s_ = (expr);             \
        if (s_ != SCL_OK) return s_; \
    } while (0)

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v, size_t a = kAlign) { return (v + a - 1) / a * a; }

// ------------------------------------------------------------------- arena

// First-fit sub-allocator over one caller-owned device buffer.  Blocks are
// 256-byte aligned; adjacent free blocks coalesce.  Thread-safe.
class Arena {
  public:
    void init(char* base, size_t size);
    void* alloc(size_t bytes);
    void release(void* p);
    size_t free_bytes();
    size_t largest_free();
    bool owns(const void* p) const {
        return (const char*)p >= base_ && (const char*)p < base_ + size_;
    }

  private:
    std::mutex mu_;
    char* base_ = nullptr;
    size_t size_ = 0;
    std::map<size_t, size_t> free_;            // offset -> bytes
    std::unordered_map<size_t, size_t> used_;  // offset -> bytes
};

// --------------------------------------------------------------- partitions

struct Partition {
    scl_dtype dtype;
    uint64_t n;
    void* d0;
    void* d1;
    void* block;   // arena block owned by the library, or null (wrapped)
};

// -------------------------------------------------------------- launch shape

struct Shape {
    int block = 256;       // threads that process data
    int ipt = 4;           // 128-bit vectors per thread per chunk
    int ctas_per_sm = 0;   // 0 = as many as fit
    int path = PATH_LDG;   // PATH_LDG or PATH_TMA (uint32 / fp32 kernels only)
    int stages = 0;        // TMA ring depth (0 = first compiled for the shape)
};

const KernelEntry* find_entry(int mask, int block, int ipt, int path = PATH_LDG, int stages = 0);
inline const KernelEntry* find_entry(int mask, const Shape& s) {
    return find_entry(mask, s.block, s.ipt, s.path, s.stages);
}
// Make a kernel launchable with its dynamic shared memory (idempotent).
int prepare_entry(const KernelEntry* e);
int mask_of_kind(uint32_t kind);
int resolve_kind(scl_dtype dt, int kernel, int reduce, uint32_t* kind);

// ------------------------------------------------------------------ scratch

// Device scratch of one launch stream: header words, tickets and flags (zero
// between launches), partial slots.  Grows on demand from the arena.
struct Scratch {
    uint32_t* hdr = nullptr;
    uint32_t* tickets = nullptr;
    uint32_t* flags = nullptr;
    size_t task_cap = 0;
    StreamPartial* spart = nullptr;
    size_t spart_cap = 0;
    uint32_t* kpart = nullptr;
    size_t kpart_cap = 0;
    StreamPartial* fpart = nullptr;
    size_t fpart_cap = 0;
    void* radix = nullptr;          // the large-key reduce's bucket tables (async calls)
    size_t radix_cap = 0;
    std::vector<void*> blocks;
};

// ------------------------------------------------------------------- planner

struct Plan {
    std::vector<DevTask> tasks;
    std::vector<uint32_t> seg_task;
    std::vector<uint32_t> kp_first;
    std::vector<KPiece> kpieces;
    std::vector<uint32_t> fold_tasks;
    uint32_t grid = 1;
    uint32_t nseg_stream = 0;
    uint32_t sslots = 0;
    uint32_t kslots = 0;
    uint32_t fold_gridx = 0;
    int mask = M_U32;
    Shape shape;
};

struct Ctx;
// Build the launch plan of `tasks` (validated).  Result pointers of the
// DevTasks are left null; the caller points them at its result array.
// `shape`, if set, replaces the context's shape for the plan's kernel family.
int plan_tasks(Ctx* c, const scl_task* tasks, uint32_t n, Plan* out,
               const Shape* shape = nullptr);

// Device image of a plan plus its own scratch, in one arena block.
struct PlanImage {
    void* block = nullptr;
    size_t bytes = 0;
    DevTask* tasks = nullptr;
    uint32_t* seg_task = nullptr;
    uint32_t* kp_first = nullptr;
    KPiece* kpieces = nullptr;
    uint32_t* fold_tasks = nullptr;
    scl_result* results = nullptr;
    uint32_t* hdr = nullptr;
    uint32_t* tickets = nullptr;
    uint32_t* flags = nullptr;
    StreamPartial* spart = nullptr;
    uint32_t* kpart = nullptr;
    StreamPartial* fpart = nullptr;
    size_t plan_bytes = 0;   // leading bytes holding the uploaded plan
    size_t zero_off = 0, zero_bytes = 0;  // region to zero once (hdr, tickets, flags)
};

// Scratch that outlives one launch: counters, tickets and flags that the
// kernels return to zero, results the kernel writes in place (may be pinned
// host memory mapped for the device), and where the error word is published.
struct ExternalScratch {
    uint32_t* hdr = nullptr;       // H_WORDS words, zero
    uint32_t* tickets = nullptr;   // task_cap words, zero
    uint32_t* flags = nullptr;     // task_cap words, zero
    size_t task_cap = 0;
    scl_result* results = nullptr; // task_cap results (device-usable address)
    uint32_t* err_out = nullptr;   // device-usable address, written at kernel end
};

// Lay out `p` in a new arena block; fill `host` with the bytes to upload
// (plan_bytes long) with result pointers set; fill `args`.  With `ext`, the
// counters, results and error word live there instead of in the block, and
// nothing in the block needs zeroing.
int build_image(Ctx* c, Plan& p, PlanImage* img, std::vector<char>* host, KernelArgs* args,
                const ExternalScratch* ext = nullptr);

// Launch a planned image (persistent kernel, then the keyed fold if needed).
int launch_plan(Ctx* c, const Plan& p, const KernelArgs& args, cudaStream_t st);

// ---------------------------------------------------------------- context

struct Server;
struct DevServer;

struct Ctx {
    int device = 0;
    int sms = 0;
    int l2_bytes = 0;
    uint64_t arena_bytes = 0;
    uint64_t hbm_budget = 0;                  // scl_config.hbm_budget_bytes
    std::atomic<uint64_t> resident_bytes{0};  // bytes of partitions the library owns
    Arena arena;
    std::recursive_mutex mu;
    std::unordered_map<uint64_t, Partition> parts;
    uint64_t next_part = 1;
    // Defaults: the fastest shapes measured on GB300 (vector-load kernels):
    // 256x8 for the streaming families and the mixed kernel; 512x4 for the
    // keyed-only kernel (two CTAs of 72 KB per SM, 32 warps).
    Shape shape[M_NUM] = {Shape{256, 8, 0, PATH_LDG, 0}, Shape{256, 8, 0, PATH_LDG, 0},
                          Shape{512, 4, 0, PATH_LDG, 0}, Shape{256, 8, 0, PATH_LDG, 0}};
    std::map<const void*, int> occ_cache;
    int large_path = SCL_LARGE_AUTO;   // scl_set_large_path
    int batch_split = 1;               // scl_set_batch_split
    // Scratch of single-partition launches, one per stream, so that launches
    // on different streams may overlap on the device.
    std::unordered_map<cudaStream_t, Scratch> single_by_stream;
    Scratch& single_for(cudaStream_t st) { return single_by_stream[st]; }
    scl_result* d_result = nullptr;        // single-call result slot
    scl_result* h_result = nullptr;        // pinned, mapped: [0] result, [1] error word
    scl_result* dh_result = nullptr;       // device address of h_result
    uint32_t* d_kout = nullptr;            // single-call keyed outputs (counts|sums|sums64)
    std::string tune_path;
    std::unique_ptr<Server> server;
    std::unique_ptr<DevServer> devserver;

    const Partition* part(scl_part h) const {
        auto it = parts.find(h);
        return it == parts.end() ? nullptr : &it->second;
    }
    Shape shape_for(int mask) const;
    uint32_t grid_max(int mask, const Shape& sh);
};

int ensure_scratch(Ctx* c, Scratch* s, size_t tasks, size_t sslots, size_t kslots, size_t fparts);
void fill_task(DevTask* t, const Partition& p, uint32_t kind, const float* coef, uint32_t nk);

// Single-partition launch (scl_map_reduce*, scl_keyed_reduce*).
int run_single(Ctx* c, const Partition& p, uint32_t kind, const float* coef, uint32_t nk,
               uint32_t* counts, float* sums, double* sums64, scl_result* dres, cudaStream_t st,
               uint32_t* err_out = nullptr);

// Global count of kernel launches made by the library (graph replays included).
void count_launches(uint64_t n);

// Tuning cache and the autotuner.
int autotune(Ctx* c, const scl_autotune_config* cfg, cudaStream_t st, scl_autotune_report* rep);
int load_tuning(Ctx* c, const char* path);
int save_tuning(Ctx* c, const char* path);

}  // namespace scl

struct scl_ctx : scl::Ctx {};
