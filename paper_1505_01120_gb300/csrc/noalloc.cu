// noalloc.cu -- a map+reduce entry point that allocates no memory at all.
//
// Some callers cannot allocate device memory when they need a result:
// plug-ins living inside a host application that has already claimed all of
// the GPU's memory through its own pool, and latency-critical paths that
// cannot afford the implicit device synchronisation of cudaMalloc / cudaFree.  scl_map_reduce_noalloc serves them: it needs no context, no
// arena and no pinned staging buffer.  The caller passes the input array and
// a device scl_result slot; the only scratch is the file-scope device array
// below, which every GPU that loads the library keeps until the process exits.
//
// The kernel is the same persistent map/reduce kernel the context API uses,
// at the launch shape 256 threads x 4 vectors per thread, so a result equals
// what scl_map_reduce returns for the same partition when that context's
// family runs at that shape (scl_set_shape).
#include <stddef.h>
#include <string.h>

#include <mutex>

#include "runtime.h"

namespace {

using namespace scl;

constexpr int kNaBlock = 256;
constexpr int kNaIpt = 4;
constexpr uint32_t kNaMaxSegments = 4096;
constexpr int kNaMaxDevices = 64;

// Everything one call needs besides its input and output.
struct NoAllocScratch {
    uint32_t hdr[H_WORDS];      // segment counter, exit counter, error word
    uint32_t ticket[4];         // the task's ticket
    uint32_t flags[4];
    StreamPartial part[kNaMaxSegments];
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// The largest accepted partition must fit the partial slots at the launch shape.
static_assert(stream_nseg(SCL_NOALLOC_MAX_ELEMENTS,
                          stream_seg_elems(SCL_NOALLOC_MAX_ELEMENTS, kNaBlock * kNaIpt * 4)) <=
                  kNaMaxSegments,
              "SCL_NOALLOC_MAX_ELEMENTS exceeds the scratch's segment partials");
static_assert(offsetof(NoAllocScratch, part) == 96, "counters cleared per call: 96 bytes");

struct DeviceSetup {
    bool ready = false;
    NoAllocScratch* scratch = nullptr;   // device address of g_noalloc_scratch
    int sms = 0;
    int per_sm[2] = {0, 0};              // resident CTAs: uint32 kernel, fp32 kernel
};

std::mutex g_setup_mu;
DeviceSetup g_setup[kNaMaxDevices];

// Once per device, with that device current: resolve the array's device
// address (host code only ever sees a host-side stand-in for the symbol) and
// the launch limits.  The cache is per device ordinal: it assumes the
// device's primary context lives as long as the library (a cudaDeviceReset,
// or a caller's own driver-API context, would need the lookup again).
int setup_device(int dev, DeviceSetup** out) {
    std::lock_guard<std::mutex> g(g_setup_mu);
    DeviceSetup& s = g_setup[dev];
    if (!s.ready) {
        void* p = nullptr;
        SCL_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        SCL_CUDA(cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev));
        const int masks[2] = {M_U32, M_F32};
        for (int i = 0; i < 2; ++i) {
            const KernelEntry* e = find_entry(masks[i], kNaBlock, kNaIpt);
            if (!e) return fail(SCL_E_STATE, "default-shape kernel missing");
            int nb = 0;
            SCL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, e->fn, kNaBlock,
                                                                   e->dyn_smem));
            s.per_sm[i] = nb > 0 ? nb : 1;
        }
        s.scratch = static_cast<NoAllocScratch*>(p);
        s.ready = true;
    }
    *out = &s;
    return SCL_OK;
}

}  // namespace

extern "C" int scl_map_reduce_noalloc(const void* dev_in, scl_dtype dtype, uint64_t n,
                                      scl_map_kernel kernel, const float coef[3],
                                      scl_reduce reduce, void* stream, scl_result* dev_out) {
    clear_error();
    if (!dev_out) return fail(SCL_E_INVALID, "null device result pointer");
    if (n && !dev_in) return fail(SCL_E_INVALID, "null input pointer");
    if ((uintptr_t)dev_in % 4) return fail(SCL_E_INVALID, "input must be 4-byte aligned");
    if (n > SCL_NOALLOC_MAX_ELEMENTS)
        return fail(SCL_E_INVALID,
                    "scl_map_reduce_noalloc takes at most %llu elements (got %llu); its "
                    "fixed scratch holds %u segment partials",
                    (unsigned long long)SCL_NOALLOC_MAX_ELEMENTS, (unsigned long long)n,
                    kNaMaxSegments);
    if (dtype == SCL_KV_I32_F32)
        return fail(SCL_E_UNSUPPORTED, "scl_map_reduce_noalloc has no keyed variant");
    uint32_t kind;
    SCL_TRY(resolve_kind(dtype, kernel, reduce, &kind));

    int dev = 0;
    SCL_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) return fail(SCL_E_INVALID, "device %d out of range", dev);
    DeviceSetup* s = nullptr;
    SCL_TRY(setup_device(dev, &s));

    const int mask = mask_of_kind(kind);
    const KernelEntry* e = find_entry(mask, kNaBlock, kNaIpt);
    if (!e) return fail(SCL_E_STATE, "default-shape kernel missing");

    KernelArgs a;
    memset(&a, 0, sizeof a);
    Partition p{dtype, n, const_cast<void*>(dev_in), nullptr, nullptr};
    fill_task(&a.single, p, kind, coef, 0);
    DevTask& t = a.single;
    t.result = dev_out;
    t.seg_elems = stream_seg_elems(n, (uint32_t)(kNaBlock * kNaIpt * 4));
    t.nseg = stream_nseg(n, t.seg_elems);
    if (t.nseg > kNaMaxSegments)
        return fail(SCL_E_INVALID, "partition needs %u segments, scratch holds %u", t.nseg,
                    kNaMaxSegments);
    a.nseg_stream = t.nseg;
    NoAllocScratch* sc = s->scratch;
    a.spart = sc->part;
    a.tickets = sc->ticket;
    a.task_flags = sc->flags;
    a.hdr = sc->hdr;

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // The array keeps whatever the previous call left; the counters and the
    // ticket must start at zero.  (The partial slots are written before they
    // are read.)
    SCL_CUDA(cudaMemsetAsync(sc, 0, offsetof(NoAllocScratch, part), st));
    const uint32_t gmax = (uint32_t)(s->sms * s->per_sm[mask == M_U32 ? 0 : 1]);
    const uint32_t grid = t.nseg < gmax ? t.nseg : gmax;
    void* params[] = {&a};
    SCL_CUDA(cudaLaunchKernel(e->fn, dim3(grid), dim3(kNaBlock), params, e->dyn_smem, st));
    count_launches(1);
    return SCL_OK;
}
