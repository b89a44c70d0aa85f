// kern_radix.cu -- instantiates the bucket-partitioned keyed reduce kernels.
#include "kernels_radix.cuh"

namespace scl {

const void* radix_hist_fn() { return (const void*)&dev::k_radix_hist<kRadixBlock>; }
const void* radix_scan_fn() { return (const void*)&dev::k_radix_scan<kRadixScanBlock>; }
// The plain form stages its input with TMA (3 CTAs per SM at up to 256
// buckets); the hot-id form keeps register loads, since its hot table leaves
// room for only 2 CTAs per SM with the input buffer.
#define SCL_SCATTER(LT)                                                               \
    (hot ? (const void*)&dev::k_radix_scatter<kRadixBlock, LT, true, radix_scatter_tma(true)> \
         : (const void*)&dev::k_radix_scatter<kRadixBlock, LT, false, radix_scatter_tma(false)>)
const void* radix_scatter_fn(uint32_t log_t, bool hot) {
    switch (log_t) {
        case 12: return SCL_SCATTER(12);
        case 13: return SCL_SCATTER(13);
        case 14: return SCL_SCATTER(14);
        default: return nullptr;
    }
}
#undef SCL_SCATTER

// Block sizes as radix_reduce_block() gives them.
const void* radix_reduce_fn(uint32_t log_t) {
    switch (log_t) {
        case 12: return (const void*)&dev::k_radix_reduce<512, 12>;
        case 13: return (const void*)&dev::k_radix_reduce<1024, 13>;
        case 14: return (const void*)&dev::k_radix_reduce<1024, 14>;
        default: return nullptr;
    }
}

}  // namespace scl
