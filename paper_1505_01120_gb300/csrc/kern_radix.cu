// kern_radix.cu -- instantiates the bucket-partitioned keyed reduce kernels.
#include "kernels_radix.cuh"

namespace scl {

const void* radix_hist_fn() { return (const void*)&dev::k_radix_hist<kRadixBlock>; }
const void* radix_scan_fn() { return (const void*)&dev::k_radix_scan<kRadixScanBlock>; }
const void* radix_scatter_fn(uint32_t log_t, bool hot) {
    switch (log_t) {
        case 12: return hot ? (const void*)&dev::k_radix_scatter<kRadixBlock, 12, true>
                            : (const void*)&dev::k_radix_scatter<kRadixBlock, 12, false>;
        case 13: return hot ? (const void*)&dev::k_radix_scatter<kRadixBlock, 13, true>
                            : (const void*)&dev::k_radix_scatter<kRadixBlock, 13, false>;
        case 14: return hot ? (const void*)&dev::k_radix_scatter<kRadixBlock, 14, true>
                            : (const void*)&dev::k_radix_scatter<kRadixBlock, 14, false>;
        default: return nullptr;
    }
}

// Block sizes as radix_reduce_block() gives them.
const void* radix_reduce_fn(uint32_t log_t) {
    switch (log_t) {
        case 12: return (const void*)&dev::k_radix_reduce<512, 12>;
        case 13: return (const void*)&dev::k_radix_reduce<512, 13>;
        case 14: return (const void*)&dev::k_radix_reduce<1024, 14>;
        default: return nullptr;
    }
}

}  // namespace scl
