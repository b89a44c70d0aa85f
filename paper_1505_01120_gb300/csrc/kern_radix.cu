// kern_radix.cu -- instantiates the bucket-partitioned keyed reduce kernels.
#include "kernels_radix.cuh"

namespace scl {

const void* radix_hist_fn() { return (const void*)&dev::k_radix_hist<kRadixBlock>; }
const void* radix_scan_fn() { return (const void*)&dev::k_radix_scan<kRadixScanBlock>; }
const void* radix_scatter_fn(bool staged) {
    return staged ? (const void*)&dev::k_radix_scatter<kRadixBlock, true>
                  : (const void*)&dev::k_radix_scatter<kRadixBlock, false>;
}
const void* radix_reduce_fn() { return (const void*)&dev::k_radix_reduce<kRadixBlock>; }

}  // namespace scl
