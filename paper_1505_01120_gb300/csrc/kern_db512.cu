// kern_db512.cu -- k_doorbell instantiations with 512-thread CTAs.
#include "kernels_db.cuh"

namespace scl {
const void* doorbell_kernel_512(int ipt) {
    SCL_DB_ENTRY(512, 2)
    SCL_DB_ENTRY(512, 4)
    SCL_DB_ENTRY(512, 8)
    return nullptr;
}
}  // namespace scl
