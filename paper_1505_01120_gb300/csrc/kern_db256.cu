// kern_db256.cu -- k_doorbell instantiations with 256-thread CTAs.
#include "kernels_db.cuh"

namespace scl {
const void* doorbell_kernel_256(int ipt) {
    SCL_DB_ENTRY(256, 2)
    SCL_DB_ENTRY(256, 4)
    SCL_DB_ENTRY(256, 8)
    return nullptr;
}
}  // namespace scl
