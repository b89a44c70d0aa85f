// kern_tma.cu -- TMA bulk-copy pipeline instantiations (uint32 and fp32 kinds).
// Ring depth is chosen so a CTA holds about 96 KB of stages (two CTAs per SM).
#include "kernels_tma.cuh"

namespace scl {

#define SCL_TMA_SET(M)                                                      \
    SCL_TMA_SHAPE(M, 256, 2, 12), SCL_TMA_SHAPE(M, 256, 4, 6),             \
    SCL_TMA_SHAPE(M, 256, 4, 4), SCL_TMA_SHAPE(M, 256, 8, 3),              \
    SCL_TMA_SHAPE(M, 512, 2, 6), SCL_TMA_SHAPE(M, 512, 4, 3)

const KernelEntry* kernel_table_tma_u32(int* count) {
    static const KernelEntry tab[] = {SCL_TMA_SET(M_U32)};
    *count = (int)(sizeof(tab) / sizeof(tab[0]));
    return tab;
}

const KernelEntry* kernel_table_tma_f32(int* count) {
    static const KernelEntry tab[] = {SCL_TMA_SET(M_F32)};
    *count = (int)(sizeof(tab) / sizeof(tab[0]));
    return tab;
}

}  // namespace scl
