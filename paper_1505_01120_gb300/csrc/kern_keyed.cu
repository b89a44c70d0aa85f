// kern_keyed.cu -- persistent map/reduce kernel instantiations for mask M_KEYED.
#include "kernels.cuh"

SCL_DEFINE_TABLE(keyed, scl::M_KEYED)

namespace scl {
// The keyed-only kernel capped at kKeyedLeanRegs registers (PATH_LEAN), for
// keyed tasks that share the SMs with a concurrent streaming launch.
const KernelEntry* kernel_table_keyed_lean(int* count) {
    static const KernelEntry tab[] = {SCL_LEAN_SHAPE(512, 2)};
    *count = (int)(sizeof(tab) / sizeof(tab[0]));
    return tab;
}
}  // namespace scl
