// kern_u32.cu -- persistent map/reduce kernel instantiations for mask M_U32.
#include "kernels.cuh"

SCL_DEFINE_TABLE(u32, scl::M_U32)
