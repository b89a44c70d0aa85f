// kern_f32.cu -- persistent map/reduce kernel instantiations for mask M_F32.
#include "kernels.cuh"

SCL_DEFINE_TABLE(f32, scl::M_F32)
