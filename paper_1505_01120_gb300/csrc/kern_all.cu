// kern_all.cu -- persistent map/reduce kernel instantiations for mask M_ALL.
#include "kernels.cuh"

SCL_DEFINE_TABLE(all, scl::M_ALL)
