// kern_keyed.cu -- persistent map/reduce kernel instantiations for mask M_KEYED.
#include "kernels.cuh"

SCL_DEFINE_TABLE(keyed, scl::M_KEYED)
