// Kernel family instantiations: 3,1 3,2.
#include "ops_impl.cuh"
HOPU_DEFINE_OPS(3, 1)
HOPU_DEFINE_OPS(3, 2)
