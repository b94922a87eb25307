// Kernel family instantiations: 3,3.
#include "ops_impl.cuh"
HOPU_DEFINE_OPS(3, 3)
