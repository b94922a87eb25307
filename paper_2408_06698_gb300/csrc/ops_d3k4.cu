// Kernel family instantiations: 3,4.
#include "ops_impl.cuh"
HOPU_DEFINE_OPS(3, 4)
