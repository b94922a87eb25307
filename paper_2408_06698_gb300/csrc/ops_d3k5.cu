// Kernel family instantiations: 3,5.
#include "ops_impl.cuh"
HOPU_DEFINE_OPS(3, 5)
