// Kernel family instantiations: 2,1 2,2 2,3 2,4.
#include "ops_impl.cuh"
HOPU_DEFINE_OPS(2, 1)
HOPU_DEFINE_OPS(2, 2)
HOPU_DEFINE_OPS(2, 3)
HOPU_DEFINE_OPS(2, 4)
