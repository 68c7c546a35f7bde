// Pair passes instantiated for D = 10.
#include "pair_impl.cuh"

VDS_PAIR_INSTANTIATE(10)
