// Pair passes instantiated for D = 3.
#include "pair_impl.cuh"

VDS_PAIR_INSTANTIATE(3)
