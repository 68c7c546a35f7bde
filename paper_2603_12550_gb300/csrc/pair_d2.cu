// Pair passes instantiated for D = 2.
#include "pair_impl.cuh"

VDS_PAIR_INSTANTIATE(2)
