// Pair passes instantiated for D = 14.
#include "pair_impl.cuh"

VDS_PAIR_INSTANTIATE(14)
