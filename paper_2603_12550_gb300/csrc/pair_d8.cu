// Pair passes instantiated for D = 8.
#include "pair_impl.cuh"

VDS_PAIR_INSTANTIATE(8)
