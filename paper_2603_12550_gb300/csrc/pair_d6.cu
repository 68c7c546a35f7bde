// Pair passes instantiated for D = 6.
#include "pair_impl.cuh"

VDS_PAIR_INSTANTIATE(6)
