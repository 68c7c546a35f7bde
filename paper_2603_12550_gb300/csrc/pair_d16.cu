// Pair passes instantiated for D = 16.
#include "pair_impl.cuh"

VDS_PAIR_INSTANTIATE(16)
