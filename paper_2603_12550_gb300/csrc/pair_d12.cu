// Pair passes instantiated for D = 12.
#include "pair_impl.cuh"

VDS_PAIR_INSTANTIATE(12)
