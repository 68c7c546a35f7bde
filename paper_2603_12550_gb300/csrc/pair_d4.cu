// Pair passes instantiated for D = 4.
#include "pair_impl.cuh"

VDS_PAIR_INSTANTIATE(4)
