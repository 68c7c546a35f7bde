// Pair passes instantiated for D = 9.
#include "pair_impl.cuh"

VDS_PAIR_INSTANTIATE(9)
