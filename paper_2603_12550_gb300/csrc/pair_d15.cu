// Pair passes instantiated for D = 15.
#include "pair_impl.cuh"

VDS_PAIR_INSTANTIATE(15)
