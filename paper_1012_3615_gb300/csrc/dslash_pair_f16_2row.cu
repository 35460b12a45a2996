// Site-pair stencil kernel instantiated for the f16_2row pair-interleaved format.
#include "dslash_pair.cuh"

BRI_INSTANTIATE_DSLASH_PAIR(bri::PairF16<6>)
