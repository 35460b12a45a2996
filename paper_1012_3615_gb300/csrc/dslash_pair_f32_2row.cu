// Site-pair stencil kernel instantiated for the f32_2row pair-interleaved format.
#include "dslash_pair.cuh"

BRI_INSTANTIATE_DSLASH_PAIR(bri::PairF32<6>)
