// Stencil apply instantiated for the f32_2row hopping-field format.
#include "dslash_kernel.cuh"

BRI_INSTANTIATE_DSLASH(bri::LinkF32<BRI_LINK_2ROW>)
