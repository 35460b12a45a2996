// Stencil apply instantiated for the f32_8p hopping-field format.
#include "dslash_kernel.cuh"

BRI_INSTANTIATE_DSLASH(bri::LinkF32<BRI_LINK_8PARAM>)
