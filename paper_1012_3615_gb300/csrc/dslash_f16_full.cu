// Stencil apply instantiated for the f16_full hopping-field format.
#include "dslash_kernel.cuh"

BRI_INSTANTIATE_DSLASH(bri::LinkF16<BRI_LINK_FULL>)
