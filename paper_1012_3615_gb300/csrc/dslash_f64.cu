// Stencil apply instantiated for the f64 hopping-field format.
#include "dslash_kernel.cuh"

BRI_INSTANTIATE_DSLASH(bri::LinkF64)
