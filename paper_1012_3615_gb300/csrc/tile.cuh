// Which lattices the shared-memory stencil kernel takes (tile shape TX..TT in common.cuh).
#pragma once
#include "common.cuh"

namespace bri {
// the tiled kernel needs every extent to be a multiple of the tile
BRI_HD bool tiled_ok(const Geom &g) {
    return g.L[0] % TX == 0 && g.L[1] % TY == 0 && g.L[2] % TZ == 0 && g.L[3] % TT == 0;
}
}  // namespace bri
