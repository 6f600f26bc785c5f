// Instantiations of the passes for axis length 256 (plane pass on 8-CTA clusters).
#include "os3d_passes.cuh"
#include "os3d_pencil.cuh"
OS3D_DEFINE_Z(256)
OS3D_DEFINE_XY(256, 256)
OS3D_DEFINE_PENCIL(256)
