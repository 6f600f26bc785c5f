// Instantiations of the passes for axis length 64.
#include "os3d_passes.cuh"
#include "os3d_pencil.cuh"
OS3D_DEFINE_Z(64)
OS3D_DEFINE_XY(64, 64)
OS3D_DEFINE_PENCIL(64)
