// Instantiations of the passes for axis length 32.
#include "os3d_passes.cuh"
#include "os3d_pencil.cuh"
OS3D_DEFINE_Z(32)
OS3D_DEFINE_XY(32, 32)
OS3D_DEFINE_PENCIL(32)
