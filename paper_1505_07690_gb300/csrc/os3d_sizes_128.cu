// Instantiations of the passes for axis length 128.
#include "os3d_passes.cuh"
#include "os3d_pencil.cuh"
OS3D_DEFINE_Z(128)
OS3D_DEFINE_XY(128, 128)
OS3D_DEFINE_PENCIL(128)
