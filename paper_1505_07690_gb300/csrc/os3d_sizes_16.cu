// Instantiations of the passes for axis length 16.
#include "os3d_passes.cuh"
#include "os3d_pencil.cuh"
OS3D_DEFINE_Z(16)
OS3D_DEFINE_XY(16, 16)
OS3D_DEFINE_PENCIL(16)
