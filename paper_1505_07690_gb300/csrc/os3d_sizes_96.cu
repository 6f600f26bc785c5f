// Instantiations of the passes for axis length 96.
#include "os3d_passes.cuh"
#include "os3d_pencil.cuh"
OS3D_DEFINE_Z(96)
OS3D_DEFINE_XY(96, 96)
OS3D_DEFINE_PENCIL(96)
