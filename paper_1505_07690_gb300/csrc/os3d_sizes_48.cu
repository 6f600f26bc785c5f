// Instantiations of the passes for axis length 48.
#include "os3d_passes.cuh"
#include "os3d_pencil.cuh"
OS3D_DEFINE_Z(48)
OS3D_DEFINE_XY(48, 48)
OS3D_DEFINE_PENCIL(48)
