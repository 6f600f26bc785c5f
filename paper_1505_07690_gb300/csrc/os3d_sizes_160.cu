// Instantiations of the passes for axis length 160: the z-pass, the pencil
// pass and the plane pass of 128 x 160 planes.
#include "os3d_passes.cuh"
#include "os3d_pencil.cuh"
OS3D_DEFINE_Z(160)
OS3D_DEFINE_XY(128, 160)
OS3D_DEFINE_PENCIL(160)
