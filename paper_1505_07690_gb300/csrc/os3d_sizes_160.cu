// Instantiations of the z-pass and the pencil pass for axis length 160.
#include "os3d_passes.cuh"
#include "os3d_pencil.cuh"
OS3D_DEFINE_Z(160)
OS3D_DEFINE_PENCIL(160)
