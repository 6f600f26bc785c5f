// Instantiations of the z-pass and the pencil pass for axis length 256.
#include "os3d_passes.cuh"
#include "os3d_pencil.cuh"
OS3D_DEFINE_Z(256)
OS3D_DEFINE_PENCIL(256)
