// Instantiations of the z-pass for nz = 160.
#include "os3d_passes.cuh"
OS3D_DEFINE_Z(160)
