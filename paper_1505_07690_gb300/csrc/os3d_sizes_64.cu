// Instantiations of the z- and xy-passes for axis length 64.
#include "os3d_passes.cuh"
OS3D_DEFINE_Z(64)
OS3D_DEFINE_XY(64, 64)
