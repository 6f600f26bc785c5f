// Instantiations of the z- and xy-passes for axis length 32.
#include "os3d_passes.cuh"
OS3D_DEFINE_Z(32)
OS3D_DEFINE_XY(32, 32)
