// Instantiations of the z- and xy-passes for axis length 16.
#include "os3d_passes.cuh"
OS3D_DEFINE_Z(16)
OS3D_DEFINE_XY(16, 16)
