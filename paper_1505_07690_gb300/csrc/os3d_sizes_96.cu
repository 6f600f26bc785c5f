// Instantiations of the z- and xy-passes for axis length 96.
#include "os3d_passes.cuh"
OS3D_DEFINE_Z(96)
OS3D_DEFINE_XY(96, 96)
