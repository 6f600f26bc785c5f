// Instantiations of the z- and xy-passes for axis length 128.
#include "os3d_passes.cuh"
OS3D_DEFINE_Z(128)
OS3D_DEFINE_XY(128, 128)
