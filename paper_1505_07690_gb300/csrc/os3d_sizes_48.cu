// Instantiations of the z- and xy-passes for axis length 48.
#include "os3d_passes.cuh"
OS3D_DEFINE_Z(48)
OS3D_DEFINE_XY(48, 48)
