// Instantiations of the z-pass for nz = 160 and the 128 x 160 xy-plane.
#include "os3d_transform.cuh"
OS3D_DEFINE_Z(160)
OS3D_DEFINE_XY(128, 160)
