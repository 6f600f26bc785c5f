// Launch-argument structures and launcher declarations shared by the C-ABI
// host code (os3d_api.cu) and the kernels (os3d_transform.cu, os3d_bank.cu).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace os3d {

constexpr int kMaxSlots = 8;    // orientation slots per launch block
constexpr int kMaxL = 32;       // maximal Legendre degree
constexpr int kTileX = 16;      // x-width of a z-pencil tile

// The angular profile h(t), t = w_hat . n in [-1, 1], in two forms:
//  e, o: h(t) = E(v) + t O(v), v = t^2 - 1/2, E and O as monomials in v;
//  a:    h(t) = sum_j a_j T_j(t) (Chebyshev), for when e, o cancel badly.
struct HEval {
  float e[13];
  float o[12];
  float a[kMaxL + 1];
  float c0;   // value used at w = 0: the spherical mean of h
};

enum ZMode { Z_FWD_PREP = 0, Z_FWD_SCORE = 1, Z_INV_SCORE = 2, Z_INV_FINAL = 3 };
enum XYMode { XY_FWD_REAL = 0, XY_FWD_SCORE = 1, XY_INV_SCORE = 2, XY_INV_REAL = 3 };

struct ZArgs {
  const float2* in;
  float2* out;
  const float* mult;        // per-voxel real factor (prep / final)
  long long slot_stride;    // elements between consecutive slot volumes of T
  int ny, nx;
  float wz, wy, wx;         // 2 pi / n per axis
  int nslots;
  int accumulate;           // inverse score: 0 -> write A, 1 -> add to A
  float nvec[kMaxSlots][3]; // orientation n_a (x, y, z) of each slot
  HEval h;
};

struct XYArgs {
  const void* in;
  void* out;
  int nz;                       // planes per volume
  int nplanes;                  // nz * slots in this launch
  long long in_a[kMaxSlots];    // element offset of the slot's input volume
  long long in_b[kMaxSlots];    // second input (antipode) or -1
  long long out_a[kMaxSlots];   // element offset of the slot's output volume
  long long out_b[kMaxSlots];   // second output (antipode) or -1
};

// launchers (return cudaGetLastError of the launch)
cudaError_t launch_z(int nz, int mode, int ev, const ZArgs& a, int grid, cudaStream_t s);
cudaError_t launch_xy(int ny, int nx, int mode, int ubf16, const XYArgs& a, int nz, int nslots,
                      cudaStream_t s);
bool xy_supported(int ny, int nx);
bool z_supported(int nz);

// FP64 bank kernels
cudaError_t launch_fit(const double* d_z, const double* d_w, int npts, int mode, int k,
                       double s_theta, int L, int n_o, double* d_out, cudaStream_t s);
cudaError_t launch_bank_M(int nz, int ny, int nx, int N, double gamma, double eps,
                          const double* d_c, int L, const double* d_slots, int nslots,
                          int n_o, float* Gs, float* GM, float* Minv, cudaStream_t s);

}  // namespace os3d
