// Launch-argument structure and launcher declarations shared by the C-ABI
// host code (os3d_api.cu) and the kernels (os3d_passes.cuh, os3d_bank.cu).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

namespace os3d {

constexpr int kMaxSlots = 12;   // orientation slots per launch block
constexpr int kAutoSlots = 11;  // block size when the caller leaves it to the library
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
  float2 e2[13], o2[12];   // (e_k, e_k) and (o_k, o_k): operands of two-lane FMAs
};

// z-passes (DFT along z of 16-wide pencil tiles):
//  Z_FWD_PREP : T0 -> DFT_z -> x mult (G/n^3)                     -> f_hat
//  Z_FWD_SCORE: f_hat x h(w_hat . n_s) -> IDFT_z, every slot      -> T_s
//  Z_INV_SCORE: T_s -> DFT_z -> x h(w_hat . n_s), sum over slots  -> A
//  Z_INV_FINAL: A x mult (G/(n^3 max(M,eps))) -> IDFT_z           -> T0
enum ZMode { Z_FWD_PREP = 0, Z_FWD_SCORE = 1, Z_INV_SCORE = 2, Z_INV_FINAL = 3 };
// xy-passes (2D DFT of z-planes: a whole plane per CTA; 256^2 planes: an 8-CTA cluster
// per plane; XY_FWD_SCORE on 256^2 planes four independent quarter-plane CTAs, on
// 128^2 planes with complex64 scores two half-plane CTAs):
//  XY_FWD_REAL : f (real) -> DFT_xy                                -> T0
//  XY_FWD_SCORE: T_s -> IDFT_xy -> U_a, U_b = conj U_a              (HBM store)
//  XY_INV_SCORE: U_a + conj U_b (HBM load) -> DFT_xy               -> T_s
//  XY_INV_REAL : T0 -> IDFT_xy -> real part                        -> f
//  XY_SOFT     : T_s -> IDFT_xy -> m_s Phi(.) -> DFT_xy             -> T_s (in place)
//                (Phi the soft threshold |u|^p sgn(u) per part, m_s = 2 for a pair)
// XY_INV_WSCORE: XY_INV_SCORE on the weighted input 2 g (w_a U_a + conj(w_b U_b))
// (the gradient of g sum w |U|^2, folded into the load; complex64 U)
// XY_WENERGY: XY_SOFT with m_s Phi replaced by 2 g (w_a + w_b) (the gradient of
// g sum w |U|^2 for U_b = conj U_a), sum (w_a + w_b) |U_a|^2 of each unit into
// epart[epart_base + unit]
enum XYMode { XY_FWD_REAL = 0, XY_FWD_SCORE = 1, XY_INV_SCORE = 2, XY_INV_REAL = 3, XY_SOFT = 4,
              XY_INV_WSCORE = 5, XY_WENERGY = 6 };

struct PassArgs {
  const void* in;
  const void* in2;            // Z_INV_FINAL: second partial sum (or null)
  void* out;
  const float* mult;          // per-voxel real factor (z prep / final)
  long long in_off;           // element offset of the input volume
  long long out_off;          // element offset of the output volume
  long long slot_stride;      // elements between consecutive T volumes
  long long ua[kMaxSlots];    // element offset of U_a of each slot
  long long ub[kMaxSlots];    // element offset of U_b = antipode, or -1
  int nz, ny, nx;
  float wz, wy, wx;           // 2 pi / n per axis
  int nslots;
  int accumulate;             // Z_INV_SCORE: 0 -> A = sum, 1 -> A += sum
  float power;                // XY_SOFT / soft threshold: exponent p > 0
  int disc;                   // 1: 16-column z tiles outside the disc |w_xy| < pi are
                              // skipped by the z-passes and read as zero / not written
                              // by the plane passes (not by the pencil passes)
  float nvec[kMaxSlots][3];   // orientation n_a (x, y, z) of each slot
  const float* wgt;           // XY_INV_WSCORE, XY_WENERGY: weight per element, U's layout
  const float* gscale;        // XY_INV_WSCORE, XY_WENERGY: the scalar g (device; or null
                              // for 1 in XY_WENERGY)
  double* epart;              // XY_WENERGY: per-unit energy sums
  long long epart_base;       // XY_WENERGY: index of this launch's first unit
  HEval h;
};

// Strided pencil passes (x and y directions of planes that the xy-pass
// cannot hold): modes and line geometry, see os3d_pencil.cuh.
enum PencilMode {
  PN_C2C = 0,   // complex -> complex (in place allowed); blockIdx.y = slot
  PN_R2C = 1,   // real f -> complex (forward DFT)
  PN_C2R = 2,   // complex -> real part (inverse DFT)
  PN_C2U = 3,   // T_s -> U_a and U_b = conj U_a (inverse DFT)
  PN_U2C = 4    // U_a + conj U_b -> T_s (forward DFT)
};

struct PencilGeom {
  int group;
  long long gstride, lstride, estride;
};

// launchers (return cudaGetLastError of the launch)
cudaError_t launch_z(int nz, int mode, int ev, const PassArgs& a, int grid_tiles,
                     cudaStream_t s);
cudaError_t launch_xy(int ny, int nx, int mode, int ubf16, const PassArgs& a, cudaStream_t s);
bool xy_supported(int ny, int nx);
bool z_supported(int nz);

// |u|^p for other exponents, kept out of line so that the unrolled DFT
// kernels that call the soft threshold stay small
static __device__ __noinline__ float soft_pow(float m, float p) { return powf(m, p); }

// Soft threshold Phi(u) = |u|^p sgn(u) of one real number (Sec. 4.1); the
// common exponent 1.5 as |u| sqrt(|u|).
__device__ __forceinline__ float soft_part(float u, float p) {
  const float m = fabsf(u);
  const float r = (p == 1.5f) ? m * sqrtf(m) : (p == 1.0f ? m : soft_pow(m, p));
  return copysignf(r, u);
}

// elementwise kernels (os3d_elementwise.cu)
cudaError_t launch_approx_sum(const void* U, int ubf16, int n_o, long long nvox, float w,
                              float* out, cudaStream_t s);
cudaError_t launch_soft_scores(const void* in, void* out, int ubf16, long long count,
                               float power, cudaStream_t s);
// weighted energy L = sum w |U|^2 (os3d_elementwise.cu): block partial sums
// into scratch[1 ..], their sum into scratch[0] and *loss (when not null);
// the gradient G = 2 g w U with g read on the device. w may be null (w = 1).
constexpr int kMaxEnergyBlocks = 4096;
cudaError_t launch_energy(const void* U, const float* w, int ubf16, long long count,
                          double* scratch, float* loss, cudaStream_t s);
cudaError_t launch_energy_grad(const void* U, const float* w, int ubf16, long long count,
                               const float* g, void* G, cudaStream_t s);
// the sum of scratch[1 .. n] in index order into scratch[0] and *loss
cudaError_t launch_energy_final(double* scratch, long long n, float* loss, cudaStream_t s);
// y = *g x over count floats (y may be x)
cudaError_t launch_scale_by(const float* x, float* y, long long count, const float* g,
                            cudaStream_t s);
// in place on a.nslots volumes of a.out, a.slot_stride apart, nvox each;
// slot s scaled by 2 when a.ub[s] >= 0 (an antipodal pair)
cudaError_t launch_soft_slots(const PassArgs& a, long long nvox, cudaStream_t s);

// Linear left-invariant diffusion (os3d_diffusion.cu): per-frequency
// integration of the orientation vector; orientation sets up to 68.
constexpr int kMaxOrientE = 68;   // largest orientation set of the diffusion kernel
constexpr int kEStride = 72;      // propagator rows and columns held (a multiple of 8)
struct EnhanceArgs {
  const float2* fh;           // f_hat G / n^3
  float2* A;                  // out: fh * n^3 h^T E h (then x G/(n^3 max(M,eps)), IDFT);
                              // zero on entry outside the listed frequencies
  const int4* seg;            // in-ball row segments {z, y, kx0, first index}
  int nseg, n_in;             // segments; listed frequencies
  int mirror;                 // 1: the list covers half the ball, results go to w and -w
  int nz, ny, nx;
  float wz, wy, wx;           // 2 pi / n per axis
  float n3;                   // nz ny nx
  int n_o;
  int steps;                  // Strang steps K
  float half_dt;              // t / (2K)
  float D11, D33;
  int paired;                 // 1: an antipodally closed set, integrated as its n_o/2 pairs
  float nvec[kMaxOrientE][3];      // orientations (paired: the pairs' first members)
  float Et[kEStride * kEStride];   // exp(dt D44 L) transposed: Et[j kEStride + i] = E[i][j],
                                   // zero outside i, j < n_o; paired: the blocks C = A + B
                                   // (rows and columns 0 ..) and D = A - B (from the
                                   // kernel's block offset) of E = [[A, B], [B, A]]
  HEval h;
};
cudaError_t launch_enhance(const EnhanceArgs& a, int ev, cudaStream_t s);
// rows per block of the paired integration for a closed set of n_o vectors, or -1
int enhance_pair_block(int n_o);
// The same integration with the propagator product on the tensor cores
// (os3d_diffusion_tc.cu), for orientation sets of up to 176 vectors.
struct EnhanceTCArgs {
  const float2* fh;           // f_hat G / n^3
  float2* A;                  // out: fh * n^3 h^T E h (zero on entry outside the listed frequencies)
  const int4* seg;            // in-ball row segments {z, y, kx0, first index}
  const unsigned char* prep;  // E_hi | E_lo (canonical layout, half) | orientations (NP x 3 float)
  unsigned* err;              // bounded waits that ran out (device counter, or null)
  int nseg, n_in, mirror;
  int nz, ny, nx;
  float wz, wy, wx, n3;
  int n_o, steps;
  float half_dt, D11, D33;
  float inv_se;               // 1 / (the power of two E was scaled by)
  HEval h;
};
cudaError_t launch_enhance_tc(const EnhanceTCArgs& a, int ev, cudaStream_t s);
int tc_padded_orientations(int n_o);   // N_o padded to the kernel's size, or -1
// self-test of the bounded mbarrier wait (64 threads, one CTA)
cudaError_t launch_wait_selftest(unsigned long long limit_ns, int arrive, unsigned* timeouts,
                                 cudaStream_t s);
size_t tc_prep_bytes(int np);
// E (n x n FP64) and the orientations in the kernel's device layout; returns
// the factor that undoes the power-of-two scale applied to E
float tc_prepare(const double* E, const double* orient, int n, int np, std::vector<unsigned char>& out);
// host: the frequencies inside the ball |w| < pi (a superset by 1e-12 in
// |w|^2) as row segments {z, y, kx0, first index}: rows of constant (kz, ky)
// with kx in [kx0, -kx0] (or [0, a] for the row through the origin when
// `half`); with `half` only kz > 0, or kz = 0 and ky > 0, and that half row.
std::vector<int4> ball_segments(int nz, int ny, int nx, bool half, int* n_in);
// host: exp(tau L) of the discrete Laplace-Beltrami operator (n x n, FP64);
// returns the spherical-harmonic degree used, or -1
int angular_propagator(const double* V, int n, int sh_degree, double tau, std::vector<double>& E);

// launch accounting shared with the serving engine (os3d_api.cu)
bool profiling_enabled();
void add_launch_count(unsigned long long n);

// FP64 bank kernels
cudaError_t launch_fit(const double* d_z, const double* d_w, int npts, int mode, int k,
                       double s_theta, int L, int n_o, int profile, double* d_out,
                       cudaStream_t s);
cudaError_t launch_bank_M(int nz, int ny, int nx, int N, double gamma, double eps,
                          const double* d_c, int L, const double* d_slots, int nslots,
                          int n_o, int mirror, float* Gs, float* GM, float* Minv,
                          cudaStream_t s);

}  // namespace os3d
