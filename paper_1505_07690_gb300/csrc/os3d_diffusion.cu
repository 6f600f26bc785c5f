// Linear left-invariant diffusion on R^3 x| S^2 (Sec. 4.1 with a constant
// diagonal D_ij) inside Upsilon f = W^{*,ext} Phi_t W f (sm_103a).
//
// All three operators are linear and commute with translations, so in the
// Fourier domain of x the whole cascade acts on f_hat(w) through one real
// number per frequency:
//   m(w) = G(w)^2 h(w)^T E(w) h(w) / max(M(w), eps),  h_i(w) = h(w_hat . n_i),
// where E(w) is the Strang product of K steps
//   diag(exp(-dt/2 r_i(w)))  exp(dt D44 L)  diag(exp(-dt/2 r_i(w))),
// r_i(w) = D11 (|w|^2 - (w.n_i)^2) + D33 (w.n_i)^2 the symbol of the spatial
// generators for orientation n_i, and L the discrete Laplace-Beltrami operator
// on the orientation set (the angular generators A4^2 + A5^2). The score is
// never formed: one thread integrates the N_o-vector h(w) of its frequency
// through the K steps. The angular propagator exp(dt D44 L) is computed on the
// host in FP64 (closed form through real spherical harmonics) and passed as a
// kernel parameter.
#include <algorithm>
#include <cmath>
#include <vector>
#include "os3d_passes.cuh"

namespace os3d {

namespace {

constexpr int kEThreads = 128;
constexpr double kPiH = 3.141592653589793238462643383279502884;

// One thread per frequency voxel; NP = padded orientation count (multiple of 4).
template <int NP>
constexpr size_t enhance_smem() {
  return sizeof(float) * ((size_t)NP * NP + (size_t)NP * kEThreads + 3 * NP);
}

template <int NP, int EV>
__global__ void __launch_bounds__(kEThreads)
enhance_kernel(const __grid_constant__ EnhanceArgs a) {
  extern __shared__ __align__(16) float esm[];
  float* Et = esm;                                   // Et[j * NP + i] = E[i][j]
  float (*col)[kEThreads] = reinterpret_cast<float (*)[kEThreads]>(esm + NP * NP);
  float (*nv)[3] = reinterpret_cast<float (*)[3]>(esm + NP * NP + NP * kEThreads);
  const int t = threadIdx.x;
  for (int q = t; q < NP * NP; q += kEThreads) {
    const int j = q / NP, i = q % NP;
    Et[q] = (i < a.n_o && j < a.n_o) ? a.E[i * kMaxOrientE + j] : 0.f;
  }
  for (int q = t; q < NP * 3; q += kEThreads)
    nv[q / 3][q % 3] = (q / 3 < a.n_o) ? a.nvec[q / 3][q % 3] : 0.f;
  __syncthreads();

  const long long nvox = (long long)a.nz * a.ny * a.nx;
  const float pi2 = 9.869604401089358f;
  for (long long v = (long long)blockIdx.x * kEThreads + t; v < nvox;
       v += (long long)gridDim.x * kEThreads) {
    const int ix = int(v % a.nx), iy = int((v / a.nx) % a.ny), iz = int(v / ((long long)a.nx * a.ny));
    const float wx = float(ix >= (a.nx + 1) / 2 ? ix - a.nx : ix) * a.wx;
    const float wy = float(iy >= (a.ny + 1) / 2 ? iy - a.ny : iy) * a.wy;
    const float wz = float(iz >= (a.nz + 1) / 2 ? iz - a.nz : iz) * a.wz;
    const float r2 = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
    if (r2 >= pi2) {
      a.A[v] = make_float2(0.f, 0.f);
      continue;
    }
    const float ri = r2 > 0.f ? rsqrtf(r2) : 0.f;
    float F[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const float tau = fmaf(wx, nv[i][0], fmaf(wy, nv[i][1], wz * nv[i][2]));
      const float rate = fmaf(a.D11, r2 - tau * tau, a.D33 * tau * tau);
      F[i] = expf(-a.half_dt * rate);
      float hv = 0.f;
      if (i < a.n_o) hv = r2 > 0.f ? eval_h<EV>(a.h, tau * ri) : a.h.c0;
      col[i][t] = hv * F[i];
    }
    for (int s = 0; s < a.steps; ++s) {
      float acc[NP];
#pragma unroll
      for (int i = 0; i < NP; ++i) acc[i] = 0.f;
#pragma unroll 2
      for (int j = 0; j < NP; ++j) {
        const float vj = col[j][t];
        const float4* row = reinterpret_cast<const float4*>(Et + j * NP);
#pragma unroll
        for (int i4 = 0; i4 < NP / 4; ++i4) {
          const float4 e = row[i4];
          acc[4 * i4 + 0] = fmaf(e.x, vj, acc[4 * i4 + 0]);
          acc[4 * i4 + 1] = fmaf(e.y, vj, acc[4 * i4 + 1]);
          acc[4 * i4 + 2] = fmaf(e.z, vj, acc[4 * i4 + 2]);
          acc[4 * i4 + 3] = fmaf(e.w, vj, acc[4 * i4 + 3]);
        }
      }
      const bool last = s == a.steps - 1;
#pragma unroll
      for (int i = 0; i < NP; ++i) col[i][t] = acc[i] * (last ? F[i] : F[i] * F[i]);
    }
    float sum = 0.f;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      if (i < a.n_o) {
        const float tau = fmaf(wx, nv[i][0], fmaf(wy, nv[i][1], wz * nv[i][2]));
        const float hv = r2 > 0.f ? eval_h<EV>(a.h, tau * ri) : a.h.c0;
        sum = fmaf(hv, col[i][t], sum);
      }
    }
    const float2 fh = a.fh[v];
    const float m = sum * a.n3;
    a.A[v] = make_float2(fh.x * m, fh.y * m);
  }
}

template <int NP>
cudaError_t launch_np(const EnhanceArgs& a, int ev, cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long nvox = (long long)a.nz * a.ny * a.nx;
  const long long need = (nvox + kEThreads - 1) / kEThreads;
  const int grid = (int)std::max(1LL, std::min(need, (long long)nsm * 8));
  constexpr size_t sm = enhance_smem<NP>();
  auto k = ev == 0 ? enhance_kernel<NP, 0> : (ev == 1 ? enhance_kernel<NP, 1> : enhance_kernel<NP, 2>);
  const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k<<<grid, kEThreads, sm, s>>>(a);
  return cudaGetLastError();
}

// ---- host: discrete Laplace-Beltrami propagator (FP64) --------------------
// Orthonormal real spherical harmonics up to degree l at the unit vectors:
// N_lm P_l^|m|(z) cos(m phi) / sin(|m| phi), N_lm^2 = (2 - delta_m0)
// (2l+1)/(4 pi) (l-|m|)!/(l+|m|)!. (Any basis of the degree-l spaces gives the
// same operator; unit norms on the sphere make a harmonic that vanishes on the
// orientation set show up as a near-zero Gram pivot.)
void real_sh(int lmax, const double* V, int n, std::vector<double>& Y, std::vector<int>& deg) {
  const int nb = (lmax + 1) * (lmax + 1);
  Y.assign((size_t)n * nb, 0.0);
  deg.assign(nb, 0);
  int c = 0;
  for (int l = 0; l <= lmax; ++l)
    for (int m = -l; m <= l; ++m) deg[c++] = l;
  for (int p = 0; p < n; ++p) {
    const double x = V[3 * p], y = V[3 * p + 1], z = std::max(-1.0, std::min(1.0, V[3 * p + 2]));
    const double ph = std::atan2(y, x), sn = std::sqrt(std::max(0.0, 1.0 - z * z));
    // P[l][m], m <= l, by the standard recurrences
    std::vector<double> P((size_t)(lmax + 1) * (lmax + 1), 0.0);
    auto at = [&](int l, int m) -> double& { return P[(size_t)l * (lmax + 1) + m]; };
    at(0, 0) = 1.0;
    for (int m = 1; m <= lmax; ++m) at(m, m) = -(2.0 * m - 1.0) * sn * at(m - 1, m - 1);
    for (int m = 0; m < lmax; ++m) at(m + 1, m) = (2.0 * m + 1.0) * z * at(m, m);
    for (int m = 0; m <= lmax; ++m)
      for (int l = m + 2; l <= lmax; ++l)
        at(l, m) = ((2.0 * l - 1.0) * z * at(l - 1, m) - (l + m - 1.0) * at(l - 2, m)) / (l - m);
    int q = 0;
    for (int l = 0; l <= lmax; ++l)
      for (int m = -l; m <= l; ++m, ++q) {
        const int am = m < 0 ? -m : m;
        double ratio = 1.0;   // (l - |m|)! / (l + |m|)!
        for (int k = l - am + 1; k <= l + am; ++k) ratio /= k;
        const double nrm = std::sqrt((m == 0 ? 1.0 : 2.0) * (2 * l + 1) / (4.0 * kPiH) * ratio);
        Y[(size_t)p * nb + q] =
            nrm * at(l, am) * (m < 0 ? std::sin(am * ph) : std::cos(am * ph));
      }
  }
}

// Cholesky of the Gram matrix Y^T Y; false when a pivot falls below 1e-12 of
// the largest diagonal entry (harmonics that are dependent on the set).
bool gram_cholesky(const std::vector<double>& Y, int n, int nb, std::vector<double>& Yn,
                   std::vector<double>& R) {
  Yn = Y;
  R.assign((size_t)nb * nb, 0.0);
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j) {
      double s = 0.0;
      for (int p = 0; p < n; ++p) s += Yn[(size_t)p * nb + i] * Yn[(size_t)p * nb + j];
      R[(size_t)i * nb + j] = s;
    }
  double dmax = 0.0;
  for (int j = 0; j < nb; ++j) dmax = std::max(dmax, R[(size_t)j * nb + j]);
  for (int j = 0; j < nb; ++j) {   // in place, upper factor
    double d = R[(size_t)j * nb + j];
    for (int q = 0; q < j; ++q) d -= R[(size_t)q * nb + j] * R[(size_t)q * nb + j];
    if (!(d > 1e-12 * dmax)) return false;
    d = std::sqrt(d);
    R[(size_t)j * nb + j] = d;
    for (int i = j + 1; i < nb; ++i) {
      double s = R[(size_t)j * nb + i];
      for (int q = 0; q < j; ++q) s -= R[(size_t)q * nb + j] * R[(size_t)q * nb + i];
      R[(size_t)j * nb + i] = s / d;
    }
  }
  return true;
}

}  // namespace

// exp(tau L) = I + Y (exp(tau Lambda) - I) (Y^T Y)^-1 Y^T for the discrete
// Laplace-Beltrami operator L = Y Lambda Y^+ (Lambda = -l(l+1) per degree);
// exact because Y^+ Y = I. Degree: `sh_degree`, or if 0 the largest l with
// (l+1)^2 <= n whose harmonics are independent on the set. Returns the degree
// used, or -1 if that basis is dependent.
int angular_propagator(const double* V, int n, int sh_degree, double tau, std::vector<double>& E) {
  int l = sh_degree;
  const bool automatic = l <= 0;
  if (automatic) {
    l = 0;
    while ((l + 2) * (l + 2) <= n) ++l;
  }
  std::vector<double> Y, Yn, R;
  std::vector<int> deg;
  for (;; --l) {
    real_sh(l, V, n, Y, deg);
    const int nb = (l + 1) * (l + 1);
    if (nb <= n && gram_cholesky(Y, n, nb, Yn, R)) break;
    if (!automatic || l == 0) return -1;
  }
  const int nb = (l + 1) * (l + 1);
  // B = (Y^T Y)^-1 Y^T (nb x n) by two triangular solves per column
  std::vector<double> B((size_t)nb * n);
  std::vector<double> y(nb);
  for (int p = 0; p < n; ++p) {
    for (int i = 0; i < nb; ++i) {   // R^T y = Yn[p, :]
      double s = Yn[(size_t)p * nb + i];
      for (int q = 0; q < i; ++q) s -= R[(size_t)q * nb + i] * y[q];
      y[i] = s / R[(size_t)i * nb + i];
    }
    for (int i = nb - 1; i >= 0; --i) {   // R x = y
      double s = y[i];
      for (int q = i + 1; q < nb; ++q) s -= R[(size_t)i * nb + q] * y[q];
      y[i] = s / R[(size_t)i * nb + i];
    }
    for (int i = 0; i < nb; ++i) B[(size_t)i * n + p] = y[i];
  }
  E.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    E[(size_t)i * n + i] = 1.0;
    for (int q = 0; q < nb; ++q) {
      const double g = std::expm1(-tau * deg[q] * (deg[q] + 1.0)) * Yn[(size_t)i * nb + q];
      if (g == 0.0) continue;
      for (int j = 0; j < n; ++j) E[(size_t)i * n + j] += g * B[(size_t)q * n + j];
    }
  }
  return l;
}

cudaError_t launch_enhance(const EnhanceArgs& a, int ev, cudaStream_t s) {
  const int n = a.n_o;
  if (n <= 8) return launch_np<8>(a, ev, s);
  if (n <= 12) return launch_np<12>(a, ev, s);
  if (n <= 20) return launch_np<20>(a, ev, s);
  if (n <= 44) return launch_np<44>(a, ev, s);
  if (n <= kMaxOrientE) return launch_np<kMaxOrientE>(a, ev, s);
  return cudaErrorInvalidValue;
}

}  // namespace os3d
