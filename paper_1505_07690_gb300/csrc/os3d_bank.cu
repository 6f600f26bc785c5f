// FP64 kernels of the wavelet bank (sm_103a): the zonal spherical-harmonic
// fit of the orientation distribution (Sec. 3.2) and the stability function
// M_psi (Sec. 2.1) with its clamped inverse (Sec. 3.1). Both run once per
// bank; FP64 is used here because the normal equations of the fit and the
// division by M are where single precision would lose digits.
#include "os3d_kernels.cuh"

namespace os3d {

namespace {

constexpr double kPiD = 3.141592653589793238462643383279502884;
constexpr int kFitThreads = 256;
constexpr int kFitChunk = 128;
constexpr int kMaxSpline = 8;

// Centred cardinal B-spline B^k(x) by the two-term recurrence
//   B^m(y) = [ (y + (m+1)/2) B^{m-1}(y + 1/2) + ((m+1)/2 - y) B^{m-1}(y - 1/2) ] / m
// starting from the indicator B^0 of (-1/2, 1/2) (Sec. 3.1).
__device__ double bspline_dev(double x, int k) {
  double b[kMaxSpline + 1];
  // level 0 at offsets k/2 - i, i = 0..k
  for (int i = 0; i <= k; ++i) {
    const double y = x + 0.5 * k - i;
    b[i] = (y > -0.5 && y < 0.5) ? 1.0 : 0.0;
  }
  for (int m = 1; m <= k; ++m) {
    for (int i = 0; i <= k - m; ++i) {
      const double y = x + 0.5 * (k - m) - i;
      b[i] = ((y + 0.5 * (m + 1)) * b[i] + (0.5 * (m + 1) - y) * b[i + 1]) / m;
    }
  }
  return b[0];
}

// One CTA. out[0..L] = b (Legendre coefficients of A), out[L+1..2L+1] = c
// (Funk + anti-symmetrised, normalised).
//  mode 1: least squares sum_p (A(theta_p) - sum_l b_l P_l(z_p))^2 on the given
//          sphere samples (the paper's pseudo-inverse, restricted to m = 0);
//  mode 0: projection b_l = (2l+1)/2 sum_p w_p A(theta_p) P_l(z_p).
__global__ void __launch_bounds__(kFitThreads)
fit_kernel(const double* __restrict__ zt, const double* __restrict__ wt, int npts, int mode,
           int k, double s_theta, int L, int n_o, int profile, double* __restrict__ out) {
  __shared__ double P[kFitChunk][kMaxL + 2];
  __shared__ double Gm[(kMaxL + 1) * (kMaxL + 1)];
  __shared__ double rv[kMaxL + 1];
  const int nl = L + 1;
  const int ne = (mode == 1 ? nl * nl : 0) + nl;
  constexpr int kMaxPer = ((kMaxL + 1) * (kMaxL + 2) + kFitThreads - 1) / kFitThreads;
  double acc[kMaxPer];
  for (int i = 0; i < kMaxPer; ++i) acc[i] = 0.0;

  for (int base = 0; base < npts; base += kFitChunk) {
    const int p = threadIdx.x;
    if (p < kFitChunk) {
      if (base + p < npts) {
        const double z = zt[2 * (base + p)];
        const double th = zt[2 * (base + p) + 1];
        double pm = 1.0, pl = z;
        P[p][0] = 1.0;
        if (L >= 1) P[p][1] = z;
        for (int l = 1; l < L; ++l) {
          const double pn = ((2 * l + 1) * z * pl - l * pm) / (l + 1);
          pm = pl;
          pl = pn;
          P[p][l + 1] = pn;
        }
        P[p][kMaxL + 1] = wt[base + p] * bspline_dev(th / s_theta, k);
      } else {
        for (int l = 0; l <= L; ++l) P[p][l] = 0.0;
        P[p][kMaxL + 1] = 0.0;
      }
    }
    __syncthreads();
    const int cnt = min(kFitChunk, npts - base);
    for (int i = 0; i < kMaxPer; ++i) {
      const int e = threadIdx.x + kFitThreads * i;
      if (e >= ne) break;
      double s = 0.0;
      if (mode == 1 && e < nl * nl) {
        const int l = e / nl, m = e % nl;
        for (int q = 0; q < cnt; ++q) s += P[q][l] * P[q][m];
      } else {
        const int l = e - (mode == 1 ? nl * nl : 0);
        for (int q = 0; q < cnt; ++q) s += P[q][l] * P[q][kMaxL + 1];
      }
      acc[i] += s;
    }
    __syncthreads();
  }
  for (int i = 0; i < kMaxPer; ++i) {
    const int e = threadIdx.x + kFitThreads * i;
    if (e >= ne) break;
    if (mode == 1 && e < nl * nl) Gm[e] = acc[i];
    else rv[e - (mode == 1 ? nl * nl : 0)] = acc[i];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;

  double b[kMaxL + 1];
  if (mode == 0) {
    for (int l = 0; l <= L; ++l) b[l] = 0.5 * (2 * l + 1) * rv[l];
  } else {
    // Cholesky G = R^T R (in place, upper part), then two triangular solves
    for (int j = 0; j < nl; ++j) {
      double d = Gm[j * nl + j];
      for (int q = 0; q < j; ++q) d -= Gm[q * nl + j] * Gm[q * nl + j];
      d = sqrt(d);
      Gm[j * nl + j] = d;
      for (int i = j + 1; i < nl; ++i) {
        double s = Gm[j * nl + i];
        for (int q = 0; q < j; ++q) s -= Gm[q * nl + j] * Gm[q * nl + i];
        Gm[j * nl + i] = s / d;
      }
    }
    double y[kMaxL + 1];
    for (int i = 0; i < nl; ++i) {
      double s = rv[i];
      for (int q = 0; q < i; ++q) s -= Gm[q * nl + i] * y[q];
      y[i] = s / Gm[i * nl + i];
    }
    for (int i = nl - 1; i >= 0; --i) {
      double s = y[i];
      for (int q = i + 1; q < nl; ++q) s -= Gm[i * nl + q] * b[q];
      b[i] = s / Gm[i * nl + i];
    }
  }
  // cake wavelet (profile 0): Funk transform c^e_l = 2 pi P_l(0) b_l and
  // anti-symmetrisation c^o_l = (1 - (-1)^l) b_l (Sec. 3.2); plate detector
  // (profile 1): h = A, c_l = b_l (Sec. 3.1). Then kappa (M averages to one).
  double c[kMaxL + 1];
  double p0 = 1.0;   // P_l(0): P_{l+2}(0) = -(l+1)/(l+2) P_l(0)
  for (int l = 0; l <= L; ++l) {
    if (profile == 1) {
      c[l] = b[l];
    } else if (l % 2 == 0) {
      c[l] = 2.0 * kPiD * p0 * b[l];
      p0 = -p0 * (l + 1) / (l + 2);
    } else {
      c[l] = 2.0 * b[l];
    }
  }
  double ss = 0.0;
  for (int l = 0; l <= L; ++l) ss += c[l] * c[l] / (2 * l + 1);
  const double kappa = 1.0 / sqrt(n_o * ss);
  for (int l = 0; l <= L; ++l) {
    out[l] = b[l];
    out[nl + l] = kappa * c[l];
  }
}

// M(w) = G(|w|)^2 sum_i h(w_hat . n_i)^2 in FP64, with h = sum_l c_l P_l.
// A slot is an orientation a, optionally with its antipode b = -a; for the
// pair h(t)^2 + h(-t)^2 = 2 (h_even^2 + h_odd^2).
// Outputs (float): Gs = G / n^3, GM = G / (n^3 max(M, eps)), Minv = 1/max(M, eps)
// (all zero outside the ball |w| < pi). With `mirror` (every slot a pair, so
// M(-w) = M(w)) only the planes iz <= nz/2 are computed and each value is
// written at w and at -w; the recurrence gives h_even(-t) = h_even(t) and
// h_odd(-t) = -h_odd(t) exactly, so a voxel reached from both sides gets the
// same bits.
__global__ void __launch_bounds__(256)
bank_M_kernel(int nz, int ny, int nx, int N, double tscale, double eps,
              const double* __restrict__ cg, int L, const double* __restrict__ slots,
              int nslots, int n_o, int mirror, float* Gs, float* GM, float* Minv) {
  __shared__ double c[kMaxL + 1], al[kMaxL + 1], be[kMaxL + 1];
  __shared__ double sl[4 * 256];
  if (threadIdx.x <= L) {
    c[threadIdx.x] = cg[threadIdx.x];
    const int l = threadIdx.x;
    al[l] = double(2 * l + 1) / double(l + 1);
    be[l] = double(l) / double(l + 1);
  }
  const long long nvox = (long long)nz * ny * nx;
  const long long nwork = mirror ? (long long)(nz / 2 + 1) * ny * nx : nvox;
  const double inv_n = 1.0 / double(nvox);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v0 = (long long)blockIdx.x * blockDim.x; v0 < nwork; v0 += stride) {
    const long long v = v0 + threadIdx.x;
    double M = 0.0, g = 0.0;
    bool inside = false;
    double wh[3] = {0.0, 0.0, 0.0};
    bool dc = false;
    long long mv = -1;   // the voxel of -w, when it is written from here too
    if (v < nwork) {
      const int ix = int(v % nx), iy = int((v / nx) % ny), iz = int(v / ((long long)nx * ny));
      if (mirror) {
        const long long m = ((long long)(iz ? nz - iz : 0) * ny + (iy ? ny - iy : 0)) * nx +
                            (ix ? nx - ix : 0);
        if (m != v) mv = m;
      }
      const int kx = ix >= (nx + 1) / 2 ? ix - nx : ix;
      const int ky = iy >= (ny + 1) / 2 ? iy - ny : iy;
      const int kz = iz >= (nz + 1) / 2 ? iz - nz : iz;
      const double wx = 2.0 * kPiD * kx / nx, wy = 2.0 * kPiD * ky / ny, wz = 2.0 * kPiD * kz / nz;
      const double r2 = wx * wx + wy * wy + wz * wz;
      inside = r2 < kPiD * kPiD;
      if (inside) {
        const double xg = r2 / tscale;
        double s = 1.0, term = 1.0;
        for (int q = 1; q <= N; ++q) {
          term *= xg / q;
          s += term;
        }
        g = exp(-xg) * s;
        dc = r2 == 0.0;
        if (!dc) {
          const double ri = 1.0 / sqrt(r2);
          wh[0] = wx * ri;
          wh[1] = wy * ri;
          wh[2] = wz * ri;
        }
      }
    }
    // slot loop in chunks staged through shared memory
    for (int sb = 0; sb < nslots; sb += 256) {
      __syncthreads();
      const int cnt = min(256, nslots - sb);
      if (threadIdx.x < cnt)
        for (int q = 0; q < 4; ++q) sl[4 * threadIdx.x + q] = slots[4 * (sb + threadIdx.x) + q];
      __syncthreads();
      if (inside && !dc) {
        for (int s = 0; s < cnt; ++s) {
          const double t = wh[0] * sl[4 * s] + wh[1] * sl[4 * s + 1] + wh[2] * sl[4 * s + 2];
          double pm = 1.0, pl = t, he = c[0], ho = (L >= 1) ? c[1] * t : 0.0;
          for (int l = 1; l < L; ++l) {
            const double pn = al[l] * t * pl - be[l] * pm;
            pm = pl;
            pl = pn;
            if ((l + 1) & 1) ho += c[l + 1] * pn;
            else he += c[l + 1] * pn;
          }
          if (sl[4 * s + 3] != 0.0) M += 2.0 * (he * he + ho * ho);
          else M += (he + ho) * (he + ho);
        }
      }
    }
    if (v < nwork) {
      float gs = 0.f, gm = 0.f, mi = 0.f;
      if (inside) {
        if (dc) M = double(n_o) * c[0] * c[0];
        M *= g * g;
        const double inv = 1.0 / fmax(M, eps);
        gs = float(g * inv_n);
        gm = float(g * inv_n * inv);
        mi = float(inv);
      }
      Gs[v] = gs;
      GM[v] = gm;
      Minv[v] = mi;
      if (mv >= 0) {
        Gs[mv] = gs;
        GM[mv] = gm;
        Minv[mv] = mi;
      }
    }
  }
}

}  // namespace

cudaError_t launch_fit(const double* d_zt, const double* d_w, int npts, int mode, int k,
                       double s_theta, int L, int n_o, int profile, double* d_out,
                       cudaStream_t s) {
  fit_kernel<<<1, kFitThreads, 0, s>>>(d_zt, d_w, npts, mode, k, s_theta, L, n_o, profile, d_out);
  return cudaGetLastError();
}

cudaError_t launch_bank_M(int nz, int ny, int nx, int N, double gamma, double eps,
                          const double* d_c, int L, const double* d_slots, int nslots,
                          int n_o, int mirror, float* Gs, float* GM, float* Minv, cudaStream_t s) {
  const double tscale = 2.0 * (gamma * kPiD) * (gamma * kPiD) / (1.0 + 2.0 * N);
  const long long nvox = (long long)nz * ny * nx;
  long long blocks = (nvox + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  bank_M_kernel<<<(int)blocks, 256, 0, s>>>(nz, ny, nx, N, tscale, eps, d_c, L, d_slots, nslots,
                                            n_o, mirror, Gs, GM, Minv);
  return cudaGetLastError();
}

}  // namespace os3d
