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
// never formed: each CTA integrates the N_o-vectors h(w) of 128 frequencies
// through the K steps. The angular propagator exp(dt D44 L) is computed on the
// host in FP64 (closed form through real spherical harmonics) and passed as a
// kernel parameter.
#include <algorithm>
#include <cmath>
#include <vector>
#include "os3d_passes.cuh"

namespace os3d {

namespace {

constexpr double kPiH = 3.141592653589793238462643383279502884;

// Antipodally closed sets (PB > 0). L commutes with the antipodal
// permutation, so with the pairs' first members first E = [[A, B], [B, A]],
// and the spatial factors of n and -n are equal (r_i depends on (w.n_i)^2):
// the Strang steps map s = v_a + v_b by C = A + B and d = v_a - v_b by
// D = A - B independently. With h(t) = E(v) + t O(v) (even and odd parts):
// s_0 = 2 E F, d_0 = 2 t O F, and h^T v = sum over pairs of E s + t O d.
// Rows [0, PB) hold s, rows [PB, 2 PB) hold d (PB the pair count padded to a
// multiple of R), so every warp's rows lie in one block and it reads only
// that block's columns: half the multiply-adds of the full product.
template <int EV>
__device__ __forceinline__ void eval_h_parts(const HEval& h, float t, float& he, float& ho) {
  if constexpr (EV < 2) {
    constexpr int NE = EV == 0 ? 9 : 13;
    constexpr int NO = NE - 1;
    const float v = fmaf(t, t, -0.5f);
    float e = h.e[NE - 1];
#pragma unroll
    for (int k = NE - 2; k >= 0; --k) e = fmaf(e, v, h.e[k]);
    float o = h.o[NO - 1];
#pragma unroll
    for (int k = NO - 2; k >= 0; --k) o = fmaf(o, v, h.o[k]);
    he = e;
    ho = t * o;
  } else {
    const float hp = eval_h<EV>(h, t), hm = eval_h<EV>(h, -t);
    he = 0.5f * (hp + hm);
    ho = 0.5f * (hp - hm);
  }
}

// One CTA per tile of TV = 128 listed frequencies, NP / R warps; NP = the
// orientation count padded to a multiple of R rows per warp (R = 6 or 8),
// or for a closed set 2 PB rows.
// Per Strang step warp w accumulates rows R w .. R w + R - 1 of E V, each
// lane 4 consecutive frequencies: per propagator column j a lane reads its 4
// vector entries with one 16-byte shared load and the R propagator entries,
// the same for the whole warp, as R/2 8-byte shared broadcasts, and issues
// 2R two-lane FMAs over pairs of adjacent rows. The tile is written back in place after a barrier.
// Vectors are stored [orientation][frequency], rows of TV floats.
constexpr int kTV = 128;

template <int NP>
constexpr size_t enhance_smem() {
  return sizeof(float) * ((size_t)NP * NP + 2 * (size_t)NP * kTV + 3 * NP + 5 * kTV) +
         sizeof(int) * 2 * kTV;
}

template <int NP, int R, int EV, int PB = 0>
__global__ void __launch_bounds__(32 * NP / R)
enhance_kernel(const __grid_constant__ EnhanceArgs a) {
  static_assert(R % 2 == 0 && NP % R == 0 && NP % 2 == 0 && NP <= kEStride,
                "R propagator rows per warp, in pairs; NP^2 floats keep V 16-byte aligned");
  static_assert(PB == 0 || (2 * PB == NP && PB % R == 0), "each warp's rows in one block");
  constexpr int NT = 32 * NP / R, TV = kTV;
  extern __shared__ __align__(16) float esm[];
  float* Es = esm;                       // Es[j * NP + i] = E[i][j]
  float* V = Es + NP * NP;               // [i][q]
  float* F = V + NP * TV;                // half-step factors exp(-dt/2 r_i)
  float* nv = F + NP * TV;               // orientations (3 per row)
  float* geo = nv + 3 * NP;              // wx, wy, wz, 1/|w|, |w|^2 per slot
  int* vox = reinterpret_cast<int*>(geo + 5 * TV);
  int* mvox = vox + TV;
  const int t = threadIdx.x;
  const int i0 = R * (t >> 5), q0 = 4 * (t & 31);
  // columns of E this warp reads: [jb, jb + nj) (zero beyond n_o, or beyond
  // the pair count in each block)
  const int np2 = a.n_o / 2;
  const int nj = PB ? (np2 + 1) & ~1 : (a.n_o + 1) & ~1;
  const int jb = (PB && i0 >= PB) ? PB : 0;
  // row i's orientation (paired: its pair's first member), or -1 for padding
  auto orient_of = [&](int i) {
    if constexpr (PB > 0) {
      const int r = i < PB ? i : i - PB;
      return r < np2 ? r : -1;
    } else {
      return i < a.n_o ? i : -1;
    }
  };

  for (int q = t; q < NP * NP; q += NT) Es[q] = a.Et[(q / NP) * kEStride + q % NP];
  for (int q = t; q < 3 * NP; q += NT) {
    const int o = PB ? (q / 3 < np2 ? q / 3 : -1) : (q / 3 < a.n_o ? q / 3 : -1);
    nv[q] = o >= 0 ? a.nvec[o][q % 3] : 0.f;
  }

  const int ntiles = (a.n_in + TV - 1) / TV;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();   // previous tile done with the slot data
    // ---- slots: frequency of every listed index of the tile
    for (int q = t; q < TV; q += NT) {
      const int g = tile * TV + q;
      vox[q] = -1;
      mvox[q] = -1;
      if (g < a.n_in) {
        int lo = 0, hi = a.nseg - 1;   // last segment with first index <= g
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (a.seg[mid].w <= g) lo = mid;
          else hi = mid - 1;
        }
        const int4 sg = a.seg[lo];
        const int kx = sg.z + (g - sg.w);
        const int z = sg.x, y = sg.y, x = kx < 0 ? kx + a.nx : kx;
        vox[q] = (z * a.ny + y) * a.nx + x;
        if (a.mirror) {
          const int mz = z ? a.nz - z : 0, my = y ? a.ny - y : 0, mx = x ? a.nx - x : 0;
          const int m = (mz * a.ny + my) * a.nx + mx;
          if (m != vox[q]) mvox[q] = m;
        }
        const float wz = float(z >= (a.nz + 1) / 2 ? z - a.nz : z) * a.wz;
        const float wy = float(y >= (a.ny + 1) / 2 ? y - a.ny : y) * a.wy;
        const float wx = float(kx) * a.wx;
        const float r2 = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
        geo[q] = wx;
        geo[TV + q] = wy;
        geo[2 * TV + q] = wz;
        geo[3 * TV + q] = r2 > 0.f ? rsqrtf(r2) : 0.f;
        geo[4 * TV + q] = r2;
      }
    }
    __syncthreads();
    // ---- F and the initial vector h F
    for (int p = t; p < NP * TV; p += NT) {
      const int i = p / TV, q = p % TV;
      const int o = orient_of(i);
      float f = 1.f, hv = 0.f;
      if (vox[q] >= 0 && o >= 0) {
        const float tau = fmaf(geo[q], nv[3 * o], fmaf(geo[TV + q], nv[3 * o + 1], geo[2 * TV + q] * nv[3 * o + 2]));
        const float r2 = geo[4 * TV + q];
        f = expf(-a.half_dt * fmaf(a.D11, r2 - tau * tau, a.D33 * tau * tau));
        if constexpr (PB > 0) {   // s_0 = 2 E F, d_0 = 2 t O F
          float he = a.h.c0, ho = 0.f;
          if (r2 > 0.f) eval_h_parts<EV>(a.h, tau * geo[3 * TV + q], he, ho);
          hv = 2.f * (i < PB ? he : ho);
        } else {
          hv = r2 > 0.f ? eval_h<EV>(a.h, tau * geo[3 * TV + q]) : a.h.c0;
        }
      }
      F[i * TV + q] = f;
      V[i * TV + q] = hv * f;
    }
    __syncthreads();
    // ---- K Strang steps: V <- F^2 (E V) (F at the last step)
    for (int s = 0; s < a.steps; ++s) {
      float2 acc[R / 2][4];   // acc[r][c]: rows i0 + 2r, i0 + 2r + 1 at frequency q0 + c
#pragma unroll
      for (int r = 0; r < R / 2; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.f, 0.f);
#pragma unroll 1
      for (int j0 = jb; j0 < jb + nj; j0 += 2) {
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const int j = j0 + jj;
          const float4 v = *reinterpret_cast<const float4*>(V + j * TV + q0);
          const float2 vv[4] = {make_float2(v.x, v.x), make_float2(v.y, v.y),
                                make_float2(v.z, v.z), make_float2(v.w, v.w)};
#pragma unroll
          for (int r = 0; r < R / 2; ++r) {
            const float2 er = *reinterpret_cast<const float2*>(Es + j * NP + i0 + 2 * r);
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = fma2(er, vv[c], acc[r][c]);
          }
        }
      }
      const bool last = s == a.steps - 1;
      __syncthreads();   // every thread has read V
#pragma unroll
      for (int r = 0; r < R / 2; ++r) {
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int off = (i0 + 2 * r + hh) * TV + q0;
          const float4 f = *reinterpret_cast<const float4*>(F + off);
          float2 w01 = make_float2(f.x, f.y), w23 = make_float2(f.z, f.w);
          if (!last) {
            w01 = mul2(w01, w01);
            w23 = mul2(w23, w23);
          }
          const float2 a01 = hh ? make_float2(acc[r][0].y, acc[r][1].y)
                                : make_float2(acc[r][0].x, acc[r][1].x);
          const float2 a23 = hh ? make_float2(acc[r][2].y, acc[r][3].y)
                                : make_float2(acc[r][2].x, acc[r][3].x);
          const float2 p01 = mul2(a01, w01), p23 = mul2(a23, w23);
          *reinterpret_cast<float4*>(V + off) = make_float4(p01.x, p01.y, p23.x, p23.y);
        }
      }
      __syncthreads();
    }
    // ---- m = n^3 h^T V per slot (products in place, then column sums)
    for (int p = t; p < NP * TV; p += NT) {
      const int i = p / TV, q = p % TV;
      const int o = orient_of(i);
      float hv = 0.f;
      if (vox[q] >= 0 && o >= 0) {
        const float tau = fmaf(geo[q], nv[3 * o], fmaf(geo[TV + q], nv[3 * o + 1], geo[2 * TV + q] * nv[3 * o + 2]));
        if constexpr (PB > 0) {   // h^T v = sum E s + t O d
          float he = a.h.c0, ho = 0.f;
          if (geo[4 * TV + q] > 0.f) eval_h_parts<EV>(a.h, tau * geo[3 * TV + q], he, ho);
          hv = i < PB ? he : ho;
        } else {
          hv = geo[4 * TV + q] > 0.f ? eval_h<EV>(a.h, tau * geo[3 * TV + q]) : a.h.c0;
        }
      }
      V[i * TV + q] *= hv;
    }
    __syncthreads();
    for (int q = t; q < TV; q += NT) {
      if (vox[q] < 0) continue;
      float sum = 0.f;
      for (int i = 0; i < (PB ? NP : a.n_o); ++i) sum += V[i * TV + q];
      const float m = sum * a.n3;
      const float2 fh = a.fh[vox[q]];
      a.A[vox[q]] = make_float2(fh.x * m, fh.y * m);
      if (mvox[q] >= 0) {
        const float2 fm = a.fh[mvox[q]];
        a.A[mvox[q]] = make_float2(fm.x * m, fm.y * m);
      }
    }
  }
}

template <int NP, int R, int PB = 0>
cudaError_t launch_np(const EnhanceArgs& a, int ev, cudaStream_t s) {
  constexpr int NT = 32 * NP / R;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  constexpr size_t sm = enhance_smem<NP>();
  auto k = ev == 0 ? enhance_kernel<NP, R, 0, PB>
                    : (ev == 1 ? enhance_kernel<NP, R, 1, PB> : enhance_kernel<NP, R, 2, PB>);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, sm);
  if (e != cudaSuccess) return e;
  const int ntiles = (a.n_in + kTV - 1) / kTV;
  const int grid = std::max(1, std::min(ntiles, nsm * std::max(per_sm, 1)));
  k<<<grid, NT, sm, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

std::vector<int4> ball_segments(int nz, int ny, int nx, bool half, int* n_in) {
  const double pi = kPiH, lim = pi * pi * (1.0 + 1e-12);
  std::vector<int4> seg;
  int total = 0;
  auto sgn = [](int k, int n) { return k >= (n + 1) / 2 ? k - n : k; };
  for (int z = 0; z < nz; ++z) {
    const int kz = sgn(z, nz);
    for (int y = 0; y < ny; ++y) {
      const int ky = sgn(y, ny);
      if (half && (kz < 0 || (kz == 0 && ky < 0))) continue;
      const double wz = 2.0 * pi * kz / nz, wy = 2.0 * pi * ky / ny;
      const double c = wz * wz + wy * wy;
      if (!(c < lim)) continue;
      int amax = (nx - 1) / 2;   // largest positive signed index
      int ar = 0;
      while (ar + 1 <= amax) {
        const double wx = 2.0 * pi * (ar + 1) / nx;
        if (!(wx * wx + c < lim)) break;
        ++ar;
      }
      const bool origin_row = half && kz == 0 && ky == 0;
      const int kx0 = origin_row ? 0 : -ar;
      const int cnt = ar - kx0 + 1;
      seg.push_back(make_int4(z, y, kx0, total));
      total += cnt;
    }
  }
  *n_in = total;
  return seg;
}

namespace {

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

int enhance_pair_block(int n_o) {
  for (int pb : {4, 6, 12, 24, 36})
    if (n_o / 2 <= pb) return pb;
  return -1;
}

cudaError_t launch_enhance(const EnhanceArgs& a, int ev, cudaStream_t s) {
  const int n = a.n_o;
  if (a.paired) {   // (2 PB rows, rows per warp, PB)
    switch (enhance_pair_block(n)) {
      case 4: return launch_np<8, 4, 4>(a, ev, s);
      case 6: return launch_np<12, 6, 6>(a, ev, s);
      case 12: return launch_np<24, 6, 12>(a, ev, s);
      case 24: return launch_np<48, 6, 24>(a, ev, s);
      case 36: return launch_np<72, 6, 36>(a, ev, s);
      default: return cudaErrorInvalidValue;
    }
  }
  // (rows, rows per warp): no padding for the 12- and 42-orientation sets
  if (n <= 8) return launch_np<8, 8>(a, ev, s);
  if (n <= 12) return launch_np<12, 6>(a, ev, s);
  if (n <= 24) return launch_np<24, 8>(a, ev, s);
  if (n <= 42) return launch_np<42, 6>(a, ev, s);
  if (n <= 48) return launch_np<48, 8>(a, ev, s);
  if (n <= kMaxOrientE) return launch_np<kEStride, 8>(a, ev, s);
  return cudaErrorInvalidValue;
}

}  // namespace os3d
