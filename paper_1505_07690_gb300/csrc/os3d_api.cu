// C-ABI of the orientation-score library: argument checks, host-side FP64
// geometry (orientation sets, tessellation, quadrature, Chebyshev form of the
// angular profile), bank construction and the launch sequence of the
// forward, inverse and adjoint transforms.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <array>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/os3d.h"
#include "os3d_kernels.cuh"

namespace os3d {
// per-size launchers (os3d_sizes_*.cu)
#define OS3D_DECL_Z(N) \
  cudaError_t launch_z_##N(int, int, const PassArgs&, int, cudaStream_t);
#define OS3D_DECL_XY(NY, NX) \
  cudaError_t launch_xy_##NY##_##NX(int, int, const PassArgs&, cudaStream_t);
OS3D_DECL_Z(16) OS3D_DECL_Z(32) OS3D_DECL_Z(48) OS3D_DECL_Z(64) OS3D_DECL_Z(96)
OS3D_DECL_Z(128) OS3D_DECL_Z(160) OS3D_DECL_Z(256)
OS3D_DECL_XY(16, 16) OS3D_DECL_XY(32, 32) OS3D_DECL_XY(48, 48) OS3D_DECL_XY(64, 64)
OS3D_DECL_XY(96, 96) OS3D_DECL_XY(128, 128) OS3D_DECL_XY(256, 256) OS3D_DECL_XY(128, 160)
#define OS3D_DECL_PN(N)                                                                   \
  cudaError_t launch_pencil_##N(int, int, int, const PassArgs&, const PencilGeom&, long long, \
                                int, cudaStream_t);
OS3D_DECL_PN(16) OS3D_DECL_PN(32) OS3D_DECL_PN(48) OS3D_DECL_PN(64) OS3D_DECL_PN(96)
OS3D_DECL_PN(128) OS3D_DECL_PN(160) OS3D_DECL_PN(256)

cudaError_t launch_pencil(int n, int mode, int dir, int ub, const PassArgs& a, const PencilGeom& g,
                          long long nlines, int nslots, cudaStream_t s) {
  switch (n) {
    case 16: return launch_pencil_16(mode, dir, ub, a, g, nlines, nslots, s);
    case 32: return launch_pencil_32(mode, dir, ub, a, g, nlines, nslots, s);
    case 48: return launch_pencil_48(mode, dir, ub, a, g, nlines, nslots, s);
    case 64: return launch_pencil_64(mode, dir, ub, a, g, nlines, nslots, s);
    case 96: return launch_pencil_96(mode, dir, ub, a, g, nlines, nslots, s);
    case 128: return launch_pencil_128(mode, dir, ub, a, g, nlines, nslots, s);
    case 160: return launch_pencil_160(mode, dir, ub, a, g, nlines, nslots, s);
    case 256: return launch_pencil_256(mode, dir, ub, a, g, nlines, nslots, s);
    default: return cudaErrorInvalidValue;
  }
}

bool z_supported(int nz) {
  return nz == 16 || nz == 32 || nz == 48 || nz == 64 || nz == 96 || nz == 128 || nz == 160 ||
         nz == 256;
}
bool xy_supported(int ny, int nx) {
  return (ny == nx &&
          (nx == 16 || nx == 32 || nx == 48 || nx == 64 || nx == 96 || nx == 128 || nx == 256)) ||
         (ny == 128 && nx == 160);
}
// planes the fused score-domain plane pass holds (every plane of the plane pass)
bool soft_plane_supported(int ny, int nx) { return xy_supported(ny, nx); }
// CTAs per plane of the plane passes (the kernels' XYSplit)
int plane_ctas(int ny, int nx) { return (ny == 256 && nx == 256) ? 8 : 1; }
cudaError_t launch_z(int nz, int mode, int ev, const PassArgs& a, int tiles, cudaStream_t s) {
  switch (nz) {
    case 16: return launch_z_16(mode, ev, a, tiles, s);
    case 32: return launch_z_32(mode, ev, a, tiles, s);
    case 48: return launch_z_48(mode, ev, a, tiles, s);
    case 64: return launch_z_64(mode, ev, a, tiles, s);
    case 96: return launch_z_96(mode, ev, a, tiles, s);
    case 128: return launch_z_128(mode, ev, a, tiles, s);
    case 160: return launch_z_160(mode, ev, a, tiles, s);
    case 256: return launch_z_256(mode, ev, a, tiles, s);
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t launch_xy(int ny, int nx, int mode, int ub, const PassArgs& a, cudaStream_t s) {
  if (ny == 128 && nx == 160) return launch_xy_128_160(mode, ub, a, s);
  if (ny != nx) return cudaErrorInvalidValue;
  switch (nx) {
    case 16: return launch_xy_16_16(mode, ub, a, s);
    case 32: return launch_xy_32_32(mode, ub, a, s);
    case 48: return launch_xy_48_48(mode, ub, a, s);
    case 64: return launch_xy_64_64(mode, ub, a, s);
    case 96: return launch_xy_96_96(mode, ub, a, s);
    case 128: return launch_xy_128_128(mode, ub, a, s);
    case 256: return launch_xy_256_256(mode, ub, a, s);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace os3d

using namespace os3d;

struct os3d_bank {
  int dev = 0;
  int dims[3] = {0, 0, 0};
  long long nvox = 0;
  int n_o = 0;
  os3d_params p{};
  std::vector<double> orient;          // n_o x 3
  std::vector<int> slot_a, slot_b;     // orientation pairs (b = -1: unpaired)
  int block_slots = 1;
  std::vector<double> b, c;            // Legendre coefficients (L+1 each)
  HEval h{};
  int ev = 0;                          // wavelet evaluation form (see HEval)
  float* Gs = nullptr;                 // G / n^3
  float* GM = nullptr;                 // G / (n^3 max(M, eps))
  float* Minv = nullptr;               // 1 / max(M, eps), 0 outside the ball
  int4* seg = nullptr;                 // frequencies inside the ball, as row segments
  unsigned* err = nullptr;             // device counter of bounded waits that ran out
  int nseg = 0, n_in = 0;              // (half of them when every orientation is paired)
  int mirror = 0;
  mutable void* ws = nullptr;          // default workspace, allocated by the first call
                                       // that passes no workspace of its own
  mutable std::mutex ws_mu;
  // the tensor-core diffusion's propagator in the kernel's layout, for the
  // last (dt D44, degree) it was computed for
  mutable std::mutex tc_mu;
  mutable double tc_tau = -1.0;
  mutable int tc_degree = -1;
  mutable float tc_inv_se = 1.f;
  mutable std::vector<unsigned char> tc_prep;
  cudaStream_t side[2] = {nullptr, nullptr};   // consecutive blocks alternate between these
  cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
  size_t ws_bytes = 0;
};

namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

// ---------------------------------------------------------------------------
// host geometry (FP64)
// ---------------------------------------------------------------------------
using V3 = std::array<double, 3>;

V3 normed(const V3& a) {
  const double n = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  return {a[0] / n, a[1] / n, a[2] / n};
}

void icosahedron(std::vector<V3>& V, std::vector<std::array<int, 3>>& F) {
  const double phi = (1.0 + std::sqrt(5.0)) / 2.0;
  V.clear();
  for (double s1 : {1.0, -1.0})
    for (double s2 : {1.0, -1.0}) {
      const V3 a = {0.0, s1, s2 * phi};
      V.push_back(normed(a));
      V.push_back(normed({a[1], a[2], a[0]}));
      V.push_back(normed({a[2], a[0], a[1]}));
    }
  // faces: triples of mutually nearest vertices
  const int n = (int)V.size();
  auto d2 = [&](int i, int j) {
    double s = 0;
    for (int q = 0; q < 3; ++q) s += (V[i][q] - V[j][q]) * (V[i][q] - V[j][q]);
    return s;
  };
  double emin = 1e9;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) emin = std::min(emin, d2(i, j));
  auto adj = [&](int i, int j) { return std::fabs(d2(i, j) - emin) < 1e-9; };
  F.clear();
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      for (int k = j + 1; k < n; ++k)
        if (adj(i, j) && adj(j, k) && adj(i, k)) F.push_back({i, j, k});
}

void octahedron(std::vector<V3>& V, std::vector<std::array<int, 3>>& F) {
  V = {{1.0, 0.0, 0.0}, {-1.0, 0.0, 0.0}, {0.0, 1.0, 0.0},
       {0.0, -1.0, 0.0}, {0.0, 0.0, 1.0}, {0.0, 0.0, -1.0}};
  F.clear();
  for (int a = 0; a < 2; ++a)
    for (int b = 2; b < 4; ++b)
      for (int c = 4; c < 6; ++c) F.push_back({a, b, c});   // one face per octant
}

void subdivide(std::vector<V3>& V, std::vector<std::array<int, 3>>& F) {
  std::map<std::pair<int, int>, int> mid;
  auto m = [&](int a, int b) {
    const auto key = std::make_pair(std::min(a, b), std::max(a, b));
    auto it = mid.find(key);
    if (it != mid.end()) return it->second;
    V.push_back(normed({V[a][0] + V[b][0], V[a][1] + V[b][1], V[a][2] + V[b][2]}));
    mid[key] = (int)V.size() - 1;
    return (int)V.size() - 1;
  };
  std::vector<std::array<int, 3>> F2;
  for (const auto& f : F) {
    const int ab = m(f[0], f[1]), bc = m(f[1], f[2]), ca = m(f[2], f[0]);
    F2.push_back({f[0], ab, ca});
    F2.push_back({ab, f[1], bc});
    F2.push_back({ca, bc, f[2]});
    F2.push_back({ab, bc, ca});
  }
  F.swap(F2);
}

// canonical order: representatives by decreasing z then azimuth, then antipodes
bool canonical_order(const std::vector<V3>& V, std::vector<V3>& out) {
  constexpr double tol = 1e-9;
  std::vector<V3> reps;
  for (const auto& p : V) {
    const bool rep = p[2] > tol || (std::fabs(p[2]) <= tol &&
                                    (p[1] > tol || (std::fabs(p[1]) <= tol && p[0] > 0.0)));
    if (rep) reps.push_back(p);
  }
  auto az = [&](const V3& p) {
    const double a = std::atan2(p[1], p[0]);
    return a <= -kPi + tol ? kPi : a;
  };
  std::stable_sort(reps.begin(), reps.end(), [&](const V3& p, const V3& q) {
    if (std::fabs(p[2] - q[2]) > tol) return p[2] > q[2];
    return az(p) < az(q);
  });
  if (2 * reps.size() != V.size()) return false;
  out = reps;
  for (const auto& p : reps) out.push_back({-p[0], -p[1], -p[2]});
  return true;
}

// points of the icosahedron of tessellation order nu (10 nu^2 + 2 points)
std::vector<V3> tessellation(int nu) {
  std::vector<V3> V;
  std::vector<std::array<int, 3>> F;
  icosahedron(V, F);
  std::map<std::tuple<long long, long long, long long>, V3> pts;
  for (const auto& f : F)
    for (int i = 0; i <= nu; ++i)
      for (int j = 0; j <= nu - i; ++j) {
        const int k = nu - i - j;
        V3 p;
        for (int q = 0; q < 3; ++q) p[q] = (i * V[f[0]][q] + j * V[f[1]][q] + k * V[f[2]][q]) / nu;
        p = normed(p);
        const auto key = std::make_tuple(std::llround(p[0] * 1e9), std::llround(p[1] * 1e9),
                                         std::llround(p[2] * 1e9));
        pts[key] = p;
      }
  std::vector<V3> out;
  for (const auto& kv : pts) out.push_back(kv.second);
  return out;
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on P_n
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int l = 1; l < n; ++l) {
        const double p2 = ((2 * l + 1) * z * p1 - l * p0) / (l + 1);
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

double legendre_sum(const std::vector<double>& c, double t) {
  double pm = 1.0, pl = t, s = c[0];
  const int L = (int)c.size() - 1;
  if (L >= 1) s += c[1] * t;
  for (int l = 1; l < L; ++l) {
    const double pn = ((2 * l + 1) * t * pl - l * pm) / (l + 1);
    pm = pl;
    pl = pn;
    s += c[l + 1] * pn;
  }
  return s;
}

// Chebyshev coefficients a_j of the degree-L polynomial h(t) = sum_l c_l P_l(t):
// interpolation at the L+1 Chebyshev points is exact for this degree.
std::vector<double> legendre_to_chebyshev(const std::vector<double>& c) {
  const int L = (int)c.size() - 1, n = L + 1;
  std::vector<double> fv(n), a(n, 0.0);
  for (int j = 0; j < n; ++j) fv[j] = legendre_sum(c, std::cos(kPi * (j + 0.5) / n));
  for (int m = 0; m < n; ++m) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += fv[j] * std::cos(kPi * m * (j + 0.5) / n);
    a[m] = (m == 0 ? 1.0 : 2.0) * s / n;
  }
  return a;
}

// h(t) = sum_l c_l P_l(t) = E(v) + t O(v) with v = t^2 - 1/2: monomial
// coefficients of h (Legendre recurrence on coefficient vectors), split into
// even and odd parts, then re-centred from s = t^2 to v = s - 1/2.
void split_monomial(const std::vector<double>& c, std::vector<double>& e, std::vector<double>& o) {
  const int L = (int)c.size() - 1;
  std::vector<double> m(L + 1, 0.0), pm(L + 2, 0.0), pl(L + 2, 0.0), pn(L + 2, 0.0);
  pm[0] = 1.0;                 // P_0
  m[0] += c[0];
  if (L >= 1) {
    pl[1] = 1.0;               // P_1
    m[1] += c[1];
  }
  for (int l = 1; l < L; ++l) {
    std::fill(pn.begin(), pn.end(), 0.0);
    for (int j = 0; j <= l; ++j) pn[j + 1] += (2.0 * l + 1.0) / (l + 1.0) * pl[j];
    for (int j = 0; j <= l - 1; ++j) pn[j] -= double(l) / (l + 1.0) * pm[j];
    for (int j = 0; j <= l + 1; ++j) m[j] += c[l + 1] * pn[j];
    pm.swap(pl);
    pl.swap(pn);
  }
  auto recentre = [](const std::vector<double>& s) {
    // sum_j s_j (v + 1/2)^j = sum_k r_k v^k
    const int n = (int)s.size();
    std::vector<double> r(n, 0.0);
    for (int j = 0; j < n; ++j) {
      double binom = 1.0;   // C(j, k) (1/2)^(j-k), k from j down to 0
      double pw = 1.0;
      for (int k = j; k >= 0; --k) {
        r[k] += s[j] * binom * pw;
        binom = binom * k / double(j - k + 1);
        pw *= 0.5;
      }
    }
    return r;
  };
  std::vector<double> se, so;
  for (int j = 0; j <= L; j += 2) se.push_back(m[j]);
  for (int j = 1; j <= L; j += 2) so.push_back(m[j]);
  e = recentre(se);
  o = recentre(so);
}

bool axis_ok(int n) { return z_supported(n); }

os3d_status check_params(const os3d_params& p) {
  if (p.k < 0 || p.k > 8 || !(p.s_theta > 0.0) || p.L < 0 || p.L > kMaxL || p.N < 0 || p.N > 64 ||
      !(p.gamma > 0.0 && p.gamma < 1.0) || !(p.eps > 0.0) || (p.fit_mode != 0 && p.fit_mode != 1) ||
      p.block_slots < 0 || p.block_slots > kMaxSlots || (p.overlap != 0 && p.overlap != 1) ||
      (p.profile != 0 && p.profile != 1))
    return OS3D_EINVAL;
  return OS3D_OK;
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

bool fault_is(const char* what) {
  const char* e = std::getenv("OS3D_FAULT");
  return e && std::strcmp(e, what) == 0;
}

// ---------------------------------------------------------------------------
// diagnostics: launch counter and optional per-kernel CUDA-event timing
// ---------------------------------------------------------------------------
std::atomic<unsigned long long> g_launches{0};
std::atomic<int> g_profile{0};
std::mutex g_prof_mu;
struct ProfRec {
  int kind;
  cudaEvent_t a, b;
};
std::vector<ProfRec> g_prof_pending;
std::vector<cudaEvent_t> g_event_pool;
unsigned long long g_prof_launches[OS3D_KIND_COUNT] = {};
double g_prof_ms[OS3D_KIND_COUNT] = {};

cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

template <class F>
cudaError_t counted_launch(int kind, cudaStream_t s, F&& launch) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (g_profile.load()) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    a = take_event();
    b = take_event();
    if (a) cudaEventRecord(a, s);
  }
  const cudaError_t e = launch();
  if (e == cudaSuccess) g_launches.fetch_add(1);
  if (a && b) {
    cudaEventRecord(b, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_pending.push_back({kind, a, b});
  }
  return e;
}

}  // namespace

bool os3d::profiling_enabled() { return g_profile.load() != 0; }
void os3d::add_launch_count(unsigned long long n) { g_launches.fetch_add(n); }

namespace {

os3d_status current_device_matches(const os3d_bank* b) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return OS3D_ECUDA;
  return dev == b->dev ? OS3D_OK : OS3D_EINVAL;
}

}  // namespace

// ===========================================================================
extern "C" {

const char* os3d_status_string(os3d_status s) {
  switch (s) {
    case OS3D_OK: return "ok";
    case OS3D_EINVAL: return "invalid argument";
    case OS3D_ENOMEM: return "device allocation failed";
    case OS3D_ECUDA: return "CUDA error";
    case OS3D_ETIMEOUT: return "timed out";
    case OS3D_EUNSUPPORTED: return "unsupported grid size";
  }
  return "unknown status";
}

os3d_status os3d_default_params(os3d_params* p) {
  if (!p) return OS3D_EINVAL;
  p->k = 2;
  p->s_theta = 0.7;
  p->L = 16;
  p->N = 8;
  p->gamma = 0.8;
  p->eps = 1e-4;
  p->fit_mode = 1;
  p->block_slots = 0;
  p->overlap = 1;
  p->profile = 0;
  return OS3D_OK;
}

os3d_status os3d_icosa_orientations(int subdiv, double* out, int capacity, int* n_o) {
  if (subdiv < 0 || subdiv > 4 || !n_o) return OS3D_EINVAL;
  const int n = 10 * (1 << (2 * subdiv)) + 2;
  *n_o = n;
  if (!out || capacity < n) return OS3D_EINVAL;
  std::vector<V3> V;
  std::vector<std::array<int, 3>> F;
  icosahedron(V, F);
  for (int s = 0; s < subdiv; ++s) subdivide(V, F);
  std::vector<V3> o;
  if ((int)V.size() != n || !canonical_order(V, o)) return OS3D_EINVAL;
  for (int i = 0; i < n; ++i)
    for (int q = 0; q < 3; ++q) out[3 * i + q] = o[i][q];
  return OS3D_OK;
}

os3d_status os3d_octa_orientations(int subdiv, double* out, int capacity, int* n_o) {
  if (subdiv < 0 || subdiv > 5 || !n_o) return OS3D_EINVAL;
  const int n = 4 * (1 << (2 * subdiv)) + 2;
  *n_o = n;
  if (!out || capacity < n) return OS3D_EINVAL;
  std::vector<V3> V;
  std::vector<std::array<int, 3>> F;
  octahedron(V, F);
  for (int s = 0; s < subdiv; ++s) subdivide(V, F);
  std::vector<V3> o;
  if ((int)V.size() != n || !canonical_order(V, o)) return OS3D_EINVAL;
  for (int i = 0; i < n; ++i)
    for (int q = 0; q < 3; ++q) out[3 * i + q] = o[i][q];
  return OS3D_OK;
}

os3d_status os3d_make_wavelets(const int dims[3], const double* orient, int n_o,
                               const os3d_params* pp, void* stream, os3d_bank** out) {
  if (!dims || !orient || !out || n_o < 1) return OS3D_EINVAL;
  *out = nullptr;
  os3d_params p;
  if (pp) p = *pp;
  else os3d_default_params(&p);
  if (check_params(p) != OS3D_OK) return OS3D_EINVAL;
  for (int i = 0; i < n_o; ++i) {
    const double* v = orient + 3 * i;
    const double nn = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (!(std::fabs(nn - 1.0) < 1e-6)) return OS3D_EINVAL;
  }
  const int nz = dims[0], ny = dims[1], nx = dims[2];
  if (nz < 1 || ny < 1 || nx < 1) return OS3D_EINVAL;
  if (!axis_ok(nz) || !axis_ok(ny) || !axis_ok(nx) || nx % kTileX) return OS3D_EUNSUPPORTED;
  if (fault_is("alloc")) return OS3D_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;

  os3d_bank* b = new (std::nothrow) os3d_bank();
  if (!b) return OS3D_ENOMEM;
  auto fail = [&](os3d_status st) {
    os3d_destroy_bank(b);
    return st;
  };
  if (cudaGetDevice(&b->dev) != cudaSuccess) return fail(OS3D_ECUDA);
  b->dims[0] = nz;
  b->dims[1] = ny;
  b->dims[2] = nx;
  b->nvox = (long long)nz * ny * nx;
  b->n_o = n_o;
  b->p = p;
  b->orient.assign(orient, orient + 3 * n_o);

  // antipodal pairs
  std::vector<int> used(n_o, 0);
  for (int i = 0; i < n_o; ++i) {
    if (used[i]) continue;
    used[i] = 1;
    int partner = -1;
    for (int j = 0; j < n_o && partner < 0; ++j) {
      if (used[j]) continue;
      double d = 0;
      for (int q = 0; q < 3; ++q) d = std::max(d, std::fabs(orient[3 * i + q] + orient[3 * j + q]));
      if (d < 1e-9) partner = j;
    }
    if (partner >= 0) used[partner] = 1;
    b->slot_a.push_back(i);
    b->slot_b.push_back(partner);
  }
  const int nslots = (int)b->slot_a.size();
  const size_t vol_c64 = sizeof(float2) * (size_t)b->nvox;
  if (p.block_slots > 0) {
    b->block_slots = p.block_slots;
  } else {
    // long blocks: fewer, longer launches; with the two side streams the
    // intermediates of consecutive blocks overlap in time (measured at
    // 128^3 x 162, forward + inverse: 2.26, 2.24, 2.22, 2.24 ms for blocks of
    // 8, 10, 11, 12 pairs; 2.69 ms at 3)
    b->block_slots = kAutoSlots;
  }
  b->block_slots = std::min(b->block_slots, nslots);
  // f_hat, two partial orientation sums, one per-volume intermediate and two
  // sets of block intermediates (for the two side streams)
  b->ws_bytes = vol_c64 * (4 + 2 * b->block_slots);

  // device allocations
  if (cudaMalloc(&b->Gs, sizeof(float) * b->nvox) != cudaSuccess ||
      cudaMalloc(&b->GM, sizeof(float) * b->nvox) != cudaSuccess ||
      cudaMalloc(&b->Minv, sizeof(float) * b->nvox) != cudaSuccess ||
      cudaMalloc(&b->err, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    return fail(OS3D_ENOMEM);
  }
  if (cudaMemsetAsync(b->err, 0, sizeof(unsigned), s) != cudaSuccess) return fail(OS3D_ECUDA);
  {
    bool all_paired = true;
    for (int q : b->slot_b) all_paired = all_paired && q >= 0;
    b->mirror = all_paired ? 1 : 0;
    const std::vector<int4> sg = ball_segments(nz, ny, nx, all_paired, &b->n_in);
    b->nseg = (int)sg.size();
    if (b->nseg > 0) {
      if (cudaMalloc(&b->seg, sizeof(int4) * sg.size()) != cudaSuccess) {
        cudaGetLastError();
        return fail(OS3D_ENOMEM);
      }
      if (cudaMemcpy(b->seg, sg.data(), sizeof(int4) * sg.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess)
        return fail(OS3D_ECUDA);
    }
  }
  for (int i = 0; i < 2; ++i)
    if (cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_join[i], cudaEventDisableTiming) != cudaSuccess)
      return fail(OS3D_ECUDA);
  if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess)
    return fail(OS3D_ECUDA);

  // (a1) sample points for the zonal fit
  std::vector<double> zt, wt;
  if (p.fit_mode == 1) {
    for (const auto& q : tessellation(15)) {
      const double z = std::max(-1.0, std::min(1.0, q[2]));
      zt.push_back(z);
      zt.push_back(std::acos(z));
      wt.push_back(1.0);
    }
  } else {
    std::vector<double> edges = {0.0};
    std::vector<double> kn;
    for (int j = 0; j <= p.k + 1; ++j) {
      const double t = std::fabs(p.s_theta * (j - 0.5 * (p.k + 1)));
      if (t > 0.0 && t < kPi) kn.push_back(t);
    }
    std::sort(kn.begin(), kn.end());
    kn.erase(std::unique(kn.begin(), kn.end()), kn.end());
    for (double t : kn) edges.push_back(t);
    edges.push_back(kPi);
    std::vector<double> gx, gw;
    gauss_legendre(64, gx, gw);
    for (size_t e = 0; e + 1 < edges.size(); ++e) {
      const double lo = edges[e], hi = edges[e + 1];
      for (size_t q = 0; q < gx.size(); ++q) {
        const double th = 0.5 * (hi - lo) * gx[q] + 0.5 * (hi + lo);
        zt.push_back(std::cos(th));
        zt.push_back(th);
        wt.push_back(0.5 * (hi - lo) * gw[q] * std::sin(th));
      }
    }
  }
  const int npts = (int)wt.size();
  const int L = p.L;
  DevBuf dzt, dwt, dout, dc, dslots;
  if (cudaMalloc(&dzt.p, sizeof(double) * zt.size()) != cudaSuccess ||
      cudaMalloc(&dwt.p, sizeof(double) * wt.size()) != cudaSuccess ||
      cudaMalloc(&dout.p, sizeof(double) * 2 * (L + 1)) != cudaSuccess ||
      cudaMalloc(&dslots.p, sizeof(double) * 4 * nslots) != cudaSuccess) {
    cudaGetLastError();
    return fail(OS3D_ENOMEM);
  }
  if (cudaMemcpyAsync(dzt.p, zt.data(), sizeof(double) * zt.size(), cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(dwt.p, wt.data(), sizeof(double) * wt.size(), cudaMemcpyHostToDevice, s))
    return fail(OS3D_ECUDA);
  if (launch_fit((const double*)dzt.p, (const double*)dwt.p, npts, p.fit_mode, p.k, p.s_theta, L,
                 n_o, p.profile, (double*)dout.p, s) != cudaSuccess)
    return fail(OS3D_ECUDA);
  std::vector<double> bc(2 * (L + 1));
  if (cudaMemcpyAsync(bc.data(), dout.p, sizeof(double) * bc.size(), cudaMemcpyDeviceToHost, s) ||
      cudaStreamSynchronize(s))
    return fail(OS3D_ECUDA);
  b->b.assign(bc.begin(), bc.begin() + L + 1);
  b->c.assign(bc.begin() + L + 1, bc.end());
  for (double v : bc)
    if (!std::isfinite(v)) return fail(OS3D_EINVAL);

  // Chebyshev form for the FP32 transform kernels
  const std::vector<double> ch = legendre_to_chebyshev(b->c);
  for (int j = 0; j <= kMaxL; ++j) b->h.a[j] = j <= L ? (float)ch[j] : 0.f;
  b->h.c0 = (float)b->c[0];
  // split monomial form h(t) = E(t^2 - 1/2) + t O(t^2 - 1/2) when it is well conditioned
  b->ev = 2;
  if (L <= 24) {
    std::vector<double> e, o;
    split_monomial(b->c, e, o);
    double hmax = 0.0, amp = 0.0;
    for (int q = 0; q <= 2000; ++q) hmax = std::max(hmax, std::fabs(legendre_sum(b->c, -1.0 + q / 1000.0)));
    for (double v : e) amp += std::fabs(v);
    for (double v : o) amp += std::fabs(v);
    if (hmax > 0.0 && amp <= 4000.0 * hmax) {
      b->ev = L <= 16 ? 0 : 1;
      for (int k = 0; k < 13; ++k) b->h.e[k] = k < (int)e.size() ? (float)e[k] : 0.f;
      for (int k = 0; k < 12; ++k) b->h.o[k] = k < (int)o.size() ? (float)o[k] : 0.f;
      for (int k = 0; k < 13; ++k) b->h.e2[k] = make_float2(b->h.e[k], b->h.e[k]);
      for (int k = 0; k < 12; ++k) b->h.o2[k] = make_float2(b->h.o[k], b->h.o[k]);
    }
  }

  // (a3) M and the per-voxel factors, FP64
  std::vector<double> sl(4 * nslots);
  for (int q = 0; q < nslots; ++q) {
    for (int d = 0; d < 3; ++d) sl[4 * q + d] = orient[3 * b->slot_a[q] + d];
    sl[4 * q + 3] = b->slot_b[q] >= 0 ? 1.0 : 0.0;
  }
  if (cudaMemcpyAsync(dslots.p, sl.data(), sizeof(double) * sl.size(), cudaMemcpyHostToDevice, s))
    return fail(OS3D_ECUDA);
  if (launch_bank_M(nz, ny, nx, p.N, p.gamma, p.eps, (const double*)dout.p + (L + 1), L,
                    (const double*)dslots.p, nslots, n_o, b->mirror, b->Gs, b->GM, b->Minv,
                    s) != cudaSuccess)
    return fail(OS3D_ECUDA);
  // the temporaries are freed when this function returns: wait for the kernels
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(OS3D_ECUDA);
  *out = b;
  return OS3D_OK;
}

os3d_status os3d_bank_info(const os3d_bank* b, size_t* ws, size_t* footprint) {
  if (!b) return OS3D_EINVAL;
  if (ws) *ws = b->ws_bytes;
  // one volume through forward + inverse: its complex64 score and two images
  if (footprint) *footprint = sizeof(float2) * (size_t)b->nvox * b->n_o + 2 * sizeof(float) * (size_t)b->nvox;
  return OS3D_OK;
}

os3d_status os3d_bank_wait_errors(const os3d_bank* b, unsigned* count, int reset) {
  if (!b || !count) return OS3D_EINVAL;
  if (current_device_matches(b) != OS3D_OK) return OS3D_EINVAL;
  if (cudaMemcpy(count, b->err, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
    return OS3D_ECUDA;
  if (reset && cudaMemset(b->err, 0, sizeof(unsigned)) != cudaSuccess) return OS3D_ECUDA;
  return OS3D_OK;
}

os3d_status os3d_bank_resident_bytes(const os3d_bank* b, size_t* bytes) {
  if (!b || !bytes) return OS3D_EINVAL;
  std::lock_guard<std::mutex> lk(b->ws_mu);
  *bytes = 3 * sizeof(float) * (size_t)b->nvox + sizeof(int4) * (size_t)b->nseg +
           (b->ws ? b->ws_bytes : 0);
  return OS3D_OK;
}

os3d_status os3d_bank_coefficients(const os3d_bank* bk, double* bo, double* co) {
  if (!bk) return OS3D_EINVAL;
  if (bo) std::copy(bk->b.begin(), bk->b.end(), bo);
  if (co) std::copy(bk->c.begin(), bk->c.end(), co);
  return OS3D_OK;
}

os3d_status os3d_bank_minv(const os3d_bank* bk, float* minv, void* stream) {
  if (!bk) return OS3D_EINVAL;
  if (!minv) return OS3D_OK;
  if (current_device_matches(bk) != OS3D_OK) return OS3D_EINVAL;
  if (cudaMemcpyAsync(minv, bk->Minv, sizeof(float) * bk->nvox, cudaMemcpyDeviceToDevice,
                      (cudaStream_t)stream) != cudaSuccess)
    return OS3D_ECUDA;
  return OS3D_OK;
}

os3d_status os3d_destroy_bank(os3d_bank* b) {
  if (!b) return OS3D_EINVAL;
  if (b->Gs) cudaFree(b->Gs);
  if (b->GM) cudaFree(b->GM);
  if (b->Minv) cudaFree(b->Minv);
  if (b->seg) cudaFree(b->seg);
  if (b->err) cudaFree(b->err);
  if (b->ws) cudaFree(b->ws);
  for (int i = 0; i < 2; ++i) {
    if (b->side[i]) cudaStreamDestroy(b->side[i]);
    if (b->ev_join[i]) cudaEventDestroy(b->ev_join[i]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  delete b;
  return OS3D_OK;
}

}  // extern "C"

// ===========================================================================
// transforms
// ===========================================================================
namespace {

struct Work {
  float2* fh;     // f_hat G / n^3
  float2* A[2];   // partial orientation sums (one per side stream)
  float2* T0;     // per-volume intermediate
  float2* T[2];   // block intermediates (one set per side stream)
};

Work carve_base(const os3d_bank* b, void* base_ptr) {
  float2* base = (float2*)base_ptr;
  const long long n = b->nvox;
  Work w;
  w.fh = base;
  w.A[0] = base + n;
  w.A[1] = base + 2 * n;
  w.T0 = base + 3 * n;
  w.T[0] = base + 4 * n;
  w.T[1] = base + (4 + b->block_slots) * n;
  return w;
}

// The caller's workspace, or the bank's own, which the first call that needs
// it allocates (cudaMalloc; outside stream capture).
os3d_status workspace_for(const os3d_bank* b, void* ws, Work* out) {
  if (!ws) {
    std::lock_guard<std::mutex> lk(b->ws_mu);
    if (!b->ws) {
      if (fault_is("alloc_ws") || cudaMalloc(&b->ws, b->ws_bytes) != cudaSuccess) {
        cudaGetLastError();
        b->ws = nullptr;
        return OS3D_ENOMEM;
      }
    }
    ws = b->ws;
  }
  *out = carve_base(b, ws);
  return OS3D_OK;
}

// fork the two side streams off `s` / join them back into `s`
cudaError_t fork_side(const os3d_bank* b, cudaStream_t s) {
  cudaError_t e = cudaEventRecord(b->ev_fork, s);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(b->side[i], b->ev_fork, 0);
  return e;
}
cudaError_t join_side(const os3d_bank* b, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaEventRecord(b->ev_join[i], b->side[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev_join[i], 0);
  }
  return e;
}

PassArgs args_base(const os3d_bank* b) {
  PassArgs a{};
  a.nz = b->dims[0];
  a.ny = b->dims[1];
  a.nx = b->dims[2];
  a.wz = float(2.0 * kPi / b->dims[0]);
  a.wy = float(2.0 * kPi / b->dims[1]);
  a.wx = float(2.0 * kPi / b->dims[2]);
  a.slot_stride = b->nvox;
  a.nslots = 1;
  a.h = b->h;
  // tiles outside the disc are skipped only where the cluster plane pass
  // (which honours the skip) consumes or produces the block intermediates
  a.disc = xy_supported(b->dims[1], b->dims[2]) ? 1 : 0;
  for (int j = 0; j < kMaxSlots; ++j) a.ub[j] = -1;
  return a;
}

// slots [s0, s0 + ns) of volume v: orientations and score offsets
void set_slots(const os3d_bank* b, PassArgs& a, int v, int s0, int ns) {
  const long long n = b->nvox;
  a.nslots = ns;
  for (int j = 0; j < ns; ++j) {
    const int ia = b->slot_a[s0 + j], ib = b->slot_b[s0 + j];
    for (int d = 0; d < 3; ++d) a.nvec[j][d] = (float)b->orient[3 * ia + d];
    a.ua[j] = ((long long)v * b->n_o + ia) * n;
    a.ub[j] = ib >= 0 ? ((long long)v * b->n_o + ib) * n : -1;
  }
}

os3d_status check_call(const os3d_bank* b, const void* x, const void* y, int batch, int udtype,
                       void* ws) {
  if (!b || !x || !y || batch < 1) return OS3D_EINVAL;
  if (udtype != OS3D_U_C64 && udtype != OS3D_U_BF16X2) return OS3D_EINVAL;
  if (ws && (reinterpret_cast<uintptr_t>(ws) & 255)) return OS3D_EINVAL;
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15) return OS3D_EINVAL;
  return current_device_matches(b);
}

#define OS3D_CK(call)                             \
  do {                                            \
    if ((call) != cudaSuccess) return OS3D_ECUDA; \
  } while (0)

// One xy-pass of `mode`: the cluster kernel when a z-plane fits it, otherwise
// a pencil pass along x and one along y (the y pass in place on complex data).
cudaError_t launch_plane(const os3d_bank* b, int mode, int ub, const PassArgs& a, cudaStream_t s) {
  const int nz = b->dims[0], ny = b->dims[1], nx = b->dims[2];
  if (xy_supported(ny, nx)) return launch_xy(ny, nx, mode, ub, a, s);
  const long long P = (long long)ny * nx;
  const PencilGeom gx{ny, P, nx, 1};    // lines = rows, elements contiguous
  const PencilGeom gy{nx, P, 1, nx};    // lines = columns, elements nx apart
  const long long lx = (long long)nz * ny, ly = (long long)nz * nx;
  const int ns = (mode == XY_FWD_SCORE || mode == XY_INV_SCORE) ? a.nslots : 1;
  PassArgs c = a;   // complex work array for the in-place y pass
  cudaError_t e;
  switch (mode) {
    case XY_FWD_REAL:   // f -> DFT_x -> out, then DFT_y in place
      g_launches.fetch_add(1);   // counted_launch counts one of the two
      e = launch_pencil(nx, PN_R2C, -1, 0, a, gx, lx, 1, s);
      if (e != cudaSuccess) return e;
      c.in = a.out;
      c.in_off = a.out_off;
      return launch_pencil(ny, PN_C2C, -1, 0, c, gy, ly, 1, s);
    case XY_INV_REAL:   // IDFT_y in place on in, then IDFT_x -> real out
      g_launches.fetch_add(1);
      c.out = const_cast<void*>(a.in);
      c.out_off = a.in_off;
      e = launch_pencil(ny, PN_C2C, 1, 0, c, gy, ly, 1, s);
      if (e != cudaSuccess) return e;
      return launch_pencil(nx, PN_C2R, 1, 0, a, gx, lx, 1, s);
    case XY_FWD_SCORE:  // IDFT_y in place on T_s, then IDFT_x -> U_a, U_b
      g_launches.fetch_add(1);
      c.out = const_cast<void*>(a.in);
      e = launch_pencil(ny, PN_C2C, 1, 0, c, gy, ly, ns, s);
      if (e != cudaSuccess) return e;
      return launch_pencil(nx, PN_C2U, 1, ub, a, gx, lx, ns, s);
    case XY_INV_SCORE:  // U_a + conj U_b -> DFT_x -> T_s, then DFT_y in place
      g_launches.fetch_add(1);
      e = launch_pencil(nx, PN_U2C, -1, ub, a, gx, lx, ns, s);
      if (e != cudaSuccess) return e;
      c.in = a.out;
      return launch_pencil(ny, PN_C2C, -1, 0, c, gy, ly, ns, s);
    default: return cudaErrorInvalidValue;
  }
}

// The score-domain step of Upsilon on a block of intermediates T_s (in
// place): the fused plane kernel, or for other planes the pencil passes
// IDFT_y, IDFT_x, the soft threshold, DFT_x, DFT_y.
cudaError_t launch_plane_soft(const os3d_bank* b, const PassArgs& a, cudaStream_t s) {
  const int nz = b->dims[0], ny = b->dims[1], nx = b->dims[2];
  if (soft_plane_supported(ny, nx)) return launch_xy(ny, nx, XY_SOFT, 0, a, s);
  const long long P = (long long)ny * nx;
  const PencilGeom gx{ny, P, nx, 1};
  const PencilGeom gy{nx, P, 1, nx};
  const long long lx = (long long)nz * ny, ly = (long long)nz * nx;
  PassArgs c = a;
  c.in = a.out;
  c.in_off = c.out_off = 0;
  g_launches.fetch_add(4);   // five launches, one counted by counted_launch
  cudaError_t e = launch_pencil(ny, PN_C2C, 1, 0, c, gy, ly, a.nslots, s);
  if (e == cudaSuccess) e = launch_pencil(nx, PN_C2C, 1, 0, c, gx, lx, a.nslots, s);
  if (e == cudaSuccess) e = launch_soft_slots(c, b->nvox, s);
  if (e == cudaSuccess) e = launch_pencil(nx, PN_C2C, -1, 0, c, gx, lx, a.nslots, s);
  if (e == cudaSuccess) e = launch_pencil(ny, PN_C2C, -1, 0, c, gy, ly, a.nslots, s);
  return e;
}

size_t u_elem_bytes(int udtype) { return udtype == OS3D_U_BF16X2 ? 4 : 8; }

// f_hat G / n^3 of volume v of f into w.fh (a4)
os3d_status prep_fhat(const os3d_bank* b, const float* f, int v, const Work& w, cudaStream_t s) {
  const int nz = b->dims[0], ny = b->dims[1], nx = b->dims[2];
  const int tiles = ny * (nx / kTileX);
  PassArgs x0 = args_base(b);
  x0.in = f;
  x0.in_off = (long long)v * b->nvox;
  x0.out = w.T0;
  OS3D_CK(counted_launch(OS3D_KIND_XY_FWD_REAL, s,
                         [&] { return launch_plane(b, XY_FWD_REAL, 0, x0, s); }));
  PassArgs zp = args_base(b);
  zp.in = w.T0;
  zp.out = w.fh;
  zp.mult = b->Gs;
  OS3D_CK(counted_launch(OS3D_KIND_Z_FWD_PREP, s,
                         [&] { return launch_z(nz, Z_FWD_PREP, 0, zp, tiles, s); }));
  return OS3D_OK;
}

// f = Re IDFT[ (A_0 + A_1) x mult ] of volume v into fout (end of a6 / a7)
os3d_status finish_real(const os3d_bank* b, const Work& w, int nblocks, const float* mult,
                        float* fout, int v, cudaStream_t s) {
  const int nz = b->dims[0], ny = b->dims[1], nx = b->dims[2];
  const int tiles = ny * (nx / kTileX);
  PassArgs zf = args_base(b);
  zf.in = w.A[0];
  zf.in2 = (b->p.overlap && nblocks >= 2) ? w.A[1] : nullptr;
  zf.out = w.T0;
  zf.mult = mult;
  OS3D_CK(counted_launch(OS3D_KIND_Z_INV_FINAL, s,
                         [&] { return launch_z(nz, Z_INV_FINAL, 0, zf, tiles, s); }));
  PassArgs xf = args_base(b);
  xf.in = w.T0;
  xf.out = fout;
  xf.out_off = (long long)v * b->nvox;
  OS3D_CK(counted_launch(OS3D_KIND_XY_INV_REAL, s,
                         [&] { return launch_plane(b, XY_INV_REAL, 0, xf, s); }));
  return OS3D_OK;
}

// inverse (use_m = true) or adjoint (use_m = false). Consecutive blocks of
// orientation pairs alternate between the two side streams (each with its own
// intermediates and partial sum), so one block's xy-pass overlaps the other's
// z-pass.
// wgt, gscale: the weighted adjoint Re W^*(2 g w U) (the plane pass's weighted
// load; complex64 U on plane-pass grids), else null
os3d_status backward_impl(const os3d_bank* b, const void* U, int udtype, int batch, float* fout,
                          void* ws, cudaStream_t s, bool use_m, const float* wgt = nullptr,
                          const float* gscale = nullptr) {
  Work w;
  if (const os3d_status e = workspace_for(b, ws, &w)) return e;
  const int nz = b->dims[0], ny = b->dims[1], nx = b->dims[2];
  const int nslots = (int)b->slot_a.size();
  const int tiles = ny * (nx / kTileX);
  for (int v = 0; v < batch; ++v) {
    if (b->p.overlap) OS3D_CK(fork_side(b, s));
    int q = 0;
    for (int s0 = 0; s0 < nslots; s0 += b->block_slots, ++q) {
      const int ns = std::min(b->block_slots, nslots - s0);
      const int k = b->p.overlap ? (q & 1) : 0;
      cudaStream_t st = b->p.overlap ? b->side[k] : s;
      PassArgs xa = args_base(b);
      set_slots(b, xa, v, s0, ns);
      xa.in = U;
      xa.out = w.T[k];
      xa.wgt = wgt;
      xa.gscale = gscale;
      const int mode = wgt ? XY_INV_WSCORE : XY_INV_SCORE;
      OS3D_CK(counted_launch(OS3D_KIND_XY_INV_SCORE, st,
                             [&] { return launch_plane(b, mode, udtype, xa, st); }));
      PassArgs za = xa;
      za.in = w.T[k];
      za.out = w.A[k];
      za.accumulate = b->p.overlap ? q >= 2 : q >= 1;
      OS3D_CK(counted_launch(OS3D_KIND_Z_INV_SCORE, st,
                             [&] { return launch_z(nz, Z_INV_SCORE, b->ev, za, tiles, st); }));
    }
    if (b->p.overlap) OS3D_CK(join_side(b, s));
    const os3d_status st = finish_real(b, w, q, use_m ? b->GM : b->Gs, fout, v, s);
    if (st != OS3D_OK) return st;
  }
  return OS3D_OK;
}

os3d_status forward_impl(const os3d_bank* b, const float* f, int batch, void* U, int udtype,
                         void* ws, cudaStream_t s) {
  Work w;
  if (const os3d_status e = workspace_for(b, ws, &w)) return e;
  const int nz = b->dims[0], ny = b->dims[1], nx = b->dims[2];
  const int nslots = (int)b->slot_a.size();
  const int tiles = ny * (nx / kTileX);
  for (int v = 0; v < batch; ++v) {
    // (a4) f_hat G / n^3
    const os3d_status st = prep_fhat(b, f, v, w, s);
    if (st != OS3D_OK) return st;
    // (a5) per block of orientation pairs, alternating between the side streams
    if (b->p.overlap) OS3D_CK(fork_side(b, s));
    int q = 0;
    for (int s0 = 0; s0 < nslots; s0 += b->block_slots, ++q) {
      const int ns = std::min(b->block_slots, nslots - s0);
      const int k = b->p.overlap ? (q & 1) : 0;
      cudaStream_t st = b->p.overlap ? b->side[k] : s;
      PassArgs za = args_base(b);
      set_slots(b, za, v, s0, ns);
      za.in = w.fh;
      za.out = w.T[k];
      OS3D_CK(counted_launch(OS3D_KIND_Z_FWD_SCORE, st,
                             [&] { return launch_z(nz, Z_FWD_SCORE, b->ev, za, tiles, st); }));
      PassArgs xa = za;
      xa.in = w.T[k];
      xa.out = U;
      OS3D_CK(counted_launch(OS3D_KIND_XY_FWD_SCORE, st,
                             [&] { return launch_plane(b, XY_FWD_SCORE, udtype, xa, st); }));
    }
    if (b->p.overlap) OS3D_CK(join_side(b, s));
  }
  return OS3D_OK;
}

// Upsilon f = W^{*,ext} Phi W f (Sec. 4.1): per block, the z-pass of the
// forward transform, the fused score-domain step and the z-pass of the
// inverse; the score itself is never stored.
os3d_status upsilon_impl(const os3d_bank* b, const float* f, int batch, float* fout, float power,
                         void* ws, cudaStream_t s) {
  Work w;
  if (const os3d_status e = workspace_for(b, ws, &w)) return e;
  const int nz = b->dims[0], ny = b->dims[1], nx = b->dims[2];
  const int nslots = (int)b->slot_a.size();
  const int tiles = ny * (nx / kTileX);
  for (int v = 0; v < batch; ++v) {
    const os3d_status st = prep_fhat(b, f, v, w, s);
    if (st != OS3D_OK) return st;
    if (b->p.overlap) OS3D_CK(fork_side(b, s));
    int q = 0;
    for (int s0 = 0; s0 < nslots; s0 += b->block_slots, ++q) {
      const int ns = std::min(b->block_slots, nslots - s0);
      const int k = b->p.overlap ? (q & 1) : 0;
      cudaStream_t st2 = b->p.overlap ? b->side[k] : s;
      PassArgs za = args_base(b);
      set_slots(b, za, v, s0, ns);
      za.in = w.fh;
      za.out = w.T[k];
      // the pencil passes of the score-domain step read every column of T
      za.disc = soft_plane_supported(ny, nx) ? 1 : 0;
      OS3D_CK(counted_launch(OS3D_KIND_Z_FWD_SCORE, st2,
                             [&] { return launch_z(nz, Z_FWD_SCORE, b->ev, za, tiles, st2); }));
      PassArgs xa = za;
      xa.in = w.T[k];
      xa.out = w.T[k];
      xa.power = power;
      OS3D_CK(counted_launch(OS3D_KIND_XY_SOFT, st2,
                             [&] { return launch_plane_soft(b, xa, st2); }));
      PassArgs zi = za;
      zi.in = w.T[k];
      zi.out = w.A[k];
      zi.accumulate = b->p.overlap ? q >= 2 : q >= 1;
      OS3D_CK(counted_launch(OS3D_KIND_Z_INV_SCORE, st2,
                             [&] { return launch_z(nz, Z_INV_SCORE, b->ev, zi, tiles, st2); }));
    }
    if (b->p.overlap) OS3D_CK(join_side(b, s));
    const os3d_status st3 = finish_real(b, w, q, b->GM, fout, v, s);
    if (st3 != OS3D_OK) return st3;
  }
  return OS3D_OK;
}

// Weighted energy L = sum w |W f|^2 and its gradient Re W^*(2 g w W f) in one
// sweep per block: the z-pass of the forward transform, the weighted
// score-domain step (per-unit energies into scratch[1 ..]), the z-pass of the
// adjoint; then the final sum of the unit energies in index order.
long long energy_units(const os3d_bank* b, int batch) {
  return (long long)batch * (long long)b->slot_a.size() * b->dims[0] *
         plane_ctas(b->dims[1], b->dims[2]);
}

os3d_status score_energy_impl(const os3d_bank* b, const float* f, const float* wgt,
                              const float* g, int batch, float* loss, float* grad_f,
                              double* scratch, void* ws, cudaStream_t s) {
  Work w;
  if (const os3d_status e = workspace_for(b, ws, &w)) return e;
  const int nz = b->dims[0], ny = b->dims[1], nx = b->dims[2];
  const int nslots = (int)b->slot_a.size();
  const int tiles = ny * (nx / kTileX);
  for (int v = 0; v < batch; ++v) {
    const os3d_status st = prep_fhat(b, f, v, w, s);
    if (st != OS3D_OK) return st;
    if (b->p.overlap) OS3D_CK(fork_side(b, s));
    int q = 0;
    for (int s0 = 0; s0 < nslots; s0 += b->block_slots, ++q) {
      const int ns = std::min(b->block_slots, nslots - s0);
      const int k = b->p.overlap ? (q & 1) : 0;
      cudaStream_t st2 = b->p.overlap ? b->side[k] : s;
      PassArgs za = args_base(b);
      set_slots(b, za, v, s0, ns);
      za.in = w.fh;
      za.out = w.T[k];
      OS3D_CK(counted_launch(OS3D_KIND_Z_FWD_SCORE, st2,
                             [&] { return launch_z(nz, Z_FWD_SCORE, b->ev, za, tiles, st2); }));
      PassArgs xa = za;
      xa.in = w.T[k];
      xa.out = w.T[k];
      xa.wgt = wgt;
      xa.gscale = g;
      xa.epart = scratch + 1;
      xa.epart_base = ((long long)v * nslots + s0) * nz * plane_ctas(ny, nx);
      OS3D_CK(counted_launch(OS3D_KIND_XY_SOFT, st2,
                             [&] { return launch_xy(ny, nx, XY_WENERGY, 0, xa, st2); }));
      PassArgs zi = za;
      zi.in = w.T[k];
      zi.out = w.A[k];
      zi.accumulate = b->p.overlap ? q >= 2 : q >= 1;
      OS3D_CK(counted_launch(OS3D_KIND_Z_INV_SCORE, st2,
                             [&] { return launch_z(nz, Z_INV_SCORE, b->ev, zi, tiles, st2); }));
    }
    if (b->p.overlap) OS3D_CK(join_side(b, s));
    const os3d_status st3 = finish_real(b, w, q, b->Gs, grad_f, v, s);
    if (st3 != OS3D_OK) return st3;
  }
  OS3D_CK(counted_launch(OS3D_KIND_ENERGY, s, [&] {
    return launch_energy_final(scratch, energy_units(b, batch), loss, s);
  }));
  return OS3D_OK;
}

// Linear diffusion with the propagator product on the tensor cores (sets of
// more than kMaxOrientE orientations): E and the orientations go to the
// device in the kernel's layout (in the workspace's second block
// intermediate, which the enhancement does not otherwise use).
os3d_status enhance_tensor(const os3d_bank* b, const float* f, int batch, float* f_out,
                           const os3d_diffusion* d, double tau, void* ws, cudaStream_t s) {
  Work w;
  if (const os3d_status we = workspace_for(b, ws, &w)) return we;
  const int np = tc_padded_orientations(b->n_o);
  EnhanceTCArgs e{};
  unsigned char* dprep = reinterpret_cast<unsigned char*>(w.T[1]);
  {
    // exp(tau L) in FP64 on the host, prepared once per (tau, degree)
    std::lock_guard<std::mutex> lk(b->tc_mu);
    if (b->tc_prep.empty() || b->tc_tau != tau || b->tc_degree != d->sh_degree) {
      std::vector<double> E;
      if (angular_propagator(b->orient.data(), b->n_o, d->sh_degree, tau, E) < 0) return OS3D_EINVAL;
      b->tc_inv_se = tc_prepare(E.data(), b->orient.data(), b->n_o, np, b->tc_prep);
      b->tc_tau = tau;
      b->tc_degree = d->sh_degree;
    }
    if (b->tc_prep.size() > sizeof(float2) * (size_t)b->nvox * b->block_slots)
      return OS3D_EUNSUPPORTED;
    e.inv_se = b->tc_inv_se;
    OS3D_CK(cudaMemcpyAsync(dprep, b->tc_prep.data(), b->tc_prep.size(), cudaMemcpyHostToDevice, s));
  }
  e.fh = w.fh;
  e.A = w.A[0];
  e.seg = b->seg;
  e.prep = dprep;
  e.err = b->err;
  e.nseg = b->nseg;
  e.n_in = b->n_in;
  e.mirror = b->mirror;
  e.nz = b->dims[0];
  e.ny = b->dims[1];
  e.nx = b->dims[2];
  e.wz = float(2.0 * kPi / b->dims[0]);
  e.wy = float(2.0 * kPi / b->dims[1]);
  e.wx = float(2.0 * kPi / b->dims[2]);
  e.n3 = float(b->nvox);
  e.n_o = b->n_o;
  e.steps = d->steps;
  e.half_dt = float(0.5 * d->t / d->steps);
  e.D11 = float(d->D11);
  e.D33 = float(d->D33);
  e.h = b->h;
  for (int v = 0; v < batch; ++v) {
    os3d_status r = prep_fhat(b, f, v, w, s);
    if (r != OS3D_OK) return r;
    OS3D_CK(cudaMemsetAsync(w.A[0], 0, sizeof(float2) * b->nvox, s));
    if (b->n_in > 0)
      OS3D_CK(counted_launch(OS3D_KIND_ENHANCE, s, [&] { return launch_enhance_tc(e, b->ev, s); }));
    r = finish_real(b, w, 1, b->GM, f_out, v, s);
    if (r != OS3D_OK) return r;
  }
  // (an upload from pageable memory is staged before cudaMemcpyAsync returns,
  // so the host copy of E may go)
  return OS3D_OK;
}

}  // namespace

extern "C" {

os3d_status os3d_forward(const os3d_bank* b, const float* f, int batch, void* U,
                         os3d_udtype udtype, void* ws, void* stream) {
  const os3d_status st = check_call(b, f, U, batch, udtype, ws);
  if (st != OS3D_OK) return st;
  return forward_impl(b, f, batch, U, udtype, ws, (cudaStream_t)stream);
}

os3d_status os3d_inverse(const os3d_bank* b, const void* U, os3d_udtype udtype, int batch,
                         float* f_out, void* ws, void* stream) {
  const os3d_status st = check_call(b, U, f_out, batch, udtype, ws);
  if (st != OS3D_OK) return st;
  return backward_impl(b, U, udtype, batch, f_out, ws, (cudaStream_t)stream, true);
}

os3d_status os3d_adjoint(const os3d_bank* b, const void* G, os3d_udtype udtype, int batch,
                         float* grad_f, void* ws, void* stream) {
  const os3d_status st = check_call(b, G, grad_f, batch, udtype, ws);
  if (st != OS3D_OK) return st;
  return backward_impl(b, G, udtype, batch, grad_f, ws, (cudaStream_t)stream, false);
}

os3d_status os3d_adjoint_weighted(const os3d_bank* b, const void* U, const float* w,
                                  const float* g, os3d_udtype udtype, int batch, float* grad_f,
                                  void* ws, void* stream) {
  const os3d_status st = check_call(b, U, grad_f, batch, udtype, ws);
  if (st != OS3D_OK) return st;
  if (!w || !g || (reinterpret_cast<uintptr_t>(w) & 15) || (reinterpret_cast<uintptr_t>(g) & 3))
    return OS3D_EINVAL;
  if (udtype != OS3D_U_C64 || !xy_supported(b->dims[1], b->dims[2])) return OS3D_EUNSUPPORTED;
  return backward_impl(b, U, udtype, batch, grad_f, ws, (cudaStream_t)stream, false, w, g);
}

os3d_status os3d_score_energy_scratch(const os3d_bank* b, int batch, size_t* doubles) {
  if (!b || batch < 1 || !doubles) return OS3D_EINVAL;
  *doubles = (size_t)(1 + energy_units(b, batch));
  return OS3D_OK;
}

os3d_status os3d_score_energy_grad(const os3d_bank* b, const float* f, const float* w,
                                   const float* g, int batch, float* loss, float* grad_f,
                                   double* scratch, size_t scratch_doubles, void* ws,
                                   void* stream) {
  const os3d_status st = check_call(b, f, grad_f, batch, OS3D_U_C64, ws);
  if (st != OS3D_OK) return st;
  if (!w || !scratch || (reinterpret_cast<uintptr_t>(w) & 15) ||
      (reinterpret_cast<uintptr_t>(scratch) & 7) || (reinterpret_cast<uintptr_t>(g) & 3) ||
      (reinterpret_cast<uintptr_t>(loss) & 3))
    return OS3D_EINVAL;
  if (scratch_doubles < (size_t)(1 + energy_units(b, batch))) return OS3D_EINVAL;
  if (!soft_plane_supported(b->dims[1], b->dims[2])) return OS3D_EUNSUPPORTED;
  return score_energy_impl(b, f, w, g, batch, loss, grad_f, scratch, ws, (cudaStream_t)stream);
}

os3d_status os3d_scale_by(const float* x, float* y, long long count, const float* g,
                          void* stream) {
  if (count < 0 || (count > 0 && (!x || !y || !g)) ||
      ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15) ||
      (reinterpret_cast<uintptr_t>(g) & 3))
    return OS3D_EINVAL;
  if (count == 0) return OS3D_OK;
  cudaStream_t s = (cudaStream_t)stream;
  OS3D_CK(counted_launch(OS3D_KIND_ENERGY_GRAD, s,
                         [&] { return launch_scale_by(x, y, count, g, s); }));
  return OS3D_OK;
}

os3d_status os3d_approx_reconstruct(const os3d_bank* b, const void* U, os3d_udtype udtype,
                                    int batch, float* f_out, void* stream) {
  const os3d_status st = check_call(b, U, f_out, batch, udtype, nullptr);
  if (st != OS3D_OK) return st;
  const double c0 = b->c[0];
  if (!(std::fabs(c0) > 0.0) || !std::isfinite(c0)) return OS3D_EINVAL;
  const float wgt = (float)(1.0 / (b->n_o * c0));
  cudaStream_t s = (cudaStream_t)stream;
  const size_t eb = u_elem_bytes(udtype);
  for (int v = 0; v < batch; ++v) {
    const char* Uv = (const char*)U + (size_t)v * b->n_o * b->nvox * eb;
    float* fv = f_out + (size_t)v * b->nvox;
    OS3D_CK(counted_launch(OS3D_KIND_APPROX, s, [&] {
      return launch_approx_sum(Uv, udtype == OS3D_U_BF16X2, b->n_o, b->nvox, wgt, fv, s);
    }));
  }
  return OS3D_OK;
}

os3d_status os3d_project(const os3d_bank* b, const void* U, os3d_udtype udtype, int batch,
                         void* U_out, void* ws, void* stream) {
  os3d_status st = check_call(b, U, U_out, batch, udtype, ws);
  if (st != OS3D_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // the reconstructed image lives in the second block intermediate of the
  // workspace, which neither transform touches while it is needed
  Work pw;
  if (const os3d_status e = workspace_for(b, ws, &pw)) return e;
  float* fs = reinterpret_cast<float*>(pw.T[1]);
  const size_t vb = (size_t)b->n_o * b->nvox * u_elem_bytes(udtype);
  for (int v = 0; v < batch; ++v) {
    st = backward_impl(b, (const char*)U + v * vb, udtype, 1, fs, ws, s, true);
    if (st == OS3D_OK) st = forward_impl(b, fs, 1, (char*)U_out + v * vb, udtype, ws, s);
    if (st != OS3D_OK) return st;
  }
  return OS3D_OK;
}

os3d_status os3d_soft_threshold(const void* in, void* out, os3d_udtype udtype, long long count,
                                double power, void* stream) {
  if (!in || !out || count < 0 || count % 4 != 0) return OS3D_EINVAL;
  if (udtype != OS3D_U_C64 && udtype != OS3D_U_BF16X2) return OS3D_EINVAL;
  if (!(power > 0.0) || !std::isfinite(power)) return OS3D_EINVAL;
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) return OS3D_EINVAL;
  if (count == 0) return OS3D_OK;
  cudaStream_t s = (cudaStream_t)stream;
  OS3D_CK(counted_launch(OS3D_KIND_SOFT, s, [&] {
    return launch_soft_scores(in, out, udtype == OS3D_U_BF16X2, count, (float)power, s);
  }));
  return OS3D_OK;
}

static_assert(OS3D_ENERGY_SCRATCH_DOUBLES == 1 + kMaxEnergyBlocks,
              "the energy scratch holds the sum and one partial per block");

os3d_status os3d_weighted_energy(const void* U, const float* w, os3d_udtype udtype,
                                 long long count, double* scratch, float* loss, void* stream) {
  if (!scratch || count < 0 || count % 4 != 0 || (count > 0 && !U)) return OS3D_EINVAL;
  if (udtype != OS3D_U_C64 && udtype != OS3D_U_BF16X2) return OS3D_EINVAL;
  if (((reinterpret_cast<uintptr_t>(U) | reinterpret_cast<uintptr_t>(w)) & 15) ||
      (reinterpret_cast<uintptr_t>(scratch) & 7) || (reinterpret_cast<uintptr_t>(loss) & 3))
    return OS3D_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // an empty score still gets its (zero) sum written
  OS3D_CK(counted_launch(OS3D_KIND_ENERGY, s, [&] {
    return launch_energy(U, w, udtype == OS3D_U_BF16X2, count, scratch, loss, s);
  }));
  g_launches.fetch_add(1);   // counted_launch counts one of the two
  return OS3D_OK;
}

os3d_status os3d_weighted_energy_grad(const void* U, const float* w, os3d_udtype udtype,
                                      long long count, const float* g, void* G, void* stream) {
  if (count < 0 || count % 4 != 0 || (count > 0 && (!U || !g || !G))) return OS3D_EINVAL;
  if (udtype != OS3D_U_C64 && udtype != OS3D_U_BF16X2) return OS3D_EINVAL;
  if (((reinterpret_cast<uintptr_t>(U) | reinterpret_cast<uintptr_t>(w) |
        reinterpret_cast<uintptr_t>(G)) & 15) || (reinterpret_cast<uintptr_t>(g) & 3))
    return OS3D_EINVAL;
  if (count == 0) return OS3D_OK;
  cudaStream_t s = (cudaStream_t)stream;
  OS3D_CK(counted_launch(OS3D_KIND_ENERGY_GRAD, s, [&] {
    return launch_energy_grad(U, w, udtype == OS3D_U_BF16X2, count, g, G, s);
  }));
  return OS3D_OK;
}

os3d_status os3d_default_diffusion(os3d_diffusion* d) {
  if (!d) return OS3D_EINVAL;
  d->t = 10.0;
  d->steps = 8;
  d->D11 = 0.0;
  d->D33 = 1.0;
  d->D44 = 0.01;
  d->sh_degree = 0;
  return OS3D_OK;
}

os3d_status os3d_angular_propagator(const double* orient, int n, int sh_degree, double tau,
                                    double* E, int* degree_used) {
  if (!orient || !E || n < 1 || !(tau >= 0.0) || !std::isfinite(tau) || sh_degree < 0 ||
      sh_degree > 15)
    return OS3D_EINVAL;
  std::vector<double> e;
  const int l = angular_propagator(orient, n, sh_degree, tau, e);
  if (l < 0) return OS3D_EINVAL;
  std::copy(e.begin(), e.end(), E);
  if (degree_used) *degree_used = l;
  return OS3D_OK;
}

os3d_status os3d_enhance_linear(const os3d_bank* b, const float* f, int batch, float* f_out,
                                const os3d_diffusion* d, void* ws, void* stream) {
  const os3d_status st = check_call(b, f, f_out, batch, OS3D_U_C64, ws);
  if (st != OS3D_OK) return st;
  if (!d) return OS3D_EINVAL;
  auto ok = [](double x) { return std::isfinite(x) && x >= 0.0; };
  if (!ok(d->t) || !ok(d->D11) || !ok(d->D33) || !ok(d->D44) || d->steps < 1 ||
      d->steps > 4096 || d->sh_degree < 0 || d->sh_degree > 15)
    return OS3D_EINVAL;
  const bool tensor = b->n_o > kMaxOrientE;
  if (tensor && tc_padded_orientations(b->n_o) < 0) return OS3D_EUNSUPPORTED;
  const double dt = d->t / d->steps;
  if (tensor) return enhance_tensor(b, f, batch, f_out, d, dt * d->D44, ws, (cudaStream_t)stream);
  std::vector<double> E;
  if (angular_propagator(b->orient.data(), b->n_o, d->sh_degree, dt * d->D44, E) < 0)
    return OS3D_EINVAL;
  static thread_local EnhanceArgs e;   // ~20 KB: kept off the stack
  e = EnhanceArgs{};
  e.nz = b->dims[0];
  e.ny = b->dims[1];
  e.nx = b->dims[2];
  e.wz = float(2.0 * kPi / b->dims[0]);
  e.wy = float(2.0 * kPi / b->dims[1]);
  e.wx = float(2.0 * kPi / b->dims[2]);
  e.n3 = float(b->nvox);
  e.n_o = b->n_o;
  e.steps = d->steps;
  e.half_dt = float(0.5 * dt);
  e.D11 = float(d->D11);
  e.D33 = float(d->D33);
  // an antipodally closed set as its pairs (E = [[A, B], [B, A]]; the kernel
  // takes C = A + B and D = A - B), else the full propagator
  const int np2 = b->n_o / 2;
  const int pb = b->mirror ? enhance_pair_block(b->n_o) : -1;
  e.paired = pb > 0 && (int)b->slot_a.size() == np2;
  if (e.paired) {
    for (int i = 0; i < np2; ++i) {
      const int ai = b->slot_a[i];
      for (int q = 0; q < 3; ++q) e.nvec[i][q] = float(b->orient[3 * ai + q]);
      for (int j = 0; j < np2; ++j) {
        const double A = E[(size_t)ai * b->n_o + b->slot_a[j]];
        const double B = E[(size_t)ai * b->n_o + b->slot_b[j]];
        e.Et[j * kEStride + i] = float(A + B);
        e.Et[(pb + j) * kEStride + pb + i] = float(A - B);
      }
    }
  } else {
    for (int i = 0; i < b->n_o; ++i) {
      for (int q = 0; q < 3; ++q) e.nvec[i][q] = float(b->orient[3 * i + q]);
      for (int j = 0; j < b->n_o; ++j) e.Et[j * kEStride + i] = float(E[(size_t)i * b->n_o + j]);
    }
  }
  e.h = b->h;
  cudaStream_t s = (cudaStream_t)stream;
  Work w;
  if (const os3d_status we = workspace_for(b, ws, &w)) return we;
  e.fh = w.fh;
  e.A = w.A[0];
  e.seg = b->seg;
  e.nseg = b->nseg;
  e.n_in = b->n_in;
  e.mirror = b->mirror;
  for (int v = 0; v < batch; ++v) {
    os3d_status r = prep_fhat(b, f, v, w, s);
    if (r != OS3D_OK) return r;
    OS3D_CK(cudaMemsetAsync(w.A[0], 0, sizeof(float2) * b->nvox, s));
    if (b->n_in > 0)
      OS3D_CK(counted_launch(OS3D_KIND_ENHANCE, s, [&] { return launch_enhance(e, b->ev, s); }));
    r = finish_real(b, w, 1, b->GM, f_out, v, s);
    if (r != OS3D_OK) return r;
  }
  return OS3D_OK;
}

os3d_status os3d_upsilon(const os3d_bank* b, const float* f, int batch, float* f_out,
                         double power, void* ws, void* stream) {
  const os3d_status st = check_call(b, f, f_out, batch, OS3D_U_C64, ws);
  if (st != OS3D_OK) return st;
  if (!(power > 0.0) || !std::isfinite(power)) return OS3D_EINVAL;
  return upsilon_impl(b, f, batch, f_out, (float)power, ws, (cudaStream_t)stream);
}

}  // extern "C"

// ===========================================================================
// Forward transform with its scratch in a fixed static device array.
//
// For callers that cannot allocate device memory when they run the
// transform: a process whose device memory belongs to a framework's pool
// allocator it may not bypass, or a latency-critical loop in which a
// cudaMalloc (which can synchronise the device) is not acceptable. The
// scratch lives in g_static_scratch below, a file-scope __device__ array of
// OS3D_STATIC_MAX_VOXELS x 3 complex values (6 MiB) that every GPU which
// loads this library holds until the process exits. Its device address is
// looked up on the first call made in each CUDA context of a device (the
// context's unique id is kept with the address, so a context created anew,
// e.g. after cudaDeviceReset, gets a fresh lookup); that first call must
// therefore come before any stream capture.
// ===========================================================================
namespace {

constexpr long long kStaticMaxVoxels = OS3D_STATIC_MAX_VOXELS;
// f_hat, one per-volume intermediate and one block intermediate (one pair)
static __device__ __align__(256) float2 g_static_scratch[3 * kStaticMaxVoxels];

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kStaticMaxDevices] = {};
unsigned long long g_static_ctx[kStaticMaxDevices] = {};   // context id of each address

// Unique id (driver API cuCtxGetId, reached through the runtime's entry-point
// query, so no link against the driver library) of the current context; 0
// when it cannot be determined.
unsigned long long current_context_id() {
  using GetCurrent = int (*)(void**);
  using GetId = int (*)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* a = nullptr;
    void* b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) ==
            cudaSuccess && qa == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) ==
            cudaSuccess && qb == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<GetCurrent>(a);
      get_id = reinterpret_cast<GetId>(b);
    }
    cudaGetLastError();
  });
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// device address of g_static_scratch in the current context
os3d_status static_scratch_address(float2** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices)
    return OS3D_ECUDA;
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev] || ctx == 0 || g_static_ctx[dev] != ctx) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return OS3D_ECUDA;
    }
    g_static_ptr[dev] = p;
    g_static_ctx[dev] = ctx;
  }
  *out = static_cast<float2*>(g_static_ptr[dev]);
  return OS3D_OK;
}

}  // namespace

extern "C" {

os3d_status os3d_forward_static(const os3d_bank* b, const float* f, int batch, void* U,
                                os3d_udtype udtype, void* stream) {
  const os3d_status st = check_call(b, f, U, batch, udtype, nullptr);
  if (st != OS3D_OK) return st;
  if (b->nvox > kStaticMaxVoxels) return OS3D_EINVAL;   // larger than the static scratch
  float2* scratch = nullptr;
  const os3d_status sa = static_scratch_address(&scratch);
  if (sa != OS3D_OK) return sa;
  // every scratch element is written before it is read within a call, so no
  // clearing is needed between calls
  float2* fh = scratch;
  float2* T0 = scratch + b->nvox;
  float2* T = scratch + 2 * b->nvox;
  cudaStream_t s = (cudaStream_t)stream;
  const int nz = b->dims[0], ny = b->dims[1], nx = b->dims[2];
  const int nslots = (int)b->slot_a.size();
  const int tiles = ny * (nx / kTileX);
  const long long n = b->nvox;
  for (int v = 0; v < batch; ++v) {
    PassArgs x0 = args_base(b);
    x0.in = f;
    x0.in_off = (long long)v * n;
    x0.out = T0;
    OS3D_CK(counted_launch(OS3D_KIND_XY_FWD_REAL, s,
                           [&] { return launch_plane(b, XY_FWD_REAL, 0, x0, s); }));
    PassArgs zp = args_base(b);
    zp.in = T0;
    zp.out = fh;
    zp.mult = b->Gs;
    OS3D_CK(counted_launch(OS3D_KIND_Z_FWD_PREP, s,
                           [&] { return launch_z(nz, Z_FWD_PREP, 0, zp, tiles, s); }));
    for (int s0 = 0; s0 < nslots; ++s0) {   // one orientation pair at a time
      PassArgs za = args_base(b);
      set_slots(b, za, v, s0, 1);
      za.in = fh;
      za.out = T;
      OS3D_CK(counted_launch(OS3D_KIND_Z_FWD_SCORE, s,
                             [&] { return launch_z(nz, Z_FWD_SCORE, b->ev, za, tiles, s); }));
      PassArgs xa = za;
      xa.in = T;
      xa.out = U;
      OS3D_CK(counted_launch(OS3D_KIND_XY_FWD_SCORE, s,
                             [&] { return launch_plane(b, XY_FWD_SCORE, udtype, xa, s); }));
    }
  }
  return OS3D_OK;
}

}  // extern "C"

extern "C" {

unsigned long long os3d_launch_count(void) { return g_launches.load(); }

os3d_status os3d_wait_selftest(double limit_s, int arrive, unsigned* timeouts) {
  if (!timeouts || !(limit_s > 0.0) || limit_s > 10.0) return OS3D_EINVAL;
  unsigned* d = nullptr;
  if (cudaMalloc(&d, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    return OS3D_ENOMEM;
  }
  os3d_status st = OS3D_OK;
  if (cudaMemset(d, 0, sizeof(unsigned)) != cudaSuccess ||
      launch_wait_selftest((unsigned long long)(limit_s * 1e9), arrive ? 1 : 0, d, nullptr) !=
          cudaSuccess ||
      cudaMemcpy(timeouts, d, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
    st = OS3D_ECUDA;
  cudaFree(d);
  return st;
}

os3d_status os3d_profile_enable(int on) {
  g_profile.store(on ? 1 : 0);
  return OS3D_OK;
}

os3d_status os3d_profile_read(int kind, unsigned long long* launches, double* ms) {
  if (kind < 0 || kind >= OS3D_KIND_COUNT) return OS3D_EINVAL;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (const auto& r : g_prof_pending) {
    float t = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess)
      return OS3D_ECUDA;
    g_prof_launches[r.kind] += 1;
    g_prof_ms[r.kind] += t;
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_prof_pending.clear();
  if (launches) *launches = g_prof_launches[kind];
  if (ms) *ms = g_prof_ms[kind];
  return OS3D_OK;
}

os3d_status os3d_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (int k = 0; k < OS3D_KIND_COUNT; ++k) {
    g_prof_launches[k] = 0;
    g_prof_ms[k] = 0.0;
  }
  for (const auto& r : g_prof_pending) {
    cudaEventSynchronize(r.b);
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_prof_pending.clear();
  return OS3D_OK;
}

const char* os3d_kernel_kind_name(int kind) {
  static const char* names[OS3D_KIND_COUNT] = {
      "xy_fwd_real", "xy_fwd_score", "xy_inv_score", "xy_inv_real", "z_fwd_prep", "z_fwd_score",
      "z_inv_score", "z_inv_final", "xy_soft", "approx_sum", "soft_threshold", "enhance_linear",
      "weighted_energy", "weighted_energy_grad"};
  return (kind >= 0 && kind < OS3D_KIND_COUNT) ? names[kind] : "unknown";
}

}  // extern "C"
