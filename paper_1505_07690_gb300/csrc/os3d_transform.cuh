// Fused FFT passes of the orientation-score transform (sm_103a).
//
// The 3D DFT of every orientation is split into two passes so that only U
// touches HBM:
//   * z-pass: DFT along z of 16-wide pencil tiles, fused with the wavelet
//     evaluation psi_hat_a = G(|w|) h(w_hat . n_a) (G is folded into the
//     per-volume factors) and, in the inverse, with the orientation sum;
//   * xy-pass: 2D DFT of one z-plane in shared memory, fused with the U
//     store (forward; U_a and its antipode U_b = conj(U_a) for a real image)
//     or the U load (inverse; P = U_a + conj(U_b)).
// Per orientation pair the intermediate volume T stays L2-resident.
//
// Forward (Eq. construction1Discrete): U_a = IDFT[ f_hat G h_a ].
// Inverse (Eq. Reconstruction1Discrete with the Sec. 3.1 clamp): for a real
// image only the Hermitian part of sum_i psi_hat_i DFT(U_i) matters, and
// with psi_hat_{-n}(w) = psi_hat_n(-w) the pair (a, b = -a) contributes
// Herm[ G h_a DFT(U_a + conj U_b) ]; hence
//   f = Re IDFT[ G / max(M, eps) * sum_slots h_a DFT(U_a + conj U_b) ].
#pragma once
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <algorithm>
#include "os3d_fft.cuh"
#include "os3d_kernels.cuh"

namespace os3d {

__device__ __forceinline__ int signed_index(int k, int n) { return k >= (n + 1) / 2 ? k - n : k; }

// Angular profile h at t = w_hat . n. EV 0 / 1: h(t) = E(v) + t O(v), v = t^2 - 1/2,
// E and O in the monomial basis of v evaluated by Horner's rule (9 + 8 or
// 13 + 12 coefficients); chosen on the host only when the coefficients show
// no cancellation. EV 2: sum_{j<=32} a_j T_j(t) by Clenshaw's recurrence.
template <int EV>
__device__ __forceinline__ float eval_h(const HEval& h, float t) {
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
    return fmaf(t, o, e);
  } else {
    float b1 = 0.f, b2 = 0.f;
    const float t2 = t + t;
#pragma unroll
    for (int j = kMaxL; j >= 1; --j) {
      const float b0 = fmaf(t2, b1, h.a[j] - b2);
      b2 = b1;
      b1 = b0;
    }
    return fmaf(t, b1, h.a[0] - b2);
  }
}

// ----------------------------------------------------------------------------
// z-pass
// ----------------------------------------------------------------------------
template <int NZ, int MODE, int EV>
__global__ void __launch_bounds__(kTileX * Plan<NZ>::R2)
z_kernel(const __grid_constant__ ZArgs a) {
  constexpr int R1 = Plan<NZ>::R1, R2 = Plan<NZ>::R2;
  constexpr int TW = kTileX;
  constexpr int J3 = (R1 + R2 - 1) / R2;   // step-2 items per thread (k1 = n2 + R2 j < R1)
  constexpr int DIR = (MODE == Z_FWD_PREP || MODE == Z_INV_SCORE) ? -1 : +1;

  __shared__ float2 tile[NZ * TW];
  __shared__ float2 tws[NZ];

  const int t = threadIdx.x;
  const int xl = t % TW, n2 = t / TW;
  const int tiles_x = a.nx / TW;
  const int y = blockIdx.x / tiles_x;
  const int x = (blockIdx.x % tiles_x) * TW + xl;
  const long long plane = (long long)a.ny * a.nx;
  const long long col = (long long)y * a.nx + x;

  fill_twiddles<NZ, DIR>(tws);
  __syncthreads();
  float2 tw[R1];
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) tw[k1] = tws[(n2 * k1) % NZ];

  const float wy = float(signed_index(y, a.ny)) * a.wy;
  const float wx = float(signed_index(x, a.nx)) * a.wx;
  const float rxy2 = fmaf(wy, wy, wx * wx);
  const bool dc_col = (y == 0) && (x == 0) && (n2 == 0);

  // step 1 (R1-point DFT of the thread's stride-R2 elements) + twiddle + store
  auto step1_store = [&](float2 (&v)[R1]) {
    dft<R1, DIR>(v);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      const float2 w = (k1 == 0) ? v[k1] : cmul(v[k1], tw[k1]);
      tile[(n2 + R2 * k1) * TW + xl] = w;
    }
  };
  // step 2 (R2-point DFT over n2 for k1 = n2 + R2 j)
  auto step2_load = [&](int j, float2 (&w)[R2]) {
    const int k1 = n2 + R2 * j;
#pragma unroll
    for (int m = 0; m < R2; ++m) w[m] = tile[(m + R2 * k1) * TW + xl];
    dft<R2, DIR>(w);
  };

  if constexpr (MODE == Z_FWD_PREP) {
    float2 v[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) v[n1] = a.in[(long long)(n2 + R2 * n1) * plane + col];
    step1_store(v);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < J3; ++j) {
      const int k1 = n2 + R2 * j;
      if (R1 % R2 != 0 && k1 >= R1) break;
      float2 w[R2];
      step2_load(j, w);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        const long long o = (long long)(k1 + R1 * k2) * plane + col;
        a.out[o] = cscale(w[k2], a.mult[o]);
      }
    }
  } else if constexpr (MODE == Z_INV_FINAL) {
    float2 v[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      const long long o = (long long)(n2 + R2 * n1) * plane + col;
      v[n1] = cscale(a.in[o], a.mult[o]);
    }
    step1_store(v);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < J3; ++j) {
      const int k1 = n2 + R2 * j;
      if (R1 % R2 != 0 && k1 >= R1) break;
      float2 w[R2];
      step2_load(j, w);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) a.out[(long long)(k1 + R1 * k2) * plane + col] = w[k2];
    }
  } else if constexpr (MODE == Z_FWD_SCORE) {
    // geometry of the step-1 input frequencies k_z = n2 + R2 n1
    float fr[R1], fi[R1], ur[R1], rr[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      const int kz = n2 + R2 * n1;
      const float2 f = a.in[(long long)kz * plane + col];
      fr[n1] = f.x;
      fi[n1] = f.y;
      const float wz = float(signed_index(kz, NZ)) * a.wz;
      const float r2 = fmaf(wz, wz, rxy2);
      const float ri = r2 > 0.f ? rsqrtf(r2) : 0.f;
      ur[n1] = wz * ri;
      rr[n1] = ri;
    }
    for (int s = 0; s < a.nslots; ++s) {
      const float dxy = fmaf(wx, a.nvec[s][0], wy * a.nvec[s][1]);
      const float nz = a.nvec[s][2];
      float2 v[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) {
        float h = eval_h<EV>(a.h, fmaf(rr[n1], dxy, ur[n1] * nz));
        if (n1 == 0 && dc_col) h = a.h.c0;
        v[n1] = make_float2(fr[n1] * h, fi[n1] * h);
      }
      step1_store(v);
      __syncthreads();
      float2* out = a.out + (long long)s * a.slot_stride;
#pragma unroll
      for (int j = 0; j < J3; ++j) {
        const int k1 = n2 + R2 * j;
        if (R1 % R2 != 0 && k1 >= R1) break;
        float2 w[R2];
        step2_load(j, w);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) out[(long long)(k1 + R1 * k2) * plane + col] = w[k2];
      }
      __syncthreads();
    }
  } else {  // Z_INV_SCORE
    // geometry of the step-2 output frequencies k_z = k1 + R1 k2
    float ur[J3 * R2], rr[J3 * R2];
    float2 acc[J3 * R2];
#pragma unroll
    for (int j = 0; j < J3; ++j) {
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        const int kz = min(n2 + R2 * j, R1 - 1) + R1 * k2;
        const float wz = float(signed_index(kz, NZ)) * a.wz;
        const float r2 = fmaf(wz, wz, rxy2);
        const float ri = r2 > 0.f ? rsqrtf(r2) : 0.f;
        ur[j * R2 + k2] = wz * ri;
        rr[j * R2 + k2] = ri;
        acc[j * R2 + k2] = make_float2(0.f, 0.f);
      }
    }
    for (int s = 0; s < a.nslots; ++s) {
      const float2* in = a.in + (long long)s * a.slot_stride;
      float2 v[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) v[n1] = in[(long long)(n2 + R2 * n1) * plane + col];
      step1_store(v);
      __syncthreads();
      const float dxy = fmaf(wx, a.nvec[s][0], wy * a.nvec[s][1]);
      const float nz = a.nvec[s][2];
#pragma unroll
      for (int j = 0; j < J3; ++j) {
        if (R1 % R2 != 0 && n2 + R2 * j >= R1) break;
        float2 w[R2];
        step2_load(j, w);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          const int p = j * R2 + k2;
          float h = eval_h<EV>(a.h, fmaf(rr[p], dxy, ur[p] * nz));
          if (p == 0 && dc_col) h = a.h.c0;
          acc[p].x = fmaf(h, w[k2].x, acc[p].x);
          acc[p].y = fmaf(h, w[k2].y, acc[p].y);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < J3; ++j) {
      if (R1 % R2 != 0 && n2 + R2 * j >= R1) break;
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        const long long o = (long long)(n2 + R2 * j + R1 * k2) * plane + col;
        float2 r = acc[j * R2 + k2];
        if (a.accumulate) r = cadd(r, a.out[o]);
        a.out[o] = r;
      }
    }
  }
}

// ----------------------------------------------------------------------------
// xy-pass: 2D DFT of one (ny, nx) plane held in shared memory. Persistent:
// each CTA walks the planes blockIdx.x, blockIdx.x + gridDim.x, ...
// Shared layout: row pitch P = nx + 8 (rows alternate 64-byte halves of the
// bank space) and, inside each aligned group of R2x columns, the column index
// XOR-ed with the group index, so that the row-contiguous step-2 reads, the
// strided step-1 writes and the column accesses are all conflict-free.
// ----------------------------------------------------------------------------
template <int NY, int NX>
struct XYCfg {
  static constexpr int R1x = Plan<NX>::R1, R2x = Plan<NX>::R2;
  static constexpr int R1y = Plan<NY>::R1, R2y = Plan<NY>::R2;
  static_assert((R2x & (R2x - 1)) == 0, "R2x must be a power of two");
  static constexpr bool ok(int nt) {
    return nt % 32 == 0 && (NY * R2x) % nt == 0 && nt % R2x == 0 && (NY * R1x) % nt == 0 &&
           nt % R2y == 0 && NX % (nt / R2y) == 0 && (NX * R1y) % nt == 0;
  }
  static constexpr int pick() {
    for (int nt = 512; nt >= 32; nt -= 32)
      if (ok(nt)) return nt;
    return 0;
  }
  static constexpr int NT = pick();
  static_assert(NT > 0, "no thread count fits this plane");
  static constexpr int P = NX + 8;
  static constexpr int JX1 = NY * R2x / NT;
  static constexpr int JX3 = NY * R1x / NT;
  static constexpr int CW = NT / R2y;
  static constexpr int JY1 = NX / CW;
  static constexpr int JY3 = NX * R1y / NT;
  static constexpr size_t smem_bytes = sizeof(float2) * (size_t(NY) * P + NX + NY);
  static __device__ __forceinline__ int phys(int r, int x) {
    return r * P + (x ^ ((x / R2x) & (R2x - 1)));
  }
  // x step-2 item j of thread t: row r and frequency k1
  static __device__ __forceinline__ void x2_item(int t, int j, int& r, int& k1) {
    const int lane = t & 31, w = t >> 5;
    if constexpr (R1x == 16 && R2x == 8 && NT % 32 == 0 && (NY / 2) % (NT / 32) == 0) {
      k1 = (lane & 7) + 8 * (lane >> 4);
      r = 2 * (w + (NT / 32) * j) + ((lane >> 3) & 1);
    } else if constexpr (R1x == 8 && R2x == 8 && (NY / 4) % (NT / 32) == 0) {
      k1 = lane & 7;
      r = 4 * (w + (NT / 32) * j) + (lane >> 3);
    } else {
      const int q = t + NT * j;
      r = q / R1x;
      k1 = q % R1x;
    }
  }
};

template <int UBF16>
__device__ __forceinline__ float2 load_u(const void* base, long long i) {
  if constexpr (UBF16) {
    const unsigned int raw = __ldcs(reinterpret_cast<const unsigned int*>(base) + i);
    __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&raw);
    return __bfloat1622float2(b);
  } else {
    return __ldcs(reinterpret_cast<const float2*>(base) + i);
  }
}
template <int UBF16>
__device__ __forceinline__ void store_u(void* base, long long i, float2 v) {
  if constexpr (UBF16) {
    __nv_bfloat162 b = __floats2bfloat162_rn(v.x, v.y);
    __stcs(reinterpret_cast<unsigned int*>(base) + i, *reinterpret_cast<unsigned int*>(&b));
  } else {
    __stcs(reinterpret_cast<float2*>(base) + i, v);
  }
}

template <int NY, int NX, int MODE, int UBF16>
__global__ void __launch_bounds__(XYCfg<NY, NX>::NT, 1)
xy_kernel(const __grid_constant__ XYArgs a) {
  using C = XYCfg<NY, NX>;
  constexpr int R1x = C::R1x, R2x = C::R2x, R1y = C::R1y, R2y = C::R2y;
  constexpr int NT = C::NT;
  constexpr int DIR = (MODE == XY_FWD_REAL || MODE == XY_INV_SCORE) ? -1 : +1;

  extern __shared__ float2 sm[];
  float2* plane = sm;
  float2* twx = sm + NY * C::P;
  float2* twy = twx + NX;

  const int t = threadIdx.x;
  const long long P = (long long)NY * NX;

  fill_twiddles<NX, DIR>(twx);
  fill_twiddles<NY, DIR>(twy);
  __syncthreads();
  const int n2x = t % R2x, r0x = t / R2x;
  float2 twr[R1x];
#pragma unroll
  for (int k1 = 0; k1 < R1x; ++k1) twr[k1] = twx[(n2x * k1) % NX];

  for (int p = blockIdx.x; p < a.nplanes; p += gridDim.x) {
    const int s = p / a.nz, z = p - s * a.nz;
    const long long zoff = (long long)z * P;
    // ---- x direction, step 1: global -> registers -> DFT_R1 -> shared
    {
      const long long ia = a.in_a[s] + zoff;
      const long long ib = a.in_b[s] + zoff;
#pragma unroll
      for (int j = 0; j < C::JX1; ++j) {
        const int r = r0x + (NT / R2x) * j;
        float2 v[R1x];
#pragma unroll
        for (int n1 = 0; n1 < R1x; ++n1) {
          const long long e = (long long)r * NX + n2x + R2x * n1;
          if constexpr (MODE == XY_FWD_REAL) {
            v[n1] = make_float2(__ldg(reinterpret_cast<const float*>(a.in) + ia + e), 0.f);
          } else if constexpr (MODE == XY_INV_SCORE) {
            float2 u = load_u<UBF16>(a.in, ia + e);
            if (a.in_b[s] >= 0) u = cadd(u, cconj(load_u<UBF16>(a.in, ib + e)));
            v[n1] = u;
          } else {
            v[n1] = reinterpret_cast<const float2*>(a.in)[ia + e];
          }
        }
        dft<R1x, DIR>(v);
#pragma unroll
        for (int k1 = 0; k1 < R1x; ++k1)
          plane[C::phys(r, n2x + R2x * k1)] = (k1 == 0) ? v[k1] : cmul(v[k1], twr[k1]);
      }
    }
    __syncthreads();
    // ---- x direction, step 2
    {
      float2 w[C::JX3][R2x];
#pragma unroll
      for (int j = 0; j < C::JX3; ++j) {
        int r, k1;
        C::x2_item(t, j, r, k1);
#pragma unroll
        for (int m = 0; m < R2x; ++m) w[j][m] = plane[C::phys(r, m + R2x * k1)];
        dft<R2x, DIR>(w[j]);
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < C::JX3; ++j) {
        int r, k1;
        C::x2_item(t, j, r, k1);
#pragma unroll
        for (int k2 = 0; k2 < R2x; ++k2) plane[C::phys(r, k1 + R1x * k2)] = w[j][k2];
      }
    }
    __syncthreads();
    // ---- y direction, step 1 (in place, item-private positions)
    {
      const int n2 = t / C::CW;
      float2 tw[R1y];
#pragma unroll
      for (int k1 = 0; k1 < R1y; ++k1) tw[k1] = twy[(n2 * k1) % NY];
#pragma unroll
      for (int j = 0; j < C::JY1; ++j) {
        const int c = t % C::CW + C::CW * j;
        float2 u[R1y];
#pragma unroll
        for (int n1 = 0; n1 < R1y; ++n1) u[n1] = plane[C::phys(n2 + R2y * n1, c)];
        dft<R1y, DIR>(u);
#pragma unroll
        for (int k1 = 0; k1 < R1y; ++k1)
          plane[C::phys(n2 + R2y * k1, c)] = (k1 == 0) ? u[k1] : cmul(u[k1], tw[k1]);
      }
    }
    __syncthreads();
    // ---- y direction, step 2 + store
    {
      const long long oa = a.out_a[s] + zoff;
      const long long ob = a.out_b[s] + zoff;
#pragma unroll
      for (int j = 0; j < C::JY3; ++j) {
        const int q = t + NT * j;
        const int c = q % NX, k1 = q / NX;
        float2 w[R2y];
#pragma unroll
        for (int m = 0; m < R2y; ++m) w[m] = plane[C::phys(m + R2y * k1, c)];
        dft<R2y, DIR>(w);
#pragma unroll
        for (int k2 = 0; k2 < R2y; ++k2) {
          const long long e = (long long)(k1 + R1y * k2) * NX + c;
          if constexpr (MODE == XY_FWD_SCORE) {
            store_u<UBF16>(a.out, oa + e, w[k2]);
            if (a.out_b[s] >= 0) store_u<UBF16>(a.out, ob + e, cconj(w[k2]));
          } else if constexpr (MODE == XY_INV_REAL) {
            reinterpret_cast<float*>(a.out)[oa + e] = w[k2].x;
          } else {
            reinterpret_cast<float2*>(a.out)[oa + e] = w[k2];
          }
        }
      }
    }
    __syncthreads();   // the plane buffer is rewritten by the next plane
  }
}

// ----------------------------------------------------------------------------
// xy-pass on a 2-CTA cluster: CTA h of the pair holds rows [h NY/2, (h+1) NY/2)
// for the x direction and columns [h NX/2, (h+1) NX/2) for the y direction.
// The x step-2 outputs are written straight into the owner's y-layout buffer
// (local or distributed shared memory), so the transpose costs no extra pass,
// and a half plane (74 KB at 128^2) lets two clusters share an SM.
// ----------------------------------------------------------------------------
template <int NY, int NX>
struct XY2Cfg {
  static constexpr int NYH = NY / 2, NXH = NX / 2;
  static constexpr int R1x = Plan<NX>::R1, R2x = Plan<NX>::R2;
  static constexpr int R1y = Plan<NY>::R1, R2y = Plan<NY>::R2;
  static_assert((R2x & (R2x - 1)) == 0, "R2x must be a power of two");
  static constexpr bool ok(int nt) {
    return nt % 32 == 0 && (NYH * R2x) % nt == 0 && nt % R2x == 0 && (NYH * R1x) % nt == 0 &&
           nt % R2y == 0 && NXH % (nt / R2y) == 0 && (NXH * R1y) % nt == 0;
  }
  static constexpr int pick() {
    for (int nt = 256; nt >= 32; nt -= 32)
      if (ok(nt)) return nt;
    return 0;
  }
  static constexpr int NT = pick();
  static_assert(NT > 0, "no thread count fits this half plane");
  static constexpr int PX = NX + 8;    // x layout: NYH rows of NX (swizzled) columns
  static constexpr int PY = NXH + 8;   // y layout: NY rows of NXH columns
  static constexpr int BUF = (NYH * PX > NY * PY) ? NYH * PX : NY * PY;
  static constexpr int JX1 = NYH * R2x / NT;
  static constexpr int JX3 = NYH * R1x / NT;
  static constexpr int CW = NT / R2y;
  static constexpr int JY1 = NXH / CW;
  static constexpr int JY3 = NXH * R1y / NT;
  static constexpr size_t smem_bytes = sizeof(float2) * (size_t(BUF) + NX + NY);
  static __device__ __forceinline__ int xphys(int r, int x) {
    return r * PX + (x ^ ((x / R2x) & (R2x - 1)));
  }
  static __device__ __forceinline__ void x2_item(int t, int j, int& r, int& k1) {
    const int lane = t & 31, w = t >> 5;
    if constexpr (R1x == 16 && R2x == 8 && (NYH / 2) % (NT / 32) == 0) {
      k1 = (lane & 7) + 8 * (lane >> 4);
      r = 2 * (w + (NT / 32) * j) + ((lane >> 3) & 1);
    } else if constexpr (R1x == 8 && R2x == 8 && (NYH / 4) % (NT / 32) == 0) {
      k1 = lane & 7;
      r = 4 * (w + (NT / 32) * j) + (lane >> 3);
    } else {
      const int q = t + NT * j;
      r = q / R1x;
      k1 = q % R1x;
    }
  }
};

// 32-bit shared-memory address of a generic pointer into this CTA's shared memory
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
// the same offset in the shared memory of CTA `rank` of this cluster
__device__ __forceinline__ unsigned map_cluster_rank(unsigned a, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster_f2(unsigned addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y)
               : "memory");
}

template <int NY, int NX, int MODE, int UBF16>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(XY2Cfg<NY, NX>::NT, 2)
xy2_kernel(const __grid_constant__ XYArgs a) {
  namespace cg = cooperative_groups;
  using C = XY2Cfg<NY, NX>;
  constexpr int R1x = C::R1x, R2x = C::R2x, R1y = C::R1y, R2y = C::R2y;
  constexpr int NT = C::NT, NYH = C::NYH, NXH = C::NXH;
  constexpr int DIR = (MODE == XY_FWD_REAL || MODE == XY_INV_SCORE) ? -1 : +1;

  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ float2 sm[];
  float2* buf = sm;
  float2* twx = sm + C::BUF;
  float2* twy = twx + NX;
  const int h = (int)cluster.block_rank();
  const unsigned peer_base = map_cluster_rank(smem_addr(buf), (unsigned)(h ^ 1));

  const int t = threadIdx.x;
  const long long P = (long long)NY * NX;
  fill_twiddles<NX, DIR>(twx);
  fill_twiddles<NY, DIR>(twy);
  __syncthreads();
  const int n2x = t % R2x, r0x = t / R2x;

  const int cl = blockIdx.x / 2, ncl = gridDim.x / 2;
  for (int p = cl; p < a.nplanes; p += ncl) {
    const int s = p / a.nz, z = p - s * a.nz;
    const long long zoff = (long long)z * P;
    // ---- x direction, step 1 on this CTA's rows
    {
      const long long ia = a.in_a[s] + zoff;
      const long long ib = a.in_b[s] + zoff;
      float2 tw[R1x];
#pragma unroll
      for (int k1 = 0; k1 < R1x; ++k1) tw[k1] = twx[(n2x * k1) % NX];
#pragma unroll
      for (int j = 0; j < C::JX1; ++j) {
        const int r = r0x + (NT / R2x) * j;
        const long long row = (long long)(h * NYH + r) * NX;
        float2 v[R1x];
#pragma unroll
        for (int n1 = 0; n1 < R1x; ++n1) {
          const long long e = row + n2x + R2x * n1;
          if constexpr (MODE == XY_FWD_REAL) {
            v[n1] = make_float2(__ldg(reinterpret_cast<const float*>(a.in) + ia + e), 0.f);
          } else if constexpr (MODE == XY_INV_SCORE) {
            float2 u = load_u<UBF16>(a.in, ia + e);
            if (a.in_b[s] >= 0) u = cadd(u, cconj(load_u<UBF16>(a.in, ib + e)));
            v[n1] = u;
          } else {
            v[n1] = reinterpret_cast<const float2*>(a.in)[ia + e];
          }
        }
        dft<R1x, DIR>(v);
#pragma unroll
        for (int k1 = 0; k1 < R1x; ++k1)
          buf[C::xphys(r, n2x + R2x * k1)] = (k1 == 0) ? v[k1] : cmul(v[k1], tw[k1]);
      }
    }
    __syncthreads();
    // ---- x direction, step 2; outputs go to the owner of their column
    {
      float2 w[C::JX3][R2x];
#pragma unroll
      for (int j = 0; j < C::JX3; ++j) {
        int r, k1;
        C::x2_item(t, j, r, k1);
#pragma unroll
        for (int m = 0; m < R2x; ++m) w[j][m] = buf[C::xphys(r, m + R2x * k1)];
        dft<R2x, DIR>(w[j]);
      }
      cluster.sync();   // both halves have read their x-layout buffers
#pragma unroll
      for (int j = 0; j < C::JX3; ++j) {
        int r, k1;
        C::x2_item(t, j, r, k1);
        const int row = (h * NYH + r) * C::PY;
#pragma unroll
        for (int k2 = 0; k2 < R2x; ++k2) {
          const int c = k1 + R1x * k2;
          // column owner: compile-time when NX/2 is a multiple of R1x
          const int owner = (NXH % R1x == 0) ? (k2 >= NXH / R1x) : (c >= NXH);
          const int idx = row + c - owner * NXH;
          if (owner == h) buf[idx] = w[j][k2];
          else st_cluster_f2(peer_base + 8u * (unsigned)idx, w[j][k2]);
        }
      }
      cluster.sync();   // this CTA's y-layout buffer is complete
    }
    // ---- y direction, step 1 on this CTA's columns (in place)
    {
      const int n2 = t / C::CW;
      float2 tw[R1y];
#pragma unroll
      for (int k1 = 0; k1 < R1y; ++k1) tw[k1] = twy[(n2 * k1) % NY];
#pragma unroll
      for (int j = 0; j < C::JY1; ++j) {
        const int c = t % C::CW + C::CW * j;
        float2 u[R1y];
#pragma unroll
        for (int n1 = 0; n1 < R1y; ++n1) u[n1] = buf[(n2 + R2y * n1) * C::PY + c];
        dft<R1y, DIR>(u);
#pragma unroll
        for (int k1 = 0; k1 < R1y; ++k1)
          buf[(n2 + R2y * k1) * C::PY + c] = (k1 == 0) ? u[k1] : cmul(u[k1], tw[k1]);
      }
    }
    __syncthreads();
    // ---- y direction, step 2 + store
    {
      const long long oa = a.out_a[s] + zoff;
      const long long ob = a.out_b[s] + zoff;
#pragma unroll
      for (int j = 0; j < C::JY3; ++j) {
        const int q = t + NT * j;
        const int c = q % NXH, k1 = q / NXH;
        float2 w[R2y];
#pragma unroll
        for (int m = 0; m < R2y; ++m) w[m] = buf[(m + R2y * k1) * C::PY + c];
        dft<R2y, DIR>(w);
#pragma unroll
        for (int k2 = 0; k2 < R2y; ++k2) {
          const long long e = (long long)(k1 + R1y * k2) * NX + h * NXH + c;
          if constexpr (MODE == XY_FWD_SCORE) {
            store_u<UBF16>(a.out, oa + e, w[k2]);
            if (a.out_b[s] >= 0) store_u<UBF16>(a.out, ob + e, cconj(w[k2]));
          } else if constexpr (MODE == XY_INV_REAL) {
            reinterpret_cast<float*>(a.out)[oa + e] = w[k2].x;
          } else {
            reinterpret_cast<float2*>(a.out)[oa + e] = w[k2];
          }
        }
      }
    }
    __syncthreads();   // the buffer is rewritten by the next plane's x step 1
  }
  cluster.sync();      // no CTA leaves while its peer may still write into it
}

// ----------------------------------------------------------------------------
// per-size launchers
// ----------------------------------------------------------------------------
template <int NZ>
cudaError_t launch_z_n(int mode, int ev, const ZArgs& a, int grid, cudaStream_t s) {
  const dim3 block(kTileX * Plan<NZ>::R2);
  switch (mode) {
    case Z_FWD_PREP: z_kernel<NZ, Z_FWD_PREP, 0><<<grid, block, 0, s>>>(a); break;
    case Z_INV_FINAL: z_kernel<NZ, Z_INV_FINAL, 0><<<grid, block, 0, s>>>(a); break;
    case Z_FWD_SCORE:
      if (ev == 0) z_kernel<NZ, Z_FWD_SCORE, 0><<<grid, block, 0, s>>>(a);
      else if (ev == 1) z_kernel<NZ, Z_FWD_SCORE, 1><<<grid, block, 0, s>>>(a);
      else z_kernel<NZ, Z_FWD_SCORE, 2><<<grid, block, 0, s>>>(a);
      break;
    case Z_INV_SCORE:
      if (ev == 0) z_kernel<NZ, Z_INV_SCORE, 0><<<grid, block, 0, s>>>(a);
      else if (ev == 1) z_kernel<NZ, Z_INV_SCORE, 1><<<grid, block, 0, s>>>(a);
      else z_kernel<NZ, Z_INV_SCORE, 2><<<grid, block, 0, s>>>(a);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int NY, int NX>
constexpr bool use_cluster_xy() {
  return NY == NX && NX >= 64;
}

template <int NY, int NX, int MODE, int UB>
cudaError_t launch_xy_one(const XYArgs& a, int nz, int nslots, cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  XYArgs b = a;
  b.nz = nz;
  b.nplanes = nz * nslots;
  if constexpr (use_cluster_xy<NY, NX>()) {
    using C = XY2Cfg<NY, NX>;
    auto k = xy2_kernel<NY, NX, MODE, UB>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::smem_bytes);
    if (e != cudaSuccess) return e;
    // two clusters (four CTAs of half a plane) per pair of SMs
    const int clusters = std::min(b.nplanes, std::max(nsm, 1));
    k<<<2 * clusters, C::NT, C::smem_bytes, s>>>(b);
  } else {
    using C = XYCfg<NY, NX>;
    auto k = xy_kernel<NY, NX, MODE, UB>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::smem_bytes);
    if (e != cudaSuccess) return e;
    const int grid = std::min(b.nplanes, std::max(nsm, 1));
    k<<<grid, C::NT, C::smem_bytes, s>>>(b);
  }
  return cudaGetLastError();
}

template <int NY, int NX>
cudaError_t launch_xy_n(int mode, int ubf16, const XYArgs& a, int nz, int nslots, cudaStream_t s) {
  switch (mode) {
    case XY_FWD_REAL: return launch_xy_one<NY, NX, XY_FWD_REAL, 0>(a, nz, nslots, s);
    case XY_INV_REAL: return launch_xy_one<NY, NX, XY_INV_REAL, 0>(a, nz, nslots, s);
    case XY_FWD_SCORE:
      return ubf16 ? launch_xy_one<NY, NX, XY_FWD_SCORE, 1>(a, nz, nslots, s)
                   : launch_xy_one<NY, NX, XY_FWD_SCORE, 0>(a, nz, nslots, s);
    case XY_INV_SCORE:
      return ubf16 ? launch_xy_one<NY, NX, XY_INV_SCORE, 1>(a, nz, nslots, s)
                   : launch_xy_one<NY, NX, XY_INV_SCORE, 0>(a, nz, nslots, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace os3d

// Per-size translation units instantiate these.
#define OS3D_DEFINE_Z(N)                                                                   \
  namespace os3d {                                                                         \
  cudaError_t launch_z_##N(int mode, int lpad, const ZArgs& a, int grid, cudaStream_t s) { \
    return launch_z_n<N>(mode, lpad, a, grid, s);                                          \
  }                                                                                        \
  }
#define OS3D_DEFINE_XY(NY, NX)                                                             \
  namespace os3d {                                                                         \
  cudaError_t launch_xy_##NY##_##NX(int mode, int ub, const XYArgs& a, int nz, int ns,     \
                                    cudaStream_t s) {                                      \
    return launch_xy_n<NY, NX>(mode, ub, a, nz, ns, s);                                    \
  }                                                                                        \
  }
