// Fused DFT passes of the orientation-score transform (sm_103a).
//
// The 3D DFT of every orientation is split into a z-pass (DFT along z of
// 16-wide pencil tiles) and an xy-pass (2D DFT of z-planes: a whole plane per
// CTA, or for 256^2 planes an 8-CTA cluster per plane; the forward score pass
// on 256^2 planes as four independent quarter-plane CTAs and on 128^2 planes
// with complex64 scores as two half-plane CTAs), with the per-orientation
// intermediate T passed through L2:
//   forward  (Eq. construction1Discrete):  U_a = IDFT_xy IDFT_z [ f_hat G h_a ]
//            z-pass : f_hat tile (read once per block) x h(w_hat . n_a) -> IDFT_z -> T_a
//            xy-pass: T_a -> IDFT_xy -> U_a and U_b = conj U_a           (HBM)
//   inverse  (Eq. Reconstruction1Discrete with the clamp of Sec. 3.1):
//            xy-pass: U_a + conj U_b (HBM) -> DFT_xy -> T_a
//            z-pass : T_a -> DFT_z -> x h(w_hat . n_a), summed over the block -> A
//            then f = Re IDFT[ A G / (n^3 max(M, eps)) ].
// For a real image U_{-n} = conj U_n, and the real reconstruction needs only
// the Hermitian part of sum_i psi_hat_i DFT(U_i), which for the pair
// (a, b = -a) is Herm[ G h_a DFT(U_a + conj U_b) ] (psi_hat_{-n}(w) =
// psi_hat_n(-w)); so one transform serves each antipodal pair.
#pragma once
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <algorithm>
#include "os3d_fft.cuh"
#include "os3d_kernels.cuh"

namespace os3d {

__device__ __forceinline__ int signed_index(int k, int n) { return k >= (n + 1) / 2 ? k - n : k; }

// True when every column (kx, ky) of the 16-wide z tile holding DFT index x
// lies strictly outside the disc |w_xy| < pi, where psi_hat vanishes for
// every kz: 4 (kx^2/nx^2 + ky^2/ny^2) > 1 for the tile's smallest |kx|
// (exact integer test; the boundary itself counts as inside).
__device__ __forceinline__ bool tile_outside(int x, int y, int nx, int ny) {
  const int x0 = x & ~(kTileX - 1);
  const int kx = x0 < (nx + 1) / 2 ? x0 : (x0 + kTileX - 1 < (nx + 1) / 2 ? 0 : nx - (x0 + kTileX - 1));
  const long long ky = signed_index(y, ny);
  const long long a = (long long)kx * kx * ny * ny + ky * ky * (long long)nx * nx;
  return 4 * a > (long long)nx * nx * ny * ny;
}

// Angular profile h at t = w_hat . n. EV 0 / 1: h(t) = E(v) + t O(v), v = t^2 - 1/2,
// E and O in the monomial basis of v by Horner's rule (9 + 8 or 13 + 12
// coefficients), chosen on the host only when the coefficients show no
// cancellation. EV 2: sum_{j<=32} a_j T_j(t) by Clenshaw's recurrence.
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

// h at the two points t.x and t.y at once (two-lane FMAs for the split forms).
template <int EV>
__device__ __forceinline__ float2 eval_h2(const HEval& h, float2 t) {
  if constexpr (EV < 2) {
    constexpr int NE = EV == 0 ? 9 : 13;
    constexpr int NO = NE - 1;
    const float2 v = fma2(t, t, make_float2(-0.5f, -0.5f));
    float2 e = h.e2[NE - 1];
#pragma unroll
    for (int k = NE - 2; k >= 0; --k) e = fma2k(e, v, h.e2[k]);
    float2 o = h.o2[NO - 1];
#pragma unroll
    for (int k = NO - 2; k >= 0; --k) o = fma2k(o, v, h.o2[k]);
    return fma2(t, o, e);
  } else {
    return make_float2(eval_h<EV>(h, t.x), eval_h<EV>(h, t.y));
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

// ----------------------------------------------------------------------------
// shared-memory and cluster helpers (inline PTX)
// ----------------------------------------------------------------------------
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
// cluster-wide barrier with release/acquire ordering of shared-memory accesses
__device__ __forceinline__ void cluster_sync_acqrel() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" :::
                   "memory");
}
// Asynchronous prefetch of `bytes` (multiple of 16, 16-byte aligned) of
// global memory into L2; no completion to wait for.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile(
      "{\n\t.reg .u64 ga;\n\t"
      "cvta.to.global.u64 ga, %0;\n\t"
      "cp.async.bulk.prefetch.L2.global [ga], %1;\n\t}" ::"l"(p), "r"(bytes)
      : "memory");
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// ----------------------------------------------------------------------------
// z-pass: DFT along z of a 16-wide pencil tile (all slots of the block)
// ----------------------------------------------------------------------------
template <int NZ, int MODE, int EV>
__global__ void __launch_bounds__(kTileX * Plan<NZ>::R2, Plan<NZ>::R2 >= 16 ? 2 : 4)
z_kernel(const __grid_constant__ PassArgs a) {
  constexpr int R1 = Plan<NZ>::R1, R2 = Plan<NZ>::R2;
  constexpr int TW = kTileX;
  constexpr int J3 = (R1 + R2 - 1) / R2;   // step-2 items per thread (k1 = n2 + R2 j < R1)
  constexpr int DIR = (MODE == Z_FWD_PREP || MODE == Z_INV_SCORE) ? -1 : +1;

  __shared__ float2 tile[NZ * TW];     // step-1 / step-2 exchange
  __shared__ float2 keep[NZ * TW];     // forward: f_hat tile; inverse: slot sum
  __shared__ float2 tws[NZ];

  const int t = threadIdx.x;
  const int xl = t % TW, n2 = t / TW;
  const int tiles_x = a.nx / TW;
  const int y = blockIdx.x / tiles_x;
  const int x = (blockIdx.x % tiles_x) * TW + xl;
  const long long plane = (long long)a.ny * a.nx;
  const long long col = (long long)y * a.nx + x;

  if constexpr (MODE == Z_FWD_SCORE || MODE == Z_INV_SCORE) {
    if (a.disc && tile_outside(x, y, a.nx, a.ny)) {
      // psi_hat = 0 on the whole tile: the forward leaves T unwritten (the
      // plane pass reads zeros there); the inverse's sum stays zero
      if (MODE == Z_INV_SCORE && !a.accumulate)
        for (int z = n2; z < NZ; z += R2)
          reinterpret_cast<float2*>(a.out)[(long long)z * plane + col] = make_float2(0.f, 0.f);
      return;
    }
  }
  fill_twiddles<NZ, DIR>(tws);
  const float wy = float(signed_index(y, a.ny)) * a.wy;
  const float wx = float(signed_index(x, a.nx)) * a.wx;
  const float rxy2 = fmaf(wy, wy, wx * wx);
  const bool dc_col = (y == 0) && (x == 0);

  // step 1 (R1-point DFT of the thread's stride-R2 elements) + twiddle + store
  auto step1 = [&](float2 (&v)[R1]) {
    dft<R1, DIR>(v);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1)
      tile[(n2 + R2 * k1) * TW + xl] = (k1 == 0) ? v[k1] : cmul(v[k1], tws[(n2 * k1) % NZ]);
  };
  // step 2 (R2-point DFT over n2 for k1 = n2 + R2 j)
  auto step2 = [&](int j, float2 (&w)[R2]) {
    const int k1 = n2 + R2 * j;
#pragma unroll
    for (int m = 0; m < R2; ++m) w[m] = tile[(m + R2 * k1) * TW + xl];
    dft<R2, DIR>(w);
  };

  if constexpr (MODE == Z_FWD_PREP || MODE == Z_INV_FINAL) {
    float2 v[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      const long long e = (long long)(n2 + R2 * n1) * plane + col;
      float2 in = reinterpret_cast<const float2*>(a.in)[a.in_off + e];
      if (MODE == Z_INV_FINAL && a.in2) in = cadd(in, reinterpret_cast<const float2*>(a.in2)[e]);
      v[n1] = MODE == Z_INV_FINAL ? cscale(in, a.mult[e]) : in;
    }
    __syncthreads();   // twiddle table
    step1(v);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < J3; ++j) {
      const int k1 = n2 + R2 * j;
      if (R1 % R2 != 0 && k1 >= R1) break;
      float2 w[R2];
      step2(j, w);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        const long long e = (long long)(k1 + R1 * k2) * plane + col;
        reinterpret_cast<float2*>(a.out)[a.out_off + e] =
            MODE == Z_FWD_PREP ? cscale(w[k2], a.mult[e]) : w[k2];
      }
    }
  } else if constexpr (MODE == Z_FWD_SCORE) {
    // f_hat tile staged once, then for each slot: x h -> IDFT_z -> T_s
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      const int z = n2 + R2 * n1;
      keep[z * TW + xl] = reinterpret_cast<const float2*>(a.in)[(long long)z * plane + col];
    }
    static_assert(R1 % 2 == 0, "points are evaluated in pairs");
    float2 ur[R1 / 2], rr[R1 / 2];   // w_z / |w| and 1 / |w| at the step-1 frequencies (pairs)
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      const float wz = float(signed_index(n2 + R2 * n1, NZ)) * a.wz;
      const float r2 = fmaf(wz, wz, rxy2);
      const float ri = r2 > 0.f ? rsqrtf(r2) : 0.f;
      (n1 % 2 ? ur[n1 / 2].y : ur[n1 / 2].x) = wz * ri;
      (n1 % 2 ? rr[n1 / 2].y : rr[n1 / 2].x) = ri;
    }
    __syncthreads();
    for (int s = 0; s < a.nslots; ++s) {
      const float dxy = fmaf(wx, a.nvec[s][0], wy * a.nvec[s][1]);
      const float nz = a.nvec[s][2];
      const float2 dxy2 = make_float2(dxy, dxy), nz2 = make_float2(nz, nz);
      float2 v[R1];
#pragma unroll
      for (int m = 0; m < R1 / 2; ++m) {
        float2 hv = eval_h2<EV>(a.h, fma2(rr[m], dxy2, mul2(ur[m], nz2)));
        if (m == 0 && n2 == 0 && dc_col) hv.x = a.h.c0;
        v[2 * m] = cscale(keep[(n2 + R2 * 2 * m) * TW + xl], hv.x);
        v[2 * m + 1] = cscale(keep[(n2 + R2 * (2 * m + 1)) * TW + xl], hv.y);
      }
      step1(v);
      __syncthreads();
      float2* out = reinterpret_cast<float2*>(a.out) + (long long)s * a.slot_stride;
#pragma unroll
      for (int j = 0; j < J3; ++j) {
        const int k1 = n2 + R2 * j;
        if (R1 % R2 != 0 && k1 >= R1) break;
        float2 w[R2];
        step2(j, w);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) out[(long long)(k1 + R1 * k2) * plane + col] = w[k2];
      }
      __syncthreads();
    }
  } else {  // Z_INV_SCORE: for each slot T_s -> DFT_z -> x h, summed into A
    static_assert(R2 % 2 == 0, "points are evaluated in pairs");
    float2 ur[J3 * R2 / 2], rr[J3 * R2 / 2];   // at the step-2 output frequencies (pairs)
#pragma unroll
    for (int j = 0; j < J3; ++j) {
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        const int kz = min(n2 + R2 * j, R1 - 1) + R1 * k2;
        const float wz = float(signed_index(kz, NZ)) * a.wz;
        const float r2 = fmaf(wz, wz, rxy2);
        const float ri = r2 > 0.f ? rsqrtf(r2) : 0.f;
        const int p = j * R2 + k2;
        (p % 2 ? ur[p / 2].y : ur[p / 2].x) = wz * ri;
        (p % 2 ? rr[p / 2].y : rr[p / 2].x) = ri;
      }
    }
#pragma unroll
    for (int j = 0; j < J3; ++j) {
      if (R1 % R2 != 0 && n2 + R2 * j >= R1) break;
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        const int z = n2 + R2 * j + R1 * k2;
        keep[z * TW + xl] = a.accumulate
                                ? reinterpret_cast<const float2*>(a.out)[(long long)z * plane + col]
                                : make_float2(0.f, 0.f);
      }
    }
    __syncthreads();   // twiddle table
    for (int s = 0; s < a.nslots; ++s) {
      const float2* in = reinterpret_cast<const float2*>(a.in) + (long long)s * a.slot_stride;
      float2 v[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) v[n1] = in[(long long)(n2 + R2 * n1) * plane + col];
      step1(v);
      __syncthreads();
      const float dxy = fmaf(wx, a.nvec[s][0], wy * a.nvec[s][1]);
      const float nz = a.nvec[s][2];
      const float2 dxy2 = make_float2(dxy, dxy), nz2 = make_float2(nz, nz);
#pragma unroll
      for (int j = 0; j < J3; ++j) {
        if (R1 % R2 != 0 && n2 + R2 * j >= R1) break;
        float2 w[R2];
        step2(j, w);
#pragma unroll
        for (int k2 = 0; k2 < R2; k2 += 2) {
          const int p = (j * R2 + k2) / 2;
          float2 hv = eval_h2<EV>(a.h, fma2(rr[p], dxy2, mul2(ur[p], nz2)));
          if (p == 0 && n2 == 0 && dc_col) hv.x = a.h.c0;
          float2& d0 = keep[(n2 + R2 * j + R1 * k2) * TW + xl];
          d0.x = fmaf(hv.x, w[k2].x, d0.x);
          d0.y = fmaf(hv.x, w[k2].y, d0.y);
          float2& d1 = keep[(n2 + R2 * j + R1 * (k2 + 1)) * TW + xl];
          d1.x = fmaf(hv.y, w[k2 + 1].x, d1.x);
          d1.y = fmaf(hv.y, w[k2 + 1].y, d1.y);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < J3; ++j) {
      if (R1 % R2 != 0 && n2 + R2 * j >= R1) break;
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        const int z = n2 + R2 * j + R1 * k2;
        reinterpret_cast<float2*>(a.out)[(long long)z * plane + col] = keep[z * TW + xl];
      }
    }
  }
}

// ----------------------------------------------------------------------------
// xy-pass on NS CTAs per z-plane: one (a whole plane per CTA) for planes up
// to 128^2, a cluster of 8 for 256^2 planes. CTA h holds rows
// [h NY/NS, (h+1) NY/NS) of a z-plane for the x direction and columns
// [h NX/NS, (h+1) NX/NS) for the y direction; the x step-2 outputs go straight
// into the owner's y-layout buffer (its own shared memory, or for NS > 1
// distributed shared memory). An eighth of a 256^2 plane (84 KB) lets two
// CTAs share an SM, so one CTA's loads overlap the other's DFTs.
// Shared layout: x layout row pitch NX + 8 (rows alternate 64-byte halves of
// the bank space) with an XOR swizzle inside each group of R2x columns; y
// layout row pitch NX/NS + 8. Work units: (plane, slot) for the score modes,
// planes for the real modes; CTAs (clusters) loop over units.
// ----------------------------------------------------------------------------
// CTAs per plane (NS) and the largest thread count per CTA. Planes up to
// 128^2: a whole plane per CTA (up to 139 KB of shared memory and 512
// threads), so every exchange stays in the CTA, with block barriers instead
// of cluster barriers (faster than half planes on 2-CTA clusters by 5 % at
// 128^2 and 7-21 % for the smaller planes). 256^2: an eighth of a plane per
// CTA on 8-CTA clusters.
template <int NY, int NX> struct XYSplit { static constexpr int NS = 1, NTMAX = 512; };
template <> struct XYSplit<256, 256> { static constexpr int NS = 8, NTMAX = 256; };

// barrier between the phases of a plane: the whole cluster, or for a plane
// held by one CTA the block
template <int NS>
__device__ __forceinline__ void plane_sync() {
  if constexpr (NS == 1) __syncthreads();
  else cluster_sync_acqrel();
}

template <int NY, int NX, int NS = XYSplit<NY, NX>::NS, int NTMAX = XYSplit<NY, NX>::NTMAX>
struct XYCfg {
  static constexpr int NYH = NY / NS, NXH = NX / NS;   // rows / columns of one CTA
  static constexpr int R1x = Plan<NX>::R1, R2x = Plan<NX>::R2;
  static constexpr int R1y = Plan<NY>::R1, R2y = Plan<NY>::R2;
  static_assert((R2x & (R2x - 1)) == 0, "R2x must be a power of two");
  static constexpr bool ok(int nt) {
    // (a rectangular plane may leave the last pass of y step 1 partial)
    return nt % 32 == 0 && (NYH * R2x) % nt == 0 && nt % R2x == 0 && (NYH * R1x) % nt == 0 &&
           nt % R2y == 0 && (NY != NX || NXH % (nt / R2y) == 0) && (NXH * R1y) % nt == 0;
  }
  static constexpr int pick() {
    for (int nt = NTMAX; nt >= 32; nt -= 32)
      if (ok(nt)) return nt;
    return 0;
  }
  static constexpr int NT = pick();
  static_assert(NT > 0, "no thread count fits this half plane");
  static constexpr int PX = NX + 8;     // x layout pitch (float2)
  static constexpr int PY = NXH + 8;    // y layout pitch (float2)
  static constexpr int BUF = (NYH * PX > NY * PY) ? NYH * PX : NY * PY;
  static constexpr int JX1 = NYH * R2x / NT;
  static constexpr int JX3 = NYH * R1x / NT;
  static constexpr int CW = NT / R2y;
  static constexpr int JY1 = (NXH + CW - 1) / CW;
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

template <int NY, int NX, int MODE, int UBF16>
__global__ void __cluster_dims__(XYSplit<NY, NX>::NS, 1, 1)
    __launch_bounds__(XYCfg<NY, NX>::NT, XYSplit<NY, NX>::NS == 1 ? 1 : 2)
xy_kernel(const __grid_constant__ PassArgs a) {
  using C = XYCfg<NY, NX>;
  constexpr int NS = XYSplit<NY, NX>::NS;
  constexpr int R1x = C::R1x, R2x = C::R2x, R1y = C::R1y, R2y = C::R2y;
  constexpr int NT = C::NT, NYH = C::NYH, NXH = C::NXH;
  constexpr bool INV = MODE == XY_INV_SCORE || MODE == XY_INV_WSCORE;   // score -> T
  constexpr int DIR = (MODE == XY_FWD_REAL || INV) ? -1 : +1;
  static_assert(MODE != XY_INV_WSCORE || !UBF16, "the weighted load takes complex64 scores");

  extern __shared__ __align__(16) float2 sm[];
  float2* work = sm;
  float2* twx = sm + C::BUF;
  float2* twy = twx + NX;

  const int t = threadIdx.x;
  const int h = (int)cluster_rank();
  unsigned peer_base[NS];   // the work buffer of every CTA of the cluster
#pragma unroll
  for (int q = 0; q < NS; ++q) peer_base[q] = map_cluster_rank(smem_addr(work), (unsigned)q);
  const long long P = (long long)NY * NX;
  const int cl = blockIdx.x / NS, ncl = gridDim.x / NS;
  const int nsl = (MODE == XY_FWD_SCORE || INV) ? a.nslots : 1;
  float c2 = 0.f;   // 2 g of the weighted load
  if constexpr (MODE == XY_INV_WSCORE) c2 = 2.f * __ldg(a.gscale);
  const int nunits = a.nz * nsl;

  fill_twiddles<NX, DIR>(twx);
  fill_twiddles<NY, DIR>(twy);
  __syncthreads();

  for (int u = cl; u < nunits; u += ncl) {
    const int z = u % a.nz, s = u / a.nz;
    const long long zoff = (long long)z * P;
    // ---- x direction, step 1 on this CTA's rows (global -> registers -> shared)
    {
      long long ia, ib = -1;
      if constexpr (INV) {
        ia = a.ua[s];
        ib = a.ub[s];
      } else if constexpr (MODE == XY_FWD_SCORE) {
        ia = (long long)s * a.slot_stride;
      } else {
        ia = a.in_off;
      }
      const int n2 = t % R2x, r0 = t / R2x;
      float2 tw[R1x];
#pragma unroll
      for (int k1 = 0; k1 < R1x; ++k1) tw[k1] = twx[(n2 * k1) % NX];
#pragma unroll
      for (int j = 0; j < C::JX1; ++j) {
        const int r = r0 + (NT / R2x) * j;
        const long long row = zoff + (long long)(h * NYH + r) * NX;
        float2 v[R1x];
#pragma unroll
        for (int n1 = 0; n1 < R1x; ++n1) {
          const long long e = row + n2 + R2x * n1;
          if constexpr (MODE == XY_FWD_REAL) {
            v[n1] = make_float2(__ldg(reinterpret_cast<const float*>(a.in) + ia + e), 0.f);
          } else if constexpr (MODE == XY_INV_SCORE) {
            float2 q = load_u<UBF16>(a.in, ia + e);
            if (ib >= 0) q = cadd(q, cconj(load_u<UBF16>(a.in, ib + e)));
            v[n1] = q;
          } else if constexpr (MODE == XY_INV_WSCORE) {
            float2 q = cscale(load_u<0>(a.in, ia + e), __ldcs(a.wgt + ia + e));
            if (ib >= 0) q = cadd(q, cconj(cscale(load_u<0>(a.in, ib + e), __ldcs(a.wgt + ib + e))));
            v[n1] = cscale(q, c2);
          } else if constexpr (MODE == XY_FWD_SCORE) {
            v[n1] = (a.disc && tile_outside(n2 + R2x * n1, h * NYH + r, NX, NY))
                        ? make_float2(0.f, 0.f)
                        : reinterpret_cast<const float2*>(a.in)[ia + e];
          } else {
            v[n1] = reinterpret_cast<const float2*>(a.in)[ia + e];
          }
        }
        dft<R1x, DIR>(v);
#pragma unroll
        for (int k1 = 0; k1 < R1x; ++k1)
          work[C::xphys(r, n2 + R2x * k1)] = (k1 == 0) ? v[k1] : cmul(v[k1], tw[k1]);
      }
    }
    __syncthreads();
    // the input rows of this CTA's next unit go to L2 while this one runs
    if (t == 0 && (MODE == XY_FWD_SCORE || INV) && u + ncl < nunits) {
      const int zn = (u + ncl) % a.nz, sn = (u + ncl) / a.nz;
      const long long rows = (long long)zn * P + (long long)h * NYH * NX;
      constexpr unsigned esz = (INV && UBF16) ? 4u : 8u;
      constexpr unsigned bytes = (unsigned)(NYH * NX) * esz;
      const char* base = reinterpret_cast<const char*>(a.in);
      if constexpr (MODE == XY_FWD_SCORE) {
        prefetch_l2(base + 8 * ((long long)sn * a.slot_stride + rows), bytes);
      } else {
        prefetch_l2(base + esz * (a.ua[sn] + rows), bytes);
        if (a.ub[sn] >= 0) prefetch_l2(base + esz * (a.ub[sn] + rows), bytes);
        if constexpr (MODE == XY_INV_WSCORE) {
          prefetch_l2(a.wgt + a.ua[sn] + rows, bytes / 2);
          if (a.ub[sn] >= 0) prefetch_l2(a.wgt + a.ub[sn] + rows, bytes / 2);
        }
      }
    }
    // ---- x direction, step 2; outputs go to the owner of their column
    {
      float2 w[C::JX3][R2x];
#pragma unroll
      for (int j = 0; j < C::JX3; ++j) {
        int r, k1;
        C::x2_item(t, j, r, k1);
#pragma unroll
        for (int m = 0; m < R2x; ++m) w[j][m] = work[C::xphys(r, m + R2x * k1)];
        dft<R2x, DIR>(w[j]);
      }
      // both halves have read their x-layout buffers before either writes into
      // the other's (release/acquire orders these reads before the peer's stores)
      plane_sync<NS>();
#pragma unroll
      for (int j = 0; j < C::JX3; ++j) {
        int r, k1;
        C::x2_item(t, j, r, k1);
        const int row = (h * NYH + r) * C::PY;
#pragma unroll
        for (int k2 = 0; k2 < R2x; ++k2) {
          const int c = k1 + R1x * k2;
          const int owner = (NXH % R1x == 0) ? (k2 / (NXH / R1x)) : (c / NXH);
          const int idx = row + c - owner * NXH;
          if (owner == h) work[idx] = w[j][k2];
          else st_cluster_f2(peer_base[owner] + 8u * (unsigned)idx, w[j][k2]);
        }
      }
      plane_sync<NS>();   // this CTA's y-layout buffer is complete
    }
    // ---- y direction, step 1 (in place)
    {
      const int n2 = t / C::CW;
      float2 tw[R1y];
#pragma unroll
      for (int k1 = 0; k1 < R1y; ++k1) tw[k1] = twy[(n2 * k1) % NY];
#pragma unroll
      for (int j = 0; j < C::JY1; ++j) {
        const int c = t % C::CW + C::CW * j;
        if (NXH % C::CW != 0 && c >= NXH) break;
        float2 u1[R1y];
#pragma unroll
        for (int n1 = 0; n1 < R1y; ++n1) u1[n1] = work[(n2 + R2y * n1) * C::PY + c];
        dft<R1y, DIR>(u1);
#pragma unroll
        for (int k1 = 0; k1 < R1y; ++k1)
          work[(n2 + R2y * k1) * C::PY + c] = (k1 == 0) ? u1[k1] : cmul(u1[k1], tw[k1]);
      }
    }
    __syncthreads();
    // ---- y direction, step 2 + store
    {
      long long o, ob = -1;
      if constexpr (MODE == XY_FWD_SCORE) {
        o = a.ua[s];
        ob = a.ub[s];
      } else if constexpr (INV) {
        o = (long long)s * a.slot_stride;
      } else {
        o = a.out_off;
      }
      const long long zo = zoff + h * NXH;
#pragma unroll
      for (int j = 0; j < C::JY3; ++j) {
        const int q = t + NT * j;
        const int c = q % NXH, k1 = q / NXH;
        float2 w[R2y];
#pragma unroll
        for (int m = 0; m < R2y; ++m) w[m] = work[(m + R2y * k1) * C::PY + c];
        dft<R2y, DIR>(w);
#pragma unroll
        for (int k2 = 0; k2 < R2y; ++k2) {
          const long long e = zo + (long long)(k1 + R1y * k2) * NX + c;
          if constexpr (MODE == XY_FWD_SCORE) {
            store_u<UBF16>(a.out, o + e, w[k2]);
            if (ob >= 0) store_u<UBF16>(a.out, ob + e, cconj(w[k2]));
          } else if constexpr (MODE == XY_INV_REAL) {
            reinterpret_cast<float*>(a.out)[o + e] = w[k2].x;
          } else if constexpr (INV) {
            if (!(a.disc && tile_outside(h * NXH + c, k1 + R1y * k2, NX, NY)))
              reinterpret_cast<float2*>(a.out)[o + e] = w[k2];
          } else {
            reinterpret_cast<float2*>(a.out)[o + e] = w[k2];
          }
        }
      }
    }
    __syncthreads();    // work is rewritten by the next x step 1
  }
  plane_sync<NS>();   // no CTA leaves while its peer may still write into it
}

// ----------------------------------------------------------------------------
// Forward score pass (T_s -> IDFT_xy -> U_a, U_b = conj U_a) on F independent
// parts of each plane split by the output row modulo F: F = 4 for 256^2
// planes, too large for one CTA, and F = 2 for 128^2 planes (two half-plane
// CTAs of 256 threads and 72 KB per SM; a CTA that runs alone on its SM
// leaves room for z-pass CTAs of the other stream beside it).
// The rows y = F k + h (h < F) of the 2D DFT of an NY x NX plane a are the
// (NY/F)-point DFT along y of the folded rows
//   b_h[r] = W^{h r} sum_{q < F} a[r + (NY/F) q] w_F^{h q},   r < NY/F,
// W = exp(DIR 2 pi i / NY), w_F = W^{NY/F} (split the input row as
// r + (NY/F) q: W^{(r + (NY/F) q)(F k + h)} = W_{NY/F}^{r k} W^{h r} w_F^{h q}).
// So each part is a whole (NY/F) x NX plane transform in one CTA (the
// machinery of xy_kernel on a 64 x 256 or 64 x 128 plane), with no exchange
// between CTAs: the CTA reads the whole input plane (the F parts of a plane
// run on consecutive CTAs, so all but one of the F reads of each input row
// come from L2) and writes every F-th output row. At
// 256^3 x 42 this forward pass takes 3.3-3.4 instead of 4.2 ms per step
// (complex64; BF16 scores 2.5 instead of 3.6 ms) against the 8-CTA cluster
// pass; the inverse stays on the cluster pass, where the four reads of both
// U_a and U_b per part made the same fold slower (6.2 against 3.9 ms). At
// 128^3 x 162 the halves take the forward + inverse step from 2.087 to
// 2.063 ms (complex64): alone the half-plane pass is 5 % faster (102 against
// 107 us per 11-pair launch), in the step it takes about as long, and the
// z-pass beside it is faster (0.69 against 0.78 ms per step).
// ----------------------------------------------------------------------------
template <int NY, int NX> struct XYFold { static constexpr int F = 1; };
template <> struct XYFold<256, 256> { static constexpr int F = 4; };
template <> struct XYFold<128, 128> { static constexpr int F = 2; };

template <int NY, int NX>
struct XYFoldCfg {
  static constexpr int F = XYFold<NY, NX>::F;
  static constexpr int NH = NY / F;
  static constexpr int MINB = F == 2 ? 2 : 1;   // CTAs per SM
  using C = XYCfg<NH, NX, 1, 512 / MINB>;
  // work buffer, twiddles along x (NX) and y (NH), fold factors W^m (m < NY)
  static constexpr size_t smem_bytes = sizeof(float2) * (size_t(C::BUF) + NX + NH + NY);
};

template <int NY, int NX, int UBF16>
__global__ void __launch_bounds__(XYFoldCfg<NY, NX>::C::NT, XYFoldCfg<NY, NX>::MINB)
xy_fold_kernel(const __grid_constant__ PassArgs a) {
  using FC = XYFoldCfg<NY, NX>;
  using C = typename FC::C;
  constexpr int F = FC::F, NH = FC::NH;
  constexpr int R1x = C::R1x, R2x = C::R2x, R1y = C::R1y, R2y = C::R2y;
  constexpr int NT = C::NT;
  constexpr int DIR = +1;
  static_assert(F == 2 || F == 4, "halves or quarters of planes");
  static_assert(NY % F == 0 && C::NYH == NH && C::NXH == NX, "one part of a plane per CTA");

  extern __shared__ __align__(16) float2 sm[];
  float2* work = sm;
  float2* twx = sm + C::BUF;
  float2* twy = twx + NX;
  float2* twf = twy + NH;   // W^m, m < NY: the fold factors

  const int t = threadIdx.x;
  const long long P = (long long)NY * NX;
  const long long PART = (long long)NH * NX;   // elements of one part of a plane
  const int nunits = F * a.nz * a.nslots;

  fill_twiddles<NX, DIR>(twx);
  fill_twiddles<NH, DIR>(twy);
  fill_twiddles<NY, DIR>(twf);
  __syncthreads();

  // T_s at element e of the plane (row y, column x); zero on the tiles
  // outside the disc, which the z-pass does not write
  auto input = [&](int s, long long e, int y, int x) -> float2 {
    return (a.disc && tile_outside(x, y, NX, NY))
               ? make_float2(0.f, 0.f)
               : reinterpret_cast<const float2*>(a.in)[(long long)s * a.slot_stride + e];
  };

  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int hf = u % F, pl = u / F;
    const int z = pl % a.nz, s = pl / a.nz;
    const long long zoff = (long long)z * P;
    // ---- x direction, step 1 on the folded rows (global -> registers -> shared)
    {
      const int n2 = t % R2x, r0 = t / R2x;
      float2 tw[R1x];
#pragma unroll
      for (int k1 = 0; k1 < R1x; ++k1) tw[k1] = twx[(n2 * k1) % NX];
#pragma unroll
      for (int j = 0; j < C::JX1; ++j) {
        const int r = r0 + (NT / R2x) * j;
        const long long row = zoff + (long long)r * NX;
        float2 v[R1x];
#pragma unroll
        for (int n1 = 0; n1 < R1x; ++n1) v[n1] = input(s, row + n2 + R2x * n1, r, n2 + R2x * n1);
#pragma unroll
        for (int q = 1; q < F; ++q) {
          float2 w[R1x];
#pragma unroll
          for (int n1 = 0; n1 < R1x; ++n1)
            w[n1] = input(s, row + q * PART + n2 + R2x * n1, r + q * NH, n2 + R2x * n1);
          // x w_F^{h q}, the same power for the whole CTA
          switch ((q * hf * (4 / F)) & 3) {
            case 0:
#pragma unroll
              for (int n1 = 0; n1 < R1x; ++n1) v[n1] = cadd(v[n1], w[n1]);
              break;
            case 1:
#pragma unroll
              for (int n1 = 0; n1 < R1x; ++n1) v[n1] = cadd(v[n1], cmul_i<DIR>(w[n1]));
              break;
            case 2:
#pragma unroll
              for (int n1 = 0; n1 < R1x; ++n1) v[n1] = csub(v[n1], w[n1]);
              break;
            default:
#pragma unroll
              for (int n1 = 0; n1 < R1x; ++n1) v[n1] = cadd(v[n1], cmul_i<-DIR>(w[n1]));
              break;
          }
        }
        if (hf) {
          const float2 om = twf[r * hf];
#pragma unroll
          for (int n1 = 0; n1 < R1x; ++n1) v[n1] = cmul(v[n1], om);
        }
        dft<R1x, DIR>(v);
#pragma unroll
        for (int k1 = 0; k1 < R1x; ++k1)
          work[C::xphys(r, n2 + R2x * k1)] = (k1 == 0) ? v[k1] : cmul(v[k1], tw[k1]);
      }
    }
    __syncthreads();
    // this CTA's part of the rows of its next unit's input plane goes to L2
    // while this unit runs (the F CTAs of a plane cover it together)
    if (t == 0 && u + (int)gridDim.x < nunits) {
      const int un = u + (int)gridDim.x;
      const int pn = un / F, hn = un % F;
      const int zn = pn % a.nz, sn = pn / a.nz;
      const long long base = (long long)zn * P + hn * PART;
      prefetch_l2(reinterpret_cast<const float2*>(a.in) + (long long)sn * a.slot_stride + base,
                  (unsigned)(NH * NX * sizeof(float2)));
    }
    // ---- x direction, step 2 (x layout -> y layout, in the same buffer)
    {
      float2 w[C::JX3][R2x];
#pragma unroll
      for (int j = 0; j < C::JX3; ++j) {
        int r, k1;
        C::x2_item(t, j, r, k1);
#pragma unroll
        for (int m = 0; m < R2x; ++m) w[j][m] = work[C::xphys(r, m + R2x * k1)];
        dft<R2x, DIR>(w[j]);
      }
      __syncthreads();   // every x-layout read is done before the y layout is written
#pragma unroll
      for (int j = 0; j < C::JX3; ++j) {
        int r, k1;
        C::x2_item(t, j, r, k1);
#pragma unroll
        for (int k2 = 0; k2 < R2x; ++k2) work[r * C::PY + k1 + R1x * k2] = w[j][k2];
      }
      __syncthreads();
    }
    // ---- y direction (NY/F points), step 1 (in place)
    {
      const int n2 = t / C::CW;
      float2 tw[R1y];
#pragma unroll
      for (int k1 = 0; k1 < R1y; ++k1) tw[k1] = twy[(n2 * k1) % NH];
#pragma unroll
      for (int j = 0; j < C::JY1; ++j) {
        const int c = t % C::CW + C::CW * j;
        if (NX % C::CW != 0 && c >= NX) break;
        float2 u1[R1y];
#pragma unroll
        for (int n1 = 0; n1 < R1y; ++n1) u1[n1] = work[(n2 + R2y * n1) * C::PY + c];
        dft<R1y, DIR>(u1);
#pragma unroll
        for (int k1 = 0; k1 < R1y; ++k1)
          work[(n2 + R2y * k1) * C::PY + c] = (k1 == 0) ? u1[k1] : cmul(u1[k1], tw[k1]);
      }
    }
    __syncthreads();
    // ---- y direction, step 2 + store of the output rows F k + h
    {
      const long long o = a.ua[s], ob = a.ub[s];
#pragma unroll
      for (int j = 0; j < C::JY3; ++j) {
        const int q = t + NT * j;
        const int c = q % NX, k1 = q / NX;
        float2 w[R2y];
#pragma unroll
        for (int m = 0; m < R2y; ++m) w[m] = work[(m + R2y * k1) * C::PY + c];
        dft<R2y, DIR>(w);
#pragma unroll
        for (int k2 = 0; k2 < R2y; ++k2) {
          const int y = F * (k1 + R1y * k2) + hf;
          const long long e = zoff + (long long)y * NX + c;
          store_u<UBF16>(a.out, o + e, w[k2]);
          if (ob >= 0) store_u<UBF16>(a.out, ob + e, cconj(w[k2]));
        }
      }
    }
    __syncthreads();   // work is rewritten by the next unit
  }
}


// ----------------------------------------------------------------------------
// Score-domain step of Upsilon = W^{*,ext} Phi W (Sec. 4.1) for one block of
// orientation pairs, fused into one plane pass, in place on T_s:
//   T_s <- DFT_xy[ m_s Phi( IDFT_xy T_s ) ]
// Phi is the soft threshold |u|^p sgn(u) of the real and imaginary parts;
// m_s = 2 for an antipodal pair (the inverse takes V_a + conj V_b and Phi
// commutes with conjugation, so V_b = conj V_a), 1 for an unpaired slot.
// The score U_s = IDFT_xy T_s exists only in shared memory. Layout and
// exchanges as xy_kernel: IDFT along x on this CTA's rows, exchange, IDFT
// along y on its columns; the y step-2 outputs go back to the rows they were
// read from (y index k1 + R1y k2 in row R2y k1 + k2), the DFT along y reads
// them through that map, exchanges back to rows, and the DFT along x writes
// T_s.
// ----------------------------------------------------------------------------
// WEIGHTED = 1 (XY_WENERGY): the score-domain step of the gradient of the
// weighted energy L = sum w |U|^2 instead: for the pair (a, b = -a) the
// adjoint's input 2 g (w_a U_a + conj(w_b U_b)) is 2 g (w_a + w_b) U_a (w is
// real and U_b = conj U_a), 2 g w_a U_a for an unpaired slot, and the energy
// of the unit, sum (w_a + w_b) |U_a|^2, goes to epart (FP32 over a thread's
// elements, FP64 over the block in a fixed order; one sum per CTA of the
// plane's cluster, at index unit x NS + rank).
template <int NY, int NX, int WEIGHTED>
__global__ void __cluster_dims__(XYSplit<NY, NX>::NS, 1, 1)
    __launch_bounds__(XYCfg<NY, NX>::NT, XYSplit<NY, NX>::NS == 1 ? 1 : 2)
xy_soft_kernel(const __grid_constant__ PassArgs a) {
  using C = XYCfg<NY, NX>;
  constexpr int NS = XYSplit<NY, NX>::NS;
  constexpr int R1x = C::R1x, R2x = C::R2x, R1y = C::R1y, R2y = C::R2y;
  constexpr int NT = C::NT, NYH = C::NYH, NXH = C::NXH;
  __shared__ double ered[WEIGHTED ? NT / 32 : 1];   // WEIGHTED: the warps' energy sums
  float c2 = 0.f;                    // WEIGHTED: 2 g
  if constexpr (WEIGHTED) c2 = 2.f * (a.gscale ? __ldg(a.gscale) : 1.f);

  extern __shared__ __align__(16) float2 sm[];
  float2* work = sm;
  float2* twx = sm + C::BUF;   // exp(+2 pi i m / NX); the DFT uses the conjugates
  float2* twy = twx + NX;

  const int t = threadIdx.x;
  const int h = (int)cluster_rank();
  unsigned peer_base[NS];   // the work buffer of every CTA of the cluster
#pragma unroll
  for (int q = 0; q < NS; ++q) peer_base[q] = map_cluster_rank(smem_addr(work), (unsigned)q);
  const long long P = (long long)NY * NX;
  const int cl = blockIdx.x / NS, ncl = gridDim.x / NS;
  const int nunits = a.nz * a.nslots;
  // row of the y-layout that holds y index n after the IDFT along y
  auto yrow = [](int n) { return R2y * (n % R1y) + n / R1y; };

  fill_twiddles<NX, +1>(twx);
  fill_twiddles<NY, +1>(twy);
  __syncthreads();

  for (int u = cl; u < nunits; u += ncl) {
    const int z = u % a.nz, s = u / a.nz;
    float2* T = reinterpret_cast<float2*>(a.out) + (long long)s * a.slot_stride + (long long)z * P;
    if (t == 0 && u + ncl < nunits) {
      const int zn = (u + ncl) % a.nz, sn = (u + ncl) / a.nz;
      prefetch_l2(reinterpret_cast<const float2*>(a.out) + (long long)sn * a.slot_stride +
                      (long long)zn * P + (long long)h * NYH * NX,
                  (unsigned)(NYH * NX * sizeof(float2)));
    }
    const float scale = a.ub[s] >= 0 ? 2.f : 1.f;
    if constexpr (WEIGHTED) {
      // this CTA's rows of the unit's weights go to L2 while the IDFT runs
      // (the cluster's CTAs together cover the plane)
      if (t == 32) {
        const long long rows = (long long)z * P + (long long)h * NYH * NX;
        constexpr unsigned wbytes = (unsigned)(NYH * NX) * 4u;
        prefetch_l2(a.wgt + a.ua[s] + rows, wbytes);
        if (a.ub[s] >= 0) prefetch_l2(a.wgt + a.ub[s] + rows, wbytes);
      }
    }
    // ---- (1) IDFT along x, step 1 (global -> registers -> shared)
    {
      const int n2 = t % R2x, r0 = t / R2x;
      float2 tw[R1x];
#pragma unroll
      for (int k1 = 0; k1 < R1x; ++k1) tw[k1] = twx[(n2 * k1) % NX];
#pragma unroll 1
      for (int j = 0; j < C::JX1; ++j) {
        const int r = r0 + (NT / R2x) * j;
        const float2* row = T + (long long)(h * NYH + r) * NX;
        float2 v[R1x];
#pragma unroll
        for (int n1 = 0; n1 < R1x; ++n1)
          v[n1] = (a.disc && tile_outside(n2 + R2x * n1, h * NYH + r, NX, NY))
                      ? make_float2(0.f, 0.f)
                      : row[n2 + R2x * n1];
        dft<R1x, +1>(v);
#pragma unroll
        for (int k1 = 0; k1 < R1x; ++k1)
          work[C::xphys(r, n2 + R2x * k1)] = (k1 == 0) ? v[k1] : cmul(v[k1], tw[k1]);
      }
    }
    __syncthreads();
    // ---- (2) IDFT along x, step 2; outputs to the owner of their column
    {
      float2 w[C::JX3][R2x];
#pragma unroll
      for (int j = 0; j < C::JX3; ++j) {
        int r, k1;
        C::x2_item(t, j, r, k1);
#pragma unroll
        for (int m = 0; m < R2x; ++m) w[j][m] = work[C::xphys(r, m + R2x * k1)];
        dft<R2x, +1>(w[j]);
      }
      plane_sync<NS>();   // both halves have read their x layouts
#pragma unroll
      for (int j = 0; j < C::JX3; ++j) {
        int r, k1;
        C::x2_item(t, j, r, k1);
        const int row = (h * NYH + r) * C::PY;
#pragma unroll
        for (int k2 = 0; k2 < R2x; ++k2) {
          const int c = k1 + R1x * k2;
          const int owner = (NXH % R1x == 0) ? (k2 / (NXH / R1x)) : (c / NXH);
          const int idx = row + c - owner * NXH;
          if (owner == h) work[idx] = w[j][k2];
          else st_cluster_f2(peer_base[owner] + 8u * (unsigned)idx, w[j][k2]);
        }
      }
      plane_sync<NS>();   // this CTA's y layout is complete
    }
    // ---- (3) IDFT along y, step 1 (in place)
    {
      const int n2 = t / C::CW;
      float2 tw[R1y];
#pragma unroll
      for (int k1 = 0; k1 < R1y; ++k1) tw[k1] = twy[(n2 * k1) % NY];
#pragma unroll 1
      for (int j = 0; j < C::JY1; ++j) {
        const int c = t % C::CW + C::CW * j;
        if (NXH % C::CW != 0 && c >= NXH) break;
        float2 u1[R1y];
#pragma unroll
        for (int n1 = 0; n1 < R1y; ++n1) u1[n1] = work[(n2 + R2y * n1) * C::PY + c];
        dft<R1y, +1>(u1);
#pragma unroll
        for (int k1 = 0; k1 < R1y; ++k1)
          work[(n2 + R2y * k1) * C::PY + c] = (k1 == 0) ? u1[k1] : cmul(u1[k1], tw[k1]);
      }
    }
    __syncthreads();
    // ---- (4) IDFT along y, step 2: U_s; m_s Phi(U_s) (or the weighted
    // gradient) back into the rows read
    float en = 0.f;   // WEIGHTED: this thread's part of the unit's energy
#pragma unroll 1
    for (int j = 0; j < C::JY3; ++j) {
      const int q = t + NT * j;
      const int c = q % NXH, k1 = q / NXH;
      float2 w[R2y];
#pragma unroll
      for (int m = 0; m < R2y; ++m) w[m] = work[(m + R2y * k1) * C::PY + c];
      dft<R2y, +1>(w);
#pragma unroll
      for (int k2 = 0; k2 < R2y; ++k2) {
        if constexpr (WEIGHTED) {
          const long long e = (long long)z * P + (long long)(k1 + R1y * k2) * NX + h * NXH + c;
          float ww = __ldcs(a.wgt + a.ua[s] + e);
          if (a.ub[s] >= 0) ww += __ldcs(a.wgt + a.ub[s] + e);
          en = fmaf(ww, fmaf(w[k2].x, w[k2].x, w[k2].y * w[k2].y), en);
          work[(R2y * k1 + k2) * C::PY + c] = cscale(w[k2], c2 * ww);
        } else {
          work[(R2y * k1 + k2) * C::PY + c] = make_float2(scale * soft_part(w[k2].x, a.power),
                                                          scale * soft_part(w[k2].y, a.power));
        }
      }
    }
    if constexpr (WEIGHTED) {
      double d = (double)en;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
      if ((t & 31) == 0) ered[t >> 5] = d;
    }
    __syncthreads();
    if constexpr (WEIGHTED) {
      // ered is written again only after the barriers of the next unit
      if (t == 0) {
        double sum = 0.0;
#pragma unroll
        for (int i = 0; i < NT / 32; ++i) sum += ered[i];
        a.epart[a.epart_base + (long long)u * NS + h] = sum;
      }
    }
    // ---- (5) DFT along y, step 1 (in place through the row map)
    {
      const int n2 = t / C::CW;
      float2 tw[R1y];
#pragma unroll
      for (int k1 = 0; k1 < R1y; ++k1) tw[k1] = cconj(twy[(n2 * k1) % NY]);
#pragma unroll 1
      for (int j = 0; j < C::JY1; ++j) {
        const int c = t % C::CW + C::CW * j;
        if (NXH % C::CW != 0 && c >= NXH) break;
        float2 u1[R1y];
#pragma unroll
        for (int n1 = 0; n1 < R1y; ++n1) u1[n1] = work[yrow(n2 + R2y * n1) * C::PY + c];
        dft<R1y, -1>(u1);
#pragma unroll
        for (int k1 = 0; k1 < R1y; ++k1)
          work[yrow(n2 + R2y * k1) * C::PY + c] = (k1 == 0) ? u1[k1] : cmul(u1[k1], tw[k1]);
      }
    }
    __syncthreads();
    // ---- (6) DFT along y, step 2; outputs to the owner of their row
    {
      float2 w[C::JY3][R2y];
#pragma unroll
      for (int j = 0; j < C::JY3; ++j) {
        const int q = t + NT * j;
        const int c = q % NXH, k1 = q / NXH;
#pragma unroll
        for (int m = 0; m < R2y; ++m) w[j][m] = work[yrow(m + R2y * k1) * C::PY + c];
        dft<R2y, -1>(w[j]);
      }
      plane_sync<NS>();   // both halves have read their y layouts
#pragma unroll
      for (int j = 0; j < C::JY3; ++j) {
        const int q = t + NT * j;
        const int c = q % NXH, k1 = q / NXH;
#pragma unroll
        for (int k2 = 0; k2 < R2y; ++k2) {
          const int ky = k1 + R1y * k2;
          const int owner = ky / NYH;
          const int idx = C::xphys(ky - owner * NYH, h * NXH + c);
          if (owner == h) work[idx] = w[j][k2];
          else st_cluster_f2(peer_base[owner] + 8u * (unsigned)idx, w[j][k2]);
        }
      }
      plane_sync<NS>();   // this CTA's x layout is complete
    }
    // ---- (7) DFT along x, step 1 (in place on this CTA's rows)
    {
      const int n2 = t % R2x, r0 = t / R2x;
      float2 tw[R1x];
#pragma unroll
      for (int k1 = 0; k1 < R1x; ++k1) tw[k1] = cconj(twx[(n2 * k1) % NX]);
#pragma unroll 1
      for (int j = 0; j < C::JX1; ++j) {
        const int r = r0 + (NT / R2x) * j;
        float2 v[R1x];
#pragma unroll
        for (int n1 = 0; n1 < R1x; ++n1) v[n1] = work[C::xphys(r, n2 + R2x * n1)];
        dft<R1x, -1>(v);
#pragma unroll
        for (int k1 = 0; k1 < R1x; ++k1)
          work[C::xphys(r, n2 + R2x * k1)] = (k1 == 0) ? v[k1] : cmul(v[k1], tw[k1]);
      }
    }
    __syncthreads();
    // ---- (8) DFT along x, step 2 -> T_s
#pragma unroll 1
    for (int j = 0; j < C::JX3; ++j) {
      int r, k1;
      C::x2_item(t, j, r, k1);
      float2 w[R2x];
#pragma unroll
      for (int m = 0; m < R2x; ++m) w[m] = work[C::xphys(r, m + R2x * k1)];
      dft<R2x, -1>(w);
      float2* row = T + (long long)(h * NYH + r) * NX;
#pragma unroll
      for (int k2 = 0; k2 < R2x; ++k2)
        if (!(a.disc && tile_outside(k1 + R1x * k2, h * NYH + r, NX, NY)))
          row[k1 + R1x * k2] = w[k2];
    }
    __syncthreads();    // work is rewritten by the next unit
  }
  plane_sync<NS>();   // no CTA leaves while its peer may still write into it
}

template <int NY, int NX, int WEIGHTED>
cudaError_t launch_xy_soft_one(const PassArgs& a, cudaStream_t s) {
  using C = XYCfg<NY, NX>;
  constexpr int NS = XYSplit<NY, NX>::NS;
  auto k = xy_soft_kernel<NY, NX, WEIGHTED>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)C::smem_bytes);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // a whole plane per CTA: as many CTAs as are resident at once; clusters:
  // two CTAs per SM
  int per_sm = 2;
  if constexpr (NS == 1) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, C::NT, C::smem_bytes);
    if (e != cudaSuccess) return e;
    per_sm = std::max(1, per_sm);
  }
  const int clusters =
      std::max(1, std::min(a.nz * a.nslots, NS == 1 ? per_sm * nsm : per_sm * nsm / NS));
  k<<<NS * clusters, C::NT, C::smem_bytes, s>>>(a);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// per-size launchers
// ----------------------------------------------------------------------------
template <int NZ>
cudaError_t launch_z_n(int mode, int ev, const PassArgs& a, int tiles, cudaStream_t s) {
  const dim3 block(kTileX * Plan<NZ>::R2);
  switch (mode) {
    case Z_FWD_PREP: z_kernel<NZ, Z_FWD_PREP, 0><<<tiles, block, 0, s>>>(a); break;
    case Z_INV_FINAL: z_kernel<NZ, Z_INV_FINAL, 0><<<tiles, block, 0, s>>>(a); break;
    case Z_FWD_SCORE:
      if (ev == 0) z_kernel<NZ, Z_FWD_SCORE, 0><<<tiles, block, 0, s>>>(a);
      else if (ev == 1) z_kernel<NZ, Z_FWD_SCORE, 1><<<tiles, block, 0, s>>>(a);
      else z_kernel<NZ, Z_FWD_SCORE, 2><<<tiles, block, 0, s>>>(a);
      break;
    case Z_INV_SCORE:
      if (ev == 0) z_kernel<NZ, Z_INV_SCORE, 0><<<tiles, block, 0, s>>>(a);
      else if (ev == 1) z_kernel<NZ, Z_INV_SCORE, 1><<<tiles, block, 0, s>>>(a);
      else z_kernel<NZ, Z_INV_SCORE, 2><<<tiles, block, 0, s>>>(a);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int NY, int NX, int MODE, int UB>
cudaError_t launch_xy_one(const PassArgs& a, cudaStream_t s) {
  using C = XYCfg<NY, NX>;
  auto k = xy_kernel<NY, NX, MODE, UB>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)C::smem_bytes);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int nsl = (MODE == XY_FWD_SCORE || MODE == XY_INV_SCORE || MODE == XY_INV_WSCORE)
                      ? a.nslots : 1;
  // two CTAs per SM, NS per cluster, looping over units; a whole plane per CTA:
  // as many CTAs as are resident at once
  constexpr int NS = XYSplit<NY, NX>::NS;
  int per_sm = 2;
  if constexpr (NS == 1) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, C::NT, C::smem_bytes);
    if (e != cudaSuccess) return e;
    per_sm = std::max(1, per_sm);
  }
  const int clusters = std::max(1, std::min(a.nz * nsl, NS == 1 ? per_sm * nsm : 2 * nsm / NS));
  k<<<NS * clusters, C::NT, C::smem_bytes, s>>>(a);
  return cudaGetLastError();
}

// the forward score pass on folded parts of planes (xy_fold_kernel): as many
// CTAs as are resident at once, a multiple of F so that the parts of a plane
// run side by side
template <int NY, int NX, int UB>
cudaError_t launch_xy_fold_one(const PassArgs& a, cudaStream_t s) {
  using FC = XYFoldCfg<NY, NX>;
  constexpr int F = FC::F;
  auto k = xy_fold_kernel<NY, NX, UB>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)FC::smem_bytes);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, FC::C::NT, FC::smem_bytes);
  if (e != cudaSuccess) return e;
  const int units = F * a.nz * a.nslots;
  const int grid = std::max(F, std::min(units, std::max(1, per_sm) * nsm) / F * F);
  k<<<grid, FC::C::NT, FC::smem_bytes, s>>>(a);
  return cudaGetLastError();
}

template <int NY, int NX>
cudaError_t launch_xy_n(int mode, int ub, const PassArgs& a, cudaStream_t s) {
  if constexpr (XYFold<NY, NX>::F == 4) {
    if (mode == XY_FWD_SCORE)
      return ub ? launch_xy_fold_one<NY, NX, 1>(a, s) : launch_xy_fold_one<NY, NX, 0>(a, s);
  } else if constexpr (XYFold<NY, NX>::F == 2) {
    // halves of 128^2 planes for complex64 scores only (with BF16 scores the
    // whole-plane pass measured 0.5 % faster per step)
    if (mode == XY_FWD_SCORE && !ub) return launch_xy_fold_one<NY, NX, 0>(a, s);
  }
  switch (mode) {
    case XY_FWD_REAL: return launch_xy_one<NY, NX, XY_FWD_REAL, 0>(a, s);
    case XY_INV_REAL: return launch_xy_one<NY, NX, XY_INV_REAL, 0>(a, s);
    case XY_FWD_SCORE:
      return ub ? launch_xy_one<NY, NX, XY_FWD_SCORE, 1>(a, s)
                : launch_xy_one<NY, NX, XY_FWD_SCORE, 0>(a, s);
    case XY_INV_SCORE:
      return ub ? launch_xy_one<NY, NX, XY_INV_SCORE, 1>(a, s)
                : launch_xy_one<NY, NX, XY_INV_SCORE, 0>(a, s);
    case XY_INV_WSCORE:
      if (ub) return cudaErrorInvalidValue;
      return launch_xy_one<NY, NX, XY_INV_WSCORE, 0>(a, s);
    case XY_SOFT: return launch_xy_soft_one<NY, NX, 0>(a, s);
    case XY_WENERGY: return launch_xy_soft_one<NY, NX, 1>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace os3d

// Per-size translation units instantiate these.
#define OS3D_DEFINE_Z(N)                                                                   \
  namespace os3d {                                                                         \
  cudaError_t launch_z_##N(int mode, int ev, const PassArgs& a, int tiles, cudaStream_t s) { \
    return launch_z_n<N>(mode, ev, a, tiles, s);                                           \
  }                                                                                        \
  }
#define OS3D_DEFINE_XY(NY, NX)                                                             \
  namespace os3d {                                                                         \
  cudaError_t launch_xy_##NY##_##NX(int mode, int ub, const PassArgs& a, cudaStream_t s) {  \
    return launch_xy_n<NY, NX>(mode, ub, a, s);                                            \
  }                                                                                        \
  }
