// Strided pencil pass: a 1D DFT along one axis for 16 parallel lines per CTA.
// Used for the x and y directions of grids whose z-planes do not fit the
// cluster xy-pass (planes larger than 128^2, or not square); the z direction
// always uses z_kernel. Lines of the volume are numbered L = 0 .. nlines-1;
// line L starts at (L / group) * gstride + (L % group) * lstride and its
// elements are estride apart. A CTA takes 16 consecutive lines of one group.
//   x axis: group = ny, gstride = ny nx, lstride = nx, estride = 1
//   y axis: group = nx, gstride = ny nx, lstride = 1,  estride = nx
#pragma once
#include <cuda_bf16.h>
#include "os3d_fft.cuh"
#include "os3d_kernels.cuh"

namespace os3d {

template <int UBF16>
__device__ __forceinline__ float2 pn_load_u(const void* base, long long i) {
  if constexpr (UBF16) {
    const unsigned int raw = __ldcs(reinterpret_cast<const unsigned int*>(base) + i);
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw));
  } else {
    return __ldcs(reinterpret_cast<const float2*>(base) + i);
  }
}
template <int UBF16>
__device__ __forceinline__ void pn_store_u(void* base, long long i, float2 v) {
  if constexpr (UBF16) {
    __nv_bfloat162 b = __floats2bfloat162_rn(v.x, v.y);
    __stcs(reinterpret_cast<unsigned int*>(base) + i, *reinterpret_cast<unsigned int*>(&b));
  } else {
    __stcs(reinterpret_cast<float2*>(base) + i, v);
  }
}

template <int N, int MODE, int DIR, int UBF16>
__global__ void __launch_bounds__(kTileX * Plan<N>::R2)
pencil_kernel(const __grid_constant__ PassArgs a, const __grid_constant__ PencilGeom g) {
  constexpr int R1 = Plan<N>::R1, R2 = Plan<N>::R2;
  constexpr int TW = kTileX;
  constexpr int J3 = (R1 + R2 - 1) / R2;
  __shared__ float2 tile[N * TW];
  __shared__ float2 tws[N];

  const int t = threadIdx.x;
  const int xl = t % TW, n2 = t / TW;
  const long long L = (long long)blockIdx.x * TW + xl;
  const long long line = (L / g.group) * g.gstride + (L % g.group) * g.lstride;
  const int s = blockIdx.y;

  fill_twiddles<N, DIR>(tws);
  float2 v[R1];
#pragma unroll
  for (int n1 = 0; n1 < R1; ++n1) {
    const long long e = line + (long long)(n2 + R2 * n1) * g.estride;
    if constexpr (MODE == PN_R2C) {
      v[n1] = make_float2(__ldg(reinterpret_cast<const float*>(a.in) + a.in_off + e), 0.f);
    } else if constexpr (MODE == PN_U2C) {
      float2 q = pn_load_u<UBF16>(a.in, a.ua[s] + e);
      if (a.ub[s] >= 0) q = cadd(q, cconj(pn_load_u<UBF16>(a.in, a.ub[s] + e)));
      v[n1] = q;
    } else {
      v[n1] = reinterpret_cast<const float2*>(a.in)[a.in_off + (long long)s * a.slot_stride + e];
    }
  }
  __syncthreads();   // twiddle table
  dft<R1, DIR>(v);
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1)
    tile[(n2 + R2 * k1) * TW + xl] = (k1 == 0) ? v[k1] : cmul(v[k1], tws[(n2 * k1) % N]);
  __syncthreads();
#pragma unroll
  for (int j = 0; j < J3; ++j) {
    const int k1 = n2 + R2 * j;
    if (R1 % R2 != 0 && k1 >= R1) break;
    float2 w[R2];
#pragma unroll
    for (int m = 0; m < R2; ++m) w[m] = tile[(m + R2 * k1) * TW + xl];
    dft<R2, DIR>(w);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const long long e = line + (long long)(k1 + R1 * k2) * g.estride;
      if constexpr (MODE == PN_C2R) {
        reinterpret_cast<float*>(a.out)[a.out_off + e] = w[k2].x;
      } else if constexpr (MODE == PN_C2U) {
        pn_store_u<UBF16>(a.out, a.ua[s] + e, w[k2]);
        if (a.ub[s] >= 0) pn_store_u<UBF16>(a.out, a.ub[s] + e, cconj(w[k2]));
      } else {
        reinterpret_cast<float2*>(a.out)[a.out_off + (long long)s * a.slot_stride + e] = w[k2];
      }
    }
  }
}

template <int N>
cudaError_t launch_pencil_n(int mode, int dir, int ub, const PassArgs& a, const PencilGeom& g,
                            long long nlines, int nslots, cudaStream_t s) {
  const dim3 block(kTileX * Plan<N>::R2);
  const dim3 grid((unsigned)(nlines / kTileX), (unsigned)nslots);
#define OS3D_PN(M, D, U) pencil_kernel<N, M, D, U><<<grid, block, 0, s>>>(a, g)
  switch (mode) {
    case PN_C2C:
      if (dir < 0) OS3D_PN(PN_C2C, -1, 0);
      else OS3D_PN(PN_C2C, 1, 0);
      break;
    case PN_R2C: OS3D_PN(PN_R2C, -1, 0); break;
    case PN_C2R: OS3D_PN(PN_C2R, 1, 0); break;
    case PN_C2U:
      if (ub) OS3D_PN(PN_C2U, 1, 1);
      else OS3D_PN(PN_C2U, 1, 0);
      break;
    case PN_U2C:
      if (ub) OS3D_PN(PN_U2C, -1, 1);
      else OS3D_PN(PN_U2C, -1, 0);
      break;
    default: return cudaErrorInvalidValue;
  }
#undef OS3D_PN
  return cudaGetLastError();
}

}  // namespace os3d

#define OS3D_DEFINE_PENCIL(N)                                                               \
  namespace os3d {                                                                          \
  cudaError_t launch_pencil_##N(int mode, int dir, int ub, const PassArgs& a,               \
                                const PencilGeom& g, long long nlines, int nslots,          \
                                cudaStream_t s) {                                           \
    return launch_pencil_n<N>(mode, dir, ub, a, g, nlines, nslots, s);                      \
  }                                                                                         \
  }
