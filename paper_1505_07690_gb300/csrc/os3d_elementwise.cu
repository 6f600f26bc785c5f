// Streaming kernels of the score domain (sm_103a): the orientation sum of the
// approximate reconstruction (Eq. Reconstruction2Approximation) and the soft
// threshold Phi(U) = |U|^p sgn(U) of Sec. 4.1, on whole scores and on the
// per-block intermediates. All are HBM-bound: 16-byte vector loads and
// stores, one pass over their data.
#include <cuda_bf16.h>
#include <algorithm>
#include "os3d_kernels.cuh"

namespace os3d {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float bf16_lo(unsigned v) { return __uint_as_float(v << 16); }

// out[x] = w sum_i Re U_i[x] for 4 consecutive voxels per thread.
template <int UBF16>
__global__ void __launch_bounds__(kThreads)
approx_sum_kernel(const void* __restrict__ U, int n_o, long long nvox, float w,
                  float* __restrict__ out) {
  const long long q = (long long)blockIdx.x * kThreads + threadIdx.x;   // quad index
  if (4 * q >= nvox) return;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  if constexpr (UBF16) {
    const uint4* p = reinterpret_cast<const uint4*>(U) + q;
    const long long step = nvox / 4;
#pragma unroll 8
    for (int i = 0; i < n_o; ++i) {
      const uint4 v = __ldcs(p + i * step);
      s0 += bf16_lo(v.x);
      s1 += bf16_lo(v.y);
      s2 += bf16_lo(v.z);
      s3 += bf16_lo(v.w);
    }
  } else {
    const float4* p = reinterpret_cast<const float4*>(U) + 2 * q;
    const long long step = nvox / 2;
#pragma unroll 8
    for (int i = 0; i < n_o; ++i) {
      const float4 a = __ldcs(p + i * step);
      const float4 b = __ldcs(p + i * step + 1);
      s0 += a.x;
      s1 += a.z;
      s2 += b.x;
      s3 += b.z;
    }
  }
  reinterpret_cast<float4*>(out)[q] = make_float4(w * s0, w * s1, w * s2, w * s3);
}

// Phi on every part of `count` complex elements (a multiple of 4), in place allowed.
template <int UBF16>
__global__ void __launch_bounds__(kThreads)
soft_scores_kernel(const void* in, void* out, long long count, float p) {
  const long long stride = (long long)gridDim.x * kThreads;
  if constexpr (UBF16) {
    const uint4* src = reinterpret_cast<const uint4*>(in);
    uint4* dst = reinterpret_cast<uint4*>(out);
    for (long long q = (long long)blockIdx.x * kThreads + threadIdx.x; 4 * q < count; q += stride) {
      uint4 v = __ldcs(src + q);
      unsigned* e = reinterpret_cast<unsigned*>(&v);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&e[j]));
        __nv_bfloat162 b = __floats2bfloat162_rn(soft_part(f.x, p), soft_part(f.y, p));
        e[j] = *reinterpret_cast<unsigned*>(&b);
      }
      __stcs(dst + q, v);
    }
  } else {
    const float4* src = reinterpret_cast<const float4*>(in);
    float4* dst = reinterpret_cast<float4*>(out);
    for (long long q = (long long)blockIdx.x * kThreads + threadIdx.x; 2 * q < count; q += stride) {
      const float4 v = __ldcs(src + q);
      __stcs(dst + q, make_float4(soft_part(v.x, p), soft_part(v.y, p), soft_part(v.z, p),
                                  soft_part(v.w, p)));
    }
  }
}

// m_s Phi on slot s = blockIdx.y of the block intermediates, in place.
__global__ void __launch_bounds__(kThreads)
soft_slots_kernel(const __grid_constant__ PassArgs a, long long nvox) {
  const int s = blockIdx.y;
  const float scale = a.ub[s] >= 0 ? 2.f : 1.f;
  float4* T = reinterpret_cast<float4*>(reinterpret_cast<float2*>(a.out) + s * a.slot_stride);
  const long long q = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (2 * q >= nvox) return;
  const float4 v = T[q];
  T[q] = make_float4(scale * soft_part(v.x, a.power), scale * soft_part(v.y, a.power),
                     scale * soft_part(v.z, a.power), scale * soft_part(v.w, a.power));
}

int grid_for(long long items) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long need = (items + kThreads - 1) / kThreads;
  return (int)std::max(1LL, std::min(need, (long long)nsm * 16));
}

}  // namespace

cudaError_t launch_approx_sum(const void* U, int ubf16, int n_o, long long nvox, float w,
                              float* out, cudaStream_t s) {
  const long long quads = nvox / 4;
  const unsigned grid = (unsigned)((quads + kThreads - 1) / kThreads);
  if (ubf16) approx_sum_kernel<1><<<grid, kThreads, 0, s>>>(U, n_o, nvox, w, out);
  else approx_sum_kernel<0><<<grid, kThreads, 0, s>>>(U, n_o, nvox, w, out);
  return cudaGetLastError();
}

cudaError_t launch_soft_scores(const void* in, void* out, int ubf16, long long count,
                               float power, cudaStream_t s) {
  if (ubf16) soft_scores_kernel<1><<<grid_for(count / 4), kThreads, 0, s>>>(in, out, count, power);
  else soft_scores_kernel<0><<<grid_for(count / 2), kThreads, 0, s>>>(in, out, count, power);
  return cudaGetLastError();
}

cudaError_t launch_soft_slots(const PassArgs& a, long long nvox, cudaStream_t s) {
  const dim3 grid((unsigned)((nvox / 2 + kThreads - 1) / kThreads), (unsigned)a.nslots);
  soft_slots_kernel<<<grid, kThreads, 0, s>>>(a, nvox);
  return cudaGetLastError();
}

}  // namespace os3d
