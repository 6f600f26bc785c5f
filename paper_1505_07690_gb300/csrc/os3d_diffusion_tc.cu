// Linear left-invariant diffusion (Sec. 4.1, constant diagonal D_ij) with the
// propagator product on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The same per-frequency integration as enhance_kernel (os3d_diffusion.cu):
// for each listed frequency w the N_o-vector v = h(w) F(w) goes through K
// Strang steps v <- F (E (F v)), F = diag(exp(-dt/2 r_i(w))), E = exp(dt D44 L),
// and m(w) = h^T v. Here a CTA of one warpgroup takes 128 frequencies at a
// time and each step is the GEMM
//   D[q][i] = sum_j V[q][j] E[i][j]      (M = 128 frequencies, N = K = N_o padded to 16)
// issued by one thread as tcgen05.mma kind::f16 with FP32 accumulation in
// tensor memory. FP32 accuracy from half-precision operands: every operand is
// split into a high and a low half, x = x_hi + x_lo, and D = V_hi E_hi^T +
// V_hi E_lo^T + V_lo E_hi^T (the dropped V_lo E_lo^T is below 2^-22 of the
// result). E is scaled once by a power of two so that max |E| is in [1/2, 1),
// every row of V (one frequency) before every step likewise, so that the low
// halves stay in the normal range of half precision; the scales are undone
// exactly in FP32.
//
// Thread q owns frequency q of the tile, which is lane q of tensor memory: it
// computes its geometry, h and the spatial factors F (kept in tensor memory,
// columns N..2N-1, next to the accumulator in columns 0..N-1), reads its row
// of D back after each step, applies F^2 (F after the last step) and writes
// the next V_hi / V_lo row into shared memory in the canonical K-major layout
// (8 x 16-byte core matrices). Waits for the MMA are bounded (1 s of global
// time); a wait that runs out counts in a.err and the kernel carries on.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>
#include <cuda_fp16.h>
#include "os3d_passes.cuh"

namespace os3d {

namespace {

constexpr int kTVtc = 128;   // frequencies per tile = M of the MMA

__device__ __forceinline__ unsigned long long gtimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity,
                                                  unsigned long long limit_ns = 1000000000ull) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer_ns();
  while (!mbar_try(bar, parity))
    if (gtimer_ns() - t0 > limit_ns) return false;
  return true;
}

// Self-test of the bounded wait: one CTA waits on an mbarrier of its own;
// with `arrive` thread 0 arrives first (the wait completes), otherwise
// nothing ever arrives and every thread's wait runs out after limit_ns.
__global__ void wait_selftest_kernel(unsigned long long limit_ns, int arrive, unsigned* timeouts) {
  __shared__ __align__(8) unsigned long long mb;
  const unsigned bar = smem_addr(&mb);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0)
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
  if (!mbar_wait_bounded(bar, 0, limit_ns)) atomicAdd(timeouts, 1u);
}
// shared-memory matrix descriptor, no swizzle: start address, LBO (next core
// matrix along K), SBO (next 8-row group along M / N), descriptor version 1
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((addr >> 4) & 0x3FFF) |
         ((unsigned long long)((lbo >> 4) & 0x3FFF) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// instruction descriptor, kind::f16: f16 A and B (K-major), f32 D, M x N
constexpr unsigned idesc_f16(int M, int N) {
  return (1u << 4) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_f16(unsigned dtm, unsigned long long da, unsigned long long db,
                                        unsigned idesc, unsigned acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtm),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tmem_st16(unsigned taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}
// power of two s with max|x| s in [1/2, 1) (1 for an all-zero row; bounded
// so that s stays finite for subnormal maxima)
__device__ __forceinline__ float row_scale(float vmax) {
  if (!(vmax > 0.f)) return 1.f;
  int e;
  frexpf(vmax, &e);
  return ldexpf(1.f, -max(e, -120));
}
__device__ __forceinline__ unsigned pack_h2(__half a, __half b) {
  return (unsigned)__half_as_ushort(a) | ((unsigned)__half_as_ushort(b) << 16);
}

template <int NP>
struct TcLayout {
  static constexpr int TV = kTVtc;
  static constexpr unsigned LBO = 128;                  // core matrices along K
  static constexpr unsigned SBO = (NP / 8) * 128;       // 8-row groups
  static constexpr size_t EBYTES = (size_t)NP * NP * 2; // one half-precision E
  static constexpr size_t VBYTES = (size_t)TV * NP * 2; // one half-precision V
  static constexpr size_t OFF_V = 2 * EBYTES;
  static constexpr size_t OFF_NV = 2 * EBYTES + 2 * VBYTES;
  static constexpr size_t OFF_RED = OFF_NV + sizeof(float) * 3 * NP;    // 4 x 128 floats
  static constexpr size_t OFF_MISC = OFF_RED + sizeof(float) * 4 * TV;  // tmem slot, 2 mbarriers
  static constexpr size_t BYTES = OFF_MISC + 32;
  static constexpr int TCOLS = 2 * NP <= 32 ? 32 : 2 * NP <= 64 ? 64 : 2 * NP <= 128 ? 128
                             : 2 * NP <= 256 ? 256 : 512;
  static_assert(NP % 16 == 0 && NP <= 256 && 2 * NP <= 512, "orientations padded to 16, <= 256");
  static_assert(OFF_MISC % 16 == 0, "alignment");
};

// Splits row q (16 columns of chunk c, already scaled) into the high and low
// halves and stores them as the two 16-byte core-matrix rows of chunk c.
template <int NP>
__device__ __forceinline__ void store_split(unsigned char* sVhi, unsigned char* sVlo, int q, int c,
                                            const float (&x)[16]) {
  using L = TcLayout<NP>;
  unsigned hi[8], lo[8];
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const __half h0 = __float2half_rn(x[2 * p]), h1 = __float2half_rn(x[2 * p + 1]);
    const __half l0 = __float2half_rn(x[2 * p] - __half2float(h0));
    const __half l1 = __float2half_rn(x[2 * p + 1] - __half2float(h1));
    hi[p] = pack_h2(h0, h1);
    lo[p] = pack_h2(l0, l1);
  }
  const size_t off = (size_t)(q / 8) * L::SBO + (size_t)(2 * c) * L::LBO + (q % 8) * 16;
  *reinterpret_cast<uint4*>(sVhi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
  *reinterpret_cast<uint4*>(sVhi + off + L::LBO) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
  *reinterpret_cast<uint4*>(sVlo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
  *reinterpret_cast<uint4*>(sVlo + off + L::LBO) = make_uint4(lo[4], lo[5], lo[6], lo[7]);
}

// 16 tensor-memory columns of this thread's lane into r, without the wait:
// several are issued before one tcgen05.wait::ld
__device__ __forceinline__ void tmem_ld16_async(unsigned taddr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
// the wait for the loads issued so far; the values pass through an empty asm
// after it, so no use of them can be scheduled before the wait
template <int G>
__device__ __forceinline__ void tmem_wait(float (&v)[G][16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int g = 0; g < G; ++g)
#pragma unroll
    for (int j = 0; j < 16; ++j) asm volatile("" : "+f"(v[g][j]));
}

// Column split of the tile: two MMA groups (columns [0, N0) and [N0, NP),
// each with its own commit), each served by two warpgroups; four warpgroups
// on the same 128 lanes, each with a contiguous range of 16-column chunks.
template <int NP>
struct TcSplit {
  static constexpr int NCH = NP / 16;
  static constexpr int CG0 = (NCH + 1) / 2;            // chunks of MMA group 0
  static constexpr int N0 = 16 * CG0, N1 = NP - N0;    // columns of the two groups
  static __host__ __device__ constexpr int begin(int wg) {
    return wg == 0 ? 0 : wg == 1 ? (CG0 + 1) / 2 : wg == 2 ? CG0 : CG0 + (NCH - CG0 + 1) / 2;
  }
  static __host__ __device__ constexpr int end(int wg) { return wg == 3 ? NCH : begin(wg + 1); }
  static __host__ __device__ constexpr int most() {   // most chunks of one warpgroup
    int m = 0;
    for (int w = 0; w < 4; ++w) m = end(w) - begin(w) > m ? end(w) - begin(w) : m;
    return m;
  }
  static_assert(N1 >= 16, "both MMA groups non-empty");
};

template <int NP, int EV>
__global__ void __launch_bounds__(512, 1) enhance_tc_kernel(const __grid_constant__ EnhanceTCArgs a) {
  using L = TcLayout<NP>;
  using S = TcSplit<NP>;
  constexpr int TV = L::TV, NCH = NP / 16, NWG = 4;
  constexpr int G = 1;                // chunks loaded per wait (16 warps hide the latency)
  extern __shared__ __align__(128) unsigned char esm[];
  unsigned char* sEhi = esm;
  unsigned char* sElo = esm + L::EBYTES;
  unsigned char* sVhi = esm + L::OFF_V;
  unsigned char* sVlo = sVhi + L::VBYTES;
  float* nv = reinterpret_cast<float*>(esm + L::OFF_NV);
  float* red = reinterpret_cast<float*>(esm + L::OFF_RED);   // per-row partials of the warpgroups
  unsigned* tslot = reinterpret_cast<unsigned*>(esm + L::OFF_MISC);
  const unsigned bar0 = smem_addr(esm + L::OFF_MISC + 16), bar1 = bar0 + 8;
  const int t = threadIdx.x, warp = t >> 5, q = t & (TV - 1), wg = t / TV;
  const int cbeg = S::begin(wg), cend = S::end(wg);
  const unsigned my_bar = wg < 2 ? bar0 : bar1;

  // E_hi, E_lo (prepared on the host in the canonical layout) and orientations
  for (size_t o = 16 * (size_t)t; o < 2 * L::EBYTES; o += 16 * 512)
    *reinterpret_cast<uint4*>(esm + o) = *reinterpret_cast<const uint4*>(a.prep + o);
  for (int o = t; o < 3 * NP; o += 512)
    nv[o] = reinterpret_cast<const float*>(a.prep + 2 * L::EBYTES)[o];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tslot)),
                 "n"(L::TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tslot;
  const unsigned lane_sel = (unsigned)(32 * (warp & 3)) << 16;   // lanes 32 (w % 4) ..
  const unsigned tD = tmem + lane_sel, tF = tmem + lane_sel + NP;
  constexpr unsigned IDESC0 = idesc_f16(TV, S::N0), IDESC1 = idesc_f16(TV, S::N1);
  unsigned phase = 0;
  bool lost = false;

  // reduction of the row's partial values of the four warpgroups
  auto row_reduce = [&](float m, bool take_max) {
    red[wg * TV + q] = m;
    __syncthreads();
    float r = red[q];
#pragma unroll
    for (int g = 1; g < NWG; ++g) r = take_max ? fmaxf(r, red[g * TV + q]) : r + red[g * TV + q];
    __syncthreads();
    return r;
  };
  // V_hi / V_lo of this thread's chunks from the accumulator columns, scaled by sc
  auto split_to_smem = [&](float sc) {
#pragma unroll 1
    for (int c0 = cbeg; c0 < cend; c0 += G) {
      float x[G][16];
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (c0 + g < cend) tmem_ld16_async(tD + 16 * (c0 + g), x[g]);
      tmem_wait<G>(x);
#pragma unroll
      for (int g = 0; g < G; ++g) {
        if (c0 + g < cend) {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) x[g][jj] *= sc;
          store_split<NP>(sVhi, sVlo, q, c0 + g, x[g]);
        }
      }
    }
  };

  const int ntiles = (a.n_in + TV - 1) / TV;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // ---- this thread's frequency
    const int gi = tile * TV + q;
    int vox = -1, mvox = -1;
    float wx = 0.f, wy = 0.f, wz = 0.f, r2 = 0.f, rinv = 0.f;
    if (gi < a.n_in) {
      int lo = 0, hi = a.nseg - 1;   // last segment with first index <= gi
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.seg[mid].w <= gi) lo = mid;
        else hi = mid - 1;
      }
      const int4 sg = a.seg[lo];
      const int kx = sg.z + (gi - sg.w);
      const int z = sg.x, y = sg.y, x = kx < 0 ? kx + a.nx : kx;
      vox = (z * a.ny + y) * a.nx + x;
      if (a.mirror) {
        const int mz = z ? a.nz - z : 0, my = y ? a.ny - y : 0, mx = x ? a.nx - x : 0;
        const int m = (mz * a.ny + my) * a.nx + mx;
        if (m != vox) mvox = m;
      }
      wz = float(z >= (a.nz + 1) / 2 ? z - a.nz : z) * a.wz;
      wy = float(y >= (a.ny + 1) / 2 ? y - a.ny : y) * a.wy;
      wx = float(kx) * a.wx;
      r2 = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
      rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
    }
    auto h_of = [&](float tau) { return r2 > 0.f ? eval_h<EV>(a.h, tau * rinv) : a.h.c0; };
    // ---- F into tensor memory, V0 = h F (unscaled) into the accumulator columns
    float vmax = 0.f;
#pragma unroll 1
    for (int c = cbeg; c < cend; ++c) {
      float Fv[16], Vv[16];
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const int i = 16 * c + jj;
        Fv[jj] = 0.f;
        Vv[jj] = 0.f;
        if (vox >= 0 && i < a.n_o) {
          const float tau = fmaf(wx, nv[3 * i], fmaf(wy, nv[3 * i + 1], wz * nv[3 * i + 2]));
          Fv[jj] = expf(-a.half_dt * fmaf(a.D11, r2 - tau * tau, a.D33 * tau * tau));
          Vv[jj] = h_of(tau) * Fv[jj];
          vmax = fmaxf(vmax, fabsf(Vv[jj]));
        }
      }
      tmem_st16(tF + 16 * c, Fv);
      tmem_st16(tD + 16 * c, Vv);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    float sq = row_scale(row_reduce(vmax, true));
    split_to_smem(sq);
    float msum = 0.f;
#pragma unroll 1
    for (int s = 0; s < a.steps; ++s) {
      // ---- D = V E^T (three products of the split operands) in two column
      // groups, each completing on its own mbarrier; one thread issues
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (t == 0) {
        const unsigned vh = smem_addr(sVhi), vl = smem_addr(sVlo);
#pragma unroll
        for (int grp = 0; grp < 2; ++grp) {
          const unsigned eh = smem_addr(sEhi) + (grp ? (S::N0 / 8) * L::SBO : 0u);
          const unsigned el = smem_addr(sElo) + (grp ? (S::N0 / 8) * L::SBO : 0u);
          const unsigned dcol = tmem + (grp ? (unsigned)S::N0 : 0u);
          const unsigned id = grp ? IDESC1 : IDESC0;
#pragma unroll 1
          for (int kk = 0; kk < NCH; ++kk)
            mma_f16(dcol, smem_desc(vh + kk * 2 * L::LBO, L::LBO, L::SBO),
                    smem_desc(eh + kk * 2 * L::LBO, L::LBO, L::SBO), id, kk > 0);
#pragma unroll 1
          for (int kk = 0; kk < NCH; ++kk)
            mma_f16(dcol, smem_desc(vh + kk * 2 * L::LBO, L::LBO, L::SBO),
                    smem_desc(el + kk * 2 * L::LBO, L::LBO, L::SBO), id, 1);
#pragma unroll 1
          for (int kk = 0; kk < NCH; ++kk)
            mma_f16(dcol, smem_desc(vl + kk * 2 * L::LBO, L::LBO, L::SBO),
                    smem_desc(eh + kk * 2 * L::LBO, L::LBO, L::SBO), id, 1);
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  grp ? bar1 : bar0)
              : "memory");
        }
      }
      if (!mbar_wait_bounded(my_bar, phase)) lost = true;
      phase ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // ---- W = F^2 D (F D after the last step), scales undone; this
      // thread's chunks of W stay in registers until the row's scale is known
      const bool last = s == a.steps - 1;
      const float undo = a.inv_se / sq;
      float wmax = 0.f;
      float wv[S::most()][16];
#pragma unroll
      for (int ci = 0; ci < S::most(); ++ci) {
        const int c = cbeg + ci;
        if (c >= cend) break;
        float d[1][16], f[1][16];
        tmem_ld16_async(tD + 16 * c, d[0]);
        tmem_ld16_async(tF + 16 * c, f[0]);
        tmem_wait<1>(d);
        tmem_wait<1>(f);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const float w = d[0][jj] * undo * (last ? f[0][jj] : f[0][jj] * f[0][jj]);
          wv[ci][jj] = w;
          wmax = fmaxf(wmax, fabsf(w));
        }
        if (last) {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int i = 16 * c + jj;
            if (vox >= 0 && i < a.n_o) {
              const float tau = fmaf(wx, nv[3 * i], fmaf(wy, nv[3 * i + 1], wz * nv[3 * i + 2]));
              msum = fmaf(h_of(tau), wv[ci][jj], msum);
            }
          }
        }
      }
      if (!last) {
        // the row's maximum over the four warpgroups: one barrier (red is
        // written again only after the next step's barrier)
        red[wg * TV + q] = wmax;
        __syncthreads();
        float r = red[q];
#pragma unroll
        for (int g = 1; g < NWG; ++g) r = fmaxf(r, red[g * TV + q]);
        sq = row_scale(r);
#pragma unroll
        for (int ci = 0; ci < S::most(); ++ci) {
          const int c = cbeg + ci;
          if (c >= cend) break;
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) wv[ci][jj] *= sq;
          store_split<NP>(sVhi, sVlo, q, c, wv[ci]);
        }
      }
    }
    // m = h^T v: the warpgroups' partial sums of the row
    const float mtot = row_reduce(msum, false);
    if (wg == 0 && vox >= 0) {
      const float m = mtot * a.n3;
      const float2 fh = a.fh[vox];
      a.A[vox] = make_float2(fh.x * m, fh.y * m);
      if (mvox >= 0) {
        const float2 fm = a.fh[mvox];
        a.A[mvox] = make_float2(fm.x * m, fm.y * m);
      }
    }
  }
  if (lost && (t & 127) == 0 && a.err) atomicAdd(a.err, 1u);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(L::TCOLS)
                 : "memory");
}

template <int NP, int EV>
cudaError_t launch_tc_np(const EnhanceTCArgs& a, cudaStream_t s) {
  using L = TcLayout<NP>;
  auto k = enhance_tc_kernel<NP, EV>;
  // shared memory requested so that the resident CTAs never ask for more
  // tensor-memory columns than an SM has (512)
  const int max_ctas = 512 / L::TCOLS;
  const size_t smem = std::max(L::BYTES, (size_t)(227 * 1024) / max_ctas - 1024);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 512, smem);
  if (e != cudaSuccess) return e;
  per_sm = std::max(1, std::min(per_sm, max_ctas));
  const int ntiles = (a.n_in + kTVtc - 1) / kTVtc;
  const int grid = std::max(1, std::min(ntiles, nsm * per_sm));
  k<<<grid, 512, smem, s>>>(a);
  return cudaGetLastError();
}

template <int NP>
cudaError_t launch_tc_ev(const EnhanceTCArgs& a, int ev, cudaStream_t s) {
  if (ev == 0) return launch_tc_np<NP, 0>(a, s);
  if (ev == 1) return launch_tc_np<NP, 1>(a, s);
  return launch_tc_np<NP, 2>(a, s);
}

// half-precision bits of x, round to nearest even (host)
unsigned short half_bits(float x) { return __half_as_ushort(__float2half_rn(x)); }
float half_value(unsigned short b) { return __half2float(__ushort_as_half(b)); }

}  // namespace

cudaError_t launch_wait_selftest(unsigned long long limit_ns, int arrive, unsigned* timeouts,
                                 cudaStream_t s) {
  wait_selftest_kernel<<<1, 64, 0, s>>>(limit_ns, arrive, timeouts);
  return cudaGetLastError();
}

int tc_padded_orientations(int n_o) {
  for (int np : {48, 64, 96, 128, 176})
    if (n_o <= np) return np;
  return -1;
}

size_t tc_prep_bytes(int np) { return 2 * (size_t)np * np * 2 + sizeof(float) * 3 * np; }

// Host: E (n x n, row-major FP64) and the orientations into the kernel's
// layout: E scaled by a power of two, split into half-precision high and low
// parts, each in the canonical K-major layout (element (i, j) at byte
// (i/8) SBO + (j/8) 128 + (i%8) 16 + (j%8) 2), zero-padded to np; then the
// orientations as np x 3 floats. Returns 1 / scale.
float tc_prepare(const double* E, const double* orient, int n, int np, std::vector<unsigned char>& out) {
  out.assign(tc_prep_bytes(np), 0);
  double emax = 0.0;
  for (int q = 0; q < n * n; ++q) emax = std::max(emax, std::fabs(E[q]));
  int e = 0;
  if (emax > 0.0) std::frexp(emax, &e);
  const double scale = std::ldexp(1.0, -e);
  const size_t sbo = (size_t)(np / 8) * 128;
  unsigned short* hi = reinterpret_cast<unsigned short*>(out.data());
  unsigned short* lo = hi + (size_t)np * np;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const size_t off = ((size_t)(i / 8) * sbo + (size_t)(j / 8) * 128 + (i % 8) * 16 + (j % 8) * 2) / 2;
      const float x = (float)(E[(size_t)i * n + j] * scale);
      const double xd = E[(size_t)i * n + j] * scale;
      hi[off] = half_bits(x);
      lo[off] = half_bits((float)(xd - (double)half_value(hi[off])));
    }
  float* nvp = reinterpret_cast<float*>(out.data() + 2 * (size_t)np * np * 2);
  for (int i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d) nvp[3 * i + d] = (float)orient[3 * i + d];
  return (float)(1.0 / scale);
}

cudaError_t launch_enhance_tc(const EnhanceTCArgs& a, int ev, cudaStream_t s) {
  switch (tc_padded_orientations(a.n_o)) {
    case 48: return launch_tc_ev<48>(a, ev, s);
    case 64: return launch_tc_ev<64>(a, ev, s);
    case 96: return launch_tc_ev<96>(a, ev, s);
    case 128: return launch_tc_ev<128>(a, ev, s);
    case 176: return launch_tc_ev<176>(a, ev, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace os3d
