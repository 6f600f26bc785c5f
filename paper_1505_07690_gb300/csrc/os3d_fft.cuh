// In-register DFT codelets and two-stage FFT plans for the orientation-score
// kernels (sm_103a).
//
// A length-N transform along one axis is split N = R1 * R2 (Cooley-Tukey,
// "four step"): with input index n = n2 + R2*n1 and output index
// k = k1 + R1*k2,
//   X[k1 + R1 k2] = sum_{n2} W_R2^{n2 k2} W_N^{n2 k1} sum_{n1} x[n2 + R2 n1] W_R1^{n1 k1}.
// Step 1 (one thread per n2) is a DFT_R1 held in registers followed by the
// twiddle W_N^{n2 k1}; the data are exchanged through shared memory; step 2
// (one thread per k1) is a DFT_R2 in registers. The codelets below are
// written from the DFT definition; composite sizes are composed at compile
// time with constant twiddles computed by a constexpr series.
#pragma once
#include <cuda_runtime.h>
#include <type_traits>

namespace os3d {

// ----------------------------------------------------------------------------
// compile-time cos/sin(2 pi m / n) (Taylor series after reduction to [-pi, pi])
// ----------------------------------------------------------------------------
constexpr double kPi = 3.141592653589793238462643383279502884;

constexpr double ct_sin_red(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 40; ++k) {
    term *= -x * x / double((2 * k) * (2 * k + 1));
    sum += term;
  }
  return sum;
}
constexpr double ct_cos_red(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 40; ++k) {
    term *= -x * x / double((2 * k - 1) * (2 * k));
    sum += term;
  }
  return sum;
}
// angle 2 pi m / n reduced to [-pi, pi]
constexpr double ct_angle(long m, long n) {
  long r = ((m % n) + n) % n;
  if (2 * r > n) r -= n;
  return 2.0 * kPi * double(r) / double(n);
}
constexpr double ct_cos2pi(long m, long n) { return ct_cos_red(ct_angle(m, n)); }
constexpr double ct_sin2pi(long m, long n) { return ct_sin_red(ct_angle(m, n)); }

// ----------------------------------------------------------------------------
// complex helpers
// ----------------------------------------------------------------------------
// Complex sums use the packed two-lane FP32 instructions of sm_100+ (one
// instruction for both parts, rounded like two scalar adds).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
// d = a b + c and d = a b lane by lane (two-lane FP32, rounded like fmaf / a * b)
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
// as fma2, with c read as one 64-bit operand (a pair held in parameter memory)
__device__ __forceinline__ float2 fma2k(float2 a, float2 b, const float2& c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "fma.rn.f32x2 rd, ra, rb, %6;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y),
        "l"(*reinterpret_cast<const unsigned long long*>(&c)));
  return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// multiply by -i (dir = -1) or +i (dir = +1):  (+i)(x + iy) = -y + ix
template <int DIR> __device__ __forceinline__ float2 cmul_i(float2 a) {
  return DIR > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int I, int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// x * W_R^M with W_R = exp(DIR * 2 pi i / R); DIR = -1 forward, +1 inverse.
template <int R, int M, int DIR>
__device__ __forceinline__ float2 twiddle_ct(float2 x) {
  constexpr int m = ((M % R) + R) % R;
  if constexpr (m == 0) {
    return x;
  } else if constexpr (2 * m == R) {
    return make_float2(-x.x, -x.y);
  } else if constexpr (4 * m == R) {
    return cmul_i<DIR>(x);
  } else if constexpr (4 * m == 3 * R) {
    return cmul_i<-DIR>(x);
  } else if constexpr ((8 * m) % R == 0) {
    // odd multiples of pi/4: |cos| = |sin| = sqrt(1/2)
    constexpr float h = 0.70710678118654752440f;
    constexpr double c = ct_cos2pi(m, R);
    constexpr double s = DIR * ct_sin2pi(m, R);
    // (x + iy)(c + is) with c = +-h, s = +-h
    constexpr float cs = c > 0 ? h : -h;
    constexpr float ss = s > 0 ? h : -h;
    if constexpr ((c > 0) == (s > 0)) {
      return make_float2(cs * (x.x - x.y), cs * (x.x + x.y));
    } else {
      return make_float2(cs * (x.x + x.y), cs * (x.y - x.x));
    }
    (void)ss;
  } else {
    constexpr float c = float(ct_cos2pi(m, R));
    constexpr float s = float(DIR * ct_sin2pi(m, R));
    return make_float2(fmaf(x.x, c, -x.y * s), fmaf(x.x, s, x.y * c));
  }
}

// ----------------------------------------------------------------------------
// DFT_R in registers, natural order in and out, unnormalised.
// ----------------------------------------------------------------------------
constexpr int ct_first_factor(int r) {
  return (r % 4 == 0 && r != 8) ? 4 : (r % 2 == 0 ? 2 : (r % 3 == 0 ? 3 : (r % 5 == 0 ? 5 : r)));
}

template <int R, int DIR>
__device__ __forceinline__ void dft(float2* v) {
  if constexpr (R == 1) {
    return;
  } else if constexpr (R == 2) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if constexpr (R == 3) {
    constexpr float s3 = 0.86602540378443864676f;   // sin(2 pi / 3)
    float2 t1 = cadd(v[1], v[2]);
    float2 t2 = make_float2(fmaf(-0.5f, t1.x, v[0].x), fmaf(-0.5f, t1.y, v[0].y));
    float2 d = csub(v[1], v[2]);
    // DIR * i * s3 * d
    float2 e = cmul_i<DIR>(cscale(d, s3));
    v[0] = cadd(v[0], t1);
    v[1] = cadd(t2, e);
    v[2] = csub(t2, e);
  } else if constexpr (R == 4) {
    float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    float2 t2 = cadd(v[1], v[3]), t3 = cmul_i<DIR>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  } else if constexpr (R == 5) {
    constexpr float c1 = float(ct_cos2pi(1, 5)), c2 = float(ct_cos2pi(2, 5));
    constexpr float s1 = float(ct_sin2pi(1, 5)), s2 = float(ct_sin2pi(2, 5));
    float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    float2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    float2 a1 = make_float2(fmaf(c1, t1.x, fmaf(c2, t2.x, v[0].x)), fmaf(c1, t1.y, fmaf(c2, t2.y, v[0].y)));
    float2 a2 = make_float2(fmaf(c2, t1.x, fmaf(c1, t2.x, v[0].x)), fmaf(c2, t1.y, fmaf(c1, t2.y, v[0].y)));
    float2 b1 = make_float2(fmaf(s1, t3.x, s2 * t4.x), fmaf(s1, t3.y, s2 * t4.y));
    float2 b2 = make_float2(fmaf(s2, t3.x, -s1 * t4.x), fmaf(s2, t3.y, -s1 * t4.y));
    // X_k = a + DIR * i * b   (W^k = cos + DIR i sin)
    float2 e1 = cmul_i<DIR>(b1), e2 = cmul_i<DIR>(b2);
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(a1, e1);
    v[4] = csub(a1, e1);
    v[2] = cadd(a2, e2);
    v[3] = csub(a2, e2);
  } else {
    constexpr int A = ct_first_factor(R);
    constexpr int B = R / A;
    static_assert(A * B == R && A > 1 && B > 1, "unsupported DFT size");
    float2 y[R];
    static_for<0, B>([&](auto n2c) {
      constexpr int n2 = decltype(n2c)::value;
      float2 t[A];
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) t[n1] = v[n2 + B * n1];
      dft<A, DIR>(t);
      static_for<0, A>([&](auto k1c) {
        constexpr int k1 = decltype(k1c)::value;
        y[n2 * A + k1] = twiddle_ct<R, n2 * k1, DIR>(t[k1]);
      });
    });
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      float2 t[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) t[n2] = y[n2 * A + k1];
      dft<B, DIR>(t);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = t[k2];
    }
  }
}

// ----------------------------------------------------------------------------
// Two-stage plans N = R1 * R2 for the supported axis lengths.
// ----------------------------------------------------------------------------
template <int N> struct Plan;
template <> struct Plan<16>  { static constexpr int R1 = 4,  R2 = 4; };
template <> struct Plan<32>  { static constexpr int R1 = 8,  R2 = 4; };
template <> struct Plan<48>  { static constexpr int R1 = 12, R2 = 4; };
template <> struct Plan<64>  { static constexpr int R1 = 8,  R2 = 8; };
template <> struct Plan<96>  { static constexpr int R1 = 12, R2 = 8; };
template <> struct Plan<128> { static constexpr int R1 = 16, R2 = 8; };
template <> struct Plan<160> { static constexpr int R1 = 20, R2 = 8; };
template <> struct Plan<256> { static constexpr int R1 = 16, R2 = 16; };

// Twiddle table W_N^m = exp(DIR 2 pi i m / N), m < N, in shared memory.
template <int N, int DIR>
__device__ __forceinline__ void fill_twiddles(float2* tw) {
  for (int m = threadIdx.x; m < N; m += blockDim.x) {
    float s, c;
    sincospif(2.0f * float(m) / float(N), &s, &c);
    tw[m] = make_float2(c, DIR * s);
  }
}

}  // namespace os3d
