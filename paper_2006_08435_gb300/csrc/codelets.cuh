// Register-resident DFT codelets for the 1D transforms of the separable 3D
// DFT (the paper, section "Approach": 1D FFTs along x, then y, then z).
//
// DFT<R, DIR>::run(v) replaces v[0..R) by X[k] = sum_n v[n] W_R^(n k),
// W_R = exp(DIR * 2 pi i / R), natural order in and out, R in
// {1,2,3,4,5,6,8,9,10,12,15,16,24,32,40,48,64}.  Radices 2, 3, 4, 5 are written out;
// composite R = R1*R2 is the four-step split
//   a[n1][k2] = DFT_R2 over n2 of v[n1 + R1 n2],   a[n1][k2] *= W_R^(n1 k2),
//   X[k2 + R2 k1] = DFT_R1 over n1 of a[n1][k2],
// with every index a compile-time constant so the twiddles fold into
// literal constants (trivial ones become swaps and sign flips).
//
// The constants cos(2 pi m / R), sin(2 pi m / R) are evaluated at compile
// time by a Taylor series in double precision written here (no math library
// call), then rounded to float.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#define FFT3D_HD __host__ __device__ __forceinline__

namespace fft3d {

// ---------------------------------------------------------------- complex ops
// Complex add/sub as one packed two-lane FP32 instruction on sm_100+
// (add/sub.rn.f32x2: the same IEEE round-to-nearest as two scalar adds).
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000) && !defined(FFT3D_NO_F32X2)
__device__ __forceinline__ unsigned long long pack2(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
  return unpack2(r);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
  return unpack2(r);
}
// Lane-wise a * b + c and a * b (fma/mul.rn.f32x2).
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)), "l"(pack2(c)));
  return unpack2(r);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
  return unpack2(r);
}
#else
FFT3D_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
FFT3D_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
FFT3D_HD float2 fma2(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
}
FFT3D_HD float2 mul2(float2 a, float2 b) { return make_float2(a.x * b.x, a.y * b.y); }
#endif
FFT3D_HD float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// a * w with w a forward (DIR = -1) table twiddle; the inverse uses conj(w).
template <int DIR>
FFT3D_HD float2 cmul_tw(float2 a, float2 w) {
  if constexpr (DIR < 0)
    return make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
  else
    return make_float2(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
}

// a * (S * i), S = +1 or -1:  i (x + i y) = -y + i x.
template <int S>
FFT3D_HD float2 mul_i(float2 a) {
  if constexpr (S > 0)
    return make_float2(-a.y, a.x);
  else
    return make_float2(a.y, -a.x);
}

// ------------------------------------------------ compile-time trigonometry
constexpr double kPi = 3.14159265358979323846264338327950288;

__host__ __device__ constexpr double series_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 30; ++k) {
    term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double series_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 30; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}
// angle 2 pi m / R reduced to [-pi, pi] on the integer before the series.
__host__ __device__ constexpr double turn_angle(int m, int R) {
  int r = ((m % R) + R) % R;
  if (2 * r > R) r -= R;
  return 2.0 * kPi * (double)r / (double)R;
}
__host__ __device__ constexpr double turn_cos(int m, int R) { return series_cos(turn_angle(m, R)); }
__host__ __device__ constexpr double turn_sin(int m, int R) { return series_sin(turn_angle(m, R)); }

// ---------------------------------------------------- static unrolled loops
template <int I, int N, class F>
FFT3D_HD void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// a * W_R^M with W_R = exp(DIR 2 pi i / R), all compile-time.
template <int M, int R, int DIR>
FFT3D_HD float2 twc(float2 a) {
  constexpr int m = ((M % R) + R) % R;
  if constexpr (m == 0) {
    return a;
  } else if constexpr (2 * m == R) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (4 * m == R) {
    return mul_i<DIR>(a);
  } else if constexpr (4 * m == 3 * R) {
    return mul_i<-DIR>(a);
  } else if constexpr ((8 * m) % R == 0) {
    // odd multiple of an eighth turn: (+-1 +- i) / sqrt(2)
    constexpr int k = 8 * m / R;
    constexpr float h = 0.70710678118654752440f;
    constexpr float cr = (k == 1 || k == 7) ? 1.0f : -1.0f;
    constexpr float ci = ((k == 1 || k == 3) ? 1.0f : -1.0f) * (float)DIR;
    return make_float2((cr * a.x - ci * a.y) * h, (ci * a.x + cr * a.y) * h);
  } else {
    constexpr float c = (float)turn_cos(m, R);
    constexpr float s = (float)((double)DIR * turn_sin(m, R));
    return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
  }
}

// ------------------------------------------------------------------ codelets
__host__ __device__ constexpr int first_factor(int R) {
  return R == 64 ? 8 : R == 48 ? 4 : R == 40 ? 8 : R == 32 ? 4 : R == 24 ? 8 : R == 16 ? 4
         : R == 12 ? 4 : R % 2 == 0 ? 2 : R % 3 == 0 ? 3 : R;
}

template <int R, int DIR>
struct DFT {
  static_assert(R == 6 || R == 8 || R == 9 || R == 10 || R == 12 || R == 15 || R == 16 ||
                    R == 24 || R == 32 || R == 40 || R == 48 || R == 64,
                "unsupported codelet radix");
  static constexpr int R1 = first_factor(R);
  static constexpr int R2 = R / R1;
  static FFT3D_HD void run(float2* v);
};

template <int DIR>
struct DFT<1, DIR> {
  static FFT3D_HD void run(float2*) {}
};

template <int DIR>
struct DFT<2, DIR> {
  static FFT3D_HD void run(float2* v) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <int DIR>
struct DFT<3, DIR> {
  static FFT3D_HD void run(float2* v) {
    // W = -1/2 + DIR i sqrt(3)/2
    constexpr float h3 = 0.86602540378443864676f;
    const float2 a = v[0], t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
    const float2 m = make_float2(a.x - 0.5f * t1.x, a.y - 0.5f * t1.y);
    const float2 r = mul_i<DIR>(cscale(t2, h3));
    v[0] = cadd(a, t1);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
  }
};

template <int DIR>
struct DFT<4, DIR> {
  static FFT3D_HD void run(float2* v) {
    const float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const float2 s13 = cadd(v[1], v[3]), d13 = mul_i<DIR>(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
  }
};

template <int DIR>
struct DFT<5, DIR> {
  static FFT3D_HD void run(float2* v) {
    constexpr float c1 = 0.30901699437494742410f;   // cos(2 pi/5)
    constexpr float c2 = -0.80901699437494742410f;  // cos(4 pi/5)
    constexpr float s1 = 0.95105651629515357212f;   // sin(2 pi/5)
    constexpr float s2 = 0.58778525229247312917f;   // sin(4 pi/5)
    const float2 x0 = v[0];
    const float2 t1 = cadd(v[1], v[4]), t3 = csub(v[1], v[4]);
    const float2 t2 = cadd(v[2], v[3]), t4 = csub(v[2], v[3]);
    const float2 a1 = make_float2(x0.x + c1 * t1.x + c2 * t2.x, x0.y + c1 * t1.y + c2 * t2.y);
    const float2 a2 = make_float2(x0.x + c2 * t1.x + c1 * t2.x, x0.y + c2 * t1.y + c1 * t2.y);
    const float2 b1 = mul_i<DIR>(make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
    const float2 b2 = mul_i<DIR>(make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
    v[0] = cadd(x0, cadd(t1, t2));
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
  }
};

template <int R, int DIR>
FFT3D_HD void DFT<R, DIR>::run(float2* v) {
  float2 a[R1][R2];
  static_for<0, R1>([&](auto I1) {
    constexpr int n1 = decltype(I1)::value;
    static_for<0, R2>([&](auto I2) { a[n1][decltype(I2)::value] = v[n1 + R1 * decltype(I2)::value]; });
    DFT<R2, DIR>::run(a[n1]);
    static_for<1, R2>([&](auto K2) {
      constexpr int k2 = decltype(K2)::value;
      a[n1][k2] = twc<n1 * k2, R, DIR>(a[n1][k2]);
    });
  });
  static_for<0, R2>([&](auto K2) {
    constexpr int k2 = decltype(K2)::value;
    float2 b[R1];
    static_for<0, R1>([&](auto I1) { b[decltype(I1)::value] = a[decltype(I1)::value][k2]; });
    DFT<R1, DIR>::run(b);
    static_for<0, R1>([&](auto K1) { v[k2 + R2 * decltype(K1)::value] = b[decltype(K1)::value]; });
  });
}

}  // namespace fft3d
