// fft.cuh -- register-level small DFTs and the two-stage shared-memory pencil FFT used by the
// pair-potential chain (Eq. e:vij evaluated "in reciprocal space using Fourier transform",
// section II).  Everything is templated on the real type T (float for the mixed form, double
// for the plain form) and on compile-time lengths; there is no runtime radix dispatch.
//
// Direction D = -1 is the forward transform sum_n x_n e^{-2 pi i n k / R}, D = +1 the inverse
// (unnormalised).  Constants of the small DFTs come from a compile-time Taylor series written
// here (not from any library); the per-length stage twiddles are a host-made table.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace ace {

template <typename T>
struct alignas(2 * sizeof(T)) cpx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) {
  return {a.x + b.x, a.y + b.y};
}
template <typename T>
__device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) {
  return {a.x - b.x, a.y - b.y};
}
template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cpx<T> cscale(cpx<T> a, T s) {
  return {a.x * s, a.y * s};
}
#ifndef ACE_NO_F32X2
// FP32 complex adds, subtracts and real scalings as packed f32x2 instructions (sm_100 family):
// one instruction per complex operation, each lane rounded to nearest like the scalar forms.
__device__ __forceinline__ unsigned long long f2_pack(cpx<float> a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ cpx<float> f2_unpack(unsigned long long v) {
  cpx<float> r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ cpx<float> operator+(cpx<float> a, cpx<float> b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(r);
}
__device__ __forceinline__ cpx<float> operator-(cpx<float> a, cpx<float> b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
  return f2_unpack(r);
}
__device__ __forceinline__ cpx<float> cscale(cpx<float> a, float s) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(cpx<float>{s, s})));
  return f2_unpack(r);
}
#endif

// multiply by D*i (D = -1: -i, D = +1: +i)
template <int D, typename T>
__device__ __forceinline__ cpx<T> rot(cpx<T> a) {
  return D < 0 ? cpx<T>{a.y, -a.x} : cpx<T>{-a.y, a.x};
}

// ---------------------------------------------------------------------------------------
// Compile-time cos / sin of 2 pi e / R: reduce to [-pi, pi] and sum the Taylor series.
// ---------------------------------------------------------------------------------------
constexpr double kPi = 3.141592653589793238462643383279502884;

__host__ __device__ constexpr double ct_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 40; ++k) {
    term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double ct_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 40; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double ct_angle(int e, int R) {
  const int a = ((e % R) + R) % R;
  return (2 * a <= R) ? 2.0 * kPi * a / R : 2.0 * kPi * (a - R) / R;
}
// exact zeros/ones where the angle is a multiple of pi/2
__host__ __device__ constexpr double ct_cos2pi(int e, int R) {
  const int a = ((e % R) + R) % R;
  if (4 * a == R || 4 * a == 3 * R) return 0.0;
  if (a == 0) return 1.0;
  if (2 * a == R) return -1.0;
  return ct_cos(ct_angle(e, R));
}
__host__ __device__ constexpr double ct_sin2pi(int e, int R) {
  const int a = ((e % R) + R) % R;
  if (a == 0 || 2 * a == R) return 0.0;
  if (4 * a == R) return 1.0;
  if (4 * a == 3 * R) return -1.0;
  return ct_sin(ct_angle(e, R));
}

// w_R^{D e} = cos(2 pi e/R) + D i sin(2 pi e/R)
template <int R, int E, int D>
struct Tw {
  static constexpr double re = ct_cos2pi(E, R);
  static constexpr double im = D * ct_sin2pi(E, R);
};

template <int R, int E, int D, typename T>
__device__ __forceinline__ cpx<T> twc(cpx<T> a) {
  constexpr int e = E % R;
  if constexpr (e == 0) {
    return a;
  } else if constexpr (4 * e == R) {
    return rot<D>(a);
  } else if constexpr (2 * e == R) {
    return {-a.x, -a.y};
  } else if constexpr (4 * e == 3 * R) {
    return rot<-D>(a);
  } else {
    const T c = (T)Tw<R, e, D>::re, s = (T)Tw<R, e, D>::im;
    return {a.x * c - a.y * s, a.x * s + a.y * c};
  }
}

template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F &&f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// ---------------------------------------------------------------------------------------
// Small DFTs in registers: natural order in, natural order out.
// ---------------------------------------------------------------------------------------
template <int R, int D, typename T>
struct Dft;

template <int D, typename T>
struct Dft<1, D, T> {
  static __device__ __forceinline__ void run(cpx<T> *) {}
};

template <int D, typename T>
struct Dft<2, D, T> {
  static __device__ __forceinline__ void run(cpx<T> *x) {
    const cpx<T> a = x[0], b = x[1];
    x[0] = a + b;
    x[1] = a - b;
  }
};

template <int D, typename T>
struct Dft<3, D, T> {
  static __device__ __forceinline__ void run(cpx<T> *x) {
    constexpr double s3 = 0.8660254037844386467637231707529361834714;  // sin(2 pi / 3)
    const cpx<T> t = x[1] + x[2];
    const cpx<T> d = x[1] - x[2];
    const cpx<T> m = {x[0].x - (T)0.5 * t.x, x[0].y - (T)0.5 * t.y};
    const cpx<T> r = rot<D>(cscale(d, (T)s3));
    x[0] = x[0] + t;
    x[1] = m + r;
    x[2] = m - r;
  }
};

template <int D, typename T>
struct Dft<4, D, T> {
  static __device__ __forceinline__ void run(cpx<T> *x) {
    const cpx<T> a = x[0] + x[2], b = x[0] - x[2];
    const cpx<T> c = x[1] + x[3], d = rot<D>(x[1] - x[3]);
    x[0] = a + c;
    x[2] = a - c;
    x[1] = b + d;
    x[3] = b - d;
  }
};

template <int D, typename T>
struct Dft<5, D, T> {
  static __device__ __forceinline__ void run(cpx<T> *x) {
    constexpr double c1 = ct_cos2pi(1, 5), c2 = ct_cos2pi(2, 5);
    constexpr double s1 = ct_sin2pi(1, 5), s2 = ct_sin2pi(2, 5);
    const cpx<T> a1 = x[1] + x[4], b1 = x[1] - x[4];
    const cpx<T> a2 = x[2] + x[3], b2 = x[2] - x[3];
    const cpx<T> x0 = x[0];
    const cpx<T> p1 = {x0.x + (T)c1 * a1.x + (T)c2 * a2.x, x0.y + (T)c1 * a1.y + (T)c2 * a2.y};
    const cpx<T> p2 = {x0.x + (T)c2 * a1.x + (T)c1 * a2.x, x0.y + (T)c2 * a1.y + (T)c1 * a2.y};
    const cpx<T> q1 = rot<D>(cpx<T>{(T)s1 * b1.x + (T)s2 * b2.x, (T)s1 * b1.y + (T)s2 * b2.y});
    const cpx<T> q2 = rot<D>(cpx<T>{(T)s2 * b1.x - (T)s1 * b2.x, (T)s2 * b1.y - (T)s1 * b2.y});
    x[0] = x0 + a1 + a2;
    x[1] = p1 + q1;
    x[4] = p1 - q1;
    x[2] = p2 + q2;
    x[3] = p2 - q2;
  }
};

// Composite R = P * Q by one Cooley-Tukey step in registers:
//   n = Q n1 + n2, k = k1 + P k2:  X[k1 + P k2] = sum_n2 w_Q^{n2 k2} w_R^{n2 k1} sum_n1 w_P^{n1 k1} x[Q n1 + n2]
template <int P, int Q, int D, typename T>
struct DftCT {
  static __device__ __forceinline__ void run(cpx<T> *x) {
    constexpr int R = P * Q;
    cpx<T> y[R];
    static_for<Q>([&](auto n2c) {
      constexpr int n2 = decltype(n2c)::value;
      cpx<T> t[P];
      static_for<P>([&](auto n1c) { t[decltype(n1c)::value] = x[Q * decltype(n1c)::value + n2]; });
      Dft<P, D, T>::run(t);
      static_for<P>([&](auto k1c) {
        constexpr int k1 = decltype(k1c)::value;
        y[n2 * P + k1] = twc<R, n2 * k1, D>(t[k1]);
      });
    });
    static_for<P>([&](auto k1c) {
      constexpr int k1 = decltype(k1c)::value;
      cpx<T> t[Q];
      static_for<Q>([&](auto n2c) { t[decltype(n2c)::value] = y[decltype(n2c)::value * P + k1]; });
      Dft<Q, D, T>::run(t);
      static_for<Q>([&](auto k2c) { x[k1 + P * decltype(k2c)::value] = t[decltype(k2c)::value]; });
    });
  }
};

// Inverse of a modulo m (a, m coprime), by search: compile time only.
constexpr int ct_inv_mod(int a, int m) {
  for (int x = 1; x < m; ++x)
    if ((a * x) % m == 1) return x;
  return m == 1 ? 0 : -1;
}

// Composite R = P * Q with gcd(P, Q) = 1 by the prime-factor (Good-Thomas) mapping: input
// n = (Q n1 + P n2) mod R, output k = (Q (Q^-1 mod P) k1 + P (P^-1 mod Q) k2) mod R.  The cross
// terms of n k are multiples of R, so X is a plain P x Q two-dimensional DFT with no twiddles.
template <int P, int Q, int D, typename T>
struct DftPFA {
  static constexpr int R = P * Q, A = ct_inv_mod(Q % P, P), B = ct_inv_mod(P % Q, Q);
  static_assert(A >= 0 && B >= 0, "factors must be coprime");
  static __device__ __forceinline__ void run(cpx<T> *x) {
    cpx<T> y[R];
    static_for<Q>([&](auto n2c) {
      constexpr int n2 = decltype(n2c)::value;
      cpx<T> t[P];
      static_for<P>([&](auto n1c) { t[decltype(n1c)::value] = x[(Q * decltype(n1c)::value + P * n2) % R]; });
      Dft<P, D, T>::run(t);
      static_for<P>([&](auto k1c) { y[n2 * P + decltype(k1c)::value] = t[decltype(k1c)::value]; });
    });
    static_for<P>([&](auto k1c) {
      constexpr int k1 = decltype(k1c)::value;
      cpx<T> t[Q];
      static_for<Q>([&](auto n2c) { t[decltype(n2c)::value] = y[decltype(n2c)::value * P + k1]; });
      Dft<Q, D, T>::run(t);
      static_for<Q>([&](auto k2c) { x[(Q * A * k1 + P * B * decltype(k2c)::value) % R] = t[decltype(k2c)::value]; });
    });
  }
};

template <int D, typename T> struct Dft<6, D, T> : DftPFA<2, 3, D, T> {};
template <int D, typename T> struct Dft<8, D, T> : DftCT<2, 4, D, T> {};
template <int D, typename T> struct Dft<9, D, T> : DftCT<3, 3, D, T> {};
template <int D, typename T> struct Dft<10, D, T> : DftPFA<2, 5, D, T> {};
template <int D, typename T> struct Dft<12, D, T> : DftPFA<3, 4, D, T> {};
template <int D, typename T> struct Dft<15, D, T> : DftPFA<3, 5, D, T> {};
template <int D, typename T> struct Dft<16, D, T> : DftCT<4, 4, D, T> {};
template <int D, typename T> struct Dft<18, D, T> : DftPFA<2, 9, D, T> {};
template <int D, typename T> struct Dft<20, D, T> : DftPFA<4, 5, D, T> {};
template <int D, typename T> struct Dft<25, D, T> : DftCT<5, 5, D, T> {};
template <int D, typename T> struct Dft<27, D, T> : DftCT<3, 9, D, T> {};

// ---------------------------------------------------------------------------------------
// Factorisation L = R1 * R2 used by the two-stage pencil FFT (both factors in registers).
// ---------------------------------------------------------------------------------------
template <int L>
struct Factor;
#define ACE_FACTOR(L_, A_, B_)                \
  template <>                                 \
  struct Factor<L_> {                         \
    static constexpr int R1 = A_, R2 = B_;    \
    static_assert(A_ * B_ == L_, "factor");   \
  };
ACE_FACTOR(2, 2, 1)
ACE_FACTOR(3, 3, 1)
ACE_FACTOR(4, 4, 1)
ACE_FACTOR(5, 5, 1)
ACE_FACTOR(6, 3, 2)
ACE_FACTOR(8, 4, 2)
ACE_FACTOR(9, 3, 3)
ACE_FACTOR(10, 5, 2)
ACE_FACTOR(12, 4, 3)
ACE_FACTOR(15, 5, 3)
ACE_FACTOR(16, 4, 4)
ACE_FACTOR(18, 6, 3)
ACE_FACTOR(20, 5, 4)
ACE_FACTOR(24, 6, 4)
ACE_FACTOR(25, 5, 5)
ACE_FACTOR(27, 9, 3)
ACE_FACTOR(30, 6, 5)
ACE_FACTOR(32, 8, 4)
ACE_FACTOR(36, 6, 6)
ACE_FACTOR(40, 8, 5)
ACE_FACTOR(45, 9, 5)
ACE_FACTOR(48, 8, 6)
ACE_FACTOR(50, 10, 5)
ACE_FACTOR(54, 9, 6)
ACE_FACTOR(60, 12, 5)
ACE_FACTOR(64, 8, 8)
ACE_FACTOR(72, 9, 8)
ACE_FACTOR(75, 15, 5)
ACE_FACTOR(80, 16, 5)
ACE_FACTOR(81, 9, 9)
ACE_FACTOR(90, 10, 9)
ACE_FACTOR(96, 12, 8)
ACE_FACTOR(100, 10, 10)
ACE_FACTOR(108, 12, 9)
ACE_FACTOR(120, 12, 10)
ACE_FACTOR(125, 25, 5)
ACE_FACTOR(128, 16, 8)
ACE_FACTOR(135, 15, 9)
ACE_FACTOR(144, 12, 12)
ACE_FACTOR(150, 15, 10)
ACE_FACTOR(160, 16, 10)
ACE_FACTOR(162, 18, 9)
ACE_FACTOR(180, 15, 12)
ACE_FACTOR(192, 16, 12)
ACE_FACTOR(200, 20, 10)
ACE_FACTOR(216, 18, 12)
ACE_FACTOR(225, 15, 15)
ACE_FACTOR(240, 16, 15)
ACE_FACTOR(243, 27, 9)
ACE_FACTOR(250, 25, 10)
ACE_FACTOR(256, 16, 16)
#undef ACE_FACTOR

}  // namespace ace
