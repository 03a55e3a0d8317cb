// Register-resident DFTs of compile-time size for the two-level FFT engine.
//
// dft_reg<N, INV>(v) transforms v[0..N-1] in registers, natural order in and out:
//   v[k] <- sum_n v[n] exp(-+2 pi i n k / N)   (INV selects the + sign, no 1/N scale)
// N = 2, 3, 4, 5 are written out; larger N = P Q split as
//   n = Q a + b, k = k1 + P k2:  Y_b[k1] = DFT_P over a of v[Q a + b],
//   Y_b[k1] *= w_N^(b k1),  X[k1 + P k2] = DFT_Q over b of Y_b[k1].
// Every index and twiddle is a compile-time constant after unrolling; twiddles are
// evaluated at compile time in double precision by constexpr series below.
#pragma once

#include <type_traits>

#include "fft_engine.cuh"

namespace vp {

// ---- compile-time cos / sin of 2 pi k / N -----------------------------------------
// Range reduction is exact (rational k / N folded into [0, 1/8] by the symmetries of
// sine and cosine); the remaining angle |x| <= pi/4 is summed by Taylor series to
// double precision.
namespace ct {

constexpr double kPi = 3.141592653589793238462643383279502884;

__host__ __device__ constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int i = 1; i < 14; ++i) {
    term *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
    sum += term;
  }
  return sum;
}

__host__ __device__ constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int i = 1; i < 14; ++i) {
    term *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
    sum += term;
  }
  return sum;
}

// cos(2 pi k / N) and sin(2 pi k / N) for integers k, N > 0.
__host__ __device__ constexpr void cos_sin(long long k, long long N, double& c, double& s) {
  k %= N;
  if (k < 0) k += N;
  // angle fraction t = k / N of a full turn; work in units of 1 / (8 N)
  const long long e = 8 * k;  // t = e / (8 N)
  const long long oct = e / N;  // octant 0..7
  const long long r = e - oct * N;  // remainder in [0, N): angle = (oct + r / N) * pi / 4
  // phase inside the octant, in [0, pi/4)
  const double x = (double)r / (double)N * (kPi / 4.0);
  const double sx = taylor_sin(x), cx = taylor_cos(x);
  const double y = kPi / 4.0 - x;  // complementary angle for odd octants
  const double sy = taylor_sin(y), cy = taylor_cos(y);
  double cc = 0.0, ss = 0.0;
  switch (oct) {
    case 0: cc = cx; ss = sx; break;    // theta = x
    case 1: cc = sy; ss = cy; break;    // theta = pi/2 - y
    case 2: cc = -sx; ss = cx; break;   // theta = pi/2 + x
    case 3: cc = -cy; ss = sy; break;   // theta = pi - y
    case 4: cc = -cx; ss = -sx; break;  // theta = pi + x
    case 5: cc = -sy; ss = -cy; break;  // theta = 3pi/2 - y
    case 6: cc = sx; ss = -cx; break;   // theta = 3pi/2 + x
    default: cc = cy; ss = -sy; break;  // theta = 2pi - y
  }
  c = cc;
  s = ss;
}

// cos and sin of 2 pi k / N for k = 0..N-1, rounded to float, built at compile time.
template <int N>
struct TwTab {
  float c[N];
  float s[N];
};
template <int N>
__host__ __device__ constexpr TwTab<N> make_twtab() {
  TwTab<N> t{};
  for (int k = 0; k < N; ++k) {
    double cc = 0.0, ss = 0.0;
    cos_sin(k, N, cc, ss);
    t.c[k] = (float)cc;
    t.s[k] = (float)ss;
  }
  return t;
}

// Smallest useful first factor of N for the register split.
__host__ __device__ constexpr int first_factor(int N) {
  if (N % 4 == 0 && N != 8 && N != 16 && N != 32) return 4;
  if (N == 8) return 2;
  if (N == 16) return 4;
  if (N == 32) return 4;
  if (N % 2 == 0) return 2;
  if (N % 3 == 0) return 3;
  if (N % 5 == 0) return 5;
  return N;
}

}  // namespace ct

// v * w_N^(k) with w_N = exp(-2 pi i / N) (or its conjugate for INV); k constant.
template <int N, bool INV>
__device__ __forceinline__ float2 twiddle_const(float2 v, int k) {
  k %= N;
  if (k == 0) return v;
  if (4 * k == N) return mul_mi<INV>(v);                       // -i
  if (2 * k == N) return make_float2(-v.x, -v.y);              // -1
  if (4 * k == 3 * N) return mul_mi<!INV>(v);                  // +i
  constexpr ct::TwTab<N> tab = ct::make_twtab<N>();
  return mul_const<INV>(v, tab.c[k], -tab.s[k]);  // exp(-i theta) = (cos, -sin)
}

// acc + v * w_N^(k), k constant: the powers +-1 and +-i fold into the add.
template <int N, bool INV>
__device__ __forceinline__ float2 add_twiddled(float2 acc, float2 v, int k) {
  k %= N;
  if (k == 0) return cadd(acc, v);
  if (2 * k == N) return csub(acc, v);
  if (4 * k == N) return add_mi<INV>(acc, v);
  if (4 * k == 3 * N) return sub_mi<INV>(acc, v);
  return cadd(acc, twiddle_const<N, INV>(v, k));
}

template <int N, bool INV>
__device__ __forceinline__ void dft_reg(float2* v) {
  if constexpr (N == 1) {
    return;
  } else if constexpr (N == 2) {
    dft2<INV>(v[0], v[1]);
  } else if constexpr (N == 3) {
    dft3<INV>(v);
  } else if constexpr (N == 4) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  } else if constexpr (N == 5) {
    dft5<INV>(v);
  } else {
    constexpr int P = ct::first_factor(N);
    constexpr int Q = N / P;
    static_assert(P * Q == N && P > 1 && Q > 1, "unsupported register DFT size");
    float2 y[N];  // y[b * P + k1]
#pragma unroll
    for (int b = 0; b < Q; ++b) {
      float2 u[P];
#pragma unroll
      for (int a = 0; a < P; ++a) u[a] = v[Q * a + b];
      dft_reg<P, INV>(u);
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) y[b * P + k1] = twiddle_const<N, INV>(u[k1], b * k1);
    }
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      float2 z[Q];
#pragma unroll
      for (int b = 0; b < Q; ++b) z[b] = y[b * P + k1];
      dft_reg<Q, INV>(z);
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) v[k1 + P * k2] = z[k2];
    }
  }
}

// f(std::integral_constant<int, i>) for i = I .. E-1, each i a compile-time constant.
template <int I, int E, typename F>
__device__ __forceinline__ void static_for(F& f) {
  if constexpr (I < E) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, E>(f);
  }
}

// dft_reg<N, INV> for an input whose entries v[n], n >= NZ, are zero: those entries are
// neither read nor added.  A zero-padded line (NZ = N / 2) saves the first butterfly
// layer and half the loads.  Outputs that the caller never reads are removed by the
// compiler as dead code, so a cropped output needs no variant of its own.
template <int N, bool INV, int NZ>
__device__ __forceinline__ void dft_reg_nz(float2* v) {
  if constexpr (NZ >= N) {
    dft_reg<N, INV>(v);
  } else if constexpr (NZ <= 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = make_float2(0.f, 0.f);
  } else if constexpr (NZ == 1) {
#pragma unroll
    for (int k = 1; k < N; ++k) v[k] = v[0];
  } else if constexpr (N <= 5) {
    // X[k] = sum_{n < NZ} v[n] w_N^(n k), written out
    float2 x[NZ];
#pragma unroll
    for (int n = 0; n < NZ; ++n) x[n] = v[n];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      float2 acc = x[0];
#pragma unroll
      for (int n = 1; n < NZ; ++n) acc = add_twiddled<N, INV>(acc, x[n], n * k);
      v[k] = acc;
    }
  } else {
    // the split of dft_reg; row b of the first level holds v[Q a + b], nonzero for
    // Q a + b < NZ, and rows b >= NZ are zero altogether
    constexpr int P = ct::first_factor(N);
    constexpr int Q = N / P;
    constexpr int NZ2 = NZ < Q ? NZ : Q;
    float2 y[NZ2 * P];
    auto row = [&](auto bc) {
      constexpr int b = decltype(bc)::value;
      constexpr int na = (NZ - b + Q - 1) / Q < P ? (NZ - b + Q - 1) / Q : P;
      float2 u[P];
#pragma unroll
      for (int a = 0; a < na; ++a) u[a] = v[Q * a + b];
      dft_reg_nz<P, INV, na>(u);
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) y[b * P + k1] = twiddle_const<N, INV>(u[k1], b * k1);
    };
    static_for<0, NZ2>(row);
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      float2 z[Q];
#pragma unroll
      for (int b = 0; b < NZ2; ++b) z[b] = y[b * P + k1];
      dft_reg_nz<Q, INV, NZ2>(z);
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) v[k1 + P * k2] = z[k2];
    }
  }
}

}  // namespace vp
