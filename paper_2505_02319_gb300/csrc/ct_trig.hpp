// Compile-time cosine and sine of 2 pi k / n, for FFT twiddle factors that
// become immediate operands of the kernels' instructions.
//
// The angle is reduced exactly, in integer arithmetic, to the nearest quarter
// turn j and a remainder r = k/n - j/4 with |r| <= 1/8 of a turn; cos and sin
// of 2 pi r (|2 pi r| <= pi/4) come from their Taylor series, 14 terms each
// (truncation below 1e-25), and the quarter turn is restored by the identities
// cos(t + j pi/2), sin(t + j pi/2).  Plain C++17, no device code: the values
// are folded by the host compiler and checked against a library on the CPU.
#pragma once

namespace ikr {

struct CtCosSin {
  double c, s;
};

constexpr double kCtPi = 3.14159265358979323846264338327950288;

constexpr double ct_sin_series(double x) {
  double term = x, sum = x;
  for (int i = 1; i <= 14; ++i) {
    term *= -(x * x) / (double)((2 * i) * (2 * i + 1));
    sum += term;
  }
  return sum;
}

constexpr double ct_cos_series(double x) {
  double term = 1.0, sum = 1.0;
  for (int i = 1; i <= 14; ++i) {
    term *= -(x * x) / (double)((2 * i - 1) * (2 * i));
    sum += term;
  }
  return sum;
}

// (cos, sin) of 2 pi k / n, n > 0, any integer k
constexpr CtCosSin ct_cossin(long long k, long long n) {
  long long m = k % n;
  if (m < 0) m += n;
  const long long j = (8 * m + n) / (2 * n);                 // nearest quarter turn, 0..4
  const double r = (double)(4 * m - j * n) / (double)(4 * n);  // remaining fraction of a turn
  const double t = 2.0 * kCtPi * r;
  const double c = ct_cos_series(t), s = ct_sin_series(t);
  switch (j & 3) {
    case 0: return CtCosSin{c, s};
    case 1: return CtCosSin{-s, c};
    case 2: return CtCosSin{-c, -s};
    default: return CtCosSin{s, -c};
  }
}

template <int N, int K> struct CtTwiddle {
  static constexpr CtCosSin v = ct_cossin(K, N);
  static constexpr double c = v.c, s = v.s;
};

}  // namespace ikr
