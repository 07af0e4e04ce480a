// The Gaussian sketch's table of normal quantiles, host code only.
//
// W[i, b] = q_j / (2^8 sqrt(w)) for cell j = h >> 50 of the hash h of entry (i, b), with
//   q_j = round(2^8 Phi^{-1}((j + 1/2) 2^-14)),  |q_j| <= 1026,
// Phi the standard normal CDF: N(0, 1) quantiles of 2^14 equiprobable cells on a grid of 2^-8.
#pragma once

#include <cmath>
#include <cstdint>

namespace lpk {

constexpr int kGaussBits = 14;

// Phi^{-1} by bisection on Phi(z) = erfc(-z / sqrt 2) / 2 over [-10, 0] to the resolution of
// FP64 (the cells below 1/2; the upper half by symmetry, q_{N-1-j} = -q_j).  No table value
// lies within 1e-5 of a rounding tie, far above the error of this evaluation, so any accurate
// evaluation of Phi^{-1} gives the same integers.
inline void gauss_grid(int16_t* q) {
  constexpr int N = 1 << kGaussBits;
  for (int j = 0; j < N / 2; ++j) {
    const double p = (j + 0.5) / N;
    double lo = -10.0, hi = 0.0;
    for (int it = 0; it < 80; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (0.5 * std::erfc(-mid * 0.70710678118654752440) < p)
        lo = mid;
      else
        hi = mid;
    }
    const long v = std::lrint(256.0 * 0.5 * (lo + hi));
    q[j] = (int16_t)v;
    q[N - 1 - j] = (int16_t)(-v);
  }
}

}  // namespace lpk
