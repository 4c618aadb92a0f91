// Device helpers of the manufactured solutions (Sec. 3.3): the 1D factors
// G_a(s) = s^2 (1-s)^2 sin(a pi s) of the seeded stream functions and their
// derivatives, exact by the Leibniz rule.  Shared by the 3D and 2D
// right-hand-side kernels and the 2D error kernel.
#pragma once

#include <cmath>

namespace stk {

// d^n/ds^n of s^2 (1-s)^2
__device__ __forceinline__ double poly_d(double s, int n) {
  switch (n) {
    case 0: return s * s * (1.0 - s) * (1.0 - s);
    case 1: return 2.0 * s - 6.0 * s * s + 4.0 * s * s * s;
    case 2: return 2.0 - 12.0 * s + 12.0 * s * s;
    case 3: return -12.0 + 24.0 * s;
    case 4: return 24.0;
  }
  return 0.0;
}

// G_a^(n)(s) for n = 0..3 by the Leibniz rule, from one sincos
__device__ __forceinline__ void G_all(int a, double s, double* out) {
  const double w = a * M_PI;
  double sv, cv;
  sincos(w * s, &sv, &cv);
  const double trig[4] = {sv, cv, -sv, -cv};  // sin(ws + j pi/2)
  const int binom[4][4] = {{1, 0, 0, 0}, {1, 1, 0, 0}, {1, 2, 1, 0}, {1, 3, 3, 1}};
  const double wpow[4] = {1.0, w, w * w, w * w * w};
  for (int n = 0; n < 4; ++n) {
    // term j: C(n, j) P^(j) w^(n-j) sin(ws + (n-j) pi/2)
    double acc = 0.0;
    for (int j = 0; j <= n; ++j) acc += binom[n][j] * poly_d(s, j) * wpow[n - j] * trig[(n - j) & 3];
    out[n] = acc;
  }
}

}  // namespace stk
