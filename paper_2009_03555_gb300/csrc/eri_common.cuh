// eri_common.cuh -- device data layout and the FP64 Boys function of the
// HFX library (screened contracted-Gaussian ERIs and exchange build).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hfx {

constexpr int kMaxL = 2;                 // s, p, d shells
constexpr int kMaxLtot = 4 * kMaxL;      // highest quartet angular momentum
constexpr double kTwoPi52 = 34.98683665524972497;  // 2 pi^{5/2}
constexpr double kSqrtPiHalf = 0.88622692545275801365;  // sqrt(pi)/2

// ---------------------------------------------------------------- records
// One primitive pair (a, b) of a shell pair (A, B): the Gaussian product
// exp(-a r_A^2) exp(-b r_B^2) = K_ab exp(-p r_P^2) (Sec. 2, shell pairs).
struct __align__(16) PrimPair {
  double p;      // a + b
  double kp;     // c_a c_b K_ab / p   (normalised contraction coefficients)
  double oo2p;   // 1 / (2p)
  double P[3];   // (a A + b B) / p
  double PA[3];  // P - A
  double bound;  // primitive self-repulsion estimate used for pair screening
};

// One significant shell pair, oriented so that l_A >= l_B.
struct __align__(16) PairRec {
  int A, B;        // shell indices
  int poff, pcnt;  // primitive pairs [poff, poff + pcnt)
  double AB[3];    // A - B (horizontal recursion)
  double Q;        // Schwarz bound sqrt(max |(ab|ab)|)   (Sec. 2, Eq. schwarz)
};

// A batch of quartets: bra pair `bra` against ket pairs [k0, k1) of the
// ket class's Q-sorted list.  The batch is the unit handed out by the device
// work queue (Sec. 3, Algorithms 1-3: the batched ERIs' start/end indexes).
struct __align__(16) Desc {
  int bra, k0, k1, pad;
};

// Geometry of one primitive quartet for the vertical recursion.
template <typename R>
struct VrrGeo {
  R PA[3], QC[3], WP[3], WQ[3];
  R oo2p, oo2q, oo2pq, rop, roq;
};

// ---------------------------------------------------------- Boys function
// F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt on a grid T_k = k / 16, k = 0..960
// (T <= 60), columns m = 0..14 and a last column exp(-T_k).  Built once per
// device by a kernel (power-series evaluation) and passed to every kernel.
constexpr int kBoysNT = 961;
constexpr int kBoysCols = 16;
constexpr double kBoysTmax = 60.0;
constexpr double kBoysStep = 1.0 / 16.0;

// Newton-Raphson refinement of a single-precision reciprocal seed:
// r <- r (2 - x r), quadratic convergence, two steps reach FP64 rounding.
__device__ __forceinline__ double rcp_nr(double x) {
  double r = (double)(1.0f / (float)x);
  r = r * fma(-x, r, 2.0);
  r = r * fma(-x, r, 2.0);
  return r;
}

// Newton-Raphson refinement of a single-precision 1/sqrt seed:
// y <- y (3 - x y^2) / 2.
__device__ __forceinline__ double rsqrt_nr(double x) {
  double y = (double)rsqrtf((float)x);
  y = y * fma(-0.5 * x, y * y, 1.5);
  y = y * fma(-0.5 * x, y * y, 1.5);
  return y;
}

// F_0..F_L at T, FP64.  T < 60: seventh-order Taylor expansion of F_L about the
// nearest grid point, exp(-T) from the tabulated exp(-T_k) times a Taylor
// series of exp(T_k - T), then downward recursion
//     F_m = (2 T F_{m+1} + exp(-T)) / (2m + 1).
// T >= 60: F_0 = sqrt(pi/T)/2 and upward F_{m+1} = (2m+1) F_m / (2T)
// (exp(-60) is below FP64 resolution of every F_m, m <= 8, there).
template <int L>
__device__ __forceinline__ void boys_fp64(const double* __restrict__ tab, double T, double* F) {
  if (T < kBoysTmax) {
    const int it = __double2int_rn(T * 16.0);
    const double x = it * kBoysStep - T;  // T_k - T, |x| <= 1/32
    const double* row = tab + it * kBoysCols;
    double f = __ldg(row + L + 6);
    f = fma(f, x * (1.0 / 6.0), __ldg(row + L + 5));
    f = fma(f, x * (1.0 / 5.0), __ldg(row + L + 4));
    f = fma(f, x * (1.0 / 4.0), __ldg(row + L + 3));
    f = fma(f, x * (1.0 / 3.0), __ldg(row + L + 2));
    f = fma(f, x * (1.0 / 2.0), __ldg(row + L + 1));
    f = fma(f, x, __ldg(row + L));
    F[L] = f;
    if (L > 0) {
      double e = fma(x, 1.0 / 5040.0, 1.0 / 720.0);
      e = fma(e, x, 1.0 / 120.0);
      e = fma(e, x, 1.0 / 24.0);
      e = fma(e, x, 1.0 / 6.0);
      e = fma(e, x, 0.5);
      e = fma(e, x, 1.0);
      e = fma(e, x, 1.0);
      const double ex = __ldg(row + 15) * e;
      const double t2 = 2.0 * T;
#pragma unroll
      for (int m = L - 1; m >= 0; --m) F[m] = fma(t2, F[m + 1], ex) * (1.0 / (2 * m + 1));
    }
  } else {
    const double r = rsqrt_nr(T);
    F[0] = kSqrtPiHalf * r;
    const double h = 0.5 * r * r;
#pragma unroll
    for (int m = 0; m < L; ++m) F[m + 1] = F[m] * ((2 * m + 1) * h);
  }
}

}  // namespace hfx
