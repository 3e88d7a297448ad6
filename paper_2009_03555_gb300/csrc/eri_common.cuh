// eri_common.cuh -- device data layout, the FP64 Boys function and the
// per-primitive-quartet prologue of the HFX library (screened
// contracted-Gaussian ERIs and exchange build).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hfx {

// Checked builds (compiled with -DHFX_CHECKED): every global index of the
// split-kernel path is tested before use; an index outside its array is
// reported with printf and the access is skipped.  Release builds compile the
// tests away.
#ifdef HFX_CHECKED
}  // namespace hfx
#include <cstdio>
namespace hfx {
static __device__ __noinline__ bool hfx_oob(const char* what, long long i, long long n, int cls) {
  printf("HFX_CHECKED class %d %s: index %lld outside [0, %lld) (block %d thread %d)\n", cls, what, i, n,
         (int)blockIdx.x, (int)threadIdx.x);
  return false;
}
#define HFX_IN(i, n, what, cls) \
  (((long long)(i) >= 0 && (long long)(i) < (long long)(n)) || hfx_oob(what, (long long)(i), (long long)(n), cls))
#else
#define HFX_IN(i, n, what, cls) true
#endif


constexpr int kMaxL = 2;                 // s, p, d shells
constexpr int kMaxLtot = 4 * kMaxL;      // highest quartet angular momentum
constexpr double kTwoPi52 = 34.98683665524972497;  // 2 pi^{5/2}
constexpr double kSqrtPiHalf = 0.88622692545275801365;  // sqrt(pi)/2

enum Kernel { kCoulomb = 0, kErfc = 1, kErf = 2 };

// ---------------------------------------------------------------- records
// One primitive pair (a, b) of a shell pair (A, B): the Gaussian product
// exp(-a r_A^2) exp(-b r_B^2) = K_ab exp(-p r_P^2) (Gaussian product theorem).
// Within a shell pair the primitive pairs are sorted by descending `bound`.
struct __align__(16) PrimPair {
  double p;       // a + b
  double kp;      // c_a c_b K_ab / p   (normalised contraction coefficients, FP64)
  double oo2p;    // 1 / (2p)
  double P[3];    // (a A + b B) / p
  double PA[3];   // P - A
  float Phi[3], Plo[3];  // P as double-single (hi + lo) for the mixed path
  float PAf[3];   // P - A, FP32 copy for the mixed path
  float oo2pf;    // 1 / (2p), FP32
  float pf, plo;  // p as double-single
  float kpf;      // kp, FP32
  float bound;    // sqrt of the s-type self-repulsion of the primitive product
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
  int bra, k0, k1, sys;  // sys: index into the build's system table
};

// Geometry of one primitive quartet for the vertical recursion.
template <typename R>
struct VrrGeo {
  R PA[3], QC[3], WP[3], WQ[3];
  R oo2p, oo2q, oo2pq, rop, roq;
};

// Accumulation of one primitive contribution into a contracted integral.
// FP64: plain sum.  FP32: compensated (Kahan) summation; the running
// compensation is subtracted once after the primitive loop.  The primitive
// contributions of a contracted quartet alternate in sign and cancel, and the
// compensation keeps FP32 sums within a few ulp of an FP64 sum.
template <typename R>
__device__ __forceinline__ void kacc(R& s, R& c, R v) {
  s += v;
}
template <>
__device__ __forceinline__ void kacc<float>(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Butterfly reduce-scatter over a warp: every lane contributes 32 values and on
// return lane j holds the sum over the 32 lanes of v[j] (five exchange steps,
// 31 shuffles per lane; v is clobbered).
template <typename R>
__device__ __forceinline__ R reduce_scatter32(R (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int sft = 16; sft >= 1; sft >>= 1) {
    const bool up = (lane & sft) != 0;
#pragma unroll
    for (int i = 0; i < sft; ++i) {
      const R send = up ? v[i] : v[i + sft];
      const R keep = up ? v[i + sft] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, sft);
    }
  }
  return v[0];
}

// Warp sum of one 32-target chunk of the split recursion: every lane holds
// 32 values and lane j returns the sum over the lanes of v[j].  Default: a
// transposition through `buf` (32 rows of 36 R in shared memory, 16-byte
// aligned): each lane stores its row with vector stores and sums its column
// as a pairwise tree, trading the butterfly's 62 selects and 31 shuffles for
// 8 (FP32) or 16 (FP64) vector stores and 32 loads, bank-conflict free (row
// stride 36); measured 3-13 % faster per split class on GB300, with the same
// results to the last digits printed.  HFX_SHFL_REDUCE (build switch) selects
// the butterfly reduce-scatter above.
#ifndef HFX_SHFL_REDUCE
#define HFX_SMEM_REDUCE
#endif
constexpr int kChunkBufStride = 36;
constexpr int kChunkBufElems = 32 * kChunkBufStride;
template <typename R>
__device__ __forceinline__ R chunk_reduce32(R (&v)[32], R* buf) {
#ifdef HFX_SMEM_REDUCE
  const int lane = threadIdx.x & 31;
  R* row = buf + lane * kChunkBufStride;
  if constexpr (sizeof(R) == 4) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      reinterpret_cast<float4*>(row)[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  } else {
#pragma unroll
    for (int k = 0; k < 16; ++k) reinterpret_cast<double2*>(row)[k] = make_double2(v[2 * k], v[2 * k + 1]);
  }
  __syncwarp();
  // the column, summed as a pairwise tree (the butterfly's summation order
  // and error growth)
  R t[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) t[j] = buf[j * kChunkBufStride + lane];
  __syncwarp();
#pragma unroll
  for (int h = 16; h > 0; h >>= 1)
#pragma unroll
    for (int i = 0; i < h; ++i) t[i] += t[i + h];
  return t[0];
#else
  (void)buf;
  return reduce_scatter32<R>(v);
#endif
}

// ---------------------------------------------------------- Boys function
// F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt.  For every top order L = 0..8 the
// table holds, on the grid T_k = k / 16 (k = 0..960, T <= 60), the Taylor
// coefficients F_{L+j}(T_k) / j!, j = 0..6, and exp(-T_k) in the last column:
// tab[(L * kBoysNT + k) * 8 + j].  Built once per basis by a kernel
// (power-series evaluation of F_m).
constexpr int kBoysNT = 961;
constexpr int kBoysCols = 8;
constexpr int kBoysNL = 9;
constexpr double kBoysTmax = 60.0;
constexpr double kBoysStep = 1.0 / 16.0;

// Newton-Raphson refinement of a single-precision reciprocal seed:
// r <- r + r (1 - x r); each step doubles the correct bits (24 -> 48 -> 96).
template <int STEPS>
__device__ __forceinline__ double rcp_nr(double x) {
  double r = (double)(1.0f / (float)x);
#pragma unroll
  for (int i = 0; i < STEPS; ++i) r = fma(r, fma(-x, r, 1.0), r);
  return r;
}

// Newton-Raphson refinement of a single-precision 1/sqrt seed:
// y <- y + y (1 - x y^2) / 2.
template <int STEPS>
__device__ __forceinline__ double rsqrt_nr(double x) {
  double y = (double)rsqrtf((float)x);
#pragma unroll
  for (int i = 0; i < STEPS; ++i) y = fma(0.5 * y, fma(-x * y, y, 1.0), y);
  return y;
}

// F_0..F_L at T in FP64.  T < 60: sixth-order Taylor expansion of F_L about
// the nearest grid point (|T - T_k| <= 1/32, truncation < 1e-15 F_L), exp(-T)
// from exp(-T_k) times a Taylor series of exp(T_k - T), then the downward
// recursion F_m = (2 T F_{m+1} + exp(-T)) / (2m + 1) (stable downward).
// T >= 60: F_0 = sqrt(pi/T)/2 and F_{m+1} = (2m+1) F_m / (2T); exp(-60) is
// below the FP64 resolution of every F_m, m <= 8, there.
template <int L, int RSQ_STEPS>
__device__ __forceinline__ void boys_fp64(const double* __restrict__ tab, double T, double* F) {
  if (T < kBoysTmax) {
    const int it = __double2int_rn(T * 16.0);
#ifdef HFX_CHECKED
    if (!HFX_IN(it, kBoysNT, "boys_fp64 grid", L)) return;
#endif
    const double x = fma((double)it, kBoysStep, -T);  // T_k - T
    const double* row = tab + ((size_t)L * kBoysNT + it) * kBoysCols;
    const double2* r2 = reinterpret_cast<const double2*>(row);
    const double2 c01 = __ldg(r2), c23 = __ldg(r2 + 1), c45 = __ldg(r2 + 2), c6e = __ldg(r2 + 3);
    double f = fma(c6e.x, x, c45.y);
    f = fma(f, x, c45.x);
    f = fma(f, x, c23.y);
    f = fma(f, x, c23.x);
    f = fma(f, x, c01.y);
    f = fma(f, x, c01.x);
    F[L] = f;
    if (L > 0) {
      double e = fma(x, 1.0 / 5040.0, 1.0 / 720.0);
      e = fma(e, x, 1.0 / 120.0);
      e = fma(e, x, 1.0 / 24.0);
      e = fma(e, x, 1.0 / 6.0);
      e = fma(e, x, 0.5);
      e = fma(e, x, 1.0);
      e = fma(e, x, 1.0);
      const double ex = c6e.y * e;
      const double t2 = 2.0 * T;
#pragma unroll
      for (int m = L - 1; m >= 0; --m) F[m] = fma(t2, F[m + 1], ex) * (1.0 / (2 * m + 1));
    }
  } else {
    const double r = rsqrt_nr<RSQ_STEPS>(T);
    F[0] = kSqrtPiHalf * r;
    const double h = 0.5 * r * r;
#pragma unroll
    for (int m = 0; m < L; ++m) F[m + 1] = F[m] * ((2 * m + 1) * h);
  }
}

// Per-primitive-quartet prologue, FP64: argument T = rho |PQ|^2, prefactor
// 2 pi^{5/2} K_ab K_cd / (p q sqrt(p+q)) and the auxiliary integrals
//   Coulomb:     G_m = pref F_m(T)
//   erf(w r)/r:  G_m = pref f^{m+1/2} F_m(f T),   f = w^2 / (w^2 + rho)
//   erfc(w r)/r: Coulomb - erf   (Sec. 2, Eq. ERI-SR)
// The difference of the erfc kernel is taken in FP64 before any rounding.
// NR = Newton steps of the reciprocals (2: FP64 path, 1: mixed path, whose
// outputs are rounded to FP32 next).  Returns 1/(p+q) and PQ through args.
template <int L, int NR>
__device__ __forceinline__ void prologue(const double* __restrict__ boys, int kernel, double omega2,
                                         const PrimPair& pb, const PrimPair& pk, double* G, double& inv_s,
                                         double* PQ) {  // FP64 path
  const double s = pb.p + pk.p;
  inv_s = rcp_nr<NR>(s);
  const double rho = pb.p * pk.p * inv_s;
  PQ[0] = pb.P[0] - pk.P[0];
  PQ[1] = pb.P[1] - pk.P[1];
  PQ[2] = pb.P[2] - pk.P[2];
  const double T = rho * fma(PQ[0], PQ[0], fma(PQ[1], PQ[1], PQ[2] * PQ[2]));
  const double pref = (kTwoPi52 * pb.kp) * pk.kp * rsqrt_nr<NR>(s);
  double F[L + 1];
  if (kernel != kErf) {
    boys_fp64<L, NR>(boys, T, F);
    if (kernel == kCoulomb) {
#pragma unroll
      for (int m = 0; m <= L; ++m) G[m] = pref * F[m];
      return;
    }
  }
  const double f = omega2 * rcp_nr<NR>(omega2 + rho);
  double Fw[L + 1];
  boys_fp64<L, NR>(boys, f * T, Fw);
  double c = f * rsqrt_nr<NR>(f);  // f^{1/2}, then f^{m+1/2}
  if (kernel == kErfc) {
#pragma unroll
    for (int m = 0; m <= L; ++m) {
      G[m] = pref * fma(-c, Fw[m], F[m]);
      c *= f;
    }
  } else {
#pragma unroll
    for (int m = 0; m <= L; ++m) {
      G[m] = pref * (c * Fw[m]);
      c *= f;
    }
  }
}

}  // namespace hfx
