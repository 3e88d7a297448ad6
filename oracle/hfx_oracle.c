/*
 * hfx_oracle.c -- plain FP64 CPU oracle for Hartree-Fock exchange construction.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * What it computes (paper Sec. 2):
 *   - contracted Cartesian Gaussian shells, axial normalisation;
 *   - electron repulsion integrals (ERIs) with the full Coulomb kernel 1/r
 *     (Sec. 2, full-range ERI definition) and the screened kernels
 *     erf(w r)/r and erfc(w r)/r (Sec. 2, Eq. ERI-SR, w = 0.11 bohr^-1);
 *   - Schwarz bounds Q_IJ = sqrt(max |(ij|ij)|)  (Sec. 2, Eq. schwarz);
 *   - density screening  P_scr * Q_IJ * Q_KL <= eps  (Sec. 2, Eq. dmscreening);
 *   - the exchange matrix K_ij = sum_kl (ik|jl) P_kl (Eq. H-HFX without -1/2),
 *     either from canonical shell quartets and the 8-fold permutation symmetry
 *     (Sec. 2) or by brute force over all ordered shell quartets.
 *
 * The ERI method is the McMurchie-Davidson Hermite scheme (Hermite expansion
 * coefficients E_t^{ij} and Hermite Coulomb integrals R_{tuv}); the Boys
 * function is a long-double power series (argument < 35) or erf plus upward
 * recursion (argument >= 35), then downward recursion.  This is a different
 * route from the GPU path on purpose.
 *
 * Attenuated kernels: the erf(w r)/r integral equals the Coulomb one with the
 * Hermite exponent alpha replaced by alpha' = alpha w^2/(alpha + w^2) and an
 * overall factor sqrt(alpha'/alpha); erfc = Coulomb - erf, applied at the base
 * R^n_{000} values (the Hermite recursion is linear in them).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define LMAX 2             /* s, p, d */
#define LTOT (4 * LMAX)    /* highest total angular momentum of a quartet */
#define MAXC 6             /* Cartesian components of a d shell */

static const long double PI_L = 3.141592653589793238462643383279502884L;

static int ncart(int l) { return (l + 1) * (l + 2) / 2; }

/* Cartesian exponents of component k of a shell of angular momentum l,
 * lexicographic order: x, y, z; xx, xy, xz, yy, yz, zz. */
static void cart(int l, int k, int e[3]) {
  int idx = 0;
  for (int lx = l; lx >= 0; --lx)
    for (int ly = l - lx; ly >= 0; --ly) {
      if (idx == k) { e[0] = lx; e[1] = ly; e[2] = l - lx - ly; return; }
      ++idx;
    }
}

static double dfact(int n) { /* n!! for n >= -1 */
  double r = 1.0;
  for (int k = n; k > 1; k -= 2) r *= k;
  return r;
}

/* ---------------------------------------------------------------- Boys */
/* F_m(x) = int_0^1 t^{2m} exp(-x t^2) dt, m = 0..mmax.
 * x < 35: F_mmax from the series e^{-x} sum_k (2x)^k / ((2m+1)(2m+3)...(2m+2k+1)),
 *         all terms positive, evaluated in long double; then downward
 *         F_m = (2x F_{m+1} + e^{-x}) / (2m+1).
 * x >= 35: F_0 = sqrt(pi/x) erf(sqrt x) / 2, upward F_{m+1} = ((2m+1) F_m - e^{-x}) / (2x). */
void oracle_boys(int mmax, double xd, double *F) {
  long double x = xd;
  if (x < 35.0L) {
    long double term = 1.0L / (2 * mmax + 1), sum = term;
    for (int k = 1; k < 2000; ++k) {
      term *= 2.0L * x / (2 * mmax + 2 * k + 1);
      sum += term;
      if (term < 1e-22L * sum) break;
    }
    long double ex = expl(-x);
    long double f = ex * sum;
    F[mmax] = (double)f;
    for (int m = mmax - 1; m >= 0; --m) {
      f = (2.0L * x * f + ex) / (2 * m + 1);
      F[m] = (double)f;
    }
  } else {
    long double ex = expl(-x);
    long double f = 0.5L * sqrtl(PI_L / x) * erfl(sqrtl(x));
    F[0] = (double)f;
    for (int m = 0; m < mmax; ++m) {
      f = ((2 * m + 1) * f - ex) / (2.0L * x);
      F[m + 1] = (double)f;
    }
  }
}

/* ------------------------------------------------------- normalisation */
/* Axial primitive normalisation N(a) = (2a/pi)^{3/4} (4a)^{l/2} / sqrt((2l-1)!!),
 * then the contracted axial component x^l is scaled to unit self-overlap. */
void oracle_normalize(int n_shells, const int *l, const int *prim_off, const double *alpha,
                      const double *coef_raw, double *coef_out) {
  for (int s = 0; s < n_shells; ++s) {
    int L = l[s], p0 = prim_off[s], p1 = prim_off[s + 1];
    double df = dfact(2 * L - 1);
    for (int k = p0; k < p1; ++k) {
      double a = alpha[k];
      coef_out[k] = coef_raw[k] * pow(2.0 * a / M_PI, 0.75) * pow(4.0 * a, 0.5 * L) / sqrt(df);
    }
    double S = 0.0;
    for (int k = p0; k < p1; ++k)
      for (int m = p0; m < p1; ++m) {
        double g = alpha[k] + alpha[m];
        S += coef_out[k] * coef_out[m] * df / pow(2.0 * g, L) * pow(M_PI / g, 1.5);
      }
    double sc = 1.0 / sqrt(S);
    for (int k = p0; k < p1; ++k) coef_out[k] *= sc;
  }
}

/* ------------------------------------------ Hermite expansion coefficients */
/* E[i][j][t] for one Cartesian axis, i <= la, j <= lb, t <= i + j, for the
 * Gaussian product of exponents a (centre A) and b (centre B):
 *   E^{00}_0 = exp(-ab/(a+b) X_AB^2)
 *   E^{i+1,j}_t = E^{ij}_{t-1}/(2p) + X_PA E^{ij}_t + (t+1) E^{ij}_{t+1}
 *   E^{i,j+1}_t = E^{ij}_{t-1}/(2p) + X_PB E^{ij}_t + (t+1) E^{ij}_{t+1}   */
typedef double ecoef_t[LMAX + 1][LMAX + 1][2 * LMAX + 2];

static void hermite_E(int la, int lb, double a, double b, double Ax, double Bx, ecoef_t E) {
  double p = a + b, Px = (a * Ax + b * Bx) / p, XPA = Px - Ax, XPB = Px - Bx, XAB = Ax - Bx;
  memset(E, 0, sizeof(ecoef_t));
  E[0][0][0] = exp(-a * b / p * XAB * XAB);
  for (int i = 0; i <= la; ++i)
    for (int j = 0; j <= lb; ++j) {
      if (i == 0 && j == 0) continue;
      for (int t = 0; t <= i + j; ++t) {
        double v = 0.0;
        if (i > 0) {
          if (t > 0) v += E[i - 1][j][t - 1] / (2.0 * p);
          if (t <= i - 1 + j) v += XPA * E[i - 1][j][t];
          if (t + 1 <= i - 1 + j) v += (t + 1) * E[i - 1][j][t + 1];
        } else {
          if (t > 0) v += E[i][j - 1][t - 1] / (2.0 * p);
          if (t <= i + j - 1) v += XPB * E[i][j - 1][t];
          if (t + 1 <= i + j - 1) v += (t + 1) * E[i][j - 1][t + 1];
        }
        E[i][j][t] = v;
      }
    }
}

/* ----------------------------------------------- Hermite Coulomb integrals */
/* R[t][u][v] = R^0_{tuv}, t+u+v <= Ltot, from the base values R^n_{000}:
 *   R^n_{t+1,u,v} = t R^{n+1}_{t-1,u,v} + X_PQ R^{n+1}_{t,u,v}  (same for u, v). */
typedef double rtab_t[LTOT + 1][LTOT + 1][LTOT + 1];

static void hermite_R(int Ltot, const double *base, double X, double Y, double Z, rtab_t R) {
  static __thread double Rn[LTOT + 1][LTOT + 1][LTOT + 1][LTOT + 1];
  for (int n = 0; n <= Ltot; ++n) Rn[n][0][0][0] = base[n];
  for (int N = 1; N <= Ltot; ++N)
    for (int n = 0; n <= Ltot - N; ++n)
      for (int t = N; t >= 0; --t)
        for (int u = N - t; u >= 0; --u) {
          int v = N - t - u;
          double r;
          if (t > 0)
            r = (t > 1 ? (t - 1) * Rn[n + 1][t - 2][u][v] : 0.0) + X * Rn[n + 1][t - 1][u][v];
          else if (u > 0)
            r = (u > 1 ? (u - 1) * Rn[n + 1][t][u - 2][v] : 0.0) + Y * Rn[n + 1][t][u - 1][v];
          else
            r = (v > 1 ? (v - 1) * Rn[n + 1][t][u][v - 2] : 0.0) + Z * Rn[n + 1][t][u][v - 1];
          Rn[n][t][u][v] = r;
        }
  for (int t = 0; t <= Ltot; ++t)
    for (int u = 0; u <= Ltot - t; ++u)
      for (int v = 0; v <= Ltot - t - u; ++v) R[t][u][v] = Rn[0][t][u][v];
}

/* ----------------------------------------------------------- the basis */
typedef struct {
  int n_shells;
  const double *xyz;    /* n_shells x 3 shell centres */
  const int *l;         /* n_shells */
  const int *prim_off;  /* n_shells + 1 */
  const double *alpha;  /* exponents */
  const double *coef;   /* normalised contraction coefficients */
  const long long *func_off; /* n_shells + 1 */
  int nbf;
} basis_t;

enum { KERNEL_COULOMB = 0, KERNEL_ERFC = 1, KERNEL_ERF = 2 };

/* Base values R^n_{000}, n = 0..Ltot, for Hermite exponent alpha, squared
 * distance R2, for the selected kernel. */
static void base_values(int Ltot, int kernel, double omega, double alpha, double R2, double *base) {
  double F[LTOT + 1], Fw[LTOT + 1];
  double full[LTOT + 1], att[LTOT + 1];
  if (kernel != KERNEL_ERF) {
    oracle_boys(Ltot, alpha * R2, F);
    double m2a = 1.0;
    for (int n = 0; n <= Ltot; ++n) { full[n] = m2a * F[n]; m2a *= -2.0 * alpha; }
  }
  if (kernel != KERNEL_COULOMB) {
    double w2 = omega * omega, ap = alpha * w2 / (alpha + w2), sc = sqrt(ap / alpha);
    oracle_boys(Ltot, ap * R2, Fw);
    double m2a = 1.0;
    for (int n = 0; n <= Ltot; ++n) { att[n] = sc * m2a * Fw[n]; m2a *= -2.0 * ap; }
  }
  for (int n = 0; n <= Ltot; ++n) {
    if (kernel == KERNEL_COULOMB) base[n] = full[n];
    else if (kernel == KERNEL_ERF) base[n] = att[n];
    else base[n] = full[n] - att[n];
  }
}

/* Contracted shell-quartet integrals (IJ|KL), out[((a*nJ + b)*nK + c)*nL + d]. */
static void shell_quartet(const basis_t *B, int I, int J, int K, int L, int kernel, double omega,
                          double *out) {
  const int sh[4] = {I, J, K, L};
  int l[4], n[4], comp[4][MAXC][3];
  for (int s = 0; s < 4; ++s) {
    l[s] = B->l[sh[s]];
    n[s] = ncart(l[s]);
    for (int k = 0; k < n[s]; ++k) cart(l[s], k, comp[s][k]);
  }
  const double *A = B->xyz + 3 * I, *Bc = B->xyz + 3 * J, *C = B->xyz + 3 * K, *D = B->xyz + 3 * L;
  int Lab = l[0] + l[1], Lcd = l[2] + l[3], Ltot = Lab + Lcd;
  int ntot = n[0] * n[1] * n[2] * n[3];
  memset(out, 0, sizeof(double) * ntot);

  ecoef_t Eab[3], Ecd[3];
  rtab_t R;
  double base[LTOT + 1];
  /* W[c][d][t][u][v]: ket-side contraction with R for fixed ket components */
  static __thread double W[MAXC][MAXC][2 * LMAX + 1][2 * LMAX + 1][2 * LMAX + 1];

  for (int ia = B->prim_off[I]; ia < B->prim_off[I + 1]; ++ia)
    for (int ib = B->prim_off[J]; ib < B->prim_off[J + 1]; ++ib) {
      double a = B->alpha[ia], b = B->alpha[ib], p = a + b;
      double cab = B->coef[ia] * B->coef[ib];
      double P[3];
      for (int x = 0; x < 3; ++x) {
        P[x] = (a * A[x] + b * Bc[x]) / p;
        hermite_E(l[0], l[1], a, b, A[x], Bc[x], Eab[x]);
      }
      for (int ic = B->prim_off[K]; ic < B->prim_off[K + 1]; ++ic)
        for (int id = B->prim_off[L]; id < B->prim_off[L + 1]; ++id) {
          double c = B->alpha[ic], d = B->alpha[id], q = c + d;
          double ccd = B->coef[ic] * B->coef[id];
          double Q[3];
          for (int x = 0; x < 3; ++x) {
            Q[x] = (c * C[x] + d * D[x]) / q;
            hermite_E(l[2], l[3], c, d, C[x], D[x], Ecd[x]);
          }
          double alpha = p * q / (p + q);
          double X = P[0] - Q[0], Y = P[1] - Q[1], Z = P[2] - Q[2];
          base_values(Ltot, kernel, omega, alpha, X * X + Y * Y + Z * Z, base);
          hermite_R(Ltot, base, X, Y, Z, R);
          double pref = 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p + q)) * cab * ccd;

          for (int kc = 0; kc < n[2]; ++kc)
            for (int kd = 0; kd < n[3]; ++kd) {
              const int *ec = comp[2][kc], *ed = comp[3][kd];
              int tx = ec[0] + ed[0], ty = ec[1] + ed[1], tz = ec[2] + ed[2];
              for (int t = 0; t <= Lab; ++t)
                for (int u = 0; u <= Lab - t; ++u)
                  for (int v = 0; v <= Lab - t - u; ++v) {
                    double s = 0.0;
                    for (int tau = 0; tau <= tx; ++tau)
                      for (int nu = 0; nu <= ty; ++nu)
                        for (int phi = 0; phi <= tz; ++phi) {
                          double e = Ecd[0][ec[0]][ed[0]][tau] * Ecd[1][ec[1]][ed[1]][nu] *
                                     Ecd[2][ec[2]][ed[2]][phi];
                          double sgn = ((tau + nu + phi) & 1) ? -1.0 : 1.0;
                          s += sgn * e * R[t + tau][u + nu][v + phi];
                        }
                    W[kc][kd][t][u][v] = s;
                  }
            }
          for (int ka = 0; ka < n[0]; ++ka)
            for (int kb = 0; kb < n[1]; ++kb) {
              const int *ea = comp[0][ka], *eb = comp[1][kb];
              for (int kc = 0; kc < n[2]; ++kc)
                for (int kd = 0; kd < n[3]; ++kd) {
                  double s = 0.0;
                  for (int t = 0; t <= ea[0] + eb[0]; ++t)
                    for (int u = 0; u <= ea[1] + eb[1]; ++u)
                      for (int v = 0; v <= ea[2] + eb[2]; ++v)
                        s += Eab[0][ea[0]][eb[0]][t] * Eab[1][ea[1]][eb[1]][u] *
                             Eab[2][ea[2]][eb[2]][v] * W[kc][kd][t][u][v];
                  out[((ka * n[1] + kb) * n[2] + kc) * n[3] + kd] += pref * s;
                }
            }
        }
    }
}

static void fill_basis(basis_t *B, int n_shells, const double *xyz, const int *l, const int *prim_off,
                       const double *alpha, const double *coef, const long long *func_off) {
  B->n_shells = n_shells; B->xyz = xyz; B->l = l; B->prim_off = prim_off;
  B->alpha = alpha; B->coef = coef; B->func_off = func_off;
  B->nbf = (int)func_off[n_shells];
}

/* Integrals of a list of shell quartets; quartet q's block starts at out_off[q]. */
void oracle_quartets(int n_shells, const double *xyz, const int *l, const int *prim_off,
                     const double *alpha, const double *coef, const long long *func_off,
                     int n_q, const int *quartets /* n_q x 4 */, int kernel, double omega,
                     const long long *out_off, double *out) {
  basis_t B;
  fill_basis(&B, n_shells, xyz, l, prim_off, alpha, coef, func_off);
#pragma omp parallel for schedule(dynamic, 1)
  for (int q = 0; q < n_q; ++q) {
    const int *s = quartets + 4 * q;
    shell_quartet(&B, s[0], s[1], s[2], s[3], kernel, omega, out + out_off[q]);
  }
}

/* Schwarz bounds Q[I*ns + J] = sqrt(max_{i in I, j in J} |(ij|ij)|), run's kernel. */
void oracle_schwarz(int n_shells, const double *xyz, const int *l, const int *prim_off,
                    const double *alpha, const double *coef, const long long *func_off, int kernel,
                    double omega, double *Q) {
  basis_t B;
  fill_basis(&B, n_shells, xyz, l, prim_off, alpha, coef, func_off);
#pragma omp parallel for schedule(dynamic, 1)
  for (int I = 0; I < n_shells; ++I) {
    double buf[MAXC * MAXC * MAXC * MAXC];
    for (int J = 0; J <= I; ++J) {
      shell_quartet(&B, I, J, I, J, kernel, omega, buf);
      int nI = ncart(l[I]), nJ = ncart(l[J]);
      double mx = 0.0;
      for (int a = 0; a < nI; ++a)
        for (int b = 0; b < nJ; ++b) {
          double v = fabs(buf[((a * nJ + b) * nI + a) * nJ + b]);
          if (v > mx) mx = v;
        }
      Q[I * n_shells + J] = Q[J * n_shells + I] = sqrt(mx);
    }
  }
}

/* Pmax[I*ns + J] = max_{i in I, j in J} |P_ij|  (Sec. 2, density screening). */
static void shell_pmax(const basis_t *B, const double *P, double *Pm) {
  int ns = B->n_shells, nbf = B->nbf;
  for (int I = 0; I < ns; ++I)
    for (int J = 0; J < ns; ++J) {
      double mx = 0.0;
      for (long long i = B->func_off[I]; i < B->func_off[I + 1]; ++i)
        for (long long j = B->func_off[J]; j < B->func_off[J + 1]; ++j) {
          double v = fabs(P[i * nbf + j]);
          if (v > mx) mx = v;
        }
      Pm[I * ns + J] = mx;
    }
}

/* Survival of shell quartet (A B | C D) (bra A,B; ket C,D).
 * screen = 0: everything survives.  screen = 1: Q_AB Q_CD > tau, and
 * P_scr = max(Pmax_AC, Pmax_AD, Pmax_BC, Pmax_BD) > 0, and, if dscreen,
 * P_scr Q_AB Q_CD > eps. */
static int survives(int ns, const double *Q, const double *Pm, int screen, double tau, int dscreen,
                    double eps, int A, int Bs, int C, int D) {
  if (!screen) return 1;
  double qq = Q[A * ns + Bs] * Q[C * ns + D];
  if (!(qq > tau)) return 0;
  double ps = Pm[A * ns + C];
  if (Pm[A * ns + D] > ps) ps = Pm[A * ns + D];
  if (Pm[Bs * ns + C] > ps) ps = Pm[Bs * ns + C];
  if (Pm[Bs * ns + D] > ps) ps = Pm[Bs * ns + D];
  if (!(ps > 0.0)) return 0;
  if (dscreen && !(ps * qq > eps)) return 0;
  return 1;
}

/* K_ij = sum_kl (ik|jl) P_kl over surviving quartets (dense nbf x nbf, FP64).
 * brute = 1: loop over all ordered shell quartets (I K | J L) and add
 *            (ik|jl) P_kl to K_ij directly (the definition, Eq. H-HFX).
 * brute = 0: loop over canonical quartets (I>=J, K>=L, IJ>=KL) and apply the
 *            8 index permutations of Sec. 2 with degeneracy weights.
 * bra_stride/bra_offset: only canonical bra pairs with index % stride == offset
 *            (a bounded sample for timing; stride 1 = everything).
 * Returns the number of surviving (canonical or ordered) shell quartets. */
long long oracle_build_K(int n_shells, const double *xyz, const int *l, const int *prim_off,
                         const double *alpha, const double *coef, const long long *func_off,
                         const double *P, int kernel, double omega, int screen, double tau,
                         int dscreen, double eps, int brute, int bra_stride, int bra_offset,
                         int nthreads, double *K) {
  basis_t B;
  fill_basis(&B, n_shells, xyz, l, prim_off, alpha, coef, func_off);
  int ns = n_shells, nbf = B.nbf;
  double *Q = (double *)calloc((size_t)ns * ns, sizeof(double));
  double *Pm = (double *)calloc((size_t)ns * ns, sizeof(double));
  if (screen) oracle_schwarz(ns, xyz, l, prim_off, alpha, coef, func_off, kernel, omega, Q);
  shell_pmax(&B, P, Pm);
  memset(K, 0, sizeof(double) * (size_t)nbf * nbf);
  long long count = 0;
  if (nthreads <= 0) nthreads = 1;
  if (bra_stride <= 0) bra_stride = 1;
  long long npair = (long long)ns * (ns + 1) / 2;

#pragma omp parallel num_threads(nthreads) reduction(+ : count)
  {
    double *Kt = (double *)calloc((size_t)nbf * nbf, sizeof(double));
    double g[MAXC * MAXC * MAXC * MAXC];
    if (brute) {
#pragma omp for schedule(dynamic, 1) collapse(2)
      for (int I = 0; I < ns; ++I)
        for (int Ks = 0; Ks < ns; ++Ks)
          for (int J = 0; J < ns; ++J)
            for (int Ls = 0; Ls < ns; ++Ls) {
              if (!survives(ns, Q, Pm, screen, tau, dscreen, eps, I, Ks, J, Ls)) continue;
              ++count;
              shell_quartet(&B, I, Ks, J, Ls, kernel, omega, g);
              int nI = ncart(l[I]), nK = ncart(l[Ks]), nJ = ncart(l[J]), nL = ncart(l[Ls]);
              for (int a = 0; a < nI; ++a)
                for (int k = 0; k < nK; ++k)
                  for (int b = 0; b < nJ; ++b)
                    for (int d = 0; d < nL; ++d) {
                      long long i = func_off[I] + a, kk = func_off[Ks] + k;
                      long long j = func_off[J] + b, ll = func_off[Ls] + d;
                      Kt[i * nbf + j] += g[((a * nK + k) * nJ + b) * nL + d] * P[kk * nbf + ll];
                    }
            }
    } else {
#pragma omp for schedule(dynamic, 1)
      for (long long ij = 0; ij < npair; ++ij) {
        if (ij % bra_stride != bra_offset) continue;
        int I = (int)floor((sqrt(8.0 * (double)ij + 1.0) - 1.0) / 2.0);
        while ((long long)I * (I + 1) / 2 > ij) --I;
        while ((long long)(I + 1) * (I + 2) / 2 <= ij) ++I;
        int J = (int)(ij - (long long)I * (I + 1) / 2);
        for (int Kq = 0; Kq <= I; ++Kq)
          for (int Lq = 0; Lq <= Kq; ++Lq) {
            long long kl = (long long)Kq * (Kq + 1) / 2 + Lq;
            if (kl > ij) continue;
            if (!survives(ns, Q, Pm, screen, tau, dscreen, eps, I, J, Kq, Lq)) continue;
            ++count;
            shell_quartet(&B, I, J, Kq, Lq, kernel, omega, g);
            double fac = 1.0;
            if (I == J) fac *= 0.5;
            if (Kq == Lq) fac *= 0.5;
            if (ij == kl) fac *= 0.5;
            int nI = ncart(l[I]), nJ = ncart(l[J]), nK = ncart(l[Kq]), nL = ncart(l[Lq]);
            for (int a = 0; a < nI; ++a)
              for (int b = 0; b < nJ; ++b)
                for (int c = 0; c < nK; ++c)
                  for (int d = 0; d < nL; ++d) {
                    double v = fac * g[((a * nJ + b) * nK + c) * nL + d];
                    long long ia = func_off[I] + a, ib = func_off[J] + b;
                    long long ic = func_off[Kq] + c, id = func_off[Lq] + d;
                    /* (ab|cd) (ba|cd) (ab|dc) (ba|dc) (cd|ab) (dc|ab) (cd|ba) (dc|ba):
                     * an integral (xy|zw) adds (xy|zw) P_yw to K_xz. */
                    Kt[ia * nbf + ic] += v * P[ib * nbf + id];
                    Kt[ib * nbf + ic] += v * P[ia * nbf + id];
                    Kt[ia * nbf + id] += v * P[ib * nbf + ic];
                    Kt[ib * nbf + id] += v * P[ia * nbf + ic];
                    Kt[ic * nbf + ia] += v * P[id * nbf + ib];
                    Kt[id * nbf + ia] += v * P[ic * nbf + ib];
                    Kt[ic * nbf + ib] += v * P[id * nbf + ia];
                    Kt[id * nbf + ib] += v * P[ic * nbf + ia];
                  }
          }
      }
    }
#pragma omp critical
    {
      for (long long x = 0; x < (long long)nbf * nbf; ++x) K[x] += Kt[x];
    }
    free(Kt);
  }
  free(Q);
  free(Pm);
  return count;
}

/* The exchange block K_IJ (functions of shell I x functions of shell J) of a
 * list of shell pairs, straight from the definition (Eq. H-HFX without -1/2):
 * K_ij = sum over all ordered shell pairs (K, L) whose quartet (I K | J L)
 * survives the screening, of sum_{k in K, l in L} (ik|jl) P_kl.
 * Only the Schwarz bounds Q_IK and Q_JL of the listed shells are computed,
 * so single blocks of large systems cost O(n_shells^2) predicate tests and
 * one shell quartet per surviving (K, L).
 * out_off[p]: start of pair p's nI x nJ block in K_out (row-major).
 * W1_out, W0_out (same layout, may be NULL): over the same surviving (K, L),
 *   W1_ij = sum Q_IK Q_JL sum_{k,l} |P_kl|   and   W0_ij = sum sum_{k,l} |P_kl|,
 * the weights with which a per-integral error bound (relative to Q_IK Q_JL,
 * or absolute) carries into K_ij.
 * Returns the number of surviving ordered shell quartets. */
long long oracle_K_shell_pairs(int n_shells, const double *xyz, const int *l, const int *prim_off,
                               const double *alpha, const double *coef, const long long *func_off,
                               const double *P, int kernel, double omega, int screen, double tau,
                               int dscreen, double eps, int n_pairs, const int *pairs /* n x 2 */,
                               const long long *out_off, int nthreads, double *K_out, double *W1_out,
                               double *W0_out) {
  basis_t B;
  fill_basis(&B, n_shells, xyz, l, prim_off, alpha, coef, func_off);
  int ns = n_shells, nbf = B.nbf;
  double *Pm = (double *)calloc((size_t)ns * ns, sizeof(double));
  double *Q = (double *)calloc((size_t)ns * ns, sizeof(double));
  shell_pmax(&B, P, Pm);
  if (nthreads <= 0) nthreads = 1;
  long long count = 0;
  for (int q = 0; q < n_pairs; ++q) {
    const int I = pairs[2 * q], J = pairs[2 * q + 1];
    const int nI = ncart(l[I]), nJ = ncart(l[J]);
    /* Schwarz rows of I and J (the run's kernel), written into the dense table
     * the screening predicate reads */
    if (screen) {
      const int rows[2] = {I, J};
      for (int r = 0; r < 2; ++r) {
        const int X = rows[r];
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 8)
        for (int Y = 0; Y < ns; ++Y) {
          double buf[MAXC * MAXC * MAXC * MAXC];
          shell_quartet(&B, X, Y, X, Y, kernel, omega, buf);
          int nX = ncart(l[X]), nY = ncart(l[Y]);
          double mx = 0.0;
          for (int a = 0; a < nX; ++a)
            for (int b = 0; b < nY; ++b) {
              double v = fabs(buf[((a * nY + b) * nX + a) * nY + b]);
              if (v > mx) mx = v;
            }
          Q[X * ns + Y] = Q[Y * ns + X] = sqrt(mx);
        }
      }
    }
    double *Kb = K_out + out_off[q];
    memset(Kb, 0, sizeof(double) * nI * nJ);
    if (W1_out) memset(W1_out + out_off[q], 0, sizeof(double) * nI * nJ);
    if (W0_out) memset(W0_out + out_off[q], 0, sizeof(double) * nI * nJ);
    long long cnt = 0;
#pragma omp parallel num_threads(nthreads) reduction(+ : cnt)
    {
      double kt[MAXC * MAXC] = {0}, w1[MAXC * MAXC] = {0}, w0[MAXC * MAXC] = {0};
      double g[MAXC * MAXC * MAXC * MAXC];
#pragma omp for schedule(dynamic, 1)
      for (int Ks = 0; Ks < ns; ++Ks)
        for (int Ls = 0; Ls < ns; ++Ls) {
          if (!survives(ns, Q, Pm, screen, tau, dscreen, eps, I, Ks, J, Ls)) continue;
          ++cnt;
          shell_quartet(&B, I, Ks, J, Ls, kernel, omega, g);
          const int nK = ncart(l[Ks]), nL = ncart(l[Ls]);
          double pabs = 0.0;
          for (int k = 0; k < nK; ++k)
            for (int d = 0; d < nL; ++d) pabs += fabs(P[(func_off[Ks] + k) * nbf + func_off[Ls] + d]);
          const double qq = screen ? Q[I * ns + Ks] * Q[J * ns + Ls] : 0.0;
          for (int a = 0; a < nI; ++a)
            for (int b = 0; b < nJ; ++b) {
              double s = 0.0;
              for (int k = 0; k < nK; ++k)
                for (int d = 0; d < nL; ++d)
                  s += g[((a * nK + k) * nJ + b) * nL + d] * P[(func_off[Ks] + k) * nbf + func_off[Ls] + d];
              kt[a * nJ + b] += s;
              w1[a * nJ + b] += qq * pabs;
              w0[a * nJ + b] += pabs;
            }
        }
#pragma omp critical
      {
        for (int x = 0; x < nI * nJ; ++x) {
          Kb[x] += kt[x];
          if (W1_out) W1_out[out_off[q] + x] += w1[x];
          if (W0_out) W0_out[out_off[q] + x] += w0[x];
        }
      }
    }
    count += cnt;
  }
  free(Q);
  free(Pm);
  return count;
}

/* Number of canonical shell quartets (each unordered pair of shell pairs
 * once) that survive the screening of Sec. 2 (the predicate of survives()),
 * counted without evaluating any quartet: Schwarz bounds of every shell pair
 * with the run's kernel, pairs ranked by descending Q, and for each pair a the
 * pairs b ranked at or before a with Q_a Q_b > tau (a prefix of the ranking)
 * tested one by one.  Q_out (ns x ns, may be NULL) receives the bounds. */
typedef struct { double q; int i, j; } qpair_t;

static int qpair_desc(const void *x, const void *y) {
  const qpair_t *a = (const qpair_t *)x, *b = (const qpair_t *)y;
  if (a->q != b->q) return a->q > b->q ? -1 : 1;
  if (a->i != b->i) return a->i < b->i ? -1 : 1;
  return a->j < b->j ? -1 : (a->j > b->j);
}

long long oracle_count_quartets(int n_shells, const double *xyz, const int *l, const int *prim_off,
                                const double *alpha, const double *coef, const long long *func_off,
                                const double *P, int kernel, double omega, double tau, int dscreen, double eps,
                                int nthreads, double *Q_out) {
  basis_t B;
  fill_basis(&B, n_shells, xyz, l, prim_off, alpha, coef, func_off);
  int ns = n_shells;
  double *Q = (double *)calloc((size_t)ns * ns, sizeof(double));
  double *Pm = (double *)calloc((size_t)ns * ns, sizeof(double));
  oracle_schwarz(ns, xyz, l, prim_off, alpha, coef, func_off, kernel, omega, Q);
  shell_pmax(&B, P, Pm);
  long long npair = (long long)ns * (ns + 1) / 2;
  qpair_t *pr = (qpair_t *)malloc(sizeof(qpair_t) * (size_t)npair);
  long long k = 0;
  for (int I = 0; I < ns; ++I)
    for (int J = 0; J <= I; ++J) {
      pr[k].q = Q[I * ns + J];
      pr[k].i = I;
      pr[k].j = J;
      ++k;
    }
  qsort(pr, (size_t)npair, sizeof(qpair_t), qpair_desc);
  if (nthreads <= 0) nthreads = 1;
  long long count = 0;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 256) reduction(+ : count)
  for (long long a = 0; a < npair; ++a) {
    const double qa = pr[a].q;
    /* last b with qa q_b > tau (q descending) */
    long long lo = 0, hi = a + 1;  /* search in [0, a] */
    while (lo < hi) {
      long long mid = (lo + hi) / 2;
      if (qa * pr[mid].q > tau) lo = mid + 1;
      else hi = mid;
    }
    for (long long b = 0; b < lo; ++b)
      if (survives(ns, Q, Pm, 1, tau, dscreen, eps, pr[a].i, pr[a].j, pr[b].i, pr[b].j)) ++count;
  }
  if (Q_out) memcpy(Q_out, Q, sizeof(double) * (size_t)ns * ns);
  free(pr);
  free(Q);
  free(Pm);
  return count;
}

/* ------------------------------------------------------------------------
 * Periodic systems (Sec. 2, Eq. H-HFX): mu runs over the home cell, nu, lambda
 * and sigma over the cells N, G, H of the auxiliary supercell.
 * ------------------------------------------------------------------------ */

/* Rows b_i of (A^T)^{-1} for the lattice A (rows a_i): n_i = b_i . L for the
 * lattice vector L = sum n_i a_i.  Returns 0 for a singular lattice. */
static int reciprocal_rows(const double *A, double *b) {
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  if (!(fabs(det) > 0.0)) return 0;
  /* b_i = (a_j x a_k) / det, (i, j, k) cyclic */
  for (int i = 0; i < 3; ++i) {
    const double *aj = A + 3 * ((i + 1) % 3), *ak = A + 3 * ((i + 2) % 3);
    b[3 * i + 0] = (aj[1] * ak[2] - aj[2] * ak[1]) / det;
    b[3 * i + 1] = (aj[2] * ak[0] - aj[0] * ak[2]) / det;
    b[3 * i + 2] = (aj[0] * ak[1] - aj[1] * ak[0]) / det;
  }
  return 1;
}

/* The images kept in the extended set: every translate R_a + n1 a1 + n2 a2 +
 * n3 a3 (n != 0) of a home atom a that lies within r_ext of at least one home
 * atom.  Rows (a, n1, n2, n3), atom by atom, shifts in lexicographic order;
 * at most max_out rows are written.  Returns the number of images, -1 for a
 * singular lattice or a negative radius. */
long long oracle_periodic_images(int n_atoms, const double *atom_xyz, const double *lattice, double r_ext,
                                 long long max_out, int *out) {
  double b[9];
  if (!reciprocal_rows(lattice, b) || r_ext < 0.0) return -1;
  double diam = 0.0;
  for (int a = 0; a < n_atoms; ++a)
    for (int c = 0; c < n_atoms; ++c) {
      double d2 = 0.0;
      for (int k = 0; k < 3; ++k) d2 += (atom_xyz[3 * a + k] - atom_xyz[3 * c + k]) * (atom_xyz[3 * a + k] - atom_xyz[3 * c + k]);
      if (sqrt(d2) > diam) diam = sqrt(d2);
    }
  /* a kept image has |L| <= r_ext + diam, hence |n_i| <= |b_i| (r_ext + diam) */
  double bmax = 0.0;
  for (int i = 0; i < 3; ++i) {
    double nb = sqrt(b[3 * i] * b[3 * i] + b[3 * i + 1] * b[3 * i + 1] + b[3 * i + 2] * b[3 * i + 2]);
    if (nb > bmax) bmax = nb;
  }
  const int m = (int)ceil(bmax * (r_ext + diam)) + 1;
  long long count = 0;
  for (int a = 0; a < n_atoms; ++a)
    for (int n1 = -m; n1 <= m; ++n1)
      for (int n2 = -m; n2 <= m; ++n2)
        for (int n3 = -m; n3 <= m; ++n3) {
          if (n1 == 0 && n2 == 0 && n3 == 0) continue;
          double x[3];
          for (int k = 0; k < 3; ++k)
            x[k] = atom_xyz[3 * a + k] + n1 * lattice[k] + n2 * lattice[3 + k] + n3 * lattice[6 + k];
          int near = 0;
          for (int c = 0; c < n_atoms && !near; ++c) {
            double d2 = 0.0;
            for (int k = 0; k < 3; ++k) d2 += (x[k] - atom_xyz[3 * c + k]) * (x[k] - atom_xyz[3 * c + k]);
            near = sqrt(d2) <= r_ext;
          }
          if (!near) continue;
          if (count < max_out) {
            out[4 * count + 0] = a;
            out[4 * count + 1] = n1;
            out[4 * count + 2] = n2;
            out[4 * count + 3] = n3;
          }
          ++count;
        }
  return count;
}

/* Exchange rows of a periodic system (Eq. H-HFX without the -1/2):
 *   K^G_{mu lambda} = sum_{N,H} sum_{nu,sigma} P^{H-N}_{nu sigma} (mu^0 nu^N | lambda^G sigma^H)
 * for mu in the home cell and lambda^G in the extended set (home atoms first,
 * in home order, then the images of oracle_periodic_images in its order);
 * nu^N and sigma^H run over the extended set.
 * Real-space density at the Gamma point (Eq. dm with a single k-point):
 * P^L_{nu sigma} = P_{nu sigma} (the home-cell density) when the atoms of
 * nu^0 and sigma^L are at most r_P apart, and 0 otherwise.
 * Screening as in survives(), with the Schwarz bounds and shell maxima of P
 * over the extended set.  Home shells: grouped by atom in atom order
 * (shell_atom), coefficients normalised.  ext_out: (n_ext x 4) rows
 * (home atom, n1, n2, n3), n_ext = n_atoms + the image count; K_rows:
 * home nbf x extended nbf, row-major.  The sum is taken by brute force over
 * all ordered shell triples (K, J, L) for every home shell I.
 * Returns the number of surviving ordered shell quartets, -1 on bad input. */
long long oracle_K_periodic(int n_shells, const int *shell_atom, const int *l, const int *prim_off,
                            const double *alpha, const double *coef, const long long *func_off, int n_atoms,
                            const double *atom_xyz, const double *lattice, double r_ext, double r_P,
                            const double *P_home, int kernel, double omega, int screen, double tau, int dscreen,
                            double eps, int nthreads, int *ext_out, double *K_rows) {
  for (int s = 1; s < n_shells; ++s)
    if (shell_atom[s] < shell_atom[s - 1]) return -1;
  const long long n_img = oracle_periodic_images(n_atoms, atom_xyz, lattice, r_ext, 0, NULL);
  if (n_img < 0) return -1;
  const int n_ext = n_atoms + (int)n_img;
  int *img = (int *)malloc(sizeof(int) * 4 * (size_t)(n_img + 1));
  oracle_periodic_images(n_atoms, atom_xyz, lattice, r_ext, n_img, img);
  for (int a = 0; a < n_atoms; ++a) {
    ext_out[4 * a] = a;
    ext_out[4 * a + 1] = ext_out[4 * a + 2] = ext_out[4 * a + 3] = 0;
  }
  memcpy(ext_out + 4 * (size_t)n_atoms, img, sizeof(int) * 4 * (size_t)n_img);
  free(img);

  /* home atom -> its shells [s0, s1) and functions [f0, f1) */
  int *as0 = (int *)calloc((size_t)n_atoms + 1, sizeof(int));
  for (int s = 0; s < n_shells; ++s) as0[shell_atom[s] + 1]++;
  for (int a = 0; a < n_atoms; ++a) as0[a + 1] += as0[a];
  const int nbf_home = (int)func_off[n_shells];

  /* extended shells: each extended atom carries its home atom's shells */
  int ens = 0, enp = 0;
  for (int X = 0; X < n_ext; ++X) {
    const int h = ext_out[4 * X];
    ens += as0[h + 1] - as0[h];
    enp += prim_off[as0[h + 1]] - prim_off[as0[h]];
  }
  double *exyz = (double *)malloc(sizeof(double) * 3 * (size_t)ens);
  double *axyz = (double *)malloc(sizeof(double) * 3 * (size_t)n_ext);
  int *el = (int *)malloc(sizeof(int) * (size_t)ens);
  int *epo = (int *)malloc(sizeof(int) * ((size_t)ens + 1));
  double *eal = (double *)malloc(sizeof(double) * (size_t)enp);
  double *eco = (double *)malloc(sizeof(double) * (size_t)enp);
  long long *efo = (long long *)malloc(sizeof(long long) * ((size_t)ens + 1));
  int *eatom_f0 = (int *)malloc(sizeof(int) * ((size_t)n_ext + 1));
  int es = 0;
  epo[0] = 0;
  efo[0] = 0;
  for (int X = 0; X < n_ext; ++X) {
    const int *e = ext_out + 4 * X;
    for (int k = 0; k < 3; ++k)
      axyz[3 * X + k] = atom_xyz[3 * e[0] + k] + e[1] * lattice[k] + e[2] * lattice[3 + k] + e[3] * lattice[6 + k];
    eatom_f0[X] = (int)efo[es];
    for (int s = as0[e[0]]; s < as0[e[0] + 1]; ++s, ++es) {
      for (int k = 0; k < 3; ++k) exyz[3 * es + k] = axyz[3 * X + k];
      el[es] = l[s];
      const int np = prim_off[s + 1] - prim_off[s];
      memcpy(eal + epo[es], alpha + prim_off[s], sizeof(double) * np);
      memcpy(eco + epo[es], coef + prim_off[s], sizeof(double) * np);
      epo[es + 1] = epo[es] + np;
      efo[es + 1] = efo[es] + ncart(l[s]);
    }
  }
  eatom_f0[n_ext] = (int)efo[ens];
  const long long nbf = efo[ens];

  /* P over the extended set, block by block of atom pairs */
  double *Pe = (double *)calloc((size_t)(nbf * nbf), sizeof(double));
  for (int X = 0; X < n_ext; ++X)
    for (int Y = 0; Y < n_ext; ++Y) {
      double d2 = 0.0;
      for (int k = 0; k < 3; ++k) d2 += (axyz[3 * X + k] - axyz[3 * Y + k]) * (axyz[3 * X + k] - axyz[3 * Y + k]);
      if (sqrt(d2) > r_P) continue;
      const int hx = ext_out[4 * X], hy = ext_out[4 * Y];
      const long long fx = func_off[as0[hx]], fy = func_off[as0[hy]];
      const int nx = eatom_f0[X + 1] - eatom_f0[X], ny = eatom_f0[Y + 1] - eatom_f0[Y];
      for (int i = 0; i < nx; ++i)
        for (int j = 0; j < ny; ++j)
          Pe[(eatom_f0[X] + i) * nbf + eatom_f0[Y] + j] = P_home[(fx + i) * nbf_home + fy + j];
    }

  basis_t B;
  fill_basis(&B, ens, exyz, el, epo, eal, eco, efo);
  double *Q = (double *)calloc((size_t)ens * ens, sizeof(double));
  double *Pm = (double *)calloc((size_t)ens * ens, sizeof(double));
  if (screen) oracle_schwarz(ens, exyz, el, epo, eal, eco, efo, kernel, omega, Q);
  shell_pmax(&B, Pe, Pm);
  memset(K_rows, 0, sizeof(double) * (size_t)nbf_home * (size_t)nbf);
  if (nthreads <= 0) nthreads = 1;
  long long count = 0;
#pragma omp parallel num_threads(nthreads) reduction(+ : count)
  {
    double *Kt = (double *)calloc((size_t)nbf_home * (size_t)nbf, sizeof(double));
    double g[MAXC * MAXC * MAXC * MAXC];
#pragma omp for schedule(dynamic, 1) collapse(2)
    for (int I = 0; I < n_shells; ++I) /* the home shells are the first n_shells extended shells */
      for (int Ks = 0; Ks < ens; ++Ks)
        for (int J = 0; J < ens; ++J)
          for (int Ls = 0; Ls < ens; ++Ls) {
            if (!survives(ens, Q, Pm, screen, tau, dscreen, eps, I, Ks, J, Ls)) continue;
            ++count;
            shell_quartet(&B, I, Ks, J, Ls, kernel, omega, g);
            const int nI = ncart(el[I]), nK = ncart(el[Ks]), nJ = ncart(el[J]), nL = ncart(el[Ls]);
            for (int a = 0; a < nI; ++a)
              for (int k = 0; k < nK; ++k)
                for (int c = 0; c < nJ; ++c)
                  for (int d = 0; d < nL; ++d)
                    Kt[(efo[I] + a) * nbf + efo[J] + c] +=
                        g[((a * nK + k) * nJ + c) * nL + d] * Pe[(efo[Ks] + k) * nbf + efo[Ls] + d];
          }
#pragma omp critical
    {
      for (long long x = 0; x < (long long)nbf_home * nbf; ++x) K_rows[x] += Kt[x];
    }
    free(Kt);
  }
  free(Q); free(Pm); free(Pe); free(as0); free(exyz); free(axyz); free(el); free(epo); free(eal); free(eco);
  free(efo); free(eatom_f0);
  return count;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
