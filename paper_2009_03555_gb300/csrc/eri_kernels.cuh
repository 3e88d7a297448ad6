// eri_kernels.cuh -- per-class kernel templates of the HFX library:
//   * k_build_K   persistent exchange-build kernel: warps pull quartet batches
//                 from a device work queue (atomic counter), screen each
//                 quartet, evaluate its contracted ERIs and scatter the four
//                 exchange contributions into atom-pair-blocked K;
//   * k_schwarz   Schwarz bounds Q_AB = sqrt(max |(ab|ab)|) of shell pairs;
//   * k_eval      raw shell-quartet integrals (diagnostics and tests).
// Included once per angular-momentum class by the generated tu_*.cu files.
#pragma once
#include <cuda_runtime.h>

#include "eri_common.cuh"

namespace hfx {

constexpr int kThreadsK = 128;

enum Kernel { kCoulomb = 0, kErfc = 1, kErf = 2 };

struct BuildArgs {
  const PairRec* bra_pairs;
  const PrimPair* bra_prims;
  const PairRec* ket_pairs;
  const PrimPair* ket_prims;
  const Desc* desc;
  int n_desc;
  int* counter;           // work-queue head (zeroed before the launch)
  int same_class;         // bra class == ket class: canonical k >= bra rank
  const double* boys;     // Boys table
  int kernel;             // Kernel
  double omega2;          // omega^2 of the attenuated kernels
  int screen;             // Schwarz + P_scr > 0 tests on
  double tau;             // Schwarz threshold
  int dscreen;            // density screening on
  double eps;             // density-screening threshold
  int route;              // 0: all quartets, 1: only bound <= promote, 2: only bound > promote
  double promote;         // FP64 promotion bound on Q_AB Q_CD P_scr
  const double* pmax;     // n_shells x n_shells shell-pair max |P|
  int ns;
  const double* P;        // block-sparse P values
  double* K;              // block-sparse K values (accumulated, not symmetrised)
  const long long* blk_off;  // n_atoms x n_atoms block offsets, -1 = absent
  int n_atoms;
  const int* sh_atom;     // atom of each shell
  const int* sh_loc;      // first function of each shell within its atom
  const int* atom_nf;     // functions per atom
  unsigned long long* n_done;  // [0] quartets computed, [1] primitive quartets computed
};

struct SchwarzArgs {
  const PairRec* pairs;   // all shell pairs
  const PrimPair* prims;
  const int* pair_class;
  int n_pairs;
  int cls;                // pair class handled by this launch
  const double* boys;
  int kernel;
  double omega2;
  double* Q;              // out: Schwarz bound per pair
};

struct EvalArgs {
  const PairRec* pairs;
  const PrimPair* prims;
  const int4* quartets;     // (bra pair, ket pair, class, unused) per item
  const long long* out_off; // per item
  const int4* strides;      // per item: output strides of canonical a, b, c, d
  int n;
  int cls;
  const double* boys;
  int kernel;
  double omega2;
  double* out;
};

// Auxiliary integrals G_m = [00|00]^(m), m = 0..L, FP64.
//   Coulomb: G_m = pref F_m(T)
//   erf(w r)/r:  G_m = pref f^{m+1/2} F_m(f T),  f = w^2 / (w^2 + rho)
//   erfc(w r)/r: Coulomb - erf   (Sec. 2, Eq. ERI-SR)
template <int L>
__device__ __forceinline__ void aux_integrals(const double* __restrict__ boys, int kernel, double omega2,
                                              double T, double rho, double pref, double* G) {
  double F[L + 1];
  if (kernel != kErf) {
    boys_fp64<L>(boys, T, F);
    if (kernel == kCoulomb) {
#pragma unroll
      for (int m = 0; m <= L; ++m) G[m] = pref * F[m];
      return;
    }
  }
  const double f = omega2 * rcp_nr(omega2 + rho);
  double Fw[L + 1];
  boys_fp64<L>(boys, f * T, Fw);
  double s = pref * (f * rsqrt_nr(f));
  if (kernel == kErfc) {
#pragma unroll
    for (int m = 0; m <= L; ++m) {
      G[m] = fma(-s, Fw[m], pref * F[m]);
      s *= f;
    }
  } else {
#pragma unroll
    for (int m = 0; m <= L; ++m) {
      G[m] = s * Fw[m];
      s *= f;
    }
  }
}

// Contracted integrals (ab|cd) of one shell quartet into out[NOUT]
// (index ((a NB + b) NC + c) ND + d).  The per-primitive-quartet prologue
// (argument T, prefactor, Boys function) is FP64; the recursions, the
// contraction and the horizontal recursion run in R.
template <class C, typename R>
__device__ __forceinline__ void contracted_quartet(const PairRec& bra, const PrimPair* __restrict__ bprims,
                                                   const PairRec& ket, const PrimPair* __restrict__ kprims,
                                                   const double* __restrict__ boys, int kernel,
                                                   double omega2, R* __restrict__ out) {
  R acc[C::NACC];
#pragma unroll
  for (int i = 0; i < C::NACC; ++i) acc[i] = R(0);
  for (int ib = 0; ib < bra.pcnt; ++ib) {
    const PrimPair pb = bprims[bra.poff + ib];
    for (int ik = 0; ik < ket.pcnt; ++ik) {
      const PrimPair pk = kprims[ket.poff + ik];
      const double s = pb.p + pk.p;
      const double inv_s = rcp_nr(s);
      const double rho = pb.p * pk.p * inv_s;
      const double PQx = pb.P[0] - pk.P[0], PQy = pb.P[1] - pk.P[1], PQz = pb.P[2] - pk.P[2];
      const double T = rho * fma(PQx, PQx, fma(PQy, PQy, PQz * PQz));
      const double pref = kTwoPi52 * pb.kp * pk.kp * rsqrt_nr(s);
      double Gd[C::L + 1];
      aux_integrals<C::L>(boys, kernel, omega2, T, rho, pref, Gd);
      R G[C::L + 1];
#pragma unroll
      for (int m = 0; m <= C::L; ++m) G[m] = R(Gd[m]);
      VrrGeo<R> g;
      const R rinv = R(inv_s);
      const R rop = R(pk.p) * rinv, roq = R(pb.p) * rinv;
      g.PA[0] = R(pb.PA[0]); g.PA[1] = R(pb.PA[1]); g.PA[2] = R(pb.PA[2]);
      g.QC[0] = R(pk.PA[0]); g.QC[1] = R(pk.PA[1]); g.QC[2] = R(pk.PA[2]);
      const R qx = R(PQx), qy = R(PQy), qz = R(PQz);
      g.WP[0] = -rop * qx; g.WP[1] = -rop * qy; g.WP[2] = -rop * qz;
      g.WQ[0] = roq * qx; g.WQ[1] = roq * qy; g.WQ[2] = roq * qz;
      g.oo2p = R(pb.oo2p);
      g.oo2q = R(pk.oo2p);
      g.oo2pq = R(0.5) * rinv;
      g.rop = rop;
      g.roq = roq;
      C::template vrr<R>(G, g, acc);
    }
  }
  C::template hrr<R>(acc, R(bra.AB[0]), R(bra.AB[1]), R(bra.AB[2]), R(ket.AB[0]), R(ket.AB[1]),
                     R(ket.AB[2]), out);
}

// The four exchange contributions of canonical quartet (AB|CD) with integrals
// g = (ab|cd) and degeneracy weight fac (Sec. 2, 8-fold symmetry; Alg. 4):
//   K_AC += g P_BD,  K_BC += g P_AD,  K_AD += g P_BC,  K_BD += g P_AC.
// The other four permutations give the transposes; K is symmetrised after the
// build.  Blocks outside the sparsity pattern are skipped (P is zero there and
// K is not stored there).  Accumulation into K is FP64.
template <class C, typename R>
__device__ __forceinline__ void scatter_K(const BuildArgs& a, int sA, int sB, int sC, int sD,
                                          const R* __restrict__ g, double fac) {
  constexpr int NA = C::NA, NB = C::NB, NC = C::NC, ND = C::ND;
  const int na = a.n_atoms;
  const int atA = a.sh_atom[sA], atB = a.sh_atom[sB], atC = a.sh_atom[sC], atD = a.sh_atom[sD];
  const int lA = a.sh_loc[sA], lB = a.sh_loc[sB], lC = a.sh_loc[sC], lD = a.sh_loc[sD];
  const int nfC = a.atom_nf[atC], nfD = a.atom_nf[atD];
  const long long oAC = a.blk_off[atA * na + atC], oAD = a.blk_off[atA * na + atD];
  const long long oBC = a.blk_off[atB * na + atC], oBD = a.blk_off[atB * na + atD];
  const double* __restrict__ P = a.P;
  double* K = a.K;
  if (oAC >= 0 && oBD >= 0) {  // K_AC += g P_BD ; K_BD += g P_AC
    R pBD[NB * ND], pAC[NA * NC];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int d = 0; d < ND; ++d) pBD[b * ND + d] = R(__ldg(P + oBD + (long long)(lB + b) * nfD + lD + d));
#pragma unroll
    for (int x = 0; x < NA; ++x)
#pragma unroll
      for (int c = 0; c < NC; ++c) pAC[x * NC + c] = R(__ldg(P + oAC + (long long)(lA + x) * nfC + lC + c));
#pragma unroll
    for (int x = 0; x < NA; ++x)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        R s = R(0);
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int d = 0; d < ND; ++d) s += g[((x * NB + b) * NC + c) * ND + d] * pBD[b * ND + d];
        atomicAdd(K + oAC + (long long)(lA + x) * nfC + lC + c, fac * (double)s);
      }
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        R s = R(0);
#pragma unroll
        for (int x = 0; x < NA; ++x)
#pragma unroll
          for (int c = 0; c < NC; ++c) s += g[((x * NB + b) * NC + c) * ND + d] * pAC[x * NC + c];
        atomicAdd(K + oBD + (long long)(lB + b) * nfD + lD + d, fac * (double)s);
      }
  }
  if (oBC >= 0 && oAD >= 0) {  // K_BC += g P_AD ; K_AD += g P_BC
    R pAD[NA * ND], pBC[NB * NC];
#pragma unroll
    for (int x = 0; x < NA; ++x)
#pragma unroll
      for (int d = 0; d < ND; ++d) pAD[x * ND + d] = R(__ldg(P + oAD + (long long)(lA + x) * nfD + lD + d));
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int c = 0; c < NC; ++c) pBC[b * NC + c] = R(__ldg(P + oBC + (long long)(lB + b) * nfC + lC + c));
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        R s = R(0);
#pragma unroll
        for (int x = 0; x < NA; ++x)
#pragma unroll
          for (int d = 0; d < ND; ++d) s += g[((x * NB + b) * NC + c) * ND + d] * pAD[x * ND + d];
        atomicAdd(K + oBC + (long long)(lB + b) * nfC + lC + c, fac * (double)s);
      }
#pragma unroll
    for (int x = 0; x < NA; ++x)
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        R s = R(0);
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int c = 0; c < NC; ++c) s += g[((x * NB + b) * NC + c) * ND + d] * pBC[b * NC + c];
        atomicAdd(K + oAD + (long long)(lA + x) * nfD + lD + d, fac * (double)s);
      }
  }
}

// Persistent exchange-build kernel for one quartet class.  The device work
// queue replaces the paper's master/sub-master/worker message passing
// (Sec. 3, Algorithms 1-3): lane 0 of a warp takes the next batch descriptor
// with one atomicAdd on the queue head (the master's "send the indexes of the
// batched ERIs"); the warp then hands the batch's quartets to its 32 lanes in
// groups of 32 (the sub-master level); a head past the end is the terminal
// token.  Each lane runs the body of Algorithm 4 for its quartet: screen,
// compute the shell quartet, accumulate into K.
template <class C, typename R>
__global__ void __launch_bounds__(kThreadsK) k_build_K(const BuildArgs a) {
  const int lane = threadIdx.x & 31;
  unsigned long long done = 0, pdone = 0;
  for (;;) {
    int d = 0;
    if (lane == 0) d = atomicAdd(a.counter, 1);
    d = __shfl_sync(0xffffffffu, d, 0);
    if (d >= a.n_desc) break;
    const Desc ds = a.desc[d];
    const PairRec bra = a.bra_pairs[ds.bra];
    for (int kb = ds.k0; kb < ds.k1; kb += 32) {
      const int k = kb + lane;
      if (k >= ds.k1) continue;
      const PairRec ket = a.ket_pairs[k];
      const double qq = bra.Q * ket.Q;
      bool go = true;
      double pscr = 0.0;
      if (a.screen || a.route) {
        const double* pm = a.pmax;
        const int ns = a.ns;
        pscr = fmax(fmax(pm[bra.A * ns + ket.A], pm[bra.A * ns + ket.B]),
                    fmax(pm[bra.B * ns + ket.A], pm[bra.B * ns + ket.B]));
      }
      if (a.screen) {
        go = (qq > a.tau) && (pscr > 0.0);
        if (go && a.dscreen) go = pscr * qq > a.eps;
      }
      if (go && a.route) {
        const bool big = qq * pscr > a.promote;
        go = (a.route == 1) ? !big : big;
      }
      if (!go) continue;
      double fac = 1.0;
      if (bra.A == bra.B) fac *= 0.5;
      if (ket.A == ket.B) fac *= 0.5;
      if (a.same_class && k == ds.bra) fac *= 0.5;
      R out[C::NOUT];
      contracted_quartet<C, R>(bra, a.bra_prims, ket, a.ket_prims, a.boys, a.kernel, a.omega2, out);
      scatter_K<C, R>(a, bra.A, bra.B, ket.A, ket.B, out, fac);
      ++done;
      pdone += (unsigned long long)(bra.pcnt * ket.pcnt);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    done += __shfl_down_sync(0xffffffffu, done, o);
    pdone += __shfl_down_sync(0xffffffffu, pdone, o);
  }
  if (lane == 0 && done) {
    atomicAdd(a.n_done, done);
    atomicAdd(a.n_done + 1, pdone);
  }
}

// Schwarz bounds of every shell pair of pair class `cls` (Sec. 2, Eq. schwarz):
// Q_AB = sqrt(max_{a in A, b in B} |(ab|ab)|), FP64, with the run's kernel.
template <class C>
__global__ void __launch_bounds__(64) k_schwarz(const SchwarzArgs a) {
  if constexpr (C::bra_class == C::ket_class) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_pairs || a.pair_class[i] != a.cls) return;
    const PairRec pr = a.pairs[i];
    double out[C::NOUT];
    contracted_quartet<C, double>(pr, a.prims, pr, a.prims, a.boys, a.kernel, a.omega2, out);
    double mx = 0.0;
#pragma unroll
    for (int x = 0; x < C::NA; ++x)
#pragma unroll
      for (int b = 0; b < C::NB; ++b) mx = fmax(mx, fabs(out[((x * C::NB + b) * C::NA + x) * C::NB + b]));
    a.Q[i] = sqrt(mx);
  }
}

// Raw integrals of listed quartets of this class, written with per-item strides
// so the caller receives them in the shell order it asked for.
template <class C, typename R>
__global__ void __launch_bounds__(64) k_eval(const EvalArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int4 q = a.quartets[i];
  if (q.z != a.cls) return;
  const PairRec bra = a.pairs[q.x], ket = a.pairs[q.y];
  R out[C::NOUT];
  contracted_quartet<C, R>(bra, a.prims, ket, a.prims, a.boys, a.kernel, a.omega2, out);
  const int4 st = a.strides[i];
  double* o = a.out + a.out_off[i];
#pragma unroll
  for (int x = 0; x < C::NA; ++x)
#pragma unroll
    for (int b = 0; b < C::NB; ++b)
#pragma unroll
      for (int c = 0; c < C::NC; ++c)
#pragma unroll
        for (int d = 0; d < C::ND; ++d)
          o[x * st.x + b * st.y + c * st.z + d * st.w] = (double)out[((x * C::NB + b) * C::NC + c) * C::ND + d];
}

// Host-side launchers, one set per class (declared in class_dispatch.h).
template <class C>
void launch_build_K(const BuildArgs& a, int fp32, int grid, cudaStream_t s) {
  if (fp32)
    k_build_K<C, float><<<grid, kThreadsK, 0, s>>>(a);
  else
    k_build_K<C, double><<<grid, kThreadsK, 0, s>>>(a);
}

template <class C>
int occupancy_build_K(int fp32) {
  int nb = 0;
  if (fp32)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_build_K<C, float>, kThreadsK, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_build_K<C, double>, kThreadsK, 0);
  return nb < 1 ? 1 : nb;
}

template <class C>
void launch_schwarz(const SchwarzArgs& a, cudaStream_t s) {
  if (a.n_pairs > 0) k_schwarz<C><<<(a.n_pairs + 63) / 64, 64, 0, s>>>(a);
}

template <class C>
void launch_eval(const EvalArgs& a, int fp32, cudaStream_t s) {
  if (a.n <= 0) return;
  if (fp32)
    k_eval<C, float><<<(a.n + 63) / 64, 64, 0, s>>>(a);
  else
    k_eval<C, double><<<(a.n + 63) / 64, 64, 0, s>>>(a);
}

}  // namespace hfx

#define HFX_INSTANTIATE_CLASS(CL)                                                                   \
  namespace hfx {                                                                                   \
  void launch_K_##CL(const BuildArgs& a, int fp32, int grid, cudaStream_t s) {                      \
    launch_build_K<CL>(a, fp32, grid, s);                                                           \
  }                                                                                                 \
  int occupancy_K_##CL(int fp32) { return occupancy_build_K<CL>(fp32); }                            \
  void launch_schwarz_##CL(const SchwarzArgs& a, cudaStream_t s) { launch_schwarz<CL>(a, s); }      \
  void launch_eval_##CL(const EvalArgs& a, int fp32, cudaStream_t s) { launch_eval<CL>(a, fp32, s); } \
  }
