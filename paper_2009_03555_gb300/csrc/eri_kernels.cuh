// eri_kernels.cuh -- per-class kernel templates of the HFX library:
//   * k_build_K        persistent exchange-build kernel, one thread per shell
//                      quartet (classes with fewer than 90 accumulators): warps
//                      pull quartet batches from a device work queue (atomic
//                      counter), screen the quartets, compact the survivors so
//                      every lane works, evaluate the contracted ERIs and
//                      scatter the four exchange contributions into
//                      atom-pair-blocked K;
//   * k_build_K_split  the same with one warp per shell quartet and the lanes
//                      on its primitive quartets (the d-shell classes), warps
//                      of a block in lockstep rounds for the long recursions;
//   * k_build_K_coop   a table-interpreter variant of the warp-per-quartet
//                      kernel, used only when the build selects it;
//   * k_schwarz, k_schwarz_warp  Schwarz bounds Q_AB = sqrt(max |(ab|ab)|) of
//                      shell pairs (a thread or a warp per pair);
//   * k_eval           raw shell-quartet integrals (diagnostics and tests).
// Included once per angular-momentum class by the generated tu_*.cu files.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

#include "boys_ds.cuh"
#include "eri_common.cuh"

namespace hfx {

constexpr int kThreadsK = 128;
constexpr int kWarpsK = kThreadsK / 32;

// Everything one system contributes to a build: its pair lists, density and
// exchange matrices, pattern tables and Pmax.  Kernels read it from a device
// table indexed by the system id of each batch descriptor, so one launch per
// quartet class serves any number of systems (a single build is a batch of 1).
struct SysArgs {
  const PairRec* pairs[6];  // significant shell pairs per pair class, Q-sorted
  const PrimPair* prims[6];
  const double* pmax;       // n_shells x n_shells shell-pair max |P|
  const double* P;          // block-sparse P values
  double* K;                // block-sparse K values (accumulated, not symmetrised)
  const long long* blk_off; // n_atoms x n_atoms block offsets, -1 = absent
  const int* sh_atom;       // atom of each shell
  const int* sh_loc;        // first function of each shell within its atom
  const int* atom_nf;       // functions per atom
  const int* sh_l;          // angular momentum of each shell
  const int* blk_x;         // pattern blocks (CSR order): atoms, value offsets
  const int* blk_y;
  const long long* blk_val_off;
  long long n_values;
  int n_blocks;
  int ns;
  int n_atoms;
  int n_pairs[6];           // entries of pairs[c]
  long long n_prims[6];     // entries of prims[c]
  // Periodic cell as an extended atom set: its home atoms and their shells
  // come first (equal to n_atoms and ns for a molecule).  Only quartets with a
  // home-cell shell are evaluated: they are the ones that reach the home rows
  // K^G_{mu lambda} (mu in the home cell, Sec. 2, Eq. H-HFX).
  int n_home_atoms;
  int n_home_shells;
};

struct BuildArgs {
  const SysArgs* sys;     // device table of systems
  const Desc* desc;       // batches of this quartet class (Desc::sys = system id)
  int n_desc;             // batches this launch takes: desc[desc_first + i * desc_stride], i < n_desc
  int desc_first, desc_stride;  // one rank's share of a sharded build (0, 1: every batch)
  int n_sys;              // entries of sys
  int* counter;           // work-queue head (zeroed before the launch)
  int bra_class, ket_class;
  int same_class;         // bra class == ket class: canonical k >= bra rank
  const double* boys;     // Boys Taylor tables (FP64)
  const float* boysf;     // the same tables as double-single (mixed path)
  int kernel;             // Kernel
  double omega2;          // omega^2 of the attenuated kernels
  float omega2_hi, omega2_lo;  // the same as a double-single pair (mixed path)
  int screen;             // Schwarz + P_scr > 0 tests on
  double tau;             // Schwarz threshold
  int dscreen;            // density screening on
  double eps;             // density-screening threshold
  float eps_prim;         // primitive quartets with bound_ab bound_cd below this are skipped
  int prim_dscreen;       // 1: the primitive cutoff applies to bound_ab bound_cd P_scr instead
  int route;              // 0: all quartets, 1: only bound <= promote, 2: only bound > promote
  double promote;         // FP64 promotion bound on Q_AB Q_CD P_scr
  int promote_prims;      // promotion per primitive quartet: route 1 takes every quartet and, in those
                          // above the bound, the primitive quartets with bound_ab bound_cd P_scr <= promote;
                          // route 2 the primitive quartets above it
  unsigned long long* n_done;  // [0] quartets computed, [1] primitive quartets computed
};

// What the primitive prologue and recursion read besides the pair data.
struct EriParams {
  const double* boys;
  const float* boysf;
  int kernel;
  double omega2;
  ds w2;           // omega^2 as a double-single pair (mixed path)
  float eps_prim;  // primitive quartets with bound_ab bound_cd below this are skipped
  float prim_hi;   // ... and those above this (the other pass of a promotion per primitive quartet)
};

#ifndef HFX_PT_PREFETCH
#define HFX_PT_PREFETCH -1  // ket primitive-pair prefetch: -1 per class (C::PT_PREFETCH), 0 never, 1 always
#endif

// The primitive quartets of one quartet that a launch evaluates: bound
// products bound_ab bound_cd in [lo, hi] (see quartet_prim_range).
struct PrimRange {
  float lo, hi;
};

__device__ __forceinline__ EriParams eri_params(const BuildArgs& a) {
  return EriParams{a.boys, a.boysf, a.kernel, a.omega2, ds{a.omega2_hi, a.omega2_lo}, a.eps_prim, 3.0e38f};
}

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
  const float* boysf;
  int kernel;
  double omega2;
  float omega2_hi, omega2_lo;
  double* out;
};

// Contracted integrals (ab|cd) of one shell quartet into out[NOUT]
// (index ((a NB + b) NC + c) ND + d).  The per-primitive-quartet prologue
// (argument, prefactor, Boys function, erfc difference) is FP64; the
// recursions, the contraction and the horizontal recursion run in R.
// Primitive pairs are sorted by descending bound, so the loops stop at the
// first primitive quartet whose bound product falls below the range (pr).
// Returns the number of primitive quartets evaluated.
template <class C, typename R>
__device__ __forceinline__ int contracted_quartet(const PairRec& bra, const PrimPair* __restrict__ bprims,
                                                  const PairRec& ket, const PrimPair* __restrict__ kprims,
                                                  const double* __restrict__ boys,
                                                  const float* __restrict__ boysf, int kernel, double omega2,
                                                  ds w2, PrimRange pr, R* __restrict__ out) {
  constexpr bool kMixed = sizeof(R) == 4;
  constexpr int NR = kMixed ? 1 : 2;
  constexpr bool kPrefetch = HFX_PT_PREFETCH < 0 ? C::PT_PREFETCH : HFX_PT_PREFETCH > 0;
  R acc[C::NACC], comp[C::NACC];
#pragma unroll
  for (int i = 0; i < C::NACC; ++i) {
    acc[i] = R(0);
    comp[i] = R(0);
  }
  int n = 0;
  const float kmax = ket.pcnt > 0 ? kprims[ket.poff].bound : 0.f;
  for (int ib = 0; ib < bra.pcnt; ++ib) {
    const PrimPair pb = bprims[bra.poff + ib];
    if (pb.bound * kmax < pr.lo) break;
    // classes with C::PT_PREFETCH load the next ket primitive pair while this
    // one is evaluated (measured per class: faster where it costs no
    // occupancy); HFX_PT_PREFETCH=0/1 turns it off/on for every class
    PrimPair pk_next;
    if constexpr (kPrefetch) {
      if (ket.pcnt > 0) pk_next = kprims[ket.poff];
    }
    for (int ik = 0; ik < ket.pcnt; ++ik) {
      PrimPair pk;
      if constexpr (kPrefetch) {
        pk = pk_next;
        if (ik + 1 < ket.pcnt) pk_next = kprims[ket.poff + ik + 1];
      } else {
        pk = kprims[ket.poff + ik];
      }
      const float bb = pb.bound * pk.bound;
      if (bb < pr.lo) break;
      if (bb > pr.hi) continue;
      ++n;
      R G[C::L + 1], PQ[3], rinv;
      if constexpr (kMixed) {
        prologue_ds<C::L>(boysf, kernel, w2, pb, pk, G, rinv, PQ);
      } else {
        double inv_s;
        prologue<C::L, NR>(boys, kernel, omega2, pb, pk, G, inv_s, PQ);
        rinv = inv_s;
      }
      VrrGeo<R> g;
      if constexpr (kMixed) {
        g.PA[0] = pb.PAf[0]; g.PA[1] = pb.PAf[1]; g.PA[2] = pb.PAf[2];
        g.QC[0] = pk.PAf[0]; g.QC[1] = pk.PAf[1]; g.QC[2] = pk.PAf[2];
        g.oo2p = pb.oo2pf;
        g.oo2q = pk.oo2pf;
      } else {
        g.PA[0] = pb.PA[0]; g.PA[1] = pb.PA[1]; g.PA[2] = pb.PA[2];
        g.QC[0] = pk.PA[0]; g.QC[1] = pk.PA[1]; g.QC[2] = pk.PA[2];
        g.oo2p = pb.oo2p;
        g.oo2q = pk.oo2p;
      }
      const R rop = (kMixed ? R(pk.pf) : R(pk.p)) * rinv, roq = (kMixed ? R(pb.pf) : R(pb.p)) * rinv;
      const R qx = PQ[0], qy = PQ[1], qz = PQ[2];
      g.WP[0] = -rop * qx; g.WP[1] = -rop * qy; g.WP[2] = -rop * qz;
      g.WQ[0] = roq * qx; g.WQ[1] = roq * qy; g.WQ[2] = roq * qz;
      g.oo2pq = R(0.5) * rinv;
      g.rop = rop;
      g.roq = roq;
      C::template vrr<R>(G, g, acc, comp);
    }
  }
  if constexpr (kMixed) {
#pragma unroll
    for (int i = 0; i < C::NACC; ++i) acc[i] -= comp[i];
  }
  C::template hrr<R>(acc, R(bra.AB[0]), R(bra.AB[1]), R(bra.AB[2]), R(ket.AB[0]), R(ket.AB[1]),
                     R(ket.AB[2]), out);
  return n;
}

// The four exchange contributions of canonical quartet (AB|CD) with integrals
// g = (ab|cd) and degeneracy weight fac (Sec. 2, 8-fold symmetry; Alg. 4):
//   K_AC += g P_BD,  K_BC += g P_AD,  K_AD += g P_BC,  K_BD += g P_AC.
// The other four permutations give the transposes; K is symmetrised after the
// build.  Blocks outside the sparsity pattern are skipped (P is zero there and
// K is not stored there).  Accumulation into K is FP64.
template <class C, typename R>
__device__ __forceinline__ void scatter_K(const SysArgs& a, int sA, int sB, int sC, int sD,
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

// P_scr of quartet (AB|CD): the largest |P| over the four exchange blocks
// AC, AD, BC, BD it contracts with (Sec. 2, Eq. dmscreening).
__device__ __forceinline__ double quartet_pscr(const SysArgs& S, const PairRec& bra, const PairRec& ket) {
  const double* pm = S.pmax;
  const int ns = S.ns;
  return fmax(fmax(__ldg(pm + bra.A * ns + ket.A), __ldg(pm + bra.A * ns + ket.B)),
              fmax(__ldg(pm + bra.B * ns + ket.A), __ldg(pm + bra.B * ns + ket.B)));
}

// Primitive cutoff of one quartet.  A primitive quartet adds at most about
// bound_ab bound_cd |P| to any K element, so with prim_dscreen the cutoff is
// applied to that product (the density screening of Eq. dmscreening carried
// down to primitives): eps_prim / P_scr on the bound product.
__device__ __forceinline__ float quartet_prim_cutoff(const BuildArgs& a, const SysArgs& S, const PairRec& bra,
                                                     const PairRec& ket) {
  if (!a.prim_dscreen) return a.eps_prim;
  const double pscr = quartet_pscr(S, bra, ket);
  return pscr > 0.0 ? (float)fmin((double)a.eps_prim / pscr, 3.0e38) : 3.0e38f;
}

// The range of primitive quartets a launch evaluates of one quartet.
// Without promotion, or for a quartet below the promotion bound, [cutoff, inf).  With promotion per
// primitive quartet, a quartet above the bound (Q_AB Q_CD P_scr > promote)
// splits at thr = promote / P_scr: the FP32 launch takes [cutoff, thr], the
// FP64 launch (thr, inf) and the cutoff; together every primitive quartet of
// the cutoff's range runs exactly once.
__device__ __forceinline__ PrimRange quartet_prim_range(const BuildArgs& a, const SysArgs& S, const PairRec& bra,
                                                        const PairRec& ket) {
  const float eps = quartet_prim_cutoff(a, S, bra, ket);
  PrimRange r{eps, 3.0e38f};
  if (a.promote_prims && a.route) {
    const double pscr = quartet_pscr(S, bra, ket);
    if (bra.Q * ket.Q * pscr > a.promote) {
      const float thr = (float)fmin(a.promote / pscr, 3.0e38);
      if (a.route == 1)
        r.hi = thr;
      else
        r.lo = fmaxf(eps, nextafterf(thr, 3.4e38f));
    }
  }
  return r;
}

// Screening of quartet (bra | ket k) (Sec. 2: Eq. schwarz and Eq. dmscreening;
// exact skip when every P block it touches is zero) and precision routing.
__device__ __forceinline__ bool keep_quartet(const BuildArgs& a, const SysArgs& S, const PairRec& bra,
                                             const PairRec& ket) {
  const int nh = S.n_home_shells;
  if (min(min(bra.A, bra.B), min(ket.A, ket.B)) >= nh) return false;  // no home-cell shell
  const double qq = bra.Q * ket.Q;
  double pscr = 0.0;
  if (a.screen || a.route) pscr = quartet_pscr(S, bra, ket);
  if (a.screen) {
    if (!(qq > a.tau) || !(pscr > 0.0)) return false;
    if (a.dscreen && !(pscr * qq > a.eps)) return false;
  }
  if (a.route) {
    const bool big = qq * pscr > a.promote;
    if (a.promote_prims && a.route == 1) return true;  // big quartets split by primitive quartet
    return (a.route == 1) ? !big : big;
  }
  return true;
}

// Number of primitive quartets of (bra|ket) inside the range pr: the
// primitive pairs are sorted by descending bound, so for each bra primitive
// pair the kept ket primitive pairs are a prefix (a staircase).
__device__ __forceinline__ int prim_quartet_count(const PrimPair* __restrict__ bp, const PairRec& bra,
                                                  const PrimPair* __restrict__ kp, const PairRec& ket, PrimRange pr) {
  const float kmax = ket.pcnt > 0 ? kp[ket.poff].bound : 0.f;
  int n = 0;
  for (int ib = 0; ib < bra.pcnt; ++ib) {
    const float b = bp[bra.poff + ib].bound;
    if (b * kmax < pr.lo) break;
    for (int ik = 0; ik < ket.pcnt; ++ik) {
      const float bb = b * kp[ket.poff + ik].bound;
      if (bb < pr.lo) break;
      if (bb <= pr.hi) ++n;
    }
  }
  return n;
}

// Bitonic sort, descending, of the 32 * NPER keys of a warp; key position
// p = 32 j + lane is held by `lane` in k[j].  Strides below 32 exchange
// between lanes (shuffles), larger strides between a lane's registers.
template <int NPER>
__device__ __forceinline__ void warp_sort_desc(unsigned (&k)[NPER]) {
  const int lane = threadIdx.x & 31;
  constexpr int N = 32 * NPER;
#pragma unroll
  for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride >= 32) {
        const int js = stride >> 5;
#pragma unroll
        for (int j = 0; j < NPER; ++j) {
          if (j & js) continue;
          const bool desc = ((j * 32) & size) == 0;
          const unsigned a0 = k[j], a1 = k[j | js];
          const unsigned hi = a0 > a1 ? a0 : a1, lo = a0 > a1 ? a1 : a0;
          k[j] = desc ? hi : lo;
          k[j | js] = desc ? lo : hi;
        }
      } else {
#pragma unroll
        for (int j = 0; j < NPER; ++j) {
          const unsigned v = __shfl_xor_sync(0xffffffffu, k[j], stride);
          const bool lower = (lane & stride) == 0;
          const bool desc = ((j * 32 + lane) & size) == 0;
          const unsigned hi = k[j] > v ? k[j] : v, lo = k[j] > v ? v : k[j];
          k[j] = (lower == desc) ? hi : lo;
        }
      }
    }
  }
}

// Survivors a warp collects before it sorts and runs them (power of two,
// 32..256).
#ifndef HFX_SORT_CAP
#define HFX_SORT_CAP 256
#endif
constexpr int kSortCap = HFX_SORT_CAP;
// HFX_PT_MINB (build switch, > 0) overrides every class's PT_MIN_BLOCKS.
#ifndef HFX_PT_MINB
#define HFX_PT_MINB 0
#endif
template <class C>
struct PerThreadShape {
  static constexpr int MIN_BLOCKS = HFX_PT_MINB > 0 ? HFX_PT_MINB : C::PT_MIN_BLOCKS;
};
static_assert(kSortCap >= 32 && kSortCap <= 256 && (kSortCap & (kSortCap - 1)) == 0, "HFX_SORT_CAP");

// Persistent exchange-build kernel for one quartet class.  The device work
// queue replaces the paper's master/sub-master/worker message passing
// (Sec. 3, Algorithms 1-3): lane 0 of a warp takes the next batch descriptor
// with one atomicAdd on the queue head (the master handing out the indexes of
// the batched ERIs); a head past the end is the terminal token.  The warp
// screens the batch's quartets 32 at a time and appends the survivors to a
// per-warp queue in shared memory (ballot + prefix count), so lanes never idle
// on screened-out quartets.  Each lane runs one quartet at a time (the body of
// Algorithm 4: compute the shell quartet, accumulate into K), and its loop
// over primitive quartets stops at the primitive cutoff, so quartets differ
// in length.  Once kSortCap survivors are queued the warp counts the
// primitive quartets of each, sorts them by that count (bitonic, in
// registers) and runs them in rounds of 32 in that order: the lanes of a
// round then have quartets of nearly equal length.
template <class C, typename R>
__global__ void __launch_bounds__(kThreadsK, PerThreadShape<C>::MIN_BLOCKS) k_build_K(const BuildArgs a) {
  constexpr int NPER = kSortCap / 32;
  __shared__ int4 s_queue[kWarpsK][kSortCap + 32];
  __shared__ unsigned s_key[kWarpsK][kSortCap];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int4* Qw = s_queue[warp];
  unsigned* Kw = s_key[warp];
  int qn = 0;
  unsigned long long done = 0, pdone = 0;

  auto process = [&](int4 it) {  // (system, bra, ket)
    const SysArgs& S = a.sys[it.x];
    const PairRec bra = S.pairs[a.bra_class][it.y];
    const PairRec ket = S.pairs[a.ket_class][it.z];
    double fac = 1.0;
    if (bra.A == bra.B) fac *= 0.5;
    if (ket.A == ket.B) fac *= 0.5;
    if (a.same_class && it.y == it.z) fac *= 0.5;
    R out[C::NOUT];
    pdone += (unsigned long long)contracted_quartet<C, R>(bra, S.prims[a.bra_class], ket, S.prims[a.ket_class],
                                                          a.boys, a.boysf, a.kernel, a.omega2,
                                                          ds{a.omega2_hi, a.omega2_lo},
                                                          quartet_prim_range(a, S, bra, ket), out);
    scatter_K<C, R>(S, bra.A, bra.B, ket.A, ket.B, out, fac);
    ++done;
  };

  // the first m (<= kSortCap) queued quartets, longest first in rounds of 32
  auto run_sorted = [&](int m) {
    unsigned k[NPER];
#pragma unroll
    for (int j = 0; j < NPER; ++j) {
      const int p = 32 * j + lane;
      k[j] = 0u;  // padding sorts last
      if (p < m) {
        const int4 it = Qw[p];
        const SysArgs& S = a.sys[it.x];
        const PairRec bra = S.pairs[a.bra_class][it.y];
        const PairRec ket = S.pairs[a.ket_class][it.z];
        const int n = prim_quartet_count(S.prims[a.bra_class], bra, S.prims[a.ket_class], ket,
                                         quartet_prim_range(a, S, bra, ket));
        k[j] = ((unsigned)(n + 1) << 8) | (unsigned)p;
      }
    }
    warp_sort_desc<NPER>(k);
#pragma unroll
    for (int j = 0; j < NPER; ++j) Kw[32 * j + lane] = k[j];
    __syncwarp();
    const int rounds = (m + 31) >> 5;
#pragma unroll 1
    for (int r = 0; r < rounds; ++r) {
      const unsigned key = Kw[32 * r + lane];
      if (key != 0u) process(Qw[key & 0xffu]);
    }
    __syncwarp();
  };

  for (;;) {
    int d = 0;
    if (lane == 0) d = atomicAdd(a.counter, 1);
    d = __shfl_sync(0xffffffffu, d, 0);
    if (d >= a.n_desc) break;
    const Desc ds = a.desc[a.desc_first + (long long)d * a.desc_stride];
    const SysArgs& S = a.sys[ds.sys];
    const PairRec bra = S.pairs[a.bra_class][ds.bra];
    const PairRec* __restrict__ kets = S.pairs[a.ket_class];
    for (int kb = ds.k0; kb < ds.k1; kb += 32) {
      const int k = kb + lane;
      bool ok = false;
      if (k < ds.k1) ok = keep_quartet(a, S, bra, kets[k]);
      const unsigned m = __ballot_sync(0xffffffffu, ok);
      if (ok) Qw[qn + __popc(m & ((1u << lane) - 1u))] = make_int4(ds.sys, ds.bra, k, 0);
      qn += __popc(m);
      __syncwarp();
      if (qn >= kSortCap) {
        run_sorted(kSortCap);
        if (lane < qn - kSortCap) Qw[lane] = Qw[kSortCap + lane];
        __syncwarp();
        qn -= kSortCap;
      }
    }
  }
  if (qn > 0) run_sorted(qn);
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


// ------------------------------------------------------------ cooperative
// Table-interpreter variant for classes with many contracted accumulators
// (selected at build time by the generator's accumulator threshold; by
// default no class uses it, the warp-split kernel being faster): one warp per
// shell quartet.  The 32 lanes compute the FP64 prologue of 32 primitive
// quartets at once into a per-warp buffer; the warp then walks the vertical
// recursion of each primitive quartet level by level (node tables emitted by
// the generator, intermediates in shared memory), every lane owning a slice of
// the contracted accumulators, which therefore stay in registers.  The
// horizontal recursion and the four exchange contractions are spread over the
// lanes the same way.
constexpr int kThreadsCoop = 64;
constexpr int kGeo = 17;  // PA[3] QC[3] WP[3] WQ[3] oo2p oo2q oo2pq rop roq

template <class C, typename R>
struct CoopLayout {
  using T = typename C::Coop;
  static constexpr int WS = 2 * T::VRR_SLOTS > T::HRR_SLOTS ? 2 * T::VRR_SLOTS : T::HRR_SLOTS;
  static constexpr int PB = C::L + 1 + kGeo;              // prologue record per primitive quartet
  static constexpr int PBUF = 32 * PB > 160 ? 32 * PB : 160;  // also holds the four P blocks
  static constexpr int PER_WARP = WS + PBUF + 64;          // + geometry of the two current quartets
  static constexpr int NPL = (C::NACC + 31) / 32;          // accumulators per lane
  static constexpr size_t bytes() { return (size_t)(kThreadsCoop / 32) * PER_WARP * sizeof(R); }
};

#ifdef HFX_CHECKED
// Checked builds: the n1 x n2 sub-block at rows l1.., columns l2.. of the
// pattern block at offset o (row length nf) lies inside the value array.
template <class C>
__device__ __forceinline__ bool ep_blocks_ok(const SysArgs& S, const BuildArgs& a, long long o, int l1, int n1, int nf, int l2,
                             int n2, const char* what) {
  const int cc = a.bra_class * 10 + a.ket_class;
  return HFX_IN(o + (long long)l1 * nf + l2, S.n_values, what, cc) &&
         HFX_IN(o + (long long)(l1 + n1 - 1) * nf + l2 + n2 - 1, S.n_values, what, cc) &&
         HFX_IN(l2 + n2 - 1, nf, what, cc);
}
#endif

// Horizontal recursion (node tables, shared memory) on the contracted
// [e0|f0] held in ws[0..NACC-1]; the outputs land in the slots the class's
// output table names.  Whole warp.
template <class C, typename R>
__device__ __forceinline__ void quartet_hrr(const PairRec& bra, const PairRec& ket, R* ws) {
  using T = typename C::Coop;
  const int lane = threadIdx.x & 31;
  const uint4* __restrict__ hrr = T::hrr();
  const int* __restrict__ hlev = T::hlev();
  const R ab0 = R(bra.AB[0]), ab1 = R(bra.AB[1]), ab2 = R(bra.AB[2]);
  const R cd0 = R(ket.AB[0]), cd1 = R(ket.AB[1]), cd2 = R(ket.AB[2]);
  for (int l = 1; l <= T::N_HLEV; ++l) {
    const int n1 = __ldg(hlev + l + 1);
    for (int n = __ldg(hlev + l) + lane; n < n1; n += 32) {
      const uint4 x = __ldg(hrr + n);
      const int kind = (x.x >> 16) & 3, axis = (x.x >> 18) & 3;
      const R c = (kind == 2) ? (axis == 0 ? ab0 : (axis == 1 ? ab1 : ab2))
                              : (axis == 0 ? cd0 : (axis == 1 ? cd1 : cd2));
      ws[x.x & 0xffff] = ws[x.y & 0xffff] + c * ws[x.y >> 16];
    }
    __syncwarp();
  }
}

// Horizontal recursion, then the four exchange contributions (see
// scatter_K) spread over the lanes.  Whole warp.
template <class C, typename R>
__device__ __forceinline__ void quartet_epilogue(const BuildArgs& a, const SysArgs& S, const PairRec& bra,
                                                 const PairRec& ket, int bi, int ki, R* ws, R* pbuf) {
  using T = typename C::Coop;
  const int lane = threadIdx.x & 31;
  quartet_hrr<C, R>(bra, ket, ws);
  // four exchange contributions (see scatter_K), outputs spread over lanes
  constexpr int NA = C::NA, NB = C::NB, NC = C::NC, ND = C::ND;
  const unsigned short* __restrict__ outs = T::out();
  double fac = 1.0;
  if (bra.A == bra.B) fac *= 0.5;
  if (ket.A == ket.B) fac *= 0.5;
  if (a.same_class && bi == ki) fac *= 0.5;
  const int na = S.n_atoms;
  const int sA = bra.A, sB = bra.B, sC = ket.A, sD = ket.B;
#ifdef HFX_CHECKED
  {
    const int cc = a.bra_class * 10 + a.ket_class;
    if (!HFX_IN(sA, S.ns, "ep sA", cc) || !HFX_IN(sB, S.ns, "ep sB", cc) || !HFX_IN(sC, S.ns, "ep sC", cc) ||
        !HFX_IN(sD, S.ns, "ep sD", cc))
      return;
    const int t0 = S.sh_atom[sA], t1 = S.sh_atom[sB], t2 = S.sh_atom[sC], t3 = S.sh_atom[sD];
    if (!HFX_IN(t0, na, "ep atA", cc) || !HFX_IN(t1, na, "ep atB", cc) || !HFX_IN(t2, na, "ep atC", cc) ||
        !HFX_IN(t3, na, "ep atD", cc))
      return;
  }
#endif
  const int atA = S.sh_atom[sA], atB = S.sh_atom[sB], atC = S.sh_atom[sC], atD = S.sh_atom[sD];
  const int lA = S.sh_loc[sA], lB = S.sh_loc[sB], lC = S.sh_loc[sC], lD = S.sh_loc[sD];
  const int nfC = S.atom_nf[atC], nfD = S.atom_nf[atD];
  const long long oAC = S.blk_off[atA * na + atC], oAD = S.blk_off[atA * na + atD];
  const long long oBC = S.blk_off[atB * na + atC], oBD = S.blk_off[atB * na + atD];
#ifdef HFX_CHECKED
  const bool h1 = oAC >= 0 && oBD >= 0 && ep_blocks_ok<C>(S, a, oAC, lA, C::NA, nfC, lC, C::NC, "AC") &&
                  ep_blocks_ok<C>(S, a, oBD, lB, C::NB, nfD, lD, C::ND, "BD");
  const bool h2 = oBC >= 0 && oAD >= 0 && ep_blocks_ok<C>(S, a, oBC, lB, C::NB, nfC, lC, C::NC, "BC") &&
                  ep_blocks_ok<C>(S, a, oAD, lA, C::NA, nfD, lD, C::ND, "AD");
#else
  const bool h1 = oAC >= 0 && oBD >= 0, h2 = oBC >= 0 && oAD >= 0;
#endif
  // P blocks into the (now free) prologue buffer: BD | AC | AD | BC
  R* pBD = pbuf;
  R* pAC = pBD + NB * ND;
  R* pAD = pAC + NA * NC;
  R* pBC = pAD + NA * ND;
  for (int e = lane; e < NB * ND; e += 32)
    pBD[e] = h1 ? R(__ldg(S.P + oBD + (long long)(lB + e / ND) * nfD + lD + e % ND)) : R(0);
  for (int e = lane; e < NA * NC; e += 32)
    pAC[e] = h1 ? R(__ldg(S.P + oAC + (long long)(lA + e / NC) * nfC + lC + e % NC)) : R(0);
  for (int e = lane; e < NA * ND; e += 32)
    pAD[e] = h2 ? R(__ldg(S.P + oAD + (long long)(lA + e / ND) * nfD + lD + e % ND)) : R(0);
  for (int e = lane; e < NB * NC; e += 32)
    pBC[e] = h2 ? R(__ldg(S.P + oBC + (long long)(lB + e / NC) * nfC + lC + e % NC)) : R(0);
  __syncwarp();
  constexpr int N1 = NA * NC, N2 = N1 + NB * ND, N3 = N2 + NB * NC, N4 = N3 + NA * ND;
  for (int o = lane; o < N4; o += 32) {
    R s = R(0);
    if (o < N1) {  // K_AC[x][c] += sum_{b,d} g P_BD
      if (!h1) continue;
      const int x = o / NC, c = o % NC;
      for (int b = 0; b < NB; ++b)
        for (int d = 0; d < ND; ++d) s += ws[__ldg(outs + ((x * NB + b) * NC + c) * ND + d)] * pBD[b * ND + d];
      atomicAdd(S.K + oAC + (long long)(lA + x) * nfC + lC + c, fac * (double)s);
    } else if (o < N2) {  // K_BD[b][d] += sum_{x,c} g P_AC
      if (!h1) continue;
      const int b = (o - N1) / ND, d = (o - N1) % ND;
      for (int x = 0; x < NA; ++x)
        for (int c = 0; c < NC; ++c) s += ws[__ldg(outs + ((x * NB + b) * NC + c) * ND + d)] * pAC[x * NC + c];
      atomicAdd(S.K + oBD + (long long)(lB + b) * nfD + lD + d, fac * (double)s);
    } else if (o < N3) {  // K_BC[b][c] += sum_{x,d} g P_AD
      if (!h2) continue;
      const int b = (o - N2) / NC, c = (o - N2) % NC;
      for (int x = 0; x < NA; ++x)
        for (int d = 0; d < ND; ++d) s += ws[__ldg(outs + ((x * NB + b) * NC + c) * ND + d)] * pAD[x * ND + d];
      atomicAdd(S.K + oBC + (long long)(lB + b) * nfC + lC + c, fac * (double)s);
    } else {  // K_AD[x][d] += sum_{b,c} g P_BC
      if (!h2) continue;
      const int x = (o - N3) / ND, d = (o - N3) % ND;
      for (int b = 0; b < NB; ++b)
        for (int c = 0; c < NC; ++c) s += ws[__ldg(outs + ((x * NB + b) * NC + c) * ND + d)] * pBC[b * NC + c];
      atomicAdd(S.K + oAD + (long long)(lA + x) * nfD + lD + d, fac * (double)s);
    }
  }
  __syncwarp();
}


template <class C, typename R>
__device__ __forceinline__ void coop_accumulate(const EriParams& a, const PairRec& bra,
                                                const PrimPair* __restrict__ bprims, const PairRec& ket,
                                                const PrimPair* __restrict__ kprims, R* ws, R* pbuf, R* sg,
                                                unsigned long long& pdone) {
  using T = typename C::Coop;
  using Lay = CoopLayout<C, R>;
  constexpr bool kMixed = sizeof(R) == 4;
  constexpr int NR = kMixed ? 1 : 2;
  constexpr int NG = C::L + 1;
  const int lane = threadIdx.x & 31;
  R acc[Lay::NPL], comp[Lay::NPL];
#pragma unroll
  for (int k = 0; k < Lay::NPL; ++k) {
    acc[k] = R(0);
    comp[k] = R(0);
  }
  const uint4* __restrict__ vrr = T::vrr();
  const int* __restrict__ vlev = T::vlev();
  const int* __restrict__ vsplit = T::vsplit();
  const unsigned short* __restrict__ tgt = T::tgt();
  const int nk = ket.pcnt, total = bra.pcnt * ket.pcnt;
  for (int t0 = 0; t0 < total; t0 += 32) {
    const int t = t0 + lane;
    bool valid = false;
    if (t < total) {
      const int ib = t / nk, ik = t - ib * nk;
      const PrimPair& pb = bprims[bra.poff + ib];
      const PrimPair& pk = kprims[ket.poff + ik];
      const float bb = pb.bound * pk.bound;
      valid = bb >= a.eps_prim && bb <= a.prim_hi;
      if (valid) {
        R* rec = pbuf + lane * Lay::PB;
        R G[NG], PQ[3], rinv;
        if constexpr (kMixed) {
          prologue_ds<C::L>(a.boysf, a.kernel, a.w2, pb, pk, G, rinv, PQ);
        } else {
          double inv_s;
          prologue<C::L, NR>(a.boys, a.kernel, a.omega2, pb, pk, G, inv_s, PQ);
          rinv = inv_s;
        }
#pragma unroll
        for (int m = 0; m < NG; ++m) rec[m] = G[m];
        R* geo = rec + NG;
        const R rop = (kMixed ? R(pk.pf) : R(pk.p)) * rinv, roq = (kMixed ? R(pb.pf) : R(pb.p)) * rinv;
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          geo[x] = kMixed ? R(pb.PAf[x]) : R(pb.PA[x]);
          geo[3 + x] = kMixed ? R(pk.PAf[x]) : R(pk.PA[x]);
          geo[6 + x] = -rop * PQ[x];
          geo[9 + x] = roq * PQ[x];
        }
        geo[12] = kMixed ? R(pb.oo2pf) : R(pb.oo2p);
        geo[13] = kMixed ? R(pk.oo2pf) : R(pk.oo2p);
        geo[14] = R(0.5) * rinv;
        geo[15] = rop;
        geo[16] = roq;
      }
    }
    unsigned mask = __ballot_sync(0xffffffffu, valid);
    __syncwarp();
    pdone += __popc(mask);
    // two primitive quartets per pass (two independent chains per node)
    R* ws1 = ws + T::VRR_SLOTS;
    while (mask) {
      const int j0 = __ffs(mask) - 1;
      mask &= mask - 1;
      int j1 = -1;
      if (mask) {
        j1 = __ffs(mask) - 1;
        mask &= mask - 1;
      }
      const R* rec0 = pbuf + j0 * Lay::PB;
      const R* rec1 = pbuf + (j1 >= 0 ? j1 : j0) * Lay::PB;
      const R live1 = j1 >= 0 ? R(1) : R(0);
      if (lane < NG) {
        ws[1 + lane] = rec0[lane];
        ws1[1 + lane] = live1 * rec1[lane];
      }
      if (lane < kGeo) {
        sg[lane] = rec0[NG + lane];
        sg[32 + lane] = rec1[NG + lane];
      }
      if (lane == 0) {
        ws[0] = R(0);
        ws1[0] = R(0);
      }
      __syncwarp();
      const R oo2pq0 = sg[14], oo2pq1 = sg[32 + 14];
      const R h0b = sg[12], r0b = sg[15], h1b = sg[32 + 12], r1b = sg[32 + 15];
      const R h0k = sg[13], r0k = sg[16], h1k = sg[32 + 13], r1k = sg[32 + 16];
      for (int l = 1; l <= C::L; ++l) {
        const int nb = __ldg(vlev + l), ns = __ldg(vsplit + l), n1 = __ldg(vlev + l + 1);
        for (int n = nb + lane; n < ns; n += 32) {  // bra nodes: PA, WP, 1/(2p), rho/p
          const uint4 x = __ldg(vrr + n);
          const int axis = (x.x >> 18) & 3;
          const R k1 = R((x.x >> 20) & 15);
          const int s0 = x.y & 0xffff, s1 = x.y >> 16, s2 = x.z & 0xffff, s3 = x.z >> 16;
          const R v0 = sg[axis] * ws[s0] + sg[6 + axis] * ws[s1] + k1 * h0b * (ws[s2] - r0b * ws[s3]);
          const R v1 = sg[32 + axis] * ws1[s0] + sg[38 + axis] * ws1[s1] + k1 * h1b * (ws1[s2] - r1b * ws1[s3]);
          ws[x.x & 0xffff] = v0;
          ws1[x.x & 0xffff] = v1;
        }
        for (int n = ns + lane; n < n1; n += 32) {  // ket nodes: QC, WQ, 1/(2q), rho/q, 1/(2(p+q))
          const uint4 x = __ldg(vrr + n);
          const int axis = (x.x >> 18) & 3;
          const R k1 = R((x.x >> 20) & 15), k2 = R((x.x >> 24) & 15);
          const int s0 = x.y & 0xffff, s1 = x.y >> 16, s2 = x.z & 0xffff, s3 = x.z >> 16, s4 = x.w;
          const R v0 = sg[3 + axis] * ws[s0] + sg[9 + axis] * ws[s1] + k1 * h0k * (ws[s2] - r0k * ws[s3]) +
                       k2 * oo2pq0 * ws[s4];
          const R v1 = sg[35 + axis] * ws1[s0] + sg[41 + axis] * ws1[s1] +
                       k1 * h1k * (ws1[s2] - r1k * ws1[s3]) + k2 * oo2pq1 * ws1[s4];
          ws[x.x & 0xffff] = v0;
          ws1[x.x & 0xffff] = v1;
        }
        __syncwarp();
      }
#pragma unroll
      for (int k = 0; k < Lay::NPL; ++k) {
        const int tt = lane + 32 * k;
        if (tt < C::NACC) {
          const int sl = __ldg(tgt + tt);
          kacc<R>(acc[k], comp[k], ws[sl]);
          kacc<R>(acc[k], comp[k], ws1[sl]);
        }
      }
      __syncwarp();
    }
  }
  // contracted [e0|f0] into HRR slots 0..NACC-1
#pragma unroll
  for (int k = 0; k < Lay::NPL; ++k) {
    const int tt = lane + 32 * k;
    if (tt < C::NACC) ws[tt] = kMixed ? acc[k] - comp[k] : acc[k];
  }
  __syncwarp();
}

template <class C, typename R>
__device__ __forceinline__ void coop_quartet(const BuildArgs& a, const SysArgs& S, int bi, int ki, R* ws, R* pbuf,
                                             R* sg, unsigned long long& pdone) {
  const PairRec bra = S.pairs[a.bra_class][bi], ket = S.pairs[a.ket_class][ki];
  EriParams ep = eri_params(a);
  const PrimRange r = quartet_prim_range(a, S, bra, ket);
  ep.eps_prim = r.lo;
  ep.prim_hi = r.hi;
  coop_accumulate<C, R>(ep, bra, S.prims[a.bra_class], ket, S.prims[a.ket_class], ws, pbuf, sg, pdone);
  quartet_epilogue<C, R>(a, S, bra, ket, bi, ki, ws, pbuf);
}

// Persistent cooperative kernel: same device work queue and screening as
// k_build_K; the survivors of each 32-quartet screening round are processed
// one after the other by the whole warp.
template <class C, typename R>
__global__ void __launch_bounds__(kThreadsCoop) k_build_K_coop(const BuildArgs a) {
  using Lay = CoopLayout<C, R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  R* base = reinterpret_cast<R*>(smem_raw) + warp * Lay::PER_WARP;
  R* ws = base;
  R* pbuf = base + Lay::WS;
  R* sg = pbuf + Lay::PBUF;
  unsigned long long done = 0, pdone = 0;
  for (;;) {
    int d = 0;
    if (lane == 0) d = atomicAdd(a.counter, 1);
    d = __shfl_sync(0xffffffffu, d, 0);
    if (d >= a.n_desc) break;
    const Desc ds = a.desc[a.desc_first + (long long)d * a.desc_stride];
#ifdef HFX_CHECKED
    {
      const int cc = a.bra_class * 10 + a.ket_class;
      if (!HFX_IN(ds.sys, a.n_sys, "desc.sys", cc)) continue;
      const SysArgs& S0 = a.sys[ds.sys];
      if (!HFX_IN(ds.bra, S0.n_pairs[a.bra_class], "desc.bra", cc)) continue;
      if (ds.k1 > ds.k0 && (!HFX_IN(ds.k0, S0.n_pairs[a.ket_class], "desc.k0", cc) ||
                            !HFX_IN(ds.k1 - 1, S0.n_pairs[a.ket_class], "desc.k1", cc)))
        continue;
    }
#endif
    const SysArgs& S = a.sys[ds.sys];
    const PairRec bra = S.pairs[a.bra_class][ds.bra];
    const PairRec* __restrict__ kets = S.pairs[a.ket_class];
    for (int kb = ds.k0; kb < ds.k1; kb += 32) {
      const int k = kb + lane;
      bool ok = false;
      if (k < ds.k1) ok = keep_quartet(a, S, bra, kets[k]);
      unsigned m = __ballot_sync(0xffffffffu, ok);
      done += __popc(m);
      while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1;
        coop_quartet<C, R>(a, S, ds.bra, kb + j, ws, pbuf, sg, pdone);
      }
    }
  }
  if (lane == 0 && done) {
    atomicAdd(a.n_done, done);
    atomicAdd(a.n_done + 1, pdone);
  }
}


// ------------------------------------------------------------------ split
// Classes with a medium-large accumulator set run one warp per shell quartet
// with the lanes on different primitive quartets: every lane evaluates the
// generated straight-line vertical recursion of its own primitive quartet and
// the finished targets are reduced over the warp 32 at a time
// (reduce_scatter32), so lane j keeps only the accumulators 32k + j.
// Primitive quartets that survive the bound test are compacted into a
// per-warp queue first, so passes run with full lanes.
//
// The recursion of these classes is thousands of straight-line instructions,
// more than the SM's instruction cache holds, so warps that run it at
// different places each stream their own instructions from L2 and stall on
// instruction fetch.  For those classes (SplitShape::LOCKSTEP) the warps of a
// block advance in rounds: in each round every warp with work runs one pass
// (or the epilogue of a finished quartet, or finds its next quartet), then the
// block meets at a barrier.  The passes of one round start together and run
// the same code, so one instruction stream serves the whole block.  Shapes
// (measured on GB300, 100-atom HSE build; SplitShape): in FP32 one 12- or
// 16-warp lockstep block per SM, the chunk accumulators in shared memory so
// that the recursion fits 168 or 128 registers; the FP32 (dd|dd) pass and the
// FP64 kernels one 8-warp block at 255 registers; recursions below
// HFX_LOCKSTEP_MIN_FLOPS flops without a class setting of their own, three
// independent 4-warp blocks per SM at <= 168 registers.
#ifndef HFX_LOCKSTEP_MIN_FLOPS
#define HFX_LOCKSTEP_MIN_FLOPS 1400
#endif
#ifndef HFX_WIDE_MIN_FLOPS
#define HFX_WIDE_MIN_FLOPS 2000
#endif
// Lockstep classes below HFX_WIDE_MIN_FLOPS run blocks of HFX_MID_WARPS warps
// (4: three blocks per SM; 12: one block per SM, all twelve warps in one
// lockstep stream).
#ifndef HFX_MID_WARPS
#define HFX_MID_WARPS 4
#endif
// Opt-in cap on the warps per block of the FP64 warp-split kernels
// (HFX_SPLIT64_MAX_WARPS=4: the FP64 (dd|dd) pass in 4-warp blocks, its shape
// before the horizontal recursion reused its workspace slots).
#ifndef HFX_SPLIT64_MAX_WARPS
#define HFX_SPLIT64_MAX_WARPS 8
#endif
// Warps per lockstep block of the FP32 wide classes (from HFX_WIDE_MIN_FLOPS
// recursion flops up) and mid classes, unless the class sets its own
// (C::SPLIT_WARPS).  Blocks of more than eight warps run at <= 168 (12 warps)
// or <= 128 (16) registers with the chunk accumulators in shared memory.
// Measured on GB300 (100-atom HSE build): 12-warp blocks against 8 make
// (dd|dp) 25 %, (dd|pp) 25 %, (dd|ds) 15 % and (dp|dp) 12 % faster; more warps
// share each stretch of the instruction stream and hide each other's fetch.
#ifndef HFX_WIDE_WARPS
#define HFX_WIDE_WARPS 12
#endif
#ifndef HFX_MID_WARPS_F32
#define HFX_MID_WARPS_F32 HFX_MID_WARPS
#endif
// HFX_LOCKSTEP64=0: the FP64 warp-split kernels without lockstep rounds.
#ifndef HFX_LOCKSTEP64
#define HFX_LOCKSTEP64 1
#endif
template <class C, typename R>
struct SplitShape {
  static constexpr bool F32 = sizeof(R) == 4;
  static constexpr bool LOCKSTEP = (C::VRR_FLOPS >= HFX_LOCKSTEP_MIN_FLOPS && (F32 || HFX_LOCKSTEP64)) ||
                                   (F32 && C::SPLIT_WARPS > 8);
  // a horizontal-recursion workspace above 32 KB per warp leaves room for
  // 4-warp blocks only.  With its slots reused once their values are dead no
  // class needs that much ((dd|dd): 2844 slots, 22 KB in FP64), so the FP64
  // (dd|dd) pass runs eight warps per SM (188 KB of shared memory) like FP32
  static constexpr bool BIG_HRR = C::Coop::HRR_SLOTS * sizeof(R) > 4096 * sizeof(double);
  static constexpr bool WIDE = C::VRR_FLOPS >= HFX_WIDE_MIN_FLOPS && !BIG_HRR;
  static constexpr bool MID = LOCKSTEP && !WIDE && !BIG_HRR;
  static constexpr int RULE = WIDE ? (F32 ? HFX_WIDE_WARPS : 8) : (MID ? (F32 ? HFX_MID_WARPS_F32 : HFX_MID_WARPS) : 4);
  static constexpr int WANT = (F32 && C::SPLIT_WARPS > 0) ? C::SPLIT_WARPS : RULE;
  // bound on the per-warp shared memory of a block with the accumulators in
  // shared memory (the layout below): more than eight warps only where the
  // block fits
  static constexpr size_t BIG_PER_WARP = (size_t)C::Coop::HRR_SLOTS + 160 + 4 +
                                         (C::Coop::HRR_SLOTS >= kChunkBufElems ? 0 : kChunkBufElems + 4) +
                                         2 * 32 * (C::NCHUNK | 1) + 4;
  static constexpr int WARPS_FIT = (WANT > 8 && WANT * BIG_PER_WARP * sizeof(R) > 227 * 1024) ? 8 : WANT;
  static constexpr bool CAPPED = !F32 && WARPS_FIT > HFX_SPLIT64_MAX_WARPS;
  static constexpr int WARPS = CAPPED ? HFX_SPLIT64_MAX_WARPS : WARPS_FIT;
  static constexpr int THREADS = 32 * WARPS;
  static constexpr int MIN_BLOCKS = (WARPS >= 8 || BIG_HRR || CAPPED) ? 1 : 3;
};

// Split classes with C::SPLIT_SMEM_ACC keep their FP32 chunk accumulators
// and compensations in shared memory instead of registers (chosen per class
// by timing: it removes the register spill of (dp|pp)); HFX_SPLIT_SMEM_ACC
// moves them there for every FP32 class.  (The FP64 (dd|dd) pass has no room
// for them beside eight warps' workspaces.)
template <class C, typename R>
struct SplitLayout {
  using T = typename C::Coop;
#ifdef HFX_SPLIT_SMEM_ACC
  static constexpr bool SMEM_ACC = sizeof(R) == 4;
#else
  static constexpr bool SMEM_ACC = sizeof(R) == 4 && (C::SPLIT_SMEM_ACC || SplitShape<C, R>::WARPS > 8);
#endif
  // 16-byte alignment (the per-warp regions, and the reduction buffer, which
  // takes vector stores)
  static constexpr int ALIGN = 16 / (int)sizeof(R);
  static constexpr int align_up(int n) { return (n + ALIGN - 1) / ALIGN * ALIGN; }
  static constexpr int PER_WARP_BASE = T::HRR_SLOTS + 160;  // HRR workspace + four P blocks
#ifdef HFX_SMEM_REDUCE
  // chunk-reduction buffer: the idle HRR workspace when it is large enough,
  // otherwise after the P blocks at the next 16-byte boundary
  static constexpr bool RED_IN_WS = T::HRR_SLOTS >= kChunkBufElems;
  static constexpr int RED_OFF = RED_IN_WS ? 0 : align_up(PER_WARP_BASE);
  static constexpr int RED_END = RED_IN_WS ? PER_WARP_BASE : RED_OFF + kChunkBufElems;
#else
  static constexpr int RED_OFF = 0;
  static constexpr int RED_END = PER_WARP_BASE;
#endif
  // shared-memory accumulators and compensations: lane-major with an odd
  // stride (no bank conflicts), after everything else (the HRR workspace holds
  // the reduction buffer during the passes and the recursion in the epilogue,
  // which reads the accumulators)
  static constexpr int ACC_STRIDE = C::NCHUNK | 1;
  static constexpr int ACC_WORDS = SMEM_ACC ? 2 * 32 * ACC_STRIDE : 0;
  static constexpr int ACC_OFF = align_up(RED_END);
  static constexpr int PER_WARP = align_up(ACC_OFF + ACC_WORDS);
  static_assert(RED_OFF % ALIGN == 0 && ACC_OFF % ALIGN == 0 && PER_WARP % ALIGN == 0,
                "16-byte aligned shared-memory regions");
  __device__ static R* red_buf(R* ws) { return ws + RED_OFF; }
  __device__ static R* acc_base(R* ws) { return ws + ACC_OFF; }
  static constexpr size_t bytes() { return (size_t)SplitShape<C, R>::WARPS * PER_WARP * sizeof(R); }
  static_assert(bytes() <= 227 * 1024, "split-kernel shared memory per block");
};

// One pass: prologue and vertical recursion of primitive quartet t of the
// shell quartet (bra | ket) on every lane (t < 0: idle lane, zero inputs),
// targets reduced over the warp into acc/comp.
template <class C, typename R>
__device__ __forceinline__ void split_pass(const EriParams& a, const PrimPair* __restrict__ bprims,
                                           const PrimPair* __restrict__ kprims, int bpoff, int kpoff, int nk, int t,
                                           R* acc, R* comp, R* red) {
  constexpr bool kMixed = sizeof(R) == 4;
  constexpr int NR = kMixed ? 1 : 2;
  constexpr int NG = C::L + 1;
  R G[NG], PQ[3] = {R(0), R(0), R(0)}, rinv = R(0);
#pragma unroll
  for (int m = 0; m < NG; ++m) G[m] = R(0);
  VrrGeo<R> g;
#pragma unroll
  for (int x = 0; x < 3; ++x) g.PA[x] = g.QC[x] = R(0);
  g.oo2p = g.oo2q = R(0);
  R rop = R(0), roq = R(0);
  if (t >= 0) {
    const int ib = t / nk, ik = t - ib * nk;
    const PrimPair& pb = bprims[bpoff + ib];
    const PrimPair& pk = kprims[kpoff + ik];
    if constexpr (kMixed) {
      prologue_ds<C::L>(a.boysf, a.kernel, a.w2, pb, pk, G, rinv, PQ);
    } else {
      double inv_s;
      prologue<C::L, NR>(a.boys, a.kernel, a.omega2, pb, pk, G, inv_s, PQ);
      rinv = inv_s;
    }
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      g.PA[x] = kMixed ? R(pb.PAf[x]) : R(pb.PA[x]);
      g.QC[x] = kMixed ? R(pk.PAf[x]) : R(pk.PA[x]);
    }
    g.oo2p = kMixed ? R(pb.oo2pf) : R(pb.oo2p);
    g.oo2q = kMixed ? R(pk.oo2pf) : R(pk.oo2p);
    rop = (kMixed ? R(pk.pf) : R(pk.p)) * rinv;
    roq = (kMixed ? R(pb.pf) : R(pb.p)) * rinv;
  }
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    g.WP[x] = -rop * PQ[x];
    g.WQ[x] = roq * PQ[x];
  }
  g.oo2pq = R(0.5) * rinv;
  g.rop = rop;
  g.roq = roq;
  C::template vrr_split<R>(G, g, acc, comp, red);
}

#ifdef HFX_CHECKED
// Checked builds: the work-queue batch and the primitive ranges it leads to.
__device__ __forceinline__ bool split_desc_ok(const BuildArgs& a, const Desc& ds) {
  const int cc = a.bra_class * 10 + a.ket_class;
  if (!HFX_IN(ds.sys, a.n_sys, "desc.sys", cc)) return false;
  const SysArgs& S0 = a.sys[ds.sys];
  if (!HFX_IN(ds.bra, S0.n_pairs[a.bra_class], "desc.bra", cc)) return false;
  if (ds.k1 > ds.k0 && (!HFX_IN(ds.k0, S0.n_pairs[a.ket_class], "desc.k0", cc) ||
                        !HFX_IN(ds.k1 - 1, S0.n_pairs[a.ket_class], "desc.k1", cc)))
    return false;
  return true;
}
__device__ __forceinline__ bool split_prims_ok(const BuildArgs& a, const SysArgs& S, const PairRec& bra,
                                               const PairRec& ket) {
  const int cc = a.bra_class * 10 + a.ket_class;
  // at most 16 x 16 primitive pairs per shell pair (16 primitives per shell)
  if (bra.pcnt < 0 || ket.pcnt < 0 || bra.pcnt > 256 || ket.pcnt > 256) return hfx_oob("pcnt", bra.pcnt, 256, cc);
  if (bra.pcnt > 0 && (!HFX_IN(bra.poff, S.n_prims[a.bra_class], "bra.poff", cc) ||
                       !HFX_IN(bra.poff + bra.pcnt - 1, S.n_prims[a.bra_class], "bra.poff+pcnt", cc)))
    return false;
  if (ket.pcnt > 0 && (!HFX_IN(ket.poff, S.n_prims[a.ket_class], "ket.poff", cc) ||
                       !HFX_IN(ket.poff + ket.pcnt - 1, S.n_prims[a.ket_class], "ket.poff+pcnt", cc)))
    return false;
  return true;
}
#endif

template <class C, typename R>
__global__ void __launch_bounds__(SplitShape<C, R>::THREADS, SplitShape<C, R>::MIN_BLOCKS)
    k_build_K_split(const BuildArgs a) {
  using Lay = SplitLayout<C, R>;
  constexpr bool kMixed = sizeof(R) == 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_pq[SplitShape<C, R>::WARPS][64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  R* ws = reinterpret_cast<R*>(smem_raw) + warp * Lay::PER_WARP;
  R* pbuf = ws + C::Coop::HRR_SLOTS;
  int* pq = s_pq[warp];
  unsigned long long done = 0, pdone = 0;
  // work-queue position of this warp (uniform over its lanes)
  bool exhausted = false, cur_ok = false;
  Desc cur{0, 0, 0, 0};
  int kb = 0;
  unsigned pend = 0u;  // kept kets of the current 32-ket window, not yet started
  // current shell quartet
  bool have = false;
  int bi = 0, ki = 0, bpoff = 0, kpoff = 0, nk = 1, total = 0, t0 = 0, qn = 0;
  PrimRange pr_q{a.eps_prim, 3.0e38f};  // primitive quartets of the current quartet this launch takes
  R acc_r[Lay::SMEM_ACC ? 1 : C::NCHUNK], comp_r[Lay::SMEM_ACC ? 1 : C::NCHUNK];
  R* const acc = Lay::SMEM_ACC ? Lay::acc_base(ws) + lane * Lay::ACC_STRIDE : acc_r;
  R* const comp = Lay::SMEM_ACC ? Lay::acc_base(ws) + (32 + lane) * Lay::ACC_STRIDE : comp_r;
  for (;;) {
    // A. the next shell quartet: next kept ket of the window, next window of
    //    the batch, or the next batch from the queue (Algorithms 1-3)
    while (!have && !exhausted) {
      if (pend) {
        const int j = __ffs(pend) - 1;
        pend &= pend - 1;
        const SysArgs& S = a.sys[cur.sys];
        bi = cur.bra;
        ki = kb + j;
        const PairRec bra = S.pairs[a.bra_class][bi], ket = S.pairs[a.ket_class][ki];
#ifdef HFX_CHECKED
        if (!split_prims_ok(a, S, bra, ket)) continue;
#endif
        bpoff = bra.poff;
        kpoff = ket.poff;
        pr_q = quartet_prim_range(a, S, bra, ket);
        nk = ket.pcnt > 0 ? ket.pcnt : 1;
        total = bra.pcnt * ket.pcnt;
        t0 = 0;
        qn = 0;
#pragma unroll
        for (int k = 0; k < C::NCHUNK; ++k) acc[k] = comp[k] = R(0);
        have = true;
      } else {
        if (cur_ok && kb + 32 < cur.k1) {
          kb += 32;
        } else {
          int d = 0;
          if (lane == 0) d = atomicAdd(a.counter, 1);
          d = __shfl_sync(0xffffffffu, d, 0);
          if (d >= a.n_desc) {
            exhausted = true;
            break;
          }
          cur = a.desc[a.desc_first + (long long)d * a.desc_stride];
          cur_ok = true;
#ifdef HFX_CHECKED
          cur_ok = split_desc_ok(a, cur);
          if (!cur_ok) continue;
#endif
          kb = cur.k0;
        }
        const SysArgs& S = a.sys[cur.sys];
        const PairRec bra = S.pairs[a.bra_class][cur.bra];
        const int k = kb + lane;
        bool ok = false;
        if (k < cur.k1) ok = keep_quartet(a, S, bra, S.pairs[a.ket_class][k]);
        pend = __ballot_sync(0xffffffffu, ok);
        done += __popc(pend);
      }
    }
    // B. one pass of the current quartet, or its epilogue once every
    //    surviving primitive quartet has been through a pass
    if (have) {
      const SysArgs& S = a.sys[cur.sys];
      const PrimPair* __restrict__ bprims = S.prims[a.bra_class];
      const PrimPair* __restrict__ kprims = S.prims[a.ket_class];
      while (qn < 32 && t0 < total) {
        const int t = t0 + lane;
        bool valid = false;
        if (t < total) {
          const int ib = t / nk, ik = t - ib * nk;
          const float bb = bprims[bpoff + ib].bound * kprims[kpoff + ik].bound;
          valid = bb >= pr_q.lo && bb <= pr_q.hi;
        }
        const unsigned m = __ballot_sync(0xffffffffu, valid);
        if (valid) pq[qn + __popc(m & ((1u << lane) - 1u))] = t;
        qn += __popc(m);
        t0 += 32;
        __syncwarp();
      }
      if (qn == 0) {
        const unsigned short* __restrict__ perm = C::split_perm();
#pragma unroll
        for (int k = 0; k < C::NCHUNK; ++k) {
          const int tt = lane + 32 * k;
          if (tt < C::NACC) ws[perm[tt]] = kMixed ? acc[k] - comp[k] : acc[k];
        }
        __syncwarp();
        const PairRec bra = S.pairs[a.bra_class][bi], ket = S.pairs[a.ket_class][ki];
        quartet_epilogue<C, R>(a, S, bra, ket, bi, ki, ws, pbuf);
        have = false;
      } else {
        const int take = qn < 32 ? qn : 32;
        const int t = lane < take ? pq[lane] : -1;
        __syncwarp();
        if (lane < qn - take) pq[lane] = pq[take + lane];
        __syncwarp();
        qn -= take;
        pdone += take;
        split_pass<C, R>(eri_params(a), bprims, kprims, bpoff, kpoff, nk, t, acc, comp, Lay::red_buf(ws));
      }
    }
    // C. lockstep classes: the round ends for the whole block, which stops
    //    once no warp has work left; otherwise each warp runs on by itself
    if constexpr (SplitShape<C, R>::LOCKSTEP) {
      if (!__syncthreads_or(have || !exhausted)) break;
    } else {
      if (!have && exhausted) break;
    }
  }
  if (lane == 0 && done) {
    atomicAdd(a.n_done, done);
    atomicAdd(a.n_done + 1, pdone);
  }
}

// Schwarz bounds of every shell pair of pair class `cls` (Sec. 2, Eq. schwarz):
// Q_AB = sqrt(max_{a in A, b in B} |(ab|ab)|), FP64, with the run's kernel and
// every primitive quartet.
template <class C>
__global__ void __launch_bounds__(64) k_schwarz(const SchwarzArgs a) {
  if constexpr (C::bra_class == C::ket_class) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_pairs || a.pair_class[i] != a.cls) return;
    const PairRec pr = a.pairs[i];
    double out[C::NOUT];
    contracted_quartet<C, double>(pr, a.prims, pr, a.prims, a.boys, nullptr, a.kernel, a.omega2, ds{0.f, 0.f}, PrimRange{0.f, 3.0e38f},
                                  out);
    double mx = 0.0;
#pragma unroll
    for (int x = 0; x < C::NA; ++x)
#pragma unroll
      for (int b = 0; b < C::NB; ++b) mx = fmax(mx, fabs(out[((x * C::NB + b) * C::NA + x) * C::NB + b]));
    a.Q[i] = sqrt(mx);
  }
}

// Schwarz bounds of the pairs of a pair class whose quartet class runs on the
// warp-split or cooperative build kernels: one warp per pair, the same
// accumulation as the build (FP64, every primitive quartet), the horizontal
// recursion in shared memory, then the largest diagonal |(ab|ab)|.  A thread
// per pair would hold hundreds of FP64 accumulators in local memory.
constexpr int kSchwarzWarps = 4;

template <class C>
struct SchwarzWarpLayout {
  // HRR workspace (also the chunk-reduction buffer of the shared-memory reduction,
  // idle during the passes), 16-byte aligned per warp
  static constexpr int RAW = C::COOP ? CoopLayout<C, double>::PER_WARP
                                     : (C::Coop::HRR_SLOTS > kChunkBufElems ? C::Coop::HRR_SLOTS : kChunkBufElems);
  static constexpr int PER_WARP = (RAW + 1) / 2 * 2;
  static constexpr size_t bytes() { return (size_t)kSchwarzWarps * PER_WARP * sizeof(double); }
};

template <class C>
__global__ void __launch_bounds__(32 * kSchwarzWarps) k_schwarz_warp(const SchwarzArgs a) {
  if constexpr (C::bra_class == C::ket_class && (C::SPLIT || C::COOP)) {
    using T = typename C::Coop;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* ws = reinterpret_cast<double*>(smem_raw) + warp * SchwarzWarpLayout<C>::PER_WARP;
    const EriParams p{a.boys, nullptr, a.kernel, a.omega2, ds{0.f, 0.f}, -1.f, 3.0e38f};  // every primitive quartet
    const unsigned short* __restrict__ outs = T::out();
    for (int i = blockIdx.x * kSchwarzWarps + warp; i < a.n_pairs; i += gridDim.x * kSchwarzWarps) {
      if (a.pair_class[i] != a.cls) continue;
      const PairRec pr = a.pairs[i];
      if constexpr (C::COOP) {
        using Lay = CoopLayout<C, double>;
        unsigned long long pd = 0;
        coop_accumulate<C, double>(p, pr, a.prims, pr, a.prims, ws, ws + Lay::WS, ws + Lay::WS + Lay::PBUF, pd);
      } else {
        double acc[C::NCHUNK], comp[C::NCHUNK];
#pragma unroll
        for (int k = 0; k < C::NCHUNK; ++k) acc[k] = comp[k] = 0.0;
        const int nk = pr.pcnt > 0 ? pr.pcnt : 1, total = pr.pcnt * pr.pcnt;
        for (int t0 = 0; t0 < total; t0 += 32) {
          const int t = t0 + lane < total ? t0 + lane : -1;
          split_pass<C, double>(p, a.prims, a.prims, pr.poff, pr.poff, nk, t, acc, comp, ws);
        }
        const unsigned short* __restrict__ perm = C::split_perm();
#pragma unroll
        for (int k = 0; k < C::NCHUNK; ++k) {
          const int tt = lane + 32 * k;
          if (tt < C::NACC) ws[perm[tt]] = acc[k];
        }
        __syncwarp();
      }
      quartet_hrr<C, double>(pr, pr, ws);
      double mx = 0.0;
      for (int e = lane; e < C::NA * C::NB; e += 32) {
        const int x = e / C::NB, b = e - x * C::NB;
        mx = fmax(mx, fabs(ws[outs[((x * C::NB + b) * C::NA + x) * C::NB + b]]));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) a.Q[i] = sqrt(mx);
      __syncwarp();
    }
  }
}

// Raw integrals of listed quartets of this class (every primitive quartet),
// written with per-item strides so the caller receives them in the shell
// order it asked for.
template <class C, typename R>
__global__ void __launch_bounds__(64) k_eval(const EvalArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int4 q = a.quartets[i];
  if (q.z != a.cls) return;
  const PairRec bra = a.pairs[q.x], ket = a.pairs[q.y];
  R out[C::NOUT];
  contracted_quartet<C, R>(bra, a.prims, ket, a.prims, a.boys, a.boysf, a.kernel, a.omega2,
                           ds{a.omega2_hi, a.omega2_lo}, PrimRange{0.f, 3.0e38f}, out);
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
template <class C, typename R>
void launch_build_K_t(const BuildArgs& a, int grid, cudaStream_t s) {
  if constexpr (C::COOP) {
    const size_t sm = CoopLayout<C, R>::bytes();
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_build_K_coop<C, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      attr = true;
    }
    k_build_K_coop<C, R><<<grid, kThreadsCoop, sm, s>>>(a);
  } else if constexpr (C::SPLIT) {
    const size_t sm = SplitLayout<C, R>::bytes();
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_build_K_split<C, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      attr = true;
    }
    k_build_K_split<C, R><<<grid, SplitShape<C, R>::THREADS, sm, s>>>(a);
  } else {
    k_build_K<C, R><<<grid, kThreadsK, 0, s>>>(a);
  }
}

template <class C>
void launch_build_K(const BuildArgs& a, int fp32, int grid, cudaStream_t s) {
  if (fp32)
    launch_build_K_t<C, float>(a, grid, s);
  else
    launch_build_K_t<C, double>(a, grid, s);
}

template <class C, typename R>
int occupancy_build_K_t() {
  int nb = 0;
  if constexpr (C::COOP) {
    const size_t sm = CoopLayout<C, R>::bytes();
    cudaFuncSetAttribute(k_build_K_coop<C, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_build_K_coop<C, R>, kThreadsCoop, sm);
  } else if constexpr (C::SPLIT) {
    const size_t sm = SplitLayout<C, R>::bytes();
    cudaFuncSetAttribute(k_build_K_split<C, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_build_K_split<C, R>, SplitShape<C, R>::THREADS, sm);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_build_K<C, R>, kThreadsK, 0);
  }
  return nb < 1 ? 1 : nb;
}

template <class C>
int occupancy_build_K(int fp32) {
  return fp32 ? occupancy_build_K_t<C, float>() : occupancy_build_K_t<C, double>();
}

template <class C>
void launch_schwarz(const SchwarzArgs& a, cudaStream_t s) {
  if (a.n_pairs <= 0) return;
  if constexpr (C::SPLIT || C::COOP) {
    const size_t sm = SchwarzWarpLayout<C>::bytes();
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_schwarz_warp<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      attr = true;
    }
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long need = (a.n_pairs + kSchwarzWarps - 1) / kSchwarzWarps;
    const int grid = (int)std::min<long long>(need, 8LL * nsm);
    k_schwarz_warp<C><<<grid, 32 * kSchwarzWarps, sm, s>>>(a);
  } else {
    k_schwarz<C><<<(a.n_pairs + 63) / 64, 64, 0, s>>>(a);
  }
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
