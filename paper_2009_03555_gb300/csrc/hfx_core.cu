// hfx_core.cu -- C ABI, setup pipeline and the small kernels of the HFX
// library (see include/hfx.h for the contract of every entry point).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_reduce.cuh>
#include <cub/device/device_scan.cuh>

#include "eri_kernels.cuh"
#include "generated/class_dispatch.h"
#include "generated/class_table.h"
#include "hfx.h"

using namespace hfx;

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

static hfx_status fail(hfx_status s, const std::string& m) {
  g_err = m;
  return s;
}

// Shared with the other translation units of the library.
void hfx_set_last_error(const std::string& m) { g_err = m; }

#define HFX_CK(x)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (x);                                                                  \
    if (e_ != cudaSuccess) {                                                               \
      if (e_ == cudaErrorMemoryAllocation) return fail(HFX_ERR_OOM, std::string(#x) + ": out of device memory"); \
      return fail(HFX_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_));         \
    }                                                                                      \
  } while (0)

template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  cudaError_t alloc(size_t count) {
    release();
    n = count;
    return cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
  }
};

static inline int ncart(int l) { return (l + 1) * (l + 2) / 2; }
// Primitive pairs whose bound estimate is below this are dropped when pairs are
// built (far below any quartet threshold; keeps FP32 bound products finite).
static constexpr double kPairDropBound = 1e-24;
static inline int pair_class_of(int la, int lb) { return la * (la + 1) / 2 + lb; }  // la >= lb
static inline int quartet_class_of(int cb, int ck) { return cb * (cb + 1) / 2 + ck; }  // cb >= ck
static inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------------------ handles
struct hfx_basis_s {
  int device = 0;
  int n_shells = 0, n_atoms = 0, nbf = 0, max_nprim = 0;
  // Home cell of a periodic basis (the first n_home_atoms atoms and their
  // n_home_shells shells; the images follow); a molecule is all home.
  int n_home_atoms = 0, n_home_shells = 0;
  std::vector<int> h_ext_home, h_ext_shift;  // per atom: home atom and lattice shift (n1, n2, n3)
  std::vector<double> h_atom_xyz;            // atom positions (bohr)
  std::vector<double> h_alpha;               // primitive exponents (shell S: h_poff[S] .. h_poff[S+1])
  std::vector<int> h_l, h_atom, h_np, h_poff, h_loc, h_atom_nf;
  std::vector<long long> h_sh_foff, h_atom_foff;
  DBuf<double> sh_xyz, alpha, coef, boys;
  DBuf<float> boysf;
  DBuf<int> sh_l, sh_atom, sh_poff, sh_loc, atom_nf;
};


// A build plan: the systems of one build (a single hfx_quartets, or the members
// of a batch), their device table, the per-class work-queue batches tagged with
// system ids, per-class launch shapes, counters and timing events.
struct Plan {
  int n = 0;
  int n_sm = 0;
  hfx_opts opts{};
  const double* boys = nullptr;
  const float* boysf = nullptr;
  SysArgs* h_sys = nullptr;  // pinned host copy (P and K filled per build)
  DBuf<SysArgs> d_sys;
  DBuf<double*> d_pmax;      // per-system Pmax tables
  const Desc* descp[HFX_NCLASS] = {};
  DBuf<Desc> desc_own[HFX_NCLASS];
  int n_desc[HFX_NCLASS] = {0};
  int n_block[HFX_NCLASS] = {0};
  int grid[2][HFX_NCLASS] = {{0}};  // persistent grid per (precision, class); 0 = occupancy x SMs
  int shard_rank = 0, shard_n = 1;   // batches i with i % shard_n == shard_rank (sharded builds)
  long long max_values = 0, max_ns2 = 0;
  int max_blocks = 0;
  DBuf<int> counters;                // 2 x HFX_NCLASS
  DBuf<unsigned long long> n_done;   // 2 x 2 x HFX_NCLASS
  DBuf<double> energy;               // per system
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t sys_copied = nullptr;  // the pinned table may be rewritten once this completed
  cudaEvent_t evk[2][HFX_NCLASS][2] = {};
  bool ran[2][HFX_NCLASS] = {};
  // CUDA graph of a whole build (batches)
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t side[HFX_NCLASS] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[HFX_NCLASS] = {};
  ~Plan() {
    if (h_sys) cudaFreeHost(h_sys);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (sys_copied) cudaEventDestroy(sys_copied);
    for (auto& p : evk)
      for (auto& c : p)
        for (auto& e : c)
          if (e) cudaEventDestroy(e);
    if (gexec) cudaGraphExecDestroy(gexec);
    for (auto& st : side)
      if (st) cudaStreamDestroy(st);
    if (fork_ev) cudaEventDestroy(fork_ev);
    for (auto& e : join_ev)
      if (e) cudaEventDestroy(e);
  }
};

struct hfx_quartets_s {
  hfx_basis* basis = nullptr;
  hfx_opts opts{};
  int n_sm = 0;
  // pattern
  int n_atoms = 0;
  long long n_values = 0;
  int n_blocks = 0;
  DBuf<long long> blk_off;                 // n_atoms x n_atoms
  DBuf<int> blk_x, blk_y;                  // block list
  DBuf<long long> blk_val_off;
  // pairs per class
  long long n_pairs[6] = {0};
  DBuf<PairRec> pairs[6];
  DBuf<PrimPair> prims[6];
  long long n_prim_pairs = 0;
  long long n_pairs_distance = 0;          // shell pairs kept by the distance screening (all pairs if off)
  // batches per quartet class
  DBuf<Desc> desc[HFX_NCLASS];
  int n_desc[HFX_NCLASS] = {0};
  long long n_quartets[HFX_NCLASS] = {0};
  // per-build buffers
  DBuf<double> pmax;                       // n_shells x n_shells
  DBuf<double> scratch;                    // energy accumulator
  DBuf<double> delta_K;                    // K of a density difference (hfx_build_K_delta)
  // spherical-harmonic layout (opts.spherical): the caller's P and K hold
  // 2l+1 real solid harmonics per shell; the build runs on Cartesian copies
  long long n_values_ext = 0;              // values of the caller's arrays
  DBuf<long long> blk_val_off_sph;         // block offsets in the spherical layout
  DBuf<int> atom_nf_sph;
  DBuf<long long> afoff_cart, afoff_sph;   // first function of each atom in each layout
  DBuf<int4> fmap_cart, fmap_sph;          // per function: (other layout's shell offset in the atom, l, component)
  DBuf<double> P_cart, K_cart;
  std::vector<long long> h_afoff_sph;
  long long nbf_sph = 0;
  float ms_setup = 0.f;
  float ms_setup_phase[4] = {0.f, 0.f, 0.f, 0.f};
  SysArgs h_sys{};  // this system's entry of a build table (P, K unset)
  Plan plan;        // single-system build plan
};

// ------------------------------------------------------------------ kernels
// Boys Taylor tables: for top order L = 0..8 and T_k = k/16, the coefficients
// F_{L+j}(T_k) / j!, j = 0..6, and exp(-T_k).  F_m by the power series
// F_m(T) = exp(-T) sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)) (all terms positive).
__global__ void k_boys_table(double* tab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kBoysNL * kBoysNT * kBoysCols) return;
  const int col = i % kBoysCols, it = (i / kBoysCols) % kBoysNT, L = i / (kBoysCols * kBoysNT);
  const double T = it * kBoysStep;
  if (col == kBoysCols - 1) {
    tab[i] = exp(-T);
    return;
  }
  const int m = L + col;
  double term = 1.0 / (2 * m + 1), sum = term;
  for (int k = 1; k < 2000; ++k) {
    term *= 2.0 * T / (2 * m + 2 * k + 1);
    sum += term;
    if (term < 1e-18 * sum) break;
  }
  double fact = 1.0;
  for (int j = 2; j <= col; ++j) fact *= j;
  tab[i] = exp(-T) * sum / fact;
}

// Double-single copy of the Boys tables (hi = fl(v), lo = fl(v - hi)).
__global__ void k_boys_split(const double* tab, float* tabf, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float h = (float)tab[i];
  tabf[2 * i] = h;
  tabf[2 * i + 1] = (float)(tab[i] - (double)h);
}

// F_0..F_L of the device evaluators at given arguments (diagnostics, tests).
template <int L>
__global__ void k_boys_eval(const double* tab, const float* tabf, int ds_path, int n, const double* T,
                            double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (ds_path) {
    ds F[L + 1];
    boys_ds<L>(tabf, ds_from_double(T[i]), F);
    for (int m = 0; m <= L; ++m) out[(size_t)i * (L + 1) + m] = (double)F[m].hi + (double)F[m].lo;
  } else {
    double F[L + 1];
    boys_fp64<L, 2>(tab, T[i], F);
    for (int m = 0; m <= L; ++m) out[(size_t)i * (L + 1) + m] = F[m];
  }
}

// Contraction coefficients: axial primitive normalisation
// (2a/pi)^{3/4} (4a)^{l/2} / sqrt((2l-1)!!), then unit self-overlap of the
// contracted x^l component.
__global__ void k_normalize(int ns, const int* l, const int* poff, const double* alpha, double* coef) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  const int L = l[s], p0 = poff[s], p1 = poff[s + 1];
  const double df = (L == 2) ? 3.0 : 1.0;
  for (int k = p0; k < p1; ++k) {
    const double a = alpha[k];
    coef[k] *= pow(2.0 * a / M_PI, 0.75) * pow(4.0 * a, 0.5 * L) / sqrt(df);
  }
  double S = 0.0;
  for (int k = p0; k < p1; ++k)
    for (int m = p0; m < p1; ++m) {
      const double g = alpha[k] + alpha[m];
      S += coef[k] * coef[m] * df / pow(2.0 * g, L) * pow(M_PI / g, 1.5);
    }
  const double sc = 1.0 / sqrt(S);
  for (int k = p0; k < p1; ++k) coef[k] *= sc;
}

// Shell-pair records (Gaussian product theorem) for a list of oriented pairs
// (l_A >= l_B).  Every primitive pair gets the estimate
// bound = |c_a c_b K_ab| sqrt(2 pi^{5/2} / (p^2 sqrt(2p))) (the square root of
// the s-type self-repulsion of the primitive product); pairs below `cutoff`
// are dropped and the rest are sorted by descending bound, so the ERI kernels
// can stop a primitive loop at the first negligible primitive quartet.
__global__ void k_pair_build(int n, const int2* list, const double* xyz, const int* l, const int* poff,
                             const double* alpha, const double* coef, int stride, double cutoff, PairRec* out,
                             PrimPair* prims, int* pclass) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int A = list[i].x, B = list[i].y;
  PairRec r;
  r.A = A;
  r.B = B;
  r.poff = (int)((long long)i * stride);
  double Ax = xyz[3 * A], Ay = xyz[3 * A + 1], Az = xyz[3 * A + 2];
  double Bx = xyz[3 * B], By = xyz[3 * B + 1], Bz = xyz[3 * B + 2];
  r.AB[0] = Ax - Bx;
  r.AB[1] = Ay - By;
  r.AB[2] = Az - Bz;
  const double ab2 = r.AB[0] * r.AB[0] + r.AB[1] * r.AB[1] + r.AB[2] * r.AB[2];
  PrimPair* dst = prims + (long long)i * stride;
  int cnt = 0;
  for (int ia = poff[A]; ia < poff[A + 1]; ++ia)
    for (int ib = poff[B]; ib < poff[B + 1]; ++ib) {
      const double a = alpha[ia], b = alpha[ib], p = a + b;
      const double kab = exp(-a * b / p * ab2);
      const double kp = coef[ia] * coef[ib] * kab / p;
      const double bound = fabs(kp) * sqrt(kTwoPi52 / sqrt(2.0 * p));
      if (!(bound >= cutoff)) continue;
      PrimPair q;
      q.p = p;
      q.kp = kp;
      q.oo2p = 0.5 / p;
      q.P[0] = (a * Ax + b * Bx) / p;
      q.P[1] = (a * Ay + b * By) / p;
      q.P[2] = (a * Az + b * Bz) / p;
      q.PA[0] = q.P[0] - Ax;
      q.PA[1] = q.P[1] - Ay;
      q.PA[2] = q.P[2] - Az;
      q.PAf[0] = (float)q.PA[0];
      q.PAf[1] = (float)q.PA[1];
      q.PAf[2] = (float)q.PA[2];
      q.oo2pf = (float)q.oo2p;
      q.pf = (float)p;
      q.plo = (float)(p - (double)q.pf);
      for (int x = 0; x < 3; ++x) {
        q.Phi[x] = (float)q.P[x];
        q.Plo[x] = (float)(q.P[x] - (double)q.Phi[x]);
      }
      q.kpf = (float)kp;
      q.bound = (float)bound;
      // insertion into the descending-bound order
      int j = cnt;
      while (j > 0 && dst[j - 1].bound < q.bound) {
        dst[j] = dst[j - 1];
        --j;
      }
      dst[j] = q;
      ++cnt;
    }
  r.pcnt = cnt;
  r.Q = 0.0;
  out[i] = r;
  const int la = l[A], lb = l[B];
  pclass[i] = la * (la + 1) / 2 + lb;
}

__global__ void k_qmax(int n, const double* Q, unsigned long long* qmax_bits) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double v = (i < n) ? Q[i] : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(qmax_bits, (unsigned long long)__double_as_longlong(v));
}

__global__ void k_sort_keys(int n, const double* Q, const int* pclass, unsigned long long* qkey, int* idx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  qkey[i] = ~(unsigned long long)__double_as_longlong(Q[i]);  // descending Q (Q >= 0)
  idx[i] = i;
}

__global__ void k_gather_class(int n, const int* idx, const int* pclass, int* ckey) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) ckey[i] = pclass[idx[i]];
}

__global__ void k_class_counts(int n, const int* sorted_idx, const int* pclass, const double* Q, int screen,
                               double tau, const unsigned long long* qmax_bits, int* count_all, int* count_kept) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int i = sorted_idx[j];
  const int c = pclass[i];
  atomicAdd(&count_all[c], 1);
  const double qmax = __longlong_as_double((long long)*qmax_bits);
  if (!screen || Q[i] * qmax > tau) atomicAdd(&count_kept[c], 1);
}

__global__ void k_gather_pairs(int n, const int* sorted_idx, const PairRec* pairs, const PrimPair* prims,
                               const double* Q, int stride, PairRec* out, PrimPair* out_prims) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int i = sorted_idx[j];
  PairRec r = pairs[i];
  r.Q = Q[i];
  const long long src = r.poff;
  r.poff = (int)((long long)j * stride);
  for (int k = 0; k < r.pcnt; ++k) out_prims[(long long)j * stride + k] = prims[src + k];
  out[j] = r;
}

// Work-queue batches for one quartet class: bra pair j (class cb) against the
// ket pairs of class ck whose bound passes the Schwarz test.  Ket lists are
// sorted by descending Q, so the survivors of Q_bra Q_ket > tau are a prefix;
// same class: canonical kets start at the bra's own rank.
__global__ void k_desc_count(int nb, const PairRec* bra, int nk, const PairRec* ket, int same, int screen,
                             double tau, int n_block, int* chunks, long long* nq) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  int k1 = nk;
  if (screen) {
    const double qb = bra[j].Q;
    const double thr = (qb > 0.0) ? (tau / qb) * (1.0 - 1e-12) : INFINITY;
    int lo = 0, hi = nk;  // first index with Q <= thr
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (ket[mid].Q > thr) lo = mid + 1;
      else hi = mid;
    }
    k1 = lo;
  }
  const int k0 = same ? j : 0;
  const int cnt = k1 > k0 ? k1 - k0 : 0;
  chunks[j] = (cnt + n_block - 1) / n_block;
  nq[j] = cnt;
}

__global__ void k_desc_fill(int nb, int nk, const PairRec* bra, const PairRec* ket, int same, int screen,
                            double tau, int n_block, const int* off, Desc* desc, int sys) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  int k1 = nk;
  if (screen) {
    const double qb = bra[j].Q;
    const double thr = (qb > 0.0) ? (tau / qb) * (1.0 - 1e-12) : INFINITY;
    int lo = 0, hi = nk;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (ket[mid].Q > thr) lo = mid + 1;
      else hi = mid;
    }
    k1 = lo;
  }
  const int k0 = same ? j : 0;
  int o = off[j];
  for (int k = k0; k < k1; k += n_block) {
    Desc d;
    d.bra = j;
    d.k0 = k;
    d.k1 = min(k + n_block, k1);
    d.sys = sys;
    desc[o++] = d;
  }
}

// sum_i P_i K_i (FP64), block reduction then one atomicAdd per block.  `vec`:
// both arrays 16-byte aligned, read as double2.
__global__ void k_dot(long long n, const double* __restrict__ P, const double* __restrict__ K, int vec,
                      double* out) {
  double s = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (vec) {
    const long long n2 = n / 2;
    const double2* P2 = reinterpret_cast<const double2*>(P);
    const double2* K2 = reinterpret_cast<const double2*>(K);
    for (long long j = i; j < n2; j += stride) {
      const double2 p = __ldg(P2 + j), k = __ldg(K2 + j);
      s = fma(p.x, k.x, fma(p.y, k.y, s));
    }
    if (i == 0 && (n & 1)) s = fma(P[n - 1], K[n - 1], s);
  } else {
    for (long long j = i; j < n; j += stride) s = fma(__ldg(P + j), __ldg(K + j), s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? ws[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(out, s);
  }
}

// y += x over n values (incremental exchange builds)
__global__ void k_axpy(long long n, const double* __restrict__ x, double* __restrict__ y) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) y[i] += x[i];
}

__global__ void k_pack(int n_blocks, const int* bx, const int* by, const long long* boff, const long long* afoff,
                       const int* atom_nf, long long nbf, double* dense, double* val, int unpack) {
  const int b = blockIdx.x;
  if (b >= n_blocks) return;
  const int X = bx[b], Y = by[b];
  const int nX = atom_nf[X], nY = atom_nf[Y];
  for (int e = threadIdx.x; e < nX * nY; e += blockDim.x) {
    const int r = e / nY, c = e % nY;
    const long long di = (afoff[X] + r) * nbf + afoff[Y] + c;
    if (unpack)
      dense[di] = val[boff[b] + e];
    else
      val[boff[b] + e] = dense[di];
  }
}


// Real solid harmonics of a d shell from its Cartesian components (xx, xy, xz,
// yy, yz, zz; normalisation of the x^2 component), in the order
// xy, yz, z^2, xz, x^2 - y^2:
//   sqrt3 xy, sqrt3 yz, (2 zz - xx - yy)/2, sqrt3 xz, sqrt3/2 (xx - yy);
// with the Cartesian normalisation every one of them has unit norm.  s and p
// shells are unchanged (the p order x, y, z is kept).
__device__ __forceinline__ double sph_coef(int l, int m, int c) {
  if (l < 2) return m == c ? 1.0 : 0.0;
  const double r3 = 1.7320508075688772935, h3 = 0.86602540378443864676;
  switch (m) {
    case 0: return c == 1 ? r3 : 0.0;
    case 1: return c == 4 ? r3 : 0.0;
    case 2: return c == 5 ? 1.0 : ((c == 0 || c == 3) ? -0.5 : 0.0);
    case 3: return c == 2 ? r3 : 0.0;
    default: return c == 0 ? h3 : (c == 3 ? -h3 : 0.0);
  }
}

// One layout change of every pattern block: to_sph: out = T in T^T (Cartesian
// to spherical, K); otherwise out = T^T in T (spherical to Cartesian, P).
// map_out[afoff_out[X] + r] = (offset of r's shell in atom X's input layout,
// l, component of r).
__global__ void k_sph_transform(int n_blocks, const int* __restrict__ bx, const int* __restrict__ by,
                                const long long* __restrict__ off_in, const long long* __restrict__ off_out,
                                const long long* __restrict__ afoff_out, const int* __restrict__ nf_in,
                                const int* __restrict__ nf_out, const int4* __restrict__ map_out, int to_sph,
                                const double* __restrict__ in, double* __restrict__ out) {
  const int b = blockIdx.x;
  if (b >= n_blocks) return;
  const int X = bx[b], Y = by[b];
  const int nXo = nf_out[X], nYo = nf_out[Y], nYi = nf_in[Y];
  for (int e = threadIdx.x; e < nXo * nYo; e += blockDim.x) {
    const int r = e / nYo, c = e % nYo;
    const int4 mr = map_out[afoff_out[X] + r], mc = map_out[afoff_out[Y] + c];
    const int nr = to_sph ? (mr.y + 1) * (mr.y + 2) / 2 : 2 * mr.y + 1;  // input components of the shells
    const int nc = to_sph ? (mc.y + 1) * (mc.y + 2) / 2 : 2 * mc.y + 1;
    double acc = 0.0;
    for (int i = 0; i < nr; ++i) {
      const double wr = to_sph ? sph_coef(mr.y, mr.z, i) : sph_coef(mr.y, i, mr.z);
      if (wr == 0.0) continue;
      const double* row = in + off_in[b] + (long long)(mr.x + i) * nYi + mc.x;
      for (int j = 0; j < nc; ++j) {
        const double wc = to_sph ? sph_coef(mc.y, mc.z, j) : sph_coef(mc.y, j, mc.z);
        acc = fma(wr * wc, row[j], acc);
      }
    }
    out[off_out[b] + e] = acc;
  }
}

// ---------------------------------------------------------------- batched
// Small kernels of a build over every system of a batch at once: 2-D grids,
// blockIdx.y = system, reading the system table.
__global__ void k_zero_b(const SysArgs* sys, int per_block) {
  const SysArgs& S = sys[blockIdx.y];
  const long long base = (long long)blockIdx.x * per_block;
  for (long long i = base + threadIdx.x; i < base + per_block && i < S.n_values; i += blockDim.x) S.K[i] = 0.0;
}

// Pmax per shell pair, max |P_ij| over i in I, j in J (Sec. 2, density
// screening; from the current P, every build).
__global__ void k_pmax_b(const SysArgs* sys, double* const* pmax) {
  const SysArgs& S = sys[blockIdx.y];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int ns = S.ns;
  if (t >= (long long)ns * ns) return;
  const int I = (int)(t / ns), J = (int)(t % ns);
  const int na = S.n_atoms;
  const long long o = S.blk_off[S.sh_atom[I] * na + S.sh_atom[J]];
  double mx = 0.0;
  if (o >= 0) {
    const int nI = (S.sh_l[I] + 1) * (S.sh_l[I] + 2) / 2, nJ = (S.sh_l[J] + 1) * (S.sh_l[J] + 2) / 2;
    const int nfJ = S.atom_nf[S.sh_atom[J]];
    for (int a = 0; a < nI; ++a)
      for (int b = 0; b < nJ; ++b)
        mx = fmax(mx, fabs(S.P[o + (long long)(S.sh_loc[I] + a) * nfJ + S.sh_loc[J] + b]));
  }
  pmax[blockIdx.y][t] = mx;
}

// K = K' + K'^T over each system's pattern (the scatter adds four of the
// eight permutations of a canonical quartet; the other four are transposes).
// Rows of image atoms of a periodic cell (atoms from n_home_atoms on) are set
// to zero: they only received the partial sums of the home-cell quartets.
__global__ void k_sym_b(const SysArgs* sys) {
  const SysArgs& S = sys[blockIdx.y];
  const int b = blockIdx.x;
  if (b >= S.n_blocks) return;
  const int X = S.blk_x[b], Y = S.blk_y[b];
  if (X > Y) return;
  const int nX = S.atom_nf[X], nY = S.atom_nf[Y];
  const long long oXY = S.blk_val_off[b];
  double* K = S.K;
  const double keepX = X < S.n_home_atoms ? 1.0 : 0.0, keepY = Y < S.n_home_atoms ? 1.0 : 0.0;
  if (X == Y) {
    for (int e = threadIdx.x; e < nX * nX; e += blockDim.x) {
      const int r = e / nX, c = e % nX;
      if (r < c) {
        const double v = keepX * (K[oXY + r * nX + c] + K[oXY + c * nX + r]);
        K[oXY + r * nX + c] = v;
        K[oXY + c * nX + r] = v;
      } else if (r == c) {
        K[oXY + r * nX + r] *= 2.0 * keepX;
      }
    }
  } else {
    const long long oYX = S.blk_off[Y * S.n_atoms + X];
    for (int e = threadIdx.x; e < nX * nY; e += blockDim.x) {
      const int r = e / nY, c = e % nY;
      const double v = K[oXY + r * nY + c] + K[oYX + c * nX + r];
      K[oXY + r * nY + c] = keepX * v;
      K[oYX + c * nX + r] = keepY * v;
    }
  }
}

// E_x[system] += -1/2 sum P_i K_i over a slice (E_x zeroed before).
__global__ void k_dot_b(const SysArgs* sys, int per_block, double* E) {
  const SysArgs& S = sys[blockIdx.y];
  const long long base = (long long)blockIdx.x * per_block;
  double s = 0.0;
  for (long long i = base + threadIdx.x; i < base + per_block && i < S.n_values; i += blockDim.x)
    s = fma(__ldg(S.P + i), __ldg(S.K + i), s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    if (t != 0.0) atomicAdd(E + blockIdx.y, -0.5 * t);
  }
}

// ------------------------------------------------------------------ helpers
static int device_sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

template <typename T>
static cudaError_t upload(DBuf<T>& b, const std::vector<T>& v, cudaStream_t s) {
  cudaError_t e = b.alloc(v.size());
  if (e != cudaSuccess) return e;
  if (v.empty()) return cudaSuccess;
  return cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}


// ---------------------------------------------------------------- plans
static void fill_sys(hfx_quartets_s* q) {
  hfx_basis* b = q->basis;
  SysArgs& S = q->h_sys;
  for (int c = 0; c < 6; ++c) {
    S.pairs[c] = q->pairs[c].p;
    S.prims[c] = q->prims[c].p;
    S.n_pairs[c] = (int)q->n_pairs[c];
    S.n_prims[c] = (long long)q->prims[c].n;
  }
  S.pmax = q->pmax.p;
  S.P = nullptr;
  S.K = nullptr;
  S.blk_off = q->blk_off.p;
  S.sh_atom = b->sh_atom.p;
  S.sh_loc = b->sh_loc.p;
  S.atom_nf = b->atom_nf.p;
  S.sh_l = b->sh_l.p;
  S.blk_x = q->blk_x.p;
  S.blk_y = q->blk_y.p;
  S.blk_val_off = q->blk_val_off.p;
  S.n_values = q->n_values;
  S.n_blocks = q->n_blocks;
  S.ns = b->n_shells;
  S.n_atoms = q->n_atoms;
  S.n_home_atoms = b->n_home_atoms;
  S.n_home_shells = b->n_home_shells;
}

static hfx_status plan_alloc(Plan& pl, const std::vector<hfx_quartets_s*>& m, int n_sm) {
  pl.n = (int)m.size();
  pl.n_sm = n_sm;
  pl.opts = m[0]->opts;
  pl.boys = m[0]->basis->boys.p;
  pl.boysf = m[0]->basis->boysf.p;
  HFX_CK(cudaMallocHost(&pl.h_sys, sizeof(SysArgs) * pl.n));
  HFX_CK(pl.d_sys.alloc(pl.n));
  std::vector<double*> pm(pl.n);
  for (int i = 0; i < pl.n; ++i) {
    pl.h_sys[i] = m[i]->h_sys;
    pm[i] = m[i]->pmax.p;
    pl.max_values = std::max(pl.max_values, m[i]->n_values);
    pl.max_ns2 = std::max(pl.max_ns2, (long long)m[i]->basis->n_shells * m[i]->basis->n_shells);
    pl.max_blocks = std::max(pl.max_blocks, m[i]->n_blocks);
  }
  HFX_CK(upload(pl.d_pmax, pm, 0));
  HFX_CK(pl.counters.alloc(2 * HFX_NCLASS));
  HFX_CK(pl.n_done.alloc(4 * HFX_NCLASS));
  HFX_CK(cudaMemset(pl.n_done.p, 0, 4 * HFX_NCLASS * sizeof(unsigned long long)));
  HFX_CK(pl.energy.alloc(pl.n));
  HFX_CK(cudaEventCreate(&pl.ev0));
  HFX_CK(cudaEventCreate(&pl.ev1));
  HFX_CK(cudaEventCreateWithFlags(&pl.sys_copied, cudaEventDisableTiming));
  for (auto& p : pl.evk)
    for (auto& c : p)
      for (auto& e : c) HFX_CK(cudaEventCreate(&e));
  return HFX_OK;
}

// Work-queue batches of quartet class `cls` for one system: returns the count;
// with `out`, also writes them (system id `sys`).
static hfx_status class_desc(hfx_quartets_s* q, int cls, int n_block, Desc* out, int sys, cudaStream_t s,
                             long long* n_desc_out, long long* n_quartets_out) {
  const int cb = hfx_class_table[cls][0], ck = hfx_class_table[cls][1];
  const int nb = (int)q->n_pairs[cb], nk = (int)q->n_pairs[ck];
  *n_desc_out = 0;
  if (n_quartets_out) *n_quartets_out = 0;
  if (nb == 0 || nk == 0) return HFX_OK;
  const hfx_opts& o = q->opts;
  DBuf<int> chunks, off;
  DBuf<long long> nq, nq_sum;
  HFX_CK(chunks.alloc(nb));
  HFX_CK(off.alloc(nb));
  HFX_CK(nq.alloc(nb));
  HFX_CK(nq_sum.alloc(1));
  k_desc_count<<<blocks_for(nb, 128), 128, 0, s>>>(nb, q->pairs[cb].p, nk, q->pairs[ck].p, cb == ck, o.screen, o.tau,
                                                   n_block, chunks.p, nq.p);
  size_t t1b = 0, t2b = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, t1b, chunks.p, off.p, nb, s);
  cub::DeviceReduce::Sum(nullptr, t2b, nq.p, nq_sum.p, nb, s);
  DBuf<unsigned char> tmp;
  HFX_CK(tmp.alloc(std::max(t1b, t2b)));
  t1b = tmp.n;
  HFX_CK(cub::DeviceScan::ExclusiveSum(tmp.p, t1b, chunks.p, off.p, nb, s));
  t2b = tmp.n;
  HFX_CK(cub::DeviceReduce::Sum(tmp.p, t2b, nq.p, nq_sum.p, nb, s));
  int last_off = 0, last_chunks = 0;
  long long total_q = 0;
  HFX_CK(cudaMemcpyAsync(&last_off, off.p + nb - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  HFX_CK(cudaMemcpyAsync(&last_chunks, chunks.p + nb - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  HFX_CK(cudaMemcpyAsync(&total_q, nq_sum.p, sizeof(long long), cudaMemcpyDeviceToHost, s));
  HFX_CK(cudaStreamSynchronize(s));
  *n_desc_out = (long long)last_off + last_chunks;
  if (n_quartets_out) *n_quartets_out = total_q;
  if (out && *n_desc_out > 0)
    k_desc_fill<<<blocks_for(nb, 128), 128, 0, s>>>(nb, nk, q->pairs[cb].p, q->pairs[ck].p, cb == ck, o.screen, o.tau,
                                                    n_block, off.p, out, sys);
  HFX_CK(cudaGetLastError());
  HFX_CK(cudaStreamSynchronize(s));
  return HFX_OK;
}

// The batches of class `cls` for every system of a plan, concatenated.
static hfx_status plan_class_desc(Plan& pl, const std::vector<hfx_quartets_s*>& m, int cls, int n_block,
                                  cudaStream_t s) {
  std::vector<long long> cnt(m.size());
  long long tot = 0;
  for (size_t i = 0; i < m.size(); ++i) {
    hfx_status st = class_desc(m[i], cls, n_block, nullptr, (int)i, s, &cnt[i], nullptr);
    if (st != HFX_OK) return st;
    tot += cnt[i];
  }
  if (tot > (1LL << 31) - 1) return fail(HFX_ERR_UNSUPPORTED, "too many work-queue batches; raise n_block");
  HFX_CK(pl.desc_own[cls].alloc(tot));
  long long o = 0;
  for (size_t i = 0; i < m.size(); ++i) {
    long long c = 0;
    hfx_status st = class_desc(m[i], cls, n_block, pl.desc_own[cls].p + o, (int)i, s, &c, nullptr);
    if (st != HFX_OK) return st;
    o += c;
  }
  pl.descp[cls] = pl.desc_own[cls].p;
  pl.n_desc[cls] = (int)tot;
  pl.n_block[cls] = n_block;
  return HFX_OK;
}

static int plan_grid(Plan& pl, int fp32, int cls) {
  int g = pl.grid[fp32][cls];
  if (g <= 0) g = pl.grid[fp32][cls] = kClassOps[cls].occupancy_K(fp32) * pl.n_sm;
  return g;
}

static BuildArgs plan_args(Plan& pl, int cls) {
  const hfx_opts& o = pl.opts;
  BuildArgs a;
  a.sys = pl.d_sys.p;
  a.desc = pl.descp[cls];
  // a sharded build takes every shard_n-th batch from shard_rank on
  const int nd = pl.n_desc[cls];
  a.desc_first = pl.shard_rank;
  a.desc_stride = pl.shard_n;
  a.n_desc = nd > pl.shard_rank ? (nd - pl.shard_rank + pl.shard_n - 1) / pl.shard_n : 0;
  a.n_sys = pl.n;
  a.bra_class = hfx_class_table[cls][0];
  a.ket_class = hfx_class_table[cls][1];
  a.same_class = a.bra_class == a.ket_class;
  a.boys = pl.boys;
  a.boysf = pl.boysf;
  a.kernel = o.kernel;
  a.omega2 = o.omega * o.omega;
  a.omega2_hi = (float)a.omega2;
  a.omega2_lo = (float)(a.omega2 - (double)a.omega2_hi);
  a.screen = o.screen;
  a.tau = o.tau;
  a.dscreen = o.density_screen;
  a.eps = o.eps;
  a.eps_prim = (float)o.prim_cutoff;
  a.prim_dscreen = o.prim_density_screen;
  a.promote = o.fp64_promote_bound;
  a.promote_prims = o.promote_prims;
  a.route = 0;
  a.counter = nullptr;
  a.n_done = nullptr;
  return a;
}

// Launches of the class kernels of one build (both precision passes of the
// mixed path when FP64 promotion is on).  `fork`: each class on its own
// stream branch (graph capture); `events`: per-launch timing.
static hfx_status plan_classes(Plan& pl, cudaStream_t s, bool fork, bool events) {
  const hfx_opts& o = pl.opts;
  const bool mixed = o.precision == HFX_PREC_MIXED;
  const bool promote_any = mixed && std::isfinite(o.fp64_promote_bound);
  if (fork) HFX_CK(cudaEventRecord(pl.fork_ev, s));
  for (int cls = 0; cls < HFX_NCLASS; ++cls) {
    for (int pass = 0; pass < 2; ++pass) pl.ran[pass][cls] = false;
    if (pl.n_desc[cls] == 0) continue;
    // promotion applies to classes of total angular momentum >= promote_min_l
    const bool promote = promote_any && hfx_class_table[cls][6] >= o.promote_min_l;
    const int passes = promote ? 2 : 1;
    cudaStream_t cs = s;
    if (fork) {
      cs = pl.side[cls];
      HFX_CK(cudaStreamWaitEvent(cs, pl.fork_ev, 0));
    }
    BuildArgs a = plan_args(pl, cls);
    for (int pass = 0; pass < passes; ++pass) {
      const int fp32 = mixed && pass == 0;
      a.route = promote ? (pass == 0 ? 1 : 2) : 0;
      a.counter = pl.counters.p + pass * HFX_NCLASS + cls;
      a.n_done = pl.n_done.p + 2 * (pass * HFX_NCLASS + cls);
      const int g = plan_grid(pl, fp32, cls);
      if (events) HFX_CK(cudaEventRecord(pl.evk[pass][cls][0], cs));
      kClassOps[cls].launch_K(a, fp32, g, cs);
#ifdef HFX_CHECKED
      {  // checked builds: finish each class kernel before the next (outside capture)
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(cs, &cap);
        if (cap == cudaStreamCaptureStatusNone) {
          const cudaError_t e = cudaStreamSynchronize(cs);
          if (e != cudaSuccess)
            return fail(HFX_ERR_CUDA, "class " + std::to_string(cls) + " pass " + std::to_string(pass) + ": " +
                                          cudaGetErrorString(e));
        }
      }
#endif
      if (events) HFX_CK(cudaEventRecord(pl.evk[pass][cls][1], cs));
      pl.ran[pass][cls] = true;
    }
    if (fork) {
      HFX_CK(cudaEventRecord(pl.join_ev[cls], cs));
      HFX_CK(cudaStreamWaitEvent(s, pl.join_ev[cls], 0));
    }
  }
  HFX_CK(cudaGetLastError());
  return HFX_OK;
}

// One whole build of every system of the plan (Algorithm 4 per system):
// system table upload, zero K, Pmax, class kernels, symmetrisation, E_x.
static hfx_status plan_build(Plan& pl, cudaStream_t s, bool fork, bool events) {
  HFX_CK(cudaMemcpyAsync(pl.d_sys.p, pl.h_sys, sizeof(SysArgs) * pl.n, cudaMemcpyHostToDevice, s));
  HFX_CK(cudaEventRecord(pl.sys_copied, s));
  if (events) HFX_CK(cudaEventRecord(pl.ev0, s));
  const int zper = 8192;
  if (pl.max_values > 0)
    k_zero_b<<<dim3((unsigned)((pl.max_values + zper - 1) / zper), pl.n), 256, 0, s>>>(pl.d_sys.p, zper);
  if (pl.max_ns2 > 0)
    k_pmax_b<<<dim3((unsigned)((pl.max_ns2 + 255) / 256), pl.n), 256, 0, s>>>(pl.d_sys.p, pl.d_pmax.p);
  HFX_CK(cudaMemsetAsync(pl.counters.p, 0, 2 * HFX_NCLASS * sizeof(int), s));
  HFX_CK(cudaMemsetAsync(pl.n_done.p, 0, 4 * HFX_NCLASS * sizeof(unsigned long long), s));
  hfx_status st = plan_classes(pl, s, fork, events);
  if (st != HFX_OK) return st;
  if (pl.max_blocks > 0) k_sym_b<<<dim3(pl.max_blocks, pl.n), 128, 0, s>>>(pl.d_sys.p);
  HFX_CK(cudaMemsetAsync(pl.energy.p, 0, sizeof(double) * pl.n, s));
  const int dper = 8192;
  if (pl.max_values > 0)
    k_dot_b<<<dim3((unsigned)((pl.max_values + dper - 1) / dper), pl.n), 256, 0, s>>>(pl.d_sys.p, dper,
                                                                                       pl.energy.p);
  if (events) HFX_CK(cudaEventRecord(pl.ev1, s));
  HFX_CK(cudaGetLastError());
  return HFX_OK;
}

static void plan_stats(Plan& pl, hfx_stats* out) {
  unsigned long long done[4 * HFX_NCLASS];
  cudaMemcpy(done, pl.n_done.p, sizeof(done), cudaMemcpyDeviceToHost);
  for (int c = 0; c < HFX_NCLASS; ++c) {
    out->n_quartets_computed[c] = 0;
    for (int pass = 0; pass < 2; ++pass) {
      const unsigned long long* d = done + 2 * (pass * HFX_NCLASS + c);
      // with promotion per primitive quartet the FP32 pass sees every quartet
      // and the FP64 pass again those above the bound
      if (!(pl.opts.promote_prims && pass == 1)) out->n_quartets_computed[c] += (long long)d[0];
      out->n_quartets_pass[pass][c] = (long long)d[0];
      out->n_prim_quartets_pass[pass][c] = (long long)d[1];
      float ms = 0.f;
      if (pl.ran[pass][c] && cudaEventElapsedTime(&ms, pl.evk[pass][c][0], pl.evk[pass][c][1]) == cudaSuccess)
        out->ms_class_pass[pass][c] = ms;
    }
  }
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, pl.ev0, pl.ev1) == cudaSuccess) out->ms_last_build = ms;
  cudaGetLastError();
}

// ------------------------------------------------------------------ ABI
extern "C" {

const char* hfx_last_error(void) { return g_err.c_str(); }

hfx_status hfx_get_class_info(int cls, hfx_class_info* out) {
  if (cls < 0 || cls >= HFX_NCLASS || !out) return fail(HFX_ERR_INVALID_ARG, "class index out of range");
  const int* t = hfx_class_table[cls];
  out->bra_class = t[0];
  out->ket_class = t[1];
  out->la = t[2];
  out->lb = t[3];
  out->lc = t[4];
  out->ld = t[5];
  out->n_out = t[7];
  out->vrr_flops = t[8];
  out->hrr_flops = t[9];
  out->n_acc = t[10];
  out->kernel_kind = t[11];
  return HFX_OK;
}

hfx_status hfx_create_basis(const hfx_shell_desc* shells, int n_shells, const double* atom_xyz, int n_atoms,
                            void* stream, hfx_basis** out) {
  if (!out) return fail(HFX_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_shells <= 0 || n_atoms <= 0 || !shells || !atom_xyz)
    return fail(HFX_ERR_INVALID_ARG, "need at least one shell and one atom");
  cudaStream_t s = (cudaStream_t)stream;
  auto* b = new hfx_basis_s();
  cudaGetDevice(&b->device);
  b->n_shells = n_shells;
  b->n_atoms = n_atoms;
  std::vector<double> xyz(3 * (size_t)n_shells), alpha, coef;
  std::vector<int> poff(1, 0);
  b->h_atom_nf.assign(n_atoms, 0);
  int prev_atom = 0;
  for (int i = 0; i < n_shells; ++i) {
    const hfx_shell_desc& d = shells[i];
    if (d.l < 0 || d.l > kMaxL) {
      delete b;
      return fail(HFX_ERR_UNSUPPORTED, "shell " + std::to_string(i) + ": angular momentum must be 0, 1 or 2");
    }
    if (d.nprim < 1 || d.nprim > 16 || !d.alpha || !d.coef) {
      delete b;
      return fail(HFX_ERR_UNSUPPORTED, "shell " + std::to_string(i) + ": need 1..16 primitives");
    }
    if (d.atom < 0 || d.atom >= n_atoms || d.atom < prev_atom) {
      delete b;
      return fail(HFX_ERR_INVALID_ARG, "shells must be grouped by atom in increasing atom order");
    }
    prev_atom = d.atom;
    for (int k = 0; k < d.nprim; ++k) {
      if (!(d.alpha[k] > 0.0) || !std::isfinite(d.alpha[k]) || !std::isfinite(d.coef[k])) {
        delete b;
        return fail(HFX_ERR_INVALID_ARG, "shell " + std::to_string(i) + ": exponents must be positive and finite");
      }
      alpha.push_back(d.alpha[k]);
      coef.push_back(d.coef[k]);
    }
    poff.push_back((int)alpha.size());
    for (int x = 0; x < 3; ++x) xyz[3 * i + x] = atom_xyz[3 * d.atom + x];
    b->h_l.push_back(d.l);
    b->h_atom.push_back(d.atom);
    b->h_np.push_back(d.nprim);
    b->h_loc.push_back(b->h_atom_nf[d.atom]);
    b->h_atom_nf[d.atom] += ncart(d.l);
    b->max_nprim = std::max(b->max_nprim, d.nprim);
  }
  b->h_poff = poff;
  b->h_alpha = alpha;
  b->h_atom_foff.assign(n_atoms + 1, 0);
  for (int a = 0; a < n_atoms; ++a) b->h_atom_foff[a + 1] = b->h_atom_foff[a] + b->h_atom_nf[a];
  b->nbf = (int)b->h_atom_foff[n_atoms];
  b->h_sh_foff.resize(n_shells + 1);
  for (int i = 0; i < n_shells; ++i) b->h_sh_foff[i] = b->h_atom_foff[b->h_atom[i]] + b->h_loc[i];
  b->h_sh_foff[n_shells] = b->nbf;
  b->n_home_atoms = n_atoms;
  b->n_home_shells = n_shells;
  b->h_atom_xyz.assign(atom_xyz, atom_xyz + 3 * (size_t)n_atoms);
  b->h_ext_home.resize(n_atoms);
  for (int a = 0; a < n_atoms; ++a) b->h_ext_home[a] = a;
  b->h_ext_shift.assign(3 * (size_t)n_atoms, 0);
  cudaError_t e = cudaSuccess;
  if ((e = upload(b->sh_xyz, xyz, s)) != cudaSuccess || (e = upload(b->alpha, alpha, s)) != cudaSuccess ||
      (e = upload(b->coef, coef, s)) != cudaSuccess || (e = upload(b->sh_l, b->h_l, s)) != cudaSuccess ||
      (e = upload(b->sh_atom, b->h_atom, s)) != cudaSuccess || (e = upload(b->sh_poff, poff, s)) != cudaSuccess ||
      (e = upload(b->sh_loc, b->h_loc, s)) != cudaSuccess || (e = upload(b->atom_nf, b->h_atom_nf, s)) != cudaSuccess ||
      (e = b->boys.alloc((size_t)kBoysNL * kBoysNT * kBoysCols)) != cudaSuccess ||
      (e = b->boysf.alloc((size_t)2 * kBoysNL * kBoysNT * kBoysCols)) != cudaSuccess) {
    delete b;
    return fail(e == cudaErrorMemoryAllocation ? HFX_ERR_OOM : HFX_ERR_CUDA,
                std::string("hfx_create_basis: ") + cudaGetErrorString(e));
  }
  k_normalize<<<blocks_for(n_shells, 128), 128, 0, s>>>(n_shells, b->sh_l.p, b->sh_poff.p, b->alpha.p, b->coef.p);
  k_boys_table<<<blocks_for(kBoysNL * kBoysNT * kBoysCols, 128), 128, 0, s>>>(b->boys.p);
  k_boys_split<<<blocks_for(kBoysNL * kBoysNT * kBoysCols, 128), 128, 0, s>>>(b->boys.p, b->boysf.p,
                                                                               kBoysNL * kBoysNT * kBoysCols);
  e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    delete b;
    return fail(HFX_ERR_CUDA, std::string("hfx_create_basis: ") + cudaGetErrorString(e));
  }
  *out = b;
  return HFX_OK;
}

void hfx_destroy_basis(hfx_basis* b) { delete b; }

hfx_status hfx_create_basis_periodic(const hfx_shell_desc* shells, int n_shells, const double* atom_xyz, int n_atoms,
                                     const double* lattice, double r_ext, void* stream, hfx_basis** out) {
  if (!out) return fail(HFX_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_shells <= 0 || n_atoms <= 0 || !shells || !atom_xyz || !lattice)
    return fail(HFX_ERR_INVALID_ARG, "need at least one shell, one atom and the lattice");
  for (int i = 0; i < n_shells; ++i)
    if (shells[i].atom < 0 || shells[i].atom >= n_atoms || (i > 0 && shells[i].atom < shells[i - 1].atom))
      return fail(HFX_ERR_INVALID_ARG, "shells must be grouped by atom in increasing atom order");
  // extended set: home atoms, then the images (hfx_periodic_extend)
  const long long n_ext = hfx_periodic_extend(atom_xyz, n_atoms, lattice, r_ext, 0, nullptr, nullptr, nullptr);
  if (n_ext < 0) return HFX_ERR_INVALID_ARG;  // message set by hfx_periodic_extend
  if (n_ext > (1LL << 24)) return fail(HFX_ERR_UNSUPPORTED, "too many images");
  std::vector<int> ext_home((size_t)n_ext), ext_shift(3 * (size_t)n_ext);
  std::vector<double> xyz(3 * (size_t)n_ext);
  if (hfx_periodic_extend(atom_xyz, n_atoms, lattice, r_ext, n_ext, ext_home.data(), ext_shift.data(), xyz.data()) !=
      n_ext)
    return fail(HFX_ERR_INVALID_ARG, "extended set changed between calls");
  // every image carries its home atom's shells
  std::vector<int> first((size_t)n_atoms + 1, n_shells);
  for (int i = n_shells - 1; i >= 0; --i) first[(size_t)shells[i].atom] = i;
  for (int a = n_atoms - 1; a >= 0; --a)
    if (first[(size_t)a] > first[(size_t)a + 1]) first[(size_t)a] = first[(size_t)a + 1];
  std::vector<hfx_shell_desc> ext(shells, shells + n_shells);
  for (long long X = n_atoms; X < n_ext; ++X) {
    const int h = ext_home[(size_t)X];
    for (int S = first[(size_t)h]; S < first[(size_t)h + 1]; ++S) {
      hfx_shell_desc d = shells[S];
      d.atom = (int)X;
      ext.push_back(d);
    }
  }
  hfx_basis* b = nullptr;
  const hfx_status st = hfx_create_basis(ext.data(), (int)ext.size(), xyz.data(), (int)n_ext, stream, &b);
  if (st != HFX_OK) return st;
  b->n_home_atoms = n_atoms;
  b->n_home_shells = n_shells;
  b->h_ext_home = ext_home;
  b->h_ext_shift = ext_shift;
  *out = b;
  return HFX_OK;
}

int hfx_basis_atoms(const hfx_basis* b, int* n_home_atoms, int* ext_home, int* ext_shift) {
  if (!b) {
    fail(HFX_ERR_INVALID_ARG, "NULL basis");
    return -1;
  }
  if (n_home_atoms) *n_home_atoms = b->n_home_atoms;
  if (ext_home) std::copy(b->h_ext_home.begin(), b->h_ext_home.end(), ext_home);
  if (ext_shift) std::copy(b->h_ext_shift.begin(), b->h_ext_shift.end(), ext_shift);
  return b->n_atoms;
}


static hfx_status setup_pattern(hfx_quartets_s* q, const hfx_pattern* pat, cudaStream_t s) {
  hfx_basis* b = q->basis;
  const int na = b->n_atoms;
  if (!pat || pat->n_atoms != na || !pat->row_ptr || !pat->col)
    return fail(HFX_ERR_INVALID_ARG, "pattern must cover the basis's atoms");
  std::vector<long long> off((size_t)na * na, -1);
  std::vector<int> bx, by;
  std::vector<long long> bo;
  long long nv = 0;
  for (int X = 0; X < na; ++X) {
    if (pat->row_ptr[X + 1] < pat->row_ptr[X]) return fail(HFX_ERR_INVALID_ARG, "pattern row_ptr not monotone");
    for (int k = pat->row_ptr[X]; k < pat->row_ptr[X + 1]; ++k) {
      const int Y = pat->col[k];
      if (Y < 0 || Y >= na || off[(size_t)X * na + Y] >= 0)
        return fail(HFX_ERR_INVALID_ARG, "pattern column out of range or repeated");
      off[(size_t)X * na + Y] = nv;
      bx.push_back(X);
      by.push_back(Y);
      bo.push_back(nv);
      nv += (long long)b->h_atom_nf[X] * b->h_atom_nf[Y];
    }
  }
  for (int X = 0; X < na; ++X) {
    if (off[(size_t)X * na + X] < 0) return fail(HFX_ERR_INVALID_ARG, "pattern must contain every diagonal block");
    for (int Y = 0; Y < na; ++Y)
      if ((off[(size_t)X * na + Y] >= 0) != (off[(size_t)Y * na + X] >= 0))
        return fail(HFX_ERR_INVALID_ARG, "pattern must be symmetric");
  }
  q->n_atoms = na;
  q->n_values = nv;
  q->n_values_ext = nv;
  q->n_blocks = (int)bx.size();
  HFX_CK(upload(q->blk_off, off, s));
  HFX_CK(upload(q->blk_x, bx, s));
  HFX_CK(upload(q->blk_y, by, s));
  if (q->opts.spherical) {
    // caller's layout: 2l+1 solid harmonics per shell, blocks in the same order
    std::vector<int> nfs((size_t)na, 0), loc_sph((size_t)b->n_shells);
    for (int i = 0; i < b->n_shells; ++i) {
      loc_sph[(size_t)i] = nfs[(size_t)b->h_atom[i]];
      nfs[(size_t)b->h_atom[i]] += 2 * b->h_l[i] + 1;
    }
    std::vector<long long> afs((size_t)na + 1, 0);
    for (int X = 0; X < na; ++X) afs[(size_t)X + 1] = afs[(size_t)X] + nfs[(size_t)X];
    std::vector<int4> mc((size_t)b->nbf), ms((size_t)afs[(size_t)na]);
    for (int i = 0; i < b->n_shells; ++i) {
      const int X = b->h_atom[i], l = b->h_l[i];
      for (int c = 0; c < ncart(l); ++c)
        mc[(size_t)(b->h_atom_foff[X] + b->h_loc[i] + c)] = make_int4(loc_sph[(size_t)i], l, c, 0);
      for (int m = 0; m < 2 * l + 1; ++m)
        ms[(size_t)(afs[(size_t)X] + loc_sph[(size_t)i] + m)] = make_int4(b->h_loc[i], l, m, 0);
    }
    std::vector<long long> bos;
    long long nvs = 0;
    for (size_t k = 0; k < bx.size(); ++k) {
      bos.push_back(nvs);
      nvs += (long long)nfs[(size_t)bx[k]] * nfs[(size_t)by[k]];
    }
    q->n_values_ext = nvs;
    q->nbf_sph = afs[(size_t)na];
    q->h_afoff_sph = afs;
    HFX_CK(upload(q->blk_val_off_sph, bos, s));
    HFX_CK(upload(q->atom_nf_sph, nfs, s));
    HFX_CK(upload(q->afoff_cart, b->h_atom_foff, s));
    HFX_CK(upload(q->afoff_sph, afs, s));
    HFX_CK(upload(q->fmap_cart, mc, s));
    HFX_CK(upload(q->fmap_sph, ms, s));
    HFX_CK(q->P_cart.alloc((size_t)std::max<long long>(nv, 1)));
    HFX_CK(q->K_cart.alloc((size_t)std::max<long long>(nv, 1)));
  }
  HFX_CK(upload(q->blk_val_off, bo, s));
  return HFX_OK;
}

hfx_status hfx_build_quartets(hfx_basis* b, const hfx_opts* opts_in, const hfx_pattern* pattern, void* stream,
                              hfx_quartets** out) {
  if (!out || !b || !opts_in) return fail(HFX_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  hfx_opts o = *opts_in;
  if (o.kernel < 0 || o.kernel > 2) return fail(HFX_ERR_INVALID_ARG, "unknown kernel");
  if (o.kernel != HFX_KERNEL_COULOMB && !(o.omega > 0.0)) return fail(HFX_ERR_INVALID_ARG, "omega must be > 0");
  if (o.precision != HFX_PREC_FP64 && o.precision != HFX_PREC_MIXED)
    return fail(HFX_ERR_INVALID_ARG, "unknown precision");
  if (o.n_block <= 0) o.n_block = 128;
  if (!(o.tau >= 0.0) || !(o.eps >= 0.0) || !(o.prim_cutoff >= 0.0))
    return fail(HFX_ERR_INVALID_ARG, "thresholds must be >= 0");
  auto* q = new hfx_quartets_s();
  std::unique_ptr<hfx_quartets_s> guard(q);
  q->basis = b;
  q->opts = o;
  q->n_sm = device_sm_count();
  cudaEvent_t t0, t1;
  HFX_CK(cudaEventCreate(&t0));
  HFX_CK(cudaEventCreate(&t1));
  HFX_CK(cudaEventRecord(t0, s));
  struct PhaseEvents {  // ends of setup phases: pairs, Schwarz, sorted lists, work queues
    cudaEvent_t e[4] = {};
    ~PhaseEvents() {
      for (auto x : e)
        if (x) cudaEventDestroy(x);
    }
  } ph;
  for (auto& x : ph.e) HFX_CK(cudaEventCreate(&x));
  hfx_status st = setup_pattern(q, pattern, s);
  if (st != HFX_OK) return st;

  // 1. all shell pairs, oriented l_A >= l_B; with distance screening only the
  //    pairs whose extents reach each other (Sec. 2: NAO/distance screening)
  const int ns = b->n_shells;
  const long long npair_all = (long long)ns * (ns + 1) / 2;
  if (npair_all > (1LL << 30)) return fail(HFX_ERR_UNSUPPORTED, "too many shell pairs");
  const int stride = b->max_nprim * b->max_nprim;
  std::vector<double> reach;
  if (o.extent_eps > 0.0) {  // R_S = sqrt(ln(1/eps) / alpha_min(S))
    if (!(o.extent_eps < 1.0)) return fail(HFX_ERR_INVALID_ARG, "extent_eps must be in (0, 1)");
    reach.resize((size_t)ns);
    const double lg = std::log(1.0 / o.extent_eps);
    for (int S = 0; S < ns; ++S) {
      double amin = b->h_alpha[(size_t)b->h_poff[S]];
      for (int k = b->h_poff[S]; k < b->h_poff[S + 1]; ++k) amin = std::min(amin, b->h_alpha[(size_t)k]);
      reach[(size_t)S] = std::sqrt(lg / amin);
    }
  }
  std::vector<int2> list;
  list.reserve((size_t)(reach.empty() ? npair_all : std::min<long long>(npair_all, 1LL << 22)));
  for (int I = 0; I < ns; ++I)
    for (int J = 0; J <= I; ++J) {
      if (!reach.empty()) {
        const double* a = &b->h_atom_xyz[3 * (size_t)b->h_atom[I]];
        const double* c = &b->h_atom_xyz[3 * (size_t)b->h_atom[J]];
        const double d2 = (a[0] - c[0]) * (a[0] - c[0]) + (a[1] - c[1]) * (a[1] - c[1]) + (a[2] - c[2]) * (a[2] - c[2]);
        const double r = reach[(size_t)I] + reach[(size_t)J];
        if (d2 > r * r) continue;
      }
      int A = I, B = J;
      if (b->h_l[A] < b->h_l[B]) std::swap(A, B);
      list.push_back(make_int2(A, B));
    }
  const int npair = (int)list.size();
  q->n_pairs_distance = npair;
  if ((long long)npair * stride > (1LL << 31) - 1) return fail(HFX_ERR_UNSUPPORTED, "too many primitive pairs");
  DBuf<int2> d_list;
  DBuf<PairRec> all_pairs;
  DBuf<PrimPair> all_prims;
  DBuf<int> pclass;
  DBuf<double> Q;
  HFX_CK(upload(d_list, list, s));
  HFX_CK(all_pairs.alloc(npair));
  HFX_CK(all_prims.alloc((size_t)npair * stride));
  HFX_CK(pclass.alloc(npair));
  HFX_CK(Q.alloc(npair));
  k_pair_build<<<blocks_for(npair, 128), 128, 0, s>>>(npair, d_list.p, b->sh_xyz.p, b->sh_l.p, b->sh_poff.p,
                                                       b->alpha.p, b->coef.p, stride, kPairDropBound, all_pairs.p,
                                                       all_prims.p, pclass.p);
  HFX_CK(cudaGetLastError());

  HFX_CK(cudaEventRecord(ph.e[0], s));

  // 2. Schwarz bounds with the run's kernel (Sec. 2, Eq. schwarz)
  for (int c = 0; c < 6; ++c) {
    SchwarzArgs a;
    a.pairs = all_pairs.p;
    a.prims = all_prims.p;
    a.pair_class = pclass.p;
    a.n_pairs = npair;
    a.cls = c;
    a.boys = b->boys.p;
    a.kernel = o.kernel;
    a.omega2 = o.omega * o.omega;
    a.Q = Q.p;
    kClassOps[quartet_class_of(c, c)].launch_schwarz(a, s);
  }
  HFX_CK(cudaGetLastError());
  HFX_CK(cudaEventRecord(ph.e[1], s));

  // 3. sort pairs by (class, descending Q); significant pairs are a prefix of
  //    each class segment (Q_IJ Q_max > tau is lossless)
  DBuf<unsigned long long> qmax, key, key_out;
  DBuf<int> idx, idx_out, ckey, ckey_out, cnt;
  HFX_CK(qmax.alloc(1));
  HFX_CK(cudaMemsetAsync(qmax.p, 0, sizeof(unsigned long long), s));
  k_qmax<<<blocks_for(npair, 256), 256, 0, s>>>(npair, Q.p, qmax.p);
  HFX_CK(key.alloc(npair));
  HFX_CK(key_out.alloc(npair));
  HFX_CK(idx.alloc(npair));
  HFX_CK(idx_out.alloc(npair));
  HFX_CK(ckey.alloc(npair));
  HFX_CK(ckey_out.alloc(npair));
  k_sort_keys<<<blocks_for(npair, 256), 256, 0, s>>>(npair, Q.p, pclass.p, key.p, idx.p);
  {
    size_t tmp_bytes = 0, tmp2 = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, key.p, key_out.p, idx.p, idx_out.p, npair, 0, 64, s);
    cub::DeviceRadixSort::SortPairs(nullptr, tmp2, ckey.p, ckey_out.p, idx_out.p, idx.p, npair, 0, 3, s);
    DBuf<unsigned char> tmp;
    HFX_CK(tmp.alloc(std::max(tmp_bytes, tmp2)));
    tmp_bytes = tmp.n;
    HFX_CK(cub::DeviceRadixSort::SortPairs(tmp.p, tmp_bytes, key.p, key_out.p, idx.p, idx_out.p, npair, 0, 64, s));
    k_gather_class<<<blocks_for(npair, 256), 256, 0, s>>>(npair, idx_out.p, pclass.p, ckey.p);
    tmp_bytes = tmp.n;
    HFX_CK(cub::DeviceRadixSort::SortPairs(tmp.p, tmp_bytes, ckey.p, ckey_out.p, idx_out.p, idx.p, npair, 0, 3, s));
  }
  HFX_CK(cnt.alloc(12));
  HFX_CK(cudaMemsetAsync(cnt.p, 0, 12 * sizeof(int), s));
  k_class_counts<<<blocks_for(npair, 256), 256, 0, s>>>(npair, idx.p, pclass.p, Q.p, o.screen, o.tau, qmax.p,
                                                        cnt.p, cnt.p + 6);
  int h_cnt[12];
  HFX_CK(cudaMemcpyAsync(h_cnt, cnt.p, sizeof(h_cnt), cudaMemcpyDeviceToHost, s));
  HFX_CK(cudaStreamSynchronize(s));

  // 4. per-class significant pair lists
  long long seg = 0;
  for (int c = 0; c < 6; ++c) {
    const int nk = h_cnt[6 + c];
    q->n_pairs[c] = nk;
    HFX_CK(q->pairs[c].alloc(nk));
    HFX_CK(q->prims[c].alloc((size_t)nk * stride));
    if (nk > 0)
      k_gather_pairs<<<blocks_for(nk, 128), 128, 0, s>>>(nk, idx.p + seg, all_pairs.p, all_prims.p, Q.p, stride,
                                                         q->pairs[c].p, q->prims[c].p);
    seg += h_cnt[c];
  }
  HFX_CK(cudaGetLastError());

  HFX_CK(cudaEventRecord(ph.e[2], s));

  // 5. work-queue batches per quartet class
  for (int cb = 0; cb < 6; ++cb)
    for (int ck = 0; ck <= cb; ++ck) {
      const int cls = quartet_class_of(cb, ck);
      const int nb = (int)q->n_pairs[cb], nk = (int)q->n_pairs[ck];
      q->n_desc[cls] = 0;
      q->n_quartets[cls] = 0;
      if (nb == 0 || nk == 0) continue;
      DBuf<int> chunks, off;
      DBuf<long long> nq, nq_sum;
      HFX_CK(chunks.alloc(nb));
      HFX_CK(off.alloc(nb));
      HFX_CK(nq.alloc(nb));
      HFX_CK(nq_sum.alloc(1));
      k_desc_count<<<blocks_for(nb, 128), 128, 0, s>>>(nb, q->pairs[cb].p, nk, q->pairs[ck].p, cb == ck, o.screen,
                                                       o.tau, o.n_block, chunks.p, nq.p);
      size_t t1b = 0, t2b = 0;
      cub::DeviceScan::ExclusiveSum(nullptr, t1b, chunks.p, off.p, nb, s);
      cub::DeviceReduce::Sum(nullptr, t2b, nq.p, nq_sum.p, nb, s);
      DBuf<unsigned char> tmp;
      HFX_CK(tmp.alloc(std::max(t1b, t2b)));
      t1b = tmp.n;
      HFX_CK(cub::DeviceScan::ExclusiveSum(tmp.p, t1b, chunks.p, off.p, nb, s));
      t2b = tmp.n;
      HFX_CK(cub::DeviceReduce::Sum(tmp.p, t2b, nq.p, nq_sum.p, nb, s));
      int last_off = 0, last_chunks = 0;
      long long total_q = 0;
      HFX_CK(cudaMemcpyAsync(&last_off, off.p + nb - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
      HFX_CK(cudaMemcpyAsync(&last_chunks, chunks.p + nb - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
      HFX_CK(cudaMemcpyAsync(&total_q, nq_sum.p, sizeof(long long), cudaMemcpyDeviceToHost, s));
      HFX_CK(cudaStreamSynchronize(s));
      const long long nd = (long long)last_off + last_chunks;
      if (nd > (1LL << 31) - 1) return fail(HFX_ERR_UNSUPPORTED, "too many work-queue batches; raise n_block");
      q->n_desc[cls] = (int)nd;
      q->n_quartets[cls] = total_q;
      HFX_CK(q->desc[cls].alloc(nd));
      if (nd > 0)
        k_desc_fill<<<blocks_for(nb, 128), 128, 0, s>>>(nb, nk, q->pairs[cb].p, q->pairs[ck].p, cb == ck, o.screen,
                                                        o.tau, o.n_block, off.p, q->desc[cls].p, 0);
      HFX_CK(cudaGetLastError());
    }
  long long npp = 0;
  for (int c = 0; c < 6; ++c) {
    if (q->n_pairs[c] == 0) continue;
    std::vector<PairRec> h((size_t)q->n_pairs[c]);
    HFX_CK(cudaMemcpyAsync(h.data(), q->pairs[c].p, h.size() * sizeof(PairRec), cudaMemcpyDeviceToHost, s));
    HFX_CK(cudaStreamSynchronize(s));
    for (auto& r : h) npp += r.pcnt;
  }
  q->n_prim_pairs = npp;
  HFX_CK(cudaEventRecord(ph.e[3], s));

  // 6. per-build buffers and the single-system build plan
  HFX_CK(q->pmax.alloc((size_t)ns * ns));
  HFX_CK(q->scratch.alloc(2));
  fill_sys(q);
  {
    std::vector<hfx_quartets_s*> one(1, q);
    hfx_status pst = plan_alloc(q->plan, one, q->n_sm);
    if (pst != HFX_OK) return pst;
    for (int cls = 0; cls < HFX_NCLASS; ++cls) {
      q->plan.descp[cls] = q->desc[cls].p;
      q->plan.n_desc[cls] = q->n_desc[cls];
      q->plan.n_block[cls] = o.n_block;
    }
  }
  HFX_CK(cudaEventRecord(t1, s));
  HFX_CK(cudaEventSynchronize(t1));
  cudaEventElapsedTime(&q->ms_setup, t0, t1);
  cudaEventElapsedTime(&q->ms_setup_phase[0], t0, ph.e[0]);
  for (int k = 1; k < 4; ++k) cudaEventElapsedTime(&q->ms_setup_phase[k], ph.e[k - 1], ph.e[k]);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  HFX_CK(cudaGetLastError());
  *out = guard.release();
  return HFX_OK;
}

void hfx_destroy_quartets(hfx_quartets* q) { delete q; }

long long hfx_value_count(const hfx_quartets* q) { return q ? q->n_values_ext : -1; }

}  // extern "C"

template <typename T>
static long long dbytes(const DBuf<T>& b) {
  return (long long)(b.n * sizeof(T));
}

// Function count of every atom from a shell list (host); false on bad input.
static bool atom_function_counts(const hfx_shell_desc* shells, int n_shells, int n_atoms, std::vector<long long>& nf) {
  nf.assign((size_t)n_atoms, 0);
  for (int i = 0; i < n_shells; ++i) {
    const int a = shells[i].atom, l = shells[i].l;
    if (a < 0 || a >= n_atoms || l < 0 || l > 2) return false;
    nf[(size_t)a] += ncart(l);
  }
  return true;
}

extern "C" {

long long hfx_quartets_device_bytes(const hfx_quartets* q) {
  if (!q) return -1;
  long long n = dbytes(q->blk_off) + dbytes(q->blk_x) + dbytes(q->blk_y) + dbytes(q->blk_val_off) +
                dbytes(q->pmax) + dbytes(q->scratch) + dbytes(q->delta_K);
  for (int c = 0; c < 6; ++c) n += dbytes(q->pairs[c]) + dbytes(q->prims[c]);
  for (int c = 0; c < HFX_NCLASS; ++c) n += dbytes(q->desc[c]) + dbytes(q->plan.desc_own[c]);
  const Plan& pl = q->plan;
  n += dbytes(pl.d_sys) + dbytes(pl.d_pmax) + dbytes(pl.counters) + dbytes(pl.n_done) + dbytes(pl.energy);
  return n;
}

long long hfx_basis_device_bytes(const hfx_basis* b) {
  if (!b) return -1;
  return dbytes(b->sh_xyz) + dbytes(b->alpha) + dbytes(b->coef) + dbytes(b->boys) + dbytes(b->boysf) +
         dbytes(b->sh_l) + dbytes(b->sh_atom) + dbytes(b->sh_poff) + dbytes(b->sh_loc) + dbytes(b->atom_nf);
}

long long hfx_pattern_value_count(const hfx_shell_desc* shells, int n_shells, const hfx_pattern* pattern) {
  if (!shells || n_shells <= 0 || !pattern || !pattern->row_ptr || !pattern->col || pattern->n_atoms <= 0) return -1;
  std::vector<long long> nf;
  if (!atom_function_counts(shells, n_shells, pattern->n_atoms, nf)) return -1;
  long long nv = 0;
  for (int X = 0; X < pattern->n_atoms; ++X)
    for (int k = pattern->row_ptr[X]; k < pattern->row_ptr[X + 1]; ++k) {
      const int Y = pattern->col[k];
      if (Y < 0 || Y >= pattern->n_atoms) return -1;
      nv += nf[(size_t)X] * nf[(size_t)Y];
    }
  return nv;
}

hfx_status hfx_pack_dense_host(const hfx_shell_desc* shells, int n_shells, const hfx_pattern* pattern,
                               const double* dense, double* val) {
  if (!dense || !val) return fail(HFX_ERR_INVALID_ARG, "NULL argument");
  if (hfx_pattern_value_count(shells, n_shells, pattern) < 0)
    return fail(HFX_ERR_INVALID_ARG, "inconsistent shells or pattern");
  std::vector<long long> nf, foff((size_t)pattern->n_atoms + 1, 0);
  atom_function_counts(shells, n_shells, pattern->n_atoms, nf);
  for (int X = 0; X < pattern->n_atoms; ++X) foff[X + 1] = foff[X] + nf[(size_t)X];
  const long long nbf = foff[pattern->n_atoms];
  long long v = 0;
  for (int X = 0; X < pattern->n_atoms; ++X)
    for (int k = pattern->row_ptr[X]; k < pattern->row_ptr[X + 1]; ++k) {
      const int Y = pattern->col[k];
      for (long long i = 0; i < nf[(size_t)X]; ++i)
        for (long long j = 0; j < nf[(size_t)Y]; ++j) val[v++] = dense[(foff[X] + i) * nbf + foff[Y] + j];
    }
  return HFX_OK;
}

long long hfx_setup_bytes_estimate(const hfx_shell_desc* shells, int n_shells, const hfx_pattern* pattern) {
  if (!shells || n_shells <= 0 || !pattern || !pattern->row_ptr || !pattern->col || pattern->n_atoms <= 0) return -1;
  std::vector<long long> nf;
  if (!atom_function_counts(shells, n_shells, pattern->n_atoms, nf)) return -1;
  long long nv = 0, nblk = 0;
  for (int X = 0; X < pattern->n_atoms; ++X)
    for (int k = pattern->row_ptr[X]; k < pattern->row_ptr[X + 1]; ++k) {
      const int Y = pattern->col[k];
      if (Y < 0 || Y >= pattern->n_atoms) return -1;
      nv += nf[(size_t)X] * nf[(size_t)Y];
      ++nblk;
    }
  int max_nprim = 1;
  for (int i = 0; i < n_shells; ++i) max_nprim = std::max(max_nprim, shells[i].nprim);
  const long long ns = n_shells, na = pattern->n_atoms, npair = ns * (ns + 1) / 2;
  const long long stride = (long long)max_nprim * max_nprim;
  const long long pair_bytes = (long long)sizeof(PairRec) + stride * (long long)sizeof(PrimPair);
  // basis: shells, primitives, the two Boys tables
  const long long basis = ns * 64 + (long long)n_shells * max_nprim * 16 +
                          (long long)kBoysNL * kBoysNT * kBoysCols * (8 + 8);
  // setup peak: every shell pair with its primitive pairs, sort keys and
  // indexes (about 64 B per pair) and the class-sorted copy of the pairs (at
  // most as large); persistent: pattern tables, Pmax, work-queue batches (a
  // generous cap of two 16 B descriptors per shell pair)
  const long long pairs_all = npair * (pair_bytes + 64);
  const long long persistent = na * na * 8 + nblk * 16 + ns * ns * 8 + npair * pair_bytes +
                               npair * 2 * (long long)sizeof(Desc);
  (void)nv;
  return basis + pairs_all + persistent;
}

hfx_status hfx_build_K(hfx_quartets* q, const double* P, double* K, void* stream) {
  if (!q || !P || !K) return fail(HFX_ERR_INVALID_ARG, "NULL argument");
  Plan& pl = q->plan;
  cudaStream_t s = (cudaStream_t)stream;
  const bool sph = q->opts.spherical != 0;
  if (sph && q->n_blocks > 0)  // P = T^T P_sph T (Cartesian copy)
    k_sph_transform<<<q->n_blocks, 128, 0, s>>>(q->n_blocks, q->blk_x.p, q->blk_y.p, q->blk_val_off_sph.p,
                                                q->blk_val_off.p, q->afoff_cart.p, q->atom_nf_sph.p,
                                                q->basis->atom_nf.p, q->fmap_cart.p, 0, P, q->P_cart.p);
  HFX_CK(cudaEventSynchronize(pl.sys_copied));
  pl.h_sys[0] = q->h_sys;
  pl.h_sys[0].P = sph ? q->P_cart.p : P;
  pl.h_sys[0].K = sph ? q->K_cart.p : K;
  const hfx_status st = plan_build(pl, s, false, true);
  if (st != HFX_OK || !sph) return st;
  if (q->n_blocks > 0)  // K_sph = T K T^T
    k_sph_transform<<<q->n_blocks, 128, 0, s>>>(q->n_blocks, q->blk_x.p, q->blk_y.p, q->blk_val_off.p,
                                                q->blk_val_off_sph.p, q->afoff_sph.p, q->basis->atom_nf.p,
                                                q->atom_nf_sph.p, q->fmap_sph.p, 1, q->K_cart.p, K);
  HFX_CK(cudaGetLastError());
  return HFX_OK;
}

hfx_status hfx_build_K_shard(hfx_quartets* q, const double* P, double* K, int rank, int n_ranks, void* stream) {
  if (!q || !P || !K) return fail(HFX_ERR_INVALID_ARG, "NULL argument");
  if (n_ranks < 1 || rank < 0 || rank >= n_ranks) return fail(HFX_ERR_INVALID_ARG, "need 0 <= rank < n_ranks");
  Plan& pl = q->plan;
  pl.shard_rank = rank;
  pl.shard_n = n_ranks;
  const hfx_status st = hfx_build_K(q, P, K, stream);
  pl.shard_rank = 0;
  pl.shard_n = 1;
  return st;
}

hfx_status hfx_build_K_delta(hfx_quartets* q, const double* dP, double* K, void* stream) {
  if (!q || !dP || !K) return fail(HFX_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const long long nv = q->n_values_ext;
  if (q->delta_K.p == nullptr || q->delta_K.n < (size_t)nv) HFX_CK(q->delta_K.alloc((size_t)nv));
  const hfx_status st = hfx_build_K(q, dP, q->delta_K.p, stream);
  if (st != HFX_OK) return st;
  if (nv > 0) {
    const int blocks = (int)std::max<long long>(1, std::min<long long>(4LL * q->n_sm, (nv + 255) / 256));
    k_axpy<<<blocks, 256, 0, s>>>(nv, q->delta_K.p, K);
    HFX_CK(cudaGetLastError());
  }
  return HFX_OK;
}

hfx_status hfx_exchange_energy(hfx_quartets* q, const double* P, const double* K, double* E_x, void* stream) {
  if (!q || !P || !K || !E_x) return fail(HFX_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  HFX_CK(cudaMemsetAsync(q->scratch.p, 0, sizeof(double), s));
  // over the caller's layout (tr(P K) is the same in both: the transforms are orthogonal per shell block)
  const long long nv = q->n_values_ext;
  const int blocks = std::max(1, std::min<int>(4 * q->n_sm, (int)((nv / 2 + 255) / 256)));
  const int vec = ((reinterpret_cast<uintptr_t>(P) | reinterpret_cast<uintptr_t>(K)) & 15) == 0;
  k_dot<<<blocks, 256, 0, s>>>(nv, P, K, vec, q->scratch.p);
  double h = 0.0;
  HFX_CK(cudaMemcpyAsync(&h, q->scratch.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  HFX_CK(cudaStreamSynchronize(s));
  *E_x = -0.5 * h;
  return HFX_OK;
}

// Dense <-> values in the caller's layout (Cartesian, or spherical harmonics).
static hfx_status pack_dense(const hfx_quartets* q, double* dense, double* val, int unpack, cudaStream_t s) {
  const bool sph = q->opts.spherical != 0;
  DBuf<long long> afoff;
  HFX_CK(upload(afoff, sph ? q->h_afoff_sph : q->basis->h_atom_foff, s));
  const long long nbf = sph ? q->nbf_sph : (long long)q->basis->nbf;
  if (unpack) HFX_CK(cudaMemsetAsync(dense, 0, (size_t)nbf * (size_t)nbf * sizeof(double), s));
  if (q->n_blocks > 0)
    k_pack<<<q->n_blocks, 128, 0, s>>>(q->n_blocks, q->blk_x.p, q->blk_y.p,
                                       sph ? q->blk_val_off_sph.p : q->blk_val_off.p, afoff.p,
                                       sph ? q->atom_nf_sph.p : q->basis->atom_nf.p, nbf, dense, val, unpack);
  HFX_CK(cudaStreamSynchronize(s));
  return HFX_OK;
}

hfx_status hfx_pack_dense(const hfx_quartets* q, const double* dense, double* val, void* stream) {
  if (!q || !dense || !val) return fail(HFX_ERR_INVALID_ARG, "NULL argument");
  return pack_dense(q, const_cast<double*>(dense), val, 0, (cudaStream_t)stream);
}

hfx_status hfx_unpack_dense(const hfx_quartets* q, const double* val, double* dense, void* stream) {
  if (!q || !dense || !val) return fail(HFX_ERR_INVALID_ARG, "NULL argument");
  return pack_dense(q, dense, const_cast<double*>(val), 1, (cudaStream_t)stream);
}

hfx_status hfx_eval_quartets(hfx_basis* b, int kernel, double omega, int precision, int n, const int* quartets,
                             const long long* out_off, double* out, void* stream) {
  if (!b || (n > 0 && (!quartets || !out_off || !out))) return fail(HFX_ERR_INVALID_ARG, "NULL argument");
  if (kernel < 0 || kernel > 2) return fail(HFX_ERR_INVALID_ARG, "unknown kernel");
  if (n <= 0) return HFX_OK;
  cudaStream_t s = (cudaStream_t)stream;
  std::map<std::pair<int, int>, int> pid;
  std::vector<int2> plist;
  std::vector<int4> items((size_t)n), strides((size_t)n);
  auto orient = [&](int I, int J, bool& swapped) {
    swapped = b->h_l[I] < b->h_l[J];
    const int A = swapped ? J : I, B = swapped ? I : J;
    auto key = std::make_pair(A, B);
    auto it = pid.find(key);
    if (it != pid.end()) return it->second;
    const int id = (int)plist.size();
    pid[key] = id;
    plist.push_back(make_int2(A, B));
    return id;
  };
  for (int t = 0; t < n; ++t) {
    const int* sh = quartets + 4 * t;
    for (int k = 0; k < 4; ++k)
      if (sh[k] < 0 || sh[k] >= b->n_shells) return fail(HFX_ERR_INVALID_ARG, "shell index out of range");
    const int nI = ncart(b->h_l[sh[0]]), nJ = ncart(b->h_l[sh[1]]), nK = ncart(b->h_l[sh[2]]),
              nL = ncart(b->h_l[sh[3]]);
    const int sI = nJ * nK * nL, sJ = nK * nL, sK = nL, sL = 1;
    bool swb, swk;
    const int pb = orient(sh[0], sh[1], swb), pk = orient(sh[2], sh[3], swk);
    int sa = swb ? sJ : sI, sb = swb ? sI : sJ, sc = swk ? sL : sK, sd = swk ? sK : sL;
    const int lA = b->h_l[plist[pb].x], lB = b->h_l[plist[pb].y];
    const int lC = b->h_l[plist[pk].x], lD = b->h_l[plist[pk].y];
    int cb = pair_class_of(lA, lB), ck = pair_class_of(lC, lD);
    int bra = pb, ket = pk;
    if (cb < ck) {
      std::swap(bra, ket);
      std::swap(cb, ck);
      std::swap(sa, sc);
      std::swap(sb, sd);
    }
    items[t] = make_int4(bra, ket, quartet_class_of(cb, ck), 0);
    strides[t] = make_int4(sa, sb, sc, sd);
  }
  const int np = (int)plist.size();
  const int stride = b->max_nprim * b->max_nprim;
  DBuf<int2> d_list;
  DBuf<PairRec> pairs;
  DBuf<PrimPair> prims;
  DBuf<int> pclass;
  DBuf<int4> d_items, d_strides;
  DBuf<long long> d_off;
  HFX_CK(upload(d_list, plist, s));
  HFX_CK(pairs.alloc(np));
  HFX_CK(prims.alloc((size_t)np * stride));
  HFX_CK(pclass.alloc(np));
  HFX_CK(upload(d_items, items, s));
  HFX_CK(upload(d_strides, strides, s));
  std::vector<long long> offv(out_off, out_off + n);
  HFX_CK(upload(d_off, offv, s));
  k_pair_build<<<blocks_for(np, 128), 128, 0, s>>>(np, d_list.p, b->sh_xyz.p, b->sh_l.p, b->sh_poff.p, b->alpha.p,
                                                   b->coef.p, stride, 0.0, pairs.p, prims.p, pclass.p);
  for (int cls = 0; cls < HFX_NCLASS; ++cls) {
    EvalArgs a;
    a.pairs = pairs.p;
    a.prims = prims.p;
    a.quartets = d_items.p;
    a.out_off = d_off.p;
    a.strides = d_strides.p;
    a.n = n;
    a.cls = cls;
    a.boys = b->boys.p;
    a.boysf = b->boysf.p;
    a.kernel = kernel;
    a.omega2 = omega * omega;
    a.omega2_hi = (float)a.omega2;
    a.omega2_lo = (float)(a.omega2 - (double)a.omega2_hi);
    a.out = out;
    kClassOps[cls].launch_eval(a, precision == HFX_PREC_MIXED, s);
  }
  HFX_CK(cudaGetLastError());
  HFX_CK(cudaStreamSynchronize(s));
  return HFX_OK;
}

hfx_status hfx_boys_eval(hfx_basis* b, int precision, int mmax, int n, const double* T, double* F, void* stream) {
  if (!b || (n > 0 && (!T || !F))) return fail(HFX_ERR_INVALID_ARG, "NULL argument");
  if (mmax < 0 || mmax > kMaxLtot) return fail(HFX_ERR_INVALID_ARG, "mmax must be in 0..8");
  if (n <= 0) return HFX_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int dsp = precision == HFX_PREC_MIXED;
  const unsigned g = blocks_for(n, 128);
  switch (mmax) {
    case 0: k_boys_eval<0><<<g, 128, 0, s>>>(b->boys.p, b->boysf.p, dsp, n, T, F); break;
    case 1: k_boys_eval<1><<<g, 128, 0, s>>>(b->boys.p, b->boysf.p, dsp, n, T, F); break;
    case 2: k_boys_eval<2><<<g, 128, 0, s>>>(b->boys.p, b->boysf.p, dsp, n, T, F); break;
    case 3: k_boys_eval<3><<<g, 128, 0, s>>>(b->boys.p, b->boysf.p, dsp, n, T, F); break;
    case 4: k_boys_eval<4><<<g, 128, 0, s>>>(b->boys.p, b->boysf.p, dsp, n, T, F); break;
    case 5: k_boys_eval<5><<<g, 128, 0, s>>>(b->boys.p, b->boysf.p, dsp, n, T, F); break;
    case 6: k_boys_eval<6><<<g, 128, 0, s>>>(b->boys.p, b->boysf.p, dsp, n, T, F); break;
    case 7: k_boys_eval<7><<<g, 128, 0, s>>>(b->boys.p, b->boysf.p, dsp, n, T, F); break;
    default: k_boys_eval<8><<<g, 128, 0, s>>>(b->boys.p, b->boysf.p, dsp, n, T, F); break;
  }
  HFX_CK(cudaGetLastError());
  HFX_CK(cudaStreamSynchronize(s));
  return HFX_OK;
}

hfx_status hfx_get_stats(const hfx_quartets* q, hfx_stats* out) {
  if (!q || !out) return fail(HFX_ERR_INVALID_ARG, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  HFX_CK(cudaDeviceSynchronize());
  for (int c = 0; c < 6; ++c) out->n_pairs_significant[c] = q->n_pairs[c];
  for (int c = 0; c < HFX_NCLASS; ++c) out->n_quartets_schwarz[c] = q->n_quartets[c];
  out->n_prim_pairs = q->n_prim_pairs;
  out->n_values = q->n_values_ext;
  out->n_pairs_distance = q->n_pairs_distance;
  out->ms_setup = q->ms_setup;
  for (int k = 0; k < 4; ++k) out->ms_setup_phase[k] = q->ms_setup_phase[k];
  plan_stats(const_cast<hfx_quartets_s*>(q)->plan, out);
  return HFX_OK;
}

// ------------------------------------------------------------------ batches
struct hfx_batch_s {
  std::vector<hfx_quartets_s*> members;
  Plan plan;
  bool tuned = false;
};

hfx_status hfx_batch_create(hfx_quartets* const* members, int n, void* stream, hfx_batch** out) {
  if (!out || !members || n <= 0) return fail(HFX_ERR_INVALID_ARG, "need at least one member");
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<hfx_batch_s> b(new hfx_batch_s());
  for (int i = 0; i < n; ++i) {
    if (!members[i]) return fail(HFX_ERR_INVALID_ARG, "NULL member");
    const hfx_opts &o0 = members[0]->opts, &oi = members[i]->opts;
    if (oi.kernel != o0.kernel || oi.omega != o0.omega || oi.precision != o0.precision ||
        oi.screen != o0.screen || oi.tau != o0.tau || oi.density_screen != o0.density_screen ||
        oi.eps != o0.eps || oi.prim_cutoff != o0.prim_cutoff ||
        !(oi.fp64_promote_bound == o0.fp64_promote_bound) || oi.promote_min_l != o0.promote_min_l ||
        oi.prim_density_screen != o0.prim_density_screen || oi.promote_prims != o0.promote_prims)
      return fail(HFX_ERR_INVALID_ARG, "batch members must share kernel, precision and screening options");
    if (oi.spherical) return fail(HFX_ERR_UNSUPPORTED, "batches take Cartesian quartet lists only");
    b->members.push_back(members[i]);
  }
  hfx_status st = plan_alloc(b->plan, b->members, members[0]->n_sm);
  if (st != HFX_OK) return st;
  for (int cls = 0; cls < HFX_NCLASS; ++cls) {
    st = plan_class_desc(b->plan, b->members, cls, members[0]->opts.n_block, s);
    if (st != HFX_OK) return st;
  }
  for (int cls = 0; cls < HFX_NCLASS; ++cls) {
    HFX_CK(cudaStreamCreateWithFlags(&b->plan.side[cls], cudaStreamNonBlocking));
    HFX_CK(cudaEventCreateWithFlags(&b->plan.join_ev[cls], cudaEventDisableTiming));
  }
  HFX_CK(cudaEventCreateWithFlags(&b->plan.fork_ev, cudaEventDisableTiming));
  *out = b.release();
  return HFX_OK;
}

void hfx_batch_destroy(hfx_batch* b) { delete b; }

static void batch_set_pointers(hfx_batch_s* b, const double* const* P, double* const* K) {
  for (int i = 0; i < b->plan.n; ++i) {
    b->plan.h_sys[i] = b->members[i]->h_sys;
    b->plan.h_sys[i].P = P[i];
    b->plan.h_sys[i].K = K[i];
  }
}

hfx_status hfx_batch_build_K(hfx_batch* b, const double* const* P_vals, double* const* K_vals, int use_graph,
                             void* stream) {
  if (!b || !P_vals || !K_vals) return fail(HFX_ERR_INVALID_ARG, "NULL argument");
  for (int i = 0; i < b->plan.n; ++i)
    if (!P_vals[i] || !K_vals[i]) return fail(HFX_ERR_INVALID_ARG, "NULL P or K of a member");
  cudaStream_t s = (cudaStream_t)stream;
  Plan& pl = b->plan;
  HFX_CK(cudaEventSynchronize(pl.sys_copied));
  batch_set_pointers(b, P_vals, K_vals);
  if (!use_graph) return plan_build(pl, s, false, true);
  if (!pl.gexec) {
    // the graph reads P and K through the system table, copied from pinned
    // host memory by its first node, so one capture serves every later build
    for (int f = 0; f < 2; ++f)
      for (int cls = 0; cls < HFX_NCLASS; ++cls)
        if (pl.n_desc[cls]) plan_grid(pl, f, cls);
    cudaStream_t cap;
    HFX_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    HFX_CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed));
    hfx_status st = plan_build(pl, cap, true, false);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (st != HFX_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return fail(HFX_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&pl.gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(HFX_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  HFX_CK(cudaEventRecord(pl.ev0, s));
  HFX_CK(cudaGraphLaunch(pl.gexec, s));
  HFX_CK(cudaEventRecord(pl.sys_copied, s));
  HFX_CK(cudaEventRecord(pl.ev1, s));
  for (auto& p : pl.ran)
    for (auto& r : p) r = false;
  return HFX_OK;
}

hfx_status hfx_batch_energies(hfx_batch* b, double* E_x, void* stream) {
  if (!b || !E_x) return fail(HFX_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  HFX_CK(cudaMemcpyAsync(E_x, b->plan.energy.p, sizeof(double) * b->plan.n, cudaMemcpyDeviceToHost, s));
  HFX_CK(cudaStreamSynchronize(s));
  return HFX_OK;
}

hfx_status hfx_batch_get_stats(hfx_batch* b, hfx_stats* out) {
  if (!b || !out) return fail(HFX_ERR_INVALID_ARG, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  HFX_CK(cudaDeviceSynchronize());
  for (auto* q : b->members) {
    for (int c = 0; c < 6; ++c) out->n_pairs_significant[c] += q->n_pairs[c];
    for (int c = 0; c < HFX_NCLASS; ++c) out->n_quartets_schwarz[c] += q->n_quartets[c];
    out->n_prim_pairs += q->n_prim_pairs;
    out->n_values += q->n_values_ext;
    out->n_pairs_distance += q->n_pairs_distance;
    out->ms_setup += q->ms_setup;
    for (int k = 0; k < 4; ++k) out->ms_setup_phase[k] += q->ms_setup_phase[k];
  }
  plan_stats(b->plan, out);
  return HFX_OK;
}

// Autotuner: for every quartet class with work, time the class kernel alone on
// the batch (current P, K) for every (batch size, persistent grid) candidate
// and keep the fastest; the choice is reported through hfx_batch_get_tuning.
// The trial launches accumulate into K, which the next build zeroes.
hfx_status hfx_batch_autotune(hfx_batch* b, const double* const* P_vals, double* const* K_vals, void* stream) {
  if (!b || !P_vals || !K_vals) return fail(HFX_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  Plan& pl = b->plan;
  HFX_CK(cudaEventSynchronize(pl.sys_copied));
  batch_set_pointers(b, P_vals, K_vals);
  hfx_status st = plan_build(pl, s, false, false);  // Pmax and a warm cache
  if (st != HFX_OK) return st;
  HFX_CK(cudaStreamSynchronize(s));
  const bool mixed = pl.opts.precision == HFX_PREC_MIXED;
  const int fp32 = mixed ? 1 : 0;
  const int nblocks[3] = {32, 128, 512};
  cudaEvent_t e0, e1;
  HFX_CK(cudaEventCreate(&e0));
  HFX_CK(cudaEventCreate(&e1));
  for (int cls = 0; cls < HFX_NCLASS; ++cls) {
    if (pl.n_desc[cls] == 0) continue;
    const int occ = kClassOps[cls].occupancy_K(fp32);
    const int grids[3] = {occ * pl.n_sm, std::max(1, occ / 2) * pl.n_sm, 2 * occ * pl.n_sm};
    float best = 1e30f;
    int best_nb = pl.n_block[cls], best_g = grids[0];
    for (int inb = 0; inb < 3; ++inb) {
      st = plan_class_desc(pl, b->members, cls, nblocks[inb], s);
      if (st != HFX_OK) return st;
      for (int ig = 0; ig < 3; ++ig) {
        BuildArgs a = plan_args(pl, cls);
        a.route = 0;
        a.counter = pl.counters.p + cls;
        a.n_done = pl.n_done.p + 2 * cls;
        HFX_CK(cudaMemsetAsync(pl.counters.p + cls, 0, sizeof(int), s));
        HFX_CK(cudaEventRecord(e0, s));
        kClassOps[cls].launch_K(a, fp32, grids[ig], s);
        HFX_CK(cudaEventRecord(e1, s));
        HFX_CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
          best = ms;
          best_nb = nblocks[inb];
          best_g = grids[ig];
        }
      }
    }
    st = plan_class_desc(pl, b->members, cls, best_nb, s);
    if (st != HFX_OK) return st;
    pl.grid[fp32][cls] = best_g;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (pl.gexec) {  // launch shapes changed: capture again on the next graph build
    cudaGraphExecDestroy(pl.gexec);
    pl.gexec = nullptr;
  }
  b->tuned = true;
  HFX_CK(cudaGetLastError());
  return HFX_OK;
}

hfx_status hfx_batch_get_tuning(hfx_batch* b, int* n_block, int* grid) {
  if (!b || !n_block || !grid) return fail(HFX_ERR_INVALID_ARG, "NULL argument");
  const int fp32 = b->plan.opts.precision == HFX_PREC_MIXED ? 1 : 0;
  for (int c = 0; c < HFX_NCLASS; ++c) {
    n_block[c] = b->plan.n_desc[c] ? b->plan.n_block[c] : 0;
    grid[c] = b->plan.n_desc[c] ? plan_grid(b->plan, fp32, c) : 0;
  }
  return HFX_OK;
}

}  // extern "C"
