/*
 * hfx.h -- C ABI of the GB300 Hartree-Fock exchange (HFX) library.
 *
 * The library builds the exchange matrix of the paper's method (Sec. 2,
 * Eq. H-HFX, without its -1/2 factor)
 *
 *     K_ij = sum_kl (ik|jl) P_kl
 *
 * over contracted Cartesian Gaussian shells (s, p, d), with the full Coulomb
 * kernel 1/r (Sec. 2, full-range ERI definition) or the screened kernel
 * erfc(w r)/r (Sec. 2, Eq. ERI-SR), Schwarz screening (Sec. 2, Eq. schwarz),
 * density-matrix screening (Sec. 2, Eq. dmscreening), the 8-fold permutation
 * symmetry of the integrals (Sec. 2), sparse replicated P and K (Sec. 3), and
 * the exchange energy E_x = -1/2 sum_ij P_ij K_ij.  All compute runs in CUDA
 * kernels for sm_103a; the device work queue of the exchange kernels is the
 * single-GPU form of the paper's master/worker distribution (Sec. 3,
 * Algorithms 1-3).
 *
 * Conventions
 *   - Functions return hfx_status; no C++ exception crosses the ABI.  On error
 *     hfx_last_error() returns a message (thread-local, valid until the next
 *     call on the same thread).
 *   - "host" pointers are read during the call only and may be freed after it;
 *     "device" pointers are CUDA global memory owned by the caller.
 *   - Stream arguments are cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Asynchronous functions only enqueue work; device errors show
 *     up at the next synchronising call (hfx_exchange_energy, hfx_get_stats).
 *   - Handles are not thread-safe: use one per thread or lock around them.
 *   - Cartesian components are ordered x, y, z (p) and xx, xy, xz, yy, yz, zz
 *     (d).  A primitive x^l exp(-a r^2) is scaled to unit norm and the
 *     contracted shell to unit self-overlap of its x^l component.
 *   - Sparse matrices (P and K) are atom-pair-blocked: a symmetric pattern of
 *     atom pairs (X, Y) given as CSR over atoms; block (X, Y) holds the
 *     nf(X) x nf(Y) functions of the two atoms row-major; blocks follow the CSR
 *     order.  P and K use the same pattern and the same value layout (the
 *     paper keeps the density and exchange matrices in one sparse format,
 *     Sec. 3 and Table 1); K elements outside the pattern are not formed.
 */
#ifndef HFX_H
#define HFX_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HFX_OK = 0,
  HFX_ERR_INVALID_ARG = 1, /* bad argument or inconsistent input */
  HFX_ERR_OOM = 2,         /* device allocation failed */
  HFX_ERR_CUDA = 3,        /* CUDA runtime error (message has the detail) */
  HFX_ERR_UNSUPPORTED = 4, /* e.g. l > 2 or more than 16 primitives */
  HFX_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
  HFX_ERR_BUSY = 6         /* resource in use (server admission) */
} hfx_status;

typedef enum { HFX_KERNEL_COULOMB = 0, HFX_KERNEL_ERFC = 1, HFX_KERNEL_ERF = 2 } hfx_kernel;
typedef enum { HFX_PREC_FP64 = 0, HFX_PREC_MIXED = 1 } hfx_precision;

/* One contracted shell.  alpha/coef: host arrays of nprim exponents (bohr^-2)
 * and raw contraction coefficients (the library normalises them). */
typedef struct {
  int l;       /* 0, 1 or 2 */
  int nprim;   /* 1..16 */
  int atom;    /* index into the atom array; shells must be grouped by atom in atom order */
  int reserved;
  const double* alpha;
  const double* coef;
} hfx_shell_desc;

/* Options of one quartet list (fixed for its lifetime, like the paper's
 * pre-SCF pair lists, Sec. 2). */
typedef struct {
  int kernel;                 /* hfx_kernel */
  double omega;               /* bohr^-1, erf/erfc kernels (HSE06: 0.11, Sec. 2) */
  int screen;                 /* 1: Schwarz test Q_IJ Q_KL > tau and exact P_scr > 0 skip */
  double tau;                 /* Schwarz drop tolerance (Sec. 2, Eq. schwarz) */
  int density_screen;         /* 1: also require P_scr Q_IJ Q_KL > eps (Eq. dmscreening) */
  double eps;                 /* density-screening threshold */
  double prim_cutoff;         /* skip primitive quartets whose bound estimate product is below this (0: keep all) */
  int precision;              /* hfx_precision */
  double fp64_promote_bound;  /* MIXED: quartets with Q_IJ Q_KL P_scr above this run in FP64 */
  int n_block;                /* quartets per work-queue batch (the paper's n_block, Sec. 4); 0 = default */
  int promote_min_l;          /* MIXED: promotion only in classes with la+lb+lc+ld >= this (0: every class) */
  int prim_density_screen;    /* 1: prim_cutoff applies to bound_ab bound_cd P_scr (the largest |P| the quartet
                                 contracts with, Eq. dmscreening) instead of bound_ab bound_cd */
  int promote_prims;          /* MIXED with promotion: 1 = promote per primitive quartet: of a quartet above
                                 fp64_promote_bound only the primitive quartets with bound_ab bound_cd P_scr
                                 above it run in FP64, the others in FP32 */
  int spherical;              /* 1: P and K in real solid harmonics, 2l+1 per shell (Sec. 2: the Cartesian
                                 integrals are transformed to spherical harmonics); order per d shell:
                                 xy, yz, z^2, xz, x^2-y^2 (s, p unchanged); not for batches or the server */
  double extent_eps;          /* > 0: distance screening (Sec. 2, with the NAO cutoff radii replaced by Gaussian
                                 extents): shell S reaches R_S = sqrt(ln(1/extent_eps) / alpha_min(S)), the radius
                                 where its most diffuse primitive exp(-alpha r^2) falls to extent_eps; shell pairs
                                 farther apart than R_A + R_B are dropped before their Schwarz bounds are formed.
                                 0: off */
  int reserved2[2];
} hfx_opts;

/* Atom-pair block pattern: CSR over atoms (host arrays). */
typedef struct {
  int n_atoms;
  const int* row_ptr; /* n_atoms + 1 */
  const int* col;     /* row_ptr[n_atoms] atom indices, sorted within each row */
} hfx_pattern;

typedef struct hfx_basis_s hfx_basis;
typedef struct hfx_quartets_s hfx_quartets;
typedef struct hfx_batch_s hfx_batch;

/* Statistics of the most recent hfx_build_K on a quartet list. */
typedef struct {
  long long n_pairs_significant[6];   /* shell pairs kept per pair class (ss ps pp ds dp dd) */
  long long n_quartets_schwarz[21];   /* canonical quartets passing the Schwarz test, per class */
  long long n_quartets_computed[21];  /* quartets evaluated in the last build (after density screening) */
  long long n_prim_pairs;             /* primitive pairs kept over all significant shell pairs */
  long long n_values;                 /* length of the P / K value arrays */
  float ms_setup;                     /* hfx_build_quartets wall time */
  float ms_last_build;                /* device time of the last hfx_build_K (events) */
  /* per launch of the last build: pass 0 = FP64 path or the FP32 part of the
   * mixed path, pass 1 = the FP64-promoted part of the mixed path */
  long long n_quartets_pass[2][21];
  long long n_prim_quartets_pass[2][21]; /* primitive quartets evaluated */
  float ms_class_pass[2][21];            /* device time of each class kernel (events) */
  float ms_setup_phase[4];               /* setup: pairs, Schwarz bounds, sorted pair lists, work queues */
  long long n_pairs_distance;            /* shell pairs the distance screening kept (all pairs when it is off) */
} hfx_stats;

/* Class table entry (for throughput and roofline accounting). */
typedef struct {
  int bra_class, ket_class;   /* pair classes 0..5 = ss ps pp ds dp dd */
  int la, lb, lc, ld;
  int n_out;                  /* Cartesian integrals per quartet */
  int vrr_flops;              /* flops of the vertical recursion per primitive quartet */
  int hrr_flops;              /* flops of the horizontal recursion per quartet */
  int n_acc;                  /* contracted [e0|f0] accumulators per quartet */
  int kernel_kind;            /* 0 per-thread k_build_K, 1 warp-split k_build_K_split, 2 cooperative k_build_K_coop */
} hfx_class_info;

/* Basis creation (setup).  Copies shells, normalises contraction coefficients
 * on the device (Sec. 2: contracted GTO shells) and builds the Boys table.
 * atom_xyz: host, n_atoms x 3 (bohr).  stream: work is enqueued on it and
 * synchronised before return.  *out must be released with hfx_destroy_basis. */
hfx_status hfx_create_basis(const hfx_shell_desc* shells, int n_shells, const double* atom_xyz, int n_atoms,
                            void* stream, hfx_basis** out);

/* Pre-SCF setup (Sec. 2): shell-pair records, Schwarz bounds with the run's
 * kernel, significant pair lists sorted per class by descending bound, and
 * the work-queue batches of canonical quartets (I>=J, K>=L, IJ>=KL) that pass
 * the Schwarz test, grouped by angular-momentum class.  pattern: the sparsity
 * pattern of P and K (must be symmetric and contain every diagonal block).
 * Synchronises the stream before return. */
hfx_status hfx_build_quartets(hfx_basis* basis, const hfx_opts* opts, const hfx_pattern* pattern, void* stream,
                              hfx_quartets** out);

/* Number of doubles in the P / K value arrays of this pattern (in the
 * spherical layout when opts.spherical). */
long long hfx_value_count(const hfx_quartets* q);

/* One exchange build (Algorithm 4): zero K, shell-pair Pmax of P, screened ERI
 * evaluation with the fused exchange contraction, symmetrisation.  P_val, K_val:
 * device arrays of hfx_value_count() doubles.  Asynchronous on `stream`. */
hfx_status hfx_build_K(hfx_quartets* q, const double* P_val, double* K_val, void* stream);

/* One rank's share of a build sharded over n_ranks processes (one GPU each):
 * the work-queue batches of every quartet class with index % n_ranks == rank,
 * the interleaved static split of the paper's distributed construction
 * (Sec. 3, Algorithms 3 and 4).  K_val receives the symmetrised exchange of
 * that share (zeroed first); the sum of the K_val arrays over the ranks -- the
 * sum all-reduce of Algorithm 4 (MPI_ALLREDUCE in the paper, NCCL here) -- is
 * the K of hfx_build_K.  Every rank needs the whole P_val.  Asynchronous on
 * `stream`; HFX_ERR_INVALID_ARG unless 0 <= rank < n_ranks. */
hfx_status hfx_build_K_shard(hfx_quartets* q, const double* P_val, double* K_val, int rank, int n_ranks,
                             void* stream);

/* Incremental build: K_val += K(dP_val).  K is linear in the density
 * (Eq. H-HFX), so an SCF step n can form K(P_n) = K(P_{n-1}) + K(P_n - P_{n-1}).
 * The density screening (Eq. dmscreening) then uses the shell maxima of the
 * difference, which is small near convergence, so fewer quartets survive.
 * dP_val, K_val: device arrays of hfx_value_count() doubles; K_val holds the
 * previous exchange matrix (symmetric, as hfx_build_K leaves it).  The change
 * is built into a scratch array the quartet list keeps (hfx_value_count()
 * doubles, allocated on first use) and added to K_val.  Asynchronous on
 * `stream`; hfx_get_stats reports the quartets of the difference build. */
hfx_status hfx_build_K_delta(hfx_quartets* q, const double* dP_val, double* K_val, void* stream);

/* E_x = -1/2 sum_ij P_ij K_ij over the pattern (device reduction, FP64).
 * Synchronises the stream; *E_x is a host double. */
hfx_status hfx_exchange_energy(hfx_quartets* q, const double* P_val, const double* K_val, double* E_x,
                               void* stream);

/* Dense <-> block-sparse conversion on the device (dense: nbf x nbf row-major,
 * nbf counting 2l+1 functions per shell when opts.spherical).
 * Pack reads only the pattern's blocks; unpack writes zeros outside it. */
hfx_status hfx_pack_dense(const hfx_quartets* q, const double* dense, double* val, void* stream);
hfx_status hfx_unpack_dense(const hfx_quartets* q, const double* val, double* dense, void* stream);

/* Contracted integrals of arbitrary shell quartets (diagnostics and tests).
 * quartets: host, n x 4 shell indices (I J | K L); out_off: host, n offsets;
 * out: device; quartet q writes nI*nJ*nK*nL doubles at out + out_off[q] in
 * (i, j, k, l) row-major order.  precision selects the FP64 or mixed path.
 * Synchronises the stream. */
hfx_status hfx_eval_quartets(hfx_basis* basis, int kernel, double omega, int precision, int n,
                             const int* quartets, const long long* out_off, double* out, void* stream);

/* Boys function F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt, m = 0..mmax (mmax <= 8),
 * as the ERI kernels evaluate it (diagnostics and tests): precision FP64 uses
 * the FP64 Taylor/downward-recursion evaluator, MIXED the double-single one.
 * T: device array of n arguments (>= 0); F: device array of n x (mmax+1),
 * row-major.  Synchronises the stream. */
hfx_status hfx_boys_eval(hfx_basis* basis, int precision, int mmax, int n, const double* T, double* F,
                         void* stream);

/* E_x = -1/2 sum_i P_val[i] K_val[i] without allocating any device memory
 * (no counterpart in the paper).  For callers that cannot call cudaMalloc --
 * processes held to a fixed device-memory budget, hosts whose allocator owns
 * every device allocation, plugins that must not allocate -- and that have no
 * quartet-list handle.  P_val, K_val: device arrays of n_values doubles;
 * E_x: device pointer to one double, written asynchronously on `stream`.
 * Scratch is a static device array of 2^16 doubles (512 KiB, held on every
 * GPU that loads the library until exit); n_values above 2^28 is rejected with
 * HFX_ERR_INVALID_ARG.  Every call looks up the array's device address
 * (cudaGetSymbolAddress, no allocation), so a device reset in between is
 * harmless; the first call on a device may load the module, so make it
 * before any stream capture.
 * Every call shares the array, so calls that overlap on the GPU race: serialise
 * them.  The reduction order is fixed (two passes, no atomics). */
hfx_status hfx_exchange_energy_noalloc(const double* P_val, const double* K_val, long long n_values, double* E_x,
                                       void* stream);

/* Statistics (synchronises the device). */
hfx_status hfx_get_stats(const hfx_quartets* q, hfx_stats* out);

/* ---- Batches: several independent systems in one build ----------------
 * A batch runs the exchange builds of its members (quartet lists that share
 * kernel, precision and screening options) together: one launch per quartet
 * class over the work queues of all members, one launch for each of the small
 * per-build kernels.  With use_graph the whole build is captured once as a
 * CUDA graph (class kernels on parallel branches) and replayed afterwards;
 * P and K pointers are read through a system table that the graph copies from
 * pinned host memory, so they may change between builds.  Members must outlive
 * the batch. */
hfx_status hfx_batch_create(hfx_quartets* const* members, int n, void* stream, hfx_batch** out);

/* One build of every member: P_vals[i], K_vals[i] device arrays of member i's
 * value count.  Asynchronous on `stream`. */
hfx_status hfx_batch_build_K(hfx_batch* b, const double* const* P_vals, double* const* K_vals, int use_graph,
                             void* stream);

/* E_x of every member from the last build (host array of n doubles); syncs. */
hfx_status hfx_batch_energies(hfx_batch* b, double* E_x, void* stream);

/* Autotuner: times every quartet class alone over the batch for each work-queue
 * batch size (32, 128, 512 quartets) and persistent grid (1/2, 1, 2 x the
 * occupancy limit) and keeps the fastest per class.  Leaves K holding trial
 * sums (the next build zeroes it).  Synchronises. */
hfx_status hfx_batch_autotune(hfx_batch* b, const double* const* P_vals, double* const* K_vals, void* stream);

/* Per-class batch size and grid in use (arrays of 21; 0 for classes without work). */
hfx_status hfx_batch_get_tuning(hfx_batch* b, int* n_block, int* grid);

/* Statistics summed over members (synchronises). */
hfx_status hfx_batch_get_stats(hfx_batch* b, hfx_stats* out);

void hfx_batch_destroy(hfx_batch* b);

/* ---- Memory accounting and host-side value layout ---------------------- */

/* Device bytes held by a quartet list (pairs, primitive pairs, work queues,
 * pattern tables, Pmax, build plan) or by a basis; -1 for NULL. */
long long hfx_quartets_device_bytes(const hfx_quartets* q);
long long hfx_basis_device_bytes(const hfx_basis* basis);

/* Number of P / K values of a pattern over these shells (host only; the same
 * count hfx_value_count reports once the quartet list exists); -1 when the
 * shells or the pattern are inconsistent. */
long long hfx_pattern_value_count(const hfx_shell_desc* shells, int n_shells, const hfx_pattern* pattern);

/* Host-side pack of a dense nbf x nbf row-major matrix into the pattern's
 * value layout (blocks in CSR order, row-major inside a block). */
hfx_status hfx_pack_dense_host(const hfx_shell_desc* shells, int n_shells, const hfx_pattern* pattern,
                               const double* dense, double* val);

/* Upper estimate of the device bytes a basis plus hfx_build_quartets need at
 * their peak for these shells and pattern (all shell pairs with their
 * primitive pairs during setup, plus what stays resident); -1 on bad input. */
long long hfx_setup_bytes_estimate(const hfx_shell_desc* shells, int n_shells, const hfx_pattern* pattern);

/* ---- Periodic systems (Sec. 2, Eq. H-HFX) ------------------------------
 * The periodic exchange K^G_{mu lambda} = sum_{N,H} sum_{nu sigma}
 * P^{H-N}_{nu sigma} (mu^0 nu^N | lambda^G sigma^H) (mu in the home cell; N, G,
 * H cells of the auxiliary supercell) is built on an extended atom set: the
 * home atoms (extended atoms 0..n_home-1, in home order) followed by the
 * images, each image carrying its home atom's shells at the translated
 * centre.  hfx_create_basis_periodic builds that set inside the library;
 * hfx_build_quartets on such a basis evaluates only the quartets with at least
 * one home-cell shell (the paper's list-IJ with I in the unit cell: every
 * integral (mu^0 nu | lambda sigma) of a home row is one of them), and
 * hfx_build_K returns the home rows K^G (the leading rows of the value
 * layout) with every row of an image atom set to zero.  hfx_exchange_energy
 * then gives the exchange energy per cell, -1/2 sum over the home rows of P K. */

/* Periodic basis.  shells, atom_xyz: the home cell as for hfx_create_basis;
 * lattice: host, 3 x 3, lattice vectors a_i as rows (bohr); r_ext (bohr): the
 * images are the translates R_a + n1 a1 + n2 a2 + n3 a3 (n != 0) of home atoms
 * that lie within r_ext of at least one home atom, in the order of
 * hfx_periodic_images.  Errors as hfx_create_basis and hfx_periodic_images
 * (HFX_ERR_INVALID_ARG for a singular lattice or a negative r_ext).
 * Synchronises the stream; release with hfx_destroy_basis. */
hfx_status hfx_create_basis_periodic(const hfx_shell_desc* shells, int n_shells, const double* atom_xyz, int n_atoms,
                                     const double* lattice, double r_ext, void* stream, hfx_basis** out);

/* Atoms of a basis: returns their number (the extended set for a periodic
 * basis), -1 for NULL.  n_home_atoms (may be NULL): home atoms (all atoms of
 * a molecular basis); ext_home (may be NULL): per atom its home atom;
 * ext_shift (may be NULL): per atom its lattice shift (n1, n2, n3), zero for
 * home atoms.  Host arrays sized by the return value. */
int hfx_basis_atoms(const hfx_basis* basis, int* n_home_atoms, int* ext_home, int* ext_shift);

/* Extended atom set of a periodic cell (host only; the set
 * hfx_create_basis_periodic builds): the n_atoms home atoms, then the images of
 * hfx_periodic_images in its order.  Returns the number of extended atoms, -1
 * on bad input (message in hfx_last_error).  The first min(count, max_atoms)
 * are written: ext_home (home atom), ext_shift (n1, n2, n3; zero for home
 * atoms), ext_xyz (R_home + n1 a1 + n2 a2 + n3 a3, bohr); call with
 * max_atoms = 0 to size the arrays. */
long long hfx_periodic_extend(const double* atom_xyz, int n_atoms, const double* lattice, double r_ext,
                              long long max_atoms, int* ext_home, int* ext_shift, double* ext_xyz);

/* Distance pattern (host only): every pair of the n_atoms atoms at most r_cut
 * bohr apart, and every diagonal pair, as CSR with columns ascending.
 * Returns the number of pairs, -1 on bad input.  row_ptr (n_atoms + 1 ints)
 * and col (first max_nnz pairs) may be NULL: call once to size col.  On a
 * periodic cell's extended atoms with r_cut the density cutoff this is the
 * pattern of the real-space density P^{H-N} (Eq. dm at the Gamma point) and of
 * the exchange rows. */
long long hfx_distance_pattern(const double* atom_xyz, int n_atoms, double r_cut, int* row_ptr, int* col,
                               long long max_nnz);

/* Image table: every translate R_a + n1 a1 + n2 a2 + n3 a3 (n != 0) of a home
 * atom a lying within r_ext (bohr) of at least one home atom.
 * atom_xyz: host, n_atoms x 3; lattice: host, 3 x 3, lattice vectors a_i as
 * rows (bohr).  Images are ordered by shift (n1, n2, n3 lexicographic) and
 * then by atom.  The first min(count, max_images) are written to image_atom
 * (home atom) and image_shift (n1, n2, n3 per image); call with
 * max_images = 0 to size the arrays.  Returns the number of images, or -1
 * (message in hfx_last_error) for NULL input, a singular lattice, a negative
 * r_ext or a search beyond 1000 cells per direction. */
long long hfx_periodic_images(const double* atom_xyz, int n_atoms, const double* lattice, double r_ext,
                              long long max_images, int* image_atom, int* image_shift);

/* Real-space density of the extended set (Eq. dm at the Gamma point): for
 * every block (X, Y) of ext_pattern (CSR over the extended atoms, normally
 * the pairs within the density cutoff), the home-cell block
 * P_home(ext_home[X], ext_home[Y]) is written to val in the pattern's value
 * layout (blocks in CSR order, row-major inside a block).
 * shells: the n_shells home shells (atom < n_home_atoms, grouped by atom);
 * ext_home: host, ext_pattern->n_atoms home-atom indices; P_home: host, dense
 * home nbf x nbf row-major; val: host, hfx_pattern_value_count of the
 * extended shells and ext_pattern. */
hfx_status hfx_periodic_pack_host(const hfx_shell_desc* shells, int n_shells, int n_home_atoms, const int* ext_home,
                                  const hfx_pattern* ext_pattern, const double* P_home, double* val);

/* Real-space density of the extended set from one density block per lattice
 * vector (Eq. dm with a k-point grid: the caller forms
 * P^L = (1/N_k) sum_k exp(-i k.L) P(k), real for a grid closed under k -> -k,
 * with P^{-L} = (P^L)^T).  Every block (X, Y) of ext_pattern receives the
 * home block P^{n_Y - n_X}(home(X), home(Y)), n the lattice shifts of the
 * extended atoms (hfx_periodic_extend), from P_L[l] where L_shift[l] equals
 * n_Y - n_X; a shift difference not in the list gives a zero block.  With one
 * P_L for every shift difference this is hfx_periodic_pack_host.
 * ext_shift: host, 3 per extended atom; L_shift: host, n_L x 3; P_L: host,
 * n_L x nbf x nbf (home functions, row-major); val as for
 * hfx_periodic_pack_host.  The exchange rows built from these values are
 * K^G_{mu lambda} = sum_{N,H} P^{H-N} (mu^0 nu^N | lambda^G sigma^H) of
 * Eq. H-HFX; the caller's Fourier sum over G gives K(k). */
hfx_status hfx_periodic_pack_lattice_host(const hfx_shell_desc* shells, int n_shells, int n_home_atoms,
                                          const int* ext_home, const int* ext_shift, const hfx_pattern* ext_pattern,
                                          int n_L, const int* L_shift, const double* P_L, double* val);

/* ---- Serving: continuous batching of independent requests -------------
 * No counterpart in the paper, whose runs build one system's K once per SCF
 * iteration; a server interleaves many such SCF-like runs on one GPU.
 * A request is one system with n_builds density matrices; it is set up once
 * (basis, Schwarz pair lists, work queues: Sec. 2) and its builds run while
 * it stays resident.  hfx_server_step() admits queued requests in arrival
 * order while their estimated device memory (hfx_setup_bytes_estimate plus
 * the P and K arrays) fits under mem_budget -- a request larger than the
 * whole budget fails with HFX_ERR_OOM, otherwise the queue head waits for
 * retirements --, runs one build of every active request (requests sharing
 * kernel, precision and screening options share one batched build, see the
 * batch functions), and retires finished requests.  The setup of requests
 * admitted while others are active runs on a second stream of the server,
 * during the active requests' builds, and they join at the next step.  One
 * host thread drives a server (not thread-safe); builds run on the stream
 * given at creation, and hfx_server_step() synchronises both streams. */
typedef struct hfx_server_s hfx_server;

typedef enum {
  HFX_REQ_QUEUED = 0,
  HFX_REQ_ACTIVE = 1,
  HFX_REQ_DONE = 2,
  HFX_REQ_FAILED = 3,
  HFX_REQ_CANCELLED = 4
} hfx_request_state;

typedef struct {
  long long mem_budget; /* device bytes for admitted requests; <= 0: 80% of the free memory at creation */
  int max_active;       /* at most this many active requests; <= 0: 64 */
  int use_graph;        /* capture each batched build as a CUDA graph (re-captured when the active set changes) */
  int incremental;      /* builds after a request's first: K(P_n) = K(P_{n-1}) + K(P_n - P_{n-1}), the difference
                           screened on its own shell maxima (twice the P/K device arrays per request) */
  int reserved[3];
} hfx_server_opts;

typedef struct {
  int state;              /* hfx_request_state */
  int status;             /* hfx_status of a failed request (HFX_OK otherwise) */
  int builds_done;
  int n_builds;
  double t_submit;        /* seconds since hfx_server_create; -1 = not yet */
  double t_admit;
  double t_done;
  long long device_bytes; /* device bytes held while active */
} hfx_request_info;

typedef struct {
  long long mem_budget;
  long long used_bytes;      /* held by active requests */
  long long peak_used_bytes;
  long long builds_done;
  long long steps;
  int n_queued, n_active, max_active_seen, reserved;
} hfx_server_info;

hfx_status hfx_server_create(const hfx_server_opts* opts, void* stream, hfx_server** out);

/* Queue a request.  shells, atom_xyz, pattern, opts: copied.  P_host: host
 * array of n_builds x value-count doubles (build i reads row i), owned by the
 * caller and read until the request is done.  K_out: host array of
 * value-count doubles receiving the K of the last build (may be NULL), owned
 * by the caller.  *ticket identifies the request. */
hfx_status hfx_server_submit(hfx_server* srv, const hfx_shell_desc* shells, int n_shells, const double* atom_xyz,
                             int n_atoms, const hfx_pattern* pattern, const hfx_opts* opts, int n_builds,
                             const double* P_host, double* K_out, long long* ticket);

/* Queue a periodic request (Sec. 2, Eq. H-HFX): the home cell (shells,
 * atom_xyz, lattice as rows, r_ext) as for hfx_create_basis_periodic, which
 * its setup calls; ext_pattern: the density pattern over the extended atoms
 * (hfx_periodic_extend, e.g. hfx_distance_pattern); P_host: n_builds x value
 * count doubles in that layout (hfx_periodic_pack_host); K_out as for
 * hfx_server_submit (image rows zero).  Energies are per cell. */
hfx_status hfx_server_submit_periodic(hfx_server* srv, const hfx_shell_desc* shells, int n_shells,
                                      const double* atom_xyz, int n_atoms, const double* lattice, double r_ext,
                                      const hfx_pattern* ext_pattern, const hfx_opts* opts, int n_builds,
                                      const double* P_host, double* K_out, long long* ticket);

/* Admission, one build of every active request, retirement (see above).
 * *n_active (may be NULL): active requests after the step. */
hfx_status hfx_server_step(hfx_server* srv, int* n_active);

/* State of a request; E_x (may be NULL): host array of n_builds, the energies
 * of the builds done so far. */
hfx_status hfx_server_poll(hfx_server* srv, long long ticket, hfx_request_info* info, double* E_x);

/* Cancel a request: a queued one leaves the queue at once, an active one at
 * the next step boundary (its device memory is then released); its state
 * becomes HFX_REQ_CANCELLED.  HFX_ERR_BUSY for a finished request. */
hfx_status hfx_server_cancel(hfx_server* srv, long long ticket);

/* Test hook (failure injection on the host, no device fault): the setup of a
 * still-queued request fails with `status` when it is admitted, as a failed
 * allocation or build would; the other requests are unaffected. */
hfx_status hfx_server_inject_setup_failure(hfx_server* srv, long long ticket, int status);

/* Forget a finished (done, failed or cancelled) request; HFX_ERR_BUSY otherwise. */
hfx_status hfx_server_release(hfx_server* srv, long long ticket);

hfx_status hfx_server_get_info(hfx_server* srv, hfx_server_info* out);
void hfx_server_destroy(hfx_server* srv);

/* Static per-class information; cls in [0, 21). */
hfx_status hfx_get_class_info(int cls, hfx_class_info* out);

void hfx_destroy_basis(hfx_basis* basis);
void hfx_destroy_quartets(hfx_quartets* q);
const char* hfx_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HFX_H */
