// hfx_server.cu -- continuous-batching exchange server.
//
// Requests are independent systems, each asking for a short sequence of
// exchange builds (an SCF-like run: one build per density matrix it supplies,
// with the pair lists and work queues of the system set up once and kept
// resident on the device between its builds; Sec. 2 sets the screening lists
// up before the SCF loop for the same reason).
//
// Each hfx_server_step():
//   1. launches one build of every active request: requests with the same
//      kernel, precision and screening options share one batched build (one
//      launch per quartet class over all of their work queues, hfx_batch_*),
//      whose plan is rebuilt only when the active set changes;
//   2. while those builds run, admits queued requests in arrival order while
//      the device memory they are estimated to need fits under the server's
//      budget (a request that could never fit fails with HFX_ERR_OOM; the head
//      of the queue waits otherwise) and runs their setup on a second stream,
//      so arrivals do not stall the active requests; they join at the next
//      step (when nothing is active they are admitted first and built at once);
//   3. collects the energies and retires the requests whose last build is
//      done: copies their last K to the caller's host array, frees their
//      device memory.
// With `incremental`, every build of a request after its first is built from
// the density difference: K(P_n) = K(P_{n-1}) + K(P_n - P_{n-1}) (K is linear
// in P, Eq. H-HFX), the difference screened on its own shell maxima
// (Eq. dmscreening), which are small between SCF-like iterations.
// Periodic requests (hfx_server_submit_periodic) are set up on the library's
// periodic basis and build the home rows K^G (the energy is per cell).
//
// One host thread drives a server; its calls are not thread-safe.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "hfx.h"

void hfx_set_last_error(const std::string& m);

namespace {

hfx_status srv_fail(hfx_status s, const std::string& m) {
  hfx_set_last_error(m);
  return s;
}

bool same_options(const hfx_opts& a, const hfx_opts& b) {
  return a.kernel == b.kernel && a.omega == b.omega && a.precision == b.precision && a.screen == b.screen &&
         a.tau == b.tau && a.density_screen == b.density_screen && a.eps == b.eps && a.prim_cutoff == b.prim_cutoff &&
         (a.fp64_promote_bound == b.fp64_promote_bound ||
          (a.fp64_promote_bound != a.fp64_promote_bound && b.fp64_promote_bound != b.fp64_promote_bound)) &&
         a.promote_min_l == b.promote_min_l && a.prim_density_screen == b.prim_density_screen &&
         a.promote_prims == b.promote_prims;
}

// new P of one build into d, and d - P into d, P := new (incremental builds)
__global__ void k_delta_in(long long n, double* __restrict__ d, double* __restrict__ P) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double t = d[i];
    d[i] = t - P[i];
    P[i] = t;
  }
}

__global__ void k_add_into(long long n, const double* __restrict__ x, double* __restrict__ y) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) y[i] += x[i];
}

// E[slot] = -1/2 sum_i P_i K_i (E zeroed before; one atomicAdd per block)
__global__ void k_energy_into(long long n, const double* __restrict__ P, const double* __restrict__ K, double* E) {
  double v = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) v = fma(P[i], K[i], v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __shared__ double w[8];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += w[k];
    atomicAdd(E, -0.5 * t);
  }
}

unsigned grid_for(long long n) { return (unsigned)std::max<long long>(1, std::min<long long>(1024, (n + 255) / 256)); }

struct Request {
  long long ticket = 0;
  hfx_request_info info{};
  // inputs (host copies; P and the K destination stay owned by the caller)
  std::vector<hfx_shell_desc> shells;
  std::vector<double> prim;  // alpha then coef of every shell, back to back
  std::vector<double> xyz;
  int n_atoms = 0;               // atoms of xyz (the home cell of a periodic request)
  int pattern_atoms = 0;         // atoms of the pattern (the extended set of a periodic request)
  bool periodic = false;
  double lattice[9] = {0};
  double r_ext = 0.0;
  std::vector<int> row_ptr, col;
  hfx_opts opts{};
  const double* P_host = nullptr;  // n_builds x n_values
  double* K_out = nullptr;         // n_values, written when the last build is done
  long long n_values = 0;
  long long estimate = 0;
  bool cancel = false;          // retire at the next step boundary
  hfx_status inject = HFX_OK;   // test hook: the next setup fails with this status
  std::vector<double> E;
  // device state while active
  hfx_basis* basis = nullptr;
  hfx_quartets* q = nullptr;
  double* P = nullptr;
  double* K = nullptr;
  double* dP = nullptr;  // incremental builds: density difference and its exchange
  double* dK = nullptr;

  hfx_pattern pattern() const {
    hfx_pattern p;
    p.n_atoms = pattern_atoms;
    p.row_ptr = row_ptr.data();
    p.col = col.data();
    return p;
  }
  void release_device() {
    if (q) hfx_destroy_quartets(q);
    if (basis) hfx_destroy_basis(basis);
    if (P) cudaFree(P);
    if (K) cudaFree(K);
    if (dP) cudaFree(dP);
    if (dK) cudaFree(dK);
    q = nullptr;
    basis = nullptr;
    P = K = dP = dK = nullptr;
  }
  ~Request() { release_device(); }
};

struct Group {
  hfx_opts opts{};
  std::vector<Request*> members;
  hfx_batch* batch = nullptr;
};

}  // namespace

struct hfx_server_s {
  hfx_server_opts o{};
  cudaStream_t stream = nullptr;
  cudaStream_t setup_stream = nullptr;  // admissions overlap the active builds
  double* energies = nullptr;           // incremental builds: per-member energies of a group
  size_t n_energies = 0;
  std::chrono::steady_clock::time_point t0;
  long long next_ticket = 1;
  std::deque<Request*> queue;
  std::vector<Request*> active;
  std::map<long long, std::unique_ptr<Request>> all;
  std::vector<Group> groups;
  bool dirty = true;
  hfx_server_info stats{};

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  void drop_groups() {
    for (auto& g : groups)
      if (g.batch) hfx_batch_destroy(g.batch);
    groups.clear();
    dirty = true;
  }
  ~hfx_server_s() {
    drop_groups();
    if (setup_stream) cudaStreamDestroy(setup_stream);
    if (energies) cudaFree(energies);
  }
};

namespace {

void finish(hfx_server_s* s, Request* r, int state, hfx_status st) {
  r->info.state = state;
  r->info.status = st;
  r->info.t_done = s->now();
  if (r->info.device_bytes > 0) s->stats.used_bytes -= r->info.device_bytes;
  r->release_device();
}

// Setup of an admitted request: basis, quartet lists, P and K buffers.
hfx_status setup_request(hfx_server_s* s, Request* r) {
  if (r->inject != HFX_OK) {  // failure injected on the host (tests)
    const hfx_status st = r->inject;
    r->inject = HFX_OK;
    return srv_fail(st, "injected setup failure");
  }
  hfx_status st = r->periodic ? hfx_create_basis_periodic(r->shells.data(), (int)r->shells.size(), r->xyz.data(),
                                                          r->n_atoms, r->lattice, r->r_ext, s->setup_stream, &r->basis)
                               : hfx_create_basis(r->shells.data(), (int)r->shells.size(), r->xyz.data(), r->n_atoms,
                                                  s->setup_stream, &r->basis);
  if (st != HFX_OK) return st;
  const hfx_pattern pat = r->pattern();
  st = hfx_build_quartets(r->basis, &r->opts, &pat, s->setup_stream, &r->q);
  if (st != HFX_OK) return st;
  const size_t bytes = (size_t)std::max<long long>(r->n_values, 1) * sizeof(double);
  const int n_arrays = s->o.incremental ? 4 : 2;
  cudaError_t e = cudaMalloc(&r->P, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&r->K, bytes);
  if (e == cudaSuccess && s->o.incremental) e = cudaMalloc(&r->dP, bytes);
  if (e == cudaSuccess && s->o.incremental) e = cudaMalloc(&r->dK, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return srv_fail(e == cudaErrorMemoryAllocation ? HFX_ERR_OOM : HFX_ERR_CUDA,
                    std::string("request buffers: ") + cudaGetErrorString(e));
  }
  r->info.device_bytes =
      hfx_basis_device_bytes(r->basis) + hfx_quartets_device_bytes(r->q) + n_arrays * (long long)bytes;
  return HFX_OK;
}

// Admission into `into` (the active set, or the requests joining it at the
// end of this step); `holding`: requests already holding device memory.
hfx_status admit(hfx_server_s* s, std::vector<Request*>& into, size_t holding) {
  while (!s->queue.empty() && holding + into.size() < (size_t)s->o.max_active) {
    Request* r = s->queue.front();
    if (r->estimate > s->o.mem_budget) {
      s->queue.pop_front();
      finish(s, r, HFX_REQ_FAILED, HFX_ERR_OOM);
      continue;
    }
    if (s->stats.used_bytes + r->estimate > s->o.mem_budget && holding + into.size() > 0)
      break;  // wait for retirements
    s->queue.pop_front();
    r->info.t_admit = s->now();
    const hfx_status st = setup_request(s, r);
    if (st != HFX_OK) {
      r->info.device_bytes = 0;
      finish(s, r, HFX_REQ_FAILED, st);
      continue;
    }
    r->info.state = HFX_REQ_ACTIVE;
    s->stats.used_bytes += r->info.device_bytes;
    s->stats.peak_used_bytes = std::max(s->stats.peak_used_bytes, s->stats.used_bytes);
    into.push_back(r);
  }
  s->stats.max_active_seen = std::max(s->stats.max_active_seen, (int)(holding + into.size()));
  return HFX_OK;
}

hfx_status regroup(hfx_server_s* s) {
  s->drop_groups();
  for (Request* r : s->active) {
    Group* g = nullptr;
    for (auto& x : s->groups)
      if (same_options(x.opts, r->opts)) g = &x;
    if (!g) {
      s->groups.emplace_back();
      g = &s->groups.back();
      g->opts = r->opts;
    }
    g->members.push_back(r);
  }
  for (auto& g : s->groups) {
    std::vector<hfx_quartets*> m;
    for (Request* r : g.members) m.push_back(r->q);
    const hfx_status st = hfx_batch_create(m.data(), (int)m.size(), s->stream, &g.batch);
    if (st != HFX_OK) return st;
  }
  s->dirty = false;
  return HFX_OK;
}

}  // namespace

extern "C" {

hfx_status hfx_server_create(const hfx_server_opts* opts, void* stream, hfx_server** out) {
  if (!out) return srv_fail(HFX_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  std::unique_ptr<hfx_server_s> s(new hfx_server_s());
  if (opts) s->o = *opts;
  if (s->o.max_active <= 0) s->o.max_active = 64;
  if (s->o.mem_budget <= 0) {
    size_t fr = 0, tot = 0;
    const cudaError_t e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) return srv_fail(HFX_ERR_CUDA, std::string("cudaMemGetInfo: ") + cudaGetErrorString(e));
    s->o.mem_budget = (long long)(0.8 * (double)fr);
  }
  s->stream = (cudaStream_t)stream;
  const cudaError_t es = cudaStreamCreateWithFlags(&s->setup_stream, cudaStreamNonBlocking);
  if (es != cudaSuccess) return srv_fail(HFX_ERR_CUDA, std::string("setup stream: ") + cudaGetErrorString(es));
  s->t0 = std::chrono::steady_clock::now();
  s->stats.mem_budget = s->o.mem_budget;
  *out = s.release();
  return HFX_OK;
}

}  // extern "C"

namespace {

// Queue a request: shells, coordinates (n_atoms: home cell of a periodic
// request), the pattern over pattern_shells (the extended shells of a
// periodic request), options, densities and the K destination.
hfx_status submit_common(hfx_server* s, const hfx_shell_desc* shells, int n_shells, const double* atom_xyz,
                         int n_atoms, const hfx_shell_desc* pattern_shells, int n_pattern_shells,
                         const hfx_pattern* pattern, const hfx_opts* opts, int n_builds, const double* P_host,
                         double* K_out, long long* ticket, std::unique_ptr<Request>& r) {
  if (opts->spherical) return srv_fail(HFX_ERR_UNSUPPORTED, "the server takes Cartesian requests only");
  const long long nv = hfx_pattern_value_count(pattern_shells, n_pattern_shells, pattern);
  if (nv < 0) return srv_fail(HFX_ERR_INVALID_ARG, "inconsistent shells or pattern");
  r->ticket = s->next_ticket++;
  r->n_atoms = n_atoms;
  r->pattern_atoms = pattern->n_atoms;
  r->xyz.assign(atom_xyz, atom_xyz + 3 * (size_t)n_atoms);
  r->row_ptr.assign(pattern->row_ptr, pattern->row_ptr + pattern->n_atoms + 1);
  r->col.assign(pattern->col, pattern->col + r->row_ptr[(size_t)pattern->n_atoms]);
  size_t np = 0;
  for (int i = 0; i < n_shells; ++i) {
    if (shells[i].nprim < 1 || !shells[i].alpha || !shells[i].coef)
      return srv_fail(HFX_ERR_INVALID_ARG, "shell without primitives");
    np += (size_t)shells[i].nprim;
  }
  r->prim.resize(2 * np);
  r->shells.assign(shells, shells + n_shells);
  size_t k = 0;
  for (auto& d : r->shells) {  // point the copies at the server's own primitive arrays
    std::copy(d.alpha, d.alpha + d.nprim, r->prim.begin() + k);
    std::copy(d.coef, d.coef + d.nprim, r->prim.begin() + np + k);
    d.alpha = r->prim.data() + k;
    d.coef = r->prim.data() + np + k;
    k += (size_t)d.nprim;
  }
  r->opts = *opts;
  r->P_host = P_host;
  r->K_out = K_out;
  r->n_values = nv;
  r->estimate = hfx_setup_bytes_estimate(pattern_shells, n_pattern_shells, pattern) +
                (s->o.incremental ? 4 : 2) * std::max<long long>(nv, 1) * 8;
  r->E.assign((size_t)n_builds, 0.0);
  r->info.state = HFX_REQ_QUEUED;
  r->info.n_builds = n_builds;
  r->info.t_submit = s->now();
  r->info.t_admit = r->info.t_done = -1.0;
  *ticket = r->ticket;
  s->queue.push_back(r.get());
  s->all[r->ticket] = std::move(r);
  return HFX_OK;
}

}  // namespace

extern "C" {

hfx_status hfx_server_submit(hfx_server* s, const hfx_shell_desc* shells, int n_shells, const double* atom_xyz,
                             int n_atoms, const hfx_pattern* pattern, const hfx_opts* opts, int n_builds,
                             const double* P_host, double* K_out, long long* ticket) {
  if (!s || !shells || n_shells <= 0 || !atom_xyz || n_atoms <= 0 || !pattern || !opts || !P_host || !ticket)
    return srv_fail(HFX_ERR_INVALID_ARG, "NULL or empty argument");
  if (n_builds < 1) return srv_fail(HFX_ERR_INVALID_ARG, "n_builds must be >= 1");
  if (pattern->n_atoms != n_atoms) return srv_fail(HFX_ERR_INVALID_ARG, "pattern must cover the atoms");
  std::unique_ptr<Request> r(new Request());
  return submit_common(s, shells, n_shells, atom_xyz, n_atoms, shells, n_shells, pattern, opts, n_builds, P_host,
                       K_out, ticket, r);
}

hfx_status hfx_server_submit_periodic(hfx_server* s, const hfx_shell_desc* shells, int n_shells,
                                      const double* atom_xyz, int n_atoms, const double* lattice, double r_ext,
                                      const hfx_pattern* ext_pattern, const hfx_opts* opts, int n_builds,
                                      const double* P_host, double* K_out, long long* ticket) {
  if (!s || !shells || n_shells <= 0 || !atom_xyz || n_atoms <= 0 || !lattice || !ext_pattern || !opts ||
      !P_host || !ticket)
    return srv_fail(HFX_ERR_INVALID_ARG, "NULL or empty argument");
  if (n_builds < 1) return srv_fail(HFX_ERR_INVALID_ARG, "n_builds must be >= 1");
  for (int i = 0; i < n_shells; ++i)
    if (shells[i].atom < 0 || shells[i].atom >= n_atoms || (i > 0 && shells[i].atom < shells[i - 1].atom))
      return srv_fail(HFX_ERR_INVALID_ARG, "shells must be grouped by atom in increasing atom order");
  // the extended set the setup will build (hfx_create_basis_periodic): sizes
  // the values and the memory estimate
  const long long n_ext = hfx_periodic_extend(atom_xyz, n_atoms, lattice, r_ext, 0, nullptr, nullptr, nullptr);
  if (n_ext < 0) return HFX_ERR_INVALID_ARG;  // message set by hfx_periodic_extend
  if (ext_pattern->n_atoms != n_ext)
    return srv_fail(HFX_ERR_INVALID_ARG, "pattern must cover the extended atoms (hfx_periodic_extend)");
  std::vector<int> ext_home((size_t)n_ext), ext_shift(3 * (size_t)n_ext);
  std::vector<double> ext_xyz(3 * (size_t)n_ext);
  hfx_periodic_extend(atom_xyz, n_atoms, lattice, r_ext, n_ext, ext_home.data(), ext_shift.data(), ext_xyz.data());
  std::vector<hfx_shell_desc> ext;
  for (long long X = 0; X < n_ext; ++X)
    for (int i = 0; i < n_shells; ++i)
      if (shells[i].atom == ext_home[(size_t)X]) {
        hfx_shell_desc d = shells[i];
        d.atom = (int)X;
        ext.push_back(d);
      }
  std::unique_ptr<Request> r(new Request());
  r->periodic = true;
  std::copy(lattice, lattice + 9, r->lattice);
  r->r_ext = r_ext;
  return submit_common(s, shells, n_shells, atom_xyz, n_atoms, ext.data(), (int)ext.size(), ext_pattern, opts,
                       n_builds, P_host, K_out, ticket, r);
}

hfx_status hfx_server_step(hfx_server* s, int* n_active) {
  if (!s) return srv_fail(HFX_ERR_INVALID_ARG, "NULL server");
  // requests cancelled while active leave at this step boundary
  {
    std::vector<Request*> keep, gone;
    for (Request* r : s->active) (r->cancel ? gone : keep).push_back(r);
    if (!gone.empty()) {
      s->drop_groups();  // the batches refer to the leaving requests' quartet lists
      for (Request* r : gone) finish(s, r, HFX_REQ_CANCELLED, HFX_OK);
      s->active.swap(keep);
    }
  }
  hfx_status st = HFX_OK;
  std::vector<Request*> incoming;  // admitted during this step's builds, active from the next
  const bool overlap = !s->active.empty();
  if (!overlap) {  // nothing to overlap with: admit now and build at once
    st = admit(s, s->active, 0);
    if (st != HFX_OK) return st;
    if (!s->active.empty()) s->dirty = true;
  }
  if (n_active) *n_active = (int)s->active.size();
  if (s->active.empty()) return HFX_OK;
  if (s->dirty) {
    st = regroup(s);
    if (st != HFX_OK) return st;
  }
  // 1. this build's density of every active request, then the builds (async)
  for (Request* r : s->active) {
    const bool delta = s->o.incremental && r->info.builds_done > 0;
    const double* src = r->P_host + (size_t)r->info.builds_done * (size_t)r->n_values;
    const cudaError_t e = cudaMemcpyAsync(delta ? r->dP : r->P, src, (size_t)r->n_values * sizeof(double),
                                          cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return srv_fail(HFX_ERR_CUDA, std::string("P upload: ") + cudaGetErrorString(e));
    if (delta) k_delta_in<<<grid_for(r->n_values), 256, 0, s->stream>>>(r->n_values, r->dP, r->P);
  }
  for (auto& g : s->groups) {
    std::vector<const double*> Ps;
    std::vector<double*> Ks;
    for (Request* r : g.members) {
      const bool delta = s->o.incremental && r->info.builds_done > 0;
      Ps.push_back(delta ? r->dP : r->P);
      Ks.push_back(delta ? r->dK : r->K);
    }
    st = hfx_batch_build_K(g.batch, Ps.data(), Ks.data(), s->o.use_graph, s->stream);
    if (st != HFX_OK) return st;
  }
  // 2. admissions (setup on the second stream) while the builds run
  if (overlap) {
    st = admit(s, incoming, s->active.size());
    if (st != HFX_OK) return st;
  }
  // 3. energies, retirement
  for (auto& g : s->groups) {
    std::vector<double> E(g.members.size(), 0.0);
    if (s->o.incremental) {  // K += K(dP), then -1/2 P.K of the whole density
      if (!s->energies || s->n_energies < g.members.size()) {
        if (s->energies) cudaFree(s->energies);
        s->energies = nullptr;
        const cudaError_t e = cudaMalloc(&s->energies, std::max<size_t>(g.members.size(), 64) * sizeof(double));
        if (e != cudaSuccess) return srv_fail(HFX_ERR_OOM, std::string("energies: ") + cudaGetErrorString(e));
        s->n_energies = std::max<size_t>(g.members.size(), 64);
      }
      cudaMemsetAsync(s->energies, 0, g.members.size() * sizeof(double), s->stream);
      for (size_t i = 0; i < g.members.size(); ++i) {
        Request* r = g.members[i];
        if (r->info.builds_done > 0) k_add_into<<<grid_for(r->n_values), 256, 0, s->stream>>>(r->n_values, r->dK, r->K);
        k_energy_into<<<grid_for(r->n_values), 256, 0, s->stream>>>(r->n_values, r->P, r->K, s->energies + i);
      }
      cudaError_t e = cudaMemcpyAsync(E.data(), s->energies, E.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                      s->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
      if (e != cudaSuccess) return srv_fail(HFX_ERR_CUDA, std::string("energies: ") + cudaGetErrorString(e));
    } else {
      st = hfx_batch_energies(g.batch, E.data(), s->stream);
      if (st != HFX_OK) return st;
    }
    for (size_t i = 0; i < g.members.size(); ++i) {
      Request* r = g.members[i];
      r->E[(size_t)r->info.builds_done] = E[i];
      r->info.builds_done += 1;
      s->stats.builds_done += 1;
    }
  }
  s->stats.steps += 1;
  std::vector<Request*> still, gone;
  for (Request* r : s->active) (r->info.builds_done < r->info.n_builds ? still : gone).push_back(r);
  if (!gone.empty()) {
    s->drop_groups();  // the batches refer to the leaving requests' quartet lists
    for (Request* r : gone) {
      if (r->K_out) {
        const cudaError_t e = cudaMemcpyAsync(r->K_out, r->K, (size_t)r->n_values * sizeof(double),
                                              cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return srv_fail(HFX_ERR_CUDA, std::string("K download: ") + cudaGetErrorString(e));
      }
      finish(s, r, HFX_REQ_DONE, HFX_OK);
    }
  }
  s->active.swap(still);
  if (!incoming.empty()) {
    s->active.insert(s->active.end(), incoming.begin(), incoming.end());
    s->dirty = true;
  }
  if (n_active) *n_active = (int)s->active.size();
  return HFX_OK;
}

hfx_status hfx_server_poll(hfx_server* s, long long ticket, hfx_request_info* info, double* E_x) {
  if (!s || !info) return srv_fail(HFX_ERR_INVALID_ARG, "NULL argument");
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return srv_fail(HFX_ERR_INVALID_ARG, "unknown ticket");
  const Request* r = it->second.get();
  *info = r->info;
  if (E_x)
    for (int i = 0; i < r->info.builds_done; ++i) E_x[i] = r->E[(size_t)i];
  return HFX_OK;
}

hfx_status hfx_server_cancel(hfx_server* s, long long ticket) {
  if (!s) return srv_fail(HFX_ERR_INVALID_ARG, "NULL server");
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return srv_fail(HFX_ERR_INVALID_ARG, "unknown ticket");
  Request* r = it->second.get();
  if (r->info.state == HFX_REQ_QUEUED) {
    s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
    finish(s, r, HFX_REQ_CANCELLED, HFX_OK);
    return HFX_OK;
  }
  if (r->info.state == HFX_REQ_ACTIVE) {
    r->cancel = true;
    return HFX_OK;
  }
  return srv_fail(HFX_ERR_BUSY, "request already finished");
}

hfx_status hfx_server_inject_setup_failure(hfx_server* s, long long ticket, int status) {
  if (!s) return srv_fail(HFX_ERR_INVALID_ARG, "NULL server");
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return srv_fail(HFX_ERR_INVALID_ARG, "unknown ticket");
  if (it->second->info.state != HFX_REQ_QUEUED) return srv_fail(HFX_ERR_BUSY, "request already admitted");
  if (status == HFX_OK) return srv_fail(HFX_ERR_INVALID_ARG, "status must be an error");
  it->second->inject = (hfx_status)status;
  return HFX_OK;
}

hfx_status hfx_server_release(hfx_server* s, long long ticket) {
  if (!s) return srv_fail(HFX_ERR_INVALID_ARG, "NULL server");
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return srv_fail(HFX_ERR_INVALID_ARG, "unknown ticket");
  const int st = it->second->info.state;
  if (st != HFX_REQ_DONE && st != HFX_REQ_FAILED && st != HFX_REQ_CANCELLED)
    return srv_fail(HFX_ERR_BUSY, "request not finished");
  s->all.erase(it);
  return HFX_OK;
}

hfx_status hfx_server_get_info(hfx_server* s, hfx_server_info* out) {
  if (!s || !out) return srv_fail(HFX_ERR_INVALID_ARG, "NULL argument");
  *out = s->stats;
  out->n_queued = (int)s->queue.size();
  out->n_active = (int)s->active.size();
  return HFX_OK;
}

void hfx_server_destroy(hfx_server* s) { delete s; }

}  // extern "C"
