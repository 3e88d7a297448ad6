"""Thin ctypes binding of the HFX C ABI (include/hfx.h).

Argument marshalling only: every step of the exchange build runs in the CUDA
library ``libhfx.so`` built in-tree by ``paper_2009_03555_gb300/build.py``.
PyTorch supplies device memory (tensors) and streams.  If the library is
missing, loading fails loudly; there is no CPU fallback.

The functions carry the C names (``hfx_create_basis``, ``hfx_build_quartets``,
``hfx_build_K``, ``hfx_exchange_energy``, ...).  ``Basis`` and ``Quartets``
own the handles and release them.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhfx.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "hfx.h")

HFX_KERNEL_COULOMB, HFX_KERNEL_ERFC, HFX_KERNEL_ERF = 0, 1, 2
HFX_PREC_FP64, HFX_PREC_MIXED = 0, 1
N_CLASSES = 21
PAIR_CLASS_NAMES = ["ss", "ps", "pp", "ds", "dp", "dd"]

_STATUS = {0: "HFX_OK", 1: "HFX_ERR_INVALID_ARG", 2: "HFX_ERR_OOM", 3: "HFX_ERR_CUDA",
           4: "HFX_ERR_UNSUPPORTED", 5: "HFX_ERR_TIMEOUT", 6: "HFX_ERR_BUSY"}


class HFXError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class ShellDesc(ctypes.Structure):
    _fields_ = [("l", ctypes.c_int), ("nprim", ctypes.c_int), ("atom", ctypes.c_int),
                ("reserved", ctypes.c_int), ("alpha", ctypes.c_void_p), ("coef", ctypes.c_void_p)]


class Opts(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("omega", ctypes.c_double), ("screen", ctypes.c_int),
                ("tau", ctypes.c_double), ("density_screen", ctypes.c_int), ("eps", ctypes.c_double),
                ("prim_cutoff", ctypes.c_double), ("precision", ctypes.c_int),
                ("fp64_promote_bound", ctypes.c_double), ("n_block", ctypes.c_int),
                ("promote_min_l", ctypes.c_int), ("prim_density_screen", ctypes.c_int), ("promote_prims", ctypes.c_int),
                ("spherical", ctypes.c_int), ("extent_eps", ctypes.c_double), ("reserved2", ctypes.c_int * 2)]


class Pattern(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("n_pairs_significant", ctypes.c_longlong * 6),
                ("n_quartets_schwarz", ctypes.c_longlong * N_CLASSES),
                ("n_quartets_computed", ctypes.c_longlong * N_CLASSES),
                ("n_prim_pairs", ctypes.c_longlong), ("n_values", ctypes.c_longlong),
                ("ms_setup", ctypes.c_float), ("ms_last_build", ctypes.c_float),
                ("n_quartets_pass", (ctypes.c_longlong * N_CLASSES) * 2),
                ("n_prim_quartets_pass", (ctypes.c_longlong * N_CLASSES) * 2),
                ("ms_class_pass", (ctypes.c_float * N_CLASSES) * 2),
                ("ms_setup_phase", ctypes.c_float * 4), ("n_pairs_distance", ctypes.c_longlong)]


class ClassInfo(ctypes.Structure):
    _fields_ = [("bra_class", ctypes.c_int), ("ket_class", ctypes.c_int), ("la", ctypes.c_int),
                ("lb", ctypes.c_int), ("lc", ctypes.c_int), ("ld", ctypes.c_int), ("n_out", ctypes.c_int),
                ("vrr_flops", ctypes.c_int), ("hrr_flops", ctypes.c_int), ("n_acc", ctypes.c_int),
                ("kernel_kind", ctypes.c_int)]

KERNEL_KIND_NAMES = ("k_build_K", "k_build_K_split", "k_build_K_coop")


EXPORTED = ["hfx_create_basis", "hfx_build_quartets", "hfx_value_count", "hfx_build_K", "hfx_build_K_delta",
            "hfx_build_K_shard",
            "hfx_exchange_energy",
            "hfx_pack_dense", "hfx_unpack_dense", "hfx_eval_quartets", "hfx_boys_eval", "hfx_get_stats",
            "hfx_get_class_info", "hfx_exchange_energy_noalloc", "hfx_batch_create", "hfx_batch_build_K",
            "hfx_batch_energies", "hfx_batch_autotune", "hfx_batch_get_tuning", "hfx_batch_get_stats",
            "hfx_batch_destroy", "hfx_quartets_device_bytes", "hfx_basis_device_bytes", "hfx_pattern_value_count",
            "hfx_pack_dense_host", "hfx_setup_bytes_estimate", "hfx_server_create", "hfx_server_submit",
            "hfx_server_step", "hfx_server_poll", "hfx_server_release", "hfx_server_get_info", "hfx_server_destroy",
            "hfx_server_cancel", "hfx_server_inject_setup_failure", "hfx_periodic_images", "hfx_periodic_pack_host",
            "hfx_create_basis_periodic", "hfx_basis_atoms", "hfx_periodic_extend", "hfx_distance_pattern",
            "hfx_server_submit_periodic", "hfx_periodic_pack_lattice_host",
            "hfx_destroy_basis", "hfx_destroy_quartets", "hfx_last_error"]

_lib = None


class ServerOpts(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_longlong), ("max_active", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("incremental", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("status", ctypes.c_int), ("builds_done", ctypes.c_int),
                ("n_builds", ctypes.c_int), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("device_bytes", ctypes.c_longlong)]


class ServerInfo(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_longlong), ("used_bytes", ctypes.c_longlong),
                ("peak_used_bytes", ctypes.c_longlong), ("builds_done", ctypes.c_longlong),
                ("steps", ctypes.c_longlong), ("n_queued", ctypes.c_int), ("n_active", ctypes.c_int),
                ("max_active_seen", ctypes.c_int), ("reserved", ctypes.c_int)]


HFX_REQ_QUEUED, HFX_REQ_ACTIVE, HFX_REQ_DONE, HFX_REQ_FAILED, HFX_REQ_CANCELLED = 0, 1, 2, 3, 4


def load(path: str = LIB_PATH):
    """Load libhfx.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run paper_2009_03555_gb300/build.py (or __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    V, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    PV = ctypes.POINTER(ctypes.c_void_p)
    lib.hfx_create_basis.argtypes = [ctypes.POINTER(ShellDesc), I, V, I, V, PV]
    lib.hfx_build_quartets.argtypes = [V, ctypes.POINTER(Opts), ctypes.POINTER(Pattern), V, PV]
    lib.hfx_value_count.argtypes = [V]
    lib.hfx_value_count.restype = LL
    lib.hfx_build_K.argtypes = [V, V, V, V]
    lib.hfx_build_K_delta.argtypes = [V, V, V, V]
    lib.hfx_build_K_shard.argtypes = [V, V, V, I, I, V]
    lib.hfx_exchange_energy.argtypes = [V, V, V, ctypes.POINTER(D), V]
    lib.hfx_pack_dense.argtypes = [V, V, V, V]
    lib.hfx_unpack_dense.argtypes = [V, V, V, V]
    lib.hfx_eval_quartets.argtypes = [V, I, D, I, I, V, V, V, V]
    lib.hfx_boys_eval.argtypes = [V, I, I, I, V, V, V]
    lib.hfx_exchange_energy_noalloc.argtypes = [V, V, LL, V, V]
    lib.hfx_batch_create.argtypes = [V, I, V, PV]
    lib.hfx_batch_build_K.argtypes = [V, V, V, I, V]
    lib.hfx_batch_energies.argtypes = [V, V, V]
    lib.hfx_batch_autotune.argtypes = [V, V, V, V]
    lib.hfx_batch_get_tuning.argtypes = [V, V, V]
    lib.hfx_batch_get_stats.argtypes = [V, ctypes.POINTER(Stats)]
    lib.hfx_batch_destroy.argtypes = [V]
    lib.hfx_batch_destroy.restype = None
    lib.hfx_get_stats.argtypes = [V, ctypes.POINTER(Stats)]
    lib.hfx_get_class_info.argtypes = [I, ctypes.POINTER(ClassInfo)]
    lib.hfx_destroy_basis.argtypes = [V]
    lib.hfx_destroy_basis.restype = None
    lib.hfx_destroy_quartets.argtypes = [V]
    lib.hfx_destroy_quartets.restype = None
    lib.hfx_last_error.restype = ctypes.c_char_p
    lib.hfx_quartets_device_bytes.argtypes = [V]
    lib.hfx_basis_device_bytes.argtypes = [V]
    lib.hfx_pattern_value_count.argtypes = [ctypes.POINTER(ShellDesc), I, ctypes.POINTER(Pattern)]
    lib.hfx_pack_dense_host.argtypes = [ctypes.POINTER(ShellDesc), I, ctypes.POINTER(Pattern), V, V]
    lib.hfx_setup_bytes_estimate.argtypes = [ctypes.POINTER(ShellDesc), I, ctypes.POINTER(Pattern)]
    lib.hfx_server_create.argtypes = [ctypes.POINTER(ServerOpts), V, PV]
    lib.hfx_server_submit.argtypes = [V, ctypes.POINTER(ShellDesc), I, V, I, ctypes.POINTER(Pattern),
                                      ctypes.POINTER(Opts), I, V, V, ctypes.POINTER(LL)]
    lib.hfx_server_submit_periodic.argtypes = [V, ctypes.POINTER(ShellDesc), I, V, I, V, D, ctypes.POINTER(Pattern),
                                               ctypes.POINTER(Opts), I, V, V, ctypes.POINTER(LL)]
    lib.hfx_server_step.argtypes = [V, ctypes.POINTER(I)]
    lib.hfx_server_poll.argtypes = [V, LL, ctypes.POINTER(RequestInfo), V]
    lib.hfx_server_release.argtypes = [V, LL]
    lib.hfx_server_cancel.argtypes = [V, LL]
    lib.hfx_server_inject_setup_failure.argtypes = [V, LL, I]
    lib.hfx_server_get_info.argtypes = [V, ctypes.POINTER(ServerInfo)]
    lib.hfx_server_destroy.argtypes = [V]
    lib.hfx_server_destroy.restype = None
    lib.hfx_periodic_images.argtypes = [V, I, V, D, LL, V, V]
    lib.hfx_periodic_pack_host.argtypes = [ctypes.POINTER(ShellDesc), I, I, V, ctypes.POINTER(Pattern), V, V]
    lib.hfx_create_basis_periodic.argtypes = [ctypes.POINTER(ShellDesc), I, V, I, V, D, V, PV]
    lib.hfx_periodic_pack_lattice_host.argtypes = [ctypes.POINTER(ShellDesc), I, I, V, V, ctypes.POINTER(Pattern),
                                                   I, V, V, V]
    lib.hfx_basis_atoms.argtypes = [V, V, V, V]
    lib.hfx_periodic_extend.argtypes = [V, I, V, D, LL, V, V, V]
    lib.hfx_distance_pattern.argtypes = [V, I, D, V, V, LL]
    for name in EXPORTED:
        if name in ("hfx_quartets_device_bytes", "hfx_basis_device_bytes", "hfx_pattern_value_count",
                    "hfx_setup_bytes_estimate", "hfx_periodic_images", "hfx_periodic_extend",
                    "hfx_distance_pattern"):
            getattr(lib, name).restype = LL
        elif name not in ("hfx_value_count", "hfx_destroy_basis", "hfx_destroy_quartets", "hfx_last_error",
                          "hfx_batch_destroy", "hfx_server_destroy"):
            getattr(lib, name).restype = I
    _lib = lib
    return lib


def _check(status):
    if status != 0:
        raise HFXError(status, load().hfx_last_error().decode(errors="replace"))


def _ptr(x):
    """Device or host address of a torch tensor / numpy array (marshalling)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return x.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:  # pragma: no cover
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ----------------------------------------------------------------- C names
def shell_descs(shell_l, shell_atom, prim_off, alpha, coef):
    """hfx_shell_desc array from flat shell arrays.  Returns (descs, keep):
    ``keep`` holds the primitive arrays the descriptors point into."""
    n = len(shell_l)
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    descs = (ShellDesc * n)()
    base_a, base_c = alpha.ctypes.data, coef.ctypes.data
    for i in range(n):
        p0, p1 = int(prim_off[i]), int(prim_off[i + 1])
        descs[i].l = int(shell_l[i])
        descs[i].nprim = p1 - p0
        descs[i].atom = int(shell_atom[i])
        descs[i].alpha = base_a + 8 * p0
        descs[i].coef = base_c + 8 * p0
    return descs, (alpha, coef)


def hfx_create_basis(shell_l, shell_atom, prim_off, alpha, coef, atom_xyz, stream=None):
    """Shells from flat arrays (host numpy).  Returns the raw handle."""
    lib = load()
    descs, _keep = shell_descs(shell_l, shell_atom, prim_off, alpha, coef)
    xyz = np.ascontiguousarray(atom_xyz, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(lib.hfx_create_basis(descs, len(shell_l), _ptr(xyz), int(xyz.shape[0]), _stream(stream),
                                ctypes.byref(h)))
    return h


def make_opts(kernel=HFX_KERNEL_ERFC, omega=0.11, screen=True, tau=1e-8, density_screen=True, eps=None,
              prim_cutoff=1e-15, precision=HFX_PREC_FP64, fp64_promote_bound=math.inf, n_block=128,
              promote_min_l=0, prim_density_screen=False, promote_prims=False, spherical=False,
              extent_eps=0.0) -> Opts:
    o = Opts()
    o.kernel, o.omega, o.screen, o.tau = int(kernel), float(omega), int(bool(screen)), float(tau)
    o.density_screen = int(bool(density_screen))
    o.eps = float(tau if eps is None else eps)
    o.prim_cutoff, o.precision = float(prim_cutoff), int(precision)
    o.fp64_promote_bound, o.n_block = float(fp64_promote_bound), int(n_block)
    o.promote_min_l = int(promote_min_l)
    o.prim_density_screen = int(bool(prim_density_screen))
    o.promote_prims = int(bool(promote_prims))
    o.spherical = int(bool(spherical))
    o.extent_eps = float(extent_eps)
    return o


def pattern_from_mask(mask):
    """CSR arrays of a symmetric boolean atom-pair mask."""
    mask = np.asarray(mask, dtype=bool)
    rows = [np.nonzero(mask[i])[0] for i in range(mask.shape[0])]
    row_ptr = np.zeros(mask.shape[0] + 1, dtype=np.int32)
    row_ptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.ascontiguousarray(np.concatenate(rows).astype(np.int32)) if rows else np.zeros(0, np.int32)
    return row_ptr, col


def hfx_build_quartets(basis, opts: Opts, row_ptr, col, stream=None):
    lib = load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    pat = Pattern(len(row_ptr) - 1, row_ptr.ctypes.data, col.ctypes.data)
    h = ctypes.c_void_p()
    _check(lib.hfx_build_quartets(basis, ctypes.byref(opts), ctypes.byref(pat), _stream(stream), ctypes.byref(h)))
    return h


def hfx_value_count(q) -> int:
    return int(load().hfx_value_count(q))


def hfx_build_K(q, P_val, K_val, stream=None):
    _check(load().hfx_build_K(q, _ptr(P_val), _ptr(K_val), _stream(stream)))


def hfx_build_K_delta(q, dP_val, K_val, stream=None):
    """K_val += K(dP_val) (incremental build; see hfx.h)."""
    _check(load().hfx_build_K_delta(q, _ptr(dP_val), _ptr(K_val), _stream(stream)))


def hfx_exchange_energy(q, P_val, K_val, stream=None) -> float:
    e = ctypes.c_double()
    _check(load().hfx_exchange_energy(q, _ptr(P_val), _ptr(K_val), ctypes.byref(e), _stream(stream)))
    return float(e.value)


def hfx_pack_dense(q, dense, val, stream=None):
    _check(load().hfx_pack_dense(q, _ptr(dense), _ptr(val), _stream(stream)))


def hfx_unpack_dense(q, val, dense, stream=None):
    _check(load().hfx_unpack_dense(q, _ptr(val), _ptr(dense), _stream(stream)))


def hfx_eval_quartets(basis, kernel, omega, precision, quartets, out_off, out, stream=None):
    q = np.ascontiguousarray(np.asarray(quartets, dtype=np.int32).reshape(-1, 4))
    off = np.ascontiguousarray(out_off, dtype=np.int64)
    _check(load().hfx_eval_quartets(basis, int(kernel), float(omega), int(precision), int(q.shape[0]),
                                    _ptr(q), _ptr(off), _ptr(out), _stream(stream)))


def hfx_boys_eval(basis, precision, mmax, T, F, stream=None):
    _check(load().hfx_boys_eval(basis, int(precision), int(mmax), int(T.numel()), _ptr(T), _ptr(F),
                                _stream(stream)))


def hfx_exchange_energy_noalloc(P_val, K_val, n_values, E_x_dev, stream=None):
    """E_x into a device double without any device allocation (see hfx.h)."""
    _check(load().hfx_exchange_energy_noalloc(_ptr(P_val), _ptr(K_val), int(n_values), _ptr(E_x_dev),
                                              _stream(stream)))


def hfx_get_stats(q) -> Stats:
    st = Stats()
    _check(load().hfx_get_stats(q, ctypes.byref(st)))
    return st


def hfx_get_class_info(cls) -> ClassInfo:
    ci = ClassInfo()
    _check(load().hfx_get_class_info(int(cls), ctypes.byref(ci)))
    return ci


def hfx_destroy_basis(h):
    load().hfx_destroy_basis(h)


def hfx_destroy_quartets(h):
    load().hfx_destroy_quartets(h)


# ----------------------------------------------------------------- owners
class Basis:
    """Owns an hfx_basis built from a system with flat shell arrays
    (``shell_l``, ``shell_atom``, ``prim_off``, ``alpha``, ``coef``, ``atom_xyz``)."""

    def __init__(self, system, stream=None):
        self.system = system
        self.nbf = int(system.n_bf)
        self.handle = hfx_create_basis(system.shell_l, system.shell_atom, system.prim_off, system.alpha,
                                       system.coef, system.atom_xyz, stream)

    def eval_quartets(self, quartets, kernel=HFX_KERNEL_ERFC, omega=0.11, precision=HFX_PREC_FP64, stream=None):
        import torch
        q = np.asarray(quartets, dtype=np.int32).reshape(-1, 4)
        nf = np.array([(int(l) + 1) * (int(l) + 2) // 2 for l in self.system.shell_l])
        sizes = np.prod(nf[q], axis=1).astype(np.int64)
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        out = torch.zeros(int(off[-1]), dtype=torch.float64, device="cuda")
        hfx_eval_quartets(self.handle, kernel, omega, precision, q, off[:-1], out, stream)
        host = out.cpu().numpy()
        return [host[off[i]:off[i + 1]].reshape(tuple(int(x) for x in nf[q[i]])) for i in range(q.shape[0])]

    def boys(self, T, mmax, precision=HFX_PREC_FP64, stream=None):
        """F_0..F_mmax at the arguments T (numpy) from the device evaluators."""
        import torch
        Td = torch.as_tensor(np.ascontiguousarray(T, dtype=np.float64)).cuda()
        Fd = torch.empty((Td.numel(), mmax + 1), dtype=torch.float64, device="cuda")
        hfx_boys_eval(self.handle, precision, mmax, Td, Fd, stream)
        return Fd.cpu().numpy()

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.hfx_destroy_basis(h)
            self.handle = None


class Quartets:
    """Owns an hfx_quartets (screened quartet lists + work queue) for one
    basis, options and atom-pair pattern."""

    def __init__(self, basis, opts: Opts, mask=None, stream=None, csr=None):
        self.basis = basis
        self.opts = opts
        row_ptr, col = csr if csr is not None else pattern_from_mask(mask)
        self.handle = hfx_build_quartets(basis.handle, opts, row_ptr, col, stream)
        self.n_values = hfx_value_count(self.handle)

    def build_K(self, P_val, K_val, stream=None):
        hfx_build_K(self.handle, P_val, K_val, stream)

    def build_K_delta(self, dP_val, K_val, stream=None):
        hfx_build_K_delta(self.handle, dP_val, K_val, stream)

    def build_K_shard(self, P_val, K_val, rank, n_ranks, stream=None):
        """This rank's share of a sharded build (sum over ranks = build_K)."""
        _check(load().hfx_build_K_shard(self.handle, _ptr(P_val), _ptr(K_val), int(rank), int(n_ranks),
                                        _stream(stream)))

    def exchange_energy(self, P_val, K_val, stream=None) -> float:
        return hfx_exchange_energy(self.handle, P_val, K_val, stream)

    def pack(self, dense, val, stream=None):
        hfx_pack_dense(self.handle, dense, val, stream)

    def unpack(self, val, dense, stream=None):
        hfx_unpack_dense(self.handle, val, dense, stream)

    def stats(self) -> Stats:
        return hfx_get_stats(self.handle)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.hfx_destroy_quartets(h)
            self.handle = None


class Batch:
    """Owns an hfx_batch over several Quartets (members must stay alive)."""

    def __init__(self, members, stream=None):
        self.members = list(members)
        arr = (ctypes.c_void_p * len(self.members))(*[m.handle.value for m in self.members])
        self._arr = arr
        h = ctypes.c_void_p()
        _check(load().hfx_batch_create(arr, len(self.members), _stream(stream), ctypes.byref(h)))
        self.handle = h

    def _ptrs(self, tensors):
        return (ctypes.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])

    def build_K(self, P_vals, K_vals, use_graph=True, stream=None):
        self._keep = (self._ptrs(P_vals), self._ptrs(K_vals))
        _check(load().hfx_batch_build_K(self.handle, self._keep[0], self._keep[1], int(bool(use_graph)),
                                        _stream(stream)))

    def energies(self, stream=None):
        out = np.zeros(len(self.members))
        _check(load().hfx_batch_energies(self.handle, _ptr(out), _stream(stream)))
        return out

    def autotune(self, P_vals, K_vals, stream=None):
        p, k = self._ptrs(P_vals), self._ptrs(K_vals)
        _check(load().hfx_batch_autotune(self.handle, p, k, _stream(stream)))

    def tuning(self):
        nb = np.zeros(N_CLASSES, dtype=np.int32)
        g = np.zeros(N_CLASSES, dtype=np.int32)
        _check(load().hfx_batch_get_tuning(self.handle, _ptr(nb), _ptr(g)))
        return nb, g

    def stats(self) -> Stats:
        st = Stats()
        _check(load().hfx_batch_get_stats(self.handle, ctypes.byref(st)))
        return st

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.hfx_batch_destroy(h)
            self.handle = None


class _SystemInput:
    """Shell descriptors, coordinates and CSR pattern of one system (host)."""

    def __init__(self, system, mask):
        self.descs, self._keep = shell_descs(system.shell_l, system.shell_atom, system.prim_off, system.alpha,
                                             system.coef)
        self.n_shells = len(system.shell_l)
        self.xyz = np.ascontiguousarray(system.atom_xyz, dtype=np.float64)
        self.row_ptr, self.col = pattern_from_mask(mask)
        self.pattern = Pattern()
        self.pattern.n_atoms = int(self.xyz.shape[0])
        self.pattern.row_ptr = self.row_ptr.ctypes.data
        self.pattern.col = self.col.ctypes.data

    def value_count(self) -> int:
        n = load().hfx_pattern_value_count(self.descs, self.n_shells, ctypes.byref(self.pattern))
        if n < 0:
            raise HFXError(1, "inconsistent shells or pattern")
        return int(n)

    def pack(self, dense) -> np.ndarray:
        dense = np.ascontiguousarray(dense, dtype=np.float64)
        out = np.empty(self.value_count())
        _check(load().hfx_pack_dense_host(self.descs, self.n_shells, ctypes.byref(self.pattern), _ptr(dense),
                                          _ptr(out)))
        return out

    def setup_bytes_estimate(self) -> int:
        return int(load().hfx_setup_bytes_estimate(self.descs, self.n_shells, ctypes.byref(self.pattern)))


def hfx_periodic_images(atom_xyz, lattice, r_ext):
    """Image table of a periodic cell: (image_atom, image_shift), the home atom
    and the lattice shift (n1, n2, n3) of every image within ``r_ext`` of a
    home atom, ordered by shift and then atom (see hfx.h)."""
    lib = load()
    xyz = np.ascontiguousarray(atom_xyz, dtype=np.float64).reshape(-1, 3)
    A = np.ascontiguousarray(lattice, dtype=np.float64).reshape(3, 3)
    n = lib.hfx_periodic_images(_ptr(xyz), int(xyz.shape[0]), _ptr(A), float(r_ext), 0, None, None)
    if n < 0:
        raise HFXError(1, lib.hfx_last_error().decode(errors="replace"))
    atom = np.zeros(max(n, 1), dtype=np.int32)
    shift = np.zeros((max(n, 1), 3), dtype=np.int32)
    m = lib.hfx_periodic_images(_ptr(xyz), int(xyz.shape[0]), _ptr(A), float(r_ext), int(n), _ptr(atom),
                                _ptr(shift))
    assert m == n
    return atom[:n], shift[:n]


class ExtendedLayout:
    """Function layout of a periodic cell's extended atom set (from the
    library's ``ext_home``): every extended atom carries its home atom's
    functions, so only counts and offsets are derived here."""

    def __init__(self, home, ext_home, ext_xyz):
        nf_home = np.diff(np.asarray(home.atom_func_off))
        ns_home = np.bincount(np.asarray(home.shell_atom), minlength=home.n_atoms)
        self.atom_xyz = ext_xyz
        self.n_atoms = len(ext_home)
        self.n_shells = int(ns_home[ext_home].sum())
        self.atom_func_off = np.concatenate([[0], np.cumsum(nf_home[ext_home])]).astype(np.int64)
        self.n_bf = int(self.atom_func_off[-1])


class Periodic:
    """A periodic cell (Sec. 2, Eq. H-HFX; see the periodic section of hfx.h).

    ``system``: the home cell (flat shell arrays, shells grouped by atom);
    ``lattice``: 3 x 3 lattice vectors as rows (bohr).  The library builds the
    extended atom set (images within ``r_ext`` of a home atom,
    hfx_periodic_extend) and the density pattern (extended atoms at most
    ``r_P`` apart, hfx_distance_pattern); ``basis()`` creates the device basis
    (hfx_create_basis_periodic), whose quartet lists evaluate only quartets with
    a home-cell shell.  The first ``n_home_bf`` rows of K are K^G (the first
    ``n_home_values`` values), the image rows are zero, and hfx_exchange_energy
    gives the exchange energy per cell."""

    def __init__(self, system, lattice, r_ext=10.0, r_P=14.0):
        lib = load()
        self.home = system
        self.lattice = np.ascontiguousarray(lattice, dtype=np.float64).reshape(3, 3)
        self.r_ext, self.r_P = float(r_ext), float(r_P)
        xyz = np.ascontiguousarray(system.atom_xyz, dtype=np.float64)
        n_home = int(system.n_atoms)
        n = lib.hfx_periodic_extend(_ptr(xyz), n_home, _ptr(self.lattice), self.r_ext, 0, None, None, None)
        if n < 0:
            raise HFXError(1, lib.hfx_last_error().decode(errors="replace"))
        self.ext_home = np.zeros(n, dtype=np.int32)
        self.ext_shift = np.zeros((n, 3), dtype=np.int32)
        ext_xyz = np.zeros((n, 3))
        m = lib.hfx_periodic_extend(_ptr(xyz), n_home, _ptr(self.lattice), self.r_ext, int(n), _ptr(self.ext_home),
                                    _ptr(self.ext_shift), _ptr(ext_xyz))
        assert m == n
        self.system = ExtendedLayout(system, self.ext_home, ext_xyz)
        nnz = lib.hfx_distance_pattern(_ptr(ext_xyz), int(n), self.r_P, None, None, 0)
        if nnz < 0:
            raise HFXError(1, lib.hfx_last_error().decode(errors="replace"))
        self.row_ptr = np.zeros(n + 1, dtype=np.int32)
        self.col = np.zeros(max(int(nnz), 1), dtype=np.int32)
        lib.hfx_distance_pattern(_ptr(ext_xyz), int(n), self.r_P, _ptr(self.row_ptr), _ptr(self.col), int(nnz))
        self.col = self.col[:nnz]
        self.pattern = Pattern()
        self.pattern.n_atoms, self.pattern.row_ptr, self.pattern.col = int(n), self.row_ptr.ctypes.data, \
            self.col.ctypes.data
        self._home_descs, self._home_keep = shell_descs(system.shell_l, system.shell_atom, system.prim_off,
                                                        system.alpha, system.coef)
        nfa = np.diff(self.system.atom_func_off)
        self.n_values = int(sum(nfa[X] * nfa[self.col[self.row_ptr[X]:self.row_ptr[X + 1]]].sum()
                                for X in range(n)))
        self.n_home_bf = int(nfa[:n_home].sum())
        self.n_home_values = int(sum(nfa[X] * nfa[self.col[self.row_ptr[X]:self.row_ptr[X + 1]]].sum()
                                     for X in range(n_home)))

    @property
    def mask(self) -> np.ndarray:
        """The density pattern as a dense boolean atom-pair matrix."""
        n = len(self.ext_home)
        m = np.zeros((n, n), dtype=bool)
        for X in range(n):
            m[X, self.col[self.row_ptr[X]:self.row_ptr[X + 1]]] = True
        return m

    def basis(self, stream=None) -> "PeriodicBasis":
        return PeriodicBasis(self, stream)

    def quartets(self, opts: Opts, stream=None) -> "Quartets":
        """Basis and quartet lists of the cell on its density pattern."""
        return Quartets(self.basis(stream), opts, csr=(self.row_ptr, self.col), stream=stream)

    def pack_lattice(self, L_shift, P_L) -> np.ndarray:
        """Values of the real-space density from one home-cell block per lattice
        vector (``L_shift``: n_L x 3 integer shifts, ``P_L``: n_L x nbf x nbf),
        e.g. the Fourier sum of a k-point grid (host)."""
        L = np.ascontiguousarray(L_shift, dtype=np.int32).reshape(-1, 3)
        PL = np.ascontiguousarray(P_L, dtype=np.float64)
        out = np.empty(self.n_values)
        _check(load().hfx_periodic_pack_lattice_host(self._home_descs, len(self.home.shell_l),
                                                     int(self.home.n_atoms), _ptr(self.ext_home),
                                                     _ptr(self.ext_shift), ctypes.byref(self.pattern), int(L.shape[0]),
                                                     _ptr(L), _ptr(PL), _ptr(out)))
        return out

    def pack(self, P_home) -> np.ndarray:
        """Values of the real-space density on the extended pattern (host)."""
        P = np.ascontiguousarray(P_home, dtype=np.float64)
        out = np.empty(self.n_values)
        _check(load().hfx_periodic_pack_host(self._home_descs, len(self.home.shell_l), int(self.home.n_atoms),
                                             _ptr(self.ext_home), ctypes.byref(self.pattern), _ptr(P),
                                             _ptr(out)))
        return out


class PeriodicBasis:
    """Owns the hfx_basis of a periodic cell (hfx_create_basis_periodic)."""

    def __init__(self, per: Periodic, stream=None):
        lib = load()
        home = per.home
        descs, _keep = shell_descs(home.shell_l, home.shell_atom, home.prim_off, home.alpha, home.coef)
        xyz = np.ascontiguousarray(home.atom_xyz, dtype=np.float64)
        h = ctypes.c_void_p()
        _check(lib.hfx_create_basis_periodic(descs, len(home.shell_l), _ptr(xyz), int(home.n_atoms),
                                             _ptr(per.lattice), per.r_ext, _stream(stream), ctypes.byref(h)))
        self.handle = h
        self.nbf = per.system.n_bf
        nh = ctypes.c_int()
        n = lib.hfx_basis_atoms(h, ctypes.byref(nh), None, None)
        self.ext_home = np.zeros(n, dtype=np.int32)
        self.ext_shift = np.zeros((n, 3), dtype=np.int32)
        lib.hfx_basis_atoms(h, None, _ptr(self.ext_home), _ptr(self.ext_shift))
        self.n_home_atoms = nh.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.hfx_destroy_basis(h)
            self.handle = None


class Server:
    """Owns an hfx_server (continuous batching of SCF-like requests)."""

    def __init__(self, mem_budget=0, max_active=64, use_graph=False, incremental=False, stream=None):
        o = ServerOpts()
        o.mem_budget, o.max_active, o.use_graph = int(mem_budget), int(max_active), int(bool(use_graph))
        o.incremental = int(bool(incremental))
        h = ctypes.c_void_p()
        _check(load().hfx_server_create(ctypes.byref(o), _stream(stream), ctypes.byref(h)))
        self.handle = h
        self._req = {}

    def submit(self, system, mask, opts: Opts, P_list, want_K=True) -> int:
        """Queue one system with one dense density matrix per build."""
        inp = _SystemInput(system, mask)
        nv = inp.value_count()
        P = np.empty((len(P_list), nv))
        for i, Pi in enumerate(P_list):
            P[i] = inp.pack(Pi)
        K = np.zeros(nv) if want_K else None
        t = ctypes.c_longlong()
        _check(load().hfx_server_submit(self.handle, inp.descs, inp.n_shells, _ptr(inp.xyz), int(inp.xyz.shape[0]),
                                        ctypes.byref(inp.pattern), ctypes.byref(opts), len(P_list), _ptr(P),
                                        _ptr(K), ctypes.byref(t)))
        self._req[t.value] = (inp, P, K, len(P_list))
        return t.value

    def submit_periodic(self, per: "Periodic", opts: Opts, P_list, want_K=True) -> int:
        """Queue a periodic cell (``Periodic``: home cell, lattice, r_ext and its
        density pattern) with one dense home-cell density matrix per build."""
        nv = per.n_values
        P = np.empty((len(P_list), nv))
        for i, Pi in enumerate(P_list):
            P[i] = per.pack(Pi)
        K = np.zeros(nv) if want_K else None
        home = per.home
        descs, keep = shell_descs(home.shell_l, home.shell_atom, home.prim_off, home.alpha, home.coef)
        xyz = np.ascontiguousarray(home.atom_xyz, dtype=np.float64)
        t = ctypes.c_longlong()
        _check(load().hfx_server_submit_periodic(self.handle, descs, len(home.shell_l), _ptr(xyz), int(home.n_atoms),
                                                 _ptr(per.lattice), per.r_ext, ctypes.byref(per.pattern),
                                                 ctypes.byref(opts), len(P_list), _ptr(P), _ptr(K), ctypes.byref(t)))
        self._req[t.value] = ((descs, keep, xyz, per), P, K, len(P_list))
        return t.value

    def step(self) -> int:
        n = ctypes.c_int()
        _check(load().hfx_server_step(self.handle, ctypes.byref(n)))
        return n.value

    def poll(self, ticket):
        """(RequestInfo, energies of the builds done so far)."""
        info = RequestInfo()
        E = np.zeros(self._req[ticket][3])
        _check(load().hfx_server_poll(self.handle, int(ticket), ctypes.byref(info), _ptr(E)))
        return info, E[:info.builds_done]

    def K_values(self, ticket):
        """K values (pattern layout) of the last build of a finished request."""
        return self._req[ticket][2]

    def cancel(self, ticket):
        _check(load().hfx_server_cancel(self.handle, int(ticket)))

    def inject_setup_failure(self, ticket, status):
        _check(load().hfx_server_inject_setup_failure(self.handle, int(ticket), int(status)))

    def release(self, ticket):
        _check(load().hfx_server_release(self.handle, int(ticket)))
        self._req.pop(ticket, None)

    def info(self) -> ServerInfo:
        i = ServerInfo()
        _check(load().hfx_server_get_info(self.handle, ctypes.byref(i)))
        return i

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.hfx_server_destroy(h)
            self.handle = None
