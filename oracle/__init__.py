"""CPU oracle for Hartree-Fock exchange construction (plain FP64 C via ctypes).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product library never imports,
links or runs anything here, and this package imports nothing from the
product.  ``build()`` compiles ``hfx_oracle.c`` with gcc into
``liboracle.so`` next to it.

Functions (each cites the passage it follows):
  boys            -- Boys function F_m(x) (auxiliary of the analytic ERIs)
  normalize       -- axial normalisation of contracted Cartesian shells
  quartets        -- contracted shell-quartet ERIs, Sec. 2 (full-range ERI
                     definition; Eq. ERI-SR for erfc; erf for the complement)
  schwarz         -- Q_IJ = sqrt(max |(ij|ij)|), Sec. 2 Eq. schwarz
  build_K         -- K_ij = sum_kl (ik|jl) P_kl, Eq. H-HFX (without the -1/2),
                     Schwarz and density screening (Eq. dmscreening), either by
                     the 8-fold permutation symmetry or by brute force
  exchange_energy -- E_x = -1/2 sum_ij P_ij K_ij
  periodic_images -- the image atoms of a periodic cell's extended set
                     (Sec. 2: the cells N, G, H of Eq. H-HFX)
  K_periodic      -- exchange rows K^G_{mu lambda} of a periodic system,
                     Eq. H-HFX with the Gamma-point real-space density of
                     Eq. dm, by brute force over the extended set

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``
(closed forms, special functions from scipy/mpmath, brute-force numerical
quadrature of the six-dimensional integral, symmetry and invariance
identities); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hfx_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

KERNEL_COULOMB, KERNEL_ERFC, KERNEL_ERF = 0, 1, 2
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP).  Returns the library path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        D = ctypes.c_double
        I = ctypes.c_int
        P = ctypes.c_void_p
        lib.oracle_boys.argtypes = [I, D, P]
        lib.oracle_normalize.argtypes = [I, P, P, P, P, P]
        lib.oracle_quartets.argtypes = [I, P, P, P, P, P, P, I, P, I, D, P, P]
        lib.oracle_schwarz.argtypes = [I, P, P, P, P, P, P, I, D, P]
        lib.oracle_build_K.argtypes = [I, P, P, P, P, P, P, P, I, D, I, D, I, D, I, I, I, I, P]
        lib.oracle_build_K.restype = ctypes.c_longlong
        lib.oracle_K_shell_pairs.argtypes = [I, P, P, P, P, P, P, P, I, D, I, D, I, D, I, P, P, I, P, P, P]
        lib.oracle_K_shell_pairs.restype = ctypes.c_longlong
        lib.oracle_count_quartets.argtypes = [I, P, P, P, P, P, P, P, I, D, D, I, D, I, P]
        lib.oracle_count_quartets.restype = ctypes.c_longlong
        lib.oracle_periodic_images.argtypes = [I, P, P, D, ctypes.c_longlong, P]
        lib.oracle_periodic_images.restype = ctypes.c_longlong
        lib.oracle_K_periodic.argtypes = [I, P, P, P, P, P, P, I, P, P, D, D, P, I, D, I, D, I, D, I, P, P]
        lib.oracle_K_periodic.restype = ctypes.c_longlong
        lib.oracle_max_threads.restype = I
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def boys(mmax: int, x: float) -> np.ndarray:
    out = np.zeros(mmax + 1)
    _load().oracle_boys(int(mmax), float(x), _p(out))
    return out


class Basis:
    """Flat arrays of a ``synth.System`` as the oracle consumes them."""

    def __init__(self, sysobj):
        self.sys = sysobj
        self.n_shells = sysobj.n_shells
        self.xyz = np.ascontiguousarray(sysobj.atom_xyz[sysobj.shell_atom], dtype=np.float64)
        self.l = np.ascontiguousarray(sysobj.shell_l, dtype=np.int32)
        self.prim_off = np.ascontiguousarray(sysobj.prim_off, dtype=np.int32)
        self.alpha = np.ascontiguousarray(sysobj.alpha, dtype=np.float64)
        self.coef = normalize(sysobj)
        self.func_off = np.ascontiguousarray(sysobj.func_off, dtype=np.int64)
        self.nbf = int(self.func_off[-1])

    def args(self):
        return (self.n_shells, _p(self.xyz), _p(self.l), _p(self.prim_off), _p(self.alpha),
                _p(self.coef), _p(self.func_off))


def normalize(sysobj) -> np.ndarray:
    out = np.zeros_like(sysobj.coef, dtype=np.float64)
    raw = np.ascontiguousarray(sysobj.coef, dtype=np.float64)
    l = np.ascontiguousarray(sysobj.shell_l, dtype=np.int32)
    off = np.ascontiguousarray(sysobj.prim_off, dtype=np.int32)
    al = np.ascontiguousarray(sysobj.alpha, dtype=np.float64)
    _load().oracle_normalize(int(sysobj.n_shells), _p(l), _p(off), _p(al), _p(raw), _p(out))
    return out


def _basis(b):
    return b if isinstance(b, Basis) else Basis(b)


def quartets(basis, quads, kernel: int = KERNEL_COULOMB, omega: float = 0.11):
    """Contracted integrals of shell quartets (I J | K L); returns a list of
    arrays shaped (nI, nJ, nK, nL), Cartesian components in x,y,z /
    xx,xy,xz,yy,yz,zz order."""
    b = _basis(basis)
    q = np.ascontiguousarray(np.asarray(quads, dtype=np.int32).reshape(-1, 4))
    nf = np.diff(b.func_off)
    sizes = np.prod(nf[q], axis=1).astype(np.int64)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    out = np.zeros(int(off[-1]))
    _load().oracle_quartets(*b.args(), int(q.shape[0]), _p(q), int(kernel), float(omega),
                            _p(off), _p(out))
    return [out[off[i]:off[i + 1]].reshape(tuple(int(x) for x in nf[q[i]])) for i in range(q.shape[0])]


def schwarz(basis, kernel: int = KERNEL_COULOMB, omega: float = 0.11) -> np.ndarray:
    b = _basis(basis)
    Q = np.zeros((b.n_shells, b.n_shells))
    _load().oracle_schwarz(*b.args(), int(kernel), float(omega), _p(Q))
    return Q


def build_K(basis, P, kernel: int = KERNEL_COULOMB, omega: float = 0.11, screen: bool = False,
            tau: float = 1e-8, density_screen: bool = False, eps: float = 1e-8,
            brute: bool = False, bra_stride: int = 1, bra_offset: int = 0,
            nthreads: int | None = None):
    """K_ij = sum_kl (ik|jl) P_kl (dense FP64) and the number of surviving
    shell quartets (canonical, or ordered when ``brute``)."""
    b = _basis(basis)
    P = np.ascontiguousarray(P, dtype=np.float64)
    assert P.shape == (b.nbf, b.nbf)
    K = np.zeros_like(P)
    nt = max_threads() if nthreads is None else int(nthreads)
    n = _load().oracle_build_K(*b.args(), _p(P), int(kernel), float(omega), int(bool(screen)),
                               float(tau), int(bool(density_screen)), float(eps), int(bool(brute)),
                               int(bra_stride), int(bra_offset), nt, _p(K))
    return K, int(n)


def K_shell_pairs(basis, P, pairs, kernel: int = KERNEL_COULOMB, omega: float = 0.11,
                  screen: bool = False, tau: float = 1e-8, density_screen: bool = False,
                  eps: float = 1e-8, nthreads: int | None = None):
    """Exchange blocks K_IJ of the listed shell pairs (I, J) straight from the
    definition (all ordered (K, L) whose quartet (I K | J L) survives).
    Returns (blocks, W1, W0, n): lists of (nI, nJ) arrays -- K, the weights
    sum Q_IK Q_JL sum|P_kl| and sum |P_kl| over the surviving (K, L) -- and the
    number of surviving ordered shell quartets."""
    b = _basis(basis)
    P = np.ascontiguousarray(P, dtype=np.float64)
    assert P.shape == (b.nbf, b.nbf)
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    nf = np.diff(b.func_off)
    sizes = (nf[pr[:, 0]] * nf[pr[:, 1]]).astype(np.int64)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    K = np.zeros(int(off[-1]))
    W1 = np.zeros_like(K)
    W0 = np.zeros_like(K)
    nt = max_threads() if nthreads is None else int(nthreads)
    n = _load().oracle_K_shell_pairs(*b.args(), _p(P), int(kernel), float(omega), int(bool(screen)),
                                     float(tau), int(bool(density_screen)), float(eps), int(pr.shape[0]),
                                     _p(pr), _p(off), nt, _p(K), _p(W1), _p(W0))
    shp = [(int(nf[i]), int(nf[j])) for i, j in pr]
    cut = lambda a: [a[off[q]:off[q + 1]].reshape(shp[q]) for q in range(pr.shape[0])]
    return cut(K), cut(W1), cut(W0), int(n)


def count_quartets(basis, P, kernel: int = KERNEL_COULOMB, omega: float = 0.11, tau: float = 1e-8,
                   density_screen: bool = False, eps: float = 1e-8, nthreads: int | None = None):
    """Number of canonical shell quartets surviving Schwarz (and density)
    screening, counted without evaluating them; also returns the Schwarz
    bounds (ns x ns)."""
    b = _basis(basis)
    P = np.ascontiguousarray(P, dtype=np.float64)
    assert P.shape == (b.nbf, b.nbf)
    Q = np.zeros((b.n_shells, b.n_shells))
    nt = max_threads() if nthreads is None else int(nthreads)
    n = _load().oracle_count_quartets(*b.args(), _p(P), int(kernel), float(omega), float(tau),
                                      int(bool(density_screen)), float(eps), nt, _p(Q))
    return int(n), Q


def exchange_energy(P, K) -> float:
    """E_x = -1/2 sum_ij P_ij K_ij."""
    return float(-0.5 * np.sum(np.asarray(P) * np.asarray(K)))


def periodic_images(atom_xyz, lattice, r_ext: float) -> np.ndarray:
    """(n_images, 4) rows (home atom, n1, n2, n3): every translate of a home
    atom by n1 a1 + n2 a2 + n3 a3 (n != 0; lattice rows a_i) within ``r_ext``
    of some home atom, atom by atom, shifts in lexicographic order."""
    x = np.ascontiguousarray(atom_xyz, dtype=np.float64).reshape(-1, 3)
    A = np.ascontiguousarray(lattice, dtype=np.float64).reshape(3, 3)
    lib = _load()
    n = lib.oracle_periodic_images(int(x.shape[0]), _p(x), _p(A), float(r_ext), 0, None)
    if n < 0:
        raise ValueError("singular lattice or negative radius")
    out = np.zeros((max(int(n), 1), 4), dtype=np.int32)
    lib.oracle_periodic_images(int(x.shape[0]), _p(x), _p(A), float(r_ext), int(n), _p(out))
    return out[:int(n)]


def K_periodic(sysobj, P_home, lattice, r_ext: float, r_P: float, kernel: int = KERNEL_COULOMB,
               omega: float = 0.11, screen: bool = False, tau: float = 1e-8, density_screen: bool = False,
               eps: float = 1e-8, nthreads: int | None = None):
    """Exchange rows of a periodic system (Eq. H-HFX without the -1/2).

    Returns (K_rows, ext, n): K_rows (home nbf x extended nbf) with
    K_rows[mu, lambda^G] = sum_{N,H,nu,sigma} P^{H-N}_{nu sigma} (mu^0 nu^N | lambda^G sigma^H);
    ext (n_ext x 4) the extended atoms (home atom, n1, n2, n3), home atoms
    first, each carrying its home atom's functions in home order; n the
    number of surviving ordered shell quartets.  P^L_{nu sigma} is the home
    density P_home where the atoms of nu^0 and sigma^L are at most ``r_P``
    apart, else 0."""
    b = Basis(sysobj)
    P = np.ascontiguousarray(P_home, dtype=np.float64)
    assert P.shape == (b.nbf, b.nbf)
    x = np.ascontiguousarray(sysobj.atom_xyz, dtype=np.float64)
    A = np.ascontiguousarray(lattice, dtype=np.float64).reshape(3, 3)
    sa = np.ascontiguousarray(sysobj.shell_atom, dtype=np.int32)
    img = periodic_images(x, A, r_ext)
    ext = np.zeros((sysobj.n_atoms + img.shape[0], 4), dtype=np.int32)
    # every extended atom carries its home atom's functions
    nf_atom = np.diff(sysobj.atom_func_off)
    nbf_ext = int(nf_atom.sum() + nf_atom[img[:, 0]].sum())
    K = np.zeros((b.nbf, nbf_ext))
    nt = max_threads() if nthreads is None else int(nthreads)
    n = _load().oracle_K_periodic(b.n_shells, _p(sa), _p(b.l), _p(b.prim_off), _p(b.alpha), _p(b.coef),
                                  _p(b.func_off), int(sysobj.n_atoms), _p(x), _p(A), float(r_ext), float(r_P),
                                  _p(P), int(kernel), float(omega), int(bool(screen)), float(tau),
                                  int(bool(density_screen)), float(eps), nt, _p(ext), _p(K))
    if n < 0:
        raise ValueError("bad input (shells not grouped by atom, singular lattice or negative radius)")
    return K, ext, int(n)
