"""The generated straight-line ERI code, compiled for the host (CPU, no GPU).

The per-class headers the generator writes hold the code the kernels run:
`vrr` (per-thread vertical recursion into contracted [e0|f0] accumulators),
`vrr_split` (the same targets in 32-target chunks, each handed to the warp
reduce-scatter, with the permutation back to accumulator order) and `hrr`
(horizontal recursion to the Cartesian integrals).  Here every class is
generated with split code (in both target orders of the split recursion), compiled with g++ behind a small host shim (the
warp reduce-scatter replaced by a recorder of each chunk's 32 values) and run
on random G_m and geometry; the results must equal the Obara-Saika and
Head-Gordon-Pople recursions written out in Python (along the other axis where
there is a choice).
"""
import ctypes
import functools
import importlib.util
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_GEN = os.path.join(ROOT, "paper_2009_03555_gb300", "csrc", "gen_eri.py")

SHIM = r"""
#pragma once
#define __device__
#define __forceinline__ inline
#define __noinline__
#define __restrict__
struct uint4 { unsigned x, y, z, w; };
namespace hfx {
template <typename R> struct VrrGeo { R PA[3], QC[3], WP[3], WQ[3]; R oo2p, oo2q, oo2pq, rop, roq; };
template <typename R> inline void kacc(R& s, R& c, R v) { (void)c; s += v; }
extern double* g_sink;
extern int g_nchunk;
// host stand-in for the warp chunk reduction: record the chunk's 32 values
template <typename R> inline R chunk_reduce32(R (&v)[32], R* buf) {
  (void)buf;
  for (int i = 0; i < 32; ++i) g_sink[g_nchunk * 32 + i] = (double)v[i];
  ++g_nchunk;
  return R(0);
}
}  // namespace hfx
"""


def _gen_module():
    spec = importlib.util.spec_from_file_location("gen_eri_host", _GEN)
    g = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(g)
    return g


@pytest.fixture(scope="module", params=["grouped", "greedy"])
def built(request, tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    g = _gen_module()
    g.SPLIT_MIN_ACC = 1        # emit split code for every class
    g.COOP_MIN_ACC = 10 ** 9
    g.VRR_ORDER = request.param  # both target orders of the split recursion
    d = tmp_path_factory.mktemp("gen_host")
    g.generate(str(d))
    (d / "eri_common.cuh").write_text(SHIM)
    classes = [c[2:] for c in g.quartet_classes()]
    src = ['#include "cls_%d%d%d%d.cuh"' % c for c in classes]
    src.append("namespace hfx { double* g_sink; int g_nchunk; }")
    src.append("using namespace hfx;")
    have = {}
    for la, lb, lc, ld in classes:
        n = "Cls%d%d%d%d" % (la, lb, lc, ld)
        text = (d / f"cls_{la}{lb}{lc}{ld}.cuh").read_text()
        # per-thread code (the per-thread build kernel, Schwarz bounds, diagnostics) is in every header
        have[n] = "static void vrr(" in text and "static void hrr(" in text
        src.append(f"""
static VrrGeo<double> geo_{n}(const double* q) {{
  VrrGeo<double> g;
  for (int x = 0; x < 3; ++x) {{ g.PA[x] = q[x]; g.QC[x] = q[3 + x]; g.WP[x] = q[6 + x]; g.WQ[x] = q[9 + x]; }}
  g.oo2p = q[12]; g.oo2q = q[13]; g.oo2pq = q[14]; g.rop = q[15]; g.roq = q[16];
  return g;
}}
extern "C" int vrr_split_{n}(const double* G, const double* q, double* sink) {{
  double acc[{n}::NCHUNK], comp[{n}::NCHUNK];
  for (int i = 0; i < {n}::NCHUNK; ++i) acc[i] = comp[i] = 0.0;
  g_sink = sink; g_nchunk = 0;
  {n}::vrr_split<double>(G, geo_{n}(q), acc, comp, nullptr);
  return g_nchunk;
}}
extern "C" const unsigned short* perm_{n}() {{ return {n}::split_perm(); }}
""")
        if have[n]:
            src.append(f"""
extern "C" void vrr_{n}(const double* G, const double* q, double* acc) {{
  double comp[{n}::NACC];
  for (int i = 0; i < {n}::NACC; ++i) acc[i] = comp[i] = 0.0;
  {n}::vrr<double>(G, geo_{n}(q), acc, comp);
}}
extern "C" void hrr_{n}(const double* acc, const double* ab, const double* cd, double* out) {{
  {n}::hrr<double>(acc, ab[0], ab[1], ab[2], cd[0], cd[1], cd[2], out);
}}
""")
    (d / "host.cpp").write_text("\n".join(src))
    lib = d / "libgenhost.so"
    r = subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-I", str(d), str(d / "host.cpp"), "-o",
                        str(lib)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return g, ctypes.CDLL(str(lib)), have


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _classes():
    return [c[2:] for c in _gen_module().quartet_classes()]


@pytest.mark.parametrize("cls", _classes(), ids=lambda c: "".join(map(str, c)))
def test_generated_vrr_split_and_hrr(built, cls):
    g, lib, have = built
    la, lb, lc, ld = cls
    n = "Cls%d%d%d%d" % cls
    L = la + lb + lc + ld
    v = g.VRR(la, lb, lc, ld)
    nacc = len(v.E) * len(v.F)
    rng = np.random.default_rng(11 + sum(10 ** k * l for k, l in enumerate(cls)))
    G = rng.uniform(0.1, 1.0, L + 1)
    q = np.concatenate([rng.uniform(-1, 1, 12), rng.uniform(0.1, 1.0, 5)])
    PA, QC, WP, WQ = q[0:3], q[3:6], q[6:9], q[9:12]
    oo2p, oo2q, oo2pq, rop, roq = q[12:17]

    def sub(u, i):
        w = list(u)
        w[i] -= 1
        return tuple(w)

    @functools.lru_cache(maxsize=None)
    def r(e, f, m):  # [e0|f0]^(m), Obara-Saika
        if min(e) < 0 or min(f) < 0:
            return 0.0
        if sum(f) > 0:
            i = max(k for k in range(3) if f[k] > 0)
            f1 = sub(f, i)
            out = QC[i] * r(e, f1, m) + WQ[i] * r(e, f1, m + 1)
            if f1[i] > 0:
                out += f1[i] * oo2q * (r(e, sub(f1, i), m) - roq * r(e, sub(f1, i), m + 1))
            if e[i] > 0:
                out += e[i] * oo2pq * r(sub(e, i), f1, m + 1)
            return out
        if sum(e) > 0:
            i = max(k for k in range(3) if e[k] > 0)
            e1 = sub(e, i)
            out = PA[i] * r(e1, f, m) + WP[i] * r(e1, f, m + 1)
            if e1[i] > 0:
                out += e1[i] * oo2p * (r(sub(e1, i), f, m) - rop * r(sub(e1, i), f, m + 1))
            return out
        return G[m]

    ref = np.array([r(e, f, 0) for e in v.E for f in v.F])
    tol = dict(rtol=1e-10, atol=1e-12 * np.abs(ref).max())

    if have[n]:
        acc = np.zeros(nacc)
        getattr(lib, f"vrr_{n}")(_ptr(G), _ptr(q), _ptr(acc))
        np.testing.assert_allclose(acc, ref, **tol)

    nchunk = (nacc + 31) // 32
    sink = np.zeros(nchunk * 32)
    f = getattr(lib, f"vrr_split_{n}")
    f.restype = ctypes.c_int
    assert f(_ptr(G), _ptr(q), _ptr(sink)) == nchunk
    pf = getattr(lib, f"perm_{n}")
    pf.restype = ctypes.POINTER(ctypes.c_ushort)
    perm = np.array([pf()[t] for t in range(nacc)])
    split_acc = np.zeros(nacc)
    split_acc[perm] = sink[:nacc]  # chunk k, slot j holds target 32k + j, stored at accumulator perm[32k + j]
    np.testing.assert_allclose(split_acc, ref, **tol)
    assert np.all(sink[nacc:] == 0.0)

    # horizontal recursion of the generated per-thread code
    if not have[n]:
        return
    AB, CD = rng.uniform(-3, 3, 3), rng.uniform(-3, 3, 3)
    out = np.zeros(len(g.comps(la)) * len(g.comps(lb)) * len(g.comps(lc)) * len(g.comps(ld)))
    getattr(lib, f"hrr_{n}")(_ptr(ref), _ptr(AB), _ptr(CD), _ptr(out))
    eidx = {e: i for i, e in enumerate(v.E)}
    fidx = {f: i for i, f in enumerate(v.F)}
    nf = len(v.F)

    def step(u, i, k):
        w = list(u)
        w[i] += k
        return tuple(w)

    @functools.lru_cache(maxsize=None)
    def bra(a, b, fv):
        if sum(b) == 0:
            return ref[eidx[a] * nf + fidx[fv]]
        i = max(k for k in range(3) if b[k] > 0)
        return bra(step(a, i, 1), step(b, i, -1), fv) + AB[i] * bra(a, step(b, i, -1), fv)

    @functools.lru_cache(maxsize=None)
    def ket(a, b, c, d):
        if sum(d) == 0:
            return bra(a, b, c)
        i = max(k for k in range(3) if d[k] > 0)
        return ket(a, b, step(c, i, 1), step(d, i, -1)) + CD[i] * ket(a, b, c, step(d, i, -1))

    want = np.array([ket(a, b, c, d) for a in g.comps(la) for b in g.comps(lb) for c in g.comps(lc)
                     for d in g.comps(ld)])
    np.testing.assert_allclose(out, want, rtol=1e-10, atol=1e-10 * np.abs(want).max())
