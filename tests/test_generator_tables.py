"""Node tables of the generated ERI code (CPU, no GPU needed).

The warp kernels interpret two generated tables per angular-momentum class:
the horizontal-recursion nodes and the output slots.  The warp-split kernels
also use the permutation that maps their reduce-scatter order to accumulator
slots.  These tests check, for all 21 classes:
  * every slot index is inside the shared-memory workspace the kernels
    allocate, and nodes of one level (run by different lanes at once) never
    read a slot that another node of the same level writes;
  * the table-driven horizontal recursion, interpreted the way the kernels
    do it, equals the Head-Gordon-Pople horizontal recursion written out
    recursively (along the other Cartesian axis where there is a choice) on
    random contracted [e0|f0] values and random AB, CD;
  * the split permutation is a permutation of the accumulators, and the four
    P blocks of the exchange contraction fit the 160-value staging buffer.
"""
import functools
import importlib.util
import os

import numpy as np
import pytest

_GEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2009_03555_gb300", "csrc",
                    "gen_eri.py")


@functools.lru_cache(maxsize=1)
def _gen():
    spec = importlib.util.spec_from_file_location("gen_eri_for_tests", _GEN)
    g = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(g)
    return g


def _classes():
    return [c[2:] for c in _gen().quartet_classes()]


def _decode(node):
    x, y = node[0], node[1]
    return x & 0xFFFF, (x >> 16) & 3, (x >> 18) & 3, y & 0xFFFF, y >> 16


@pytest.mark.parametrize("cls", _classes(), ids=lambda c: "".join(map(str, c)))
def test_hrr_tables(cls):
    g = _gen()
    la, lb, lc, ld = cls
    t = g.coop_tables(la, lb, lc, ld)
    hs, nacc = t["hrr_slots"], t["nacc"]
    na, nb, nc, nd = (len(g.comps(l)) for l in cls)
    assert len(t["outs"]) == na * nb * nc * nd
    assert len(set(t["outs"])) == len(t["outs"]) and max(t["outs"]) < hs
    written = set(range(nacc))
    offs = t["hlev_off"]
    assert offs[0] == offs[1] == 0 and offs[t["n_hlev"] + 1] == len(t["hnodes"])
    for lev in range(1, t["n_hlev"] + 1):
        level = [_decode(n) for n in t["hnodes"][offs[lev]:offs[lev + 1]]]
        dsts = {d for d, *_ in level}
        for dst, kind, axis, s1, s2 in level:
            assert nacc <= dst < hs and s1 < hs and s2 < hs
            assert kind in (2, 3) and axis in (0, 1, 2)
            assert s1 in written and s2 in written  # written by an earlier level or an accumulator
            assert s1 not in dsts and s2 not in dsts
        written |= dsts

    # numerical: table interpretation against the recursion written out
    rng = np.random.default_rng(sum(10 ** k * l for k, l in enumerate(cls)))
    acc = rng.standard_normal(nacc)
    AB, CD = rng.uniform(-3, 3, 3), rng.uniform(-3, 3, 3)
    ws = np.zeros(hs)
    ws[:nacc] = acc
    for node in t["hnodes"]:  # level order: the order the kernels run them in
        dst, kind, axis, s1, s2 = _decode(node)
        ws[dst] = ws[s1] + (AB if kind == 2 else CD)[axis] * ws[s2]
    got = ws[t["outs"]]

    v = g.VRR(la, lb, lc, ld)
    eidx = {e: i for i, e in enumerate(v.E)}
    fidx = {f: i for i, f in enumerate(v.F)}
    nf = len(v.F)

    def step(u, i, k):
        w = list(u)
        w[i] += k
        return tuple(w)

    @functools.lru_cache(maxsize=None)
    def bra(a, b, f):  # (a b | f 0]
        if sum(b) == 0:
            return acc[eidx[a] * nf + fidx[f]]
        i = max(k for k in range(3) if b[k] > 0)
        return bra(step(a, i, 1), step(b, i, -1), f) + AB[i] * bra(a, step(b, i, -1), f)

    @functools.lru_cache(maxsize=None)
    def ket(a, b, c, d):  # (a b | c d)
        if sum(d) == 0:
            return bra(a, b, c)
        i = max(k for k in range(3) if d[k] > 0)
        return ket(a, b, step(c, i, 1), step(d, i, -1)) + CD[i] * ket(a, b, c, step(d, i, -1))

    ref = np.array([ket(a, b, c, d) for a in g.comps(la) for b in g.comps(lb) for c in g.comps(lc)
                    for d in g.comps(ld)])
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("cls", _classes(), ids=lambda c: "".join(map(str, c)))
def test_split_permutation_and_p_blocks(cls):
    g = _gen()
    la, lb, lc, ld = cls
    _, nchunk, _, perm = g.gen_vrr_split(la, lb, lc, ld)
    nacc = g.coop_tables(la, lb, lc, ld)["nacc"]
    assert sorted(perm) == list(range(nacc)) and nchunk == (nacc + 31) // 32
    na, nb, nc, nd = (len(g.comps(l)) for l in cls)
    assert na * nc + nb * nd + na * nd + nb * nc <= 160
