"""Node tables of the generated ERI code (CPU, no GPU needed).

The warp kernels interpret generated tables per angular-momentum class: the
horizontal-recursion nodes and the output slots, the permutation that maps the
split kernels' reduce-scatter order to accumulator slots, and (table kernel)
the vertical-recursion nodes.  These tests check, for all 21 classes:
  * every slot index is inside the shared-memory workspace the kernels
    allocate, and nodes of one level (run by different lanes at once) never
    read a slot that another node of the same level writes;
  * the table-driven horizontal recursion, interpreted the way the kernels
    do it, equals the Head-Gordon-Pople horizontal recursion written out
    recursively (along the other Cartesian axis where there is a choice) on
    random contracted [e0|f0] values and random AB, CD;
  * the split permutation is a permutation of the accumulators, and the four
    P blocks of the exchange contraction fit the 160-value staging buffer;
  * the vertical-recursion tables equal the Obara-Saika recursion written out
    recursively, likewise on random G_m and geometry.
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
    # slots are reused once their value is dead, so a level may write a slot
    # that held an accumulator or an earlier node; the lanes run one level in
    # parallel, so no level may read a slot it writes, nor write one twice
    written = set(range(nacc))
    offs = t["hlev_off"]
    assert offs[0] == offs[1] == 0 and offs[t["n_hlev"] + 1] == len(t["hnodes"])
    for lev in range(1, t["n_hlev"] + 1):
        level = [_decode(n) for n in t["hnodes"][offs[lev]:offs[lev + 1]]]
        dsts = [d for d, *_ in level]
        assert len(dsts) == len(set(dsts))
        for dst, kind, axis, s1, s2 in level:
            assert 0 <= dst < hs and s1 < hs and s2 < hs
            assert kind in (2, 3) and axis in (0, 1, 2)
            assert s1 in written and s2 in written  # written by an earlier level or an accumulator
            assert s1 not in dsts and s2 not in dsts
        written |= set(dsts)

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


@pytest.mark.parametrize("cls", _classes(), ids=lambda c: "".join(map(str, c)))
def test_vrr_tables(cls):
    """The vertical-recursion node tables (interpreted as the table kernel
    does: slot 0 = 0, slots 1..L+1 = G_0..G_L, bra nodes then ket nodes level
    by level) equal the Obara-Saika recursion written out recursively along
    the other axis where there is a choice, on random G_m and geometry."""
    g = _gen()
    la, lb, lc, ld = cls
    L = la + lb + lc + ld
    t = g.coop_tables(la, lb, lc, ld)
    rng = np.random.default_rng(7 + sum(10 ** k * l for k, l in enumerate(cls)))
    G = rng.uniform(0.1, 1.0, L + 1)
    PA, QC, WP, WQ = (rng.uniform(-1, 1, 3) for _ in range(4))
    oo2p, oo2q, oo2pq, rop, roq = rng.uniform(0.1, 1.0, 5)
    ws = np.zeros(t["vrr_slots"])
    ws[1:L + 2] = G
    for node in t["nodes"]:
        x, y, z, w = node
        dst, kind, axis = x & 0xFFFF, (x >> 16) & 3, (x >> 18) & 3
        k1, k2 = (x >> 20) & 15, (x >> 24) & 15
        s0, s1, s2, s3 = y & 0xFFFF, y >> 16, z & 0xFFFF, z >> 16
        assert max(dst, s0, s1, s2, s3, w) < t["vrr_slots"]
        if kind == 0:
            ws[dst] = PA[axis] * ws[s0] + WP[axis] * ws[s1] + k1 * oo2p * (ws[s2] - rop * ws[s3])
        else:
            ws[dst] = (QC[axis] * ws[s0] + WQ[axis] * ws[s1] + k1 * oo2q * (ws[s2] - roq * ws[s3])
                       + k2 * oo2pq * ws[w])
    got = ws[t["targets"]]

    def sub(u, i):
        v = list(u)
        v[i] -= 1
        return tuple(v)

    @functools.lru_cache(maxsize=None)
    def r(e, f, m):  # [e0|f0]^(m)
        if sum(e) < 0 or min(e) < 0 or min(f) < 0:
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

    v = g.VRR(la, lb, lc, ld)
    ref = np.array([r(e, f, 0) for e in v.E for f in v.F])
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_per_class_settings_name_classes_of_the_right_kernel():
    """The generator's per-class tables name real classes of the kernel they
    configure: launch bounds and ket prefetch only per-thread classes (fewer
    than SPLIT_MIN_ACC contracted accumulators), warps per block and
    shared-memory accumulators only warp-split classes, with 12 or 16 warps."""
    g = _gen()
    classes = {tuple(c) for c in _classes()}
    assert len(classes) == 21

    def nacc(c):
        v = g.VRR(*c)
        return len(v.E) * len(v.F)

    for c in list(g.PT_MIN_BLOCKS) + list(g.PT_PREFETCH):
        assert c in classes and nacc(c) < g.SPLIT_MIN_ACC, c
    for c in list(g.SPLIT_WARPS) + list(g.SPLIT_SMEM_ACC):
        assert c in classes and nacc(c) >= g.SPLIT_MIN_ACC, c
    assert set(g.SPLIT_WARPS.values()) <= {12, 16}
