"""Host-only helpers of the library (no GPU needed): the value layout of an
atom-pair pattern (count and dense packing) and the setup memory estimate
used for admission, checked against a plain numpy restatement."""
import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def lib():
    from paper_2009_03555_gb300 import hfx
    try:
        return hfx.load()
    except ImportError as e:  # the library is built by __graft_entry__.build()
        pytest.skip(str(e))


def _numpy_pack(s, mask, dense):
    fo = s.atom_func_off
    vals = []
    for X in range(s.n_atoms):
        for Y in np.flatnonzero(mask[X]):
            vals.append(dense[fo[X]:fo[X + 1], fo[Y]:fo[Y + 1]].ravel())
    return np.concatenate(vals)


@pytest.mark.parametrize("make", [lambda: synth.ch_chain(7, sub=5), lambda: synth.ch_cluster(5, 9)])
def test_pattern_value_count_and_pack(lib, make):
    from paper_2009_03555_gb300 import hfx
    s = make()
    mask = synth.atom_pair_mask(s, 6.0)
    inp = hfx._SystemInput(s, mask)
    dense = np.random.default_rng(3).standard_normal((s.n_bf, s.n_bf))
    ref = _numpy_pack(s, mask, dense)
    assert inp.value_count() == ref.size
    np.testing.assert_array_equal(inp.pack(dense), ref)


def test_setup_estimate_grows_with_pairs(lib):
    from paper_2009_03555_gb300 import hfx
    e = []
    for n in (4, 8, 16):
        s = synth.ch_chain(n, sub=6)
        e.append(hfx._SystemInput(s, synth.atom_pair_mask(s, 6.0)).setup_bytes_estimate())
    assert 0 < e[0] < e[1] < e[2]
    # at least every shell pair's primitive pairs (128 B each, 16 per pair)
    ns = synth.ch_chain(16, sub=6).n_shells
    assert e[2] >= ns * (ns + 1) // 2 * 16 * 128


def test_host_helpers_reject_inconsistent_input(lib):
    """Shells that name an atom outside the pattern, columns out of range and
    NULL buffers are refused (-1 or HFX_ERR_INVALID_ARG), never read past."""
    import ctypes
    from paper_2009_03555_gb300 import hfx
    s = synth.ch_chain(3, sub=7)
    inp = hfx._SystemInput(s, synth.atom_pair_mask(s, 6.0))
    assert inp.value_count() > 0
    # a pattern over fewer atoms than the shells use
    small = hfx.Pattern(2, inp.row_ptr.ctypes.data, inp.col.ctypes.data)
    assert lib.hfx_pattern_value_count(inp.descs, inp.n_shells, ctypes.byref(small)) == -1
    assert lib.hfx_setup_bytes_estimate(inp.descs, inp.n_shells, ctypes.byref(small)) == -1
    # a column index out of range
    bad_col = inp.col.copy()
    bad_col[-1] = s.n_atoms
    bad = hfx.Pattern(s.n_atoms, inp.row_ptr.ctypes.data, bad_col.ctypes.data)
    assert lib.hfx_pattern_value_count(inp.descs, inp.n_shells, ctypes.byref(bad)) == -1
    out = np.empty(inp.value_count())
    dense = np.zeros((s.n_bf, s.n_bf))
    st = lib.hfx_pack_dense_host(inp.descs, inp.n_shells, ctypes.byref(bad), hfx._ptr(dense), hfx._ptr(out))
    assert st == 1 and b"inconsistent" in lib.hfx_last_error()
    # NULL buffers
    assert lib.hfx_pack_dense_host(inp.descs, inp.n_shells, ctypes.byref(inp.pattern), None, hfx._ptr(out)) == 1
    assert lib.hfx_pattern_value_count(inp.descs, 0, ctypes.byref(inp.pattern)) == -1


def test_single_atom_pattern(lib):
    """The smallest system: one atom, its diagonal block only."""
    from paper_2009_03555_gb300 import hfx
    s = synth.ch_chain(1, sub=8)
    mask = np.ones((1, 1), dtype=bool)
    inp = hfx._SystemInput(s, mask)
    assert inp.value_count() == s.n_bf * s.n_bf
    dense = np.random.default_rng(4).standard_normal((s.n_bf, s.n_bf))
    np.testing.assert_array_equal(inp.pack(dense), dense.ravel())
