"""The C-ABI library loads and exports every function include/hfx.h declares
(no compute: runs without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hfx.h")


def declared_functions(path):
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hfx_[A-Za-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2009_03555_gb300 import build as B
    from paper_2009_03555_gb300 import hfx
    if not os.path.exists(hfx.LIB_PATH):
        B.build()
    return hfx.load()


def test_header_declares_the_boundary():
    names = declared_functions(HEADER)
    for n in ("hfx_create_basis", "hfx_build_quartets", "hfx_build_K", "hfx_exchange_energy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2009_03555_gb300 import hfx
    names = declared_functions(HEADER)
    out = subprocess.run(["nm", "-D", "--defined-only", hfx.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hfx_[A-Za-z_]+)\b", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)


def test_class_table(lib):
    from paper_2009_03555_gb300 import hfx
    seen = set()
    for c in range(hfx.N_CLASSES):
        ci = hfx.hfx_get_class_info(c)
        assert ci.la >= ci.lb and ci.lc >= ci.ld and ci.bra_class >= ci.ket_class
        n = lambda l: (l + 1) * (l + 2) // 2
        assert ci.n_out == n(ci.la) * n(ci.lb) * n(ci.lc) * n(ci.ld)
        # [e0|f0] accumulators: e over la..la+lb, f over lc..lc+ld
        ne = sum(n(l) for l in range(ci.la, ci.la + ci.lb + 1))
        nf = sum(n(l) for l in range(ci.lc, ci.lc + ci.ld + 1))
        assert ci.n_acc == ne * nf
        # kernel family by accumulator count: per-thread below 90, warp-split from 90 up
        # (the cooperative kernel is opt-in, HFX_COOP_MIN_ACC)
        assert ci.kernel_kind == (1 if ci.n_acc >= 90 else 0)
        seen.add((ci.la, ci.lb, ci.lc, ci.ld))
    assert len(seen) == 21
    with pytest.raises(hfx.HFXError):
        hfx.hfx_get_class_info(21)
