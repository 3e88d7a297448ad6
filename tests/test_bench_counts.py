"""The roofline's flop counts (CPU): the costs of the double-single operations
that bench.py composes into the mixed-path prologue count, derived here from
the device code itself (boys_ds.cuh).  Each helper's body is scanned for its
FP32 intrinsics (add, subtract, multiply: 1 flop; FMA: 2; reciprocal and
reciprocal square root seeds: 1), plain products written with '*', and calls
of the other helpers."""
import os
import re

import pytest

import bench

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2009_03555_gb300", "csrc",
                   "boys_ds.cuh")
HELPERS = ["two_sum", "fast_two_sum", "ds_add", "ds_sub", "ds_mul", "ds_mulf", "ds_addf", "ds_rcp", "ds_rsqrt"]


def _bodies():
    text = open(SRC).read()
    out = {}
    for name in HELPERS:
        m = re.search(r"__device__ __forceinline__ ds " + name + r"\(([^)]*)\)\s*\{", text)
        assert m, name
        i, depth = m.end(), 1
        while depth:
            depth += {"{": 1, "}": -1}.get(text[i], 0)
            i += 1
        out[name] = text[m.end():i - 1]
    return out


def _cost(name, bodies, memo):
    if name in memo:
        return memo[name]
    body = re.sub(r"//[^\n]*", "", bodies[name])
    n = 0
    n += len(re.findall(r"__f(?:add|sub|mul)_rn\(", body))
    n += 2 * len(re.findall(r"(?:__fmaf_rn|fmaf)\(", body))
    n += len(re.findall(r"(?:__frcp_rn|rsqrtf)\(", body))
    n += len(re.findall(r"[\w)]\s*\*\s*[\w(]", body))  # plain products such as 0.5f * y
    for other in HELPERS:
        calls = len(re.findall(r"\b" + other + r"\(", body)) if other != name else 0
        if calls:
            n += calls * _cost(other, bodies, memo)
    memo[name] = n
    return n


@pytest.fixture(scope="module")
def costs():
    bodies = _bodies()
    memo = {}
    return {h: _cost(h, bodies, memo) for h in HELPERS}


def test_double_single_operation_costs(costs):
    assert costs["two_sum"] == 6 and costs["fast_two_sum"] == 3
    assert costs["ds_add"] == bench.DS_ADD
    assert costs["ds_sub"] == bench.DS_ADD
    assert costs["ds_mul"] == bench.DS_MUL
    assert costs["ds_mulf"] == bench.DS_MULF
    assert costs["ds_addf"] == bench.DS_ADDF
    assert costs["ds_rcp"] == bench.DS_RCP
    assert costs["ds_rsqrt"] == bench.DS_RSQRT


def test_prologue_counts_grow_as_stated():
    # erfc: the attenuation factor (76), a second Boys evaluation (70 + 66 + 25 L for L > 0) and 33 per
    # G_m on top of Coulomb's 8
    for L in range(1, 9):
        c, e = bench.ds_prologue_flops(L, 0), bench.ds_prologue_flops(L, 1)
        assert e - c == 76 + (70 + 66 + 25 * L) + 25 * (L + 1)
        assert bench.ds_prologue_flops(L, 1) - bench.ds_prologue_flops(L - 1, 1) == (50 if L > 1 else 50 + 132) + 33
    assert bench.ds_prologue_flops(6, 1) == 1059 and bench.ds_prologue_flops(8, 1) == 1225
    assert bench.fp64_prologue_flops(8, 1) == 205
