"""The coupling table baked into the CUDA kernels, checked on the CPU against
the oracle.  The kernels' table comes from the build-time generator
(csrc/gen_tables.cpp: Gaunt integrals by quadrature, row-normalised, sign by
the first entry); the oracle's real CG tensors come from Racah's formula and
the real-basis change.  Both follow the same definition by different routes;
here every path, every nonzero entry and the entry ordering the kernels rely
on are compared (the table is emitted in FP32 and FP64)."""
import os
import re
import subprocess

import numpy as np
import pytest

import oracle

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2605_22698_gb300", "csrc")


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    d = tmp_path_factory.mktemp("gen")
    exe, inc = str(d / "gen_tables"), str(d / "cg_tables.inc")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, "-o", exe, os.path.join(CSRC, "gen_tables.cpp")], check=True)
    subprocess.run([exe, inc], check=True)
    text = open(inc).read()
    out = {}
    for m in re.finditer(r"struct CGTable(P?)<(\d)> \{(.*?)\n\};", text, re.S):
        key, body = (int(m.group(2)), m.group(1) == "P"), m.group(3)
        arrs = {}
        for a in re.finditer(r"static constexpr (?:int|float|double) (\w+)\[\d+\] = \{([^}]*)\};", body):
            arrs[a.group(1)] = np.array([float(x.rstrip("f")) for x in a.group(2).split(",")])
        out[key] = arrs
    assert set(out) == {(2, False), (3, False), (2, True), (3, True)}
    return out


VARIANTS = [(2, False), (3, False), (2, True), (3, True)]  # (l_max, every parity)


@pytest.mark.parametrize("L,allp", VARIANTS)
def test_paths_match_the_oracle(tables, L, allp):
    t = tables[(L, allp)]
    got = list(zip(t["l1"].astype(int), t["l2"].astype(int), t["l3"].astype(int)))
    assert got == oracle.paths(L, 3, all_parities=allp)


@pytest.mark.parametrize("L,allp", VARIANTS)
def test_entries_match_the_oracle(tables, L, allp):
    """Natural-parity paths: Gaunt integrals; odd l1 + l2 + l3 (the mixed-parity
    table): integrals of Y_l3 r.(grad Y_l1 x grad Y_l2); both against the
    oracle's Racah-based real tensors."""
    t = tables[(L, allp)]
    off = t["off"].astype(int)
    for p, (l1, l2, l3) in enumerate(oracle.paths(L, 3, all_parities=allp)):
        C = oracle.real_cg(l1, l2, l3)  # [m3][m1][m2]
        dense = np.zeros_like(C)
        for k in range(off[p], off[p + 1]):
            assert int(t["ep"][k]) == p
            i3, i1, i2 = int(t["e3"][k]), int(t["e1"][k]), int(t["e2"][k])
            assert l3 * l3 <= i3 < (l3 + 1) ** 2 and l1 * l1 <= i1 < (l1 + 1) ** 2 and l2 * l2 <= i2 < (l2 + 1) ** 2
            dense[i3 - l3 * l3, i1 - l1 * l1, i2 - l2 * l2] = t["ecd"][k]
            assert abs(t["ec"][k] - t["ecd"][k]) <= 1e-7 * abs(t["ecd"][k])
        np.testing.assert_allclose(dense, C, atol=1e-12)
        # no entry of the oracle's tensor above the emission threshold is missing
        assert off[p + 1] - off[p] == int((np.abs(C) > 1e-12).sum())


@pytest.mark.parametrize("L", [2, 3])
def test_contraction_couplings_are_the_table_paths_with_l1_le_l2(tables, L):
    t = tables[(L, False)]
    sub = [(int(a), int(b), int(c)) for a, b, c in zip(t["l1"], t["l2"], t["l3"]) if a <= b <= L]
    assert sub == oracle.sc_paths(L)
