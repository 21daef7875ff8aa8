"""The library's host algebra of the tabulated reaction M2L
(csrc/table_algebra.h, compiled on the CPU with g++) against the oracle's
independent expansion (oracle/tables.py; Sec. 3.5, eqs. identitypolyexp,
asslegendreexpcoef, metoletableform): the same index set of S integrals, and
for every operator entry the same tables with the same coefficients once the
oracle's phases i^{n+n'+1+m'-m} s_t s_s are folded in."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import tables as tb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = tmp_path_factory.mktemp("tabalg") / "check_table_algebra"
    src = os.path.join(ROOT, "tests", "cpp", "check_table_algebra.cpp")
    inc = os.path.join(ROOT, "paper_1902_05132_gb300", "csrc")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", inc, src, "-o", str(out)], check=True)
    return str(out)


@pytest.mark.parametrize("p,kl,klp,a", [(4, 0.8, 1.2, 0), (6, 1.6, 1.2, 1), (8, 1.2, 1.2, 0), (12, 0.8, 1.6, 1)])
def test_table_algebra_matches_oracle_expansion(exe, p, kl, klp, a):
    r = subprocess.run([exe, str(p), repr(kl), repr(klp), str(a)], capture_output=True, text=True, check=True)
    lines = r.stdout.strip().split("\n")
    head = [int(v) for v in lines[0].split()]
    ntab, keys = head[0], head[1:]
    ex = tb.Expansion(p, kl, klp)
    assert ntab == len(ex.index)
    assert [tuple(keys[4 * i:4 * i + 4]) for i in range(ntab)] == ex.index
    got = {}
    for ln in lines[1:]:
        v = ln.split()
        i, j, k = int(v[0]), int(v[1]), int(v[2])
        got[(i, j)] = [(int(v[3 + 3 * x]), float(v[4 + 3 * x]) + 1j * float(v[5 + 3 * x])) for x in range(k)]
    up = (a == 0)
    P = len(ex.ns)
    worst = 0.0
    for i in range(P):
        n, m = ex.ns[i], ex.ms[i]
        st = 1 if up else (-1) ** ((n + m) % 2)
        for j in range(P):
            n2, m2 = ex.ns[j], ex.ms[j]
            ss = (-1) ** n2 if up else (-1) ** (m2 % 2)
            ph = st * ss * 1j ** ((n + n2 + 1 + (m2 - m)) % 4)
            want = sorted((x, c * ph) for x, c in ex.terms[(i, j)])
            have = sorted(got.get((i, j), []))
            assert [x for x, _ in have] == [x for x, _ in want], (i, j)
            for (_, c1), (_, c2) in zip(have, want):
                worst = max(worst, abs(c1 - c2) / max(abs(c2), 1e-300))
    assert worst < 1e-11, worst
