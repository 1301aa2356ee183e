"""CPU-side checks of the C-ABI library: it loads, exports every symbol the
header declares, and its host logic (boundary extraction, monotone split)
agrees with the oracle and with the mathematics.  No kernel is launched."""
import os
import re

import numpy as np
import pytest

import gen
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2408_04466_gb300 import build
    build.build()
    import paper_2408_04466_gb300 as pkg
    return pkg


def _declared():
    src = open(os.path.join(ROOT, "include", "gwn.h")).read()
    return sorted(set(re.findall(r"GWN_API\s+[^;(]*?\b(gwn_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    so = ctypes.CDLL(lib._capi.LIB_PATH)
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(so, n), n
    assert set(names) == set(lib._capi.exported_symbols())
    assert b"sm_103a" in lib.load().gwn_version()


def _loops_to_edges(off, vid):
    edges = []
    for j in range(len(off) - 1):
        lo, hi = off[j], off[j + 1]
        for i in range(lo, hi):
            edges.append((int(vid[i]), int(vid[i + 1] if i + 1 < hi else vid[lo])))
    return edges


def _oracle_unit_edges(F):
    src, dst, m = oracle.boundary_edges(F)
    out = []
    for s, t, k in zip(src, dst, m):
        out += [(int(s), int(t))] * int(k)
    return sorted(out)


@pytest.mark.parametrize("name", ["cap", "torus", "soup", "heightfield"])
def test_boundary_extraction_matches_oracle(lib, name):
    if name == "cap":
        m = gen.icosphere_cap(subdiv=4)
        V, F = m.V, m.F
    elif name == "torus":
        m = gen.slit_torus(n_u=48, n_v=40, n_queries=16)
        V, F = m.V, m.F
    elif name == "heightfield":
        m = gen.holey_heightfield(n=96, n_holes=3)
        V, F = m.V, m.F
    else:
        rng = np.random.default_rng(3)
        V = rng.standard_normal((30, 3)).astype(np.float32)
        F = rng.integers(0, 30, (80, 3)).astype(np.int32)
        F = np.concatenate([F, F[:7], F[:3, [0, 2, 1]]])   # multiplicities 2, 0 and degenerate faces
    off, vid = lib.boundary_extract_host(F, len(V))
    got = sorted(_loops_to_edges(off, vid))
    assert got == _oracle_unit_edges(F)
    # every loop is closed and consecutive
    for j in range(len(off) - 1):
        assert off[j + 1] > off[j]
    if name == "cap":
        assert len(off) - 1 == 1
    if name == "torus":
        assert len(off) - 1 == 2 and len(vid) == 2 * 40


def test_boundary_extraction_closed_and_empty(lib):
    V, F = gen.icosphere(2)
    off, vid = lib.boundary_extract_host(F.astype(np.int32), len(V))
    assert len(off) == 1 and len(vid) == 0
    off, vid = lib.boundary_extract_host(np.zeros((0, 3), np.int32), 0)
    assert len(off) == 1 and len(vid) == 0


def test_boundary_extraction_rejects_bad_indices(lib):
    with pytest.raises(lib.GwnError):
        lib.boundary_extract_host(np.array([[0, 1, 5]], np.int32), 3)


def test_monotone_split(lib):
    rng = np.random.default_rng(0)
    for _ in range(300):
        c = rng.standard_normal(8)
        u = lib.monotone_split_host(c)
        assert u[0, 0] == 0.0 and u[-1, 1] == 1.0
        assert np.all(u[1:, 0] == u[:-1, 1])
        y = c[1::2]
        # y(u) must be monotone on every piece: check on a fine sample
        for a, b in u:
            t = np.linspace(a, b, 200)
            v = 1 - t
            yy = v ** 3 * y[0] + 3 * t * v * v * y[1] + 3 * t * t * v * y[2] + t ** 3 * y[3]
            dy = np.diff(yy)
            assert np.all(dy >= -1e-12) or np.all(dy <= 1e-12)
        # cut points are the roots of y'(u) in (0, 1)
        d0, d1, d2 = y[1] - y[0], y[2] - y[1], y[3] - y[2]
        roots = np.roots([d0 - 2 * d1 + d2, 2 * (d1 - d0), d0]) if abs(d0 - 2 * d1 + d2) > 1e-12 else \
            (np.array([-d0 / (2 * (d1 - d0))]) if d1 != d0 else np.array([]))
        roots = np.sort(np.real(roots[np.isreal(roots)]))
        roots = roots[(roots > 0) & (roots < 1)]
        assert len(u) == len(roots) + 1
        assert np.allclose(u[1:, 0], roots, atol=1e-9)
