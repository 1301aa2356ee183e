"""Pins for the 2D oracle: closed forms and agreement of three independent
methods (adaptive quadrature of the definition, Algorithm 1 with one ray in
the largest arc, and the +x-ray closed form)."""
import json
import math
import os

import numpy as np

import gen
import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def test_straight_segment():
    g = GOLD["segment_2d"]
    ctrl = np.array(g["control_points"], np.float64)
    P = np.array([g["query"]], np.float64)
    for f in (oracle.w2d_quad, oracle.w2d_alg1):
        assert abs(f(ctrl, P)[0] - g["w"]) < 1e-14
    assert abs(oracle.w2d_closed_x(ctrl, P)[0][0] - g["w"]) < 1e-14
    # arbitrary straight segments vs the atan2 of the end points
    rng = np.random.default_rng(0)
    for _ in range(50):
        s, e, p = rng.standard_normal((3, 2))
        ctrl = np.stack([s, s + (e - s) / 3, s + 2 * (e - s) / 3, e])
        a = math.atan2((s - p)[0] * (e - p)[1] - (s - p)[1] * (e - p)[0], (s - p) @ (e - p))
        for f in (oracle.w2d_quad, oracle.w2d_alg1):
            assert abs(f(ctrl, p[None])[0] - a / (2 * math.pi)) < 1e-13


def test_antipodal_arc_is_half():
    # cubic from (1,0) over the top to (-1,0): end points antipodal from 0
    k = 4 / 3 * (math.sqrt(2) - 1) * 2
    ctrl = np.array([[1, 0], [1, k], [-1, k], [-1, 0]], np.float64)
    P = np.zeros((1, 2))
    for f in (oracle.w2d_quad, oracle.w2d_alg1):
        assert abs(f(ctrl, P)[0] - GOLD["antipodal_arc_2d"]["w_abs"]) < 1e-14
    assert abs(oracle.w2d_quad(ctrl[::-1].copy(), P)[0] + 0.5) < 1e-14


def test_closed_chain_is_integer():
    # closed star-shaped chain (last control point = first)
    m = 3 * 24
    th = 2 * np.pi * np.arange(m + 1) / m
    r = 1 + 0.2 * np.cos(5 * th)
    ctrl = np.stack([r * np.cos(th), r * np.sin(th)], 1)
    ctrl[-1] = ctrl[0]
    rng = np.random.default_rng(1)
    P = rng.uniform(-1.5, 1.5, (400, 2))
    dist = oracle.dist2d(ctrl, P)
    P = P[dist > 1e-3]
    wq = oracle.w2d_quad(ctrl, P)
    inside = np.abs(wq - 1) < 1e-9
    outside = np.abs(wq) < 1e-9
    assert np.all(inside | outside) and inside.sum() > 20 and outside.sum() > 20
    wa = oracle.w2d_alg1(ctrl, P)
    wc, chi = oracle.w2d_closed_x(ctrl, P)
    assert np.abs(wa - wq).max() < 1e-12 and np.abs(wc - wq).max() < 1e-12


def test_three_methods_agree_on_the_circle_chain():
    c = gen.bezier_circle_chain()
    P = gen.grid_points(c.grids[0], np.float64)
    dist = oracle.dist2d(c.ctrl, P)
    keep = dist > 1e-4 * math.hypot(3.0, 3.0)
    wq = oracle.w2d_quad(c.ctrl, P)
    wa = oracle.w2d_alg1(c.ctrl, P)
    wc, chi = oracle.w2d_closed_x(c.ctrl, P)
    assert np.abs(wq - wa)[keep].max() < 1e-13
    assert np.abs(wq - wc)[keep].max() < 1e-13
    assert np.abs(wa - wc)[keep].max() < 1e-13


def test_chain_ray_crossings_sign_convention():
    # upward straight segment at x = 1: the +x ray from the origin crosses it
    # counter-clockwise -> +1; the -x ray misses it
    ctrl = np.array([[1, -1], [1, -0.3], [1, 0.3], [1, 1]], np.float64)
    assert oracle.chain_ray_crossings(ctrl, [0, 0], [1, 0]) == 1
    assert oracle.chain_ray_crossings(ctrl, [0, 0], [-1, 0]) == 0
    assert oracle.chain_ray_crossings(ctrl[::-1].copy(), [0, 0], [1, 0]) == -1
    # an S-shaped cubic crossed three times by the x axis
    ctrl = np.array([[1, -1], [4, 3], [-2, -3], [1, 1]], np.float64)
    g = ctrl[:, 1]
    assert oracle.chain_ray_crossings(ctrl, [-10, 0], [1, 0]) == 1   # +1 -1 +1


def test_star_chains_small_three_methods():
    ch = gen.star_chains(n_chains=3, seg_hi=64, grid_n=24, seed=2)
    for c in range(3):
        ctrl = ch.ctrl[ch.offsets[c]:ch.offsets[c + 1]].astype(np.float64)
        P = gen.grid_points(ch.grids[c], np.float64)
        g = ch.grids[c]
        diag = math.hypot(g.hi[0] - g.lo[0], g.hi[1] - g.lo[1])
        keep = oracle.dist2d(ctrl, P) > 1e-4 * diag
        wq = oracle.w2d_quad(ctrl, P)
        wc, chi = oracle.w2d_closed_x(ctrl, P)
        wa = oracle.w2d_alg1(ctrl, P)
        assert np.abs(wq - wc)[keep].max() < 1e-12
        assert np.abs(wa - wc)[keep].max() < 1e-12


def test_crossing_counts_certified_near_the_curve():
    """The +x-ray count with its certification, on curves whose crossings are
    known exactly.  (a) Two straight cubic segments (0,0)-(3,3)-(6,0): on the
    row y = 3/2 the crossings are at x = 3/2 (upward) and 9/2 (downward); a
    query 2^-40 to either side of x = 3/2 is decided correctly and certified,
    one 2^-50 away is flagged (it lies on the curve at float64 resolution).
    (b) y = x - x^2/3 on [0, 3] (one cubic, apex (3/2, 3/4)): just below the
    apex a query between the two crossings counts -1, outside them 0; on the
    apex row the count is 0 and only queries within float64 resolution of
    the apex are flagged.  (c) The chord side: a chain from (0,0) to (2,2)
    bulging to the right closes with the chord along y = x; a query 2^-40
    left or right of it is decided exactly."""
    line = np.array([[0, 0], [1, 1], [2, 2], [3, 3], [4, 2], [5, 1], [6, 0]], np.float64)
    eps = 2.0 ** -40
    P = np.array([[1.5 - eps, 1.5], [1.5 + eps, 1.5], [1.5 - 2.0 ** -50, 1.5], [1.5 + 2.0 ** -50, 1.5],
                  [0.2, 1.5], [5.0, 1.5]])
    _, chi, unc = oracle.w2d_closed_x(line, P, want_unc=True)
    assert chi[:2].tolist() == [0, -1] and not unc[:2].any()
    assert unc[2] and unc[3]
    assert chi[4:].tolist() == [0, 0] and not unc[4:].any()
    para = np.array([[0, 0], [1, 1], [2, 1], [3, 0]], np.float64)    # x = 3u, y = 3u(1-u)
    for d in (2.0 ** -30, 2.0 ** -44):
        half = math.sqrt(3.0 * d)                                   # crossings at 3/2 -+ sqrt(3 d)
        yr = 0.75 - d
        P = np.array([[1.5, yr], [1.5 - 2 * half, yr], [1.5 + 2 * half, yr]])
        _, chi, unc = oracle.w2d_closed_x(para, P, want_unc=True)
        assert chi.tolist() == [-1, 0, 0] and not unc.any(), (d, chi, unc)
    P = np.array([[0.2, 0.75], [2.9, 0.75], [1.5, 0.75 + 2.0 ** -40], [1.5, 0.75]])
    _, chi, unc = oracle.w2d_closed_x(para, P, want_unc=True)
    assert chi[:3].tolist() == [0, 0, 0] and not unc[:3].any()
    assert unc[3]                                                    # the apex itself
    bulge = np.array([[0, 0], [2, 0], [2, 0], [2, 2]], np.float64)
    P = np.array([[1.0 - eps, 1.0], [1.0 + eps, 1.0]])
    _, chi, unc = oracle.w2d_closed_x(bulge, P, want_unc=True)
    # row y = 1: the curve crosses at x = 2 - ... > 1 (upward, +1); the chord
    # (2,2) -> (0,0) crosses at x = 1 (downward): counted only left of it
    assert chi.tolist() == [0, 1] and not unc.any(), (chi, unc)
