"""The argument behind the chain pre-test's convexity test (keller_on_edge in
the CUDA sources), restated in numpy and checked by brute force.

The unfolded length of a chain is convex in the edge parameters, so its
derivative along one edge, e.(Q - A)/|Q - A| + e.(Q - B)/|Q - B| for the
neighbours A and B of the point Q on that edge, grows as Q moves along the
edge. If that derivative is positive at the edge's start (less a margin) for
every position of the neighbours on their edges, or negative at its end,
the minimum has Q (or a neighbour) off its edge. The bound of
e.(Q - Y)/|Q - Y| over Y on a segment uses the arc that the directions from
Q to the segment sweep: its extremes are at the arc's ends or at +-|e_p|,
e_p the projection of e onto the arc's plane, where e_p points into the arc.

Checked here: that bound against dense sampling of the segment, and that no
random chain rejected by the test has its true minimum (scipy) on its edges.
This restates the rule; the GPU parity tests check that the pre-test drops no
path the oracle finds."""
import numpy as np
import pytest


def _unit(v):
    return v / np.linalg.norm(v)


def cos_over_edge(e, Q, p0, es, lo, hi):
    """(min, max) of e.(Q - Y)/|Q - Y| for Y = p0 + es s, s in [lo, hi], and
    a lower bound of |Q - Y|."""
    d0, d1 = Q - p0 - es * lo, Q - p0 - es * hi
    l0, l1 = np.linalg.norm(d0), np.linalg.norm(d1)
    c0, c1 = e @ d0 / l0, e @ d1 / l1
    cmin, cmax = min(c0, c1), max(c0, c1)
    n = np.cross(d0, d1)
    nn = np.linalg.norm(n)
    dmin = min(l0, l1, nn / (hi - lo))
    if nn > 1e-3 * l0 * l1:
        u = n / nn
        en = e @ u
        pn = np.sqrt(max(0.0, 1.0 - en * en))
        ep = e - en * u
        s0, s1 = ep @ np.cross(u, d0), ep @ np.cross(d1, u)
        g0, g1 = 1e-3 * l0, 1e-3 * l1
        if s0 >= -g0 and s1 >= -g1:
            cmax = max(cmax, pn)
        if s0 <= g0 and s1 <= g1:
            cmin = min(cmin, -pn)
    else:  # an arc shorter than 1e-3 rad
        cmin, cmax = cmin - 2e-3, cmax + 2e-3
    return cmin, cmax, dmin


def keller_on_edge(W, F, S1, S2, m):
    """False when no Keller point can lie within m of edge W, its neighbours
    being point F (or a point of edge S1 when F is None) and a point of edge
    S2, both edges widened by m. Edges: (start, unit direction, length)."""
    for q in (0, 1):
        t = W[2] + m if q else -m
        Q = W[0] + W[1] * t
        if F is not None:
            d = Q - F
            d1 = np.linalg.norm(d)
            lo1 = hi1 = W[1] @ d / d1
        else:
            lo1, hi1, d1 = cos_over_edge(W[1], Q, S1[0], S1[1], -m, S1[2] + m)
        lo2, hi2, d2 = cos_over_edge(W[1], Q, S2[0], S2[1], -m, S2[2] + m)
        if not (d1 > 4 * m and d2 > 4 * m):
            return True
        err = 4e-5
        if q == 0 and lo1 + lo2 > err:
            return False
        if q == 1 and hi1 + hi2 < -err:
            return False
    return True


def _edge(rng):
    return (rng.normal(size=3) * 3, _unit(rng.normal(size=3)), rng.uniform(0.5, 4.0))


def test_cosine_bound_holds_over_the_segment():
    rng = np.random.default_rng(1)
    for _ in range(5000):
        e = _unit(rng.normal(size=3))
        Q = rng.normal(size=3) * 3
        p0, es, L = _edge(rng)
        lo, hi = -0.05, L + 0.05
        cmin, cmax, dmin = cos_over_edge(e, Q, p0, es, lo, hi)
        s = np.linspace(lo, hi, 4001)
        V = Q - p0 - es * s[:, None]
        d = np.linalg.norm(V, axis=1)
        c = V @ e / d
        assert c.min() >= cmin - 1e-9 and c.max() <= cmax + 1e-9
        assert d.min() >= dmin - 1e-9


@pytest.mark.parametrize("m", [2, 3])
def test_rejected_chains_have_their_minimum_off_an_edge(m):
    scipy_opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(2 + m)
    rejected = 0
    for _ in range(600):
        T, R = rng.normal(size=3) * 10, rng.normal(size=3) * 10
        W = [_edge(rng) for _ in range(m)]

        def length(t):
            P = [T] + [w[0] + w[1] * ti for w, ti in zip(W, t)] + [R]
            return sum(np.linalg.norm(P[i + 1] - P[i]) for i in range(len(P) - 1))

        tests = [keller_on_edge(W[0], T, None, W[1], 0.05), keller_on_edge(W[-1], R, None, W[-2], 0.05)]
        if m == 3:
            tests.append(keller_on_edge(W[1], None, W[0], W[2], 0.05))
        if all(tests):
            continue
        rejected += 1
        res = scipy_opt.minimize(length, [w[2] / 2 for w in W], method="BFGS", options={"gtol": 1e-10})
        on_edges = all(-1e-6 <= ti <= w[2] + 1e-6 for ti, w in zip(res.x, W))
        assert not on_edges, (W, T, R, res.x)
    assert rejected > 400  # the test rejects most random chains
