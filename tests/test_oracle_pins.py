"""Pins for the CPU oracle: checks against closed forms, invariants, exact
polynomial cases and an independent ODE solver, never against the oracle itself.

The paper names the method (direct summation, Hermite 4th/6th/8th order,
individual block time-steps; abstract and "Codes description") but prints no
formulas, so every pin here fixes the mathematics those names imply.  Each test
is chosen so that a plausible slip (a dropped term, a wrong sign, a wrong
coefficient or power) fails it.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import polynomial as P

pytestmark = []


# --------------------------------------------------------------------------
# Force: closed forms
# --------------------------------------------------------------------------

def test_two_body_softened_force_closed_form(orc):
    # m_j = 2 at distance 3 along x, softening 4 on j only: eps_ij^2 = max = 16.
    # |A| = m d / (d^2 + eps^2)^(3/2) = 2*3/125, pointing from i to j.
    m = np.array([1.0, 2.0])
    x = np.array([[0.0, 0, 0], [3.0, 0, 0]])
    v = np.zeros((2, 3))
    eps2 = np.array([0.0, 16.0])
    out = orc.force(m, eps2, x, v, np.zeros((2, 3)), np.zeros((2, 3)), order=8, idx=[0, 1])
    assert out["acc"][0] == pytest.approx([6.0 / 125, 0, 0], abs=1e-17)
    assert out["acc"][1] == pytest.approx([-3.0 / 125, 0, 0], abs=1e-17)
    # potential -m_j / R = -2/5 on particle 0 and -1/5 on particle 1
    assert out["pot"] == pytest.approx([-0.4, -0.2], rel=1e-15)
    # at rest with zero acceleration every time derivative vanishes
    for k in ("jerk", "snap", "crackle"):
        assert np.all(out[k] == 0)


def test_equilateral_triangle_force(orc):
    # three unit masses on a triangle of side s: each feels sqrt(3)/s^2 toward the centre
    s = 1.7
    ang = np.array([90.0, 210.0, 330.0]) * math.pi / 180
    rad = s / math.sqrt(3)
    x = np.stack([rad * np.cos(ang), rad * np.sin(ang), np.zeros(3)], axis=1)
    out = orc.force(np.ones(3), np.zeros(3), x, np.zeros((3, 3)), np.zeros((3, 3)), order=6)
    for i in range(3):
        mag = np.linalg.norm(out["acc"][i])
        assert mag == pytest.approx(math.sqrt(3) / s ** 2, rel=1e-14)
        # points to the centre
        assert np.dot(out["acc"][i], -x[i]) / (mag * rad) == pytest.approx(1.0, rel=1e-14)
    assert out["pot"] == pytest.approx([-2.0 / s] * 3, rel=1e-14)


def test_circular_relative_motion_jerk(orc):
    # Unsoftened pair in uniform circular relative motion: A rotates with the
    # angular speed w, so |J| = w|A|, |S| = w^2|A|, |C| = w^3|A| and J is
    # perpendicular to A.  Relative velocity w*d tangential; relative acc -w^2 d radial.
    d, w, mj = 0.8, 1.3, 0.7
    x = np.array([[0.0, 0, 0], [d, 0, 0]])
    v = np.array([[0.0, 0, 0], [0, w * d, 0]])
    a = np.array([[0.0, 0, 0], [-w * w * d, 0, 0]])
    jk = np.array([[0.0, 0, 0], [0, -w ** 3 * d, 0]])
    out = orc.force(np.array([1.0, mj]), np.zeros(2), x, v, a, jk, order=8, idx=[0])
    A = mj / d ** 2
    assert out["acc"][0] == pytest.approx([A, 0, 0], rel=1e-15)
    assert out["jerk"][0] == pytest.approx([0, w * A, 0], abs=1e-14)
    assert out["snap"][0] == pytest.approx([-w * w * A, 0, 0], abs=1e-14)
    assert out["crackle"][0] == pytest.approx([0, -w ** 3 * A, 0], abs=1e-14)


def _poly_traj(rng, n, deg):
    """Random polynomial trajectories x_i(t) = sum_k c_ik t^k, k <= deg."""
    return rng.normal(size=(n, 3, deg + 1)) * (0.5 ** np.arange(deg + 1))


def _eval(coef, t, der=0):
    n = coef.shape[0]
    out = np.zeros((n, 3))
    for i in range(n):
        for c in range(3):
            out[i, c] = P.polyval(t, P.polyder(coef[i, c], der) if der else coef[i, c])
    return out


def test_finite_difference_derivatives(orc):
    # Particles on prescribed cubic trajectories.  The force's J, S, C must be the
    # 1st, 2nd, 3rd time derivatives of A along those trajectories, measured by
    # Richardson-extrapolated central differences.
    rng = np.random.default_rng(7)
    n = 16
    coef = _poly_traj(rng, n, 3)
    coef[:, :, 0] += rng.normal(size=(n, 3)) * 2.0  # spread the positions out
    m = rng.uniform(0.5, 1.5, n)
    eps2 = np.full(n, 0.01)
    t0 = 0.3

    def state(t):
        return _eval(coef, t), _eval(coef, t, 1), _eval(coef, t, 2), _eval(coef, t, 3)

    def A(t):
        x, v, a, j = state(t)
        return orc.force(m, eps2, x, v, a, j, order=8)["acc"]

    x, v, a, j = state(t0)
    F = orc.force(m, eps2, x, v, a, j, order=8)

    def d1(h):
        return (A(t0 - 2 * h) - 8 * A(t0 - h) + 8 * A(t0 + h) - A(t0 + 2 * h)) / (12 * h)

    def d2(h):
        return (-A(t0 - 2 * h) + 16 * A(t0 - h) - 30 * A(t0) + 16 * A(t0 + h) - A(t0 + 2 * h)) / (12 * h * h)

    def d3(h):
        return (A(t0 - 3 * h) - 8 * A(t0 - 2 * h) + 13 * A(t0 - h) - 13 * A(t0 + h) + 8 * A(t0 + 2 * h)
                - A(t0 + 3 * h)) / (8 * h ** 3)

    h = 2e-3
    J_fd = (16 * d1(h / 2) - d1(h)) / 15
    S_fd = (16 * d2(h / 2) - d2(h)) / 15
    C_fd = (16 * d3(h / 2) - d3(h)) / 15
    scale = lambda q: np.max(np.abs(q))  # noqa: E731
    assert np.max(np.abs(F["jerk"] - J_fd)) / scale(F["jerk"]) < 1e-9
    assert np.max(np.abs(F["snap"] - S_fd)) / scale(F["snap"]) < 1e-6
    assert np.max(np.abs(F["crackle"] - C_fd)) / scale(F["crackle"]) < 1e-4


def test_total_force_antisymmetry(orc):
    # Newton's third law with symmetric pair softening: sum m_i a_i = 0 and the
    # same for every time derivative.
    rng = np.random.default_rng(3)
    n = 200
    x = rng.normal(size=(n, 3))
    v = rng.normal(size=(n, 3))
    a = rng.normal(size=(n, 3))
    j = rng.normal(size=(n, 3))
    m = rng.uniform(0.1, 1, n)
    eps2 = rng.choice([0.0, 1e-4, 1e-2], n)
    F = orc.force(m, eps2, x, v, a, j, order=8)
    for k in ("acc", "jerk", "snap", "crackle"):
        tot = (m[:, None] * F[k]).sum(axis=0)
        mag = (m[:, None] * np.abs(F[k])).sum()
        assert np.all(np.abs(tot) < 1e-15 * mag), k


def test_potential_energy_closed_form(orc):
    # equilateral triangle of masses 1, 2, 3, side 2, softening 0.5 on particle 1
    s = 2.0
    x = np.array([[0, 0, 0], [s, 0, 0], [s / 2, s * math.sqrt(3) / 2, 0]])
    v = np.array([[1.0, 0, 0], [0, 2, 0], [0, 0, 3]])
    m = np.array([1.0, 2, 3])
    eps2 = np.array([0.0, 0.25, 0.0])
    ek, ep = orc.energy(m, eps2, x, v)
    assert ek == pytest.approx(0.5 * 1 + 0.5 * 2 * 4 + 0.5 * 3 * 9, rel=1e-15)
    r_soft = math.sqrt(s * s + 0.25)
    assert ep == pytest.approx(-(1 * 2 / r_soft + 1 * 3 / s + 2 * 3 / r_soft), rel=1e-15)


def test_single_active_matches_longdouble_sum(orc):
    # N_act = 1 over N = 4096: acceleration and potential against a numpy
    # extended-precision sum of Newton's law (a second, independent evaluation).
    rng = np.random.default_rng(11)
    n = 4096
    x = rng.normal(size=(n, 3))
    m = rng.uniform(0.5, 1.5, n) / n
    eps2 = np.full(n, 1e-6)
    i = 137
    F = orc.force(m, eps2, x, np.zeros((n, 3)), np.zeros((n, 3)), order=6, idx=[i])
    xl = x.astype(np.longdouble)
    r = xl - xl[i]
    r2 = (r * r).sum(axis=1) + np.longdouble(1e-6)
    w = m.astype(np.longdouble) / (r2 * np.sqrt(r2))
    w[i] = 0
    acc = (w[:, None] * r).sum(axis=0)
    phi = -(m.astype(np.longdouble) / np.sqrt(r2))
    phi[i] = 0
    assert np.allclose(F["acc"][0], acc.astype(np.float64), rtol=1e-15, atol=0)
    assert F["pot"][0] == pytest.approx(float(phi.sum()), rel=1e-15)


# --------------------------------------------------------------------------
# Predictor, corrector, interpolation: exact on polynomials
# --------------------------------------------------------------------------

@pytest.mark.parametrize("order", [4, 6, 8])
def test_predictor_exact_on_polynomials(orc, order):
    # x(t) a polynomial of the degree the predictor reaches: 5 for orders 4/6,
    # 7 for order 8.  Predicted x, v (and a, jerk where they are predicted)
    # must equal the polynomial and its derivatives at the target time.
    deg = 7 if order == 8 else 5
    rng = np.random.default_rng(order)
    n = 5
    coef = _poly_traj(rng, n, deg)
    t0 = rng.uniform(0, 0.1, n)
    t = 0.17
    x = np.array([_eval(coef[i:i + 1], t0[i])[0] for i in range(n)])
    v = np.array([_eval(coef[i:i + 1], t0[i], 1)[0] for i in range(n)])
    d = np.zeros((n, 6, 3))
    for k in range(6):
        d[:, k] = np.array([_eval(coef[i:i + 1], t0[i], k + 2)[0] for i in range(n)])
    xp, vp, ap, jp = orc.predict(order, t, t0, x, v, d)
    assert np.allclose(xp, _eval(coef, t), rtol=1e-14, atol=1e-14)
    assert np.allclose(vp, _eval(coef, t, 1), rtol=1e-14, atol=1e-14)
    if order >= 6:
        # a is predicted to the crackle term (order 6) or to a^(5) (order 8):
        # exact, since a of this x is a polynomial of degree deg - 2
        assert np.allclose(ap, _eval(coef, t, 2), rtol=1e-13, atol=1e-13)
    if order == 8:
        assert np.allclose(jp, _eval(coef, t, 3), rtol=1e-13, atol=1e-13)


def test_predictor_truncation_is_the_stated_one(orc):
    # order 6: x to the crackle term (dt^5), v to dt^4, a to dt^3.  A particle
    # with only a^(4) non-zero is not moved at all by the order-6 predictor;
    # with only crackle it moves by c dt^5/120.
    d = np.zeros((1, 6, 3))
    d[0, 4] = [1.0, 0, 0]
    xp, vp, ap, _ = orc.predict(6, 0.5, [0.0], np.zeros((1, 3)), np.zeros((1, 3)), d)
    assert np.all(xp == 0) and np.all(vp == 0) and np.all(ap == 0)
    d[0, 4] = 0
    d[0, 3] = [1.0, 0, 0]
    xp, vp, ap, _ = orc.predict(6, 0.5, [0.0], np.zeros((1, 3)), np.zeros((1, 3)), d)
    assert xp[0, 0] == pytest.approx(0.5 ** 5 / 120, rel=1e-15)
    assert vp[0, 0] == pytest.approx(0.5 ** 4 / 24, rel=1e-15)
    assert ap[0, 0] == pytest.approx(0.5 ** 3 / 6, rel=1e-15)


@pytest.mark.parametrize("mm", [2, 3, 4])
def test_interpolation_reproduces_polynomial(orc, mm):
    # acc(t) of degree 2mm-1 is fixed by its first mm derivatives at both ends;
    # the interpolant must return its higher derivatives at the end exactly.
    # Small-integer coefficients and h = 1/4 make every input exact in double,
    # so the only error left is the oracle's own (long double) solve.
    rng = np.random.default_rng(100 + mm)
    deg = 2 * mm - 1
    coef = rng.integers(-50, 51, size=(3, deg + 1)).astype(float)
    h = 0.25
    D0 = np.array([[P.polyval(0.0, P.polyder(coef[c], k)) for c in range(3)] for k in range(mm)])
    D1 = np.array([[P.polyval(h, P.polyder(coef[c], k)) for c in range(3)] for k in range(mm)])
    want = np.array([[P.polyval(h, P.polyder(coef[c], k)) for c in range(3)] for k in range(mm, 2 * mm)])
    got = orc.interp(mm, h, D0, D1)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("order", [4, 6, 8])
def test_corrector_exact_and_order(orc, order):
    # For x(t) of degree `order` the corrector is exact (v-rule exact for a of
    # degree order-2, x-rule exact for v of degree order-1).  For degree order+1
    # the one-step error must fall as h^(order+1).
    rng = np.random.default_rng(order + 20)

    def one(deg, h):
        coef = rng.normal(size=(1, 3, deg + 1))
        x0, v0 = _eval(coef, 0.0)[0], _eval(coef, 0.0, 1)[0]
        D0 = np.array([_eval(coef, 0.0, k + 2)[0] for k in range(4)])
        D1 = np.array([_eval(coef, h, k + 2)[0] for k in range(4)])
        x1, v1 = orc.correct(order, h, x0, v0, D0, D1)
        return np.max(np.abs(x1 - _eval(coef, h)[0])), np.max(np.abs(v1 - _eval(coef, h, 1)[0]))

    ex, ev = one(order, 0.3)
    assert ex < 1e-14 and ev < 1e-14
    rng = np.random.default_rng(order + 21)
    coef = rng.normal(size=(1, 3, order + 2))
    coef[0, :, order + 1] = 1.0

    def err(h):
        x0, v0 = _eval(coef, 0.0)[0], _eval(coef, 0.0, 1)[0]
        D0 = np.array([_eval(coef, 0.0, k + 2)[0] for k in range(4)])
        D1 = np.array([_eval(coef, h, k + 2)[0] for k in range(4)])
        x1, _ = orc.correct(order, h, x0, v0, D0, D1)
        return np.max(np.abs(x1 - _eval(coef, h)[0]))

    e1, e2 = err(0.4), err(0.2)
    assert math.log2(e1 / e2) == pytest.approx(order + 1, abs=0.15)


# --------------------------------------------------------------------------
# Time step
# --------------------------------------------------------------------------

@pytest.mark.parametrize("order", [4, 6, 8])
def test_timestep_criterion_circular_orbit(orc, order):
    # For uniform circular motion a^(k) has magnitude w^k |a|, so the
    # generalised criterion gives eta / w (orders 6, 8) and the classic Aarseth
    # form sqrt(eta) / w (order 4).
    w, amp, eta = 2.5, 0.9, 0.2
    ph = 0.37
    D = np.array([[amp * w ** k * math.cos(ph + k * math.pi / 2), amp * w ** k * math.sin(ph + k * math.pi / 2), 0.0]
                  for k in range(order)])
    dt = orc.dt_criterion(order, eta, D)
    want = math.sqrt(eta) / w if order == 4 else eta / w
    assert dt == pytest.approx(want, rel=1e-14)


def _fg_series(kmax):
    """Lagrange f and g series of the Kepler problem: the k-th time derivative
    of the relative position is F_k r + G_k v, with F_k, G_k polynomials in
    u = M/r^3, p = r.v/r^2, q = v.v/r^2 - u.  They follow from r'' = -u r by
    differentiating along the orbit, with du/dt = -3up, dp/dt = q - 2p^2,
    dq/dt = -p(u + 2q) (textbook celestial mechanics).  This route uses the
    equation of motion only, none of the oracle's pair formulas."""
    import sympy as sp
    u, p, q = sp.symbols("u p q")

    def ddt(e):
        return sp.diff(e, u) * (-3 * u * p) + sp.diff(e, p) * (q - 2 * p ** 2) + sp.diff(e, q) * (-p * (u + 2 * q))

    F, G = [sp.Integer(1)], [sp.Integer(0)]
    for _ in range(kmax):
        F, G = F + [sp.expand(ddt(F[-1]) - u * G[-1])], G + [sp.expand(F[-1] + ddt(G[-1]))]
    return [sp.lambdify((u, p, q), f) for f in F], [sp.lambdify((u, p, q), g) for g in G]


_FG = {}


def _kepler_derivatives(r, v, M, kmax=9):
    """d^k r / dt^k for k = 0..kmax of the relative orbit at (r, v)."""
    if kmax not in _FG:
        _FG[kmax] = _fg_series(kmax)
    F, G = _FG[kmax]
    rr = float(r @ r)
    u = M / rr ** 1.5
    p, q = float(r @ v) / rr, float(v @ v) / rr - u
    return np.array([F[k](u, p, q) * r + G[k](u, p, q) * v for k in range(kmax + 1)])


def _kepler_state(e, t, a=1.0, M=1.0):
    """Relative position and velocity at time t after apocentre (Kepler's equation)."""
    n = math.sqrt(M / a ** 3)
    mean = math.pi + n * t
    E = mean
    for _ in range(100):
        E -= (E - e * math.sin(E) - mean) / (1 - e * math.cos(E))
    Ed = n / (1 - e * math.cos(E))
    b = a * math.sqrt(1 - e * e)
    return (np.array([a * (math.cos(E) - e), b * math.sin(E), 0.0]),
            np.array([-a * math.sin(E) * Ed, b * math.cos(E) * Ed, 0.0]))


@pytest.mark.parametrize("t", [math.pi, 2.9, 0.7])
def test_force_derivatives_on_an_eccentric_orbit(orc, t):
    # Unsoftened pair (0.3 + 0.7) on an e = 0.9 orbit, at pericentre (t = pi
    # after apocentre, where r.v = 0), just before it (where alpha, beta and
    # gamma are all large and non-zero) and far out.  Body i's acceleration is
    # (m_j / M) times the relative one, so its acc, jerk, snap and crackle are
    # (m_j / M) r^(2..5), taken from the f and g series.  Each pair term of
    # the force derivatives (the 3 alpha A of J, the 6 alpha J + 3 beta A of S,
    # the 9 alpha S + 9 beta J + 3 gamma A of C) is large here, so a dropped
    # term, a wrong coefficient or a wrong sign fails.
    M, m = 1.0, np.array([0.3, 0.7])
    r, v = _kepler_state(0.9, t, M=M)
    D = _kepler_derivatives(r, v, M, 5)
    sgn = np.array([1.0, -1.0])  # x0 - x1 = r
    frac = np.array([m[1] / M, m[0] / M])
    x = np.array([sgn[i] * frac[i] * D[0] for i in range(2)])
    vv = np.array([sgn[i] * frac[i] * D[1] for i in range(2)])
    aa = np.array([sgn[i] * frac[i] * D[2] for i in range(2)])
    jj = np.array([sgn[i] * frac[i] * D[3] for i in range(2)])
    out = orc.force(m, np.zeros(2), x, vv, aa, jj, order=8)
    for k, key in enumerate(("acc", "jerk", "snap", "crackle")):
        for i in range(2):
            want = sgn[i] * frac[i] * D[k + 2]
            assert np.max(np.abs(out[key][i] - want)) <= 1e-12 * np.linalg.norm(want), (key, i)


@pytest.mark.parametrize("order", [6, 8])
@pytest.mark.parametrize("t", [math.pi, 2.9, 0.0])
def test_timestep_criterion_off_the_circle(orc, order, t):
    # On an e = 0.9 Kepler orbit the derivative norms |a^(k)| are far from
    # the geometric sequence w^k |a| of the circle, so the criterion's
    # pairing (sqrt(|a||a^(2)|) with |a^(1)|, sqrt(|a^(p-3)||a^(p-1)|) with
    # |a^(p-2)|), its plain (not squared) norms and its 1/(p-3) power are all
    # visible.  Derivatives from the f and g series, at pericentre, near it
    # and at apocentre.
    eta = 0.2
    r, v = _kepler_state(0.9, t)
    D = _kepler_derivatives(r, v, 1.0, order + 1)[2:2 + order]
    n = [float(np.linalg.norm(d)) for d in D]
    p = order

    def crit(top, bottom, power):
        return eta * (top / bottom) ** power

    want = crit(math.sqrt(n[0] * n[2]) + n[1], math.sqrt(n[p - 3] * n[p - 1]) + n[p - 2], 1.0 / (p - 3))
    got = orc.dt_criterion(order, eta, D)
    assert got == pytest.approx(want, rel=1e-12)
    # the readings this pin tells apart differ by far more than its tolerance
    squared = crit(n[0] * n[2] + n[1] ** 2, n[p - 3] * n[p - 1] + n[p - 2] ** 2, 0.5 / (p - 3))
    swapped = crit(math.sqrt(n[0] * n[1]) + n[2], math.sqrt(n[p - 3] * n[p - 2]) + n[p - 1], 1.0 / (p - 3))
    assert abs(squared / want - 1) > 1e-3 and abs(swapped / want - 1) > 1e-2


@pytest.mark.parametrize("order", [6, 8])
def test_steps_per_orbit_on_an_eccentric_orbit(orc, order):
    # Integrate two e = 0.9 orbits (no step cap: dt_max = 1) at eta and eta/2.
    # With eta used linearly the step count doubles when eta halves (a root
    # of eta, as in the order-4 form, would give sqrt(2)).  Each step is a
    # power of two within a factor 2 below the criterion, so the count per
    # orbit lies between I and 2I, I = the integral over one orbit of
    # dt / dt_crit(t) with the criterion evaluated on the exact orbit.
    T = 2 * math.pi
    ts = np.linspace(0.0, T, 12001)
    counts = {}
    for eta in (0.2, 0.1):
        inv = [1.0 / orc.dt_criterion(order, eta, _kepler_derivatives(*_kepler_state(0.9, t), 1.0,
                                                                       order + 1)[2:2 + order]) for t in ts]
        integral = float(np.trapezoid(inv, ts))
        r, v = _kepler_state(0.9, 0.0)
        m = np.array([0.5, 0.5])
        st = orc.State(m, 0.0, np.array([0.5 * r, -0.5 * r]), np.array([0.5 * v, -0.5 * v]))
        counts[eta] = orc.integrate(st, order=order, t_end=2 * T, eta=eta, dt_max=1.0) / 2
        assert integral <= counts[eta] <= 2 * integral, (eta, counts[eta], integral)
    assert counts[0.1] / counts[0.2] == pytest.approx(2.0, rel=0.05)


@pytest.mark.parametrize("eta_s", [0.01, 0.05])
def test_startup_step_circular_binary(orc, eta_s):
    # Start-up (the integrator's first pass): acc and jerk from the force at
    # t = 0, step eta_s |a| / |j|, quantised.  On a circular unsoftened binary
    # (total mass M, separation r) each body's acc rotates at the orbital rate
    # w = sqrt(M / r^3), so |j| = w |a| and the limit is eta_s / w; the step is
    # the largest power of two not above it.  A swapped ratio, a squared eta_s
    # or a missing quantisation fails this.
    M, r = 1.0, 0.3
    w = math.sqrt(M / r ** 3)
    x = np.array([[-r / 2, 0, 0], [r / 2, 0, 0]])
    v = np.array([[0, -w * r / 2, 0], [0, w * r / 2, 0]])
    st = orc.State(np.full(2, M / 2), np.zeros(2), x, v)
    assert orc.integrate(st, order=6, t_end=0.0, eta_s=eta_s) == 0  # start-up only
    for i in range(2):
        lim = orc.dt_startup(eta_s, st.d[i, 0], st.d[i, 1])
        assert lim == pytest.approx(eta_s / w, rel=1e-13)
        assert st.dt[i] == 2.0 ** math.floor(math.log2(eta_s / w))
        assert st.t[i] == 0.0


def test_timestep_quantiser_brute_force(orc):
    dt_max, dt_min = 1.0 / 16, 2.0 ** -40
    rng = np.random.default_rng(5)
    for _ in range(400):
        lim = float(np.exp(rng.uniform(math.log(1e-6), math.log(1.0))))
        t1 = float(rng.integers(0, 1 << 20)) * 2.0 ** -int(rng.integers(8, 24))
        got = orc.dt_quantise(lim, t1, dt_max, dt_min)
        best = None
        for k in range(4, 41):
            cand = 2.0 ** -k
            if cand <= lim and cand <= dt_max and math.fmod(t1, cand) == 0.0:
                best = cand
                break
        assert got == best
    with pytest.raises(orc.OracleError):
        orc.dt_quantise(1e-13, 0.0, dt_max, dt_min)


def test_next_block_brute_force(orc):
    rng = np.random.default_rng(9)
    for _ in range(50):
        n = int(rng.integers(1, 300))
        dt = 2.0 ** -rng.integers(4, 12, n).astype(float)
        t = np.array([float(rng.integers(0, 64)) * d for d in dt])
        tb, idx = orc.next_block(t, dt)
        tn = t + dt
        assert tb == tn.min()
        assert list(idx) == [i for i in range(n) if tn[i] == tb]


# --------------------------------------------------------------------------
# Integrator
# --------------------------------------------------------------------------

def _kepler_ic(e, a=1.0, m1=0.5, m2=0.5):
    M = m1 + m2
    r = a * (1 + e)
    vrel = math.sqrt(M * (1 - e) / (a * (1 + e)))
    x = np.array([[m2 / M * r, 0, 0], [-m1 / M * r, 0, 0]])
    v = np.array([[0, m2 / M * vrel, 0], [0, -m1 / M * vrel, 0]])
    return np.array([m1, m2]), x, v


def _kepler_exact(e, t, a=1.0, M=1.0):
    """Relative position at time t from apocentre (Kepler's equation)."""
    n = math.sqrt(M / a ** 3)
    mean = math.pi + n * t  # apocentre has mean anomaly pi
    E = mean
    for _ in range(100):
        E -= (E - e * math.sin(E) - mean) / (1 - e * math.cos(E))
    return np.array([a * (math.cos(E) - e), a * math.sqrt(1 - e * e) * math.sin(E), 0.0])


def _orbit_elements(x, v, M=1.0):
    r = x[0] - x[1]
    u = v[0] - v[1]
    en = 0.5 * u @ u - M / np.linalg.norm(r)
    a = -M / (2 * en)
    h = np.cross(r, u)
    evec = np.cross(u, h) / M - r / np.linalg.norm(r)
    return a, np.linalg.norm(evec)


@pytest.mark.parametrize("e", [0.0, 0.5, 0.9])
def test_kepler_orbit(orc, e):
    # Two bodies of 0.5 each, a = 1: period 2*pi.  After 8 time units the
    # relative position must match the Kepler solution, and a, e must hold.
    m, x, v = _kepler_ic(e)
    st = orc.State(m, 0.0, x, v)
    orc.integrate(st, order=6, t_end=8.0, eta=0.05, dt_max=1.0 / 16)
    assert np.all(st.t == 8.0)
    rel = st.x[0] - st.x[1]
    assert np.max(np.abs(rel - (-_kepler_exact(e, 8.0)))) < 2e-6
    a1, e1 = _orbit_elements(st.x, st.v)
    assert a1 == pytest.approx(1.0, abs=1e-7)
    assert e1 == pytest.approx(e, abs=1e-7)


def test_kepler_period(orc):
    # Return to apocentre after one period 2*pi: sample the relative distance
    # at block times and locate its maximum near 2*pi.
    m, x, v = _kepler_ic(0.5)
    st = orc.State(m, 0.0, x, v)
    best_t, best_r = 0.0, 0.0
    t = 0.0
    while t < 7.0:
        t += 1.0 / 64
        orc.integrate(st, order=6, t_end=t, eta=0.05, dt_max=1.0 / 64)
        r = np.linalg.norm(st.x[0] - st.x[1])
        if t > 4.0 and r > best_r:
            best_t, best_r = t, r
    assert abs(best_t - 2 * math.pi) < 1.0 / 64
    assert best_r == pytest.approx(1.5, abs=1e-6)


@pytest.mark.parametrize("order", [4, 6, 8])
def test_convergence_order(orc, order):
    # Global position error of an e = 0.5 Kepler orbit after 4 time units
    # (against the Kepler-equation solution) must fall as dt^p when every step
    # is halved.  Steps are fixed by dt_max with a criterion that never binds.
    m, x, v = _kepler_ic(0.5)
    T = 4.0
    exact = -_kepler_exact(0.5, T)

    def err(dm):
        st = orc.State(m, 0.0, x, v)
        orc.integrate(st, order=order, t_end=T, eta=100.0, dt_max=dm)
        return np.max(np.abs((st.x[0] - st.x[1]) - exact))

    steps = {4: (1 / 128, 1 / 256, 1 / 512), 6: (1 / 32, 1 / 64, 1 / 128), 8: (1 / 32, 1 / 64)}[order]
    errs = [err(dm) for dm in steps]
    slopes = [math.log2(errs[k] / errs[k + 1]) for k in range(len(errs) - 1)]
    assert np.mean(slopes) == pytest.approx(order, abs=0.5), (errs, slopes)


def test_pythagorean_three_body_against_dop853(orc):
    # Burrau's problem: masses 3, 4, 5 at rest on a 3-4-5 triangle, no softening.
    # Compare with scipy's DOP853 (independent integrator, Newton's law written
    # here) before the first close encounter.
    from scipy.integrate import solve_ivp
    m = np.array([3.0, 4.0, 5.0])
    x = np.array([[1.0, 3.0, 0], [-2.0, -1.0, 0], [1.0, -1.0, 0]])
    v = np.zeros((3, 3))

    def rhs(_t, y):
        p = y[:9].reshape(3, 3)
        acc = np.zeros((3, 3))
        for i in range(3):
            for j in range(3):
                if i != j:
                    r = p[j] - p[i]
                    acc[i] += m[j] * r / np.linalg.norm(r) ** 3
        return np.concatenate([y[9:], acc.ravel()])

    t_end = 1.5
    sol = solve_ivp(rhs, (0, t_end), np.concatenate([x.ravel(), v.ravel()]), method="DOP853",
                    rtol=1e-13, atol=1e-13)
    ref = sol.y[:9, -1].reshape(3, 3)
    for order, eta in ((6, 0.1), (8, 0.2)):
        st = orc.State(m, 0.0, x, v)
        orc.integrate(st, order=order, t_end=t_end, eta=eta, dt_max=1.0 / 64)
        assert np.all(st.t == t_end)
        assert np.max(np.abs(st.x - ref)) < 1e-8, order


def test_conservation_plummer_1k(orc):
    # Plummer N = 1024, order 6, eta 0.2 to t = 0.125: energy, linear and
    # angular momentum conserved at the synchronised end time.
    from paper_1312_1789_b300 import ics
    wl = ics.standard_workload(0)
    st = orc.State(wl.m, wl.eps2, wl.x, wl.v)
    E0 = sum(orc.energy(wl.m, wl.eps2, wl.x, wl.v, nthreads=8))
    P0 = (wl.m[:, None] * wl.v).sum(axis=0)
    L0 = (wl.m[:, None] * np.cross(wl.x, wl.v)).sum(axis=0)
    orc.integrate(st, order=6, t_end=0.125, nthreads=8)
    assert np.all(st.t == 0.125)
    E1 = sum(orc.energy(st.m, st.eps2, st.x, st.v, nthreads=8))
    assert abs((E1 - E0) / E0) < 1e-9
    P1 = (st.m[:, None] * st.v).sum(axis=0)
    L1 = (st.m[:, None] * np.cross(st.x, st.v)).sum(axis=0)
    pscale = (st.m[:, None] * np.abs(st.v)).sum()
    assert np.max(np.abs(P1 - P0)) < 1e-10 * pscale
    assert np.max(np.abs(L1 - L0)) < 1e-10 * pscale


# --------------------------------------------------------------------------
# Initial conditions (shared input generator, checked with the oracle energy)
# --------------------------------------------------------------------------

def test_plummer_ic_properties(orc):
    from scipy import stats

    from paper_1312_1789_b300 import ics
    n = 4096
    m, x, v = ics.plummer(n, 1234)
    ek, ep = orc.energy(m, np.zeros(n), x, v, nthreads=8)
    assert ek + ep == pytest.approx(-0.25, abs=0.03)
    assert 2 * ek / abs(ep) == pytest.approx(1.0, abs=0.08)
    r = np.linalg.norm(x, axis=1)
    p = stats.kstest(r, lambda rr: ics.plummer_enclosed_mass(rr)).pvalue
    assert p > 0.01


def test_plummer_ic_energy_tends_to_henon_units(orc):
    """The Plummer generator scales by the model's analytic energy (no pair
    sum), so the sampled E = T + W misses -1/4 by the sampling noise alone,
    O(N^-1/2): small at 65536 particles, and larger at 1024.  A wrong length
    or velocity unit would leave an offset that does not shrink with N."""
    from paper_1312_1789_b300 import ics
    dev = {}
    for n, seeds in ((1024, range(6)), (65536, range(2))):
        e, q = [], []
        for s in seeds:
            m, x, v = ics.plummer(n, 2000 + s)
            ek, ep = orc.energy(m, np.zeros(n), x, v, nthreads=8)
            e.append(ek + ep + 0.25)
            q.append(2 * ek / abs(ep) - 1.0)
        dev[n] = (np.sqrt(np.mean(np.square(e))), np.sqrt(np.mean(np.square(q))))
    assert dev[65536][0] < 0.004 and dev[65536][1] < 0.012
    assert dev[65536][0] < dev[1024][0] and dev[65536][1] < dev[1024][1]


def test_hernquist_ic_properties(orc):
    from scipy import stats

    from paper_1312_1789_b300 import ics
    n = 4096
    m, x, v = ics.hernquist(n, 4321)
    ek, ep = orc.energy(m, np.zeros(n), x, v, nthreads=8)
    assert ek + ep == pytest.approx(-0.25, abs=0.04)
    assert 2 * ek / abs(ep) == pytest.approx(1.0, abs=0.1)
    r = np.linalg.norm(x, axis=1)
    cdf = lambda rr: np.minimum(ics.hernquist_enclosed_mass(rr) / ics.HERNQUIST_MASS_CUT, 1.0)  # noqa: E731
    p = stats.kstest(r, cdf).pvalue
    assert p > 0.01


# --------------------------------------------------------------------------
# Noise floor of interpolated derivatives (reduced-precision reading)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("order", [4, 6, 8])
def test_noise_floor_brackets_the_true_derivatives(orc, order):
    # acc(t) an exact polynomial of degree 2mm-1, so the interpolant recovers
    # its derivatives exactly; perturb every input by relative rounding up to
    # eps.  The perturbed derivatives must stay within their floors of the true
    # ones, and the floored norms must never exceed the true norms.
    mm = order // 2
    eps = np.array([3e-7, 1e-6, 2e-6, 2e-5])
    rng = np.random.default_rng(300 + order)
    for trial in range(50):
        coef = rng.normal(size=(3, 2 * mm))
        h = float(2.0 ** -rng.integers(2, 12))
        D0 = np.array([[P.polyval(0.0, P.polyder(coef[c], k)) for c in range(3)] for k in range(mm)])
        D1 = np.array([[P.polyval(h, P.polyder(coef[c], k)) for c in range(3)] for k in range(mm)])
        true = np.array([[P.polyval(h, P.polyder(coef[c], k)) for c in range(3)] for k in range(mm, 2 * mm)])

        def jitter(D):
            out = D.copy()
            for r in range(mm):
                u = rng.normal(size=3)
                out[r] += eps[r] * np.linalg.norm(D[r]) * rng.uniform(0, 1) * u / np.linalg.norm(u)
            return out

        P0, P1 = jitter(D0), jitter(D1)
        got = orc.interp(mm, h, P0, P1)
        N = orc.noise_floor(mm, h, P0, P1, eps)
        for q in range(mm):
            # rounding of the floor itself: relative 1e-12 of the terms
            slack = 1e-9 * N[q] + 1e-12 * np.linalg.norm(true[q])
            assert np.linalg.norm(got[q] - true[q]) <= N[q] * (1 + 2 * max(eps)) + slack
            assert max(np.linalg.norm(got[q]) - N[q], 0.0) <= np.linalg.norm(true[q]) + slack


@pytest.mark.parametrize("order", [4, 6, 8])
def test_zero_noise_floor_is_the_plain_criterion(orc, order):
    rng = np.random.default_rng(order)
    mm = order // 2
    D0 = rng.normal(size=(mm, 3))
    Dfull = rng.normal(size=(2 * mm, 3))
    assert orc.dt_criterion_floored(order, 0.2, 0.01, D0, Dfull, [0, 0, 0, 0]) == orc.dt_criterion(order, 0.2, Dfull)
    # a floor that swamps every interpolated derivative leaves no constraint
    assert orc.dt_criterion_floored(order, 0.2, 1e-6, D0, Dfull, [1e-3] * 4) == math.inf


def test_noisy_forces_do_not_collapse_the_step(orc):
    # A circular orbit whose forces carry 1e-6 relative rounding, started with
    # a step far below the resolvable one: with the floor the step grows to the
    # eta-limited value instead of collapsing.
    w = 1.0
    eta = 0.2
    rng = np.random.default_rng(1)

    def derivs(t, k0, k1):
        return np.array([[math.cos(w * t + k * math.pi / 2), math.sin(w * t + k * math.pi / 2), 0.0]
                         for k in range(k0, k1)]) * (-(w ** np.arange(k0, k1)))[:, None]

    for floored in (False, True):
        eps = [1e-6, 1e-6, 1e-6, 1e-6] if floored else [0, 0, 0, 0]
        h, t = 2.0 ** -12, 0.0
        for _ in range(60):
            D0 = derivs(t, 0, 3) * (1 + 1e-6 * rng.normal(size=(3, 1)))
            D1 = derivs(t + h, 0, 3) * (1 + 1e-6 * rng.normal(size=(3, 1)))
            hi = orc.interp(3, h, D0, D1)
            crit = orc.dt_criterion_floored(6, eta, h, D0, np.vstack([D1, hi]), eps)
            t += h
            try:
                h = orc.dt_quantise(min(crit, 2 * h), t, 1.0, 2.0 ** -40)
            except orc.OracleError:
                h = 0.0
                break
        if floored:
            assert h == 0.125  # the largest power of two <= eta / w = 0.2
        else:
            assert h < 2.0 ** -12  # the plain criterion shrinks the step on noise
