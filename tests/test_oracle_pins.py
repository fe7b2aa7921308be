"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an identity the paper proves (EC condition, discrete SCL, free-stream
preservation, entropy identity), a finite-difference derivative, a
high-precision reference, or an exact solution.  A plausible slip (dropped
term, wrong sign, transposed operand) in the oracle fails at least one of them.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2107_12027_gb300 import workloads as wl

GAMMAS = (5.0 / 3.0, 4.0 / 3.0, 1.4)


# ---------------------------------------------------------------- coefficients
def _alpha_exact(p):
    """Solve the constraints of eq. HOCoeff exactly (Gaussian elimination over
    the rationals): sum n a_n = 1, sum n^(2s-1) a_n = 0 for s = 2..p."""
    A = [[Fraction(n ** (2 * s - 1)) for n in range(1, p + 1)] for s in range(1, p + 1)]
    b = [Fraction(1)] + [Fraction(0)] * (p - 1)
    for col in range(p):
        piv = next(r for r in range(col, p) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        b[col], b[piv] = b[piv], b[col]
        for r in range(p):
            if r != col and A[r][col] != 0:
                f = A[r][col] / A[col][col]
                A[r] = [a - f * c for a, c in zip(A[r], A[col])]
                b[r] -= f * b[col]
    return [b[r] / A[r][r] for r in range(p)]


@pytest.mark.parametrize("p", [1, 2, 3])
def test_alpha_solves_constraints(p):
    exact = _alpha_exact(p)
    np.testing.assert_allclose(oracle.alpha(p), [float(a) for a in exact], rtol=0, atol=1e-16)


def test_delta_p2_is_textbook_fourth_order_difference():
    # delta[a] = 1/2 sum alpha_n (a_{+n} - a_{-n}); for p = 2 the textbook
    # fourth-order central difference has weights 2/3 and -1/12.
    a = oracle.alpha(2)
    np.testing.assert_allclose(a / 2, [2.0 / 3.0, -1.0 / 12.0], rtol=1e-15)


# ------------------------------------------------------------------- log mean
def test_logmean_against_high_precision():
    # Error model of [[a]]/[[ln a]] with rounded logarithms: a few ulp times
    # (1 + (|ln a| + |ln b|)/|ln(b/a)|) on the direct branch, a few ulp on the
    # series branch (truncation below 1e-17 there).
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    r = wl.rng(11)
    ulp = 2.0 ** -52
    worst = 0.0
    for _ in range(600):
        a = float(np.exp(r.uniform(-5, 5)))
        gap = float(10.0 ** r.uniform(-15, 0.5))
        b = a * (1.0 + gap) if r.uniform() < 0.5 else a / (1.0 + gap)
        ref = (mp.mpf(b) - mp.mpf(a)) / (mp.log(mp.mpf(b)) - mp.log(mp.mpf(a)))
        got = oracle.logmean(a, b)
        err = abs(float((mp.mpf(got) - ref) / ref))
        cond = 1.0 + (abs(np.log(a)) + abs(np.log(b))) / max(abs(float(mp.log(mp.mpf(b) / mp.mpf(a)))), 2e-2)
        worst = max(worst, err / (ulp * cond))
    assert worst < 4.0, worst
    assert oracle.logmean(2.5, 2.5) == 2.5


# ----------------------------------------------------------- states and fluxes
def _states(n, seed, vmax=0.9):
    return wl.random_states(wl.rng(seed), n, rho=(1e-4, 10.0), p=(5e-4, 10.0), vmax=vmax)


@pytest.mark.parametrize("gamma", GAMMAS)
def test_cons2prim_round_trip(gamma):
    # The recovered pressure is conditioned by E/p (cold flows subtract large
    # nearly equal energies) and by W^2; the round trip must reach that bound.
    ulp = 2.0 ** -52
    worst = 0.0
    for w in list(_states(300, 1)) + list(_states(100, 2, vmax=0.995)):
        U = oracle.prim2cons(gamma, w)
        w2, st, it = oracle.cons2prim(gamma, U)
        assert st == 0 and it < 60
        W2 = 1.0 / (1.0 - w[1] ** 2 - w[2] ** 2)
        err = max(abs(w2[0] / w[0] - 1), abs(w2[3] / w[3] - 1), abs(w2[1] - w[1]), abs(w2[2] - w[2]))
        worst = max(worst, err / (ulp * (1.0 + U[3] / w[3]) * W2))
    assert worst < 16.0, worst


def test_cons2prim_rejects_non_admissible():
    g = 5.0 / 3.0
    assert oracle.cons2prim(g, [1.0, 2.0, 0.0, 1.5])[1] == -1     # |m| > E
    assert oracle.cons2prim(g, [-1.0, 0.0, 0.0, 1.0])[1] == -1    # D < 0


def test_flux_matches_paper_definition_at_rest():
    # At v = 0 the flux of eq. RMHDdiv2 is (0, p e_k, 0).
    F = oracle.flux(5.0 / 3.0, [2.0, 0.0, 0.0, 0.7], 1)
    np.testing.assert_allclose(F, [0.0, 0.0, 0.7, 0.0], atol=1e-15)


def _jac(f, w, h=1e-6):
    w = np.asarray(w, float)
    cols = []
    for a in range(4):
        e = np.zeros(4)
        e[a] = h * max(1.0, abs(w[a]))
        cols.append((np.asarray(f(w + e)) - np.asarray(f(w - e))) / (2 * e[a]))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("gamma", GAMMAS)
def test_entropy_variables_are_gradient_of_entropy(gamma):
    # V = eta'(U)^T (Def. 2.1): compare with central differences of eta(U(w)).
    for w in _states(20, 3, vmax=0.8):
        w = np.array([max(w[0], 0.05), w[1], w[2], max(w[3], 0.05)])
        dUdw = _jac(lambda q: oracle.prim2cons(gamma, q), w)
        detadw = _jac(lambda q: np.array([oracle.entropy(gamma, q)] * 4), w)[0]
        V_fd = np.linalg.solve(dUdw.T, detadw)
        V = oracle.entropy_vars(gamma, w)
        np.testing.assert_allclose(V, V_fd, rtol=2e-6, atol=2e-6 * np.abs(V).max())


@pytest.mark.parametrize("gamma", GAMMAS)
def test_potentials_identities(gamma):
    # eq. EntropyPotential: phi = V.U - eta, psi_k = V.F_k - q_k, q_k = eta v_k.
    for w in _states(50, 4):
        V = oracle.entropy_vars(gamma, w)
        U = oracle.prim2cons(gamma, w)
        eta = oracle.entropy(gamma, w)
        phi, psi = oracle.potentials(w)
        scale = np.abs(V * U).sum() + abs(eta)
        assert abs(V @ U - eta - phi) <= 1e-13 * scale
        for k in range(2):
            F = oracle.flux(gamma, w, k)
            sk = np.abs(V * F).sum() + abs(eta * w[1 + k])
            assert abs(V @ F - eta * w[1 + k] - psi[k]) <= 1e-13 * sk


def _pairs(n, seed):
    r = wl.rng(seed)
    A = wl.random_states(r, n)
    B = wl.random_states(r, n)
    # a third of the pairs nearly equal (exercise the log-mean series)
    k = n // 3
    B[:k] = A[:k] * (1.0 + r.uniform(-1e-9, 1e-9, (k, 4)))
    B[:k, 1:3] = np.clip(B[:k, 1:3], -0.6, 0.6)
    return A, B


@pytest.mark.parametrize("gamma", GAMMAS)
def test_two_point_flux_entropy_conservation_condition(gamma):
    # Sec. 3.1: [[V]].U~ = [[phi]], [[V]].F~_j = [[psi_j]] (B = 0).
    A, B = _pairs(600, 5)
    worst = 0.0
    for wl_, wr_ in zip(A, B):
        Ut, F1, F2 = oracle.ec_flux(gamma, wl_, wr_)
        dV = oracle.entropy_vars(gamma, wr_) - oracle.entropy_vars(gamma, wl_)
        phl, psl = oracle.potentials(wl_)
        phr, psr = oracle.potentials(wr_)
        for flux, target in ((Ut, phr - phl), (F1, psr[0] - psl[0]), (F2, psr[1] - psl[1])):
            Vl, Vr = oracle.entropy_vars(gamma, wl_), oracle.entropy_vars(gamma, wr_)
            scale = (np.abs(Vl) + np.abs(Vr)) @ np.abs(flux) + abs(phl) + abs(phr) + np.abs(psl).sum() + np.abs(psr).sum()
            worst = max(worst, abs(dV @ flux - target) / scale)
    assert worst < 2e-14, worst


@pytest.mark.parametrize("gamma", GAMMAS)
def test_two_point_flux_consistency_and_symmetry(gamma):
    # Lemma 3.1 hypotheses: F~(U, U) = F(U) and F~(l, r) = F~(r, l).
    A, B = _pairs(200, 6)
    for w, v in zip(A, B):
        Ut, F1, F2 = oracle.ec_flux(gamma, w, w)
        np.testing.assert_allclose(Ut, oracle.prim2cons(gamma, w), rtol=1e-13, atol=1e-300)
        np.testing.assert_allclose(F1, oracle.flux(gamma, w, 0), rtol=1e-13, atol=1e-14 * np.abs(F1).max())
        np.testing.assert_allclose(F2, oracle.flux(gamma, w, 1), rtol=1e-13, atol=1e-14 * np.abs(F2).max())
        a = oracle.ec_flux(gamma, w, v)
        b = oracle.ec_flux(gamma, v, w)
        for x, y in zip(a, b):
            np.testing.assert_allclose(x, y, rtol=1e-14, atol=1e-15 * np.abs(x).max())


# -------------------------------------------------------------- eigen-system
@pytest.mark.parametrize("gamma", GAMMAS)
def test_scaled_eigenvectors(gamma):
    # Sec. 4: dU/dV = R R^T and dF_1/dU = R Lambda R^{-1}; the Jacobians come
    # from central differences of the flux and state definitions.
    for w in _states(40, 7, vmax=0.85):
        w = np.array([max(w[0], 0.05), w[1], w[2], max(w[3], 0.05)])
        lam, R = oracle.eigen(gamma, w)
        dUdw = _jac(lambda q: oracle.prim2cons(gamma, q), w)
        dFdw = _jac(lambda q: oracle.flux(gamma, q, 0), w)
        dVdw = _jac(lambda q: oracle.entropy_vars(gamma, q), w)
        A = dFdw @ np.linalg.inv(dUdw)
        A0 = dUdw @ np.linalg.inv(dVdw)
        sA = np.abs(A).max() * np.abs(R).max()
        assert np.abs(A @ R - R * lam).max() < 1e-6 * sA
        assert np.abs(R @ R.T - A0).max() < 1e-6 * np.abs(A0).max()
        ev = np.sort(np.linalg.eigvals(A).real)
        np.testing.assert_allclose(np.sort(lam), ev, atol=1e-7)


def test_eigenvalues_reduce_to_sound_speed_at_rest():
    # at rest the acoustic speeds are -c, +c with c^2 = Gamma p/(rho h)
    g, rho, p = 5.0 / 3.0, 1.3, 0.4
    lam, _ = oracle.eigen(g, [rho, 0.0, 0.0, p])
    h = 1 + g * p / ((g - 1) * rho)
    c = np.sqrt(g * p / (rho * h))
    np.testing.assert_allclose(lam, [-c, 0.0, 0.0, c], atol=1e-15)


# ---------------------------------------------------------------------- WENO
@pytest.mark.parametrize("w", [3, 5])
def test_weno_exact_on_linear_data(w):
    # a linear function's edge value is reproduced exactly by every sub-stencil
    s = 0.7 + 0.3 * np.arange(w)
    mid = (w - 1) // 2
    assert abs(oracle.weno(w, 1e-6, s) - (0.7 + 0.3 * (mid + 0.5))) < 1e-14


def test_weno5_order_on_smooth_data():
    # On smooth data the left and right WENO5 values at one interface differ
    # by O(h^5) away from critical points (the dissipation's accuracy).
    errs = []
    for h in (0.1, 0.05, 0.025):
        x = 0.3 + h * np.arange(-2, 4)
        f = np.sin(x)
        left = oracle.weno(5, 1e-30, f[0:5])
        right = oracle.weno(5, 1e-30, f[5:0:-1])
        errs.append(abs(right - left))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > 4.5, rates


def test_weno5_non_oscillatory_at_a_step():
    s = np.array([0.0, 0.0, 0.0, 1.0, 1.0])
    assert abs(oracle.weno(5, 1e-6, s)) < 1e-6


# ------------------------------------------------------------------- metrics
def _dlt(a, axis, p):
    al = oracle.alpha(p)
    return sum(0.5 * al[n - 1] * (np.roll(a, -n, axis) - np.roll(a, n, axis)) for n in range(1, p + 1))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_discrete_scl_on_random_mesh(p):
    # eq. DiscSCL_O2p: sum_k delta_k[J xi_k,x_j] = 0 for any mesh (periodic).
    n = 20
    x = wl.random_mesh(n, n, wl.rng(8), amp=0.3)
    cfg = oracle.make_cfg(n, n, p=p)
    m, _ = oracle.metrics(cfg, x)
    for j in range(2):
        div = _dlt(m[0 + j], 1, p) + _dlt(m[2 + j], 0, p)
        assert np.abs(div).max() < 1e-15 * 50, np.abs(div).max()


def test_metrics_exact_on_affine_mesh():
    # x = A xi + b: J xi_x = A11, J xi_y = -A01, J eta_x = -A10, J eta_y = A00
    # (index-space xi), J = det A, also across the outflow ghost extrapolation.
    n = 12
    A = np.array([[0.09, 0.02], [-0.01, 0.07]])
    I, Jm = np.meshgrid(np.arange(n), np.arange(n))
    x = np.stack([A[0, 0] * I + A[0, 1] * Jm + 0.3, A[1, 0] * I + A[1, 1] * Jm - 0.2])
    for p in (1, 2, 3):
        cfg = oracle.make_cfg(n, n, bc=(oracle.OUTFLOW, oracle.OUTFLOW), p=p)
        m, J0 = oracle.metrics(cfg, x)
        np.testing.assert_allclose(m[0], A[1, 1], rtol=1e-12)
        np.testing.assert_allclose(m[1], -A[0, 1], rtol=1e-12)
        np.testing.assert_allclose(m[2], -A[1, 0], rtol=1e-12)
        np.testing.assert_allclose(m[3], A[0, 0], rtol=1e-12)
        np.testing.assert_allclose(J0, np.linalg.det(A), rtol=1e-12)
