"""Pins of the RMHD part of the FP64 oracle against what the paper and the
mathematics fix.

Each test checks the oracle against something other than itself: the
covariant definition of the equations (eq. RMHD: rest-mass current, the
energy-momentum tensor and the dual field tensor), identities that define the
entropy variables and potentials (Sec. 2), the EC conditions of Sec. 3.1,
finite-difference Jacobians (eigen-system), textbook wave speeds in special
configurations, and the scheme-level identities (entropy conservation,
free-stream preservation, the reduction to RHD).
"""
import numpy as np
import pytest

import oracle
from paper_2107_12027_gb300 import workloads as wl

GAMMAS = (4.0 / 3.0, 5.0 / 3.0)
G53 = 5.0 / 3.0
EPS = np.finfo(float).eps


def _states(n, seed, **kw):
    return wl.random_states_mhd(wl.rng(seed), n, **kw)


def _four_vectors(w):
    """u^alpha, b^alpha of eq. RMHD (the paper's definitions below it)."""
    v, B = w[1:4], w[5:8]
    W = 1.0 / np.sqrt(1.0 - v @ v)
    u = W * np.concatenate([[1.0], v])
    b = W * np.concatenate([[v @ B], B / W ** 2 + v * (v @ B)])
    return u, b


def _covariant_flux(gamma, w, alpha):
    """Row alpha of (rho u, T, Psi): the conserved densities for alpha = 0 and
    the fluxes along x_alpha otherwise, with T = T_f + T_m and
    Psi^{ab} = u^a b^b - u^b b^a, metric diag(-1, 1, 1, 1)."""
    rho, p = w[0], w[4]
    u, b = _four_vectors(w)
    g = np.diag([-1.0, 1.0, 1.0, 1.0])
    bb = -b[0] ** 2 + b[1:] @ b[1:]
    h = 1.0 + gamma / (gamma - 1.0) * p / rho
    T = rho * h * np.outer(u, u) + p * g + bb * (np.outer(u, u) + g / 2) - np.outer(b, b)
    Psi = np.outer(u, b) - np.outer(b, u)
    # conserved order (D, m_1..3, E, B_1..3): momentum T^{a k}, energy T^{a 0}
    return np.concatenate([[rho * u[alpha]], T[alpha, 1:], [T[alpha, 0]], Psi[alpha, 1:]])


# ------------------------------------------------------------ state and flux
@pytest.mark.parametrize("gamma", GAMMAS)
def test_cons_and_flux_match_covariant_definition(gamma):
    for w in _states(200, 1):
        U = oracle.mhd_prim2cons(gamma, w)
        ref = _covariant_flux(gamma, w, 0)
        np.testing.assert_allclose(U, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
        for d in range(3):
            F = oracle.mhd_flux(gamma, w, d)
            ref = _covariant_flux(gamma, w, d + 1)
            np.testing.assert_allclose(F, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("gamma", GAMMAS)
def test_cons2prim_round_trip(gamma):
    # Error model: the recovery resolves Z = rho h W^2 to ~eps (E + Z), so the
    # primitives carry ~eps (1 + E/p) W^2 relative error (cold, fast gas).
    worst = 0.0
    S = _states(3000, 2, rho=(1e-4, 10.0), p=(5e-4, 10.0), vmax=0.995, bmax=1.0)
    for w in S:
        U = oracle.mhd_prim2cons(gamma, w)
        w2, st, it = oracle.mhd_cons2prim(gamma, U)
        assert st == 0 and it < 100
        W2 = 1.0 / (1.0 - w[1:4] @ w[1:4])
        err = max(np.max(np.abs(w2[[0, 4]] - w[[0, 4]]) / w[[0, 4]]), np.max(np.abs(w2[1:4] - w[1:4])))
        assert np.array_equal(w2[5:], w[5:])
        worst = max(worst, err / (EPS * (1.0 + U[4] / w[4]) * W2))
    assert worst < 16.0, worst


def test_cons2prim_rejects_non_admissible():
    U = oracle.mhd_prim2cons(4.0 / 3.0, np.array([1.0, 0.1, 0.2, 0.0, 1.0, 0.3, 0.1, 0.0]))
    bad = U.copy()
    bad[0] = -1.0
    assert oracle.mhd_cons2prim(4.0 / 3.0, bad)[1] == -1
    bad = U.copy()
    bad[4] = -1.0
    assert oracle.mhd_cons2prim(4.0 / 3.0, bad)[1] == -1


# --------------------------------------------------------- entropy quantities
def _jac(f, w, rel=1e-3):
    """Jacobian of f at w by Richardson-extrapolated central differences
    (truncation O(h^4)), steps scaled by the component magnitude."""
    cols = []
    for a in range(len(w)):
        e = np.zeros(len(w))
        e[a] = 1.0
        h = rel * max(abs(w[a]), 0.05)
        D = lambda hh: (f(w + hh * e) - f(w - hh * e)) / (2 * hh)
        cols.append((4 * D(h / 2) - D(h)) / 3)
    return np.array(cols).T


@pytest.mark.parametrize("gamma", GAMMAS)
def test_entropy_variables_are_gradient_of_entropy(gamma):
    # V^T = d eta/dU = (d eta/dw) (dU/dw)^{-1}
    for w in _states(40, 3, vmax=0.8):
        deta = _jac(lambda q: np.array([oracle.mhd_entropy(gamma, q)]), w)[0]
        JU = _jac(lambda q: oracle.mhd_prim2cons(gamma, q), w)
        V = np.linalg.solve(JU.T, deta)
        Vo = oracle.mhd_entropy_vars(gamma, w)
        np.testing.assert_allclose(Vo, V, rtol=1e-7, atol=1e-7 * np.abs(Vo).max())


@pytest.mark.parametrize("gamma", GAMMAS)
def test_potentials_identities(gamma):
    # eq. EntropyPotential: phi = V.U - eta, psi_k = V.F_k + Phi B_k - q_k,
    # q_k = eta v_k; eq. Phi: Phi = Phi'(V).V (degree-one homogeneity)
    for w in _states(300, 4):
        V = oracle.mhd_entropy_vars(gamma, w)
        U = oracle.mhd_prim2cons(gamma, w)
        eta = oracle.mhd_entropy(gamma, w)
        phi, psi, Phi = oracle.mhd_potentials(w)
        sc = abs(V) @ abs(U) + abs(eta)
        assert abs(phi - (V @ U - eta)) <= 1e-13 * sc
        for k in range(3):
            F = oracle.mhd_flux(gamma, w, k)
            ref = V @ F + Phi * w[5 + k] - eta * w[1 + k]
            assert abs(psi[k] - ref) <= 1e-13 * (abs(V) @ abs(F) + abs(Phi * w[5 + k]) + abs(eta))
        P = oracle.mhd_phiprime(w)
        assert abs(P @ V - Phi) <= 1e-13 * (abs(P) @ abs(V))


@pytest.mark.parametrize("gamma", GAMMAS)
def test_phiprime_is_gradient_of_phi(gamma):
    # Phi'(V) = dPhi/dV = (dPhi/dw) (dV/dw)^{-1}
    for w in _states(30, 5, vmax=0.8):
        dPhi = _jac(lambda q: np.array([oracle.mhd_potentials(q)[2]]), w)[0]
        JV = _jac(lambda q: oracle.mhd_entropy_vars(gamma, q), w)
        ref = np.linalg.solve(JV.T, dPhi)
        np.testing.assert_allclose(oracle.mhd_phiprime(w), ref, rtol=1e-7, atol=1e-7 * np.abs(ref).max())


# ------------------------------------------------------------ two-point flux
@pytest.mark.parametrize("gamma", GAMMAS)
def test_two_point_flux_entropy_conservation_conditions(gamma):
    # Sec. 3.1: [[V]].U~ = [[phi]], [[V]].F~_j = [[psi_j]] - {{B_j}} [[Phi]]
    S = _states(1200, 6)
    worst = 0.0
    for wl_, wr_ in zip(S[0::2], S[1::2]):
        Ut, Ft = oracle.mhd_ec_flux(gamma, wl_, wr_)
        dV = oracle.mhd_entropy_vars(gamma, wr_) - oracle.mhd_entropy_vars(gamma, wl_)
        pl, sl, Pl = oracle.mhd_potentials(wl_)
        pr, sr, Pr = oracle.mhd_potentials(wr_)
        res = dV @ Ut - (pr - pl)
        worst = max(worst, abs(res) / (abs(dV) @ abs(Ut) + abs(pl) + abs(pr)))
        for j in range(3):
            rhs = sr[j] - sl[j] - 0.5 * (wl_[5 + j] + wr_[5 + j]) * (Pr - Pl)
            res = dV @ Ft[j] - rhs
            worst = max(worst, abs(res) / (abs(dV) @ abs(Ft[j]) + abs(sl[j]) + abs(sr[j])
                                           + abs(wl_[5 + j] * Pl) + abs(wr_[5 + j] * Pr)))
    assert worst < 1e-13, worst


@pytest.mark.parametrize("gamma", GAMMAS)
def test_two_point_flux_consistency_and_symmetry(gamma):
    for w in _states(100, 7):
        Ut, Ft = oracle.mhd_ec_flux(gamma, w, w)
        U = oracle.mhd_prim2cons(gamma, w)
        np.testing.assert_allclose(Ut, U, rtol=1e-12, atol=1e-13 * np.abs(U).max())
        for j in range(3):
            F = oracle.mhd_flux(gamma, w, j)
            np.testing.assert_allclose(Ft[j], F, rtol=1e-11, atol=1e-12 * np.abs(F).max())
    S = _states(100, 8)
    for a, b in zip(S[0::2], S[1::2]):
        U1, F1 = oracle.mhd_ec_flux(gamma, a, b)
        U2, F2 = oracle.mhd_ec_flux(gamma, b, a)
        np.testing.assert_array_equal(U1, U2)
        np.testing.assert_array_equal(F1, F2)


def test_two_point_flux_reduces_to_rhd():
    # Remark after eq. ECConditionCurv: B = 0 gives the RHD case
    gamma = 5.0 / 3.0
    S = wl.random_states(wl.rng(9), 100)
    for a, b in zip(S[0::2], S[1::2]):
        Ut4, F14, F24 = oracle.ec_flux(gamma, a, b)
        ext = lambda s: np.array([s[0], s[1], s[2], 0.0, s[3], 0.0, 0.0, 0.0])
        Ut, Ft = oracle.mhd_ec_flux(gamma, ext(a), ext(b))
        pick = [0, 1, 2, 4]
        for got, ref in ((Ut, Ut4), (Ft[0], F14), (Ft[1], F24)):
            np.testing.assert_allclose(got[pick], ref, rtol=1e-13, atol=1e-14 * np.abs(ref).max())
            assert np.all(got[[3, 5, 6, 7]] == 0.0)


def test_printed_R1_misses_the_ec_condition_by_a_cubic_term():
    """The reading of R_1 in U~^RMHD: as printed (1/2 {{W}}{{(b^k)^2}}, summed
    to 3) the EC condition fails by exactly -(1/8)[[beta]][[W]][[|b|^2]]; the
    oracle's 1/2 {{W (b^k)^2}} closes it.  The two differ exactly by that
    term in the U~_E and U~_m components."""
    gamma = 4.0 / 3.0
    S = _states(200, 10)
    for wl_, wr_ in zip(S[0::2], S[1::2]):
        Ut, _ = oracle.mhd_ec_flux(gamma, wl_, wr_)
        ul, bl = _four_vectors(wl_)
        ur, br = _four_vectors(wr_)
        Wl, Wr = ul[0], ur[0]
        betal, betar = wl_[0] / wl_[4], wr_[0] / wr_[4]
        b2l, b2r = bl[1:] @ bl[1:], br[1:] @ br[1:]
        # printed minus read R_1: 1/2 sum_k ({{W}}{{b_k^2}} - {{W b_k^2}}) = -1/8 [[W]][[|b|^2]]
        dR1 = -0.125 * (Wr - Wl) * (b2r - b2l)
        # propagate: U~_E = (sum u R - beta_m R1)/D_  ->  dU_E = -beta_m dR1 / D_
        W_m = 0.5 * (Wl + Wr)
        u_m = 0.5 * (ul[1:] + ur[1:])
        beta_m = 0.5 * (betal + betar)
        Dcal = beta_m * (W_m ** 2 - u_m @ u_m) / W_m
        dUE = -beta_m * dR1 / Dcal
        printed = Ut.copy()
        printed[4] += dUE
        printed[1:4] += u_m * dUE / W_m
        dV = oracle.mhd_entropy_vars(gamma, wr_) - oracle.mhd_entropy_vars(gamma, wl_)
        pl, pr = oracle.mhd_potentials(wl_)[0], oracle.mhd_potentials(wr_)[0]
        res_read = dV @ Ut - (pr - pl)
        res_printed = dV @ printed - (pr - pl)
        cubic = -0.125 * (betar - betal) * (Wr - Wl) * (b2r - b2l)
        sc = abs(dV) @ abs(Ut) + abs(pl) + abs(pr)
        assert abs(res_read) < 1e-13 * sc
        assert abs(res_printed - cubic) < 1e-12 * sc


# -------------------------------------------------------------- eigen-system
def _check_eigen(gamma, w, sep_only=True):
    lam, R = oracle.mhd_eigen(gamma, w)
    JU = _jac(lambda q: oracle.mhd_prim2cons(gamma, q), w)
    JV = _jac(lambda q: oracle.mhd_entropy_vars(gamma, q), w)
    JF = _jac(lambda q: oracle.mhd_flux(gamma, q, 0), w)
    A0 = JU @ np.linalg.inv(JV)
    # symmetrized x_1 Jacobian: dF/dU plus the Godunov-Powell column Phi' dB_1
    A = JF @ np.linalg.inv(JU) + np.outer(oracle.mhd_phiprime(w), np.eye(8)[5])
    np.testing.assert_allclose(R @ R.T, A0, rtol=0, atol=1e-8 * np.abs(A0).max())
    np.testing.assert_allclose(A @ R, R * lam, rtol=0, atol=1e-8 * np.abs(R).max())
    return lam


@pytest.mark.parametrize("gamma", GAMMAS)
def test_scaled_eigenvectors(gamma):
    # dU/dV = R R^T and dF~/dU R = R Lambda (Sec. 4) for states whose speeds
    # are separated (clusters get a canonical, non-eigen basis by design)
    n = 0
    for w in _states(60, 12, vmax=0.9, bmax=1.5):
        lam, _ = oracle.mhd_eigen(gamma, w)
        if np.min(np.diff(np.sort(lam[2:]))) < 1e-4:
            continue
        _check_eigen(gamma, w)
        n += 1
    assert n > 40


def test_eigen_exactly_degenerate_states():
    # B_t = 0 (Alfven meets a magnetosonic wave) and B_n = 0 (slow and Alfven
    # meet the entropy speed): the canonical basis spans exact eigenspaces
    gamma = 4.0 / 3.0
    for w in ([1.0, 0.3, 0.1, 0.0, 0.5, 1.0, 0.0, 0.0], [1.0, 0.3, 0.1, 0.0, 0.5, 0.0, 1.0, 0.0],
              [10.0, 0.0, 0.5, 0.0, 1.0, 1.0, 0.0, 0.0], [0.7, -0.2, 0.4, 0.1, 0.9, 0.0, 0.0, 0.0]):
        _check_eigen(gamma, np.array(w))


def test_eigen_speeds_textbook_special_cases():
    gamma = 4.0 / 3.0
    for rho, p, b in [(1.0, 0.5, 0.8), (0.3, 2.0, 1.5)]:
        rh = rho + gamma / (gamma - 1.0) * p
        cs2 = gamma * p / rh
        # at rest with B along the normal: sound +-c_s, Alfven +-b/sqrt(rho h + b^2) (twice)
        lam, _ = oracle.mhd_eigen(gamma, np.array([rho, 0, 0, 0, p, b, 0, 0]))
        va = b / np.sqrt(rh + b * b)
        ref = np.sort([-np.sqrt(cs2), -va, -va, 0, 0, va, va, np.sqrt(cs2)])
        np.testing.assert_allclose(np.sort(lam), ref, atol=1e-14)
        # at rest with B normal to the normal: fast^2 = v_A^2 + c_s^2 (1 - v_A^2), others 0
        lam, _ = oracle.mhd_eigen(gamma, np.array([rho, 0, 0, 0, p, 0, b, 0]))
        va2 = b * b / (rh + b * b)
        cf = np.sqrt(va2 + cs2 * (1 - va2))
        np.testing.assert_allclose(np.sort(lam), [-cf, 0, 0, 0, 0, 0, 0, cf], atol=1e-14)
    # B = 0 and v_3 = 0: the RHD speeds
    w = np.array([0.7, 0.3, -0.4, 0.0, 0.9, 0, 0, 0])
    lam, _ = oracle.mhd_eigen(5.0 / 3.0, w)
    l4, _ = oracle.eigen(5.0 / 3.0, w[[0, 1, 2, 4]])
    np.testing.assert_allclose(np.sort(lam), np.sort(np.concatenate([l4, [0.3] * 4])), atol=1e-14)


def test_divergence_wave_is_analytic_eigenvector():
    # column 1 is the divergence wave dB = e_1 - v_1 v (other primitives fixed),
    # speed v_1, for the symmetrized system
    gamma = 4.0 / 3.0
    for w in _states(10, 13, vmax=0.8):
        lam, R = oracle.mhd_eigen(gamma, w)
        a = np.zeros(8)
        a[5:] = np.eye(3)[0] - w[1] * w[1:4]
        JU = _jac(lambda q: oracle.mhd_prim2cons(gamma, q), w)
        r = JU @ a
        np.testing.assert_allclose(R[:, 1] / np.linalg.norm(R[:, 1]), r / np.linalg.norm(r), atol=1e-8)
        assert lam[0] == w[1] and lam[1] == w[1]


# ------------------------------------------------------------ scheme level
def _smooth(n, seed, p, w, gamma=4.0 / 3.0):
    cfg = oracle.make_cfg(n, n, gamma=gamma, p=p, w=w, phys=oracle.RMHD)
    x = wl.wavy_mesh(n, n, amp=0.05)
    prim = wl.smooth_random_state_mhd(x, wl.rng(seed))
    cons, J = oracle.init_state(cfg, prim, x)
    return cfg, cons, J, x, wl.wavy_mesh_velocity(n, n)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_ec_entropy_identity_with_powell_source(p):
    # Thm. 3.1: the EC scheme (with the Powell source) conserves the total
    # entropy on a periodic grid: sum_i (V_i . d(JU)_i/dt - phi_i dJ_i/dt) = 0,
    # here on a moving curvilinear mesh
    cfg, cons, J, x, xd = _smooth(14, 20 + p, p, 0)
    dc, dJ = oracle.rhs(cfg, cons, J, x, xd)
    prod = oracle.totals(cfg, cons, J, dc, dJ)[3]
    prim, _ = oracle.state_prim(cfg, cons, J)
    scale = 0.0
    for a in range(8):
        V = np.array([oracle.mhd_entropy_vars(cfg.gamma, prim[:, j, i])[a]
                      for j in range(cfg.ny) for i in range(cfg.nx)])
        scale += np.abs(V * dc[a].ravel()).sum()
    assert abs(prod) < 1e-13 * scale, (prod, scale)


@pytest.mark.parametrize("p", [2, 3])
def test_es_entropy_inequality(p):
    # Thm. 4.1 with the Powell source: production <= 0, smooth and
    # discontinuous periodic data
    cfg, cons, J, x, xd = _smooth(14, 30 + p, p, 5)
    assert oracle.totals(cfg, cons, J, *oracle.rhs(cfg, cons, J, x, xd))[3] < 0.0
    n = 14
    x = wl.uniform_mesh(n, n)
    prim = wl.quadrant_riemann_mhd(x, wl.quadrant_states_mhd(wl.rng(40 + p)), split=(0.5, 0.5))
    cons, J = oracle.init_state(cfg, prim, x)
    assert oracle.totals(cfg, cons, J, *oracle.rhs(cfg, cons, J, x))[3] < 0.0


@pytest.mark.parametrize("w", [0, 5])
def test_free_stream_on_moving_mesh(w):
    # Prop. 3.2: a constant state stays constant on a moving mesh
    n = 12
    cfg = oracle.make_cfg(n, n, gamma=4.0 / 3.0, p=2, w=w, phys=oracle.RMHD)
    x = wl.random_mesh(n, n, wl.rng(50), amp=0.15)
    w0 = np.array([1.3, 0.3, -0.2, 0.1, 0.7, 0.5, -0.8, 0.3])
    prim = np.ascontiguousarray(np.broadcast_to(w0[:, None, None], (8, n, n)))
    cons, J = oracle.init_state(cfg, prim, x)
    xd = wl.random_mesh(n, n, wl.rng(51), amp=0.1) - wl.uniform_mesh(n, n)
    dc, dJ = oracle.rhs(cfg, cons, J, x, np.ascontiguousarray(xd))
    U0 = oracle.mhd_prim2cons(4.0 / 3.0, w0)
    assert np.abs(dc - U0[:, None, None] * dJ[None]).max() < 1e-13 * np.abs(U0).max()


def test_mass_and_volume_conserved():
    cfg, cons, J, x, xd = _smooth(12, 60, 2, 5)
    dc, dJ = oracle.rhs(cfg, cons, J, x, xd)
    assert abs(dc[0].sum()) < 1e-13 * np.abs(dc[0]).sum()
    assert abs(dJ.sum()) < 1e-14 * max(np.abs(dJ).sum(), 1e-30) + 1e-16


def test_ec_scheme_reduces_to_rhd():
    # B = 0, v_3 = 0: the EC right-hand side equals the RHD one
    n = 12
    x = wl.wavy_mesh(n, n)
    prim4 = wl.smooth_random_state(x, wl.rng(70))
    z = 0 * prim4[0]
    prim8 = np.ascontiguousarray(np.stack([prim4[0], prim4[1], prim4[2], z, prim4[3], z, z, z]))
    c4 = oracle.make_cfg(n, n, p=2, w=0)
    c8 = oracle.make_cfg(n, n, p=2, w=0, phys=oracle.RMHD)
    xd = wl.wavy_mesh_velocity(n, n)
    d4, j4 = oracle.rhs(c4, *oracle.init_state(c4, prim4, x), x, xd)
    d8, j8 = oracle.rhs(c8, *oracle.init_state(c8, prim8, x), x, xd)
    sc = np.abs(d4).max()
    np.testing.assert_allclose(d8[[0, 1, 2, 4]], d4, rtol=0, atol=1e-13 * sc)
    assert np.all(d8[[3, 5, 6, 7]] == 0.0)
    np.testing.assert_array_equal(j8, j4)


def test_rotor_steps_keep_planar_symmetry_and_positivity():
    n = 24
    cfg = oracle.make_cfg(n, n, gamma=4.0 / 3.0, p=2, w=5, phys=oracle.RMHD,
                          bc=(oracle.OUTFLOW, oracle.OUTFLOW), period=(1.0, 1.0), alpha=800.0)
    x, prim = wl.rotor_config(n)
    cons, J = oracle.init_state(cfg, prim, x)
    for _ in range(5):
        cons, J, x, dt = oracle.rk_step(cfg, cons, J, x)
        assert dt > 0
    pr, st = oracle.state_prim(cfg, cons, J)
    assert st == 0
    assert np.all(pr[0] > 0) and np.all(pr[4] > 0)
    assert np.all(pr[3] == 0.0) and np.all(pr[7] == 0.0)


def _vortex_truncation_error(n, p, R=8.0, t=2.0):
    """max |rhs - d(JU)/dt| / max |d(JU)/dt| of the EC scheme on the analytic
    RMHD vortex on a static curvilinear mesh; d(JU)/dt of the exact solution
    by a fourth-order central difference in time (error ~1e-12)."""
    x = wl.vortex_mesh(n, R=R)
    cfg = oracle.make_cfg(n, n, period=(2 * R, 2 * R), p=p, w=0, gamma=5.0 / 3.0, phys=oracle.RMHD)
    cons, J = oracle.init_state(cfg, wl.rmhd_vortex(x, t, R=R), x)
    d = 1e-3
    U = lambda tt: oracle.init_state(cfg, wl.rmhd_vortex(x, tt, R=R), x)[0]
    dUdt = (-U(t + 2 * d) + 8 * U(t + d) - 8 * U(t - d) + U(t - 2 * d)) / (12 * d)
    rhs = oracle.rhs(cfg, cons, J, x)[0]
    return np.abs(rhs - dUdt).max() / np.abs(dUdt).max()


@pytest.mark.parametrize("p,order", [(1, 1.9), (2, 3.8), (3, 5.5)])
def test_vortex_truncation_order(p, order):
    # The 2D RMHD isentropic vortex of Sec. 6 (analytic solution, rotating
    # and moving, with a field) is an exact solution of the RMHD system; the
    # EC right-hand side approximates d(JU)/dt to order 2p (Prop. 3.1) on a
    # curvilinear mesh.  The box is [-8, 8]^2 rather than [-5, 5]^2 so that
    # the periodic wrap of the vortex's e^{-r^2/2} tails stays below 1e-12.
    e1, e2 = _vortex_truncation_error(128, p), _vortex_truncation_error(256, p)
    assert np.log2(e1 / e2) > order, (e1, e2)


def _pde_residual(fun, dim, pts, t=0.7, d=1e-3):
    """max |dU/dt + sum_k dF_k/dx_k| / max |dU/dt| of the primitive field
    fun(x [dim][1], t) at the points, by fourth-order central differences in
    t and x of the oracle's pointwise U and F_k (eq. RMHDdiv2, div B = 0)."""
    stencil = ((-1.0, 2), (8.0, 1), (-8.0, -1), (1.0, -2))
    res, scale = 0.0, 0.0
    for P in pts.T:
        w = lambda xx, tt: fun(xx.reshape(dim, 1), tt)[:, 0]
        dU = sum(c * oracle.mhd_prim2cons(G53, w(P, t + o * d)) for c, o in stencil) / (12 * d)
        r = dU.copy()
        for k in range(dim):
            e = np.zeros(dim)
            e[k] = d
            r += sum(c * oracle.mhd_flux(G53, w(P + o * e, t), k) for c, o in stencil) / (12 * d)
        res, scale = max(res, np.abs(r).max()), max(scale, np.abs(dU).max())
    return res / scale


@pytest.mark.parametrize("dim", [2, 3])
def test_analytic_vortices_solve_rmhd(dim):
    # The 2D and 3D RMHD vortices of Sec. 6 are exact solutions: the PDE's
    # residual at random points is at the level of the difference formulas'
    # error (~1e-11).  With the field's exponent as printed, exp(1 - r^2),
    # the same check leaves a residual of ~4e-4.
    pts = wl.rng(90 + dim).uniform(-2.5, 2.5, (dim, 120))
    if dim == 2:
        f = lambda x, t: wl.rmhd_vortex(x, t, R=8.0)
    else:
        f = lambda x, t: wl.rmhd_vortex3(x, t)
    assert _pde_residual(f, dim, pts) < 1e-9


def test_vortex3_is_periodic_on_its_box():
    # shifting a point by a period of [-R, R]^2 x [-5R, 5R] moves the plane
    # coordinates by a lattice vector: the field repeats
    pts = wl.rng(95).uniform(-5.0, 5.0, (3, 500)) * np.array([[1.0], [1.0], [5.0]])
    base = wl.rmhd_vortex3(pts, 0.3)
    for d, per in enumerate((10.0, 10.0, 50.0)):
        q = pts.copy()
        q[d] += per
        assert np.abs(wl.rmhd_vortex3(q, 0.3) - base).max() < 1e-13


def test_shock_cloud_states_satisfy_the_jump_conditions():
    # Sec. 6 shock-cloud: the post- and pre-shock states (the latter read as
    # rho = 1, v = 0, p = 0.05, B = (0, 0.16106, -0.16106) from the garbled
    # print) are joined by one RMHD shock: F(R) - F(L) = s (U(R) - U(L)) for a
    # single speed s in all eight components, to the printed 5-6 digits.
    L, R = np.array(wl.SHOCK_CLOUD_POST), np.array(wl.SHOCK_CLOUD_PRE)
    dU = oracle.mhd_prim2cons(G53, R) - oracle.mhd_prim2cons(G53, L)
    dF = oracle.mhd_flux(G53, R, 0) - oracle.mhd_flux(G53, L, 0)
    s = dU @ dF / (dU @ dU)
    assert np.abs(dF - s * dU).max() < 2e-6 * np.abs(dF).max()
    assert 0.83 < s < 0.85                                     # right-moving, sub-luminal
    # the print's own order of the pre-shock state is not a shock of L
    P = np.array([1.0, 0, 0, 0, 0, 0.16106, 0.16106, 0.05])
    P[4] = 1e-3     # (p = 0 is not admissible; any small pressure)
    dU = oracle.mhd_prim2cons(G53, P) - oracle.mhd_prim2cons(G53, L)
    dF = oracle.mhd_flux(G53, P, 0) - oracle.mhd_flux(G53, L, 0)
    s = dU @ dF / (dU @ dU)
    assert np.abs(dF - s * dU).max() > 1e-3 * np.abs(dF).max()


def test_shock_cloud_inflow_equals_outflow_while_the_boundary_is_uniform():
    # The 2D shock-cloud starts with the post-shock state next to its inflow
    # end, so inflow ghosts (the post-shock state) and zero-gradient ghosts
    # (copies of those nodes) hold the same data, up to the recovery's
    # rounding of the stored state: the same right-hand sides.
    x, prim = wl.rmhd_shock_cloud_config((42, 30))
    kw = dict(period=(1.4, 1.0), p=3, w=5, gamma=G53, phys=oracle.RMHD)
    c_in = oracle.make_cfg(42, 30, bc=(oracle.INFLOW, oracle.OUTFLOW), inflow=wl.SHOCK_CLOUD_POST, **kw)
    c_out = oracle.make_cfg(42, 30, bc=(oracle.OUTFLOW, oracle.OUTFLOW), **kw)
    cons, J = oracle.init_state(c_in, prim, x)
    a, b = oracle.rhs(c_in, cons, J, x), oracle.rhs(c_out, cons, J, x)
    assert np.abs(a[0] - b[0]).max() < 1e-13 * np.abs(a[0]).max()
    assert np.array_equal(a[1], b[1])
    # a different inflow state changes only the first columns
    c_x = oracle.make_cfg(42, 30, bc=(oracle.INFLOW, oracle.OUTFLOW),
                          inflow=np.array(wl.SHOCK_CLOUD_POST) * [1.1, 1, 1, 1, 1.1, 1, 1, 1], **kw)
    d = oracle.rhs(c_x, cons, J, x)[0] - a[0]
    assert np.abs(d[:, :, :3]).max() > 1e-3 * np.abs(a[0]).max()
    assert np.abs(d[:, :, 3:]).max() < 1e-13 * np.abs(a[0]).max()
