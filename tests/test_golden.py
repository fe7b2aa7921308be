"""Pins against the numbers printed in Sec. 6 (the fixtures under
tests/golden/, each record citing its example):

- the workloads' initial data and parameters are the paper's;
- the states that an example joins by a shock or a contact satisfy the
  jump conditions of the oracle's conserved variables and fluxes: to
  rounding where the paper prints 15 digits (Riemann problem III, the 3D
  shock-bubble), to rounding for the contacts of Riemann problems I and III;
- the states of Riemann problem II that meet the rest state lie on one
  isentropic simple wave, to the 4 printed digits;
- the CPU-time shares that the text states follow from the printed times
  to within one unit of their last digit, except for the 3D shock-cloud,
  where the stated 9.06% matches a total of 34h56m49s for the fine UM-O5
  run and not the printed 34h46m49s (one digit of the two is a misprint;
  nothing here depends on which)."""
import inspect
import os
from fractions import Fraction

import numpy as np

import oracle
from paper_2107_12027_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _num(tok):
    return float(Fraction(tok)) if "/" in tok else float(tok)


def _records(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                out.setdefault(line[0], []).append(line[1:])
    return out


def _data():
    return {k: np.array([_num(t) for t in v[0]]) for k, v in _records("paper_example_data.txt").items()}


def _defaults(fn):
    return {k: p.default for k, p in inspect.signature(fn).parameters.items() if p.default is not p.empty}


QUAD = ("ll", "lr", "ul", "ur")   # quadrant q = (x_1 > s_1) + 2 (x_2 > s_2) of the workloads


def _rh(gamma, left, right, direction, prim2cons=oracle.prim2cons, flux=oracle.flux):
    """Speed s of the best fit F(R) - F(L) = s (U(R) - U(L)) and the
    residual relative to the larger of the two jumps (a contact at rest has
    no flux jump)."""
    dU = prim2cons(gamma, np.asarray(right)) - prim2cons(gamma, np.asarray(left))
    dF = flux(gamma, np.asarray(right), direction) - flux(gamma, np.asarray(left), direction)
    s = dU @ dF / (dU @ dU)
    return s, np.abs(dF - s * dU).max() / max(np.abs(dF).max(), np.abs(dU).max())


def test_workload_data_are_the_papers():
    d = _data()
    for k in (1, 2, 3):
        assert np.array_equal(np.array(wl.RHD_RP_STATES[k]), np.stack([d["rp%d.%s" % (k, q)] for q in QUAD]))
    # the Riemann problems on [0,1]^2 split at (0.5, 0.5)
    x, prim = wl.rhd_rp_config(3, 9)
    assert x[0].min() == 0.0 and x[0].max() == 1.0
    assert np.array_equal(prim[:, -1, -1], d["rp3.ur"]) and np.array_equal(prim[:, 0, 0], d["rp3.ll"])
    v = _defaults(wl.rmhd_vortex)
    assert (v["R"], v["sigma"], v["B0"]) == (d["vortex2d.R"][0], d["vortex2d.sigma"][0], d["vortex2d.B0"][0])
    assert v["gamma"] == d["vortex2d.gamma"][0]
    assert _defaults(wl.vortex_mesh)["amp"] == d["vortex2d.mesh_amplitude"][0]
    # the vortex moves with the printed velocity: its data at (x, t) are those
    # at (x - t velocity, 0)
    x = wl.vortex_mesh(24, t=0.7)
    sh = x - 1.3 * d["vortex2d.velocity"][:, None, None]
    assert np.allclose(wl.rmhd_vortex(x, t=1.3), wl.rmhd_vortex(sh, t=0.0), rtol=0, atol=1e-12)
    v3 = _defaults(wl.rmhd_vortex3)
    assert (v3["R"], v3["gamma"], v3["sigma"], v3["B0"]) == tuple(
        d["vortex3d." + k][0] for k in ("R", "gamma", "sigma", "B0"))
    x = wl.vortex_mesh3(6)
    x0 = wl.uniform_mesh3((6, 6, 30), *np.reshape(d["vortex3d.box"], (3, 2)).T)
    assert np.allclose(x0, wl.vortex_mesh3(6, t=2.0), rtol=0, atol=1e-12)       # cos(pi t/4) = 0
    assert np.allclose(x, x0, rtol=0, atol=0.21)
    # a shift of x by a box period moves the plane coordinates by a printed
    # lattice vector (x -> x + 2R e_1: (40/3, 10/3)), and leaves the data (up
    # to ~4e-11: the nearest lattice image jumps where two are equally near,
    # and the vortex's tail is not quite zero there)
    lat = d["vortex3d.lattice"].reshape(2, 2)
    R = d["vortex3d.R"][0]
    assert np.allclose(lat[0], (2 * R + 2 * R / 3, 2 * R / 3), rtol=0, atol=1e-12)
    sh = x + np.array([2 * R, 0.0, 0.0])[:, None, None, None]
    assert np.allclose(wl.rmhd_vortex3(sh, t=0.05), wl.rmhd_vortex3(x, t=0.05), rtol=0, atol=1e-10)
    b = _defaults(wl.rmhd_blast2)
    assert (b["r_in"], b["r_out"]) == (d["blast2d.r_inner"][0], d["blast2d.r_outer"][0])
    assert (b["rho_in"], b["p_in"]) == tuple(d["blast2d.inner_rho_p"])
    assert (b["rho_out"], b["p_out"]) == tuple(d["blast2d.outer_rho_p"])
    assert b["Bx"] == d["blast2d.B1"][0]
    x, _ = wl.rmhd_blast2_config(5)
    assert x[0].max() == d["blast2d.half_width"][0] == -x[0].min()
    assert np.array_equal(np.array(wl.SHOCK_CLOUD_POST), d["shockcloud2d.post"])
    c = _defaults(wl.rmhd_shock_cloud)
    assert (c["x_shock"], c["r_cloud"], c["rho_cloud"]) == (
        d["shockcloud2d.x_shock"][0], d["shockcloud2d.cloud_radius"][0], d["shockcloud2d.cloud_rho"][0])
    x, prim = wl.rmhd_shock_cloud_config((15, 11))
    dom = d["shockcloud2d.domain"]
    assert np.allclose((x[0].min(), x[0].max(), x[1].min(), x[1].max()), dom, rtol=0, atol=1e-14)
    ic = np.argmin((x[0] - 0.25) ** 2 + (x[1] - 0.5) ** 2)                  # the cloud's centre
    assert tuple(d["shockcloud2d.cloud_centre"]) == (0.25, 0.5) and prim[0].flat[ic] == 30.0
    # the sphere: states inside and outside r0
    pts = np.array([[0.0, 0.3, 0.49, 0.51, 0.9], [0.0] * 5, [0.0] * 5])[:, :, None, None]
    s = wl.sphere_rp3(pts)[:, :, 0, 0]
    assert _defaults(wl.sphere_rp3)["r0"] == d["sphere3d.r0"][0]
    assert np.array_equal(s[:5, :3].T, np.stack([d["sphere3d.inside"]] * 3))
    assert np.array_equal(s[:5, 3:].T, np.stack([d["sphere3d.outside"]] * 2))
    assert not s[5:].any()
    # the shock-bubble
    pre, post, gas = (np.array(t[:5]) for t in (wl.SHOCK_BUBBLE_PRE, wl.SHOCK_BUBBLE_POST, wl.SHOCK_BUBBLE_GAS))
    assert np.array_equal(pre, d["shockbubble3d.pre"]) and np.array_equal(post, d["shockbubble3d.post"])
    assert np.array_equal(gas, d["shockbubble3d.bubble"])
    sb = _defaults(wl.rhd_shock_bubble3)
    assert sb["x_shock"] == d["shockbubble3d.x_shock"][0] and sb["radius"] == d["shockbubble3d.bubble_radius"][0]
    assert np.array_equal(np.array(sb["centre"]), d["shockbubble3d.bubble_centre"])
    x, prim = wl.rhd_shock_bubble3_config((14, 7, 7))
    dom = d["shockbubble3d.domain"]
    assert np.array_equal([x[k].min() for k in range(3)], dom[0::2])
    assert np.array_equal([x[k].max() for k in range(3)], dom[1::2])
    assert np.array_equal(prim[:5, 3, 3, -1], post) and np.array_equal(prim[:5, 3, 3, 0], pre)
    assert np.array_equal(prim[:5, 3, 3, 9], gas)                              # x_1 = 225, inside the bubble
    assert not prim[5:].any()
    x, prim = wl.rmhd_shock_cloud3_config((15, 11, 11))
    assert np.allclose([x[k].min() for k in range(3)], d["shockcloud3d.domain"][0::2], rtol=0, atol=1e-14)
    assert np.allclose([x[k].max() for k in range(3)], d["shockcloud3d.domain"][1::2], rtol=0, atol=1e-14)
    assert prim[0, 5, 5, 5] == 30.0 and tuple(d["shockcloud3d.cloud_centre"]) == (0.25, 0.5, 0.5)


def test_shock_cloud_pre_state_reading():
    # The printed pre-shock state has p = 0, which is not admissible.  The
    # reading (rho = 1, v = 0, p = 0.05, B = (0, 0.16106, -0.16106)) takes the
    # printed magnitudes in another order, with B_3 = -B_2 as behind the
    # shock; its jump conditions with the post-shock state are pinned in the
    # RMHD oracle tests.
    d = _data()
    printed = d["shockcloud2d.pre_as_printed"]
    assert printed[4] == 0.0
    assert sorted(np.abs(wl.SHOCK_CLOUD_PRE)) == sorted(printed)
    assert wl.SHOCK_CLOUD_PRE[7] == -wl.SHOCK_CLOUD_PRE[6] and d["shockcloud2d.post"][7] == -d["shockcloud2d.post"][6]


def test_rp3_shocks_satisfy_the_jump_conditions():
    # Riemann problem III: the top (x_1 = 0.5, x_2 > 0.5) and right (x_2 =
    # 0.5, x_1 > 0.5) discontinuities are single shocks.  The 15-digit state
    # makes the jump F(ur) - F(n) = s (U(ur) - U(n)) hold to rounding, with
    # the same speed for both by the data's symmetry.
    d, g = _data(), float(Fraction(5, 3))
    s1, r1 = _rh(g, d["rp3.ul"], d["rp3.ur"], 0)
    s2, r2 = _rh(g, d["rp3.lr"], d["rp3.ur"], 1)
    assert r1 < 1e-14 and r2 < 1e-14
    assert abs(s1 - s2) < 1e-14 and 0.9 < s1 < 1.0
    # the same jump through the RMHD oracle at B = 0
    wl8 = np.r_[d["rp3.ul"][:3], 0.0, d["rp3.ul"][3], 0.0, 0.0, 0.0]
    wr8 = np.r_[d["rp3.ur"][:3], 0.0, d["rp3.ur"][3], 0.0, 0.0, 0.0]
    s3, r3 = _rh(g, wl8, wr8, 0, oracle.mhd_prim2cons, oracle.mhd_flux)
    assert r3 < 1e-14 and abs(s3 - s1) < 1e-14
    # the pin sees the thermodynamics: with Gamma = 4/3 the same states are
    # far from any single jump
    assert _rh(4.0 / 3.0, d["rp3.ul"], d["rp3.ur"], 0)[1] > 1e-3


def test_shock_bubble_states_satisfy_the_jump_conditions():
    # 3D shock-bubble: the post-shock state (x_1 > 265, moving to the left)
    # and the medium (x_1 < 265) are joined by one left-moving shock
    d, g = _data(), float(Fraction(5, 3))
    pre, post = d["shockbubble3d.pre"], d["shockbubble3d.post"]
    s, r = _rh(g, pre[[0, 1, 2, 4]], post[[0, 1, 2, 4]], 0)
    assert r < 1e-14 and -0.42 < s < -0.41
    s8, r8 = _rh(g, np.r_[pre, 0, 0, 0], np.r_[post, 0, 0, 0], 0, oracle.mhd_prim2cons, oracle.mhd_flux)
    assert r8 < 1e-14 and abs(s8 - s) < 1e-14


def test_contacts_move_with_the_normal_velocity():
    # Riemann problems I and III: across each contact the pressure and the
    # normal velocity are continuous and the jump moves with that velocity:
    # F(R) - F(L) = v_n (U(R) - U(L)) with s = v_n exactly (to rounding)
    d, g = _data(), float(Fraction(5, 3))
    pairs = [("rp1", "ul", "ur", 0), ("rp1", "ll", "lr", 0), ("rp1", "ll", "ul", 1), ("rp1", "lr", "ur", 1),
             ("rp3", "ll", "ul", 1), ("rp3", "ll", "lr", 0)]
    for k, a, b, dirn in pairs:
        L, R = d["%s.%s" % (k, a)], d["%s.%s" % (k, b)]
        assert L[3] == R[3] and L[1 + dirn] == R[1 + dirn]
        s, r = _rh(g, L, R, dirn)
        assert r < 1e-14 and abs(s - L[1 + dirn]) < 1e-14


def _isentropic_invariants(gamma, w):
    """p / rho^Gamma and the Riemann invariants atanh(v) -+ (2 / sqrt(Gamma -
    1)) atanh(c_s / sqrt(Gamma - 1)) of 1D isentropic relativistic flow
    along v (no tangential velocity), with c_s^2 = Gamma p / (rho h)."""
    rho, v, p = w
    h = 1.0 + gamma / (gamma - 1.0) * p / rho
    cs = np.sqrt(gamma * p / (rho * h))
    a = np.sqrt(gamma - 1.0)
    return p / rho ** gamma, np.arctanh(v) - 2.0 / a * np.arctanh(cs / a), np.arctanh(v) + 2.0 / a * np.arctanh(cs / a)


def test_rp2_rarefactions_are_isentropic_simple_waves():
    # Riemann problem II: the rest state (ur) meets ul across x_1 = 0.5 and
    # lr across x_2 = 0.5 with no tangential velocity on either side.  A
    # right-facing rarefaction keeps the entropy p / rho^Gamma and the
    # invariant J_- = atanh(v_n) - 2/sqrt(Gamma-1) atanh(c_s/sqrt(Gamma-1));
    # the printed 4-digit states hold both to ~1e-4, and break J_+ at O(1).
    d, g = _data(), float(Fraction(5, 3))
    ur = d["rp2.ur"]
    for q, dirn in (("ul", 0), ("lr", 1)):
        w = d["rp2." + q]
        assert w[2 - dirn] == 0.0 and ur[1] == ur[2] == 0.0
        e0, jm0, jp0 = _isentropic_invariants(g, (ur[0], 0.0, ur[3]))
        e1, jm1, jp1 = _isentropic_invariants(g, (w[0], w[1 + dirn], w[3]))
        assert abs(e1 - e0) < 2e-4 and abs(jm1 - jm0) < 2e-4 * abs(jm0)
        assert abs(jp1 - jp0) > 0.1


def _seconds(t):
    out, num = 0, ""
    for ch in t:
        if ch.isdigit():
            num += ch
        else:
            out += int(num) * {"h": 3600, "m": 60, "s": 1}[ch]
            num = ""
    return out


def test_stated_cpu_time_shares_follow_from_the_printed_times():
    rec = _records("paper_cpu_times.txt")
    for ex, rows in rec.items():
        times = {}
        stated = None
        for row in rows:
            if row[0] == "stated_percent":
                stated = float(row[1])
            else:
                times[(row[0], row[1])] = _seconds(row[2])
        mm = [t for (s, _), t in times.items() if s == "MM-O5"][0]
        um = max(t for (s, _), t in times.items() if s == "UM-O5")      # the finer UM-O5 run
        share = 100.0 * mm / um
        digits = 0.1 if stated >= 10 else 0.01                             # one unit of the last printed digit
        if ex == "shockcloud3d":
            assert abs(share - stated) > 0.03                              # 9.10% from the printed times
            assert abs(share - 9.10) < 0.01
            assert abs(100.0 * mm / _seconds("34h56m49s") - stated) < digits
        else:
            assert abs(share - stated) < digits, (ex, share, stated)


def test_study_runs_the_papers_comparisons():
    # The UM-O5 against MM-O5 study of bench.py runs to the paper's final
    # times on the paper's MM-O5 meshes and its fine UM-O5 meshes (500^2 for
    # RP I and II, 600^2 for RP III), and for the blast also its coarse
    # UM-O5 mesh.
    import bench
    d, rec = _data(), _records("paper_cpu_times.txt")
    for k in (1, 2, 3):
        sizes, t_end = bench.STUDY["rp%d" % k]
        assert t_end == d["rp%d.t_end" % k][0]
        meshes = {(r[0], int(r[1].split("x")[0])) for r in rec["rp%d" % k] if r[0] != "stated_percent"}
        assert ("MM-O5", sizes[0]) in meshes
        assert ("UM-O5", sizes[2]) in meshes
    sizes, t_end = bench.STUDY["blast"]
    assert t_end == d["blast2d.t_end"][0]
    meshes = {(r[0], int(r[1].split("x")[0])) for r in rec["blast2d"] if r[0] != "stated_percent"}
    assert {("MM-O5", sizes[0]), ("UM-O5", sizes[1]), ("UM-O5", sizes[2])} <= meshes
