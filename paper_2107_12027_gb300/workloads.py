"""Seeded synthetic inputs shaped like the paper's 2D RHD tests.

This module only draws initial data and meshes (numpy PCG64, fixed seeds); it
contains none of the scheme's arithmetic, so both the CUDA path and the oracle
can be fed from it.  Arrays are structure-of-arrays, ``[comp][j][i]``, FP64.
"""
from __future__ import annotations

import numpy as np

SEED = 20210726  # base seed; workloads add a config index and a problem id


def rng(offset: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED + offset))


# ---- meshes -----------------------------------------------------------------
def uniform_mesh(nx, ny, lo=(0.0, 0.0), hi=(1.0, 1.0), periodic=(True, True)):
    """Nodes of a uniform mesh.  A periodic direction has nx distinct nodes
    spaced L/nx starting at lo; an outflow direction has nodes on both ends."""
    ax = []
    for n, a, b, per in ((nx, lo[0], hi[0], periodic[0]), (ny, lo[1], hi[1], periodic[1])):
        ax.append(a + (b - a) * np.arange(n) / (n if per else (n - 1)))
    X, Y = np.meshgrid(ax[0], ax[1])
    return np.ascontiguousarray(np.stack([X, Y]))


def wavy_mesh(nx, ny, lo=(0.0, 0.0), hi=(1.0, 1.0), amp=0.05, t=0.0, periodic=(True, True)):
    """A smooth curvilinear mesh: a uniform mesh displaced like the prescribed
    vortex mesh, x = x0 + amp cos(pi t/4) sin(2 pi k y0/L), with k chosen so the
    displacement is periodic (and zero on outflow boundaries)."""
    x0 = uniform_mesh(nx, ny, lo, hi, periodic)
    Lx, Ly = hi[0] - lo[0], hi[1] - lo[1]
    s = amp * np.cos(np.pi * t / 4.0)
    X = x0[0] + s * Lx * np.sin(2 * np.pi * (x0[1] - lo[1]) / Ly) * np.sin(np.pi * (x0[0] - lo[0]) / Lx) ** (0 if periodic[0] else 2)
    Y = x0[1] + s * Ly * np.sin(2 * np.pi * (x0[0] - lo[0]) / Lx) * np.sin(np.pi * (x0[1] - lo[1]) / Ly) ** (0 if periodic[1] else 2)
    return np.ascontiguousarray(np.stack([X, Y]))


def wavy_mesh_velocity(nx, ny, lo=(0.0, 0.0), hi=(1.0, 1.0), amp=0.05, t=0.0, periodic=(True, True)):
    """d/dt of :func:`wavy_mesh` (the prescribed mesh velocity)."""
    x0 = uniform_mesh(nx, ny, lo, hi, periodic)
    Lx, Ly = hi[0] - lo[0], hi[1] - lo[1]
    ds = -amp * np.pi / 4.0 * np.sin(np.pi * t / 4.0)
    X = ds * Lx * np.sin(2 * np.pi * (x0[1] - lo[1]) / Ly) * np.sin(np.pi * (x0[0] - lo[0]) / Lx) ** (0 if periodic[0] else 2)
    Y = ds * Ly * np.sin(2 * np.pi * (x0[0] - lo[0]) / Lx) * np.sin(np.pi * (x0[1] - lo[1]) / Ly) ** (0 if periodic[1] else 2)
    return np.ascontiguousarray(np.stack([X, Y]))


def random_mesh(nx, ny, r, amp=0.15, lo=(0.0, 0.0), hi=(1.0, 1.0), periodic=(True, True)):
    """A uniform mesh with every node jittered by up to amp of a spacing
    (non-smooth, untangled): used where an identity must hold for any mesh."""
    x0 = uniform_mesh(nx, ny, lo, hi, periodic)
    hx = (hi[0] - lo[0]) / (nx if periodic[0] else nx - 1)
    hy = (hi[1] - lo[1]) / (ny if periodic[1] else ny - 1)
    d = r.uniform(-amp, amp, size=x0.shape)
    d[0] *= hx
    d[1] *= hy
    if not periodic[0]:
        d[:, :, 0] = 0.0
        d[:, :, -1] = 0.0
    if not periodic[1]:
        d[:, 0, :] = 0.0
        d[:, -1, :] = 0.0
    return np.ascontiguousarray(x0 + d)


# ---- states -----------------------------------------------------------------
def random_states(r, n, rho=(0.1, 10.0), p=(0.01, 10.0), vmax=0.9):
    """n admissible primitive states (rho, vx, vy, p), log-uniform rho and p."""
    rho_ = np.exp(r.uniform(np.log(rho[0]), np.log(rho[1]), n))
    p_ = np.exp(r.uniform(np.log(p[0]), np.log(p[1]), n))
    sp = vmax * np.sqrt(r.uniform(0.0, 1.0, n))
    th = r.uniform(0.0, 2 * np.pi, n)
    return np.stack([rho_, sp * np.cos(th), sp * np.sin(th), p_], axis=-1)


def sine_wave(x, t=0.0):
    """Smooth density advection: rho = 1 + 0.2 sin(2 pi (x + y - 0.4 t)),
    v = (0.2, 0.2), p = 1 (an exact RHD solution)."""
    X, Y = x[0], x[1]
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * (X + Y - 0.4 * t))
    return np.ascontiguousarray(np.stack([rho, 0.2 + 0 * X, 0.2 + 0 * X, 1.0 + 0 * X]))


def smooth_random_state(x, r, amp=0.2, modes=3):
    """A smooth periodic state on [0,1]^2 with a few random Fourier modes in
    each primitive variable (used for the entropy-identity checks)."""
    X, Y = x[0], x[1]
    out = []
    for base, a in ((1.0, amp), (0.1, 0.3), (-0.1, 0.3), (1.0, amp)):
        f = base + 0 * X
        for _ in range(modes):
            kx, ky = r.integers(-2, 3, 2)
            ph = r.uniform(0, 2 * np.pi)
            f = f + a / modes * np.sin(2 * np.pi * (kx * X + ky * Y) + ph)
        out.append(f)
    return np.ascontiguousarray(np.stack(out))


def quadrant_states(r, vmax=0.9):
    """Four seeded states of a four-quadrant Riemann problem: rho in [0.1, 1],
    p in [0.01, 1], |v| in [0, vmax] with a uniform direction."""
    rho = r.uniform(0.1, 1.0, 4)
    p = r.uniform(0.01, 1.0, 4)
    sp = r.uniform(0.0, vmax, 4)
    th = r.uniform(0.0, 2 * np.pi, 4)
    return np.stack([rho, sp * np.cos(th), sp * np.sin(th), p], axis=-1)


def quadrant_riemann(x, states, split=(0.0, 0.0)):
    """Piecewise-constant data: quadrant q = (x > sx) + 2 (y > sy)."""
    q = (x[0] > split[0]).astype(int) + 2 * (x[1] > split[1]).astype(int)
    prim = np.empty((4,) + x.shape[1:])
    for c in range(4):
        prim[c] = states[q, c]
    return np.ascontiguousarray(prim)


def riemann_config(n=400, offset=1):
    """2D RHD four-quadrant Riemann problem on [-1,1]^2 with outflow
    boundaries, n x n nodes, seeded states (the 400^2 benchmark workload)."""
    x = uniform_mesh(n, n, (-1.0, -1.0), (1.0, 1.0), (False, False))
    states = quadrant_states(rng(offset))
    return x, quadrant_riemann(x, states)


def sine_config(n=64):
    """2D RHD smooth sine wave on periodic [0,1]^2, n x n nodes."""
    x = uniform_mesh(n, n, (0.0, 0.0), (1.0, 1.0), (True, True))
    return x, sine_wave(x)


def batch_sizes(nprob=256, side=(64, 512), offset=4):
    """Side lengths of the batched workload: uniform integers in [64, 512]."""
    return rng(offset).integers(side[0], side[1] + 1, size=nprob)


def batch_problem(k, n, vmax=0.5, offset=1000):
    """Problem k of the batched workload: a seeded four-quadrant Riemann
    problem on [-1,1]^2 with n x n nodes (outflow); speeds up to vmax."""
    x = uniform_mesh(n, n, (-1.0, -1.0), (1.0, 1.0), (False, False))
    return x, quadrant_riemann(x, quadrant_states(rng(offset + k), vmax=vmax))


# ---- RMHD states: prim[8] = (rho, v_1, v_2, v_3, p, B_1, B_2, B_3) -------------
def random_states_mhd(r, n, rho=(0.1, 10.0), p=(0.01, 10.0), vmax=0.9, bmax=1.5):
    """n admissible RMHD primitive states: log-uniform rho and p, |v| <= vmax
    with a uniform direction in 3D, each B component uniform in [-bmax, bmax]."""
    rho_ = np.exp(r.uniform(np.log(rho[0]), np.log(rho[1]), n))
    p_ = np.exp(r.uniform(np.log(p[0]), np.log(p[1]), n))
    d = r.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    v = d * (vmax * np.cbrt(r.uniform(0.0, 1.0, n)))[:, None]
    B = r.uniform(-bmax, bmax, (n, 3))
    return np.concatenate([rho_[:, None], v, p_[:, None], B], axis=1)


def smooth_random_state_mhd(x, r, amp=0.2, modes=3):
    """A smooth periodic RMHD state on [0,1]^2: a few random Fourier modes in
    each of the eight primitive variables (entropy-identity checks)."""
    X, Y = x[0], x[1]
    out = []
    for base, a in ((1.0, amp), (0.1, 0.3), (-0.1, 0.3), (0.05, 0.2), (1.0, amp),
                    (0.5, 0.3), (-0.3, 0.3), (0.2, 0.3)):
        f = base + 0 * X
        for _ in range(modes):
            kx, ky = r.integers(-2, 3, 2)
            ph = r.uniform(0, 2 * np.pi)
            f = f + a / modes * np.sin(2 * np.pi * (kx * X + ky * Y) + ph)
        out.append(f)
    return np.ascontiguousarray(np.stack(out))


def quadrant_states_mhd(r, vmax=0.5, bmax=1.0):
    """Four seeded RMHD quadrant states: rho in [0.1, 1], p in [0.01, 1],
    in-plane |v| in [0, vmax] with a uniform direction, v_3 = 0, B_1, B_2 in
    [-bmax, bmax], B_3 in [-bmax/2, bmax/2]."""
    rho = r.uniform(0.1, 1.0, 4)
    p = r.uniform(0.01, 1.0, 4)
    sp = r.uniform(0.0, vmax, 4)
    th = r.uniform(0.0, 2 * np.pi, 4)
    B = np.stack([r.uniform(-bmax, bmax, 4), r.uniform(-bmax, bmax, 4),
                  r.uniform(-0.5 * bmax, 0.5 * bmax, 4)], axis=-1)
    return np.concatenate([np.stack([rho, sp * np.cos(th), sp * np.sin(th), 0 * rho, p], axis=-1), B],
                          axis=1)


def quadrant_riemann_mhd(x, states, split=(0.0, 0.0)):
    """Piecewise-constant RMHD data: quadrant q = (x > sx) + 2 (y > sy)."""
    q = (x[0] > split[0]).astype(int) + 2 * (x[1] > split[1]).astype(int)
    prim = np.empty((8,) + x.shape[1:])
    for c in range(8):
        prim[c] = states[q, c]
    return np.ascontiguousarray(prim)


def rotor(x, rho_in=10.0, omega=9.95, r0=0.1, rho_out=1.0, p=1.0, Bx=1.0, r1=None):
    """The rotor: a disk r < r0 of density rho_in spinning rigidly at angular
    speed omega (|v| <= omega r0 = 0.995), background rho_out at rest,
    uniform pressure p and field B = (Bx, 0, 0).  With r1 > r0, density and
    angular speed fall linearly from the disk values at r0 to the background
    at r1 (a tapered rotor)."""
    X, Y = x[0], x[1]
    r = np.sqrt(X * X + Y * Y)
    if r1 is None:
        f = (r < r0).astype(float)
    else:
        f = np.clip((r1 - r) / (r1 - r0), 0.0, 1.0)
    z = 0 * X
    rho = rho_out + f * (rho_in - rho_out)
    om = f * omega * np.where(r < r0, 1.0, r0 / np.maximum(r, 1e-300))   # |v| continuous, <= omega r0
    vx = -om * Y
    vy = om * X
    return np.ascontiguousarray(np.stack([rho, vx, vy, z, p + z, Bx + z, z, z]))


def rotor_config(n=512, taper=None):
    """2D RMHD rotor on [-0.5,0.5]^2 with outflow boundaries, n x n nodes,
    Gamma = 4/3 (the 512^2 RMHD workload); taper = r1 for the tapered disk."""
    x = uniform_mesh(n, n, (-0.5, -0.5), (0.5, 0.5), (False, False))
    return x, rotor(x, r1=taper)


# ---- 3D (RMHD) ----------------------------------------------------------------
# Arrays [comp][k][j][i] (i fastest), the layout of the 3D C ABI.
def uniform_mesh3(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), periodic=(True, True, True)):
    """Nodes of a uniform 3D mesh (conventions of :func:`uniform_mesh`)."""
    ax = [a + (b - a) * np.arange(m) / (m if per else (m - 1)) for m, a, b, per in zip(n, lo, hi, periodic)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return np.ascontiguousarray(np.stack([X, Y, Z]))


def wavy_mesh3(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), amp=0.04, t=0.0, periodic=(True, True, True)):
    """A smooth curvilinear 3D mesh: each coordinate displaced by a product of
    sines of the other two (periodic, zero on outflow faces)."""
    x0 = uniform_mesh3(n, lo, hi, periodic)
    s = amp * np.cos(np.pi * t / 4.0)
    out = []
    for d in range(3):
        L = [hi[k] - lo[k] for k in range(3)]
        a, b = (d + 1) % 3, (d + 2) % 3
        f = np.sin(2 * np.pi * (x0[a] - lo[a]) / L[a]) * np.sin(2 * np.pi * (x0[b] - lo[b]) / L[b])
        if not periodic[d]:
            f = f * np.sin(np.pi * (x0[d] - lo[d]) / L[d]) ** 2
        out.append(x0[d] + s * L[d] * f)
    return np.ascontiguousarray(np.stack(out))


def wavy_mesh_velocity3(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), amp=0.04, t=0.0, periodic=(True, True, True)):
    """d/dt of :func:`wavy_mesh3`."""
    x0 = uniform_mesh3(n, lo, hi, periodic)
    ds = -amp * np.pi / 4.0 * np.sin(np.pi * t / 4.0)
    out = []
    for d in range(3):
        L = [hi[k] - lo[k] for k in range(3)]
        a, b = (d + 1) % 3, (d + 2) % 3
        f = np.sin(2 * np.pi * (x0[a] - lo[a]) / L[a]) * np.sin(2 * np.pi * (x0[b] - lo[b]) / L[b])
        if not periodic[d]:
            f = f * np.sin(np.pi * (x0[d] - lo[d]) / L[d]) ** 2
        out.append(ds * L[d] * f)
    return np.ascontiguousarray(np.stack(out))


def random_mesh3(n, r, amp=0.15, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), periodic=(True, True, True)):
    """A uniform 3D mesh with every node jittered by up to amp of a spacing
    (outflow faces keep their normal coordinate)."""
    x0 = uniform_mesh3(n, lo, hi, periodic)
    d = r.uniform(-amp, amp, size=x0.shape)
    for k in range(3):
        d[k] *= (hi[k] - lo[k]) / (n[k] if periodic[k] else n[k] - 1)
    for k in range(3):
        if not periodic[k]:
            sl = [slice(None)] * 3
            for end in (0, -1):
                sl[2 - k] = end
                d[(k,) + tuple(sl)] = 0.0
    return np.ascontiguousarray(x0 + d)


def smooth_random_state_mhd3(x, r, amp=0.2, modes=3):
    """A smooth periodic 3D RMHD state on [0,1]^3 with a few random Fourier
    modes in each of the eight primitive variables."""
    X, Y, Z = x[0], x[1], x[2]
    out = []
    for base, a in ((1.0, amp), (0.1, 0.3), (-0.1, 0.3), (0.05, 0.3), (1.0, amp),
                    (0.5, 0.3), (-0.3, 0.3), (0.2, 0.3)):
        f = base + 0 * X
        for _ in range(modes):
            kx, ky, kz = r.integers(-2, 3, 3)
            ph = r.uniform(0, 2 * np.pi)
            f = f + a / modes * np.sin(2 * np.pi * (kx * X + ky * Y + kz * Z) + ph)
        out.append(f)
    return np.ascontiguousarray(np.stack(out))


def blast3(x, r0=0.1, p_in=1.0, p_out=5e-4, rho_in=1e-2, rho_out=1e-4, B=(0.1, 0.0, 0.0)):
    """The 3D RMHD blast: a sphere r < r0 at pressure p_in in a background at
    p_out; density rho_in inside (reading: the paper's 2D blast explosion
    zone) and rho_out outside; at rest; uniform B."""
    X, Y, Z = x[0], x[1], x[2]
    inside = (X * X + Y * Y + Z * Z) < r0 * r0
    z = 0 * X
    rho = np.where(inside, rho_in, rho_out)
    p = np.where(inside, p_in, p_out)
    return np.ascontiguousarray(np.stack([rho, z, z, z, p, B[0] + z, B[1] + z, B[2] + z]))


def blast3_config(n=128):
    """3D RMHD blast on [-0.5,0.5]^3 with outflow faces, n^3 nodes, Gamma = 4/3
    (the 128^3 adjoint workload)."""
    x = uniform_mesh3((n, n, n), (-0.5, -0.5, -0.5), (0.5, 0.5, 0.5), (False, False, False))
    return x, blast3(x)


# ---- the 2D RMHD isentropic vortex (Sec. 6, 2D RMHD vortex example) --------
def vortex_mesh(n, t=0.0, R=5.0, amp=0.2):
    """The example's prescribed moving mesh on the periodic box [-R, R]^2 (n
    distinct nodes per direction, spacing 2R/n): x_1 = x0_1 + amp cos(pi t/4)
    sin(3 pi x0_2 / R), x_2 = x0_2 + amp cos(pi t/4) sin(3 pi x0_1 / R)."""
    x0 = uniform_mesh(n, n, (-R, -R), (R, R))
    s = amp * np.cos(np.pi * t / 4.0)
    return np.ascontiguousarray(np.stack([x0[0] + s * np.sin(3 * np.pi * x0[1] / R),
                                          x0[1] + s * np.sin(3 * np.pi * x0[0] / R)]))


def vortex_mesh_velocity(n, t=0.0, R=5.0, amp=0.2):
    """d/dt of vortex_mesh at fixed computational coordinates."""
    x0 = uniform_mesh(n, n, (-R, -R), (R, R))
    s = -amp * (np.pi / 4.0) * np.sin(np.pi * t / 4.0)
    return np.ascontiguousarray(np.stack([s * np.sin(3 * np.pi * x0[1] / R), s * np.sin(3 * np.pi * x0[0] / R)]))


def rmhd_vortex(x, t=0.0, R=5.0, gamma=5.0 / 3.0, sigma=0.2, B0=0.05):
    """The example's analytic RMHD vortex (primitives [8][...] at the points
    x [2][...] and time t): a rotated, boosted isentropic vortex moving with
    velocity (-0.5, -0.5) on the periodic box [-R, R]^2, Gamma = 5/3.

    The magnetic field of the vortex frame is B0 exp((1 - r^2)/2)(-x2, x1):
    radial balance of the rotating equilibrium, d(p + B^2/2)/dr = (rho h W^2
    v^2 - B^2)/r, gives the printed rotation rate f with the printed kappa =
    2 Gamma sigma rho + (Gamma-1) B0^2 (2 - r^2) for that field (with
    exp(1 - r^2), as the text reads, kappa's field term would be
    2 (Gamma-1) B0^2 exp(1 - r^2)(1 - r^2) instead)."""
    s2 = np.sqrt(2.0)
    xh = [np.mod(x[k] + t / 2.0 - 1.0 + R, 2.0 * R) - R for k in range(2)]
    xt = [xh[k] + (s2 - 1.0) * (xh[0] + xh[1]) / 2.0 for k in range(2)]
    r2 = xt[0] ** 2 + xt[1] ** 2
    e = np.exp(1.0 - r2)
    rho = (1.0 - sigma * e) ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    kappa = 2.0 * gamma * sigma * rho + (gamma - 1.0) * B0 ** 2 * (2.0 - r2)
    f = np.sqrt(kappa * e / (kappa * r2 * e + (gamma - 1.0) * rho + gamma * p))
    vt1, vt2 = -xt[1] * f, xt[0] * f
    den = 4.0 - 2.0 * (vt1 + vt2)
    v1 = ((2.0 + s2) * vt1 + (2.0 - s2) * vt2 - 2.0) / den
    v2 = ((2.0 + s2) * vt2 + (2.0 - s2) * vt1 - 2.0) / den
    eb = np.exp(0.5 * (1.0 - r2))       # see the docstring
    Bt1, Bt2 = -B0 * eb * xt[1], B0 * eb * xt[0]
    B1 = 0.5 * ((s2 + 1.0) * Bt1 - (s2 - 1.0) * Bt2)
    B2 = 0.5 * ((s2 + 1.0) * Bt2 - (s2 - 1.0) * Bt1)
    z = np.zeros_like(rho)
    return np.ascontiguousarray(np.stack([rho, v1, v2, z, p, B1, B2, z]))


# ---- the 3D RMHD isentropic vortex (Sec. 6, 3D RMHD vortex example) --------
def vortex_mesh3(n, t=0.0, R=5.0, amp=0.2):
    """The example's prescribed moving mesh on the periodic box [-R, R]^2 x
    [-5R, 5R] with n x n x 5n distinct nodes (spacing 2R/n): each coordinate
    displaced by amp cos(pi t/4) times the product of sines of the other two,
    sin(3 pi x0_{1,2}/R) and sin(3 pi x0_3/(5R))."""
    x0 = uniform_mesh3((n, n, 5 * n), (-R, -R, -5 * R), (R, R, 5 * R))
    return np.ascontiguousarray(x0 + np.cos(np.pi * t / 4.0) * _vortex3_shape(x0, R, amp))


def vortex_mesh3_velocity(n, t=0.0, R=5.0, amp=0.2):
    """d/dt of vortex_mesh3 at fixed computational coordinates."""
    x0 = uniform_mesh3((n, n, 5 * n), (-R, -R, -5 * R), (R, R, 5 * R))
    return np.ascontiguousarray(-(np.pi / 4.0) * np.sin(np.pi * t / 4.0) * _vortex3_shape(x0, R, amp))


def _vortex3_shape(x0, R, amp):
    s1, s2 = np.sin(3 * np.pi * x0[0] / R), np.sin(3 * np.pi * x0[1] / R)
    s3 = np.sin(3 * np.pi * x0[2] / (5 * R))
    return amp * np.stack([s2 * s3, s3 * s1, s1 * s2])


def _vortex_plane(xt, gamma, sigma, B0):
    """The rotating equilibrium of the vortex frame at the points xt [2][...]:
    (rho, p, vt [2], Bt [2]), with the field B0 exp((1 - r^2)/2)(-x2, x1) (the
    field for which radial balance gives the examples' rotation rate f and
    kappa; see rmhd_vortex)."""
    r2 = xt[0] ** 2 + xt[1] ** 2
    e = np.exp(1.0 - r2)
    rho = (1.0 - sigma * e) ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    kappa = 2.0 * gamma * sigma * rho + (gamma - 1.0) * B0 ** 2 * (2.0 - r2)
    f = np.sqrt(kappa * e / (kappa * r2 * e + (gamma - 1.0) * rho + gamma * p))
    eb = np.exp(0.5 * (1.0 - r2))
    return rho, p, (-xt[1] * f, xt[0] * f), (-B0 * eb * xt[1], B0 * eb * xt[0])


def rmhd_vortex3(x, t=0.0, R=5.0, gamma=5.0 / 3.0, sigma=0.2, B0=0.05):
    """The example's analytic 3D RMHD vortex (primitives [8][...] at the points
    x [3][...] and time t) on the periodic box [-R, R]^2 x [-5R, 5R]: the 2D
    vortex in the plane coordinates xh_k = x_k + (x_1 + x_2 + x_3)/3 + t
    (k = 1, 2), boosted along (1, 1, 1).  Shifts of x by the box's periods move
    xh on the lattice spanned by (8R/3, 2R/3) and (2R/3, 8R/3); the vortex
    frame point xt is the lattice image of xh nearest to the origin."""
    s = (x[0] + x[1] + x[2]) / 3.0 + t
    xh = np.stack([x[0] + s, x[1] + s])
    L = np.array([[8.0 * R / 3.0, 2.0 * R / 3.0], [2.0 * R / 3.0, 8.0 * R / 3.0]])   # columns: lattice
    c = np.floor(np.tensordot(np.linalg.inv(L), xh, axes=1))
    best, bd = None, None
    for a in (-1, 0, 1, 2):
        for b in (-1, 0, 1, 2):
            k = np.stack([c[0] + a, c[1] + b])
            cand = xh - np.tensordot(L, k, axes=1)
            d = cand[0] ** 2 + cand[1] ** 2
            if best is None:
                best, bd = cand, d
            else:
                m = d < bd
                best = np.where(m, cand, best)
                bd = np.where(m, d, bd)
    rho, p, vt, Bt = _vortex_plane(best, gamma, sigma, B0)
    den = 6.0 - 3.0 * (vt[0] + vt[1])
    v = [(4.0 * vt[0] + vt[1] - 3.0) / den, (4.0 * vt[1] + vt[0] - 3.0) / den, (vt[0] + vt[1] - 3.0) / den]
    B = [(5.0 * Bt[0] - Bt[1]) / 3.0, (5.0 * Bt[1] - Bt[0]) / 3.0, -(Bt[0] + Bt[1]) / 3.0]
    return np.ascontiguousarray(np.stack([rho, v[0], v[1], v[2], p, B[0], B[1], B[2]]))


# ---- the paper's 2D RHD Riemann problems I-III (Sec. 6) --------------------
# Initial data on [0,1]^2 split at x_1 = x_2 = 0.5, in the quadrant order of
# quadrant_riemann: q = (x_1 > 0.5) + 2 (x_2 > 0.5), rows (rho, v_1, v_2, p).
# Gamma = 5/3 (the section's default), outflow boundaries, t = 0.4.
RHD_RP_STATES = {
    1: ((3.0, -0.5, 0.5, 5.0), (1.5, -0.5, -0.5, 5.0),        # four contact discontinuities
        (1.0, 0.5, 0.5, 5.0), (0.5, 0.5, -0.5, 5.0)),
    2: ((1.0, -0.3529, -0.3529, 1.0), (0.5771, 0.0, -0.3529, 0.4),   # four rarefactions
        (0.5771, -0.3529, 0.0, 0.4), (1.0, 0.0, 0.0, 1.0)),
    3: ((0.5, 0.0, 0.0, 1.0), (0.1, 0.0, 0.7, 1.0),           # two contacts, two shocks
        (0.1, 0.7, 0.0, 1.0), (0.035145216124503, 0.0, 0.0, 0.162931056509027)),
}


def rhd_rp_config(k, n):
    """Riemann problem k (1, 2 or 3) of Sec. 6 on n x n nodes of [0,1]^2
    (outflow: nodes on both ends)."""
    x = uniform_mesh(n, n, (0.0, 0.0), (1.0, 1.0), (False, False))
    return x, quadrant_riemann(x, np.array(RHD_RP_STATES[k]), split=(0.5, 0.5))


def rmhd_blast2(x, r_in=0.8, r_out=1.0, rho_in=1e-2, p_in=1.0, rho_out=1e-4, p_out=5e-4, Bx=0.1):
    """The 2D RMHD blast of Sec. 6: the explosion zone r < 0.8 (rho = 0.01,
    p = 1), the ambient medium r > 1 (rho = 1e-4, p = 5e-4), a linear taper
    of rho and p in between, at rest, B = (0.1, 0, 0); Gamma = 4/3."""
    r = np.hypot(x[0], x[1])
    s = np.clip((r - r_in) / (r_out - r_in), 0.0, 1.0)       # 0 inside, 1 outside
    rho = rho_in + s * (rho_out - rho_in)
    p = p_in + s * (p_out - p_in)
    z = 0.0 * r
    return np.ascontiguousarray(np.stack([rho, z, z, z, p, Bx + z, z, z]))


def rmhd_blast2_config(n):
    """The 2D RMHD blast on n x n nodes of [-6,6]^2 with outflow boundaries."""
    x = uniform_mesh(n, n, (-6.0, -6.0), (6.0, 6.0), (False, False))
    return x, rmhd_blast2(x)


# ---- the RMHD shock-cloud interactions (Sec. 6) -----------------------------
# The planar shock's states, primitive (rho, v_1, v_2, v_3, p, B_1, B_2, B_3),
# Gamma = 5/3.  The post-shock state is printed as given.  The pre-shock
# state is printed garbled; it is read as rho = 1, v = 0, p = 0.05,
# B = (0, 0.16106, -0.16106).  With that reading the two states satisfy the
# RMHD jump conditions for a single shock speed (0.839) to the printed
# digits; the printed order does not.
SHOCK_CLOUD_POST = (3.86859, 0.68, 0.0, 0.0, 1.25115, 0.0, 0.84981, -0.84981)
SHOCK_CLOUD_PRE = (1.0, 0.0, 0.0, 0.0, 0.05, 0.0, 0.16106, -0.16106)


def rmhd_shock_cloud(x, x_shock=0.05, r_cloud=0.15, rho_cloud=30.0):
    """The shock at x_1 = x_shock moving into the pre-shock medium, which
    holds a cloud of density rho_cloud and radius r_cloud centred at (0.25,
    0.5) (2D, x [2][...]) or (0.25, 0.5, 0.5) (3D, x [3][...]); the cloud
    has the medium's velocity, pressure and field."""
    post, pre = np.array(SHOCK_CLOUD_POST), np.array(SHOCK_CLOUD_PRE)
    shocked = x[0] < x_shock
    prim = np.where(shocked[None], post.reshape((8,) + (1,) * (x.ndim - 1)),
                    pre.reshape((8,) + (1,) * (x.ndim - 1)))
    c = (0.25, 0.5, 0.5)
    r2 = sum((x[d] - c[d]) ** 2 for d in range(x.shape[0]))
    prim[0] = np.where(r2 < r_cloud ** 2, rho_cloud, prim[0])
    return np.ascontiguousarray(prim)


def rmhd_shock_cloud_config(n=(210, 150)):
    """2D shock-cloud on [-0.2,1.2] x [0,1]: inflow of the post-shock state at
    x_1 = -0.2, outflow elsewhere (n nodes per direction, both ends)."""
    x = uniform_mesh(n[0], n[1], (-0.2, 0.0), (1.2, 1.0), (False, False))
    return x, rmhd_shock_cloud(x)


def rmhd_shock_cloud3_config(n=(210, 150, 150)):
    """3D shock-cloud on [-0.2,1.2] x [0,1]^2 with the spherical cloud."""
    x = uniform_mesh3(n, (-0.2, 0.0, 0.0), (1.2, 1.0, 1.0), (False, False, False))
    return x, rmhd_shock_cloud(x)


# ---- the 3D RHD shock-bubble interaction (Sec. 6) ---------------------------
# Primitive (rho, v_1, v_2, v_3, p, B_1, B_2, B_3), Gamma = 5/3: the medium at
# rest ahead of a planar shock at x_1 = 265, the shocked gas behind it moving
# to the left, and a light bubble of radius 25 centred at (215, 0, 0).  The
# 15-digit post-shock state satisfies the RHD jump conditions with the medium
# to rounding (shock speed -0.4148).
SHOCK_BUBBLE_PRE = (1.0, 0.0, 0.0, 0.0, 0.05, 0.0, 0.0, 0.0)
SHOCK_BUBBLE_POST = (1.865225080631180, -0.196781107378299, 0.0, 0.0, 0.15, 0.0, 0.0, 0.0)
SHOCK_BUBBLE_GAS = (0.1358, 0.0, 0.0, 0.0, 0.05, 0.0, 0.0, 0.0)


def rhd_shock_bubble3(x, x_shock=265.0, centre=(215.0, 0.0, 0.0), radius=25.0):
    """The 3D shock-bubble data at the points x [3][...] (an RHD problem, here
    on the RMHD system with B = 0)."""
    pre, post, gas = (np.array(s).reshape((8, 1, 1, 1)) for s in
                      (SHOCK_BUBBLE_PRE, SHOCK_BUBBLE_POST, SHOCK_BUBBLE_GAS))
    prim = np.where((x[0] > x_shock)[None], post, pre)
    r2 = sum((x[d] - centre[d]) ** 2 for d in range(3))
    prim = np.where((r2 <= radius * radius)[None], gas, prim)
    return np.ascontiguousarray(prim)


def rhd_shock_bubble3_config(n=(325, 90, 90)):
    """The 3D shock-bubble on [0,325] x [-45,45]^2 with outflow ends (n nodes
    per direction, both ends): the zero-gradient end at x_1 = 325 keeps the
    uniform post-shock state that the shock leaves behind."""
    x = uniform_mesh3(n, (0.0, -45.0, -45.0), (325.0, 45.0, 45.0), (False, False, False))
    return x, rhd_shock_bubble3(x)


def sphere_rp3(x, r0=0.5):
    """The 3D spherically symmetric Riemann problem of Sec. 6 (an RHD
    problem, here on the RMHD system with B = 0): rho = 10, p = 40/3 for
    r < r0, rho = 1, p = 1e-2 outside, at rest."""
    r2 = x[0] ** 2 + x[1] ** 2 + x[2] ** 2
    z = 0.0 * r2
    inside = r2 < r0 * r0
    return np.ascontiguousarray(np.stack([np.where(inside, 10.0, 1.0), z, z, z,
                                          np.where(inside, 40.0 / 3.0, 1e-2), z, z, z]))
