"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check compares the oracle with something other than itself: values the paper
prints (tests/golden), hand evaluations of Eqs. (12)-(20), Gauss-Hermite moments of
the Maxwellian (Eq. 5), a 40-digit linear solve, exact invariants (conservation,
relaxation factor, symmetries), the exact Riemann solution, the sound speed
sqrt(gamma T), the Taylor-Green decay rate (Eqs. 22-23) and the Chapman-Enskog
stress (Eq. 21).  A dropped term, a wrong sign or index or a transposed operand
anywhere in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import exact
import oracle
from paper_2502_16818_gb300 import workloads as W


def model_of(w, **kw):
    d = dict(nx=w.nx, ny=w.ny, dx=w.dx, dy=w.dy, dt=w.dt, tau=w.tau, I=w.I, vg=w.vg, eg=w.eg,
             bc_x=w.bc_x, bc_y=w.bc_y)
    d.update(kw)
    return oracle.Model(**d)


def init_of(m, w):
    return oracle.init(m, w.rho, w.ux, w.uy, w.T)


VSETS = [("sod", W.VSET_SOD), ("lax", W.VSET_LAX), ("sound", W.VSET_SOUND), ("tgv", W.VSET_TGV),
         ("shock", W.VSET_SHOCK)]


def one_cell_model(vset, I):
    return oracle.Model(nx=1, ny=1, dx=1.0, dy=1.0, dt=1e-5, tau=1e-4, I=I, vg=vset[0], eg=vset[1])


# ------------------------------------------------------------------ Eqs. (2)-(3)

def test_velocity_set_eq2(golden):
    rows = golden("velocity_set_eq2.txt")
    vx, vy, eta = oracle.velocity_set((1.0, 1.0, 1.0, 1.0), (0.1, 0.2, 0.3, 0.4))
    for r in rows:
        i = int(r[0]) - 1
        assert vx[i] == float(r[1]) and vy[i] == float(r[2])
        assert eta[i] == {"a": 0.1, "b": 0.2, "c": 0.3, "d": 0.4}[r[3]]
    # group speeds scale each group (Eq. 2)
    vx, vy, _ = oracle.velocity_set((2.0, 3.0, 5.0, 7.0), (0, 0, 0, 0))
    for g, s in enumerate((2.0, 3.0, 5.0, 7.0)):
        assert np.all(np.maximum(np.abs(vx[4 * g:4 * g + 4]), np.abs(vy[4 * g:4 * g + 4])) == s)


# ---------------------------------------------------------------------- Eq. (5)

@pytest.mark.parametrize("I", [0.0, 1.0, 3.0, 2.5])
@pytest.mark.parametrize("T", [0.8, 1.7])
def test_central_moments_match_quadrature(I, T):
    rho = 1.3
    fbar = oracle.central_moments_eq(I, rho, T)
    for k, (lab, phi) in enumerate(exact.moment_rows()):
        ref = exact.maxwellian_moment(phi, I, rho, 0.0, 0.0, T, central=True)
        assert abs(fbar[k] - ref) <= 1e-13 * (1 + abs(ref)), (lab, fbar[k], ref)


# ------------------------------------------------------------------ Eqs. (6)-(7)

@pytest.mark.parametrize("name,vset", VSETS)
@pytest.mark.parametrize("I", [0.0, 3.0])
def test_feq_reproduces_maxwellian_moments(name, vset, I):
    """sum_i f_eq,i Psi_k is the Maxwellian moment of Eq. (5), both in the lab frame
    (raw) and in the comoving frame (central), for all 16 rows of Eq. (6)."""
    m = one_cell_model(vset, I)
    vx, vy, eta = oracle.velocity_set(*vset)
    rng = np.random.default_rng(7)
    for _ in range(4):
        rho = rng.uniform(0.2, 2.0)
        ux, uy = rng.uniform(-0.4, 0.4, 2)
        T = rng.uniform(0.5, 2.0)
        f = oracle.feq(m, rho, ux, uy, T)
        for central in (False, True):
            ax, ay = (vx - ux, vy - uy) if central else (vx, vy)
            for lab, phi in exact.moment_rows():
                terms = f * phi(ax, ay, eta)
                got = terms.sum()
                ref = exact.maxwellian_moment(phi, I, rho, ux, uy, T, central=central)
                scale = np.abs(terms).sum() + abs(ref)
                assert abs(got - ref) <= 1e-12 * scale, (name, lab, central, got, ref)


@pytest.mark.parametrize("name,vset", VSETS)
def test_solve_against_40_digit_solution(name, vset):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    vx, vy, eta = oracle.velocity_set(*vset)
    for ux, uy, T in [(0.0, 0.0, 1.0), (0.31, -0.12, 0.8), (0.7, 0.05, 7.9)]:
        M = oracle.central_matrix(vx, vy, eta, ux, uy)
        b = oracle.central_moments_eq(3.0, 1.0, T)
        x = oracle.solve(M, b)
        ref = np.array([float(v) for v in mpmath.lu_solve(mpmath.matrix(M.tolist()),
                                                          mpmath.matrix(b.tolist()))])
        assert np.max(np.abs(x - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_central_matrix_columns_are_monomials_of_peculiar_velocity():
    """Column i of M(u) equals the Eq. (6) monomials at v_i - u (pins the row order
    and the shift by u)."""
    vx, vy, eta = oracle.velocity_set(*W.VSET_TGV)
    M = oracle.central_matrix(vx, vy, eta, 0.13, -0.07)
    for k, (lab, phi) in enumerate(exact.moment_rows()):
        np.testing.assert_allclose(M[k], phi(vx - 0.13, vy + 0.07, eta), rtol=1e-14, atol=1e-14)


# ------------------------------------------------------------------ macroscopics

@pytest.mark.parametrize("name,vset", VSETS[:4])
def test_macros_of_single_velocity(name, vset):
    """A distribution concentrated on one velocity has rho = f_i, u = v_i and
    T = eta_i^2 / (D + I) (Eq. 4 conserved rows)."""
    I = 1.0
    m = one_cell_model(vset, I)
    vx, vy, eta = oracle.velocity_set(*vset)
    for i in range(16):
        f = np.zeros(16)
        f[i] = 0.7
        r, u, v, T = oracle.cell_macros(m, f)
        assert r == 0.7
        assert abs(u - vx[i]) < 1e-15 and abs(v - vy[i]) < 1e-15
        assert abs(T - eta[i] ** 2 / (2 + I)) < 1e-15


@pytest.mark.parametrize("name,vset", VSETS[:4])
def test_macros_of_equilibrium_roundtrip(name, vset):
    m = one_cell_model(vset, 3.0)
    f = oracle.feq(m, 0.9, 0.2, -0.1, 1.3)
    r, u, v, T = oracle.cell_macros(m, f)
    assert abs(r - 0.9) < 1e-14 and abs(u - 0.2) < 1e-13 and abs(v + 0.1) < 1e-13
    assert abs(T - 1.3) < 1e-13


@pytest.mark.parametrize("name,vset", VSETS)
def test_collision_conserves_mass_momentum_energy(name, vset):
    """sum_i (f_i - f_i^eq) {1, v_i, v_i^2 + eta_i^2} = 0 (Sec. 2, after Eq. 7)."""
    I = 1.0
    m = one_cell_model(vset, I)
    vx, vy, eta = oracle.velocity_set(*vset)
    rng = np.random.default_rng(3)
    for _ in range(10):
        f = rng.uniform(0.01, 0.2, 16)
        r, u, v, T = oracle.cell_macros(m, f)
        d = f - oracle.feq(m, r, u, v, T)
        for psi in (np.ones(16), vx, vy, vx ** 2 + vy ** 2 + eta ** 2):
            assert abs(np.dot(d, psi)) <= 1e-13 * np.dot(np.abs(f), np.abs(psi))


# ------------------------------------------------------------------ Eqs. (12)-(20)

def test_minmod_eq16(golden):
    for X, Y, out in golden("minmod_eq16.txt"):
        assert oracle.minmod(float(X), float(Y)) == float(out), (X, Y)


def test_nnd_hand_evaluations(golden):
    for r in golden("nnd_eq12_20.txt"):
        v, dr = float(r[0]), float(r[1])
        fs = [float(a) for a in r[2:7]]
        assert oracle.nnd_derivative(v, fs, dr) == pytest.approx(float(r[7]), abs=1e-15)


def test_nnd_exact_on_linear_data():
    rng = np.random.default_rng(5)
    for _ in range(20):
        a, b, v, dr = rng.normal(), rng.normal(), rng.normal() * 3, rng.uniform(0.1, 2)
        fs = a + b * np.arange(-2, 3) * dr
        assert oracle.nnd_derivative(v, fs, dr) == pytest.approx(v * b, rel=1e-12, abs=1e-12)


def _collisionless(w, **kw):
    return model_of(w, tau=1e300, **kw)


def test_advection_is_tvd_per_velocity():
    """Collision off (tau -> infinity): every f_i is advected on its own by the NND
    scheme with two-stage TVD Runge-Kutta, so its total variation never grows."""
    n = 64
    w = W.sound(n=n, ny=1, I=1.0, dt=2e-3, tau=1.0)
    x = (np.arange(n) + 0.5) / n
    w.rho = np.where((x > 0.3) & (x < 0.55), 1.5, 1.0).reshape(1, n)
    m = _collisionless(w)
    f = init_of(m, w)
    tv = lambda g: np.abs(np.diff(np.concatenate([g, g[:1]]))).sum()
    for s in range(40):
        g = oracle.step(m, f, 1)
        for i in range(16):
            assert tv(g[i, 0]) <= tv(f[i, 0]) * (1 + 1e-13) + 1e-15
        f = g


def test_advection_second_order_on_smooth_data():
    """Smooth periodic advection of each f_i at its own speed: L1 error against the
    shifted exact profile falls at second order (minmod clips only at extrema)."""
    errs = []
    for n in (64, 128, 256):
        w = W.sound(n=n, ny=1, I=1.0, dt=0.2 / n / 2.2, tau=1.0, amp=0.3)
        m = _collisionless(w)
        f0 = init_of(m, w)
        steps = n // 4
        f = oracle.step(m, f0, steps)
        t = steps * w.dt
        vx, _, _ = oracle.velocity_set(w.vg, w.eg)
        x = (np.arange(n) + 0.5) / n
        wts = oracle.feq(m, 1.0, 0.0, 0.0, 1.0)     # at u = 0, f_eq is rho times these
        e = 0.0
        for i in range(16):
            ref = wts[i] * (1.0 + 0.3 * np.sin(2 * np.pi * (x - vx[i] * t)))
            e += np.abs(f[i, 0] - ref).mean()
        errs.append(e)
    order = math.log(errs[1] / errs[2], 2)
    assert order > 1.7, errs
    assert math.log(errs[0] / errs[1], 2) > 1.5, errs


# ------------------------------------------------------------------ Eq. (1) + RK

@pytest.mark.parametrize("rk", [0, 1])
def test_pure_relaxation_factor(rk):
    """Spatially uniform f with f - f_eq orthogonal to the conserved rows: the flux
    vanishes exactly and f - f_eq shrinks by 1 - h + h^2/2 per step, h = dt/tau."""
    vset = W.VSET_TGV
    vx, vy, eta = oracle.velocity_set(*vset)
    C = np.stack([np.ones(16), vx, vy, vx ** 2 + vy ** 2 + eta ** 2])
    rng = np.random.default_rng(11)
    r = rng.normal(size=16)
    delta = r - C.T @ np.linalg.solve(C @ C.T, C @ r)
    m1 = one_cell_model(vset, 3.0)
    feq = oracle.feq(m1, 1.1, 0.05, -0.02, 0.9)
    h = 0.37
    m = oracle.Model(nx=3, ny=2, dx=1.0, dy=1.0, dt=h * 1e-3, tau=1e-3, I=3.0, vg=vset[0],
                     eg=vset[1], rk=rk)
    f0 = np.broadcast_to((feq + 0.01 * delta)[:, None, None], (16, 2, 3)).copy()
    n = 25
    f = oracle.step(m, f0, n)
    expect = feq + 0.01 * delta * (1 - h + h * h / 2) ** n
    np.testing.assert_allclose(f, np.broadcast_to(expect[:, None, None], f.shape), rtol=0,
                               atol=5e-14 * np.abs(feq).max())


def test_uniform_equilibrium_is_fixed_point():
    w = W.random_smooth(6, 5, seed=1)
    m = model_of(w)
    f0 = oracle.init(m, 0.8, 0.1, -0.05, 1.2)
    f = oracle.step(m, f0, 50)
    np.testing.assert_allclose(f, f0, rtol=0, atol=1e-13 * np.abs(f0).max())


@pytest.mark.parametrize("rk", [0, 1])
def test_global_conservation_periodic(rk):
    """Periodic box: the NND flux telescopes and the collision conserves, so total
    mass, momentum and energy stay fixed."""
    w = W.random_blocks(24, 20, seed=2, dt=4e-4, tau=1e-3)
    m = model_of(w, rk=rk)
    f = init_of(m, w)
    s0 = oracle.conserved_sums(m, f)
    f = oracle.step(m, f, 200)
    s1 = oracle.conserved_sums(m, f)
    scale = np.array([abs(s0[0]), abs(s0[0]) * 2.2, abs(s0[0]) * 2.2, abs(s0[3])])
    assert np.all(np.abs(s1 - s0) <= 1e-12 * scale), (s0, s1)


# symmetry maps of the velocity set (Eq. 2 ordering)
MIRROR_X = [2, 1, 0, 3, 5, 4, 7, 6, 10, 9, 8, 11, 13, 12, 15, 14]
TRANSPOSE = [1, 0, 3, 2, 4, 7, 6, 5, 9, 8, 11, 10, 12, 15, 14, 13]


def test_symmetry_maps_are_symmetries_of_velocity_set():
    vx, vy, eta = oracle.velocity_set(*W.VSET_TGV)
    assert np.array_equal(vx[MIRROR_X], -vx) and np.array_equal(vy[MIRROR_X], vy)
    assert np.array_equal(vx[TRANSPOSE], vy) and np.array_equal(vy[TRANSPOSE], vx)
    assert np.array_equal(eta[MIRROR_X], eta) and np.array_equal(eta[TRANSPOSE], eta)


def test_mirror_symmetry():
    w = W.random_blocks(20, 6, seed=4, dt=4e-4, tau=1e-3, bc=(W.ZERO_GRADIENT, W.PERIODIC))
    m = model_of(w)
    f = oracle.step(m, init_of(m, w), 30)
    w2 = W.random_blocks(20, 6, seed=4, dt=4e-4, tau=1e-3, bc=(W.ZERO_GRADIENT, W.PERIODIC))
    w2.rho, w2.ux, w2.uy, w2.T = (w.rho[:, ::-1].copy(), -w.ux[:, ::-1].copy(),
                                  w.uy[:, ::-1].copy(), w.T[:, ::-1].copy())
    g = oracle.step(m, init_of(m, w2), 30)
    np.testing.assert_allclose(g, f[MIRROR_X][:, :, ::-1], rtol=0, atol=1e-13 * np.abs(f).max())


def test_transpose_symmetry():
    w = W.random_blocks(12, 12, seed=6, dt=4e-4, tau=1e-3)
    m = model_of(w)
    f = oracle.step(m, init_of(m, w), 20)
    w2 = W.random_blocks(12, 12, seed=6, dt=4e-4, tau=1e-3)
    w2.rho, w2.ux, w2.uy, w2.T = w.rho.T.copy(), w.uy.T.copy(), w.ux.T.copy(), w.T.T.copy()
    g = oracle.step(m, init_of(m, w2), 20)
    np.testing.assert_allclose(g, f[TRANSPOSE].transpose(0, 2, 1), rtol=0,
                               atol=1e-13 * np.abs(f).max())


def test_one_row_equals_identical_rows():
    w = W.sod(nx=40, steps=50, dt=1e-4, tau=1e-4)
    m1 = model_of(w)
    f1 = oracle.step(m1, init_of(m1, w), 50)
    m4 = model_of(w, ny=4)
    f4 = oracle.step(m4, oracle.init(m4, np.repeat(w.rho, 4, 0), np.repeat(w.ux, 4, 0),
                                     np.repeat(w.uy, 4, 0), np.repeat(w.T, 4, 0)), 50)
    for r in range(4):
        assert np.array_equal(f4[:, r], f1[:, 0])


# ------------------------------------------------------------------ Sec. 3 physics

def test_exact_references_reproduce_paper_shock_state(golden):
    """The Ma = 15 state printed in Sec. 3.3 satisfies the Rankine-Hugoniot
    relations (gamma = 1.4) and P = rho T."""
    left, right = [[float(v) for v in r] for r in golden("ma15_post_shock.txt")]
    rho2, u2, p2, _ = exact.rankine_hugoniot(15.0, 1.4, right[0], right[4])
    assert rho2 == pytest.approx(left[0], abs=1e-4)
    assert u2 == pytest.approx(left[1], abs=1e-4)
    assert p2 == pytest.approx(left[4], abs=1e-4)
    assert left[0] * left[3] == pytest.approx(left[4], rel=1e-5)


def _riemann_l1(w, steps):
    m = model_of(w)
    f = oracle.step(m, init_of(m, w), steps)
    rho, ux, uy, T = oracle.macros(m, f)
    t = steps * w.dt
    g = W.gamma_of(w.I)
    L, R = w.extra["left"], w.extra["right"]
    ex = exact.RiemannExact((L[0], L[1], L[0] * L[2]), (R[0], R[1], R[0] * R[2]), g)
    x = w.extra["x_lo"] + (np.arange(w.nx) + 0.5) * w.dx
    ref = ex.sample((x - w.extra["x_interface"]) / t)
    l1 = np.abs(rho[0] - ref[0]).mean() * (w.extra["x_hi"] - w.extra["x_lo"])
    return l1, rho[0], ref, ex, x, t


@pytest.mark.slow
def test_sod_against_exact_riemann():
    """Sod tube (Sec. 3.1), I = 0 so gamma = 2: density approaches the exact Riemann
    solution, and the error falls with the grid."""
    errs = []
    for nx in (100, 200):
        w = W.sod(nx=nx, I=0.0, dt=5e-5 * 100 / nx, tau=5e-5)
        steps = int(round(0.2 / w.dt))
        l1, rho, ref, ex, x, t = _riemann_l1(w, steps)
        errs.append(l1)
    assert errs[1] < 0.012 and errs[1] < errs[0] * 0.8, errs
    # plateau between contact and shock within 2%
    xs = ex.u_star * t + 0.5
    plateau = (x > xs + 0.04) & (x < xs + 0.08)
    assert np.all(np.abs(rho[plateau] - ref[0][plateau]) < 0.02 * ref[0][plateau])


@pytest.mark.slow
def test_lax_against_exact_riemann_gamma_14():
    """Lax tube (Sec. 3.2) with I = 3, gamma = 1.4 as in the paper."""
    w = W.lax(nx=200, I=3.0, dt=5e-5, tau=1e-4)
    l1, rho, ref, ex, x, t = _riemann_l1(w, int(round(0.2 / w.dt)))
    assert l1 < 0.05, l1
    # shock position: the last point above the mid-density between plateau and right
    # state lies within 3 cells of the exact shock
    rho_mid = 0.5 * (ref[0].max() + 0.5)
    i_num = np.nonzero(rho > rho_mid)[0].max()
    i_ref = np.nonzero(ref[0] > rho_mid)[0].max()
    assert abs(i_num - i_ref) <= 3


def _sound_frequency(n, ny, I, tau=2e-4, dt=2e-4):
    w = W.sound(n=n, ny=ny, I=I, dt=dt, tau=tau)
    m = model_of(w)
    f = init_of(m, w)
    x = (np.arange(n) + 0.5) / n
    if ny == 1:
        basis = np.cos(2 * np.pi * x)[None, :]
    else:
        y = (np.arange(ny) + 0.5) / ny
        basis = np.outer(np.sin(2 * np.pi * y), np.cos(2 * np.pi * x))
    kmag = 2 * np.pi * (1 if ny == 1 else math.sqrt(2))
    omega_guess = math.sqrt(W.gamma_of(I)) * kmag
    steps = int(1.3 * 2 * math.pi / omega_guess / dt) + 2
    amps = [0.0]
    for s in range(steps):
        f = oracle.step(m, f, 1)
        ux = oracle.macros(m, f)[1]
        amps.append(float((ux * basis).sum()))
    a = np.array(amps)
    t = np.arange(len(a)) * dt
    zc = [t[i] - a[i] * dt / (a[i + 1] - a[i]) for i in range(1, len(a) - 1)
          if a[i] != 0 and np.sign(a[i]) != np.sign(a[i + 1])]
    return math.pi / (zc[1] - zc[0]), omega_guess


@pytest.mark.parametrize("I", [0.0, 1.0, 3.0])
def test_sound_speed_1d(I):
    """Standing acoustic mode: the velocity oscillates at omega = sqrt(gamma T) k,
    gamma = (D + I + 2)/(D + I) (Sec. 2 after Eq. 5)."""
    om, om_ref = _sound_frequency(128, 1, I)
    assert abs(om / om_ref - 1) < 2e-3, (om, om_ref)


@pytest.mark.parametrize("axis", ["x", "y"])
def test_sound_speed_anisotropic_cells(axis):
    """A 1-D standing wave along one axis of a grid whose cells are 7 times longer in
    the other direction: the frequency depends only on the spacing along the wave."""
    n, I, dt, tau = 96, 1.0, 2.5e-4, 2.5e-4
    w = W.sound(n=n, ny=1, I=I, dt=dt, tau=tau)
    if axis == "x":
        m = model_of(w, ny=2, dy=7.0 / n)
        fields = [np.repeat(a, 2, axis=0) for a in (w.rho, w.ux, w.uy, w.T)]
    else:
        m = model_of(w, nx=2, ny=n, dx=7.0 / n, dy=1.0 / n)
        fields = [np.repeat(a.reshape(n, 1), 2, axis=1) for a in (w.rho, w.ux, w.uy, w.T)]
    f = oracle.init(m, *fields)
    x = (np.arange(n) + 0.5) / n
    om_ref = math.sqrt(W.gamma_of(I)) * 2 * np.pi
    steps = int(1.3 * 2 * math.pi / om_ref / dt) + 2
    amps = [0.0]
    for _ in range(steps):
        f = oracle.step(m, f, 1)
        _, ux, uy, _ = oracle.macros(m, f)
        u = ux[0] if axis == "x" else uy[:, 0]
        amps.append(float((u * np.cos(2 * np.pi * x)).sum()))
    a = np.array(amps)
    zc = [(i - a[i] / (a[i + 1] - a[i])) * dt for i in range(1, len(a) - 1)
          if a[i] != 0 and np.sign(a[i]) != np.sign(a[i + 1])]
    om = math.pi / (zc[1] - zc[0])
    assert abs(om / om_ref - 1) < 3e-3, (axis, om, om_ref)


@pytest.mark.slow
def test_sound_speed_2d():
    om, om_ref = _sound_frequency(32, 32, 3.0, tau=4e-4, dt=4e-4)
    assert abs(om / om_ref - 1) < 5e-3, (om, om_ref)


def _tgv_rate_ratio(n, dt):
    w = W.taylor_green(n=n, I=3.0, dt=dt, tau=5e-4)
    m = model_of(w)
    f = init_of(m, w)
    k = w.extra["k"]
    X, Y = np.meshgrid((np.arange(n) + 0.5) * w.dx, (np.arange(n) + 0.5) * w.dx, indexing="xy")
    basis = np.sin(k * X) * np.cos(k * Y)
    a0 = (oracle.macros(m, f)[1] * basis).sum()
    steps = int(round(0.05 / dt))
    f = oracle.step(m, f, steps)
    rho, ux, uy, T = oracle.macros(m, f)
    rate = -math.log((ux * basis).sum() / a0) / (steps * w.dt)
    return rate / (2 * T.mean() * w.tau * k * k)


@pytest.mark.slow
def test_taylor_green_decay_rate():
    """Velocity amplitude decays as exp(-2 nu k^2 t) with nu = T tau (Eqs. 22-23 and
    the viscosity of Sec. 2); the scheme's own dissipation vanishes at second order."""
    r48 = _tgv_rate_ratio(48, 2e-4)
    r96 = _tgv_rate_ratio(96, 1e-4)
    assert abs(r96 - 1) < 0.03, (r48, r96)
    assert math.log(abs(r48 - 1) / abs(r96 - 1), 2) > 1.5, (r48, r96)


@pytest.mark.slow
def test_taylor_green_l2_slope_near_paper(golden):
    """Sec. 3.5: the relative L2 error of u_x (Eq. 25) against the analytic vortex
    falls with dx at about the slope the paper prints (loose pin)."""
    slope_paper = float(dict((r[0], r[1]) for r in golden("paper_numbers.txt"))["tgv_l2_slope"])
    errs, dxs = [], []
    t_end = 0.05
    for n in (20, 30, 40):
        w = W.taylor_green(n=n, I=3.0, dt=1e-4, tau=5e-4)
        m = model_of(w)
        steps = int(round(t_end / w.dt))
        f = oracle.step(m, init_of(m, w), steps)
        rho, ux, uy, T = oracle.macros(m, f)
        X, Y = np.meshgrid((np.arange(n) + 0.5) * w.dx, (np.arange(n) + 0.5) * w.dx, indexing="xy")
        uref, _ = exact.taylor_green_velocity(X, Y, steps * w.dt, w.extra["U0"], w.extra["k"],
                                              T.mean() * w.tau)
        errs.append(math.sqrt(np.mean(((ux - uref) / w.extra["U0"]) ** 2)))
        dxs.append(w.dx)
    slope = np.polyfit(np.log(dxs), np.log(errs), 1)[0]
    assert abs(slope - slope_paper) < 0.45, (slope, errs)


# ------------------------------------------------------------------ Eqs. (8)-(11), (21)

def test_tne_zero_at_equilibrium_and_trace_identity():
    w = W.random_blocks(16, 8, seed=9, dt=4e-4, tau=1e-3)
    m = model_of(w, I=2.0)
    f = oracle.step(m, init_of(m, w), 5)
    d = oracle.tne(m, f)
    # trace: Delta2_xx + Delta2_yy = -sum (f - f_eq) eta^2 (energy row is conserved)
    _, _, eta = oracle.velocity_set(w.vg, w.eg)
    rho, ux, uy, T = oracle.macros(m, f)
    for (y, x) in [(0, 0), (3, 5), (7, 15), (4, 9)]:
        fe = oracle.feq(m, rho[y, x], ux[y, x], uy[y, x], T[y, x])
        rhs = -np.dot(f[:, y, x] - fe, eta ** 2)
        assert d[0, y, x] + d[2, y, x] == pytest.approx(rhs, abs=1e-13)
    f0 = init_of(m, w)
    assert np.abs(oracle.tne(m, f0)).max() < 1e-12


def test_tne_brute_force_cell():
    """Each Delta* row is sum_i (f_i - f_eq,i) Psi_k(v_i - u), Eqs. (8)-(11)."""
    m = one_cell_model(W.VSET_LAX, 1.0)
    rng = np.random.default_rng(12)
    f = rng.uniform(0.02, 0.1, 16)
    r, u, v, T = oracle.cell_macros(m, f)
    fe = oracle.feq(m, r, u, v, T)
    vx, vy, eta = oracle.velocity_set(*W.VSET_LAX)
    d = oracle.tne(m, f.reshape(16, 1, 1))[:, 0, 0]
    rows = exact.moment_rows()[4:]
    for k, (lab, phi) in enumerate(rows):
        assert d[k] == pytest.approx(np.dot(f - fe, phi(vx - u, vy - v, eta)), rel=1e-14, abs=1e-14)


def test_tne_matches_chapman_enskog_eq21():
    """In a smooth compression the second-order TNE follows Eq. (21):
    Delta2_xx = 2 rho T tau ((1 - D - I)/(D + I) du_x/dx + 1/(D + I) du_y/dy)."""
    n, I = 128, 3.0
    w = W.sound(n=n, ny=1, I=I, dt=5e-4, tau=1e-3, amp=1e-2)
    m = model_of(w)
    steps = int(0.25 / math.sqrt(W.gamma_of(I)) / w.dt)    # a quarter period
    f = oracle.step(m, init_of(m, w), steps)
    rho, ux, uy, T = oracle.macros(m, f)
    d = oracle.tne(m, f)
    dudx = (np.roll(ux[0], -1) - np.roll(ux[0], 1)) / (2 * w.dx)
    K = 2.0 + I
    ce = 2 * rho[0] * T[0] * w.tau * (1 - K) / K * dudx
    err = np.sqrt(np.mean((d[0, 0] - ce) ** 2)) / np.sqrt(np.mean(ce ** 2))
    assert err < 0.1, err
