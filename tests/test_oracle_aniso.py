"""Pins of the oracle's anisotropic path (Sec. 3.6: the polynomial order may
differ per element and per direction, P_x, P_y, P_z, with mortars between
faces whose tangential degrees differ) against what the mathematics fixes:

* the geometry: the face nodes and face metric terms of two neighbours are
  one polynomial on the mortar, whatever their tangential degree pairs
  (including faces where neither side has the mortar's degrees);
* the residual: a free stream is preserved on curved elements; mass,
  momentum and energy are conserved; a linear pressure field along each
  direction is exact on an affine mesh (closed-form du/dt); a field that
  varies along x only converges spectrally in P_x and is blind to P_y, P_z;
* the BR1 gradients of polynomial velocities are exact in each direction up
  to that direction's degree;
* the time step is the closed form on a uniform state and an affine box.
"""
import numpy as np
import pytest

import oracle as O
from tests import inputs as I

G = 1.4
PI3 = ((-np.pi,) * 3, (np.pi,) * 3)

CFGS = [("euler", "lf", "standard"), ("euler", "roe", "ec"), ("euler", "ec", "kg"), ("euler", "matrix", "ir"),
        ("ns", "roe", "standard"), ("ns", "rusanov", "pirozzoli"), ("ns", "ldroe", "ducros"),
        ("ns", "ec", "morinishi")]


def _face(a, d, end):
    """Face values a[..., k, j, i] at index `end` along d, as [..., tb, ta]."""
    return np.take(a, end, axis=a.ndim - 1 - d)


def _tangential(d):
    return (1, 2) if d == 0 else (0, 2) if d == 1 else (0, 1)


def _to_mortar(f, S, M):
    """Face field f[..., tb, ta] of tangential degrees S = (S0, S1) onto the
    mortar of degrees M (interpolation, each direction its own pair)."""
    P0, _ = O.mortar_matrices(S[0], M[0])
    P1, _ = O.mortar_matrices(S[1], M[1])
    return np.einsum("ai,bj,...ji->...ba", P0, P1, f)


def _constant_state(pm, rho=1.1, v=(0.3, -0.2, 0.1), p=0.9):
    u = pm.empty()
    for e in range(pm.E):
        b = pm.block(u, e)
        b[0] = rho
        for c in range(3):
            b[1 + c] = rho * v[c]
        b[4] = p / (G - 1) + 0.5 * rho * sum(x * x for x in v)
    return u


def _mesh(shape, deg, amp, lo=PI3[0], hi=PI3[1]):
    return O.PMesh(*shape, deg, lo=lo, hi=hi, amp=amp)


# --------------------------------------------------------------------------- geometry

def test_triples_of_equal_degrees_are_the_isotropic_mesh():
    deg = I.random_degrees(12, seed=3, lo=2, hi=6)
    a = _mesh((3, 2, 2), deg, 0.06)
    b = _mesh((3, 2, 2), np.repeat(deg[:, None], 3, axis=1), 0.06)
    cfg = O.Cfg("ns", "roe", "ec", Re=200.0)
    u = I.random_state_blocks(deg, seed=5, smooth=True)
    assert np.array_equal(a.residual(cfg, u), b.residual(cfg, u))
    assert a.dt(cfg, u) == b.dt(cfg, u)


def test_geometry_rule_and_rejections():
    assert _mesh((2, 1, 1), [[4, 5, 6], [6, 4, 5]], 0.05).Ngeo == 2
    assert _mesh((2, 1, 1), [[2, 5, 6], [6, 4, 5]], 0.05).Ngeo == 1
    with pytest.raises(ValueError):
        _mesh((2, 1, 1), [[1, 3, 3], [3, 3, 3]], 0.05)   # degree 1 in one direction with a curved map
    with pytest.raises(ValueError):
        _mesh((2, 1, 1), [[3, 3, 8], [3, 3, 3]], 0.0)


def test_faces_watertight_and_one_normal():
    deg = I.random_degree_triples(27, seed=5, lo=4, hi=7)
    pm = _mesh((3, 3, 3), deg, 0.08)
    crossed = 0
    for e in range(pm.E):
        for d in range(3):
            nb = pm.neighbour(e, d, +1)
            t0, t1 = _tangential(d)
            SL, SR = (deg[e][t0], deg[e][t1]), (deg[nb][t0], deg[nb][t1])
            M = (max(SL[0], SR[0]), max(SL[1], SR[1]))
            crossed += M != SL and M != SR
            XL = _to_mortar(_face(pm.X(e), d, deg[e][d]), SL, M)
            XR = _to_mortar(_face(pm.X(nb), d, 0), SR, M)
            dx = XL - XR
            dx -= 2 * np.pi * np.round(dx / (2 * np.pi))
            assert np.abs(dx).max() < 1e-12
            AL = _to_mortar(_face(pm.Ja(e)[d], d, deg[e][d]), SL, M)
            AR = _to_mortar(_face(pm.Ja(nb)[d], d, 0), SR, M)
            # (rounding of the degree-7 curl-form differences: ~1e-12 where a
            # metric component is zero, the same order as the conforming
            # oracle's own free-stream residue)
            assert np.abs(AL - AR).max() < 4e-12 * np.abs(AR).max()
    assert crossed > 5   # faces where neither side carries the mortar's degrees


# --------------------------------------------------------------------------- residual

@pytest.mark.parametrize("phys,surf,vol", CFGS)
def test_free_stream_on_curved_anisotropic_degrees(phys, surf, vol):
    deg = I.random_degree_triples(27, seed=11, lo=2, hi=7)
    pm = _mesh((3, 3, 3), deg, 0.08)
    cfg = O.Cfg(phys, surf, vol, Re=100.0)
    r = pm.residual(cfg, _constant_state(pm))
    for e in range(pm.E):
        assert np.abs(pm.block(r, e)).max() < 2e-14 * max(pm.shape3(e)) ** 4, (e, deg[e])


@pytest.mark.parametrize("phys,surf,vol", CFGS)
def test_conservation_on_curved_anisotropic_degrees(phys, surf, vol):
    deg = I.random_degree_triples(27, seed=13, lo=2, hi=7)
    pm = _mesh((3, 3, 3), deg, 0.06)
    cfg = O.Cfg(phys, surf, vol, Re=100.0)
    u = I.random_state_blocks(deg, seed=17, smooth=True)
    r = pm.residual(cfg, u)
    tot = pm.integrals(G, u, r)[:5]
    scale = np.zeros(5)
    for e in range(pm.E):
        w = [O.lgl(int(p))[1] for p in deg[e]]
        W = pm.J(e) * w[0][None, None, :] * w[1][None, :, None] * w[2][:, None, None]
        scale += np.abs(pm.block(r, e) * W).sum(axis=(1, 2, 3))
    assert np.all(np.abs(tot) <= 1e-12 * scale.max())


@pytest.mark.parametrize("d", [0, 1, 2])
@pytest.mark.parametrize("phys,vol,surf", [("euler", "standard", "roe"), ("ns", "kg", "lf"),
                                           ("euler", "pirozzoli", "matrix"), ("ns", "standard", "ec")])
def test_linear_pressure_field_along_each_direction_is_exact(d, phys, vol, surf):
    """rho, v constant and p = p0 + a x_d on an affine mesh elongated along d:
    every flux is linear, so the residual is the exact
       d rho/dt = 0, d(rho v)/dt = -grad p, dE/dt = -gamma/(gamma-1) v.grad p.
    The field jumps across the periodic boundary normal to d: only elements
    two away from it are checked.  Degrees 1..7 in every direction.  The
    bar is the rounding floor of the same mesh: twice what a constant state
    (a = 0, exact residual 0) leaves in each element (up to ~6e-11 where
    degree-7 lifting meets degree-1 neighbours)."""
    shape = [2, 2, 2]
    shape[d] = 6
    E = 24
    deg = I.random_degree_triples(E, seed=23 + d, lo=1, hi=7)
    hi = [1.0, 1.0, 1.0]
    hi[d] = 3.0
    pm = _mesh(shape, deg, 0.0, lo=(0.0, 0.0, 0.0), hi=tuple(hi))
    rho, v, p0, a = 1.2, np.array([0.3, -0.2, 0.1]), 1.0, 0.1

    def state(a):
        u = pm.empty()
        for e in range(E):
            p = p0 + a * pm.X(e)[d]
            b = pm.block(u, e)
            b[0] = rho
            for c in range(3):
                b[1 + c] = rho * v[c]
            b[4] = p / (G - 1) + 0.5 * rho * (v @ v)
        return u

    cfg = O.Cfg(phys, surf, vol, Re=50.0)
    r = pm.residual(cfg, state(a))
    r0 = pm.residual(cfg, state(0.0))
    exact = np.zeros(5)
    exact[1 + d] = -a
    exact[4] = -G / (G - 1) * v[d] * a
    checked = 0
    for e in range(E):
        ab = (e % shape[0], (e // shape[0]) % shape[1], e // (shape[0] * shape[1]))
        if ab[d] in (0, 1, 4, 5):
            continue
        floor = np.abs(pm.block(r0, e)).max()
        assert floor < 1e-10
        assert np.abs(pm.block(r, e) - exact[:, None, None, None]).max() < 2 * floor + 1e-12, (e, deg[e])
        checked += 1
    assert checked == 8


def _x_wave_error(deg, surf="roe", vol="standard"):
    """Max-norm residual error (relative) on the density wave
    rho = 1 + 0.2 sin(2 pi x/L), v and p constant -- an exact Euler solution,
    du/dt = -(v.grad rho)(1, v, |v|^2/2) -- on a 3^3 affine mesh."""
    v, p, L = np.array([0.4, -0.3, 0.2]), 1.0, 2.0
    pm = _mesh((3, 3, 3), deg, 0.0, lo=(0.0, 0.0, 0.0), hi=(L, L, L))
    u, exact = pm.empty(), pm.empty()
    for e in range(pm.E):
        ph = 2 * np.pi * pm.X(e)[0] / L
        rho = 1 + 0.2 * np.sin(ph)
        vgr = 0.2 * np.cos(ph) * 2 * np.pi / L * v[0]
        b, x = pm.block(u, e), pm.block(exact, e)
        b[0] = rho
        x[0] = -vgr
        for c in range(3):
            b[1 + c] = rho * v[c]
            x[1 + c] = -vgr * v[c]
        b[4] = p / (G - 1) + 0.5 * rho * (v @ v)
        x[4] = -vgr * 0.5 * (v @ v)
    r = pm.residual(O.Cfg("euler", surf, vol), u)
    return np.abs(r - exact).max() / np.abs(exact).max()


@pytest.mark.parametrize("surf,vol", [("roe", "standard"), ("lf", "kg"), ("ec", "ec")])
def test_wave_along_x_converges_in_px_and_ignores_py_pz(surf, vol):
    """The wave is constant along y and z, which degree 1 represents exactly:
    (P_x, 1, 1) gives the error of (P_x, P_x, P_x) (the nodes along x are the
    same), and the error falls spectrally with P_x alone."""
    E = 27
    err = {}
    for px in (3, 5, 7):
        err[px] = _x_wave_error(np.tile([px, 1, 1], (E, 1)), surf, vol)
        iso = _x_wave_error(np.full(E, px), surf, vol)
        # (the two residuals differ by rounding only: the isotropic residual itself
        # varies along y and z by up to 4.5e-10 at P = 7, against a max|du/dt| of
        # 0.26 -- 2e-9 in these relative-error units; a 1-ulp change of the state
        # moves it by 4e-13)
        assert err[px] == pytest.approx(iso, rel=1e-6, abs=5e-9)
    assert err[5] < err[3] / 5 and err[7] < err[5] / 5, err   # (measured: 9.6x to 130x per step)
    # transverse degrees that differ between neighbours (mortars on the x faces)
    # change nothing either
    deg = np.column_stack([np.full(E, 5), I.random_degrees(E, seed=3, lo=1, hi=4), I.random_degrees(E, seed=4, lo=1, hi=4)])
    assert _x_wave_error(deg, surf, vol) == pytest.approx(err[5], rel=1e-6, abs=5e-9)


def test_br1_gradient_is_exact_per_direction():
    """v = (x^2, y, 0), rho and p constant: the conserved variables are
    polynomials of degree (4, 2, 0) along (x, y, z) (E carries |v|^2) and
    q = (v, T) of degree (2, 1, 0).  Elements with P_x >= 4, P_y >= 2,
    P_z >= 1 resolve them, every mortar interpolates the traces exactly and
    both sides agree, so the BR1 lift vanishes and grad q is exact -- on the
    elements away from the periodic boundaries, where the field jumps."""
    shape = (5, 5, 5)
    E = 125
    rng = np.random.default_rng(9)
    deg = np.column_stack([rng.integers(4, 8, E), rng.integers(2, 6, E), rng.integers(1, 4, E)]).astype(np.int32)
    pm = _mesh(shape, deg, 0.0, lo=(0.0, 0.0, 0.0), hi=(2.5, 2.5, 2.5))
    rho, p = 1.1, 0.8
    u = pm.empty()
    for e in range(E):
        X = pm.X(e)
        v = [X[0] ** 2, X[1], 0.0 * X[2]]
        b = pm.block(u, e)
        b[0] = rho
        for c in range(3):
            b[1 + c] = rho * v[c]
        b[4] = p / (G - 1) + 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
    grad = pm.gradients(O.Cfg("ns", "roe", "standard"), u)
    checked = 0
    for e in range(E):
        ab = (e % 5, (e // 5) % 5, e // 25)
        if min(ab) == 0 or max(ab) == 4:
            continue
        nx, ny, nz = pm.shape3(e)
        g = grad[12 * pm.noff[e]:12 * pm.noff[e + 1]].reshape(4, 3, nz, ny, nx)
        X = pm.X(e)
        exact = np.zeros((4, 3, nz, ny, nx))
        exact[0, 0] = 2 * X[0]
        exact[1, 1] = 1.0
        assert np.abs(g - exact).max() < 1e-11 * np.abs(exact).max(), (e, deg[e])
        checked += 1
    assert checked == 27
    # a degree too low for the field in one direction breaks it: with P_x = 3
    # and 5 alternating along y, the y faces (x tangential) interpolate E's
    # degree-3 interpolant of x^4, which is not the degree-5 one
    deg[:, 0] = [3 if ((e // 5) % 5) % 2 == 0 else 5 for e in range(E)]
    pm = _mesh(shape, deg, 0.0, lo=(0.0, 0.0, 0.0), hi=(2.5, 2.5, 2.5))
    u = pm.empty()
    for e in range(E):
        X = pm.X(e)
        b = pm.block(u, e)
        b[0] = rho
        b[1] = rho * X[0] ** 2
        b[2] = rho * X[1]
        b[3] = 0.0
        b[4] = p / (G - 1) + 0.5 * rho * (X[0] ** 4 + X[1] ** 2)
    grad = pm.gradients(O.Cfg("ns", "roe", "standard"), u)
    e = 62   # the centre element
    nx, ny, nz = pm.shape3(e)
    g = grad[12 * pm.noff[e]:12 * pm.noff[e + 1]].reshape(4, 3, nz, ny, nx)
    assert np.abs(g[3]).max() > 1e-6   # T is no longer constant on the mortars


def test_dt_closed_form_on_an_affine_box():
    """Uniform state on an affine box: Ja^d/J = (2/h_d) e_d, so
    dt = cfl 8 / max_e sum_d n_d^2 (|v_d| + c) 2/h_d  (and the viscous bound
    12 / max_e (mu/rho) sum_d n_d^4 (2/h_d)^2 when smaller)."""
    shape, L = (3, 2, 2), np.array([3.0, 1.0, 2.0])
    deg = I.random_degree_triples(12, seed=31, lo=1, hi=7)
    pm = _mesh(shape, deg, 0.0, lo=(0.0, 0.0, 0.0), hi=tuple(L))
    rho, v, p = 1.2, np.array([0.3, -0.5, 0.1]), 0.9
    u = _constant_state(pm, rho, v, p)
    c = np.sqrt(G * p / rho)
    s = 2.0 / (L / np.array(shape))
    n = deg + 1.0
    cfg = O.Cfg("euler", "lf", "standard", cfl=0.5)
    lam = max(((n[e] ** 2) * (np.abs(v) + c) * s).sum() for e in range(12))
    assert pm.dt(cfg, u) == pytest.approx(0.5 * 8 / lam, rel=1e-13)
    cfg = O.Cfg("ns", "lf", "standard", cfl=0.5, Re=0.05)
    mu = 1 / 0.05
    lamv = max((mu / rho) * ((n[e] ** 4) * s ** 2).sum() for e in range(12))
    assert pm.dt(cfg, u) == pytest.approx(min(0.5 * 8 / lam, 12 / lamv), rel=1e-13)
    assert 12 / lamv < 0.5 * 8 / lam


def test_step_conserves_and_stays_finite_on_anisotropic_tgv():
    deg = I.random_degree_triples(27, seed=41, lo=2, hi=5)
    pm = _mesh((3, 3, 3), deg, 0.05)
    cfg = O.Cfg("ns", "roe", "ec", Re=400.0)
    u = pm.ic_tgv(G, 0.1)
    g = np.zeros_like(u)
    m0 = pm.integrals(G, u)[:5]
    for _ in range(3):
        pm.rk_step(cfg, u, g)
    m1 = pm.integrals(G, u)[:5]
    assert np.all(np.isfinite(u))
    assert abs(m1[0] - m0[0]) < 1e-13 * abs(m0[0]) and abs(m1[4] - m0[4]) < 1e-13 * abs(m0[4])
