"""Pins of the oracle's per-element-degree path (Sec. 3.6: p-adaptation with
mortar coupling; the geometry follows the free-stream rules the section
cites) against what the mathematics fixes:

* the mortar operators: interpolation is exact on polynomials of the face
  degree; the projection is the L2 projection (checked against Legendre
  series truncation), reproduces face polynomials and keeps the integral;
* the geometry: the face nodes and face metric terms of two neighbours of
  different degrees are the same polynomial (watertight, one normal);
* the residual: with equal degrees it is the conforming residual (the
  conforming oracle is pinned on its own); with mixed degrees it preserves a
  free stream on curved elements, conserves mass, momentum and energy, and is
  exact where the fluxes are polynomials the elements resolve (a linear
  pressure field on an affine mesh, closed-form du/dt).
"""
import numpy as np
import pytest
from numpy.polynomial import legendre as Lg

import oracle as O
from tests import inputs as I

G = 1.4
PI3 = ((-np.pi,) * 3, (np.pi,) * 3)


# --------------------------------------------------------------------------- mortar operators

@pytest.mark.parametrize("Ns,Nm", [(s, m) for m in range(1, 8) for s in range(1, m + 1)])
def test_mortar_operators(Ns, Nm):
    Pi, P = O.mortar_matrices(Ns, Nm)
    xs, ws = O.lgl(Ns)
    xm, wm = O.lgl(Nm)
    # interpolation reproduces every polynomial of the face degree
    for k in range(Ns + 1):
        assert np.allclose(Pi @ xs ** k, xm ** k, atol=1e-13)
    # projection of x^k (k <= Nm) is its Legendre series truncated at degree Ns
    for k in range(Nm + 1):
        c = Lg.poly2leg(np.eye(k + 1)[k])[:Ns + 1]
        assert np.allclose(P @ xm ** k, Lg.legval(xs, c), atol=1e-13), k
    # it undoes the interpolation, and keeps the integral (w_s^T P = w_m^T)
    assert np.allclose(P @ Pi, np.eye(Ns + 1), atol=1e-13)
    assert np.allclose(ws @ P, wm, atol=1e-14)


def test_mortar_projection_closed_forms():
    # x^2 from degree 2 onto degree 1: the constant 1/3
    _, P = O.mortar_matrices(1, 2)
    assert np.allclose(P @ np.array([1.0, 0.0, 1.0]), [1 / 3, 1 / 3], atol=1e-15)
    # x^3 from degree 3 onto degree 2: (3/5) x at the nodes -1, 0, 1
    x3, _ = O.lgl(3)
    _, P = O.mortar_matrices(2, 3)
    assert np.allclose(P @ x3 ** 3, [-0.6, 0.0, 0.6], atol=1e-15)


# --------------------------------------------------------------------------- geometry

def _face(a, d, end):
    """Face values a[..., k, j, i] at index `end` along d, as [..., tb, ta]."""
    return np.take(a, end, axis=a.ndim - 1 - d)


def test_geometry_rule_and_rejections():
    assert O.PMesh(2, 2, 2, [4, 5, 6, 7, 4, 5, 6, 7], *PI3, amp=0.05).Ngeo == 2
    assert O.PMesh(2, 1, 1, [2, 3], *PI3, amp=0.05).Ngeo == 1
    assert O.PMesh(2, 1, 1, [1, 3], *PI3, amp=0.0).Ngeo == 1
    with pytest.raises(ValueError):
        O.PMesh(2, 1, 1, [1, 3], *PI3, amp=0.05)   # degree 1 with a curved map
    with pytest.raises(ValueError):
        O.PMesh(2, 1, 1, [3, 8], *PI3)


def test_faces_watertight_and_one_normal():
    deg = I.random_degrees(27, seed=5, lo=4, hi=7)
    pm = O.PMesh(3, 3, 3, deg, *PI3, amp=0.08)
    for e in range(pm.E):
        for d in range(3):
            nb = pm.neighbour(e, d, +1)
            NL, NR = int(deg[e]), int(deg[nb])
            lo_side, hi_side = (e, nb) if NL <= NR else (nb, e)
            Nlo, Nhi = min(NL, NR), max(NL, NR)
            Pi, _ = O.mortar_matrices(Nlo, Nhi)
            end_lo = Nlo if lo_side == e else 0
            end_hi = Nhi if hi_side == e else 0
            # node coordinates (periodic images differ by the box length)
            Xl = _face(pm.X(lo_side), d, end_lo)
            Xh = _face(pm.X(hi_side), d, end_hi)
            Xl_on_h = np.einsum("ai,bj,cji->cba", Pi, Pi, Xl)
            dx = Xl_on_h - Xh
            dx -= 2 * np.pi * np.round(dx / (2 * np.pi))
            assert np.abs(dx).max() < 1e-12
            # face metric Ja^d (the scaled normal) from both sides
            Al = _face(pm.Ja(lo_side)[d], d, end_lo)
            Ah = _face(pm.Ja(hi_side)[d], d, end_hi)
            assert np.abs(np.einsum("ai,bj,cji->cba", Pi, Pi, Al) - Ah).max() < 1e-12 * np.abs(Ah).max()


# --------------------------------------------------------------------------- residual

CFGS = [("euler", "lf", "standard"), ("euler", "roe", "ec"), ("euler", "ec", "kg"), ("euler", "matrix", "ir"),
        ("ns", "roe", "standard"), ("ns", "rusanov", "pirozzoli"), ("ns", "ldroe", "ducros"),
        ("ns", "ec", "morinishi")]


@pytest.mark.parametrize("phys,surf,vol", CFGS)
@pytest.mark.parametrize("amp", [0.0, 0.06])
def test_equal_degrees_is_the_conforming_residual(phys, surf, vol, amp):
    N = 4
    pm = O.PMesh(3, 2, 2, [N] * 12, *PI3, amp=amp)
    X = np.stack([pm.X(e) for e in range(pm.E)])
    m = O.Mesh(3, 2, 2, N, *PI3, X=X)
    cfg = O.Cfg(phys, surf, vol, Re=200.0)
    u = I.random_state(m.shape, seed=3, smooth=True)
    r = pm.residual(cfg, u.reshape(-1)).reshape(m.shape)
    ref = m.residual(cfg, u)
    assert np.abs(r - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.allclose(np.stack([pm.J(e) for e in range(pm.E)]), m.J, rtol=1e-14, atol=0)
    if phys == "ns":
        gp = pm.gradients(cfg, u.reshape(-1)).reshape(m.E, 4, 3, N + 1, N + 1, N + 1)
        gr = m.gradients(cfg, u)
        assert np.abs(gp - gr).max() <= 1e-12 * np.abs(gr).max()


def test_equal_degrees_dt_and_step_match_conforming():
    N = 3
    pm = O.PMesh(2, 2, 2, [N] * 8, *PI3)
    m = O.Mesh(2, 2, 2, N, *PI3)
    cfg = O.Cfg("ns", "roe", "ec", Re=400.0)
    u = m.ic_tgv(G, 0.1)
    assert pm.dt(cfg, u.reshape(-1)) == pytest.approx(m.dt(cfg, u), rel=1e-14)
    up, gp = u.reshape(-1).copy(), np.zeros(u.size)
    uc, gc = u.copy(), np.zeros_like(u)
    pm.rk_step(cfg, up, gp)
    m.rk3_step(cfg, uc, gc)
    assert np.abs(up.reshape(m.shape) - uc).max() <= 1e-13 * np.abs(uc).max()


def _constant_state(pm, rho=1.1, v=(0.3, -0.2, 0.1), p=0.9):
    u = pm.empty()
    for e in range(pm.E):
        b = pm.block(u, e)
        b[0] = rho
        for c in range(3):
            b[1 + c] = rho * v[c]
        b[4] = p / (G - 1) + 0.5 * rho * sum(x * x for x in v)
    return u


@pytest.mark.parametrize("phys,surf,vol", CFGS)
def test_free_stream_on_curved_mixed_degrees(phys, surf, vol):
    deg = I.random_degrees(27, seed=11, lo=2, hi=7)
    pm = O.PMesh(3, 3, 3, deg, *PI3, amp=0.08)
    cfg = O.Cfg(phys, surf, vol, Re=100.0)
    r = pm.residual(cfg, _constant_state(pm))
    # rounding grows with the derivative matrices' norm (~n^2) applied twice
    # (metric terms, fluxes): the conforming oracle leaves 2.4e-11 at n = 8 on
    # this box.  A geometry of too high a degree for the faces leaves O(0.1).
    for e in range(pm.E):
        assert np.abs(pm.block(r, e)).max() < 2e-14 * pm.n(e) ** 4, (e, deg[e])


@pytest.mark.parametrize("phys,surf,vol", CFGS)
def test_conservation_on_curved_mixed_degrees(phys, surf, vol):
    deg = I.random_degrees(27, seed=13, lo=2, hi=7)
    pm = O.PMesh(3, 3, 3, deg, *PI3, amp=0.06)
    cfg = O.Cfg(phys, surf, vol, Re=100.0)
    u = I.random_state_blocks(deg, seed=17, smooth=True)
    r = pm.residual(cfg, u)
    tot = pm.integrals(G, u, r)[:5]
    scale = np.zeros(5)
    for e in range(pm.E):
        n = pm.n(e)
        _, w = O.lgl(n - 1)
        W = pm.J(e) * w[None, None, :] * w[None, :, None] * w[:, None, None]
        scale += np.abs(pm.block(r, e) * W).sum(axis=(1, 2, 3))
    assert np.all(np.abs(tot) <= 1e-12 * scale.max())


def test_mortar_flux_is_not_the_lumped_projection():
    """Conservation and free stream alone would also hold for some wrong
    projections; the mixed-degree residual must also be exact on a resolved
    polynomial field (next test), which fails for e.g. a mass-lumped P."""
    Pi, P = O.mortar_matrices(1, 3)
    xs, ws = O.lgl(1)
    xm, wm = O.lgl(3)
    lumped = np.diag(1 / ws) @ Pi.T @ np.diag(wm)
    assert not np.allclose(lumped @ Pi, np.eye(2))
    assert np.allclose(P @ Pi, np.eye(2))


@pytest.mark.parametrize("phys", ["euler", "ns"])
@pytest.mark.parametrize("vol", ["standard", "kg", "pirozzoli"])
@pytest.mark.parametrize("surf", ["lf", "roe", "rusanov", "ldroe", "matrix", "ec"])
def test_linear_pressure_field_is_exact(phys, vol, surf):
    """rho, v constant and p = p0 + a x on an affine mesh: every flux is linear
    in the state's position, so the semi-discrete residual is the exact
       d rho/dt = 0, d(rho v)/dt = -grad p, dE/dt = -gamma/(gamma-1) v.grad p,
    and the viscous terms vanish (v constant, grad T constant).  The field
    jumps across the periodic x boundary, so only elements whose two
    x-neighbours are interior are checked; their faces couple degrees 1..7."""
    ex = 6
    deg = I.random_degrees(ex * 2 * 2, seed=23, lo=1, hi=7)
    pm = O.PMesh(ex, 2, 2, deg, lo=(0.0, 0.0, 0.0), hi=(3.0, 1.0, 1.0), amp=0.0)
    rho, v, p0, a = 1.2, np.array([0.3, -0.2, 0.1]), 1.0, 0.1
    u = pm.empty()
    for e in range(pm.E):
        X = pm.X(e)
        p = p0 + a * X[0]
        b = pm.block(u, e)
        b[0] = rho
        for c in range(3):
            b[1 + c] = rho * v[c]
        b[4] = p / (G - 1) + 0.5 * rho * (v @ v)
    cfg = O.Cfg(phys, surf, vol, Re=50.0)
    r = pm.residual(cfg, u)
    exact = np.array([0.0, -a, 0.0, 0.0, -G / (G - 1) * v[0] * a])
    checked = 0
    for e in range(pm.E):
        ix = e % ex
        if ix in (0, 1, ex - 2, ex - 1):
            continue
        assert np.abs(pm.block(r, e) - exact[:, None, None, None]).max() < 2e-11, (e, deg[e])
        checked += 1
    assert checked == 8
    assert len(set(deg.tolist())) >= 4


def _density_wave_error(lo, hi, surf, vol):
    """Max-norm residual error (relative) on the density wave
    rho = 1 + 0.2 sin(2 pi x/L), v and p constant -- an exact Euler solution
    with du/dt = -(v.grad rho)(1, v, |v|^2/2) -- on a 3^3 mesh whose elements
    draw their degrees from [lo, hi]."""
    v, p, L = np.array([0.4, -0.3, 0.2]), 1.0, 2.0
    deg = I.random_degrees(27, seed=61, lo=lo, hi=hi)
    pm = O.PMesh(3, 3, 3, deg, lo=(0.0, 0.0, 0.0), hi=(L, L, L), amp=0.0)
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
def test_spectral_convergence_across_mortars(surf, vol):
    """The error of mixed-degree meshes falls spectrally as their degree range
    rises, and stays at the level of their lowest degree's uniform mesh: the
    mortars keep the method's accuracy (measured: within 1.5x)."""
    e24, e46, e57 = (_density_wave_error(lo, hi, surf, vol) for lo, hi in ((2, 4), (4, 6), (5, 7)))
    assert e46 < e24 / 10 and e57 < e46 / 3, (e24, e46, e57)
    assert e57 < 1e-2
    assert e46 <= 2 * _density_wave_error(4, 4, surf, vol)
