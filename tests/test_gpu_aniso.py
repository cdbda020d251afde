"""Per-element, per-direction degrees (Sec. 3.6: P_x, P_y, P_z, anisotropic
p-adaptation) with mortars of per-direction degree: the GPU path
(hs3d_pmesh_create3) against the oracle's anisotropic PMesh on the same
seeded inputs, element by element.

FP64 only (the path rejects mixed precision): rel-L2 <= 1e-12 for the
geometry, the residual of every volume form and surface flux (Euler and
Navier-Stokes), the BR1 gradients through the residual, the state after RK
steps with device dt, and the quadrature diagnostics.  Degree maps mix
every degree 1..7 across directions and faces, including faces where neither
side carries the mortar's degrees.
"""
import numpy as np
import pytest

import oracle as O
from tests import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2206_09733_gb300 as hs  # noqa: E402

G = 1.4
TOL64 = 1e-12
PI3 = ((-np.pi,) * 3, (np.pi,) * 3)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2206_09733_gb300 import build
    build.build()
    hs.lib()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def pair(ex, ey, ez, deg3, lo=PI3[0], hi=PI3[1], amp=0.0):
    return (O.PMesh(ex, ey, ez, deg3, lo=lo, hi=hi, amp=amp),
            hs.PMesh(ex, ey, ez, deg3, lo=lo, hi=hi, amp=amp))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def cfgs(physics, surface, volume, precision="fp64", Re=200.0, time="rk3"):
    return (O.Cfg(physics, surface, volume, gamma=G, Re=Re, Pr=0.72, time=time),
            hs.solver_cfg(physics, surface, volume, precision, gamma=G, Re=Re, Pr=0.72, time=time))


def test_layout_is_element_order_and_matches_the_oracle():
    deg = I.random_degree_triples(30, seed=1, lo=1, hi=7)
    om, gm = pair(5, 3, 2, deg)
    assert np.array_equal(gm.offset, om.off)
    sizes = np.diff(gm.offset)
    assert np.array_equal(sizes, 5 * np.prod(deg + 1, axis=1))


@pytest.mark.parametrize("amp,lo_deg", [(0.0, 1), (0.08, 2), (0.08, 4)])
def test_geometry_matches_oracle(amp, lo_deg):
    deg = I.random_degree_triples(27, seed=3, lo=lo_deg, hi=7)
    om, gm = pair(3, 3, 3, deg, amp=amp)
    X, J = (host(t) for t in gm.geometry())
    nodes = int(om.noff[-1])
    assert np.abs(X - om._X).max() < 1e-14 * np.abs(om._X).max()
    assert rel(J, om._J) < TOL64
    assert X.size == 3 * nodes


def test_rejects_mixed_precision_and_bad_degrees():
    deg = I.random_degree_triples(8, seed=5, lo=2, hi=5)
    gm = hs.PMesh(2, 2, 2, deg, *PI3, amp=0.05)
    u = gm.empty_state()
    r = torch.empty_like(u)
    with pytest.raises(hs.HS3DError):
        gm.residual(hs.solver_cfg("euler", "roe", "standard", "mixed32"), u, r)
    bad = deg.copy()
    bad[3, 2] = 8
    with pytest.raises(hs.HS3DError):
        hs.PMesh(2, 2, 2, bad, *PI3)
    one = deg.copy()
    one[0, 1] = 1
    with pytest.raises(hs.HS3DError):
        hs.PMesh(2, 2, 2, one, *PI3, amp=0.05)


MESHES = {
    # curved, degrees 2..7 in every direction
    "curved_2to7": dict(shape=(3, 3, 3), lo=2, hi=7, amp=0.08, seed=11),
    # affine, degrees 1..7 (degree-1 directions allowed on an affine map)
    "affine_1to7": dict(shape=(4, 3, 2), lo=1, hi=7, amp=0.0, seed=12),
    # one element thick in z: its own neighbour across the z faces
    "thin_z": dict(shape=(3, 2, 1), lo=2, hi=5, amp=0.05, seed=13),
}
CASES = [("euler", "lf", "standard"), ("euler", "roe", "ec"), ("euler", "matrix", "ir"), ("euler", "ec", "kg"),
         ("ns", "roe", "standard"), ("ns", "rusanov", "pirozzoli"), ("ns", "ldroe", "ducros"),
         ("ns", "ec", "morinishi"), ("ns", "roe", "ec")]


@pytest.mark.parametrize("mesh", list(MESHES))
@pytest.mark.parametrize("phys,surf,vol", CASES)
def test_residual_fp64(mesh, phys, surf, vol):
    m = MESHES[mesh]
    E = int(np.prod(m["shape"]))
    deg = I.random_degree_triples(E, seed=m["seed"], lo=m["lo"], hi=m["hi"])
    om, gm = pair(*m["shape"], deg, amp=m["amp"])
    oc, gc = cfgs(phys, surf, vol)
    u0 = I.random_state_blocks(deg, seed=21, smooth=True)
    ref = om.residual(oc, u0)
    u = dev(u0)
    r = torch.empty_like(u)
    gm.residual(gc, u, r)
    out = host(r)
    assert rel(out, ref) < TOL64
    # element by element: none off by more than the tolerance of the whole
    scale = np.abs(ref).max()
    assert np.abs(out - ref).max() < 1e-11 * scale


def test_faces_where_neither_side_has_the_mortar_degrees():
    """Two elements along x with tangential degrees (3, 5) and (5, 3): the x
    faces carry a (5, 5) mortar that neither side has (face metric
    interpolated from the minus side)."""
    deg = np.array([[4, 3, 5], [2, 5, 3]], dtype=np.int32)
    om, gm = pair(2, 1, 1, deg, amp=0.06)
    for combo in (("ns", "roe", "ec"), ("euler", "lf", "standard")):
        oc, gc = cfgs(*combo)
        u0 = I.random_state_blocks(deg, seed=5, smooth=True)
        ref = om.residual(oc, u0)
        u = dev(u0)
        r = torch.empty_like(u)
        gm.residual(gc, u, r)
        assert rel(host(r), ref) < TOL64, combo


@pytest.mark.parametrize("phys,surf,vol,time", [("euler", "roe", "standard", "rk3"), ("ns", "lf", "ec", "rk3"),
                                                ("ns", "roe", "kg", "rk4")])
def test_rk_steps_match_oracle(phys, surf, vol, time):
    deg = I.random_degree_triples(27, seed=31, lo=2, hi=6)
    om, gm = pair(3, 3, 3, deg, amp=0.05)
    oc, gc = cfgs(phys, surf, vol, time=time)
    u0 = om.ic_tgv(G, 0.3)
    uo, go = u0.copy(), np.zeros_like(u0)
    dts = [om.rk_step(oc, uo, go) for _ in range(3)]
    u = dev(u0)
    g = torch.zeros_like(u)
    gm.run(gc, u, g, 3)
    t, steps = gm.clock()
    assert steps == 3
    assert abs(t - sum(dts)) < 1e-13 * sum(dts)
    assert rel(host(u), uo) < TOL64


def test_init_state_matches_oracle():
    deg = I.random_degree_triples(27, seed=41, lo=2, hi=7)
    om, gm = pair(3, 3, 3, deg, amp=0.05)
    u = gm.init_state(gm.empty_state(), "tgv", G, 0.1)
    assert rel(host(u), om.ic_tgv(G, 0.1)) < 1e-14
    u = gm.init_state(gm.empty_state(), "vortex", G, 0.5, 5.0, xc=0.3, yc=-0.4)
    assert rel(host(u), om.ic_vortex(G, 0.5, 5.0, xc=0.3, yc=-0.4)) < 1e-14


@pytest.mark.parametrize("with_dudt", [False, True])
def test_diagnostics_match_oracle(with_dudt):
    deg = I.random_degree_triples(27, seed=51, lo=2, hi=6)
    om, gm = pair(3, 3, 3, deg, amp=0.06)
    oc, gc = cfgs("ns", "roe", "ec")
    u0 = I.random_state_blocks(deg, seed=9, smooth=True)
    r0 = om.residual(oc, u0) if with_dudt else None
    ref = om.integrals(G, u0, r0)
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    gm.diagnostics(gc, dev(u0), out, dudt=dev(r0) if with_dudt else None)
    got = host(out)
    scale = np.abs(ref).max()
    assert np.abs(got[:5] - ref[:5]).max() < 1e-12 * scale
    if with_dudt:
        # conservation: the mass, momentum and energy integrals of du/dt vanish
        assert np.abs(got[:5]).max() < 1e-12 * got[6]
        assert abs(got[5] - ref[5]) < 1e-11 * got[6]


def test_free_stream_on_curved_anisotropic_degrees():
    deg = I.random_degree_triples(27, seed=61, lo=2, hi=7)
    _, gm = pair(3, 3, 3, deg, amp=0.08)
    rho, v, p = 1.1, (0.3, -0.2, 0.1), 0.9
    u = np.zeros(gm.size)
    for e in range(27):
        b = gm.block(u, e)
        b[0] = rho
        for c in range(3):
            b[1 + c] = rho * v[c]
        b[4] = p / (G - 1) + 0.5 * rho * sum(x * x for x in v)
    for combo in (("ns", "roe", "ec"), ("euler", "matrix", "standard")):
        _, gc = cfgs(*combo)
        r = torch.empty(gm.size, dtype=torch.float64, device="cuda")
        gm.residual(gc, dev(u), r)
        assert np.abs(host(r)).max() < 2e-14 * 8 ** 4, combo


def test_isotropic_triples_take_the_bucketed_path():
    deg = I.random_degrees(12, seed=71, lo=2, hi=6)
    g1 = hs.PMesh(3, 2, 2, deg, *PI3, amp=0.05)
    g3 = hs.PMesh(3, 2, 2, np.repeat(deg[:, None], 3, axis=1), *PI3, amp=0.05)
    assert np.array_equal(g1.offset, g3.offset)   # the degree-grouped layout
    _, gc = cfgs("ns", "roe", "ec")
    u = g1.init_state(g1.empty_state(), "tgv", G, 0.1)
    r1, r3 = torch.zeros_like(u), torch.zeros_like(u)   # (the gaps between degree groups stay untouched)
    g1.residual(gc, u, r1)
    g3.residual(gc, u, r3)
    assert torch.equal(r1, r3)


def test_run_continuation_equals_one_run():
    deg = I.random_degree_triples(27, seed=81, lo=2, hi=5)
    _, gm = pair(3, 3, 3, deg, amp=0.05)
    _, gc = cfgs("ns", "roe", "ec")
    u0 = gm.init_state(gm.empty_state(), "tgv", G, 0.2)
    a, ga = u0.clone(), torch.zeros_like(u0)
    gm.clock(reset=True)
    gm.run(gc, a, ga, 4)
    b, gb = u0.clone(), torch.zeros_like(u0)
    gm.clock(reset=True)
    gm.run(gc, b, gb, 2)
    gm.run(gc, b, gb, 2, dt=-1.0)
    assert torch.equal(a, b)
