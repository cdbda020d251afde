"""Gauss-Legendre solution nodes on the GPU against the oracle (needs a GPU).

Geometry at the Gauss points (metric polynomials of the Gauss-Lobatto map),
the residual with interpolated face traces for every physics and surface
flux (standard volume term), free stream, the rejection of split forms, the
dt rule, time stepping with both integrators, the batched server and the
quadrature diagnostics."""
import numpy as np
import pytest

import oracle as O
from tests.inputs import random_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2206_09733_gb300 as hs  # noqa: E402

TOL64 = 1e-12
G = 1.4


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2206_09733_gb300 import build
    build.build()
    hs.lib()


def pair(ex, ey, ez, N, lo=(-np.pi,) * 3, hi=(np.pi,) * 3, amp=0.0):
    return (O.Mesh(ex, ey, ez, N, lo=lo, hi=hi, amp=amp, nodes="gauss"),
            hs.Mesh(ex, ey, ez, N, lo=lo, hi=hi, amp=amp, nodes="gauss"))


def cfgs(physics, surface, precision="fp64", Re=400.0, cfl=0.5, time="rk3"):
    return (O.Cfg(physics, surface, "standard", gamma=G, Re=Re, Pr=0.72, cfl=cfl, time=time),
            hs.solver_cfg(physics, surface, "standard", precision, gamma=G, Re=Re, Pr=0.72, cfl=cfl, time=time))


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_gauss_geometry_matches_oracle(N):
    om, gm = pair(3, 2, 2, N, amp=0.1)
    X, Ja, J = (host(t) for t in gm.geometry())
    assert rel(X, om.X) < 1e-14
    assert rel(J, om.J) < TOL64
    assert rel(Ja, om.Ja) < TOL64


SURFACES = ("lf", "roe", "ec", "rusanov", "ldroe", "matrix")


@pytest.mark.parametrize("physics", ["euler", "ns"])
@pytest.mark.parametrize("surface", SURFACES)
def test_gauss_residual_parity(physics, surface):
    # smooth states: on Gauss nodes the face traces are extrapolations, which
    # turn node-wise random states non-physical (see the test below)
    om, gm = pair(3, 4, 2, 3, amp=0.1)
    u0 = random_state(om.shape, seed=13, smooth=True)
    oc, gc = cfgs(physics, surface)
    ref = om.residual(oc, u0)
    u = dev(u0)
    r = torch.empty_like(u)
    gm.residual(gc, u, r)
    out = host(r)
    assert rel(out, ref) < TOL64
    assert np.abs(out - ref).max() < 1e-11 * np.abs(ref).max()


def test_gauss_rough_state_gives_the_same_nonphysical_traces():
    """Node-wise random states extrapolate to negative pressures at some
    Gauss faces, outside the method's domain: the oracle produces
    non-finite values on the lines of those faces.  Where both results are
    finite they agree; the kernels' non-finite nodes lie inside the oracle's
    (NaN propagation differs in detail: fmax ignores a NaN operand)."""
    om, gm = pair(3, 4, 2, 3, amp=0.1)
    u0 = random_state(om.shape, seed=13)
    oc, gc = cfgs("euler", "lf")
    ref = om.residual(oc, u0)
    u = dev(u0)
    r = torch.empty_like(u)
    gm.residual(gc, u, r)
    out = host(r)
    bad = ~np.isfinite(ref)
    bad_gpu = ~np.isfinite(out)
    assert bad.any()
    assert not (bad_gpu & ~bad).any()
    ok = ~bad & ~bad_gpu
    assert rel(out[ok], ref[ok]) < TOL64


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("combo", [("ns", "roe"), ("euler", "lf"), ("ns", "matrix")])
def test_gauss_residual_parity_every_degree(N, combo):
    om, gm = pair(2, 3, 2, N, amp=0.08)
    u0 = random_state(om.shape, seed=200 + N, smooth=True)
    oc, gc = cfgs(*combo)
    ref = om.residual(oc, u0)
    u = dev(u0)
    r = torch.empty_like(u)
    gm.residual(gc, u, r)
    assert rel(host(r), ref) < TOL64


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 1, 3)])
def test_gauss_degenerate_meshes(shape):
    om, gm = pair(*shape, 3, amp=0.05)
    u0 = random_state(om.shape, seed=17, smooth=True)
    for combo in (("ns", "roe"), ("euler", "ec")):
        oc, gc = cfgs(*combo)
        ref = om.residual(oc, u0)
        u = dev(u0)
        r = torch.empty_like(u)
        gm.residual(gc, u, r)
        assert rel(host(r), ref) < TOL64, combo


def test_gauss_free_stream_and_mixed_precision():
    om, gm = pair(4, 4, 4, 4, amp=0.1)
    st = np.array([1.2, 0.36, -0.24, 0.12, 2.6])
    u0 = np.broadcast_to(st[None, :, None, None, None], gm.shape).copy()
    for surface in SURFACES:
        for physics in ("euler", "ns"):
            _, gc = cfgs(physics, surface)
            u = dev(u0)
            r = torch.empty_like(u)
            gm.residual(gc, u, r)
            assert np.abs(host(r)).max() < 1e-12, (surface, physics)
    # mixed precision on a smooth state
    u0 = random_state(om.shape, seed=19, smooth=True)
    for surface in SURFACES:
        oc, gc = cfgs("ns", surface, precision="mixed32")
        ref = om.residual(oc, u0)
        u = dev(u0)
        r = torch.empty_like(u)
        gm.residual(gc, u, r)
        assert rel(host(r), ref) < 2e-5, surface


def test_gauss_tensor_core_precision_computes_as_mixed32():
    """On Gauss-Legendre meshes the tensor-core precision selects the same
    kernels as MIXED32 (its contraction exists for Gauss-Lobatto nodes only):
    bitwise equal residuals and steps."""
    _, gm = pair(3, 3, 2, 3, amp=0.05)
    u0 = gm.init_state(gm.empty_state(), "tgv", G, 0.3)
    out = []
    for prec in ("mixed_tc", "mixed32"):
        gc = hs.solver_cfg("ns", "roe", "standard", prec, gamma=G, Re=200.0)
        r = torch.empty_like(u0)
        gm.residual(gc, u0, r)
        u, g = u0.clone(), torch.zeros_like(u0)
        gm.rk3_run(gc, u, g, 2)
        out.append((r, u))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


def test_gauss_rejects_split_forms():
    _, gm = pair(2, 2, 2, 2)
    u = gm.init_state(gm.empty_state(), "tgv", G, 0.1)
    r = torch.empty_like(u)
    with pytest.raises(hs.HS3DError) as ei:
        gm.residual(hs.solver_cfg("euler", "roe", "ec"), u, r)
    assert ei.value.status == hs.ERR_UNSUPPORTED


def test_gauss_dt_matches_oracle():
    om, gm = pair(4, 4, 4, 3, amp=0.05)
    oc, gc = cfgs("ns", "roe", Re=100.0)
    u0 = om.ic_tgv(G, 0.3)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    gm.dt(gc, dev(u0), out)
    ref = om.dt(oc, u0)
    assert abs(host(out)[0] - ref) < 1e-13 * ref


@pytest.mark.parametrize("time", ["rk3", "rk4"])
def test_gauss_vortex_steps_parity(time):
    om, gm = pair(4, 4, 2, 3, lo=(0,) * 3, hi=(10, 10, 5), amp=0.05)
    oc, gc = cfgs("euler", "roe", cfl=0.5, time=time)
    uo = om.ic_vortex(G, 0.5, 5.0)
    go = np.zeros_like(uo)
    t = 0.0
    for _ in range(10):
        t += om.dt(oc, uo)
        om.rk3_step(oc, uo, go)
    u = gm.init_state(gm.empty_state(), "vortex", G, 0.5, 5.0)
    g = torch.zeros_like(u)
    gm.clock(reset=True)
    gm.rk3_run(gc, u, g, 10)
    assert rel(host(u), uo) < TOL64
    ts, steps = gm.clock()
    assert steps == 10 and abs(ts - t) < 1e-13 * t
    # stepwise equals the graph replay
    u2 = gm.init_state(gm.empty_state(), "vortex", G, 0.5, 5.0)
    g2 = torch.zeros_like(u2)
    for _ in range(10):
        gm.rk3_step(gc, u2, g2)
    assert torch.equal(u, u2)


def test_gauss_tgv_ns_steps_parity_and_mixed():
    om, gm = pair(6, 6, 6, 3, amp=0.05)
    oc, gc = cfgs("ns", "roe", Re=1600.0)
    uo = om.ic_tgv(G, 0.1)
    go = np.zeros_like(uo)
    for _ in range(5):
        om.rk3_step(oc, uo, go)
    for prec, bar in (("fp64", TOL64), ("mixed32", 1e-5)):
        _, gc = cfgs("ns", "roe", precision=prec, Re=1600.0)
        u = gm.init_state(gm.empty_state(), "tgv", G, 0.1)
        g = torch.zeros_like(u)
        gm.rk3_run(gc, u, g, 5)
        assert rel(host(u), uo) < bar, prec


def test_gauss_diagnostics_and_conservation():
    om, gm = pair(4, 4, 4, 4, amp=0.08)
    oc, gc = cfgs("ns", "lf", Re=200.0)
    u0 = om.ic_tgv(G, 0.3)
    ref_r = om.residual(oc, u0)
    ref = om.integrals(G, u0, ref_r)
    u = dev(u0)
    r = torch.empty_like(u)
    gm.residual(gc, u, r)
    out = torch.empty(7, dtype=torch.float64, device="cuda")
    gm.diagnostics(gc, u, out, dudt=r)
    d = host(out)
    mag = om.integrals(G, u0, np.abs(ref_r))[:5]
    assert (np.abs(d[:5]) < 1e-12 * mag).all()            # discrete conservation on Gauss nodes
    assert abs(d[5] - ref[5]) < 1e-9 * ref[6]


def test_gauss_requests_in_the_server():
    """A Gauss-node request beside a Lobatto one: each matches the oracle."""
    srv = hs.Server()
    E, N, n_steps = 4, 3, 5
    tickets, outs = [], []
    for nodes in ("gauss", "lobatto"):
        mesh = hs.mesh_desc(E, E, 1, N, lo=(0, 0, 0), hi=(10, 10, 10.0 / E), nodes=nodes)
        cfg = hs.solver_cfg("euler", "roe", "standard", "fp64", cfl=0.5)
        ic = hs.ic_desc("vortex", G, 0.4, 2.0, 5.0, 5.0)
        out = np.zeros((E * E, 5, N + 1, N + 1, N + 1))
        tickets.append(srv.submit(mesh, cfg, ic, n_steps=n_steps, result=out))
        outs.append(out)
    import time
    t0 = time.time()
    done = {}
    while len(done) < len(tickets):
        for t in tickets:
            if t not in done:
                st, res = srv.poll(t)
                if st != hs.PENDING:
                    done[t] = (st, res)
        assert time.time() - t0 < 60
        time.sleep(0.002)
    for nodes, t, a in zip(("gauss", "lobatto"), tickets, outs):
        assert done[t][0] == hs.OK
        om = O.Mesh(E, E, 1, N, lo=(0, 0, 0), hi=(10, 10, 10.0 / E), nodes=nodes)
        oc = O.Cfg("euler", "roe", "standard", cfl=0.5)
        u = om.ic_vortex(G, 0.4, 2.0, xc=5.0, yc=5.0)
        g = np.zeros_like(u)
        for _ in range(n_steps):
            om.rk3_step(oc, u, g)
        assert rel(a, u) < TOL64, nodes
    srv.close()
