"""Continuous-batching server through the C-ABI (needs a GPU).

Checks: a request's result is the same alone and in a mix (bitwise: every
element's arithmetic depends only on its own request), results match the
oracle, admission under a budget smaller than the total footprint queues
requests and still completes them, and the failure paths (oversize request,
bad descriptor, injected allocation failure, non-physical state) fail the
request, not the server."""
import os
import subprocess
import sys
import time

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2206_09733_gb300 as hs  # noqa: E402

G = 1.4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2206_09733_gb300 import build
    build.build()
    hs.lib()
    torch.cuda.init()


def wait_all(srv, tickets, limit_s=120.0):
    t0 = time.time()
    out = {}
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            st, res = srv.poll(t)
            if st != hs.PENDING:
                out[t] = (st, res)
        assert time.time() - t0 < limit_s, "server did not finish in time"
        time.sleep(0.002)
    return out


def vortex_request(E, N, xc, yc, beta, Ma, precision="mixed32", volume="ec", time="rk3"):
    mesh = hs.mesh_desc(E, E, 1, N, lo=(0, 0, 0), hi=(10, 10, 10.0 / E))
    cfg = hs.solver_cfg("euler", "lf", volume, precision, cfl=0.5, time=time)
    ic = hs.ic_desc("vortex", G, Ma, beta, xc, yc)
    return mesh, cfg, ic


def test_result_same_alone_and_in_mix_and_matches_oracle():
    specs = [(4, 3, 3.1, 6.2, 2.0, 0.3), (5, 2, 7.0, 2.5, 4.0, 0.6), (3, 4, 5.0, 5.0, 1.5, 0.2),
             (4, 3, 2.0, 8.0, 3.0, 0.5), (6, 5, 6.5, 4.5, 2.5, 0.4)]
    n_steps = 6
    # alone: one at a time
    alone = []
    srv = hs.Server()
    for sp in specs:
        mesh, cfg, ic = vortex_request(*sp, precision="fp64")
        out = np.zeros((sp[0] * sp[0], 5, sp[1] + 1, sp[1] + 1, sp[1] + 1))
        t = srv.submit(mesh, cfg, ic, n_steps=n_steps, result=out)
        (st, res), = wait_all(srv, [t]).values()
        assert st == hs.OK and res.steps == n_steps
        alone.append(out)
    # mixed: all at once, plus unrelated traffic of other sizes
    outs, tickets = [], []
    for sp in specs:
        mesh, cfg, ic = vortex_request(*sp, precision="fp64")
        out = np.zeros_like(alone[len(outs)])
        tickets.append(srv.submit(mesh, cfg, ic, n_steps=n_steps, result=out))
        outs.append(out)
        m2, c2, i2 = vortex_request(4, sp[1], 5.0, 5.0, 1.0, 0.3, precision="fp64")
        srv.submit(m2, c2, i2, n_steps=3)
    res = wait_all(srv, tickets)
    for t, a, b in zip(tickets, alone, outs):
        assert res[t][0] == hs.OK
        assert np.array_equal(a, b)           # bitwise alone vs in the mix
    # and each matches the oracle
    for sp, a in zip(specs, alone):
        E, N, xc, yc, beta, Ma = sp
        om = O.Mesh(E, E, 1, N, lo=(0, 0, 0), hi=(10, 10, 10.0 / E))
        oc = O.Cfg("euler", "lf", "ec", cfl=0.5)
        u = om.ic_vortex(G, Ma, beta, xc=xc, yc=yc)
        g = np.zeros_like(u)
        for _ in range(n_steps):
            om.rk3_step(oc, u, g)
        assert np.linalg.norm(a - u) / np.linalg.norm(u) < 1e-12
    srv.close()


def test_mixed_schemes_share_the_server_and_match_the_oracle():
    """Requests with different split forms and time integrators run side by
    side (each group in its own launches) and each matches the oracle."""
    specs = [("ec", "rk4"), ("kg", "rk3"), ("pirozzoli", "rk4"), ("ducros", "rk3"), ("kg", "rk4")]
    E, N, n_steps = 4, 3, 5
    srv = hs.Server()
    tickets, outs = [], []
    for volume, time_ in specs:
        mesh, cfg, ic = vortex_request(E, N, 5.0, 5.0, 2.0, 0.4, precision="fp64", volume=volume, time=time_)
        out = np.zeros((E * E, 5, N + 1, N + 1, N + 1))
        tickets.append(srv.submit(mesh, cfg, ic, n_steps=n_steps, result=out))
        outs.append(out)
    res = wait_all(srv, tickets)
    for (volume, time_), t, a in zip(specs, tickets, outs):
        assert res[t][0] == hs.OK and res[t][1].steps == n_steps
        om = O.Mesh(E, E, 1, N, lo=(0, 0, 0), hi=(10, 10, 10.0 / E))
        oc = O.Cfg("euler", "lf", volume, cfl=0.5, time=time_)
        u = om.ic_vortex(G, 0.4, 2.0, xc=5.0, yc=5.0)
        g = np.zeros_like(u)
        for _ in range(n_steps):
            om.rk3_step(oc, u, g)
        assert np.linalg.norm(a - u) / np.linalg.norm(u) < 1e-12, (volume, time_)
    srv.close()


def test_mixed_and_tensor_core_requests_equal_single_solves():
    """Mixed-precision requests (MIXED32, and MIXED_TC which runs the same
    kernels) in one server give bitwise the states of the same solves stepped alone through
    hs3d_rk3_run (the server's captured step graph replayed across steps)."""
    # pairs of requests with the same order and scheme share their launches (item tables)
    specs = [(4, 3, "mixed_tc", "standard"), (3, 3, "mixed_tc", "standard"), (3, 4, "mixed_tc", "standard"),
             (4, 3, "mixed32", "ec"), (5, 3, "mixed32", "ec"), (5, 2, "mixed32", "standard")]
    n_steps = 5
    srv = hs.Server()
    tickets, outs = [], []
    for E, N, prec, volume in specs:
        mesh, cfg, ic = vortex_request(E, N, 4.0, 6.0, 2.0, 0.4, precision=prec, volume=volume)
        out = np.zeros((E * E, 5, N + 1, N + 1, N + 1))
        tickets.append(srv.submit(mesh, cfg, ic, n_steps=n_steps, result=out))
        outs.append(out)
    res = wait_all(srv, tickets)
    srv.close()
    for (E, N, prec, volume), t, a in zip(specs, tickets, outs):
        assert res[t][0] == hs.OK and res[t][1].steps == n_steps
        gm = hs.Mesh(E, E, 1, N, lo=(0, 0, 0), hi=(10, 10, 10.0 / E))
        u = gm.init_state(gm.empty_state(), "vortex", G, 0.4, 2.0, 4.0, 6.0)
        g = torch.zeros_like(u)
        gm.rk3_run(hs.solver_cfg("euler", "lf", volume, prec, cfl=0.5), u, g, n_steps)
        torch.cuda.synchronize()
        assert np.array_equal(a, u.cpu().numpy()), (E, N, prec, volume)


def test_t_final_is_hit_exactly():
    srv = hs.Server()
    mesh, cfg, ic = vortex_request(4, 3, 5.0, 5.0, 2.0, 0.4)
    t = srv.submit(mesh, cfg, ic, t_final=0.37)
    (st, res), = wait_all(srv, [t]).values()
    assert st == hs.OK and res.t_sim == 0.37 and res.steps > 1
    srv.close()


def test_admission_under_a_small_budget_queues_and_completes():
    # each request below needs ~1-3 MB; a 6 MB budget admits only a few at a time
    srv = hs.Server(hbm_budget_bytes=6 * 1024 * 1024)
    tickets = []
    for k in range(12):
        mesh, cfg, ic = vortex_request(4 + k % 3, 3, 5.0, 5.0, 2.0, 0.3)
        tickets.append(srv.submit(mesh, cfg, ic, n_steps=5))
    peak_running = 0
    t0 = time.time()
    while srv.stats()["finished"] < len(tickets):
        peak_running = max(peak_running, srv.stats()["running"])
        assert srv.stats()["bytes_in_use"] <= 6 * 1024 * 1024
        assert time.time() - t0 < 120
        time.sleep(0.001)
    res = wait_all(srv, tickets)
    assert all(st == hs.OK for st, _ in res.values())
    assert peak_running < len(tickets)
    srv.close()


def test_failure_paths_fail_the_request_not_the_server():
    srv = hs.Server(hbm_budget_bytes=64 * 1024 * 1024)
    # oversize request: rejected at submit
    mesh, cfg, ic = vortex_request(64, 7, 5.0, 5.0, 2.0, 0.3)
    mesh.ez = 64
    with pytest.raises(hs.HS3DError) as ei:
        srv.submit(mesh, cfg, ic, n_steps=1)
    assert ei.value.status == hs.ERR_NOMEM
    # bad descriptor
    mesh, cfg, ic = vortex_request(4, 9, 5.0, 5.0, 2.0, 0.3)
    with pytest.raises(hs.HS3DError):
        srv.submit(mesh, cfg, ic, n_steps=1)
    # non-physical initial state (a vortex strong enough to make T < 0)
    mesh, cfg, ic = vortex_request(4, 3, 5.0, 5.0, 20.0, 0.3)
    bad = srv.submit(mesh, cfg, ic, n_steps=5)
    # a healthy request alongside
    mesh, cfg, ic = vortex_request(4, 3, 5.0, 5.0, 2.0, 0.3)
    good = srv.submit(mesh, cfg, ic, n_steps=5)
    res = wait_all(srv, [bad, good])
    assert res[bad][0] == hs.ERR_NONPHYSICAL
    assert res[good][0] == hs.OK
    srv.close()


def test_injected_allocation_failure_in_child_process():
    """HS3D_FAULT_ALLOC_FAILURES=1 makes the first admission's allocation
    fail on the host; with nothing running the request fails with NOMEM and
    the next request succeeds."""
    code = r'''
import sys, time
sys.path.insert(0, ".")
import paper_2206_09733_gb300 as hs
srv = hs.Server()
m = hs.mesh_desc(4, 4, 1, 3, lo=(0, 0, 0), hi=(10, 10, 2.5))
c = hs.solver_cfg("euler", "lf", "ec", "mixed32")
i = hs.ic_desc("vortex", 1.4, 0.3, 2.0, 5.0, 5.0)
a = srv.submit(m, c, i, n_steps=2); b = srv.submit(m, c, i, n_steps=2)
t0 = time.time()
while True:
    sa, _ = srv.poll(a); sb, _ = srv.poll(b)
    if sa != hs.PENDING and sb != hs.PENDING: break
    assert time.time() - t0 < 60
    time.sleep(0.01)
print(sa, sb)
srv.close()
'''
    env = dict(os.environ, HS3D_FAULT_ALLOC_FAILURES="1")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=180)
    assert r.returncode == 0, r.stderr
    sa, sb = (int(x) for x in r.stdout.split())
    assert sa == hs.ERR_NOMEM and sb == hs.OK


def test_bounded_wait_times_out_cleanly_in_child_process():
    """HS3D_SERVER_WAIT_LIMIT_S=0 gives the server's completion wait no time:
    the running requests fail with HS3D_ERR_TIMEOUT, the process exits
    cleanly (no GPU wait is left unbounded)."""
    code = r'''
import sys, time
sys.path.insert(0, ".")
import paper_2206_09733_gb300 as hs
srv = hs.Server()
m = hs.mesh_desc(24, 24, 24, 7, lo=(0, 0, 0), hi=(10, 10, 10))
c = hs.solver_cfg("euler", "lf", "standard", "fp64")
i = hs.ic_desc("vortex", 1.4, 0.3, 2.0, 5.0, 5.0)
a = srv.submit(m, c, i, n_steps=50)
t0 = time.time()
while True:
    sa, _ = srv.poll(a)
    if sa != hs.PENDING: break
    assert time.time() - t0 < 120
    time.sleep(0.01)
print(sa)
srv.close()
'''
    env = dict(os.environ, HS3D_SERVER_WAIT_LIMIT_S="0")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert int(r.stdout.split()[-1]) == hs.ERR_TIMEOUT


def _tgv_request(E, N, precision, physics, surface, volume, amp):
    mesh = hs.mesh_desc(E, E, E, N, lo=(-np.pi,) * 3, hi=(np.pi,) * 3, amp=amp)
    cfg = hs.solver_cfg(physics, surface, volume, precision, gamma=G, Re=800.0, Pr=0.72, Ma=0.1, cfl=0.5)
    ic = hs.ic_desc("tgv", G, 0.1)
    return mesh, cfg, ic


def test_persistent_launches_equal_grid_launches_and_single_solves():
    """The persistent design (work table + persistent grids whose CTAs walk
    several tiles: groups here hold more tiles than fit on the GPU at once)
    against the grid design, and the grid design against the same solves
    stepped alone (bitwise) -- Navier-Stokes on the bulk-copy (N = 3) and
    per-thread copy (N = 2, 4) staging paths, the split and standard forms,
    FP64 and mixed precision.  The persistent kernels are instantiations of
    their own (the tile body called out of line), where the compiler may fuse
    the FP32 multiply-adds of the mixed path differently: those states agree
    to the FP32 rounding of the residual (1e-7 relative after 3 steps), the
    FP64 ones bitwise."""
    specs = [(14, 3, "mixed32", "ns", "roe", "ec", 0.05), (12, 3, "mixed32", "ns", "roe", "ec", 0.03),
             (13, 3, "mixed32", "ns", "roe", "ec", 0.0),
             (16, 2, "mixed32", "euler", "lf", "standard", 0.04), (15, 2, "mixed32", "euler", "lf", "standard", 0.0),
             (8, 4, "mixed32", "ns", "roe", "standard", 0.05), (9, 4, "mixed32", "ns", "roe", "standard", 0.02),
             (6, 3, "fp64", "ns", "roe", "ec", 0.05), (5, 3, "fp64", "ns", "roe", "ec", 0.0)]
    n_steps = 3
    finals = {}
    for mode in ("grid", "persistent"):
        srv = hs.Server(launch_mode=mode)
        tickets, outs = [], []
        for E, N, prec, phys, surf, vol, amp in specs:
            mesh, cfg, ic = _tgv_request(E, N, prec, phys, surf, vol, amp)
            out = np.zeros((E ** 3, 5, N + 1, N + 1, N + 1))
            tickets.append(srv.submit(mesh, cfg, ic, n_steps=n_steps, result=out))
            outs.append(out)
        res = wait_all(srv, tickets)
        srv.close()
        for t in tickets:
            assert res[t][0] == hs.OK and res[t][1].steps == n_steps
        finals[mode] = outs
    for spec, a, b in zip(specs, finals["grid"], finals["persistent"]):
        if spec[2] == "fp64":
            assert np.array_equal(a, b), spec
        else:
            assert np.abs(a - b).max() <= 1e-7 * np.abs(a).max(), spec
    for k in (0, 3, 5, 7):
        E, N, prec, phys, surf, vol, amp = specs[k]
        gm = hs.Mesh(E, E, E, N, lo=(-np.pi,) * 3, hi=(np.pi,) * 3, amp=amp)
        u = gm.init_state(gm.empty_state(), "tgv", G, 0.1)
        g = torch.zeros_like(u)
        gm.rk3_run(hs.solver_cfg(phys, surf, vol, prec, gamma=G, Re=800.0, Pr=0.72, Ma=0.1, cfl=0.5), u, g, n_steps)
        torch.cuda.synchronize()
        assert np.array_equal(finals["grid"][k], u.cpu().numpy()), specs[k]
