"""Mixed-precision path against the FP64 oracle: FP32 flux arithmetic on
deviations from a per-element reference state formed in FP64, the mass
divergence in float-float, FP64 state, geometry and RK accumulation.

Every residual is held to 1e-5 relative (rel-L2 over all nodes and
variables), on smooth random states for every scheme and on the Mach 0.1
Taylor-Green vortex, where the residual is a small difference of fluxes
of O(p0 = 71) and O(H = 250): rounding the state alone to FP32 moves that
residual by ~5e-4, so only the deviation formulation meets the bar there."""
import numpy as np
import pytest

import oracle as O
from tests.inputs import random_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2206_09733_gb300 as hs  # noqa: E402

G = 1.4


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2206_09733_gb300 import build
    build.build()
    hs.lib()


COMBOS = [(p, s, v) for p in ("euler", "ns") for s in ("lf", "roe", "ec", "rusanov", "ldroe", "matrix")
          for v in ("standard", "ec", "kg", "pirozzoli", "ducros", "morinishi", "ir")]


@pytest.mark.parametrize("combo", COMBOS)
def test_mixed_residual_smooth_state(combo):
    lo, hi = (-np.pi,) * 3, (np.pi,) * 3
    om = O.Mesh(3, 3, 3, 4, lo=lo, hi=hi, amp=0.1)
    gm = hs.Mesh(3, 3, 3, 4, lo=lo, hi=hi, amp=0.1)
    u0 = random_state(om.shape, seed=21, smooth=True)
    ref = om.residual(O.Cfg(*combo, Re=400.0), u0)
    u = torch.from_numpy(u0).cuda()
    r = torch.empty_like(u)
    gm.residual(hs.solver_cfg(*combo, "mixed32", Re=400.0), u, r)
    err = rel(host(r), ref)
    print(f"mixed residual rel-L2 {combo}: {err:.3e}")
    assert err < 1e-5


@pytest.mark.parametrize("N", range(1, 8))
@pytest.mark.parametrize("combo", [("euler", "lf", "standard"), ("ns", "roe", "ec"), ("ns", "matrix", "kg")])
def test_mixed_every_order(N, combo):
    """Both staging variants of the mixed element kernel (bulk copies for an
    even number of nodes per direction, per-thread asynchronous copies for
    an odd one) against the oracle: the residual of a smooth state and the
    state after three RK steps."""
    lo, hi = (-np.pi,) * 3, (np.pi,) * 3
    om = O.Mesh(3, 2, 2, N, lo=lo, hi=hi, amp=0.05)
    gm = hs.Mesh(3, 2, 2, N, lo=lo, hi=hi, amp=0.05)
    u0 = random_state(om.shape, seed=40 + N, smooth=True)
    oc = O.Cfg(*combo, Re=400.0)
    gc = hs.solver_cfg(*combo, "mixed32", Re=400.0)
    ref = om.residual(oc, u0)
    u = torch.from_numpy(u0).cuda()
    r = torch.empty_like(u)
    gm.residual(gc, u, r)
    assert rel(host(r), ref) < 1e-5
    uo, go = u0.copy(), np.zeros_like(u0)
    for _ in range(3):
        om.rk3_step(oc, uo, go)
    g = torch.zeros_like(u)
    gm.rk3_run(gc, u, g, 3)
    assert rel(host(u), uo) < 1e-5
    assert gm.clock()[1] >= 3


def test_mixed_ec_n3_partial_tile():
    """The Chandrashekar element kernel at N = 3, whose x- and y-line pair
    fluxes travel by warp shuffles: 27 elements in the default tiles of 4
    elements, so that the last tile holds an element past the end of the mesh
    (its lanes take part in the shuffles with no work), against the oracle."""
    lo, hi = (-np.pi,) * 3, (np.pi,) * 3
    om = O.Mesh(3, 3, 3, 3, lo=lo, hi=hi, amp=0.07)
    gm = hs.Mesh(3, 3, 3, 3, lo=lo, hi=hi, amp=0.07)
    u0 = random_state(om.shape, seed=77, smooth=True)
    oc = O.Cfg("ns", "roe", "ec", Re=400.0)
    gc = hs.solver_cfg("ns", "roe", "ec", "mixed32", Re=400.0)
    ref = om.residual(oc, u0)
    u = torch.from_numpy(u0).cuda()
    r = torch.empty_like(u)
    gm.residual(gc, u, r)
    assert rel(host(r), ref) < 1e-5
    uo, go = u0.copy(), np.zeros_like(u0)
    for _ in range(2):
        om.rk3_step(oc, uo, go)
    g = torch.zeros_like(u)
    gm.rk3_run(gc, u, g, 2)
    assert rel(host(u), uo) < 1e-5


@pytest.mark.parametrize("vol", ["standard", "ec", "kg"])
def test_tensor_core_precision_computes_as_mixed32(vol):
    """HS3D_MIXED_TC is accepted and runs the MIXED32 kernels (the
    contraction stays on the CUDA cores): residual and RK steps bitwise equal."""
    lo, hi = (-np.pi,) * 3, (np.pi,) * 3
    gm = hs.Mesh(3, 3, 3, 7, lo=lo, hi=hi, amp=0.05)
    u0 = torch.from_numpy(random_state(gm.shape, seed=7, smooth=True)).cuda()
    a, b = torch.empty_like(u0), torch.empty_like(u0)
    gm.residual(hs.solver_cfg("ns", "roe", vol, "mixed_tc", Re=400.0), u0, a)
    gm.residual(hs.solver_cfg("ns", "roe", vol, "mixed32", Re=400.0), u0, b)
    assert torch.equal(a, b)
    ua, ub = u0.clone(), u0.clone()
    gm.rk3_run(hs.solver_cfg("ns", "roe", vol, "mixed_tc", Re=400.0), ua, torch.zeros_like(ua), 2)
    gm.rk3_run(hs.solver_cfg("ns", "roe", vol, "mixed32", Re=400.0), ub, torch.zeros_like(ub), 2)
    assert torch.equal(ua, ub)


def test_mixed_tgv_residual_and_state():
    lo, hi = (-np.pi,) * 3, (np.pi,) * 3
    om = O.Mesh(16, 16, 16, 3, lo=lo, hi=hi, amp=0.05)
    gm = hs.Mesh(16, 16, 16, 3, lo=lo, hi=hi, amp=0.05)
    oc = O.Cfg("ns", "roe", "ec", Re=1600.0)
    gc = hs.solver_cfg("ns", "roe", "ec", "mixed32", Re=1600.0)
    u0 = om.ic_tgv(G, 0.1)
    ref = om.residual(oc, u0)
    u = torch.from_numpy(u0).cuda()
    r = torch.empty_like(u)
    gm.residual(gc, u, r)
    err_r = rel(host(r), ref)
    uo, go = u0.copy(), np.zeros_like(u0)
    for _ in range(10):
        om.rk3_step(oc, uo, go)
    g = torch.zeros_like(u)
    gm.rk3_run(gc, u, g, 10)
    err_u = rel(host(u), uo)
    per_var = [float(np.linalg.norm(host(r)[:, v] - ref[:, v]) / np.linalg.norm(ref)) for v in range(5)]
    print(f"mixed TGV 16^3: residual rel-L2 {err_r:.3e} (per variable {per_var}), "
          f"state after 10 steps rel-L2 {err_u:.3e}")
    assert err_r < 1e-5
    assert err_u < 1e-5


def test_integer_pipe_rounding_matches_hardware():
    """The mixed path's FP64->FP32 rounding (bit operations) equals the
    hardware round-to-nearest conversion on random and edge-case inputs;
    the exact widening equals the hardware FP32->FP64 conversion; the
    float-float split's low part (integer arithmetic and one int->float
    conversion) equals the hardware rounding of x - hi."""
    rng = np.random.default_rng(0)
    parts = [rng.standard_normal(1 << 20) * 10.0 ** rng.uniform(-30, 30, 1 << 20),
             rng.uniform(-1e3, 1e3, 1 << 20),
             np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.nan, 3.4028234663852886e38,
                       3.4028235677973366e38, 1.1754943508222875e-38, 1e-40, -1e-45, 1e300, -1e-300])]
    # halfway cases: float grid points plus exactly half an FP32 ulp
    f = rng.uniform(1, 2, 1 << 16).astype(np.float32).astype(np.float64)
    parts.append(f + 2.0 ** -24)
    parts.append(f - 2.0 ** -24)
    x = torch.from_numpy(np.concatenate(parts)).cuda()
    bad, bad_widen, tiny, bad_split = hs.check_rounding(x)
    assert bad == 0 and bad_widen == 0 and bad_split == 0
    assert tiny >= 3
