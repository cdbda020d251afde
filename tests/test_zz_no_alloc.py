"""hs3d_diagnostics_noalloc against hs3d_diagnostics (needs a GPU).

The no-allocation entry point serves callers that cannot allocate device
memory (for example code running during a stream capture, or inside a
framework that owns all device memory): it takes every input from the
caller and keeps its partial sums in a fixed device array.  Its results must
equal the allocating entry point's, on two calls in a row (the array keeps
the previous call's contents), with and without dudt.  This file is named to
be collected last."""
import numpy as np
import pytest

from tests.inputs import random_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2206_09733_gb300 as hs  # noqa: E402

TOL = 1e-13


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2206_09733_gb300 import build
    build.build()
    hs.lib()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_allocating_entry_point_twice():
    lo, hi = (-np.pi,) * 3, (np.pi,) * 3
    results = []
    for call, (shape, N, seed) in enumerate([((5, 4, 3), 3, 1), ((3, 3, 2), 5, 2)]):
        m = hs.Mesh(*shape, N, lo=lo, hi=hi, amp=0.08)
        cfg = hs.solver_cfg("euler", "ec", "ec", "fp64")
        u = torch.from_numpy(random_state(m.shape, seed=seed)).cuda()
        r = torch.empty_like(u)
        m.residual(cfg, u, r)
        _, _, J = m.geometry()
        for dudt in (None, r):
            ref = torch.zeros(7, dtype=torch.float64, device="cuda")
            got = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda")
            m.diagnostics(cfg, u, ref, dudt=dudt)
            hs.diagnostics_noalloc(N, m.E, 1.4, J, u, got, dudt=dudt)
            torch.cuda.synchronize()
            a, b = got.cpu().numpy(), ref.cpu().numpy()
            k = 7 if dudt is not None else 5
            assert np.all(np.isfinite(a[:k]))
            assert _rel(a[:5], b[:5]) < TOL, (call, a, b)
            if dudt is not None:
                assert abs(a[5] - b[5]) <= TOL * b[6] and _rel(a[6:7], b[6:7]) < TOL
            results.append(a.copy())
    # the second call ran on different data: it did not reuse the first's sums
    assert not np.allclose(results[0][:5], results[2][:5])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    u = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    with pytest.raises(hs.HS3DError) as ei:
        hs.diagnostics_noalloc(7, 16385, 1.4, u, u, out)      # 16385 * 512 > 8,388,608 nodes
    assert ei.value.status == hs.ERR_INVALID
    assert "capacity" in str(ei.value)


def test_noalloc_on_gauss_nodes_uses_their_weights():
    """On a mesh with Gauss-Legendre solution nodes J and u live at the Gauss
    points: the sums take the Gauss weights, as hs3d_diagnostics does."""
    lo, hi = (-np.pi,) * 3, (np.pi,) * 3
    for N in (2, 3):
        m = hs.Mesh(4, 3, 2, N, lo=lo, hi=hi, amp=0.06, nodes="gauss")
        cfg = hs.solver_cfg("euler", "roe", "standard", "fp64")
        u = torch.from_numpy(random_state(m.shape, seed=10 + N)).cuda()
        r = torch.empty_like(u)
        m.residual(cfg, u, r)
        _, _, J = m.geometry()
        for dudt in (None, r):
            ref = torch.zeros(7, dtype=torch.float64, device="cuda")
            got = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda")
            m.diagnostics(cfg, u, ref, dudt=dudt)
            hs.diagnostics_noalloc(N, m.E, 1.4, J, u, got, dudt=dudt, nodes="gauss")
            torch.cuda.synchronize()
            a, b = got.cpu().numpy(), ref.cpu().numpy()
            assert _rel(a[:5], b[:5]) < TOL, (N, a, b)
            if dudt is not None:
                assert abs(a[5] - b[5]) <= TOL * b[6] and _rel(a[6:7], b[6:7]) < TOL
        # the Lobatto weights would not do: the sums differ at O(1)
        wrong = torch.zeros(7, dtype=torch.float64, device="cuda")
        hs.diagnostics_noalloc(N, m.E, 1.4, J, u, wrong)
        torch.cuda.synchronize()
        assert _rel(wrong.cpu().numpy()[:5], b[:5]) > 1e-3


def test_noalloc_small_call_after_a_large_one():
    """A call that uses fewer partial-sum slots than the previous one reads
    only the slots it wrote (the array keeps the previous call's sums)."""
    lo, hi = (-np.pi,) * 3, (np.pi,) * 3
    for shape, N in (((16, 16, 8), 3), ((1, 1, 1), 2)):
        m = hs.Mesh(*shape, N, lo=lo, hi=hi, amp=0.05)
        cfg = hs.solver_cfg("euler", "lf", "standard", "fp64")
        u = torch.from_numpy(random_state(m.shape, seed=3)).cuda()
        _, _, J = m.geometry()
        ref = torch.zeros(7, dtype=torch.float64, device="cuda")
        got = torch.zeros(7, dtype=torch.float64, device="cuda")
        m.diagnostics(cfg, u, ref)
        hs.diagnostics_noalloc(N, m.E, 1.4, J, u, got)
        torch.cuda.synchronize()
        assert _rel(got.cpu().numpy()[:5], ref.cpu().numpy()[:5]) < TOL, shape
