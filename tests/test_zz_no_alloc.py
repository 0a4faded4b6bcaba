"""The allocation-free solve entry point (rich_solve_batch_noalloc).

Some callers cannot call cudaMalloc: code embedded in a host framework that
owns all device memory through its own pool allocator, or latency-sensitive
loops that cannot afford cudaMalloc's implicit device synchronisation.  For
them the library offers one entry point that allocates nothing and works out of
a fixed static device array.  This test calls it through the C ABI twice in a
row, on different inputs, and checks each result against the regular
rich_solve_batch entry point at the FP64 parity tolerance (1e-10 relative,
statuses equal).  It lives in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import paper_1903_08741_gb300 as R
    from paper_1903_08741_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(torch.device("cuda:0"))
    return R


def test_noalloc_matches_solve_batch_twice(R):
    from tests.inputs import PHYSICS, SOLVER
    dev = torch.device("cuda:0")
    pb = R.Problem(nx=32, nz=32, nsteps=3, dt=0.01, **PHYSICS, **SOLVER)
    for call, seed in enumerate((21, 22)):
        lk, al = O.sample_fields(32, 32, 12, seed=seed)
        lk_d, al_d = torch.from_numpy(lk).to(dev), torch.from_numpy(al).to(dev)
        q_ref, _, s_ref, _, _ = R.solve_batch(pb, lk_d, al_d)
        qoi = torch.full((12,), -1.0, dtype=torch.float64, device=dev)
        status = torch.full((12,), -7, dtype=torch.int32, device=dev)
        R.solve_batch_noalloc(pb, lk_d, al_d, qoi=qoi, status=status)
        torch.cuda.synchronize(dev)
        q, s = qoi.cpu().numpy(), status.cpu().numpy()
        q_ref, s_ref = q_ref.cpu().numpy(), s_ref.cpu().numpy()
        assert np.array_equal(s, s_ref), (call, s, s_ref)
        ok = s_ref == 0
        assert ok.sum() >= 6
        rel = np.abs(q[ok] - q_ref[ok]) / np.abs(q_ref[ok])
        assert rel.max() <= 1e-10, (call, rel.max())
        assert np.all(np.isnan(q[(s_ref == 1) | (s_ref == 3)]))


@pytest.mark.parametrize("n,prec", [(32, "mixed"), (128, "fp64")])
def test_noalloc_other_precisions_and_grids(R, n, prec):
    """Mixed precision (FP32 cycles, QoI within the mixed path's 1e-6) and a
    128^2 FP64 grid, whose 2.9 MiB slots let only five CTAs share the array
    (bit-identical results to the regular entry point at any CTA count)."""
    from tests.inputs import PHYSICS, SOLVER
    dev = torch.device("cuda:0")
    kw = dict(precision=R.MIXED) if prec == "mixed" else {}
    pb = R.Problem(nx=n, nz=n, nsteps=2, dt=0.005, **PHYSICS, **SOLVER, **kw)
    S = 12
    lk, al = O.sample_fields(n, n, S, seed=31)
    lk_d, al_d = torch.from_numpy(lk).to(dev), torch.from_numpy(al).to(dev)
    q_ref, _, s_ref, _, _ = R.solve_batch(pb, lk_d, al_d)
    for call in range(2):
        q, s = R.solve_batch_noalloc(pb, lk_d, al_d)
        torch.cuda.synchronize(dev)
        ok = (s_ref == 0) & (s == 0)
        assert ok.sum() >= S // 2
        if prec == "mixed":
            assert (torch.abs(q[ok] - q_ref[ok]) / torch.abs(q_ref[ok])).max() <= 1e-6, call
        else:
            assert torch.equal(s, s_ref) and torch.equal(q[ok], q_ref[ok]), call


def test_noalloc_rejects_oversized_grid(R):
    from tests.inputs import PHYSICS, SOLVER
    dev = torch.device("cuda:0")
    pb = R.Problem(nx=1024, nz=1024, nsteps=1, dt=0.01, **PHYSICS, **SOLVER)
    x = torch.zeros((1, 1024, 1024), dtype=torch.float64, device=dev)
    with pytest.raises(R.RichError):
        R.solve_batch_noalloc(pb, x, x)


def test_noalloc_rejects_bad_shapes_before_launch(R):
    """A field of another grid, a mismatched alpha, or a qoi / status shorter
    than the batch raise before the library is called."""
    from tests.inputs import PHYSICS, SOLVER
    dev = torch.device("cuda:0")
    pb = R.Problem(nx=16, nz=16, nsteps=1, dt=0.01, **PHYSICS, **SOLVER)
    x = torch.zeros((4, 16, 16), dtype=torch.float64, device=dev)
    l0 = R.launch_count()
    for args, kw in (((torch.zeros((4, 16, 8), dtype=torch.float64, device=dev), x), {}),
                     ((x, torch.zeros((3, 16, 16), dtype=torch.float64, device=dev)), {}),
                     ((x, x), dict(qoi=torch.zeros(3, dtype=torch.float64, device=dev))),
                     ((x, x), dict(status=torch.zeros(2, dtype=torch.int32, device=dev)))):
        with pytest.raises(R.RichError):
            R.solve_batch_noalloc(pb, *args, **kw)
    assert R.launch_count() == l0
