"""Host logic of bench.py (no GPU): the DRAM-traffic figure is reported only for
the kernel sources it was captured from, and MLMC levels are tuned for the
estimator's per-launch batch."""
import bench


def test_traffic_only_for_the_captured_sources(monkeypatch):
    sha, ratio = bench.TRAFFIC[("fp64", 512)]
    monkeypatch.setattr(bench, "fused_sha", lambda: sha)
    assert bench.captured_traffic("fp64", 512, 1e12) == ratio * 1e12
    assert bench.captured_traffic("fp64", 1024, 1e12) is None          # shape never captured
    monkeypatch.setattr(bench, "fused_sha", lambda: "0" * 64)           # kernel changed since
    assert bench.captured_traffic("fp64", 512, 1e12) is None


def test_fused_sha_covers_kernel_and_host_code():
    a = bench.fused_sha()
    assert len(a) == 64 and a == bench.fused_sha()


def test_mlmc_launch_batches_follow_the_field_buffers():
    # B = 2^31 / (16 * 256^2) = 2048 finest-level fields; level l holds B (256 / n_l)^2
    L = bench.MLMC_LEVELS
    got = [bench.mlmc_launch_batch(L, n, l) for l, n in enumerate(L["nsamples"])]
    assert got == [20000, 5000, 1200, 300, 80]
    big = dict(nsamples=(10 ** 7, 10 ** 6, 10 ** 5), n0=64, steps0=5, t_final=0.1)   # finest 256^2
    assert [bench.mlmc_launch_batch(big, n, l) for l, n in enumerate(big["nsamples"])] == [32768, 8192, 2048]
