"""Host logic of the launch-shape autotuner (no GPU): candidate shapes, cache
keys, and the shipped GB300 choices."""
import json

import pytest

from paper_1903_08741_gb300 import autotune


class _Pb:
    def __init__(self, nx, nz, precision=0, cycle=1, closure=0):
        self.nx, self.nz, self.precision, self.cycle, self.closure = nx, nz, precision, cycle, closure


def test_one_warp_shape_only_for_small_grids():
    assert autotune.shapes(_Pb(16, 16))[0] == 32
    assert autotune.shapes(_Pb(32, 32))[0] == 32
    assert 32 not in autotune.shapes(_Pb(64, 64))
    assert 32 not in autotune.shapes(_Pb(64, 32))
    assert autotune.shapes(_Pb(64, 16))[0] == 32          # 1024 cells
    for n in (16, 64, 512):
        assert autotune.shapes(_Pb(n, n))[-4:] == (128, 256, 512, 1024)


def test_keys_bucket_the_batch_and_name_cycle_and_closure():
    k = autotune._key(_Pb(128, 128), 4096, "GPU")
    assert k == "GPU|128x128|fp64|S4096"
    assert autotune._key(_Pb(128, 128, precision=1), 3000, "GPU") == "GPU|128x128|mixed|S4096"
    assert autotune._key(_Pb(32, 32, cycle=2, closure=1), 25600, "GPU") == "GPU|32x32|fp64|S32768|W2|VG"
    assert autotune._bucket(1) == 1 and autotune._bucket(80) == 128 and autotune._bucket(128) == 128


def test_cache_path_follows_the_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("RICH_TUNE_CACHE", str(tmp_path / "t.json"))
    assert autotune.cache_path() == str(tmp_path / "t.json")


def test_shipped_choices_are_valid_and_the_fastest_probed():
    with open(autotune.SHIPPED) as f:
        data = json.load(f)
    assert data
    for key, e in data.items():
        name, grid, prec = key.split("|")[:3]
        nx, nz = (int(v) for v in grid.split("x"))
        bt, mi = e["block_threads"], e["mixed_inner"]
        assert bt in (32, 128, 256, 512, 1024), key
        assert (mi == 0) if prec == "fp64" else (1 <= mi <= 16), key
        if bt == 32:
            assert nx * nz <= 32 * 32, key
        probe = e["probe_ms"]
        assert f"{bt}/{mi}" in probe
        assert probe[f"{bt}/{mi}"] == pytest.approx(min(probe.values())), key
