"""The C-ABI library builds, loads and exports every function its header declares;
the ctypes structures have the C layout.  No GPU needed."""
import ctypes as C
import os
import re
import subprocess

import pytest

import paper_1903_08741_gb300 as R
from paper_1903_08741_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(rich_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(libpath):
    names = declared_functions()
    assert "rich_solve_batch" in names and "rich_sample_fields" in names
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (rich_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    L = C.CDLL(libpath)
    for n in names:
        assert hasattr(L, n)
    assert sorted(R.exported_symbols()) == names


def test_status_strings_without_gpu(libpath):
    L = R.lib()
    assert L.rich_status_str(0) == b"ok"
    assert b"picard" in L.rich_status_str(1)
    assert b"adjoint" in L.rich_status_str(4)
    assert L.rich_set_adjoint_limits(None, 1e-11, 400) == -1
    h = C.c_void_p()
    assert L.rich_create(C.byref(h), 0) in (0, -2)   # -2 when no CUDA device is present


def test_struct_layouts_match_c(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "richards.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(rich_problem_t),'
                   ' sizeof(rich_field_t), sizeof(rich_stats_t), offsetof(rich_problem_t, precision),'
                   ' offsetof(rich_stats_t, seconds), offsetof(rich_problem_t, cycle),'
                   ' offsetof(rich_field_t, nu), offsetof(rich_field_t, corr_len_z),'
                   ' sizeof(rich_mlmc_cfg_t), offsetof(rich_mlmc_cfg_t, tune_inner),'
                   ' sizeof(rich_mlmc_result_t)); printf("%zu %zu %zu\\n", offsetof(rich_mlmc_cfg_t, bias_pairs),'
                   ' offsetof(rich_mlmc_result_t, total_rmse), offsetof(rich_mlmc_result_t, levels_for_eps));'
                   ' return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert vals == [C.sizeof(R._Problem), C.sizeof(R._Field), C.sizeof(R._Stats),
                    R._Problem.precision.offset, R._Stats.seconds.offset, R._Problem.cycle.offset,
                    R._Field.nu.offset, R._Field.corr_len_z.offset, C.sizeof(R._MlmcCfg),
                    R._MlmcCfg.tune_inner.offset, C.sizeof(R._MlmcResult), R._MlmcCfg.bias_pairs.offset,
                    R._MlmcResult.total_rmse.offset, R._MlmcResult.levels_for_eps.offset]


def test_noalloc_wrapper_rejects_bad_shapes_on_host():
    """The allocation-free wrapper checks grid shape, alpha shape and the
    lengths of qoi / status before anything reaches the library (CPU tensors
    here: the check runs before any device is touched)."""
    torch = pytest.importorskip("torch")
    pb = R.Problem(nx=16, nz=16, nsteps=1, dt=0.01)
    x = torch.zeros((4, 16, 16), dtype=torch.float64)
    bad = ((torch.zeros((4, 16, 8), dtype=torch.float64), x, None, None),
           (x, torch.zeros((3, 16, 16), dtype=torch.float64), None, None),
           (torch.zeros((16, 16), dtype=torch.float64), x, None, None),
           (x, x, torch.zeros(3, dtype=torch.float64), None),
           (x, x, None, torch.zeros(2, dtype=torch.int32)))
    for lk, al, q, s in bad:
        with pytest.raises(R.RichError):
            R.solve_batch_noalloc(pb, lk, al, qoi=q, status=s)
    assert R._check_noalloc_args(pb, x, x, None, None) == 4
