"""CPU checks of the C-ABI boundary: the library builds, loads and exports every entry point
that include/pic.h declares; parameter validation needs no GPU."""
import ctypes as C
import subprocess

import pytest

from paper_2109_04469_gb300 import build as B
from paper_2109_04469_gb300 import pic, workloads


@pytest.fixture(scope="module")
def lib():
    B.build()
    return pic.lib()


def test_every_declared_entry_point_is_exported(lib):
    names = pic.declared_functions()
    assert len(names) >= 18
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert getattr(lib, n) is not None


def test_binding_covers_the_header(lib):
    # every declared function has a ctypes signature in the binding
    import inspect

    src = inspect.getsource(pic.lib)
    for n in pic.declared_functions():
        assert f'"{n}"' in src, n


def test_struct_layout_matches_header(lib):
    # pic_params: 13 doubles + 3 int32 pairs + 2 int64 + u64 + u32/i32 pair + ...; the
    # workspace query accepts a valid struct and rejects a broken one field by field
    cfg = workloads.params("ccp_5pa_150v_128c")
    assert pic.workspace_bytes(cfg) > 0
    bad = [dict(n_cells=1), dict(weight=0.0), dict(refl_e=1.5), dict(gamma_see=-0.1),
           dict(capacity_per_species=10), dict(steps_per_rf=0), dict(eepf_bins=0),
           dict(precision=7), dict(gap_m=float("nan")), dict(capacity_per_species=2**31)]
    for b in bad:
        c = dict(cfg)
        c.update(b)
        with pytest.raises(pic.PicError) as e:
            pic.workspace_bytes(c)
        assert e.value.code == -1, b


def test_workspace_grows_with_capacity(lib):
    a = pic.workspace_bytes(workloads.params("ccp_5pa_150v_128c"))
    b = pic.workspace_bytes(workloads.params("ccp_5pa_150v_128c", capacity_per_species=10**6))
    assert b > a
    assert a % 256 == 0 and b % 256 == 0


def test_strerror(lib):
    for code in (0, -1, -2, -3, -4, -5, 1, 99):
        assert isinstance(lib.pic_strerror(code), bytes)


def test_null_handles_are_rejected(lib):
    assert lib.pic_step(None, 1) == -1
    assert lib.pic_sync(None) == -1
    assert lib.pic_diag(None, None) == -1
    h = C.c_void_p()
    p = pic.make_params(workloads.params("ccp_5pa_150v_128c"))
    # a missing workspace is refused before any CUDA call
    assert lib.pic_init(C.byref(p), None, 0, None, C.byref(h)) == -5
