"""The C-ABI library loads and exports every entry point declared in
include/ugkwp.h; argument validation and workspace sizing run without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2312_16981_gb300 import binding as B
from paper_2312_16981_gb300 import build as gpu_build
from paper_2312_16981_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    gpu_build.build()
    return B.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ugkwp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ugkwp_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    # and the binding knows all of them
    assert set(names) == set(B.FUNCTIONS)


def test_workspace_size_and_validation(lib):
    p = I.multigroup_slab()
    n = B.workspace_bytes(p)
    assert n > 2 * p.particle_capacity * 44
    bad = p.replace(G=0)
    with pytest.raises(B.UGKWPError) as e:
        B.workspace_bytes(bad)
    assert e.value.code == -1
    p2 = I.small_checkerboard()
    p2.bc = [I.BC_BLACKBODY, 0, 0, 0]
    p2.bcT = [1.0, 0, 0, 0]
    with pytest.raises(B.UGKWPError) as e:
        B.workspace_bytes(p2)
    assert e.value.code == -8


def test_init_rejects_small_workspace_without_touching_device(lib):
    p = I.small_multigroup()
    hp = B._HostProblem(p)
    h = ctypes.c_void_p()
    code = lib.ugkwp_init(ctypes.byref(hp.s), ctypes.c_void_p(256), 16, None, ctypes.byref(h))
    assert code == -7 and not h.value
    assert b"workspace" in lib.ugkwp_last_error(None)


def test_record_layout_matches_header():
    assert B.RECORD.itemsize == 8 + 6 * 4 + 9 * 8


def test_3d_validation_and_sizing(lib):
    p = I.checkerboard_3d(n=8, G=3, block=2, patch=2)
    n3 = B.workspace_bytes(p)
    # z positions and directions of both particle buffers on top of the 2D layout
    assert n3 > 2 * p.particle_capacity * (6 * 8 + 8 + 4 + 2 * 8)
    for bad, code in [(p.replace(nz=0), -1), (p.replace(dz=0.0), -1),
                      (p.replace(bc=[0, 0, 0, 0, 3, 0]), -1),
                      (p.replace(bc=[0, 0, 0, 0, I.BC_BLACKBODY, 0], bcT=[0.0] * 4 + [1.0, 0.0]), -8)]:
        with pytest.raises(B.UGKWPError) as e:
            B.workspace_bytes(bad)
        assert e.value.code == code
    # ensembles are built for 1D and 2D members
    hps = [B._HostProblem(q) for q in (p, p.replace(seed=1))]
    arr = (B.CProblem * 2)(*[hp.s for hp in hps])
    n = ctypes.c_size_t()
    assert lib.ugkwp_workspace_size_ensemble(arr, 2, ctypes.byref(n)) == -8
