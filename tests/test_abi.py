"""The C ABI library builds, loads without a GPU and exports every entry point
that include/sop.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sop.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sop_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1003_1148_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sop_create", "sop_step", "sop_forces", "sop_pairlist_rebuild", "sop_pull", "sop_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_abi():
    from paper_1003_1148_gb300 import sop
    assert sorted(sop.EXPORTED) == declared_functions()


def test_struct_layouts_match_header():
    # field order and sizes of the ctypes mirrors follow the header's structs
    from paper_1003_1148_gb300 import sop
    assert ctypes.sizeof(sop.Record) == 8 * 8
    assert ctypes.sizeof(sop.PullParams) == 4 * 3 + 4 + 8 * 2
    assert ctypes.sizeof(sop.Params) == 10 * 8 + 2 * 4 + 8 + 4 * 4 + 8
    assert ctypes.sizeof(sop.Topology) == 8 + 8 + 8 + 8 + 8


def test_create_rejects_bad_input_without_gpu_work(lib):
    # an invalid topology is rejected by validation before any CUDA call
    from paper_1003_1148_gb300 import sop
    import numpy as np
    with pytest.raises(sop.SopError) as e:
        sop.Simulation(np.zeros((4, 3)), [0, 2, 2, 4])    # empty chain
    assert e.value.status == sop.ERR_INVALID_ARG
    with pytest.raises(sop.SopError) as e:
        sop.Simulation(np.full((2, 3), np.nan), [0, 2])
    assert e.value.status == sop.ERR_INVALID_ARG
    with pytest.raises(sop.SopError) as e:
        sop.Simulation(np.zeros((2, 3)), [0, 2], params={"dt": -1.0})
    assert e.value.status == sop.ERR_INVALID_ARG
