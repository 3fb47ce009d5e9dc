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
    return sorted(set(re.findall(r"\b(sop_[a-z0-9_]+)\s*\(", src)))


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


def test_struct_layouts_match_header(tmp_path):
    """Size and every field offset of the ctypes mirrors equal what a C compiler lays out
    from include/sop.h."""
    import subprocess
    from paper_1003_1148_gb300 import sop
    mirrors = {"sop_topology": sop.Topology, "sop_params": sop.Params, "sop_pull_params": sop.PullParams,
               "sop_record": sop.Record, "sop_stats": sop.Stats, "sop_ramp_params": sop.RampParams}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "sop.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        c, f, v = line.split()
        got[(c, f)] = int(v)
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


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


def test_noise_calls_validate_before_any_cuda_call(lib):
    # n out of range and a bead range past 2^32 are rejected before any device work;
    # n = 0 is a valid empty request that touches no device
    from paper_1003_1148_gb300 import sop
    import numpy as np
    assert sop.box_muller(np.zeros((0, 4), np.uint32)).shape == (0, 3)
    assert sop.bead_noise(1, 0, 0, 0).shape == (0, 3)
    with pytest.raises(sop.SopError) as e:
        sop.bead_noise(1, 0, 2 ** 32 - 2, 4)
    assert e.value.status == sop.ERR_INVALID_ARG
    L = sop.load()   # too many items: refused without touching the (NULL) output
    assert L.sop_bead_noise(1, 0, 0, 2 ** 26 + 1, None, None) == sop.ERR_INVALID_ARG
    assert L.sop_box_muller(None, -1, None, None) == sop.ERR_INVALID_ARG
