"""CPU checks of the C-ABI library: it builds, loads, exports every function that
include/biot.h declares, and validates arguments before touching a device.
No compute call is made here."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "biot.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^BIOT_API\s+[\w\s\*]+?\b(biot_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2409_11382_gb300 import build as B
    from paper_2409_11382_gb300 import biot
    B.build()
    return biot.load_library()


def test_header_declares_the_documented_api():
    names = declared_functions()
    for must in ("biot_create", "biot_step", "biot_solve_to", "biot_read_u", "biot_read_p", "biot_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_2409_11382_gb300 import biot
    assert sorted(biot.API_FUNCTIONS) == declared_functions()


def test_struct_layout_matches_header(tmp_path):
    """The ctypes mirrors of the header's structs have the sizes and field
    offsets the C compiler gives them (compiled here from include/biot.h)."""
    import subprocess
    from paper_2409_11382_gb300 import biot
    structs = {"biot_params": biot.biot_params, "biot_side": biot.biot_side, "biot_stats": biot.biot_stats,
               "biot_request_info": biot.biot_request_info, "biot_server_stats": biot.biot_server_stats}
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "biot.h"', "int main(void) {"]
    for name, cls in structs.items():
        src.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            cfield = "lambda" if field == "lambda_" else field
            src.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {cfield}));')
    src.append("return 0; }")
    c_file = tmp_path / "layout.c"
    c_file.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c_file), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    for name, cls in structs.items():
        assert got[(name, "size")] == C.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def _params(**kw):
    from paper_2409_11382_gb300 import workloads as W
    p, sides, _ = W.terzaghi_33()
    p.update(kw)
    return p, sides


@pytest.mark.parametrize("bad", [
    dict(nx=30),            # not divisible by 2^(levels-1)
    dict(ly=2.0),           # non-square cells
    dict(alpha=1.5),
    dict(c0=0.0),
    dict(gamma=0.0),
    dict(K=0),
    dict(r=1.5),
    dict(levels=0),
    dict(mu=-1.0),
    dict(precision=7),
])
def test_invalid_parameters_are_rejected_before_device_use(lib, bad):
    from paper_2409_11382_gb300 import biot
    p, sides = _params(**bad)
    with pytest.raises(biot.BiotError) as e:
        biot.Solver(p, sides)
    assert e.value.code == biot.ERR_INVALID_ARG


def test_unpaired_periodic_side_is_rejected(lib):
    from paper_2409_11382_gb300 import biot
    p, sides = _params()
    sides = [dict(s) for s in sides]
    sides[1] = dict(eta_type=biot.PERIODIC, p_type=biot.PERIODIC)  # right periodic, left mirror
    with pytest.raises(biot.BiotError) as e:
        biot.Solver(p, sides)
    assert e.value.code == biot.ERR_INVALID_ARG


def test_missing_device_is_reported(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_2409_11382_gb300 import biot
    p, sides = _params()
    with pytest.raises(biot.BiotError) as e:
        biot.Solver(p, sides)
    assert e.value.code in (biot.ERR_NO_DEVICE, biot.ERR_CUDA)


def test_error_strings(lib):
    from paper_2409_11382_gb300 import biot
    for code in (biot.OK, biot.ERR_INVALID_ARG, biot.ERR_DIVERGED, biot.ERR_NO_DEVICE):
        assert lib.biot_error_string(code)


def test_estimate_bytes_validates_without_a_device(lib):
    from paper_2409_11382_gb300 import biot, workloads as W
    p, sides, _ = W.terzaghi_33(precision=W.FP32)
    n = biot.estimate_bytes(p, sides)
    cells = 32 * 32
    assert n > 100 * cells  # populations of all levels, flow, coupling and read-out planes
    with pytest.raises(biot.BiotError) as e:
        biot.estimate_bytes(dict(p, nx=30), sides)
    assert e.value.code == biot.ERR_INVALID_ARG


def test_server_needs_a_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_2409_11382_gb300 import biot
    with pytest.raises(biot.BiotError) as e:
        biot.Server(1 << 30, 4)
    assert e.value.code in (biot.ERR_NO_DEVICE, biot.ERR_CUDA)


def test_binding_constants_match_the_header():
    """Every numeric #define BIOT_<NAME> of the header that the binding mirrors
    as <NAME> has the same value; the option flags are all mirrored."""
    from paper_2409_11382_gb300 import biot
    text = open(HEADER).read()
    defines = dict(re.findall(r"^#define\s+BIOT_(\w+)\s+\(?(-?\d+)\)?", text, flags=re.M))
    assert "OPT_SEGMENTS" in defines and "FP32" in defines
    checked = 0
    for name, value in defines.items():
        if hasattr(biot, name):
            assert getattr(biot, name) == int(value), name
            checked += 1
    for name in defines:
        if name.startswith("OPT_"):
            assert hasattr(biot, name), name
    assert checked >= 20
