"""CPU checks of the C-ABI library: it builds, loads, exports every entry point
that include/*.h declares, and rejects bad arguments on the host without
touching a GPU."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1209_6038_gb300 import build, cloak
    build.build()
    return cloak.load()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(cloak_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    from paper_1209_6038_gb300 import cloak
    names = declared_functions()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
        assert n in cloak.SIGNATURES, f"{n} has no binding"
    assert set(cloak.SIGNATURES) <= set(names)


def test_null_handle_rejected_on_host(lib):
    d3 = (C.c_double * 3)(0, 0, 0)
    assert lib.cloak_camera_set(None, d3, d3, d3, 60.0, 10, 10) == 1
    assert b"null handle" in lib.cloak_last_error()
    assert lib.cloak_set_integrator(None, 0, 1e-3, 0, 10) == 1
    assert lib.cloak_render(None, 1, 1, 0, None, 0, None) == 1
    assert lib.cloak_trace_rays(None, 1, None, 0, None, None) == 1
    lib.cloak_destroy(None)


def test_record_layout():
    from paper_1209_6038_gb300 import cloak
    import oracle
    assert cloak.RECORD_DTYPE.itemsize == 80
    assert cloak.RECORD_DTYPE == oracle.RECORD_DTYPE


def declared_enums():
    """CLOAK_<NAME> = value pairs of every enum in include/*.h."""
    vals = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for body in re.findall(r"enum\s*\{(.*?)\}", src, flags=re.S):
            for name, v in re.findall(r"\bCLOAK_(\w+)\s*=\s*(-?\d+)", body):
                vals[name] = int(v)
    return vals


def test_binding_constants_match_the_header():
    """The Python binding's constants carry the header's enum values (precision, schedule, panels, ray
    status, error codes, ...): a value passed through the ABI means the same on both sides."""
    from paper_1209_6038_gb300 import cloak
    vals = declared_enums()
    assert len(vals) >= 35
    for name, v in vals.items():
        if name.startswith("RAY_"):
            assert cloak.RAY_STATUS[v] == name[4:], name
        else:
            assert getattr(cloak, name) == v, name


def test_fma_peak_rejects_bad_arguments_on_host(lib):
    flops = C.c_double(0.0)
    sink = C.c_void_p(16)  # never dereferenced: every call below fails its argument check before a launch
    assert lib.cloak_fma_peak(7, 1, 32, 1, sink, C.byref(flops), None) == 1   # not FP64 / FP32
    assert lib.cloak_fma_peak(0, 0, 32, 1, sink, C.byref(flops), None) == 1   # no blocks
    assert lib.cloak_fma_peak(0, 1, 48, 1, sink, C.byref(flops), None) == 1   # not a multiple of 32
    assert lib.cloak_fma_peak(0, 1, 512, 1, sink, C.byref(flops), None) == 1  # above 256 threads
    assert lib.cloak_fma_peak(0, 1, 32, 0, sink, C.byref(flops), None) == 1   # no iterations
    assert lib.cloak_fma_peak(0, 1, 32, 1, None, C.byref(flops), None) == 1   # no sink
    assert b"cloak_fma_peak" in lib.cloak_last_error()
