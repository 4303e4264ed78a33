"""The C-ABI library builds, loads and exports every symbol include/pe.h declares.

Runs without a GPU: only argument validation that fails before any device
work is exercised (no compute call).
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2412_01138_gb300 import build, pe

    build.build()
    return pe.lib()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            # function declarations: "<return type> pe_name(" at the start of a line
            names |= set(re.findall(r"^(?:pe_status|void|int32_t|const char\*)\s+(pe_[a-z0-9_]+)\(", text, re.M))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert declared, "no declarations found"
    for name in sorted(declared):
        assert hasattr(lib, name), name
    from paper_2412_01138_gb300 import pe
    assert set(pe.EXPORTED) == declared


def test_invalid_setup_arguments_rejected_before_device_work(lib):
    from paper_2412_01138_gb300 import pe

    ctx = C.c_void_p()
    n = (C.c_int32 * 1)(15)
    box = (C.c_double * 2)(0.0, 1.0)
    good = pe.pe_tableau(2, None, 0, 0)
    cases = [
        dict(d=0), dict(d=4), dict(D=0.0), dict(D=-1.0), dict(T=0.0), dict(N=0), dict(M=0),
    ]
    for kw in cases:
        args = dict(d=1, D=1.0, T=1.0, N=4, M=4)
        args.update(kw)
        st = lib.pe_setup(C.byref(ctx), args["d"], n, box, args["D"], 0.0, args["T"], args["N"], args["M"],
                          C.byref(good), C.byref(good), None)
        assert st == pe.PE_EINVAL, kw
        assert lib.pe_last_error().decode()
    # duplicate interpolation nodes (the Lagrange basis of Eq. (3-12) needs distinct nodes)
    c = (C.c_double * 2)(0.5, 0.5)
    dup = pe.pe_tableau(2, C.cast(c, C.POINTER(C.c_double)), 0, 0)
    st = lib.pe_setup(C.byref(ctx), 1, n, box, 1.0, 0.0, 1.0, 4, 4, C.byref(dup), C.byref(good), None)
    assert st == pe.PE_EINVAL and "distinct" in lib.pe_last_error().decode()
    # box with lo >= hi
    bad_box = (C.c_double * 2)(1.0, 1.0)
    st = lib.pe_setup(C.byref(ctx), 1, n, bad_box, 1.0, 0.0, 1.0, 4, 4, C.byref(good), C.byref(good), None)
    assert st == pe.PE_EINVAL
    # NULL context pointers are rejected
    assert lib.pe_parareal_iter(None, None) == pe.PE_EINVAL
    assert lib.pe_dst(0, n, None, None, None) == pe.PE_EINVAL


def _header_struct_fields(name):
    """Field names of `typedef struct { ... } name;` in include/pe.h, in declaration order."""
    import os
    import re

    src = open(os.path.join(os.path.dirname(__file__), "..", "include", "pe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    m = re.search(r"typedef struct\s*\{([^{}]*)\}\s*" + name + r"\s*;", src, re.S)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        fp = re.search(r"\(\s*\*\s*(\w+)\s*\)\s*\(", decl)  # function pointer: ret (*name)(args)
        if fp:
            fields.append(fp.group(1))
            continue
        for part in decl.split(","):  # "int32_t a, b" declares a and b
            fields.append(re.search(r"(\w+)\s*(\[[^\]]*\])*\s*$", part.strip()).group(1))
    return fields


@pytest.mark.parametrize("name", ["pe_options", "pe_term", "pe_tableau", "pe_field", "pe_forcing", "pe_result"])
def test_python_struct_mirrors_match_the_header(name):
    """The ctypes mirrors of the C-ABI structs list the header's fields in the same order."""
    from paper_2412_01138_gb300 import pe

    assert [f for f, _ in getattr(pe, name)._fields_] == _header_struct_fields(name)


def test_measurement_calls_reject_bad_arguments_before_device_work(lib):
    from paper_2412_01138_gb300 import pe

    out = C.c_double()
    assert lib.pe_measure_fma_peak(7, C.byref(out), None) == pe.PE_EINVAL
    assert lib.pe_measure_fma_peak(pe.PE_FP64, None, None) == pe.PE_EINVAL
    for budget in (0, -5, 10**9):
        assert lib.pe_probe_wait_timeout(budget, None) == pe.PE_EINVAL
        assert "budget" in lib.pe_last_error().decode()
    assert lib.pe_probe_widen_f32(None, None, -1, None) == pe.PE_EINVAL
    assert lib.pe_probe_widen_f32(None, None, 4, None) == pe.PE_EINVAL
    assert lib.pe_probe_widen_f32(None, None, 0, None) == pe.PE_OK


def test_transform_wrappers_check_buffers_before_the_library_sees_them(lib):
    """Host arrays, a wrong dtype or a buffer shorter than prod(n) never reach the kernels."""
    import numpy as np

    from paper_2412_01138_gb300 import pe

    host = np.zeros(64)
    for fn, kw in ((pe.dst, {}), (pe.dst, {"f32": True}), (pe.dst_noalloc, {}), (pe.dst_tc, {})):
        with pytest.raises(ValueError):
            fn(2, (8, 8), host, host, **kw)
    with pytest.raises(ValueError):
        pe.dst(2, (8,), host, host)  # len(n) != d


def test_solver_output_buffers_are_checked_in_the_binding():
    """pe_solve_out / pe_solve_async receive only float64 buffers of at least ndof values (host
    arrays here; device tensors take the same checks), checked before any call."""
    import numpy as np

    from paper_2412_01138_gb300 import pe

    pe._check_out(np.empty(10), 10)
    pe._check_out(np.empty(12), 10)
    for bad in (np.empty(9), np.empty(10, dtype=np.float32), np.empty(10, dtype=np.int64)):
        with pytest.raises(ValueError):
            pe._check_out(bad, 10)
    with pytest.raises(TypeError):
        pe._check_out([0.0] * 10, 10)
