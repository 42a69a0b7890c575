"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point declared in include/fde_hodlr.h, and rejects bad arguments
before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1804_05522_gb300 import binding
from paper_1804_05522_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:fde_status|void|const char\*|unsigned long long)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def cpu_lib():
    from paper_1804_05522_gb300 import build

    build.build()  # incremental: recompiles only what changed since the last build
    return binding.load()


def test_exports_every_declared_symbol(cpu_lib):
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(cpu_lib.dll, name), name
    assert set(declared) == set(binding.exported_symbols())


def test_strerror(cpu_lib):
    for s in range(6):
        assert cpu_lib.dll.fde_strerror(s)


@pytest.mark.parametrize("field,value", [("N", 1), ("alpha", 1.0), ("alpha", 2.5), ("leaf", 4), ("leaf", 512),
                                         ("tol", 0.0), ("tol", 1.0), ("h", -1.0), ("dt", 0.0), ("shift", 0.0)])
def test_bad_parameters_rejected_on_host(cpu_lib, field, value):
    op = I.fd1d(N=128).ops[0]
    p = cpu_lib.op_params(op)
    setattr(p, field, value)
    s, h = cpu_lib.hodlr_build_status(p)
    assert s == binding.FDE_ERR_ARG and not h
    assert "argument" in cpu_lib.last_error()


def test_null_arguments_rejected(cpu_lib):
    assert cpu_lib.dll.hodlr_factor(None, None) == binding.FDE_ERR_ARG
    assert cpu_lib.dll.hodlr_solve(None, None, None, 1, 1, None) == binding.FDE_ERR_ARG
    assert cpu_lib.dll.sylv_step(None, None, None, 1, None, None, None) == binding.FDE_ERR_ARG
    assert cpu_lib.dll.fde_run(None, None, None, None, None) == binding.FDE_ERR_ARG


@pytest.mark.parametrize("dim,shifts", [(1, (0.5, None)), (2, (1.0, 0.5)), (2, (0.5, 1.0))])
def test_time_loop_rejects_wrong_shift(cpu_lib, dim, shifts):
    """The time loop is implicit Euler: shift 1 in 1D (Eq. (system_FD)), 1/2 per
    side in 2D (Eq. (sylv-timestepping)); anything else is refused on the host."""
    w = I.fd1d(N=64) if dim == 1 else I.fd2d(N=64, leaf=16)
    rp = cpu_lib.run_params(w)
    rp.op_x.shift = shifts[0]
    if dim == 2:
        rp.op_y.shift = shifts[1]
    with pytest.raises(binding.FdeError) as e:
        cpu_lib.fde_run(rp, 1, 1)  # never dereferenced: the check comes first
    assert e.value.status == binding.FDE_ERR_ARG and "shift" in str(e.value)
