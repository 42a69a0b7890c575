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


def test_refused_calls_launch_nothing(cpu_lib):
    # argument errors are caught on the host before any launch: the library's
    # launch counter does not move
    c0 = cpu_lib.dll.fde_launch_count()
    p = cpu_lib.op_params(I.fd1d(N=128).ops[0])
    p.alpha = 3.0
    s, h = cpu_lib.hodlr_build_status(p)
    assert s == binding.FDE_ERR_ARG and not h
    assert cpu_lib.dll.fde_run(None, None, None, None, None) == binding.FDE_ERR_ARG
    assert cpu_lib.dll.fde_launch_count() == c0


def test_prof_query_unknown_family_is_empty(cpu_lib):
    ms, n = ctypes.c_double(-1.0), ctypes.c_longlong(-1)
    assert cpu_lib.dll.fde_prof_query(b"no_such_family", ctypes.byref(ms), ctypes.byref(n), None, None) == 0
    assert ms.value == 0.0 and n.value == 0
    assert cpu_lib.dll.fde_prof_query(None, ctypes.byref(ms), ctypes.byref(n), None, None) == binding.FDE_ERR_ARG


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
    assert cpu_lib.dll.sylv_set_refine(None, None) == binding.FDE_ERR_ARG
    assert cpu_lib.dll.sylv_get_refine(None, None) == binding.FDE_ERR_ARG
    assert cpu_lib.dll.fde_runner_load(None, None, 0, None) == binding.FDE_ERR_ARG
    assert cpu_lib.dll.fde_runner_state(None, None, None) == binding.FDE_ERR_ARG


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


def test_tree_layout_matches_oracle(cpu_lib):
    """The host tree of hodlr_build against the oracle's split rule
    (Eq. (HODLRpart)), bit for bit, over many sizes including ragged ones."""
    from oracle import fde_oracle as O

    rng = np.random.default_rng(1804)
    cases = [(1, 8), (2, 8), (8, 8), (9, 8), (1000, 64), (1024, 64), (1025, 64), (4096, 128), (16384, 256),
             (12345, 100), (65, 64), (129, 64)]
    cases += [(int(n), int(l)) for n, l in zip(rng.integers(2, 20000, 60), rng.integers(1, 300, 60))]
    for N, leaf in cases:
        L, lo, hi = cpu_lib.fde_tree_layout(N, leaf)
        tree = O.hodlr_tree(N, leaf)
        assert L == len(tree) - 1, (N, leaf)
        flat = [node for lvl in tree for node in lvl]
        assert list(zip(lo.tolist(), hi.tolist())) == flat, (N, leaf)


def test_tree_layout_rejects_bad_arguments(cpu_lib):
    L = ctypes.c_int()
    lo = np.zeros(4, dtype=np.int32)
    hi = np.zeros(4, dtype=np.int32)
    assert cpu_lib.dll.fde_tree_layout(0, 8, lo.ctypes.data, hi.ctypes.data, 4, ctypes.byref(L)) == binding.FDE_ERR_ARG
    assert cpu_lib.dll.fde_tree_layout(64, 0, lo.ctypes.data, hi.ctypes.data, 4, ctypes.byref(L)) == binding.FDE_ERR_ARG
    # 100 / 16: three levels need 15 nodes, 4 are too few; the depth is still reported
    assert cpu_lib.dll.fde_tree_layout(100, 16, lo.ctypes.data, hi.ctypes.data, 4, ctypes.byref(L)) == binding.FDE_ERR_ARG
    assert L.value == 3


def test_injected_allocation_failure_is_nomem(cpu_lib):
    """The host-side allocation hook: hodlr_build's first device allocation
    fails as if the device were out of memory; the call returns
    FDE_ERR_NOMEM before any launch, and the hook disarms itself."""
    c0 = cpu_lib.dll.fde_launch_count()
    p = cpu_lib.op_params(I.fd1d(N=128).ops[0])
    cpu_lib.fail_alloc_after(0)
    try:
        s, h = cpu_lib.hodlr_build_status(p)
    finally:
        cpu_lib.fail_alloc_after(-1)
    assert s == binding.FDE_ERR_NOMEM and not h
    assert "injected" in cpu_lib.last_error()
    assert cpu_lib.dll.fde_launch_count() == c0
