"""Thin ctypes binding of the fde_hodlr C ABI (include/fde_hodlr.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
Device buffers are passed as integer addresses (e.g. torch.Tensor.data_ptr()),
streams as integer cudaStream_t handles.  If the shared library has not been
built, load() raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libfde_hodlr.so")

FDE_OK, FDE_ERR_ARG, FDE_ERR_NOMEM, FDE_ERR_NOCONV, FDE_ERR_NUMERIC, FDE_ERR_CUDA = range(6)
FDE_FP64, FDE_FP32_REFINE, FDE_BF16_REFINE = 0, 1, 2


class OpParams(C.Structure):
    _fields_ = [("N", C.c_int), ("alpha", C.c_double), ("h", C.c_double), ("dt", C.c_double),
                ("shift", C.c_double), ("d_plus", C.c_void_p), ("d_minus", C.c_void_p),
                ("leaf", C.c_int), ("tol", C.c_double)]


class HodlrInfo(C.Structure):
    _fields_ = [("N", C.c_int), ("leaf", C.c_int), ("levels", C.c_int), ("nleaves", C.c_int),
                ("kmax", C.c_int), ("aca_rank", C.c_int), ("aca_converged", C.c_int),
                ("norm2", C.c_double), ("c", C.c_double), ("aca_tol", C.c_double)]


class RefineParams(C.Structure):
    _fields_ = [("max_sweeps", C.c_int), ("tol_update", C.c_double), ("tol_relres", C.c_double),
                ("fixed_sweeps", C.c_int)]


class RunParams(C.Structure):
    _fields_ = [("dim", C.c_int), ("op_x", OpParams), ("op_y", OpParams), ("steps", C.c_int),
                ("rank", C.c_int), ("h_src_left", C.c_void_p), ("h_src_right", C.c_void_p),
                ("h_amp", C.c_void_p), ("h_sin_amp", C.c_void_p), ("h_omega", C.c_void_p),
                ("prec", C.c_int), ("use_graph", C.c_int)]


class RunStats(C.Structure):
    _fields_ = [("setup_s", C.c_double), ("solve_s", C.c_double), ("steps_per_s", C.c_double),
                ("sweeps_total", C.c_int), ("sweeps_max", C.c_int), ("relres_max", C.c_double),
                ("kmax_x", C.c_int), ("kmax_y", C.c_int)]


class BatchOpts(C.Structure):
    _fields_ = [("threads", C.c_int), ("autotune", C.c_int)]


_P = C.c_void_p
_SIGS = {
    "hodlr_build": ([C.POINTER(OpParams), _P, C.POINTER(_P)], C.c_int),
    "hodlr_factor": ([_P, _P], C.c_int),
    "hodlr_solve": ([_P, _P, _P, C.c_int, C.c_int, _P], C.c_int),
    "hodlr_matvec": ([_P, _P, _P, C.c_int, C.c_int, _P], C.c_int),
    "hodlr_matvec_noalloc": ([_P, _P, _P, C.c_int, C.c_int, _P], C.c_int),
    "fde_runner_step_source": ([_P, _P, C.c_int, _P], C.c_int),
    "fde_batch_create": ([_P, _P, C.c_int, _P, _P, C.POINTER(_P)], C.c_int),
    "fde_batch_advance": ([_P, C.c_int], C.c_int),
    "fde_batch_state": ([_P, C.c_int, _P, _P], C.c_int),
    "fde_batch_info": ([_P, C.c_int, C.POINTER(C.c_int), _P], C.c_int),
    "fde_batch_timing": ([_P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                          C.POINTER(C.c_longlong)], C.c_int),
    "fde_batch_free": ([_P], None),
    "fde_gemm_f32": ([C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float, _P, C.c_int, C.c_longlong, _P, C.c_int,
                      C.c_longlong, C.c_float, _P, C.c_int, C.c_longlong, C.c_int, C.c_int, C.c_longlong, C.c_int, _P],
                     C.c_int),
    "hodlr_get_info": ([_P, C.POINTER(HodlrInfo)], C.c_int),
    "hodlr_to_dense": ([_P, _P, C.c_int, _P], C.c_int),
    "hodlr_get_weights": ([_P, _P], C.c_int),
    "hodlr_get_aca_pivots": ([_P, _P, _P, C.c_int, C.POINTER(C.c_int)], C.c_int),
    "hodlr_get_tree": ([_P, _P, _P, C.c_int], C.c_int),
    "hodlr_free": ([_P], None),
    "fde_tree_layout": ([C.c_int, C.c_int, _P, _P, C.c_int, C.POINTER(C.c_int)], C.c_int),
    "sylv_create": ([_P, _P, C.c_int, _P, C.POINTER(_P)], C.c_int),
    "sylv_get_refine": ([_P, C.POINTER(RefineParams)], C.c_int),
    "sylv_set_refine": ([_P, C.POINTER(RefineParams)], C.c_int),
    "sylv_step": ([_P, _P, _P, C.c_int, _P, C.POINTER(C.c_double), C.POINTER(C.c_int)], C.c_int),
    "sylv_inner_solve": ([_P, _P, _P, C.c_int, _P], C.c_int),
    "sylv_residual": ([_P, _P, _P, _P, C.c_int, _P], C.c_int),
    "sylv_flop_model": ([_P, C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
    "sylv_free": ([_P], None),
    "fde_block_interval": ([C.POINTER(OpParams), C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)],
                           C.c_int),
    "fde_fadi_shifts": ([C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.POINTER(C.c_int), _P,
                         _P, C.POINTER(C.c_double)], C.c_int),
    "fde_run": ([C.POINTER(RunParams), _P, _P, _P, C.POINTER(RunStats)], C.c_int),
    "fde_runner_create": ([C.POINTER(RunParams), _P, _P, C.POINTER(_P)], C.c_int),
    "fde_runner_advance": ([_P, C.c_int, _P], C.c_int),
    "fde_runner_load": ([_P, _P, C.c_int, _P], C.c_int),
    "fde_runner_state": ([_P, _P, _P], C.c_int),
    "fde_runner_residual": ([_P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double), _P],
                            C.c_int),
    "fde_runner_set_coefficients": ([_P, _P, _P, _P, _P, _P], C.c_int),
    "fde_runner_flop_model": ([_P, C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
    "fde_runner_step_source_async": ([_P, _P, C.c_int, _P], C.c_int),
    "fde_runner_state_async": ([_P, _P, _P], C.c_int),
    "fde_runner_sync": ([_P, _P], C.c_int),
    "fde_lowrank_create": ([_P, _P, _P, C.c_int, C.c_double, _P, _P], C.c_int),
    "fde_lowrank_advance": ([_P, C.c_int, _P], C.c_int),
    "fde_lowrank_factors": ([_P, _P, _P, C.c_int, C.POINTER(C.c_int), _P], C.c_int),
    "fde_lowrank_info": ([_P, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "fde_lowrank_free": ([_P], None),
    "fde_runner_stats": ([_P, C.POINTER(RunStats)], C.c_int),
    "fde_runner_free": ([_P], None),
    "fde_launch_count": ([], C.c_ulonglong),
    "fde_prof_enable": ([C.c_int], None),
    "fde_prof_query": ([C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.POINTER(C.c_double),
                        C.POINTER(C.c_int)], C.c_int),
    "fde_prof_reset": ([], None),
    "fde_fail_alloc_after": ([C.c_longlong], None),
    "fde_set_wait_limit": ([C.c_uint], C.c_int),
    "fde_strerror": ([C.c_int], C.c_char_p),
    "fde_last_error": ([], C.c_char_p),
}


class FdeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"fde status {status}: {msg}")
        self.status = status


class Lib:
    """Loaded library with checked wrappers named after the C entry points."""

    def __init__(self, path: str = LIB_PATH):
        if not os.path.exists(path):
            raise RuntimeError(f"fde_hodlr library not built ({path}); run __graft_entry__.build()")
        self.dll = C.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(self.dll, name)
            fn.argtypes = args
            fn.restype = res
        self._keep = []

    # -- error handling
    def check(self, status: int):
        if status != FDE_OK:
            raise FdeError(status, self.dll.fde_last_error().decode())
        return status

    def last_error(self) -> str:
        return self.dll.fde_last_error().decode()

    # -- parameter marshalling
    def op_params(self, op, d_plus=None, d_minus=None) -> OpParams:
        """fde_op_params from an inputs.OpSpec (coefficients passed as host arrays
        unless device addresses are given)."""
        dp = np.ascontiguousarray(op.d_plus, dtype=np.float64)
        dm = np.ascontiguousarray(op.d_minus, dtype=np.float64)
        self._keep += [dp, dm]
        p = OpParams(op.N, op.alpha, op.h, op.dt, op.shift,
                     d_plus if d_plus is not None else dp.ctypes.data,
                     d_minus if d_minus is not None else dm.ctypes.data, op.leaf, op.tol)
        p._arrays = (dp, dm)
        return p

    # -- HODLR
    def hodlr_build(self, params: OpParams, stream: int = 0) -> int:
        h = _P()
        self.check(self.dll.hodlr_build(C.byref(params), stream, C.byref(h)))
        return h.value

    def hodlr_build_status(self, params: OpParams, stream: int = 0):
        h = _P()
        s = self.dll.hodlr_build(C.byref(params), stream, C.byref(h))
        return s, h.value

    def hodlr_factor(self, h: int, stream: int = 0):
        self.check(self.dll.hodlr_factor(h, stream))

    def hodlr_solve(self, h: int, b: int, x: int, nrhs: int, ldb: int, stream: int = 0):
        self.check(self.dll.hodlr_solve(h, b, x, nrhs, ldb, stream))

    def hodlr_matvec(self, h: int, x: int, y: int, nrhs: int, ldx: int, stream: int = 0):
        self.check(self.dll.hodlr_matvec(h, x, y, nrhs, ldx, stream))

    def gemm_f32(self, ta, tb, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, Cm, ldc, sC, batch=1, kblk=0, kstr=0,
                 mode=-1, stream: int = 0):
        self.check(self.dll.fde_gemm_f32(int(ta), int(tb), m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, Cm, ldc, sC,
                                         batch, kblk, kstr, mode, stream))

    def hodlr_matvec_noalloc(self, h: int, x: int, y: int, nrhs: int, ldx: int, stream: int = 0):
        self.check(self.dll.hodlr_matvec_noalloc(h, x, y, nrhs, ldx, stream))

    def hodlr_get_info(self, h: int) -> HodlrInfo:
        info = HodlrInfo()
        self.check(self.dll.hodlr_get_info(h, C.byref(info)))
        return info

    def hodlr_to_dense(self, h: int, A: int, ld: int, stream: int = 0):
        self.check(self.dll.hodlr_to_dense(h, A, ld, stream))

    def hodlr_get_weights(self, h: int, N: int) -> np.ndarray:
        g = np.zeros(N + 2)
        self.check(self.dll.hodlr_get_weights(h, g.ctypes.data))
        return g

    def hodlr_get_aca_pivots(self, h: int, cap: int = 512):
        r = np.zeros(cap, dtype=np.int32)
        c = np.zeros(cap, dtype=np.int32)
        k = C.c_int()
        self.check(self.dll.hodlr_get_aca_pivots(h, r.ctypes.data, c.ctypes.data, cap, C.byref(k)))
        return r[:k.value].copy(), c[:k.value].copy()

    def hodlr_get_tree(self, h: int, levels: int):
        n = (1 << (levels + 1)) - 1
        lo = np.zeros(n, dtype=np.int32)
        hi = np.zeros(n, dtype=np.int32)
        self.check(self.dll.hodlr_get_tree(h, lo.ctypes.data, hi.ctypes.data, n))
        return lo, hi

    def hodlr_free(self, h: int):
        if h:
            self.dll.hodlr_free(h)

    def fde_tree_layout(self, N: int, leaf: int):
        """(levels, lo, hi): the host-side tree of hodlr_build, nodes in level order."""
        L = C.c_int()
        self.dll.fde_tree_layout(N, leaf, None, None, 0, C.byref(L))  # depth first
        n = (1 << (L.value + 1)) - 1
        lo = np.zeros(n, dtype=np.int32)
        hi = np.zeros(n, dtype=np.int32)
        self.check(self.dll.fde_tree_layout(N, leaf, lo.ctypes.data, hi.ctypes.data, n, C.byref(L)))
        return L.value, lo, hi

    # -- Sylvester
    def sylv_create(self, ax: int, ay: int, prec: int, stream: int = 0) -> int:
        s = _P()
        self.check(self.dll.sylv_create(ax, ay, prec, stream, C.byref(s)))
        return s.value

    def sylv_get_refine(self, s: int) -> RefineParams:
        r = RefineParams()
        self.check(self.dll.sylv_get_refine(s, C.byref(r)))
        return r

    def sylv_set_refine(self, s: int, r: RefineParams):
        self.check(self.dll.sylv_set_refine(s, C.byref(r)))

    def sylv_step(self, s: int, Cp: int, Xp: int, ld: int, stream: int = 0):
        rr = C.c_double()
        sw = C.c_int()
        self.check(self.dll.sylv_step(s, Cp, Xp, ld, stream, C.byref(rr), C.byref(sw)))
        return rr.value, sw.value

    def sylv_inner_solve(self, s: int, Cp: int, Xp: int, ld: int, stream: int = 0):
        self.check(self.dll.sylv_inner_solve(s, Cp, Xp, ld, stream))

    def sylv_residual(self, s: int, Cp: int, Xp: int, Rp: int, ld: int, stream: int = 0):
        self.check(self.dll.sylv_residual(s, Cp, Xp, Rp, ld, stream))

    def sylv_free(self, s: int):
        if s:
            self.dll.sylv_free(s)

    # -- fADI shift selection (host only)
    def fde_block_interval(self, params: OpParams, lo: int, hi: int):
        a, b = C.c_double(), C.c_double()
        self.check(self.dll.fde_block_interval(C.byref(params), lo, hi, C.byref(a), C.byref(b)))
        return a.value, b.value

    def fde_fadi_shifts(self, a: float, b: float, c: float, d: float, target: float, jmax: int = 64):
        al = np.zeros(max(jmax, 1))
        be = np.zeros(max(jmax, 1))
        J = C.c_int()
        r = C.c_double()
        self.check(self.dll.fde_fadi_shifts(a, b, c, d, target, jmax, C.byref(J), al.ctypes.data, be.ctypes.data,
                                            C.byref(r)))
        return al[:J.value].copy(), be[:J.value].copy(), r.value

    # -- time loop
    def run_params(self, w, prec: int = FDE_FP64, use_graph: int = 0) -> RunParams:
        px = self.op_params(w.ops[0])
        py = self.op_params(w.ops[1]) if w.dim == 2 else OpParams()
        FL = np.asfortranarray(w.src_left, dtype=np.float64)
        FR = np.asfortranarray(w.src_right if w.src_right is not None else np.zeros((1, 1)), dtype=np.float64)
        amp = np.ascontiguousarray(w.src_amp, dtype=np.float64)
        sa = np.ascontiguousarray(w.src_sin_amp, dtype=np.float64)
        om = np.ascontiguousarray(w.src_omega, dtype=np.float64)
        rp = RunParams(w.dim, px, py, w.steps, FL.shape[1], FL.ctypes.data, FR.ctypes.data,
                       amp.ctypes.data, sa.ctypes.data, om.ctypes.data, prec, use_graph)
        rp._arrays = (px, py, FL, FR, amp, sa, om)
        return rp

    def fde_run(self, params: RunParams, U0: int, Uout: int, stream: int = 0) -> RunStats:
        st = RunStats()
        self.check(self.dll.fde_run(C.byref(params), U0, Uout, stream, C.byref(st)))
        return st


    # -- runner (stateful time loop)
    def runner_create(self, params: RunParams, U0: int, stream: int = 0) -> int:
        r = _P()
        self.check(self.dll.fde_runner_create(C.byref(params), U0, stream, C.byref(r)))
        return r.value

    # -- factored 2D loop
    def lowrank_create(self, params: RunParams, W0: np.ndarray, Z0: np.ndarray, eps: float, stream: int = 0) -> int:
        W0 = np.asfortranarray(W0, dtype=np.float64)
        Z0 = np.asfortranarray(Z0, dtype=np.float64)
        h = _P()
        self.check(self.dll.fde_lowrank_create(C.byref(params), W0.ctypes.data, Z0.ctypes.data, W0.shape[1], eps,
                                               stream, C.byref(h)))
        return h.value

    def lowrank_advance(self, h: int, nsteps: int, stream: int = 0):
        self.check(self.dll.fde_lowrank_advance(h, nsteps, stream))

    def lowrank_factors(self, h: int, N: int, cap: int = 32, stream: int = 0):
        """(W, Z, rank): host copies of the factors, N x rank each."""
        W = np.zeros((cap, N))
        Z = np.zeros((cap, N))
        rk = C.c_int()
        self.check(self.dll.fde_lowrank_factors(h, W.ctypes.data, Z.ctypes.data, cap, C.byref(rk), stream))
        return W[:rk.value].T.copy(), Z[:rk.value].T.copy(), rk.value

    def lowrank_info(self, h: int):
        J, rm = C.c_int(), C.c_int()
        self.check(self.dll.fde_lowrank_info(h, C.byref(J), C.byref(rm)))
        return J.value, rm.value

    def lowrank_free(self, h: int):
        if h:
            self.dll.fde_lowrank_free(h)

    # -- batches
    def batch_create(self, params_list, U0_ptrs, threads=4, autotune=False, stream: int = 0) -> int:
        n = len(params_list)
        arr = (RunParams * n)(*params_list)
        ptrs = (C.c_void_p * n)(*U0_ptrs)
        opts = BatchOpts(threads, 1 if autotune else 0)
        h = _P()
        self.check(self.dll.fde_batch_create(C.cast(arr, _P), C.cast(ptrs, _P), n, C.byref(opts), stream,
                                             C.byref(h)))
        return h.value

    def batch_advance(self, b: int, nsteps: int):
        self.check(self.dll.fde_batch_advance(b, nsteps))

    def batch_state(self, b: int, i: int, U: int, stream: int = 0):
        self.check(self.dll.fde_batch_state(b, i, U, stream))

    def batch_info(self, b: int, i: int):
        leaf = C.c_int()
        st = RunStats()
        self.check(self.dll.fde_batch_info(b, i, C.byref(leaf), C.byref(st)))
        return leaf.value, st

    def batch_timing(self, b: int):
        a, t, s, n = C.c_double(), C.c_double(), C.c_double(), C.c_longlong()
        self.check(self.dll.fde_batch_timing(b, C.byref(a), C.byref(t), C.byref(s), C.byref(n)))
        return a.value, t.value, s.value, n.value

    def batch_free(self, b: int):
        if b:
            self.dll.fde_batch_free(b)

    def runner_step_source(self, r: int, F: int, ldf: int, stream: int = 0):
        self.check(self.dll.fde_runner_step_source(r, F, ldf, stream))

    def runner_step_source_async(self, r: int, F: int, ldf: int, stream: int = 0):
        self.check(self.dll.fde_runner_step_source_async(r, F, ldf, stream))

    def runner_state_async(self, r: int, U: int, stream: int = 0):
        self.check(self.dll.fde_runner_state_async(r, U, stream))

    def runner_sync(self, r: int, stream: int = 0):
        self.check(self.dll.fde_runner_sync(r, stream))

    def runner_advance(self, r: int, nsteps: int, stream: int = 0):
        self.check(self.dll.fde_runner_advance(r, nsteps, stream))

    def runner_load(self, r: int, U: int, step_index: int, stream: int = 0):
        self.check(self.dll.fde_runner_load(r, U, step_index, stream))

    def runner_state(self, r: int, U: int, stream: int = 0):
        self.check(self.dll.fde_runner_state(r, U, stream))

    def runner_residual(self, r: int, stream: int = 0):
        """(||R||_F / ||C||_F, max |R_ij|, ||R||_F) of the last step, exact FP64."""
        rr, mx, fr = C.c_double(), C.c_double(), C.c_double()
        self.check(self.dll.fde_runner_residual(r, C.byref(rr), C.byref(mx), C.byref(fr), stream))
        return rr.value, mx.value, fr.value

    def runner_flop_model(self, r: int):
        """(method flops, implementation GEMM flops) of one refinement sweep."""
        a, b = C.c_double(), C.c_double()
        self.check(self.dll.fde_runner_flop_model(r, C.byref(a), C.byref(b)))
        return a.value, b.value

    def sylv_flop_model(self, s: int):
        """(method flops, implementation GEMM flops) of one inner solve."""
        a, b = C.c_double(), C.c_double()
        self.check(self.dll.sylv_flop_model(s, C.byref(a), C.byref(b)))
        return a.value, b.value

    def runner_set_coefficients(self, r: int, dpx, dmx, dpy=None, dmy=None, stream: int = 0):
        """D_± of the next step (host arrays, or device addresses as ints)."""
        held = []  # host copies live until the call returns (it synchronises)

        def ptr(a):
            if a is None or isinstance(a, int):
                return a
            a = np.ascontiguousarray(a, dtype=np.float64)
            held.append(a)
            return a.ctypes.data
        self.check(self.dll.fde_runner_set_coefficients(r, ptr(dpx), ptr(dmx), ptr(dpy), ptr(dmy), stream))

    def runner_stats(self, r: int) -> RunStats:
        st = RunStats()
        self.check(self.dll.fde_runner_stats(r, C.byref(st)))
        return st

    def runner_free(self, r: int):
        if r:
            self.dll.fde_runner_free(r)

    # -- failure injection (tests of the error paths)
    def fail_alloc_after(self, n: int):
        self.dll.fde_fail_alloc_after(n)

    def set_wait_limit(self, iters: int):
        self.check(self.dll.fde_set_wait_limit(iters))

    # -- instrumentation
    def launch_count(self) -> int:
        return int(self.dll.fde_launch_count())

    def prof_enable(self, on: bool):
        self.dll.fde_prof_enable(1 if on else 0)

    def prof_query(self, family: str):
        """(device ms, launches, algorithmic work, kind) with kind 1 = FLOPs, 0 = bytes."""
        ms = C.c_double()
        n = C.c_longlong()
        w = C.c_double()
        k = C.c_int()
        self.check(self.dll.fde_prof_query(family.encode(), C.byref(ms), C.byref(n), C.byref(w), C.byref(k)))
        return ms.value, n.value, w.value, k.value

    def prof_reset(self):
        self.dll.fde_prof_reset()


_LIB = None


def load(path: str = LIB_PATH) -> Lib:
    global _LIB
    if _LIB is None:
        _LIB = Lib(path)
    return _LIB


def exported_symbols():
    return list(_SIGS)
