"""Thin Python binding of the C ABI in ``include/ffsrqr.h`` (argument marshalling only).

Every computation happens inside ``libffsrqr.so``; this module passes plain
pointers, sizes and a CUDA stream.  PyTorch provides device memory and streams.
If the shared library is missing the import fails loudly: there is no CPU or
library fallback.

Names mirror the C ABI (``ffsrqr_plan``, ``ffsrqr_run``, ``ffsrqr_destroy``,
``ffsrqr_status_string``, ``ffsrqr_workspace_item``); ``Plan`` is a small
convenience wrapper that owns a torch workspace tensor.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

PLAIN_FP32 = 0
MIXED = 1            # FFSRQR_MIXED_TF32X3
MIXED_TF32X3 = 1
MIXED_BF16X3 = 2
FP64 = 3

STATUS = {0: "ok", 1: "rank_deficient", 2: "swap_cap", 3: "timeout", 4: "nonfinite",
          5: "workspace", 6: "cuda", 7: "unsupported"}

ITEM = {"omega": 0, "bt": 1, "s11": 2, "q1": 3, "gt": 4, "vp": 5, "tmp": 6, "r": 7, "mt": 8, "ctl": 9}


class Opts(ctypes.Structure):
    _fields_ = [("g", ctypes.c_double), ("max_swaps", ctypes.c_int32), ("flags", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("swaps", ctypes.c_int32),
                ("g2_first", ctypes.c_double), ("g2_final", ctypes.c_double),
                ("cand_first", ctypes.c_int32), ("jacobi_sweeps", ctypes.c_int32),
                ("alpha_first", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Problem(ctypes.Structure):
    """ffsrqr_problem_t: one problem of a batch (device pointers)."""
    _fields_ = [("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("U", ctypes.c_void_p), ("ldu", ctypes.c_int64), ("S", ctypes.c_void_p),
                ("V", ctypes.c_void_p), ("ldv", ctypes.c_int64), ("piv", ctypes.c_void_p)]


class Request(ctypes.Structure):
    """ffsrqr_request_t: one request of the server (device pointers)."""
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int32), ("p", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("reserved", ctypes.c_int32), ("A", ctypes.c_void_p),
                ("lda", ctypes.c_int64), ("seed", ctypes.c_uint64), ("U", ctypes.c_void_p),
                ("ldu", ctypes.c_int64), ("S", ctypes.c_void_p), ("V", ctypes.c_void_p),
                ("ldv", ctypes.c_int64), ("piv", ctypes.c_void_p)]


class HostProblem(ctypes.Structure):
    """ffsrqr_host_problem_t: one problem of a pipe (host pointers)."""
    _fields_ = [("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("U", ctypes.c_void_p), ("ldu", ctypes.c_int64), ("S", ctypes.c_void_p),
                ("V", ctypes.c_void_p), ("ldv", ctypes.c_int64), ("piv", ctypes.c_void_p)]


class RpcaOpts(ctypes.Structure):
    """ffsrqr_rpca_opts_t."""
    _fields_ = [("mode", ctypes.c_int32), ("p", ctypes.c_int32), ("sv0", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("kmax", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("lambda_", ctypes.c_double), ("rho", ctypes.c_double), ("mu_bar_ratio", ctypes.c_double),
                ("tol", ctypes.c_double)]


class RpcaInfo(ctypes.Structure):
    """ffsrqr_rpca_info_t."""
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("rank", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("rel_residual", ctypes.c_double), ("nnz_e", ctypes.c_int64),
                ("norm2", ctypes.c_double), ("lambda_", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libffsrqr.so not built ({path}); run __graft_entry__.build() "
                           "or python -m paper_1803_01982_gb300.build")
    lib = ctypes.CDLL(path)
    P, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
    lib.ffsrqr_plan.argtypes = [ctypes.POINTER(P), i64, i64, i32, i32, i32, ctypes.POINTER(Opts),
                                ctypes.POINTER(ctypes.c_size_t)]
    lib.ffsrqr_plan.restype = ctypes.c_int
    lib.ffsrqr_plan_l.argtypes = [ctypes.POINTER(P), i64, i64, i32, i32, i32, i32, ctypes.POINTER(Opts),
                                  ctypes.POINTER(ctypes.c_size_t)]
    lib.ffsrqr_plan_l.restype = ctypes.c_int
    lib.ffsrqr_plan_rsi.argtypes = [ctypes.POINTER(P), i64, i64, i32, i32, i32, i32, ctypes.POINTER(Opts),
                                    ctypes.POINTER(ctypes.c_size_t)]
    lib.ffsrqr_plan_rsi.restype = ctypes.c_int
    lib.ffsrqr_plan_blocked.argtypes = [ctypes.POINTER(P), i64, i64, i32, i32, i32, i32, ctypes.POINTER(Opts),
                                        ctypes.POINTER(ctypes.c_size_t)]
    lib.ffsrqr_plan_blocked.restype = ctypes.c_int
    lib.ffsrqr_plan_depth.argtypes = [P]
    lib.ffsrqr_plan_depth.restype = ctypes.c_int
    lib.ffsrqr_run.argtypes = [P, P, i64, u64, P, i64, P, P, i64, P, P, P, ctypes.POINTER(Info)]
    lib.ffsrqr_run.restype = ctypes.c_int
    lib.ffsrqr_destroy.argtypes = [P]
    lib.ffsrqr_destroy.restype = ctypes.c_int
    lib.ffsrqr_status_string.argtypes = [ctypes.c_int]
    lib.ffsrqr_status_string.restype = ctypes.c_char_p
    lib.ffsrqr_last_cuda_error.argtypes = []
    lib.ffsrqr_last_cuda_error.restype = ctypes.c_char_p
    lib.ffsrqr_workspace_item.argtypes = [P, i32, ctypes.POINTER(ctypes.c_size_t),
                                          ctypes.POINTER(i64), ctypes.POINTER(i64),
                                          ctypes.POINTER(i64), ctypes.POINTER(i32)]
    lib.ffsrqr_workspace_item.restype = ctypes.c_int
    lib.ffsrqr_philox4x32_10.argtypes = [P, P, i32, P]
    lib.ffsrqr_philox4x32_10.restype = ctypes.c_int
    lib.ffsrqr_phase_times.argtypes = [P, ctypes.POINTER(ctypes.c_float), i32]
    lib.ffsrqr_phase_times.restype = ctypes.c_int
    lib.ffsrqr_phase_times_back.argtypes = [P, i32, ctypes.POINTER(ctypes.c_float), i32]
    lib.ffsrqr_phase_times_back.restype = ctypes.c_int
    lib.ffsrqr_plan_tune.argtypes = [P, P, i64, ctypes.c_uint64, P, i64, P, P, i64, P, P, P, ctypes.POINTER(i32),
                                     ctypes.POINTER(ctypes.c_float)]
    lib.ffsrqr_plan_tune.restype = ctypes.c_int
    lib.ffsrqr_plan_set_g2_rows.argtypes = [P, i32]
    lib.ffsrqr_plan_set_g2_rows.restype = ctypes.c_int
    lib.ffsrqr_launch_count.argtypes = [P]
    lib.ffsrqr_launch_count.restype = ctypes.c_int
    lib.ffsrqr_qrcp_static.argtypes = [P, i64, i32, i64, i32, P, P, P, P]
    lib.ffsrqr_qrcp_static.restype = ctypes.c_int
    lib.ffsrqr_batch_create.argtypes = [ctypes.POINTER(P), i32, P, P, P, P, i32, ctypes.POINTER(Opts), i32,
                                        ctypes.POINTER(ctypes.c_size_t)]
    lib.ffsrqr_batch_create.restype = ctypes.c_int
    lib.ffsrqr_batch_run.argtypes = [P, P, P, P, P]
    lib.ffsrqr_batch_run.restype = ctypes.c_int
    lib.ffsrqr_batch_tune.argtypes = [P, P, P, P, P, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float)]
    lib.ffsrqr_batch_tune.restype = ctypes.c_int
    lib.ffsrqr_batch_streams.argtypes = [P]
    lib.ffsrqr_batch_streams.restype = ctypes.c_int
    lib.ffsrqr_batch_set_phased.argtypes = [P, i32]
    lib.ffsrqr_batch_set_phased.restype = ctypes.c_int
    lib.ffsrqr_batch_phased.argtypes = [P]
    lib.ffsrqr_batch_phased.restype = ctypes.c_int
    lib.ffsrqr_batch_small_svd_launches.argtypes = [P]
    lib.ffsrqr_batch_small_svd_launches.restype = ctypes.c_int
    lib.ffsrqr_batch_workspace_offset.argtypes = [P, i32, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(P)]
    lib.ffsrqr_batch_workspace_offset.restype = ctypes.c_int
    lib.ffsrqr_batch_destroy.argtypes = [P]
    lib.ffsrqr_batch_destroy.restype = ctypes.c_int
    lib.ffsrqr_server_create.argtypes = [ctypes.POINTER(P), ctypes.c_size_t, i32, ctypes.POINTER(Opts)]
    lib.ffsrqr_server_create.restype = ctypes.c_int
    lib.ffsrqr_server_submit.argtypes = [P, ctypes.POINTER(Request), ctypes.POINTER(i64)]
    lib.ffsrqr_server_submit.restype = ctypes.c_int
    lib.ffsrqr_server_poll.argtypes = [P, i64, ctypes.POINTER(Info), ctypes.POINTER(ctypes.c_double)]
    lib.ffsrqr_server_poll.restype = ctypes.c_int
    lib.ffsrqr_server_wait.argtypes = [P, i64, ctypes.POINTER(Info), ctypes.POINTER(ctypes.c_double)]
    lib.ffsrqr_server_wait.restype = ctypes.c_int
    lib.ffsrqr_server_stats.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                        ctypes.POINTER(ctypes.c_size_t)]
    lib.ffsrqr_server_stats.restype = ctypes.c_int
    lib.ffsrqr_server_destroy.argtypes = [P]
    lib.ffsrqr_server_destroy.restype = ctypes.c_int
    lib.ffsrqr_server_set_phase_batch.argtypes = [P, i32]
    lib.ffsrqr_server_set_phase_batch.restype = ctypes.c_int
    lib.ffsrqr_server_pause.argtypes = [P, i32]
    lib.ffsrqr_server_pause.restype = ctypes.c_int
    lib.ffsrqr_server_phase_stats.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.ffsrqr_server_phase_stats.restype = ctypes.c_int
    lib.ffsrqr_pipe_create.argtypes = [ctypes.POINTER(P), P, ctypes.POINTER(ctypes.c_size_t)]
    lib.ffsrqr_pipe_create.restype = ctypes.c_int
    lib.ffsrqr_pipe_run.argtypes = [P, ctypes.POINTER(HostProblem), i32, P, P, P, ctypes.POINTER(Info)]
    lib.ffsrqr_pipe_run.restype = ctypes.c_int
    lib.ffsrqr_pipe_destroy.argtypes = [P]
    lib.ffsrqr_pipe_destroy.restype = ctypes.c_int
    lib.ffsrqr_plan_shape.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32),
                                      ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.ffsrqr_plan_shape.restype = ctypes.c_int
    lib.ffsrqr_tucker_plan.argtypes = [ctypes.POINTER(P), i32, i32, P, P, P, i32, i32, ctypes.POINTER(Opts),
                                       ctypes.POINTER(ctypes.c_size_t)]
    lib.ffsrqr_tucker_plan.restype = ctypes.c_int
    lib.ffsrqr_tucker_run.argtypes = [P, P, u64, P, P, P, P, P, P]
    lib.ffsrqr_tucker_run.restype = ctypes.c_int
    lib.ffsrqr_tucker_launch_count.argtypes = [P]
    lib.ffsrqr_tucker_launch_count.restype = ctypes.c_int
    lib.ffsrqr_tucker_destroy.argtypes = [P]
    lib.ffsrqr_tucker_destroy.restype = ctypes.c_int
    lib.ffsrqr_rpca_create.argtypes = [ctypes.POINTER(P), i64, i64, ctypes.POINTER(RpcaOpts),
                                       ctypes.POINTER(ctypes.c_size_t)]
    lib.ffsrqr_rpca_create.restype = ctypes.c_int
    lib.ffsrqr_rpca_run.argtypes = [P, P, i64, P, i64, P, i64, u64, P, P, ctypes.POINTER(RpcaInfo)]
    lib.ffsrqr_rpca_run.restype = ctypes.c_int
    lib.ffsrqr_rpca_launch_count.argtypes = [P]
    lib.ffsrqr_rpca_launch_count.restype = ctypes.c_int
    lib.ffsrqr_rpca_destroy.argtypes = [P]
    lib.ffsrqr_rpca_destroy.restype = ctypes.c_int
    return lib


lib = _load()

# The C names, re-exported unchanged.
ffsrqr_plan = lib.ffsrqr_plan
ffsrqr_plan_l = lib.ffsrqr_plan_l
ffsrqr_plan_depth = lib.ffsrqr_plan_depth
ffsrqr_plan_rsi = lib.ffsrqr_plan_rsi
ffsrqr_run = lib.ffsrqr_run
ffsrqr_destroy = lib.ffsrqr_destroy
ffsrqr_status_string = lib.ffsrqr_status_string
ffsrqr_last_cuda_error = lib.ffsrqr_last_cuda_error
ffsrqr_workspace_item = lib.ffsrqr_workspace_item
ffsrqr_philox4x32_10 = lib.ffsrqr_philox4x32_10
ffsrqr_phase_times = lib.ffsrqr_phase_times
ffsrqr_launch_count = lib.ffsrqr_launch_count
ffsrqr_plan_tune = lib.ffsrqr_plan_tune
ffsrqr_phase_times_back = lib.ffsrqr_phase_times_back
ffsrqr_batch_create = lib.ffsrqr_batch_create
ffsrqr_batch_run = lib.ffsrqr_batch_run
ffsrqr_batch_tune = lib.ffsrqr_batch_tune
ffsrqr_batch_streams = lib.ffsrqr_batch_streams
ffsrqr_batch_set_phased = lib.ffsrqr_batch_set_phased
ffsrqr_batch_phased = lib.ffsrqr_batch_phased
ffsrqr_batch_small_svd_launches = lib.ffsrqr_batch_small_svd_launches
ffsrqr_batch_workspace_offset = lib.ffsrqr_batch_workspace_offset
ffsrqr_batch_destroy = lib.ffsrqr_batch_destroy
ffsrqr_server_create = lib.ffsrqr_server_create
ffsrqr_server_submit = lib.ffsrqr_server_submit
ffsrqr_server_poll = lib.ffsrqr_server_poll
ffsrqr_server_wait = lib.ffsrqr_server_wait
ffsrqr_server_stats = lib.ffsrqr_server_stats
ffsrqr_server_destroy = lib.ffsrqr_server_destroy
ffsrqr_server_set_phase_batch = lib.ffsrqr_server_set_phase_batch
ffsrqr_server_pause = lib.ffsrqr_server_pause
ffsrqr_server_phase_stats = lib.ffsrqr_server_phase_stats
ffsrqr_qrcp_static = lib.ffsrqr_qrcp_static
ffsrqr_pipe_create = lib.ffsrqr_pipe_create
ffsrqr_pipe_run = lib.ffsrqr_pipe_run
ffsrqr_pipe_destroy = lib.ffsrqr_pipe_destroy
ffsrqr_plan_shape = lib.ffsrqr_plan_shape
ffsrqr_tucker_plan = lib.ffsrqr_tucker_plan
ffsrqr_tucker_run = lib.ffsrqr_tucker_run
ffsrqr_tucker_launch_count = lib.ffsrqr_tucker_launch_count
ffsrqr_tucker_destroy = lib.ffsrqr_tucker_destroy
ffsrqr_rpca_create = lib.ffsrqr_rpca_create
ffsrqr_rpca_run = lib.ffsrqr_rpca_run
ffsrqr_rpca_launch_count = lib.ffsrqr_rpca_launch_count
ffsrqr_rpca_destroy = lib.ffsrqr_rpca_destroy
TUCKER_STHOSVD = 0
TUCKER_HOSVD = 1


class FfsrqrError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        msg = lib.ffsrqr_status_string(rc).decode()
        if rc == 6:
            msg += ": " + lib.ffsrqr_last_cuda_error().decode()
        raise FfsrqrError(f"{what} returned {rc} ({msg})")


class Plan:
    """Plan + device workspace for one (m, n, k, p, mode) shape; l (>= k) is
    Alg. 9's SRQR depth (None: l = k).  rsi_q (not None): the plan runs
    randomized subspace iteration with that many iterations instead.  b (not
    None): TRQRCP's block size (Alg. 2; the sketch has b + p rows).  g2_rows
    (>= 1): Alg. 4's d-row random estimate of g2 instead of the exact one."""

    def __init__(self, m: int, n: int, k: int, p: int, mode: int = PLAIN_FP32, g: float = 2.0,
                 max_swaps: int | None = None, flags: int = 0, device=None, l: int | None = None,
                 rsi_q: int | None = None, g2_rows: int = 0, b: int | None = None):
        import torch
        self.m, self.n, self.k, self.p, self.mode = m, n, k, p, mode
        self.device = torch.device("cuda" if device is None else device)
        self.dtype = torch.float64 if mode == FP64 else torch.float32
        self.l = k if l is None else l
        opts = Opts(g, 4 * self.l if max_swaps is None else max_swaps, flags)
        self._h = ctypes.c_void_p()
        ws = ctypes.c_size_t()
        with torch.cuda.device(self.device):
            if b is not None:  # TRQRCP with block size b (Alg. 2)
                assert l is None and rsi_q is None
                _check(lib.ffsrqr_plan_blocked(ctypes.byref(self._h), m, n, k, b, p, mode, ctypes.byref(opts),
                                               ctypes.byref(ws)), "ffsrqr_plan_blocked")
            elif rsi_q is not None:  # randomized subspace iteration with rsi_q iterations
                _check(lib.ffsrqr_plan_rsi(ctypes.byref(self._h), m, n, k, p, rsi_q, mode, ctypes.byref(opts),
                                           ctypes.byref(ws)), "ffsrqr_plan_rsi")
            elif l is None:
                _check(lib.ffsrqr_plan(ctypes.byref(self._h), m, n, k, p, mode, ctypes.byref(opts),
                                       ctypes.byref(ws)), "ffsrqr_plan")
            else:
                _check(lib.ffsrqr_plan_l(ctypes.byref(self._h), m, n, k, l, p, mode, ctypes.byref(opts),
                                         ctypes.byref(ws)), "ffsrqr_plan_l")
            if g2_rows:
                self.set_g2_rows(g2_rows)
        self.workspace_bytes = ws.value
        self.workspace = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8,
                                     device=self.device)
        base = self.workspace.data_ptr()
        self._ws_off = (-base) % 256
        self._info_host = torch.zeros(ctypes.sizeof(Info), dtype=torch.uint8).pin_memory()

    def set_g2_rows(self, d: int) -> None:
        """0: exact g2 in the SRQR test; d >= 1: Alg. 4's d-row random estimate."""
        _check(lib.ffsrqr_plan_set_g2_rows(self._h, d), "ffsrqr_plan_set_g2_rows")
        self.g2_rows = d

    @property
    def ws_ptr(self) -> int:
        return self.workspace.data_ptr() + self._ws_off

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib.ffsrqr_destroy(h)
            self._h = None

    def outputs(self):
        import torch
        U = torch.empty(self.m, self.k, dtype=self.dtype, device=self.device)
        S = torch.empty(self.k, dtype=self.dtype, device=self.device)
        V = torch.empty(self.n, self.k, dtype=self.dtype, device=self.device)
        piv = torch.empty(self.n, dtype=torch.int32, device=self.device)
        return U, S, V, piv

    def run(self, A, seed: int = 0, out=None, stream=None):
        """Enqueue ffsrqr_run on ``stream`` (default: torch's current stream)."""
        import torch
        assert A.is_cuda and A.dtype == self.dtype and A.shape == (self.m, self.n)
        assert A.stride(1) == 1
        U, S, V, piv = out if out is not None else self.outputs()
        st = torch.cuda.current_stream(self.device) if stream is None else stream
        info_ptr = ctypes.cast(self._info_host.data_ptr(), ctypes.POINTER(Info))
        _check(lib.ffsrqr_run(self._h, A.data_ptr(), A.stride(0), seed, U.data_ptr(), U.stride(0),
                              S.data_ptr(), V.data_ptr(), V.stride(0), piv.data_ptr(), self.ws_ptr,
                              ctypes.c_void_p(st.cuda_stream), info_ptr), "ffsrqr_run")
        return U, S, V, piv

    def tune(self, A, seed: int = 0, out=None, stream=None):
        """Autotune the tensor-core launch configuration on A (ffsrqr_plan_tune);
        returns (config [stages of passes 1-3, Gram grid, all-stream-K flags of
        passes 1-3], best ms per run)."""
        import torch
        assert A.is_cuda and A.dtype == self.dtype and A.shape == (self.m, self.n)
        U, S, V, piv = out if out is not None else self.outputs()
        st = torch.cuda.current_stream(self.device) if stream is None else stream
        cfg, ms = (ctypes.c_int32 * 7)(), ctypes.c_float()
        _check(lib.ffsrqr_plan_tune(self._h, A.data_ptr(), A.stride(0), seed, U.data_ptr(), U.stride(0),
                                    S.data_ptr(), V.data_ptr(), V.stride(0), piv.data_ptr(), self.ws_ptr,
                                    ctypes.c_void_p(st.cuda_stream), cfg, ctypes.byref(ms)), "ffsrqr_plan_tune")
        return list(cfg), ms.value

    def info(self) -> dict:
        """Report of the last run (call after synchronising its stream)."""
        return Info.from_buffer_copy(bytes(self._info_host.numpy().tobytes())).as_dict()

    def item(self, name: str):
        """View of a workspace intermediate (see ffsrqr_workspace_item)."""
        import torch
        off = ctypes.c_size_t()
        r, c, ld = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        eb = ctypes.c_int32()
        _check(lib.ffsrqr_workspace_item(self._h, ITEM[name], ctypes.byref(off), ctypes.byref(r),
                                         ctypes.byref(c), ctypes.byref(ld), ctypes.byref(eb)),
               "ffsrqr_workspace_item")
        dt = torch.float64 if eb.value == 8 else (torch.int32 if name == "ctl" else torch.float32)
        start = self._ws_off + off.value
        nbytes = (r.value - 1) * ld.value * eb.value + c.value * eb.value
        raw = self.workspace[start:start + nbytes]
        flat = raw.view(dt)
        return torch.as_strided(flat, (r.value, c.value), (ld.value, 1))


PHASES = ["omega", "pass1_sketch", "qrcp", "panel_qr", "pass2_r12", "srqr_test", "swap_loop",
          "qr_rt", "pass3_tmp", "qr_tmp", "small_svd", "outputs",
          "tc_pass1_kernel", "tc_pass2_kernel", "tc_pass3_kernel"]
FLAG_CHECK_FINITE = 1
FLAG_PHASE_TIMES = 2
FLAG_TEST_STALL = 4


def phase_times(plan: "Plan", back: int = 0) -> dict:
    """Per-phase device milliseconds of the plan's last run (back = 0) or the
    run before it (back = 1), for a plan made with FLAG_PHASE_TIMES; waits on
    the host for that run to finish."""
    buf = (ctypes.c_float * 15)()
    cnt = lib.ffsrqr_phase_times_back(plan._h, back, buf, 15)
    if cnt < 0:
        raise FfsrqrError(f"ffsrqr_phase_times_back returned {cnt}")
    return {PHASES[i]: buf[i] for i in range(cnt)}


class Pipe:
    """Host-buffer pipeline over one plan (ffsrqr_pipe_*): each problem's A is
    copied from host memory while the previous problem computes, and the
    outputs come back to host memory."""

    def __init__(self, plan: "Plan"):
        import torch
        self.plan = plan
        self._h = ctypes.c_void_p()
        nb = ctypes.c_size_t()
        _check(lib.ffsrqr_pipe_create(ctypes.byref(self._h), plan._h, ctypes.byref(nb)), "ffsrqr_pipe_create")
        self.device_mem = torch.empty(nb.value + 256, dtype=torch.uint8, device=plan.device)
        self._off = (-self.device_mem.data_ptr()) % 256

    def host_outputs(self):
        """Pinned host U, S, V, piv for one problem."""
        import torch
        p = self.plan
        return (torch.empty(p.m, p.k, dtype=p.dtype).pin_memory(), torch.empty(p.k, dtype=p.dtype).pin_memory(),
                torch.empty(p.n, p.k, dtype=p.dtype).pin_memory(),
                torch.empty(p.n, dtype=torch.int32).pin_memory())

    def run(self, As, outs, seeds=None, stream=None):
        """Enqueue the problems (host A tensors and host output tuples) on
        ``stream`` (default: torch's current stream); synchronise it to read
        the outputs.  Returns the pinned info array."""
        import torch
        count = len(As)
        arr = (HostProblem * max(1, count))()
        for i, (A, (U, S, V, piv)) in enumerate(zip(As, outs)):
            assert not A.is_cuda and A.dtype == self.plan.dtype and A.stride(1) == 1
            arr[i] = HostProblem(A.data_ptr(), A.stride(0), 0 if seeds is None else seeds[i], U.data_ptr(),
                                 U.stride(0), S.data_ptr(), V.data_ptr(), V.stride(0), piv.data_ptr())
        self._infos = torch.zeros(max(1, count) * ctypes.sizeof(Info), dtype=torch.uint8).pin_memory()
        st = torch.cuda.current_stream(self.plan.device) if stream is None else stream
        _check(lib.ffsrqr_pipe_run(self._h, arr, count, self.device_mem.data_ptr() + self._off, self.plan.ws_ptr,
                                   ctypes.c_void_p(st.cuda_stream),
                                   ctypes.cast(self._infos.data_ptr(), ctypes.POINTER(Info))), "ffsrqr_pipe_run")
        return self._infos

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib.ffsrqr_pipe_destroy(h)
            self._h = None


class Batch:
    """Many problems of uneven sizes run as one CUDA graph (ffsrqr_batch_*).

    sizes: list of (m, n, k, p).  The workspace is one torch uint8 buffer;
    outputs() allocates each problem's (U, S, V, piv)."""

    def __init__(self, sizes, mode: int = PLAIN_FP32, streams: int = 4, g: float = 2.0, device=None):
        import torch
        self.sizes = [tuple(int(v) for v in sz) for sz in sizes]
        self.mode = mode
        self.device = torch.device("cuda" if device is None else device)
        self.dtype = torch.float64 if mode == FP64 else torch.float32
        cnt = len(self.sizes)
        arr = lambda ct, col: (ct * cnt)(*[sz[col] for sz in self.sizes])  # noqa: E731
        self._m, self._n = arr(ctypes.c_int64, 0), arr(ctypes.c_int64, 1)
        self._k, self._p = arr(ctypes.c_int32, 2), arr(ctypes.c_int32, 3)
        self._h = ctypes.c_void_p()
        ws = ctypes.c_size_t()
        opts = Opts(g, 0, 0)
        opts_p = None
        if g != 2.0:
            opts = Opts(g, 4 * max(sz[2] for sz in self.sizes), 0)
            opts_p = ctypes.byref(opts)
        _check(lib.ffsrqr_batch_create(ctypes.byref(self._h), cnt, self._m, self._n, self._k, self._p, mode,
                                       opts_p, streams, ctypes.byref(ws)), "ffsrqr_batch_create")
        self.workspace = torch.empty(ws.value + 256, dtype=torch.uint8, device=self.device)
        self._ws_off = (-self.workspace.data_ptr()) % 256
        self._info = torch.zeros(cnt * ctypes.sizeof(Info), dtype=torch.uint8).pin_memory()

    def outputs(self):
        import torch
        outs = []
        for m, n, k, p in self.sizes:
            outs.append((torch.empty(m, k, dtype=self.dtype, device=self.device),
                         torch.empty(k, dtype=self.dtype, device=self.device),
                         torch.empty(n, k, dtype=self.dtype, device=self.device),
                         torch.empty(n, dtype=torch.int32, device=self.device)))
        return outs

    def _problems(self, As, outs, seeds):
        probs = (Problem * len(self.sizes))()
        for i, (A, (U, S, V, piv)) in enumerate(zip(As, outs)):
            assert A.is_cuda and A.dtype == self.dtype and A.stride(1) == 1
            probs[i] = Problem(A.data_ptr(), A.stride(0), seeds[i], U.data_ptr(), U.stride(0), S.data_ptr(),
                               V.data_ptr(), V.stride(0), piv.data_ptr())
        return probs

    def run(self, As, outs, seeds=None, stream=None):
        import torch
        seeds = seeds or [0] * len(self.sizes)
        self._probs = self._problems(As, outs, seeds)  # kept alive: the graph was captured with it
        st = torch.cuda.current_stream(self.device) if stream is None else stream
        _check(lib.ffsrqr_batch_run(self._h, self._probs, self.workspace.data_ptr() + self._ws_off,
                                    ctypes.c_void_p(st.cuda_stream), self._info.data_ptr()), "ffsrqr_batch_run")

    def tune(self, As, outs, seeds=None, stream=None):
        import torch
        seeds = seeds or [0] * len(self.sizes)
        self._probs = self._problems(As, outs, seeds)
        st = torch.cuda.current_stream(self.device) if stream is None else stream
        chosen, ms = ctypes.c_int32(), ctypes.c_float()
        _check(lib.ffsrqr_batch_tune(self._h, self._probs, self.workspace.data_ptr() + self._ws_off,
                                     ctypes.c_void_p(st.cuda_stream), self._info.data_ptr(),
                                     ctypes.byref(chosen), ctypes.byref(ms)), "ffsrqr_batch_tune")
        return chosen.value, ms.value

    def set_phased(self, phased: bool):
        """Phase-batched graph: the small SVDs of all single-precision problems in
        one launch per cluster size (ffsrqr_batch_set_phased)."""
        _check(lib.ffsrqr_batch_set_phased(self._h, 1 if phased else 0), "ffsrqr_batch_set_phased")

    @property
    def phased(self) -> bool:
        return lib.ffsrqr_batch_phased(self._h) == 1

    def small_svd_launches(self) -> int:
        return lib.ffsrqr_batch_small_svd_launches(self._h)

    def info(self, i: int) -> dict:
        sz = ctypes.sizeof(Info)
        return Info.from_buffer_copy(bytes(self._info[i * sz:(i + 1) * sz].numpy().tobytes())).as_dict()

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            lib.ffsrqr_batch_destroy(self._h)
            self._h = ctypes.c_void_p()


class Server:
    """Request server (ffsrqr_server_*): device memory budget, slots streams."""

    def __init__(self, budget_bytes: int, slots: int = 4):
        self._h = ctypes.c_void_p()
        _check(lib.ffsrqr_server_create(ctypes.byref(self._h), budget_bytes, slots, None), "ffsrqr_server_create")
        self._keep = {}

    def submit(self, A, k: int, p: int, mode: int, out, seed: int = 0) -> int:
        U, S, V, piv = out
        m, n = A.shape
        req = Request(m, n, k, p, mode, 0, A.data_ptr(), A.stride(0), seed, U.data_ptr(), U.stride(0),
                      S.data_ptr(), V.data_ptr(), V.stride(0), piv.data_ptr())
        t = ctypes.c_int64()
        rc = lib.ffsrqr_server_submit(self._h, ctypes.byref(req), ctypes.byref(t))
        if rc != 0:
            raise FfsrqrError(f"ffsrqr_server_submit returned {rc} ({lib.ffsrqr_status_string(rc).decode()})")
        self._keep[t.value] = (A, out)  # buffers stay alive until the request finishes
        return t.value

    def wait(self, ticket: int):
        info, lat = Info(), ctypes.c_double()
        rc = lib.ffsrqr_server_wait(self._h, ticket, ctypes.byref(info), ctypes.byref(lat))
        self._keep.pop(ticket, None)
        _check(rc, "ffsrqr_server_wait")
        return info.as_dict(), lat.value

    def poll(self, ticket: int):
        info, lat = Info(), ctypes.c_double()
        rc = lib.ffsrqr_server_poll(self._h, ticket, ctypes.byref(info), ctypes.byref(lat))
        if rc == 1:
            return None
        self._keep.pop(ticket, None)
        _check(rc, "ffsrqr_server_poll")
        return info.as_dict(), lat.value

    def stats(self) -> dict:
        a, c, q, f = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_size_t()
        _check(lib.ffsrqr_server_stats(self._h, ctypes.byref(a), ctypes.byref(c), ctypes.byref(q), ctypes.byref(f)),
               "ffsrqr_server_stats")
        return {"admitted": a.value, "completed": c.value, "queued": q.value, "arena_free": f.value}

    def set_phase_batch(self, on: bool):
        """Same-phase batching of the small SVDs (ffsrqr_server_set_phase_batch)."""
        _check(lib.ffsrqr_server_set_phase_batch(self._h, 1 if on else 0), "ffsrqr_server_set_phase_batch")

    def pause(self, paused: bool):
        """Hold (True) or resume (False) admission (ffsrqr_server_pause)."""
        _check(lib.ffsrqr_server_pause(self._h, 1 if paused else 0), "ffsrqr_server_pause")

    def phase_stats(self) -> dict:
        nl, nr = ctypes.c_int64(), ctypes.c_int64()
        _check(lib.ffsrqr_server_phase_stats(self._h, ctypes.byref(nl), ctypes.byref(nr)),
               "ffsrqr_server_phase_stats")
        return {"small_svd_launches": nl.value, "grouped_requests": nr.value}

    def close(self):
        if self._h.value:
            lib.ffsrqr_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        self.close()



class Tucker:
    """Plan + device workspace for a rank-``ranks`` Tucker approximation of a
    dims[0] x ... x dims[d-1] tensor: ``method`` TUCKER_STHOSVD (Alg. 6, in
    ``order``) or TUCKER_HOSVD (Alg. 5), with Flip-Flop SRQR (oversampling p,
    ``mode``) for every unfolding."""

    def __init__(self, dims, ranks, order=None, p: int = 5, mode: int = PLAIN_FP32,
                 method: int = TUCKER_STHOSVD, g: float = 2.0, device=None):
        import torch
        self.d = len(dims)
        self.dims, self.ranks = [int(x) for x in dims], [int(x) for x in ranks]
        self.order = list(range(self.d)) if order is None else [int(x) for x in order]
        self.p, self.mode, self.method = p, mode, method
        self.device = torch.device("cuda" if device is None else device)
        self.dtype = torch.float64 if mode == FP64 else torch.float32
        d = self.d
        dims_c = (ctypes.c_int64 * d)(*self.dims)
        ranks_c = (ctypes.c_int32 * d)(*self.ranks)
        order_c = (ctypes.c_int32 * d)(*self.order)
        opts = Opts(g, 4 * max(self.ranks), 0)
        self._h = ctypes.c_void_p()
        ws = ctypes.c_size_t()
        with torch.cuda.device(self.device):
            _check(lib.ffsrqr_tucker_plan(ctypes.byref(self._h), method, d, dims_c, ranks_c, order_c, p, mode,
                                          ctypes.byref(opts), ctypes.byref(ws)), "ffsrqr_tucker_plan")
        self.workspace_bytes = ws.value
        self.workspace = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=self.device)
        self._ws_off = (-self.workspace.data_ptr()) % 256
        self._info_host = torch.zeros(d * ctypes.sizeof(Info), dtype=torch.uint8).pin_memory()

    @property
    def ws_ptr(self) -> int:
        return self.workspace.data_ptr() + self._ws_off

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib.ffsrqr_tucker_destroy(h)
            self._h = None

    def outputs(self):
        """(U_r by mode, S_r by mode, core) as torch device tensors."""
        import torch
        kw = {"dtype": self.dtype, "device": self.device}
        Us = [torch.empty(I, k, **kw) for I, k in zip(self.dims, self.ranks)]
        Ss = [torch.empty(k, **kw) for k in self.ranks]
        core = torch.empty(*self.ranks, **kw)
        return Us, Ss, core

    def run(self, X, seed: int = 0, out=None, stream=None):
        """Enqueue ffsrqr_tucker_run on ``stream`` (default: torch's current stream)."""
        import torch
        assert X.is_cuda and X.dtype == self.dtype and list(X.shape) == self.dims and X.is_contiguous()
        Us, Ss, core = out if out is not None else self.outputs()
        st = torch.cuda.current_stream(self.device) if stream is None else stream
        u_c = (ctypes.c_void_p * self.d)(*[u.data_ptr() for u in Us])
        s_c = (ctypes.c_void_p * self.d)(*[s.data_ptr() for s in Ss])
        _check(lib.ffsrqr_tucker_run(self._h, X.data_ptr(), seed, u_c, s_c, core.data_ptr(), self.ws_ptr,
                                     ctypes.c_void_p(st.cuda_stream), self._info_host.data_ptr()),
               "ffsrqr_tucker_run")
        return Us, Ss, core

    def infos(self):
        """Per-factor-step reports of the last run (after a sync)."""
        raw = bytes(self._info_host.numpy().tobytes())
        sz = ctypes.sizeof(Info)
        return [Info.from_buffer_copy(raw[j * sz:(j + 1) * sz]).as_dict() for j in range(self.d)]

    def launch_count(self) -> int:
        return lib.ffsrqr_tucker_launch_count(self._h)


class RPCA:
    """Robust PCA solver (Alg. 7, IALM with Alg. 9 as the truncated SVD) for
    m x n inputs, with its device workspace.  Options left at 0 take the C
    ABI's defaults (ffsrqr_rpca_opts_t)."""

    def __init__(self, m: int, n: int, mode: int = MIXED, p: int = 0, sv0: int = 0, max_iter: int = 0,
                 kmax: int = 0, lam: float = 0.0, rho: float = 0.0, mu_bar_ratio: float = 0.0, tol: float = 0.0,
                 device=None):
        import torch
        self.m, self.n, self.mode = m, n, mode
        self.device = torch.device("cuda" if device is None else device)
        self.dtype = torch.float64 if mode == FP64 else torch.float32
        opts = RpcaOpts(mode, p, sv0, max_iter, kmax, 0, lam, rho, mu_bar_ratio, tol)
        self._h = ctypes.c_void_p()
        ws = ctypes.c_size_t()
        with torch.cuda.device(self.device):
            _check(lib.ffsrqr_rpca_create(ctypes.byref(self._h), m, n, ctypes.byref(opts), ctypes.byref(ws)),
                   "ffsrqr_rpca_create")
        self.workspace_bytes = ws.value
        self.workspace = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=self.device)
        self._ws_off = (-self.workspace.data_ptr()) % 256

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib.ffsrqr_rpca_destroy(h)
            self._h = None

    def run(self, M, X=None, E=None, seed: int = 0, stream=None):
        """Solve for M (device, m x n); returns (X, E, info dict).  Blocking."""
        import torch
        assert M.is_cuda and M.dtype == self.dtype and M.shape == (self.m, self.n) and M.stride(1) == 1
        X = torch.empty_like(M) if X is None else X
        E = torch.empty_like(M) if E is None else E
        st = torch.cuda.current_stream(self.device) if stream is None else stream
        info = RpcaInfo()
        _check(lib.ffsrqr_rpca_run(self._h, M.data_ptr(), M.stride(0), X.data_ptr(), X.stride(0), E.data_ptr(),
                                   E.stride(0), seed, self.workspace.data_ptr() + self._ws_off,
                                   ctypes.c_void_p(st.cuda_stream), ctypes.byref(info)), "ffsrqr_rpca_run")
        return X, E, info.as_dict()

    def launch_count(self) -> int:
        return lib.ffsrqr_rpca_launch_count(self._h)
