"""Python binding of libcpd (include/cpd.h): argument marshalling only.

The functions below carry the C names and forward to the library; every step
of an iteration runs in the library's CUDA kernels. Importing this module
loads ``libcpd.so`` from the package directory and raises if it has not been
built (``python -m paper_2103_04081_gb300.build``): there is no CPU path.

``Decomposition`` is a small convenience wrapper used by the tests and the
bench; it keeps torch tensors only as device/host buffers.
"""
from __future__ import annotations

import ctypes
import json
import os

import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libcpd.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENONFINITE, EDEGENERATE, EAGAIN, EBUSY = range(9)
HOST, DEVICE = 0, 1
SAMPLE = {"euclidean": 0, "leverage": 1, "uniform": 2}
STEP = {"fixed": 0, "adagrad": 1, "decay": 2}
CONSTRAINT = {"none": 0, "nonneg": 1}
LAYOUT = {"replicas": 0, "strided": 1}
XDT = {"f64": 0, "f32": 1, "bf16": 2}
ENGINE = {"auto": 0, "simt": 1, "tensor": 2, "cluster": 3, "persistent": 4, "fused": 5}
MAX_MODES = 8


class CpdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cpd status {status}: {msg}")
        self.status = status


class cpd_config(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int32), ("R", ctypes.c_int32), ("B", ctypes.c_int32),
        ("sampling", ctypes.c_int32), ("step", ctypes.c_int32), ("x_dtype", ctypes.c_int32),
        ("dims", ctypes.c_int64 * MAX_MODES),
        ("alpha", ctypes.c_double), ("eta", ctypes.c_double), ("b", ctypes.c_double),
        ("beta", ctypes.c_double), ("gamma", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("engine", ctypes.c_int32), ("max_ctas", ctypes.c_int32),
        ("constraint", ctypes.c_int32), ("x_layout", ctypes.c_int32),
        ("tile_rows", ctypes.c_int32), ("tile_fibers", ctypes.c_int32),
        ("block", ctypes.c_int32),
    ]


class cpd_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_active", ctypes.c_int32),
                ("fit_every", ctypes.c_int32), ("no_grouping", ctypes.c_int32),
                ("strided_above_mb", ctypes.c_int32)]


class cpd_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("done", ctypes.c_int32), ("reached", ctypes.c_int32),
                ("layout", ctypes.c_int32), ("iters", ctypes.c_int64), ("fit", ctypes.c_double),
                ("tol", ctypes.c_double), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is missing: build it with "
                           "`python -m paper_2103_04081_gb300.build` (there is no CPU fallback)")
    lib = ctypes.CDLL(_LIB_PATH)
    P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    sig = {
        "cpd_init": [ctypes.POINTER(cpd_config), P, I32, P, I32, P, ctypes.POINTER(P)],
        "cpd_sgd_iters": [P, I64, P],
        "cpd_prepare": [P, I64, P],
        "cpd_gradients": [P, I32, I64, I32, P, P],
        "cpd_skrp": [P, I32, I64, I32, P, P, P, P, P],
        "cpd_fit": [P, P, P, P],
        "cpd_fit_start": [P, P],
        "cpd_fit_poll": [P, P, P],
        "cpd_get_factors": [P, P, I32, P],
        "cpd_set_factors": [P, P, I32, P],
        "cpd_get_adagrad": [P, P, I32, P],
        "cpd_set_adagrad": [P, P, I32, P],
        "cpd_get_iteration": [P, ctypes.POINTER(I64)],
        "cpd_set_iteration": [P, I64],
        "cpd_last_sample": [P, P, P, P, P],
        "cpd_last_gradient": [P, P, P],
        "cpd_sync": [P, P],
        "cpd_profile": [P, I32],
        "cpd_profile_read": [P, ctypes.POINTER(I64), ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double), P],
        "cpd_describe": [P, ctypes.c_char_p, ctypes.c_size_t],
        "cpd_destroy": [P],
        "cpd_tol_noalloc": [I32, P, I32, I32, P, P, P, P],
        "cpd_server_create": [ctypes.POINTER(cpd_server_config), ctypes.POINTER(P)],
        "cpd_submit": [P, ctypes.POINTER(cpd_config), P, I32, P, I32, ctypes.c_double, I64,
                       ctypes.POINTER(ctypes.c_uint64)],
        "cpd_poll": [P, ctypes.c_uint64, ctypes.POINTER(cpd_result), P],
        "cpd_server_wait": [P, ctypes.c_double],
        "cpd_server_stats": [P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                             ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)],
        "cpd_server_destroy": [P],
        "cpd_grad_variance": [P, I32, P, P, P],
        "cpd_autotune": [ctypes.POINTER(cpd_config), P, I32, P, I32, I64, ctypes.POINTER(cpd_config),
                         ctypes.POINTER(ctypes.c_double), P],
        "cpd_group_create": [P, I32, P, ctypes.POINTER(P)],
        "cpd_group_iters": [P, I64, P],
        "cpd_group_destroy": [P],
        "cpd_trace": [P, I32],
        "cpd_trace_read": [P, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.cpd_last_error.argtypes = []
    lib.cpd_last_error.restype = ctypes.c_char_p
    return lib


_lib = _load()


def lib() -> ctypes.CDLL:
    return _lib


def _check(st: int) -> None:
    if st != OK:
        raise CpdError(st, _lib.cpd_last_error().decode())


def make_config(dims, R, B, sampling="euclidean", step="adagrad", x_dtype="bf16", alpha=0.1,
                eta=0.1, b=1e-12, beta=1.0, gamma=1.0, seed=0, engine="auto",
                max_ctas=0, constraint="none", x_layout="replicas", tile_rows=0,
                tile_fibers=0, block=1) -> cpd_config:
    c = cpd_config()
    c.N, c.R, c.B = len(dims), int(R), int(B)
    c.sampling, c.step, c.x_dtype = SAMPLE[sampling], STEP[step], XDT[x_dtype]
    for k, d in enumerate(dims):
        c.dims[k] = int(d)
    c.alpha, c.eta, c.b, c.beta, c.gamma = alpha, eta, b, beta, gamma
    c.seed = int(seed) & (2**64 - 1)
    c.engine = ENGINE[engine]
    c.max_ctas = int(max_ctas)
    c.constraint = CONSTRAINT[constraint]
    c.x_layout = LAYOUT[x_layout]
    c.tile_rows, c.tile_fibers = int(tile_rows), int(tile_fibers)
    c.block = int(block)
    return c


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptrs(ts) -> ctypes.Array:
    return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])


def _loc(t: torch.Tensor) -> int:
    return DEVICE if t.is_cuda else HOST


# ---- C-ABI names -------------------------------------------------------

def cpd_init(cfg: cpd_config, X: torch.Tensor, A0: list, stream=None) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(_lib.cpd_init(ctypes.byref(cfg), X.data_ptr(), _loc(X), _ptrs(A0), _loc(A0[0]),
                         _stream(stream), ctypes.byref(ctx)))
    return ctx


def cpd_sgd_iters(ctx, iters: int, stream=None) -> None:
    _check(_lib.cpd_sgd_iters(ctx, int(iters), _stream(stream)))


def cpd_prepare(ctx, iters: int, stream=None) -> None:
    _check(_lib.cpd_prepare(ctx, int(iters), _stream(stream)))


def cpd_gradients(ctx, n: int, t0: int, K: int, G_out: torch.Tensor, stream=None) -> None:
    """K mini-batch gradients of mode n into the device tensor G_out (K x I_n x R float32)."""
    _check(_lib.cpd_gradients(ctx, int(n), int(t0), int(K), G_out.data_ptr(), _stream(stream)))


def cpd_skrp(ctx, n: int, t0: int, K: int, idx=None, p=None, Z=None, X=None, stream=None) -> None:
    """Alg. 3 + Alg. 1 materialised for K batches of mode n into device tensors
    (idx K*B x N int32, p K*B float64, Z K*B x R float32, X K*B x ld_n)."""
    ptr = (lambda t: t.data_ptr() if t is not None else None)
    _check(_lib.cpd_skrp(ctx, int(n), int(t0), int(K), ptr(idx), ptr(p), ptr(Z), ptr(X), _stream(stream)))


def cpd_fit(ctx, stream=None) -> tuple[float, float]:
    fit, tol = ctypes.c_double(), ctypes.c_double()
    _check(_lib.cpd_fit(ctx, ctypes.byref(fit), ctypes.byref(tol), _stream(stream)))
    return fit.value, tol.value


def cpd_fit_start(ctx, stream=None) -> None:
    _check(_lib.cpd_fit_start(ctx, _stream(stream)))


def cpd_fit_poll(ctx):
    """(fit, tol), or None while the pass started by cpd_fit_start is running."""
    fit, tol = ctypes.c_double(), ctypes.c_double()
    st = _lib.cpd_fit_poll(ctx, ctypes.byref(fit), ctypes.byref(tol))
    if st == EAGAIN:
        return None
    _check(st)
    return fit.value, tol.value


def cpd_get_factors(ctx, out: list, stream=None) -> None:
    _check(_lib.cpd_get_factors(ctx, _ptrs(out), _loc(out[0]), _stream(stream)))


def cpd_set_factors(ctx, A: list, stream=None) -> None:
    _check(_lib.cpd_set_factors(ctx, _ptrs(A), _loc(A[0]), _stream(stream)))


def cpd_get_adagrad(ctx, out: list, stream=None) -> None:
    _check(_lib.cpd_get_adagrad(ctx, _ptrs(out), _loc(out[0]), _stream(stream)))


def cpd_set_adagrad(ctx, S: list, stream=None) -> None:
    _check(_lib.cpd_set_adagrad(ctx, _ptrs(S), _loc(S[0]), _stream(stream)))


def cpd_get_iteration(ctx) -> int:
    t = ctypes.c_int64()
    _check(_lib.cpd_get_iteration(ctx, ctypes.byref(t)))
    return t.value


def cpd_set_iteration(ctx, t: int) -> None:
    _check(_lib.cpd_set_iteration(ctx, int(t)))


def cpd_last_sample(ctx, N: int, B: int, stream=None):
    n = ctypes.c_int32()
    idx = torch.empty(B, N, dtype=torch.int32)
    p = torch.empty(B, dtype=torch.float64)
    _check(_lib.cpd_last_sample(ctx, ctypes.byref(n), idx.data_ptr(), p.data_ptr(), _stream(stream)))
    return n.value, idx, p


def cpd_last_gradient(ctx, In: int, R: int, dtype, stream=None) -> torch.Tensor:
    G = torch.empty(In, R, dtype=dtype)
    _check(_lib.cpd_last_gradient(ctx, G.data_ptr(), _stream(stream)))
    return G


def cpd_sync(ctx, stream=None) -> None:
    _check(_lib.cpd_sync(ctx, _stream(stream)))


def cpd_profile(ctx, enable: bool) -> None:
    _check(_lib.cpd_profile(ctx, int(bool(enable))))


def cpd_profile_read(ctx, stream=None) -> tuple[int, float, float]:
    """(timed iterations, mean gradient-kernel ms, mean ms of the rest of an iteration)."""
    n, mg, mu = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    _check(_lib.cpd_profile_read(ctx, ctypes.byref(n), ctypes.byref(mg), ctypes.byref(mu),
                                 _stream(stream)))
    return n.value, mg.value, mu.value


def cpd_trace(ctx, enable: bool) -> None:
    _check(_lib.cpd_trace(ctx, int(bool(enable))))


def cpd_trace_read(ctx, stream=None) -> list:
    """The 64 phase timestamps (ns) of the most recent traced iteration."""
    out = (ctypes.c_uint64 * 64)()
    _check(_lib.cpd_trace_read(ctx, out, _stream(stream)))
    return [int(v) for v in out]


def cpd_describe(ctx) -> dict:
    buf = ctypes.create_string_buffer(1024)
    _check(_lib.cpd_describe(ctx, buf, 1024))
    return json.loads(buf.value.decode())


def cpd_destroy(ctx) -> None:
    _check(_lib.cpd_destroy(ctx))


def cpd_tol_noalloc(dims, R: int, x_dtype: str, X: torch.Tensor, A: list, tol_out: torch.Tensor,
                    stream=None) -> None:
    """Tol of a CP model into the device double `tol_out`, with no device allocation."""
    d = (ctypes.c_int64 * len(dims))(*[int(v) for v in dims])
    _check(_lib.cpd_tol_noalloc(len(dims), d, int(R), XDT[x_dtype], X.data_ptr(), _ptrs(A),
                                tol_out.data_ptr(), _stream(stream)))


def cpd_server_create(hbm_budget: int = 0, max_active: int = 0, fit_every: int = 0,
                      grouping: bool = True, strided_above_mb: int = 0):
    cfg = cpd_server_config()
    cfg.hbm_budget, cfg.max_active, cfg.fit_every = int(hbm_budget), int(max_active), int(fit_every)
    cfg.no_grouping = 0 if grouping else 1
    cfg.strided_above_mb = int(strided_above_mb)
    srv = ctypes.c_void_p()
    _check(_lib.cpd_server_create(ctypes.byref(cfg), ctypes.byref(srv)))
    return srv


def cpd_submit(srv, cfg: cpd_config, X: torch.Tensor, A0: list, stop_fit: float, max_iters: int) -> int:
    ticket = ctypes.c_uint64()
    _check(_lib.cpd_submit(srv, ctypes.byref(cfg), X.data_ptr(), _loc(X), _ptrs(A0), _loc(A0[0]),
                           float(stop_fit), int(max_iters), ctypes.byref(ticket)))
    return ticket.value


def cpd_poll(srv, ticket: int, A_out: list | None = None):
    """(status, result dict); status EAGAIN while the request runs or waits."""
    res = cpd_result()
    st = _lib.cpd_poll(srv, ticket, ctypes.byref(res), _ptrs(A_out) if A_out else None)
    if st not in (OK, EAGAIN):
        msg = _lib.cpd_last_error().decode()
    else:
        msg = ""
    d = {f: getattr(res, f) for f, _ in cpd_result._fields_}
    d["message"] = msg
    return st, d


def cpd_server_stats(srv) -> dict:
    """The server's budget, the bytes its requests hold, running and waiting requests."""
    b, h = ctypes.c_size_t(), ctypes.c_size_t()
    a, q = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.cpd_server_stats(srv, ctypes.byref(b), ctypes.byref(h), ctypes.byref(a), ctypes.byref(q)))
    return {"budget": b.value, "held": h.value, "active": a.value, "queued": q.value}


def cpd_server_wait(srv, timeout_s: float = 0.0) -> bool:
    st = _lib.cpd_server_wait(srv, float(timeout_s))
    if st == EAGAIN:
        return False
    _check(st)
    return True


def cpd_server_destroy(srv) -> None:
    _check(_lib.cpd_server_destroy(srv))


def cpd_grad_variance(ctx, n: int, stream=None) -> tuple[float, float]:
    """(E||G - E[G]||^2, ||E[G]||^2) of the mode-n mini-batch gradient (Thm 10)."""
    v, m = ctypes.c_double(), ctypes.c_double()
    _check(_lib.cpd_grad_variance(ctx, int(n), ctypes.byref(v), ctypes.byref(m), _stream(stream)))
    return v.value, m.value


def cpd_autotune(cfg: cpd_config, X: torch.Tensor, A0: list, iters: int = 500, stream=None):
    """(configuration with the fastest engine and CTA cap, its iterations/s)."""
    best = cpd_config()
    rate = ctypes.c_double()
    _check(_lib.cpd_autotune(ctypes.byref(cfg), X.data_ptr(), _loc(X), _ptrs(A0), _loc(A0[0]), int(iters),
                             ctypes.byref(best), ctypes.byref(rate), _stream(stream)))
    return best, rate.value


def cpd_group_create(ctxs: list, stream=None):
    """One grouped launch per iteration for all of `ctxs` (borrowed handles)."""
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    grp = ctypes.c_void_p()
    _check(_lib.cpd_group_create(arr, len(ctxs), _stream(stream), ctypes.byref(grp)))
    return grp


def cpd_group_iters(grp, iters: int, stream=None) -> None:
    _check(_lib.cpd_group_iters(grp, int(iters), _stream(stream)))


def cpd_group_destroy(grp) -> None:
    _check(_lib.cpd_group_destroy(grp))


# ---- convenience wrapper -------------------------------------------------

class Decomposition:
    """One context: owns nothing on the Python side but the handle."""

    def __init__(self, X: torch.Tensor, A0: list, stream=None, config: cpd_config | None = None, **cfg):
        if config is not None:     # a ready configuration (e.g. from cpd_autotune)
            self.dims = tuple(int(config.dims[k]) for k in range(config.N))
            self.R, self.B = int(config.R), int(config.B)
            self.x_dtype = {v: k for k, v in XDT.items()}[config.x_dtype]
            self.cfg = config
        else:
            self.dims = tuple(int(d) for d in cfg["dims"])
            self.R, self.B = int(cfg["R"]), int(cfg["B"])
            self.x_dtype = cfg.get("x_dtype", "bf16")
            self.cfg = make_config(**cfg)
        self.fdtype = torch.float64 if self.x_dtype == "f64" else torch.float32
        A0 = [a.to(self.fdtype).contiguous() for a in A0]
        self.ctx = cpd_init(self.cfg, X.contiguous(), A0, stream)

    def sgd_iters(self, iters: int, stream=None) -> None:
        cpd_sgd_iters(self.ctx, iters, stream)

    def fit(self, stream=None) -> tuple[float, float]:
        return cpd_fit(self.ctx, stream)

    def factors(self, device="cpu", stream=None) -> list:
        out = [torch.empty(d, self.R, dtype=self.fdtype, device=device) for d in self.dims]
        if device != "cpu":
            out = [o.contiguous() for o in out]
        cpd_get_factors(self.ctx, out, stream)
        if device != "cpu":
            torch.cuda.synchronize()
        return out

    def set_factors(self, A: list, stream=None) -> None:
        cpd_set_factors(self.ctx, [a.to(self.fdtype).contiguous() for a in A], stream)

    def adagrad(self) -> list:
        out = [torch.empty(d, self.R, dtype=torch.float64) for d in self.dims]
        cpd_get_adagrad(self.ctx, out)
        return out

    def set_adagrad(self, S: list) -> None:
        cpd_set_adagrad(self.ctx, [s.to(torch.float64).contiguous() for s in S])

    @property
    def t(self) -> int:
        return cpd_get_iteration(self.ctx)

    @t.setter
    def t(self, v: int) -> None:
        cpd_set_iteration(self.ctx, v)

    def last_sample(self):
        return cpd_last_sample(self.ctx, len(self.dims), self.B)

    def last_gradient(self):
        n, _, _ = self.last_sample()
        return n, cpd_last_gradient(self.ctx, self.dims[n], self.R, self.fdtype)

    def sync(self) -> None:
        cpd_sync(self.ctx)

    def grad_variance(self, n: int, stream=None) -> tuple[float, float]:
        return cpd_grad_variance(self.ctx, n, stream)

    def describe(self) -> dict:
        return cpd_describe(self.ctx)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            cpd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
