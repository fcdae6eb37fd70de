"""ctypes access to the FP64 CPU oracle in ``cpd_oracle.c``.

Test infrastructure: only the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline / reference leg use this module. It never imports the
CUDA package, and the CUDA package never imports it.

Every function marshals numpy arrays into the C oracle; the arithmetic lives
in the C file, which cites the paper's sections step by step.

Conventions: X is a dense tensor in column-major order (first index fastest,
the order of Eq. (2)), passed as a numpy array in Fortran order or as a flat
buffer together with ``dims``. Factors are float64 arrays of shape (I_k, R).
Indices are 0-based.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpd_oracle.c")
LIB_PATH = os.path.join(_HERE, "liboracle.so")

MAXN = 8
SAMPLE = {"euclidean": 0, "leverage": 1, "uniform": 2}
STEP = {"fixed": 0, "adagrad": 1, "decay": 2}
XDT = {"f64": 0, "f32": 1, "bf16": 2}
CONSTRAINT = {"none": 0, "nonneg": 1}
OK, EINVAL, EDEGENERATE = 0, 1, 6


OMP_LIB_PATH = os.path.join(_HERE, "liboracle_omp.so")


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle with gcc (-ffp-contract=off: no implicit FMA). With
    omp, the timing-only all-cores build of the same source."""
    path = OMP_LIB_PATH if omp else LIB_PATH
    if force or not os.path.exists(path) or (os.path.getmtime(path) < os.path.getmtime(_SRC)):
        tmp = path + f".tmp{os.getpid()}"
        extra = ["-DORC_OMP", "-fopenmp"] if omp else []
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fPIC", *extra,
            "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, path)
    return path


_lib = None
_lib_omp = None


def lib(omp: bool = False) -> ctypes.CDLL:
    global _lib, _lib_omp
    if omp:
        if _lib_omp is None:
            _lib_omp = ctypes.CDLL(build(omp=True))
            _declare(_lib_omp)
        return _lib_omp
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int32), ("R", ctypes.c_int32), ("B", ctypes.c_int32),
        ("sampling", ctypes.c_int32), ("step", ctypes.c_int32),
        ("x_dtype", ctypes.c_int32), ("dims", ctypes.c_int64 * MAXN),
        ("alpha", ctypes.c_double), ("eta", ctypes.c_double),
        ("b", ctypes.c_double), ("beta", ctypes.c_double),
        ("gamma", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("constraint", ctypes.c_int32), ("block", ctypes.c_int32),
    ]


@dataclass
class Config:
    """Problem and method parameters of one BrawsCPD / AdawsCPD run."""
    dims: tuple
    R: int
    B: int
    sampling: str = "euclidean"
    step: str = "adagrad"
    x_dtype: str = "f64"
    alpha: float = 0.1
    eta: float = 0.1
    b: float = 1e-12
    beta: float = 1.0
    gamma: float = 1.0
    seed: int = 0
    constraint: str = "none"
    block: int = 1          # Remark 1: fibers per sampled block (1: per-fiber sampling)
    extra: dict = field(default_factory=dict)

    def c(self) -> _Cfg:
        cfg = _Cfg()
        cfg.N = len(self.dims)
        cfg.R, cfg.B = self.R, self.B
        cfg.sampling = SAMPLE[self.sampling]
        cfg.step = STEP[self.step]
        cfg.x_dtype = XDT[self.x_dtype]
        for k, d in enumerate(self.dims):
            cfg.dims[k] = int(d)
        cfg.alpha, cfg.eta, cfg.b = self.alpha, self.eta, self.b
        cfg.constraint = CONSTRAINT[self.constraint]
        cfg.beta, cfg.gamma = self.beta, self.gamma
        cfg.seed = int(self.seed) & (2**64 - 1)
        cfg.block = int(self.block)
        return cfg


_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_u64 = ctypes.c_uint64
_dbl = ctypes.c_double


def _declare(L):
    L.orc_philox4x64.argtypes = [_p, _p, _p]
    L.orc_fiber_word.argtypes = [_u64, _i64, _i64, ctypes.c_int]
    L.orc_fiber_word.restype = _u64
    L.orc_mode_draw.argtypes = [_u64, _i64, _i32]
    L.orc_mode_draw.restype = _i32
    L.orc_weights_euclidean.argtypes = [_p, _i64, _i32, _p]
    L.orc_weights_leverage.argtypes = [_p, _i64, _i32, _p]
    L.orc_weights_leverage.restype = ctypes.c_int
    L.orc_weights.argtypes = [_i32, _p, _i64, _i32, _p]
    L.orc_weights.restype = ctypes.c_int
    L.orc_distribution.argtypes = [_p, _i64, _p]
    L.orc_distribution.restype = ctypes.c_int
    L.orc_draw.argtypes = [_p, _i64, _u64]
    L.orc_draw.restype = _i64
    L.orc_prob.argtypes = [_p, _i64, _i64]
    L.orc_prob.restype = _dbl
    L.orc_unfold_col.argtypes = [_i32, _p, _i32, _p]
    L.orc_unfold_col.restype = _i64
    L.orc_gather_fiber.argtypes = [_p, _i32, _i32, _p, _i32, _p, _p]
    L.orc_krp_row.argtypes = [_i32, _i32, _i32, _p, _p, _p]
    L.orc_gradient.argtypes = [_i64, _i32, _i32, _i64, _p, _p, _p, _p, _p]
    L.orc_update.argtypes = [ctypes.POINTER(_Cfg), _i64, _i64, _p, _p, _p]
    L.orc_gradient_for_batch.argtypes = [ctypes.POINTER(_Cfg), _i32, _p, _p, _p, _p, _p]
    L.orc_gradient_for_batch.restype = ctypes.c_int
    L.orc_step.argtypes = [ctypes.POINTER(_Cfg), _i64, _p, _p, _p, _p, _p, _p, _p]
    L.orc_sample_batch.argtypes = [ctypes.POINTER(_Cfg), _i32, _i64, _p, _p, _p, _p, _p, _p]
    L.orc_sample_batch.restype = ctypes.c_int
    L.orc_step.restype = ctypes.c_int
    L.orc_run.argtypes = [ctypes.POINTER(_Cfg), _i64, _i64, _p, _p, _p]
    L.orc_run.restype = ctypes.c_int
    L.orc_tol.argtypes = [_i32, _p, _i32, _p, _i32, _p, _p]
    L.orc_tol.restype = _dbl


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr_array(arrs):
    return (ctypes.c_void_p * len(arrs))(*[_ptr(a) for a in arrs])


def x_buffer(X: np.ndarray, x_dtype: str) -> np.ndarray:
    """Flat column-major buffer of X in the stored dtype ('bf16' = uint16 bits)."""
    if x_dtype == "bf16":
        if X.dtype != np.uint16:
            raise TypeError("bf16 tensors are passed as uint16 bit patterns")
        return np.asfortranarray(X).ravel(order="F")
    want = np.float64 if x_dtype == "f64" else np.float32
    return np.asfortranarray(X, dtype=want).ravel(order="F")


# ------------------------------------------------------------------ #
# Primitives                                                           #
# ------------------------------------------------------------------ #

def philox(ctr, key) -> list:
    c = (ctypes.c_uint64 * 4)(*[int(v) & (2**64 - 1) for v in ctr])
    k = (ctypes.c_uint64 * 2)(*[int(v) & (2**64 - 1) for v in key])
    o = (ctypes.c_uint64 * 4)()
    lib().orc_philox4x64(c, k, o)
    return [int(v) for v in o]


def fiber_word(seed: int, t: int, f: int, k: int) -> int:
    return lib().orc_fiber_word(seed, t, f, k)


def mode_draw(seed: int, t: int, N: int) -> int:
    return lib().orc_mode_draw(seed, t, N)


def weights(sampling: str, A) -> tuple[int, np.ndarray]:
    A = _f64(A)
    w = np.empty(A.shape[0])
    st = lib().orc_weights(SAMPLE[sampling], _ptr(A), A.shape[0], A.shape[1], _ptr(w))
    return st, w


def distribution(w) -> tuple[int, np.ndarray]:
    """(status, cdf): the fixed-point sampling distribution of row weights w."""
    w = _f64(w)
    out = np.zeros(w.size, dtype=np.uint64)
    st = lib().orc_distribution(_ptr(w), w.size, _ptr(out))
    return st, out


def draw(cdf: np.ndarray, x: int) -> int:
    c = np.ascontiguousarray(cdf, dtype=np.uint64)
    return lib().orc_draw(_ptr(c), c.size, int(x) & (2**64 - 1))


def prob(cdf: np.ndarray, i: int) -> float:
    c = np.ascontiguousarray(cdf, dtype=np.uint64)
    return lib().orc_prob(_ptr(c), c.size, int(i))


def unfold_col(dims, n: int, idx) -> int:
    d = np.asarray(dims, dtype=np.int64)
    i = np.asarray(idx, dtype=np.int64)
    return lib().orc_unfold_col(len(d), _ptr(d), n, _ptr(i))


def gather_fiber(X: np.ndarray, n: int, idx, x_dtype: str = "f64") -> np.ndarray:
    buf = x_buffer(X, x_dtype)
    d = np.asarray(X.shape, dtype=np.int64)
    i = np.asarray(idx, dtype=np.int64)
    out = np.empty(X.shape[n])
    lib().orc_gather_fiber(_ptr(buf), XDT[x_dtype], len(d), _ptr(d), n, _ptr(i), _ptr(out))
    return out


def krp_row(A: list, n: int, idx) -> np.ndarray:
    A = [_f64(a) for a in A]
    i = np.asarray(idx, dtype=np.int64)
    R = A[0].shape[1]
    out = np.empty(R)
    lib().orc_krp_row(len(A), R, n, _ptr_array(A), _ptr(i), _ptr(out))
    return out


def gradient(An, Zs, Xs, p, Jn: int) -> np.ndarray:
    """Eq. (11) with Xs given as (B, I_n) rows = fibers."""
    An, Zs, Xs, p = _f64(An), _f64(Zs), _f64(Xs), _f64(p)
    In, R = An.shape
    B = Zs.shape[0]
    G = np.empty((In, R))
    lib().orc_gradient(In, R, B, Jn, _ptr(An), _ptr(Zs), _ptr(Xs), _ptr(p), _ptr(G))
    return G


def update(cfg: Config, t: int, An: np.ndarray, Sn, G) -> None:
    """In-place Eq. (12) / Eq. (13a)-(13b) on float64 arrays."""
    G = _f64(G)
    c = cfg.c()
    S_ptr = _ptr(Sn) if Sn is not None else None
    lib().orc_update(ctypes.byref(c), t, An.shape[0], _ptr(An), S_ptr, _ptr(G))


def gradient_for_batch(cfg: Config, n: int, idx, X, A: list):
    """(status, p, G) for a given mini-batch idx of shape (B, N)."""
    A = [_f64(a) for a in A]
    c = cfg.c()
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    buf = x_buffer(X, cfg.x_dtype)
    p = np.empty(cfg.B)
    G = np.empty((cfg.dims[n], cfg.R))
    st = lib().orc_gradient_for_batch(ctypes.byref(c), n, _ptr(idx), _ptr(buf),
                                      _ptr_array(A), _ptr(p), _ptr(G))
    return st, p, G


def step(cfg: Config, t: int, X, A: list, S: list | None = None, xbuf=None) -> dict:
    """One iteration; A (and S) are lists of float64 arrays updated in place."""
    for a in A:
        assert a.dtype == np.float64 and a.flags.c_contiguous
    c = cfg.c()
    buf = x_buffer(X, cfg.x_dtype) if xbuf is None else xbuf
    N, B = len(cfg.dims), cfg.B
    n = ctypes.c_int32()
    idx = np.empty((B, N), dtype=np.int64)
    p = np.empty(B)
    G = np.empty((max(cfg.dims), cfg.R))
    S_arr = _ptr_array(S) if S is not None else None
    st = lib().orc_step(ctypes.byref(c), t, _ptr(buf), _ptr_array(A), S_arr,
                        ctypes.byref(n), _ptr(idx), _ptr(p), _ptr(G))
    return {"status": st, "n": n.value, "idx": idx, "p": p,
            "G": G[: cfg.dims[n.value]].copy()}


def sample_batch(cfg: Config, n: int, t: int, A: list, xbuf=None, X=None, want_fibers: bool = True) -> dict:
    """Alg. 3 + Alg. 1 for mode n with the draws of iteration t: idx (B x N,
    column n = -1), p (B), Z (B x R) and, if wanted, the fibers X_S (B x I_n)."""
    A = [_f64(a) for a in A]
    c = cfg.c()
    buf = x_buffer(X, cfg.x_dtype) if xbuf is None else xbuf
    B, N, R = cfg.B, len(cfg.dims), cfg.R
    idx = np.empty((B, N), dtype=np.int64)
    p = np.empty(B)
    Z = np.empty((B, R))
    Xs = np.empty((B, int(cfg.dims[n]))) if want_fibers else None
    st = lib().orc_sample_batch(ctypes.byref(c), n, t, _ptr(buf), _ptr_array(A), _ptr(idx), _ptr(p), _ptr(Z),
                                _ptr(Xs) if Xs is not None else None)
    return {"status": st, "idx": idx, "p": p, "Z": Z, "X": Xs}


def run(cfg: Config, t0: int, T: int, X, A: list, S: list | None = None, xbuf=None,
        omp: bool = False) -> int:
    """T iterations from t0 (A, S updated in place); omp: the all-cores build."""
    for a in A:
        assert a.dtype == np.float64 and a.flags.c_contiguous
    c = cfg.c()
    buf = x_buffer(X, cfg.x_dtype) if xbuf is None else xbuf
    S_arr = _ptr_array(S) if S is not None else None
    return lib(omp).orc_run(ctypes.byref(c), t0, T, _ptr(buf), _ptr_array(A), S_arr)


def tol(X, A: list, x_dtype: str = "f64", dims=None) -> tuple[float, float]:
    """(Tol, ||X||^2) of Sec. 5.2 by a direct residual sum over all entries."""
    A = [_f64(a) for a in A]
    if dims is None:
        dims = X.shape
        buf = x_buffer(X, x_dtype)
    else:
        buf = X
    d = np.asarray(dims, dtype=np.int64)
    xx = ctypes.c_double()
    v = lib().orc_tol(len(d), _ptr(d), A[0].shape[1], _ptr(buf), XDT[x_dtype],
                      _ptr_array(A), ctypes.byref(xx))
    return v, xx.value


def stored_values(xbuf: np.ndarray, x_dtype: str) -> np.ndarray:
    """Exact float64 values of a flat buffer of stored tensor entries: bf16 bit
    patterns are the upper half of an IEEE binary32 word, f32 and f64 widen
    exactly."""
    if x_dtype == "bf16":
        return (np.asarray(xbuf, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return np.asarray(xbuf).astype(np.float64)


def tol_blas(xbuf: np.ndarray, dims, A: list, x_dtype: str = "f64",
             chunk_cols: int = 1 << 15) -> tuple[float, float]:
    """(Tol, ||X||^2) of Sec. 5.2, the same definition as ``tol`` (a direct
    residual sum over every entry, FP64), taken over the columns of the mode-1
    unfolding in chunks so that large tensors finish in seconds:
    X_(1)(:, j) - A^(1) z_j with z_j = the Hadamard product of the rows
    A^(k)(i_k, :), k >= 2 (Eq. (3)), j numbered by Eq. (2). The product
    A^(1) z_j is a library matrix multiply."""
    A = [_f64(a) for a in A]
    dims = [int(d) for d in dims]
    I0 = dims[0]
    J = int(np.prod(dims[1:]))
    res = xx = 0.0
    for j0 in range(0, J, chunk_cols):
        j1 = min(J, j0 + chunk_cols)
        j = np.arange(j0, j1, dtype=np.int64)
        Z = np.ones((j1 - j0, A[0].shape[1]))
        for k in range(1, len(dims)):
            Z *= A[k][j % dims[k]]
            j //= dims[k]
        x = stored_values(xbuf[j0 * I0: j1 * I0], x_dtype).reshape(j1 - j0, I0)
        d = x - Z @ A[0].T
        res += float(np.einsum("ij,ij->", d, d))
        xx += float(np.einsum("ij,ij->", x, x))
    return res / xx, xx


def grad_row_scale(dims, n: int, idx, p, A: list, xbuf: np.ndarray, x_dtype: str, B: int,
                   terms: int | None = None) -> np.ndarray:
    """Componentwise size of each row of the mini-batch gradient of Eq. (11):
        scale_i = || |A^(n)_i| |H| ||  +  || sum_f s_f |x_f(i)| |z_f| ||,
    |H| = sum_f s_f |z_f| |z_f|^T, s_f = 1 / (B J_n p_f), z_f the sampled KRP
    row (Eq. (3)) and x_f the sampled fiber (Eq. (2)) of batch entry f. These
    are the sizes of the two products whose difference is G_i, against which
    the rounding error of any evaluation of G_i is measured. idx is B x N
    (column n ignored), A the factors the batch was drawn from. `terms` is the
    count of Eq. (11)'s 1/B (B / bs with sampled blocks of bs fibers)."""
    N = len(dims)
    strides = np.cumprod([1] + [int(d) for d in dims[:-1]])
    Jn = float(np.prod([float(d) for k, d in enumerate(dims) if k != n]))
    s = 1.0 / ((B if terms is None else terms) * Jn * np.asarray(p, dtype=np.float64))
    Z = np.ones((B, A[0].shape[1]))
    base = np.zeros(B, dtype=np.int64)
    for k in range(N):
        if k == n:
            continue
        ik = np.asarray(idx[:, k], dtype=np.int64)
        Z *= np.abs(A[k][ik])
        base += ik * strides[k]
    off = base[None, :] + np.arange(int(dims[n]), dtype=np.int64)[:, None] * strides[n]
    Xs = np.abs(stored_values(xbuf[off.ravel()], x_dtype).reshape(int(dims[n]), B))
    H = (Z * s[:, None]).T @ Z
    t1 = np.linalg.norm(np.abs(A[n]) @ H, axis=1)
    t2 = np.linalg.norm(Xs @ (Z * s[:, None]), axis=1)
    return t1 + t2
