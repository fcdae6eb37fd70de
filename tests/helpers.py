"""Shared helpers of the GPU parity tests: problem set-up and teacher forcing.

Both sides take their inputs from paper_2103_04081_gb300.inputs; the oracle
is fed the same stored tensor bytes and, at every teacher-forced step, the
GPU's current factors and AdaGrad state.
"""
import numpy as np
import torch

from paper_2103_04081_gb300 import inputs as IN

TOL = {"f64": dict(G=1e-11, A=1e-13), "f32": dict(G=1e-5, A=1e-6),
       "bf16": dict(G=1e-5, A=1e-6), "bf16_tensor": dict(G=2e-2, A=1e-4)}


def make_problem(dims, R, noise=1e-2, x_dtype="f32", seed=0, init_seed=1, device="cpu",
                 lognormal_rows=False, congruence=0.0, nonneg=False):
    A = IN.factors(dims, R, seed, congruence=congruence, lognormal_rows=lognormal_rows,
                   nonneg=nonneg, device=device)
    X = IN.cp_tensor(A, noise, seed, x_dtype)
    A0 = IN.init_factors(dims, R, init_seed,
                         dtype=torch.float64 if x_dtype == "f64" else torch.float32, nonneg=nonneg)
    return A, X, A0


def oracle_xbuf(X: torch.Tensor) -> np.ndarray:
    """Flat column-major host buffer of the stored tensor, as the oracle reads it."""
    t = X.detach().cpu()
    if t.dtype == torch.bfloat16:
        return t.view(torch.int16).numpy().view(np.uint16).copy()
    return t.numpy().copy()


def rel(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def teacher_forced(dec, orc, ocfg, xbuf, steps, tol_G, tol_A, check_every=1):
    """Run `steps` GPU iterations; before each checked one, start the oracle from
    the GPU's state at the same t and compare n, idx, p (bit-exact), G and A^(n)."""
    worst = {"G": 0.0, "A": 0.0}
    for q in range(steps):
        if q % check_every:
            dec.sgd_iters(1)
            continue
        t = dec.t
        A = [a.double().numpy().copy() for a in dec.factors()]
        S = [s.numpy().copy() for s in dec.adagrad()]
        out = orc.step(ocfg, t, None, A, S, xbuf=xbuf)
        assert out["status"] == orc.OK
        dec.sgd_iters(1)
        n, idx, p = dec.last_sample()
        assert n == out["n"], (t, n, out["n"])
        np.testing.assert_array_equal(idx.numpy().astype(np.int64), out["idx"])
        np.testing.assert_array_equal(p.numpy(), out["p"])
        n2, G = dec.last_gradient()
        eG = rel(G.numpy(), out["G"])
        A1 = dec.factors()
        eA = rel(A1[n].double().numpy(), A[n])
        for k in range(len(A)):
            if k != n:
                np.testing.assert_array_equal(A1[k].double().numpy(), A[k])
        assert eG <= tol_G, (t, n, eG)
        assert eA <= tol_A, (t, n, eA)
        worst["G"] = max(worst["G"], eG)
        worst["A"] = max(worst["A"], eA)
    dec.sync()
    return worst
