"""Shared helpers of the GPU parity tests: problem set-up and teacher forcing.

Both sides take their inputs from paper_2103_04081_gb300.inputs; the oracle
is fed the same stored tensor bytes and, at every teacher-forced step, the
GPU's current factors and AdaGrad state.

Tolerances. Each checked iteration compares the gradient and the updated
factor three ways:
  * the whole-matrix relative Frobenius error (the ceilings the method's
    precisions state: FP64 ~1e-11, FP32 1e-5, BF16 tensor cores 2e-2);
  * row by row, relative to a componentwise scale of the row,
        scale_i = || |A_i| |H| ||  +  || sum_f s_f |x_f(i)| |z_f| ||,
    |H| = sum_f s_f |z_f| |z_f|^T, s_f = 1/(B J_n p_f) -- the size of the two
    products whose difference is G_i (Eq. (11)), so that rounding errors are
    measured against what they scale with, not against G_i itself, which may
    be small by cancellation. A kernel bug confined to a few rows (a ragged
    row tile, a dropped fiber group, one bad column of the hi/lo split) moves
    its rows by O(1) of this scale;
  * the updated factor, whole-matrix and row by row (relative to the larger
    of its new and old norms), against the oracle's step (Eq. (12), (13a)-
    (13b), FP64) applied to the GPU's own gradient, and the AdaGrad state
    likewise. The gradient is already checked against the oracle's; checking
    the updated factor against the oracle's updated factor instead would fold
    in the step's sensitivity to g, which has no bound: on an entry's first
    AdaGrad update (S = 0) the step eta g / sqrt(b + g^2), b = 1e-12, goes from
    0 to eta as g goes from 0 to about 1e-5, so a gradient entry of a few 1e-6
    (it happens: one in 4800 entries of a 200 x 24 factor) turns an admissible
    gradient error into an O(eta) change of that entry. That comparison is
    reported as A_oracle.
The row bounds follow from the arithmetic: FP64 carries ~1e-16 per
operation; FP32 accumulations over B fibers stay within ~sqrt(B) 2^-24;
the tensor-core path represents s_f z_f as a bf16 hi/lo pair (relative
error <= 2^-16 after the two roundings), with FP32 accumulation in tensor
memory, so its rows stay near 1e-5 of their scale.
"""
import numpy as np
import torch

from paper_2103_04081_gb300 import inputs as IN

# Row bounds: about ten times the worst row error measured over every parity
# case on a GB300 (FP64 4e-16 / 9e-16, FP32 on CUDA cores 3.4e-7 / 1.6e-7,
# tensor cores 2.6e-6 / 4.8e-6), and within the rounding model above (the
# tensor-core bound 2e-5 is the bf16 hi/lo representation error 2^-16 of
# s_f z_f with room for the FP32 accumulation).
TOL = {"f64": dict(G=1e-11, A=1e-13, G_row=1e-13, A_row=1e-13),
       "f32": dict(G=1e-5, A=1e-6, G_row=3e-6, A_row=2e-6),
       "bf16": dict(G=1e-5, A=1e-6, G_row=3e-6, A_row=2e-6),
       "bf16_tensor": dict(G=2e-2, A=1e-4, G_row=2e-5, A_row=2e-5)}


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


def grad_row_scale(dims, n, idx, p, A, xbuf, x_dtype, B, terms=None):
    """scale_i of every row of G^(n) for the batch (idx, p) (see the module docstring)."""
    from oracle import oracle as O
    return O.grad_row_scale(dims, n, idx, p, A, xbuf, x_dtype, B, terms)


def row_errors(G_gpu, G_orc, scale, A_gpu, A_orc, A_prev):
    """(max scaled row error of G, max relative row error of A^(n))."""
    dG = np.linalg.norm(np.asarray(G_gpu, np.float64) - G_orc, axis=1)
    eg = float(np.max(dG / np.maximum(scale, 1e-300))) if dG.size else 0.0
    dA = np.linalg.norm(np.asarray(A_gpu, np.float64) - A_orc, axis=1)
    den = np.maximum(np.linalg.norm(A_orc, axis=1), np.linalg.norm(A_prev, axis=1))
    ea = float(np.max(np.where(den > 0, dA / np.where(den > 0, den, 1.0), dA))) if dA.size else 0.0
    return eg, ea


def teacher_forced(dec, orc, ocfg, xbuf, steps, tol_G, tol_A, check_every=1, tol_G_row=None,
                   tol_A_row=None):
    """Run `steps` GPU iterations; before each checked one, start the oracle from
    the GPU's state at the same t and compare n, idx, p (bit-exact), G and A^(n)
    (whole-matrix and row by row, see the module docstring)."""
    worst = {"G": 0.0, "A": 0.0, "G_row": 0.0, "A_row": 0.0, "A_oracle": 0.0}
    dims = tuple(int(d) for d in ocfg.dims)
    for q in range(steps):
        if q % check_every:
            dec.sgd_iters(1)
            continue
        t = dec.t
        A = [a.double().numpy().copy() for a in dec.factors()]
        A_prev = [a.copy() for a in A]
        S = [s.numpy().copy() for s in dec.adagrad()]
        S_prev = [s.copy() for s in S]
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
        # the oracle's step applied to the GPU's gradient
        adagrad = ocfg.step == "adagrad"
        A_step = A_prev[n].copy()
        S_step = S_prev[n].copy() if adagrad else None
        orc.update(ocfg, t, A_step, S_step, G.numpy())
        eA = rel(A1[n].double().numpy(), A_step)
        if adagrad:
            eS = rel(dec.adagrad()[n].numpy(), S_step)
            assert eS <= 1e-12, (t, n, "S", eS)
        for k in range(len(A)):
            if k != n:
                np.testing.assert_array_equal(A1[k].double().numpy(), A[k])
        scale = grad_row_scale(dims, n, out["idx"], out["p"], A_prev, xbuf, ocfg.x_dtype, ocfg.B,
                               ocfg.B // max(1, ocfg.block))
        eGr, eAr = row_errors(G.numpy(), out["G"], scale, A1[n].double().numpy(), A_step, A_prev[n])
        assert eG <= tol_G, (t, n, eG)
        assert eA <= tol_A, (t, n, eA)
        if tol_G_row is not None:
            assert eGr <= tol_G_row, ("row", t, n, eGr)
        if tol_A_row is not None:
            assert eAr <= tol_A_row, ("row", t, n, eAr)
        worst["G"] = max(worst["G"], eG)
        worst["A"] = max(worst["A"], eA)
        worst["G_row"] = max(worst["G_row"], eGr)
        worst["A_row"] = max(worst["A_row"], eAr)
        worst["A_oracle"] = max(worst["A_oracle"], rel(A1[n].double().numpy(), A[n]))
    dec.sync()
    return worst


def forced(dec, orc, ocfg, xbuf, steps, key, **kw):
    """teacher_forced with every tolerance of TOL[key]."""
    t = TOL[key]
    return teacher_forced(dec, orc, ocfg, xbuf, steps, t["G"], t["A"], tol_G_row=t["G_row"],
                          tol_A_row=t["A_row"], **kw)
