"""The gradient-variance diagnostic (cpd_grad_variance, Thm 10 / Table 1 /
Fig. 3) against the oracle: the exact variance by enumerating every
single-fiber mini-batch with its probability."""
import numpy as np
import pytest
import torch

from helpers import make_problem, oracle_xbuf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cpd():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2103_04081_gb300 import build
    build.build()
    from paper_2103_04081_gb300 import cpd as C
    return C


def oracle_variance(orc, dims, R, B, sampling, x_dtype, xbuf, A, n):
    """E||G - E G||^2 and ||E G||^2 of the B-draw gradient of mode n, from the
    oracle's gradient of every one-fiber batch (B draws are i.i.d.)."""
    cfg1 = orc.Config(dims=tuple(dims), R=R, B=1, sampling=sampling, x_dtype=x_dtype)
    others = [k for k in range(len(dims)) if k != n]
    mean = np.zeros((dims[n], R))
    second = 0.0
    for j in range(int(np.prod([dims[k] for k in others]))):
        idx = np.full((1, len(dims)), -1, dtype=np.int64)
        rest = j
        for k in others:                        # Eq. (2): first mode fastest
            idx[0, k] = rest % dims[k]
            rest //= dims[k]
        st, p, G = orc.gradient_for_batch(cfg1, n, idx, xbuf, A)
        assert st == orc.OK
        if p[0] == 0.0:
            continue
        mean += p[0] * G
        second += p[0] * float((G * G).sum())
    m2 = float((mean * mean).sum())
    return (second - m2) / B, m2


@pytest.mark.parametrize("dims,R,B,xdt,sampling", [
    ((6, 5, 4), 3, 7, "f32", "euclidean"),
    ((7, 6, 5), 2, 3, "f64", "leverage"),
    ((5, 6, 4, 3), 2, 11, "bf16", "uniform"),
    ((9, 8, 7), 4, 16, "bf16", "euclidean"),
])
def test_variance_matches_oracle_enumeration(cpd, orc, dims, R, B, xdt, sampling):
    _, X, A0 = make_problem(dims, R, x_dtype=xdt, lognormal_rows=True, noise=0.1)
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype=xdt,
                            sampling=sampling, step="adagrad", seed=3, engine="simt")
    xbuf = oracle_xbuf(X)
    for steps in (0, 7):                       # initial factors, then after a deferred CDF rebuild
        dec.sgd_iters(steps)
        A = [a.double().numpy() for a in dec.factors()]
        for n in range(len(dims)):
            v_gpu, m_gpu = dec.grad_variance(n)
            v_orc, m_orc = oracle_variance(orc, dims, R, B, sampling, xdt, xbuf, A, n)
            assert v_orc > 0
            assert v_gpu == pytest.approx(v_orc, rel=2e-5), (steps, n)
            assert m_gpu == pytest.approx(m_orc, rel=2e-5), (steps, n)
    dec.close()


def test_variance_diagnostic_does_not_change_the_run(cpd):
    """Completing a deferred CDF rebuild for the diagnostic leaves the run bitwise unchanged."""
    dims, R = (60, 50, 40), 6
    _, X, A0 = make_problem(dims, R, x_dtype="f32")
    mk = lambda: cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=64, x_dtype="f32",
                                   sampling="euclidean", step="adagrad", seed=9)
    a, b = mk(), mk()
    for q in range(5):
        a.sgd_iters(37)
        b.sgd_iters(37)
        b.grad_variance(q % 3)
    for x, y in zip(a.factors(), b.factors()):
        assert torch.equal(x, y)
    a.close()
    b.close()
