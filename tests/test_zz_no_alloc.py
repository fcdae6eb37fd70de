"""cpd_tol_noalloc: the relative error without any device allocation.

Callers that cannot allocate device memory (their memory is owned by another
allocator, or an allocation's device synchronisation is not affordable in
their loop) use this entry point. It must agree with cpd_fit, the context-based
entry point that computes the same Tol, on two calls in a row -- the second
call runs on scratch left over from the first.
"""
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


# cpd_fit sums at most 16 (CUDA cores) or 32 (tensor cores) squared
# residuals in FP32 before adding them to its FP64 running sum (float
# factors); the allocation-free pass accumulates every entry in FP64. For a
# BF16 tensor cpd_fit forms x_hat from bf16 hi/lo pairs on the tensor cores
# (about 2^-15 relative per product). These runs are far from converged
# (residual comparable to X), where both effects stay below the tolerances.
@pytest.mark.parametrize("xdt,dims,R,rtol", [
    ("f64", (30, 20, 25), 4, 1e-12),
    ("f32", (64, 50, 40), 6, 1e-6),
    ("bf16", (48, 40, 36, 20), 5, 2e-5),
    ("bf16", (300, 1000, 1000), 32, 2e-5),
])
def test_noalloc_tol_matches_cpd_fit_twice(cpd, xdt, dims, R, rtol):
    _, X, A0 = make_problem(dims, R, noise=0.1, x_dtype=xdt)
    Xd = X.cuda()
    dec = cpd.Decomposition(Xd, [a.cuda() for a in A0], dims=dims, R=R, B=32, x_dtype=xdt,
                            sampling="euclidean", step="adagrad", seed=4)
    dec.sgd_iters(20)
    _, tol_ref = dec.fit()
    A = dec.factors("cuda")
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        cpd.cpd_tol_noalloc(dims, R, xdt, Xd, A, out)
        torch.cuda.synchronize()
        assert out.item() == pytest.approx(tol_ref, rel=rtol)
    # a second problem on the same scratch: other sizes, then the first again
    _, X2, A2 = make_problem((17, 9, 33), 3, noise=0.5, x_dtype="f32", seed=7)
    d2 = cpd.Decomposition(X2.cuda(), [a.cuda() for a in A2], dims=(17, 9, 33), R=3, B=8,
                           x_dtype="f32", sampling="uniform", step="fixed")
    _, tol2 = d2.fit()
    cpd.cpd_tol_noalloc((17, 9, 33), 3, "f32", X2.cuda(), [a.cuda().float() for a in A2], out)
    torch.cuda.synchronize()
    assert out.item() == pytest.approx(tol2, rel=1e-6)
    cpd.cpd_tol_noalloc(dims, R, xdt, Xd, A, out)
    torch.cuda.synchronize()
    assert out.item() == pytest.approx(tol_ref, rel=rtol)
    dec.close()
    d2.close()


def test_noalloc_rejects_oversize(cpd):
    dims = (4, 1025, 1024)                      # 1,049,600 mode-1 fibers > 2^20
    A = [torch.zeros(d, 2, device="cuda") for d in dims]
    X = torch.zeros(8, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(cpd.CpdError) as e:
        cpd.cpd_tol_noalloc(dims, 2, "f32", X, A, out)
    assert e.value.status == cpd.EINVAL
    assert "at most 1048576" in str(e.value)
    # sizes whose product overflows 64 bits are refused the same way
    with pytest.raises(cpd.CpdError) as e:
        cpd.cpd_tol_noalloc((4, 2**31, 2**31, 2**31), 2, "f32", X, A + [A[0]], out)
    assert e.value.status == cpd.EINVAL


@pytest.mark.parametrize("xdt,dims,R", [("f64", (13, 9, 11), 3), ("f32", (40, 33, 17), 5),
                                        ("bf16", (21, 12, 10, 7), 4)])
def test_noalloc_tol_matches_oracle(cpd, orc, xdt, dims, R):
    """Directly against the oracle's entry-by-entry residual sum (Sec. 5.2)."""
    _, X, A0 = make_problem(dims, R, noise=0.2, x_dtype=xdt)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    cpd.cpd_tol_noalloc(dims, R, xdt, X.cuda(), [a.cuda() for a in A0], out)
    torch.cuda.synchronize()
    want, _ = orc.tol(oracle_xbuf(X), [a.double().numpy() for a in A0], xdt, dims=dims)
    assert out.item() == pytest.approx(want, rel=1e-12 if xdt == "f64" else 1e-6)


def test_noalloc_zero_tensor_gives_nan(cpd):
    dims = (5, 6, 7)
    X = torch.zeros(int(np.prod(dims)), device="cuda")
    A = [torch.ones(d, 2, device="cuda") for d in dims]
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    cpd.cpd_tol_noalloc(dims, 2, "f32", X, A, out)
    torch.cuda.synchronize()
    assert np.isnan(out.item())
