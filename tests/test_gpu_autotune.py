"""cpd_autotune: the fastest of the applicable engines and CTA caps, handed
back as a configuration whose runs are reproducible."""
import pytest
import torch

from helpers import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cpd():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2103_04081_gb300 import build
    build.build()
    from paper_2103_04081_gb300 import cpd as C
    return C


@pytest.mark.parametrize("dims,R,xdt,engine", [
    ((200, 150, 120), 24, "bf16", "auto"),
    ((90, 80, 70), 6, "f32", "auto"),
    ((200, 150, 120), 24, "bf16", "tensor"),
])
def test_autotune_returns_a_runnable_reproducible_config(cpd, dims, R, xdt, engine):
    _, X, A0 = make_problem(dims, R, x_dtype=xdt)
    X, A0 = X.cuda(), [a.cuda() for a in A0]
    cfg = cpd.make_config(dims, R, 256, x_dtype=xdt, step="adagrad", seed=3, engine=engine)
    best, rate = cpd.cpd_autotune(cfg, X, A0, iters=64)
    assert rate > 0
    assert best.engine in (1, 2, 3, 4) and best.max_ctas >= 0
    if engine == "tensor":
        assert best.engine == 2
    if xdt == "f32":
        assert best.engine == 1                      # tensor cores need BF16 tensors
    # the chosen configuration runs, and twice the same way
    outs = []
    for _ in range(2):
        ctx = cpd.cpd_init(best, X, A0)
        cpd.cpd_sgd_iters(ctx, 100)
        out = [torch.empty(d, R) for d in dims]
        cpd.cpd_get_factors(ctx, out)
        cpd.cpd_destroy(ctx)
        outs.append(out)
    for a, b in zip(*outs):
        assert torch.isfinite(a).all() and torch.equal(a, b)
