"""cpd_autotune: the fastest of the applicable engines, CTA caps and tile
shapes, handed back as a configuration whose runs are reproducible; explicit
tile shapes keep parity with the oracle."""
import pytest
import torch

from helpers import forced, make_problem, oracle_xbuf

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
    assert best.tile_rows in (0, 32, 128) and best.tile_fibers in (0, 32, 64, 128)
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


@pytest.mark.parametrize("dims,R,B,xdt,engine,rows,fibers,key", [
    ((90, 70, 50), 6, 100, "f32", "simt", 32, 24, "f32"),
    ((90, 70, 50), 6, 100, "f32", "simt", 128, 0, "f32"),
    ((260, 200, 150), 24, 256, "bf16", "tensor", 128, 32, "bf16_tensor"),
    ((260, 200, 150), 24, 256, "bf16", "cluster", 0, 64, "bf16_tensor"),
])
def test_explicit_tile_shapes_keep_parity(cpd, orc, dims, R, B, xdt, engine, rows, fibers, key):
    _, X, A0 = make_problem(dims, R, x_dtype=xdt, lognormal_rows=True)
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype=xdt,
                            sampling="euclidean", step="adagrad", seed=8, engine=engine,
                            tile_rows=rows, tile_fibers=fibers)
    d = dec.describe()
    assert d["engine"] == engine
    if fibers:
        assert d["fibers_per_cta"] == fibers and d["fiber_groups"] == (B + fibers - 1) // fibers
    if rows and engine == "simt":              # at most the longest mode, rounded up to 8
        assert d["rows_per_cta"] == min(rows, (max(dims) + 7) // 8 * 8)
    dec.sgd_iters(10)
    ocfg = orc.Config(dims=dims, R=R, B=B, sampling="euclidean", step="adagrad", x_dtype=xdt, seed=8)
    forced(dec, orc, ocfg, oracle_xbuf(X), 4, key)
    dec.close()
