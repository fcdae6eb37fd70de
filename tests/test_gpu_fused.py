"""The fused engine (cpd_config.engine = 5): gradient and step of one
iteration in one launch, a thread-block cluster per 128-row tile of A^(n)
whose CTAs split the batch and sum the partials M and H (Eq. (11)) in
distributed shared memory in ascending rank. max_ctas is its cluster size.

Teacher-forced against the FP64 oracle (draws and p_f bit-exact, G and the
updated rows within the tensor-core tolerances), bitwise reproducible under
any chunking of a call and between graph replays and plain launches, and at
the 1000^3 workload's full size in the launch the bench times."""
import numpy as np
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


def _ocfg(orc, dims, R, B, sampling, step, seed, **kw):
    return orc.Config(dims=tuple(dims), R=R, B=B, sampling=sampling, step=step, x_dtype="bf16", seed=seed, **kw)


FUSED = [
    # dims, R, B, sampling, cluster size (0 = chosen), fibers per CTA, rows per cluster
    ((200, 150, 100), 50, 300, "euclidean", 0, 48, 128),     # ragged row tile (200 = 128 + 72), 8 CTAs
    ((40, 36, 130, 28), 12, 77, "euclidean", 16, 16, 128),    # 4-way; ranks 5..15 draw no fiber
    ((129, 257, 70), 64, 2048, "leverage", 16, 128, 128),     # R = 64; tiles of 1 row (129, 257)
    ((300, 64, 90), 20, 1024, "uniform", 8, 128, 128),
    ((90, 70, 60), 8, 100, "euclidean", 1, 112, 128),         # one-CTA clusters
    ((260, 200, 150), 24, 3328, "euclidean", 16, 208, 128),   # the largest tile of fibers
    # 8 tiles of 128 rows against the 7 clusters of 16 CTAs a GB300 co-schedules:
    # clusters of 256 rows (two MMA tiles), the last one ragged (1000 = 3 x 256 + 232)
    ((1000, 40, 30), 32, 2048, "euclidean", 16, 128, 256),
]


@pytest.mark.parametrize("dims,R,B,sampling,cs,fpc,rows", FUSED)
def test_teacher_forced_fused(cpd, orc, dims, R, B, sampling, cs, fpc, rows):
    A, X, A0 = make_problem(dims, R, x_dtype="bf16", lognormal_rows=True)
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype="bf16",
                            sampling=sampling, step="adagrad", seed=77, engine="fused", max_ctas=cs)
    d = dec.describe()
    assert d["engine"] == "fused" and d["fibers_per_cta"] == fpc and d["rows_per_cta"] == rows, d
    assert d["update_grid"] == 0 and d["grad_grid"] == d["cluster"] * -(-max(dims) // rows), d
    ocfg = _ocfg(orc, dims, R, B, sampling, "adagrad", 77)
    worst = forced(dec, orc, ocfg, oracle_xbuf(X), 12, "bf16_tensor")
    print(dims, R, B, sampling, cs, worst, d)
    dec.close()


@pytest.mark.parametrize("step,kw", [("fixed", dict(alpha=0.05)), ("decay", dict(beta=0.05, gamma=2.0))])
def test_fused_other_steps_and_nonneg(cpd, orc, step, kw):
    dims, R, B = (150, 120, 90), 24, 256
    _, X, A0 = make_problem(dims, R, x_dtype="bf16", nonneg=True, noise=5e-2)
    kw = dict(kw, constraint="nonneg")
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype="bf16",
                            sampling="euclidean", step=step, seed=5, engine="fused", max_ctas=4, **kw)
    ocfg = _ocfg(orc, dims, R, B, "euclidean", step, 5, **kw)
    forced(dec, orc, ocfg, oracle_xbuf(X), 6, "bf16_tensor")
    dec.sgd_iters(300)
    assert all(bool((a >= 0).all()) for a in dec.factors())
    fit, _ = dec.fit()
    assert np.isfinite(fit)
    dec.close()


def test_fused_chunking_graph_and_plain_are_bitwise(cpd):
    """100 iterations in one call, in calls of 1, 31, 32, 5, 31, and as plain
    (profiled) launches give the same factors and AdaGrad state bit for bit."""
    dims, R, B = (220, 130, 100), 32, 1024
    _, X, A0 = make_problem(dims, R, x_dtype="bf16")
    kw = dict(dims=dims, R=R, B=B, x_dtype="bf16", sampling="euclidean", step="adagrad", seed=9,
              engine="fused", max_ctas=16)
    d1 = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], **kw)
    d1.sgd_iters(100)
    d2 = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], **kw)
    for q in (1, 31, 32, 5, 31):
        d2.sgd_iters(q)
    d3 = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], **kw)
    cpd.cpd_profile(d3.ctx, True)          # plain launches bracketed by events
    d3.sgd_iters(100)
    launches, grad_ms, _ = cpd.cpd_profile_read(d3.ctx)
    assert launches == 100 and grad_ms > 0.0
    for d in (d2, d3):
        assert d.t == 100
        for a, b in zip(d1.factors(), d.factors()):
            assert torch.equal(a, b)
        for a, b in zip(d1.adagrad(), d.adagrad()):
            assert torch.equal(a, b)
    for d in (d1, d2, d3):
        d.close()


def test_fused_follows_cluster_engine_free_run(cpd):
    """The fused and the cluster engines run the same method with different
    summation orders; over a free run of 800 iterations from the same start
    their fits agree within 1e-3 and both improve on the start."""
    dims, R, B = (300, 250, 200), 24, 1024
    _, X, A0 = make_problem(dims, R, x_dtype="bf16", noise=1e-2, lognormal_rows=True)
    fits = {}
    for engine in ("cluster", "fused"):
        d = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype="bf16",
                              sampling="euclidean", step="adagrad", seed=3, engine=engine)
        f0, _ = d.fit()
        d.sgd_iters(800)
        fits[engine], _ = d.fit()
        assert fits[engine] > f0
        d.close()
    print(fits)
    assert abs(fits["cluster"] - fits["fused"]) <= 1e-3, fits


@pytest.mark.parametrize("kw,msg", [
    (dict(max_ctas=3), "cluster size"),
    (dict(max_ctas=32), "cluster size"),
    (dict(B=4000, max_ctas=16), "208 fibers"),
    (dict(tile_fibers=32), "take no tile_rows"),
    (dict(x_dtype="f32"), "tensor-core engine"),
])
def test_fused_rejects_invalid_configs(cpd, kw, msg):
    dims, R = (64, 48, 40), 8
    base = dict(dims=dims, R=R, B=256, x_dtype="bf16", engine="fused")
    base.update(kw)
    _, X, A0 = make_problem(dims, R, x_dtype=base["x_dtype"])
    with pytest.raises(cpd.CpdError) as e:
        cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], **base)
    assert e.value.status == cpd.EINVAL and msg in str(e.value), str(e.value)


def test_fused_trace_phases_in_order(cpd):
    dims, R, B = (500, 400, 300), 32, 2048
    _, X, A0 = make_problem(dims, R, x_dtype="bf16")
    d = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype="bf16",
                          sampling="euclidean", step="adagrad", seed=1, engine="fused")
    d.sgd_iters(5)
    cpd.cpd_trace(d.ctx, True)
    d.sgd_iters(1)
    tr = cpd.cpd_trace_read(d.ctx)
    cpd.cpd_trace(d.ctx, False)
    order = [0, 15, 1, 2, 16, 3, 4, 5, 6, 7, 8, 9, 10, 17, 11, 14]
    seq = [int(tr[k]) for k in order]
    assert all(v > 0 for v in seq), seq
    assert all(b >= a for a, b in zip(seq, seq[1:])), seq
    d.close()
