"""Blocks first, then sampling (Remark 1; cpd_config.block): the batch is
B / bs sampled blocks of bs consecutive mode-n fibers. Teacher-forced against
the oracle's block sampling on every engine that takes it (indices and p_f
bit-exact, G and the step within each engine's tolerances), and block = 1
bitwise equal to per-fiber sampling."""
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


CASES = [
    # engine, x_dtype, dims, R, B, block, sampling, layout
    ("simt", "f64", (32, 24, 20), 5, 48, 4, "euclidean", "replicas"),
    ("simt", "f32", (64, 48, 30), 8, 128, 8, "leverage", "replicas"),
    ("simt", "f32", (40, 32, 24, 18), 6, 96, 4, "uniform", "replicas"),
    ("simt", "bf16", (96, 80, 72), 12, 256, 16, "euclidean", "strided"),
    ("tensor", "bf16", (200, 152, 100), 50, 304, 8, "euclidean", "replicas"),
    ("cluster", "bf16", (300, 64, 90), 20, 1024, 4, "euclidean", "replicas"),
    ("fused", "bf16", (256, 128, 96), 32, 2048, 16, "euclidean", "replicas"),
    ("fused", "bf16", (128, 96, 40, 30), 16, 512, 8, "leverage", "replicas"),
]


@pytest.mark.parametrize("engine,xdt,dims,R,B,bs,sampling,layout", CASES)
def test_teacher_forced_block_sampling(cpd, orc, engine, xdt, dims, R, B, bs, sampling, layout):
    _, X, A0 = make_problem(dims, R, x_dtype=xdt, lognormal_rows=True)
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype=xdt,
                            sampling=sampling, step="adagrad", seed=13, engine=engine, block=bs,
                            x_layout=layout)
    assert dec.describe()["engine"] == engine and dec.describe()["block"] == bs
    ocfg = orc.Config(dims=dims, R=R, B=B, sampling=sampling, step="adagrad", x_dtype=xdt, seed=13, block=bs)
    key = "bf16_tensor" if engine in ("tensor", "cluster", "fused") else xdt
    worst = forced(dec, orc, ocfg, oracle_xbuf(X), 9, key)
    n, idx, p = dec.last_sample()
    k0 = 1 if n == 0 else 0
    rows = idx.numpy().astype(int)
    assert (rows[::bs, k0] % bs == 0).all()                  # aligned blocks of the first other mode
    print(engine, xdt, dims, bs, sampling, layout, worst)
    dec.close()


def test_block_one_is_per_fiber_sampling(cpd):
    dims, R, B = (80, 60, 40), 16, 256
    _, X, A0 = make_problem(dims, R, x_dtype="bf16")
    runs = []
    for bs in (0, 1):
        d = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype="bf16",
                              sampling="euclidean", step="adagrad", seed=3, engine="cluster", block=bs)
        d.sgd_iters(70)
        runs.append(d)
    for a, b in zip(runs[0].factors(), runs[1].factors()):
        assert torch.equal(a, b)
    for d in runs:
        d.close()


def test_block_sampling_rejected_where_fibers_are_drawn_one_by_one(cpd):
    dims, R = (64, 48, 40), 8
    _, X, A0 = make_problem(dims, R, x_dtype="bf16")
    d = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=64, x_dtype="bf16", block=4)
    with pytest.raises(cpd.CpdError) as e:
        cpd.cpd_skrp(d.ctx, 0, 0, 1)
    assert e.value.status == cpd.EINVAL
    with pytest.raises(cpd.CpdError) as e:
        cpd.cpd_grad_variance(d.ctx, 0)
    assert e.value.status == cpd.EINVAL
    d.close()
