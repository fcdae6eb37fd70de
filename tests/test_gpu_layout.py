"""The strided layout (cpd_config.x_layout = CPD_LAYOUT_STRIDED): the mode-1
replica alone (X column-major, the first mode padded to a multiple of 8), the
other modes' fibers (Eq. (2)) read from it with a stride instead of from their
own replicas. The server falls back to it when a request's replicas would not
fit.

The CUDA-core engine does the same arithmetic on the same entries whichever
layout it reads them from, so a strided run is compared bit for bit with the
replica run of the same configuration, besides teacher forcing against the
oracle."""
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


CASES = [
    # dims, R, B, x_dtype, sampling, step
    ((37, 29, 23), 5, 40, "f64", "euclidean", "fixed"),
    ((61, 47, 33), 7, 64, "f32", "leverage", "adagrad"),
    ((45, 30, 26, 19), 6, 77, "bf16", "euclidean", "adagrad"),
    ((50, 44, 36), 9, 96, "bf16", "uniform", "adagrad"),
]


@pytest.mark.parametrize("dims,R,B,xdt,sampling,step", CASES)
def test_strided_matches_replicas_bitwise_and_oracle(cpd, orc, dims, R, B, xdt, sampling, step):
    _, X, A0 = make_problem(dims, R, noise=0.05, x_dtype=xdt, lognormal_rows=True)
    kw = dict(dims=dims, R=R, B=B, x_dtype=xdt, sampling=sampling, step=step, alpha=0.01, seed=23, engine="simt")
    rep = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], **kw)
    strd = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], x_layout="strided", **kw)
    assert strd.describe()["x_layout"] == "strided" and rep.describe()["x_layout"] == "replicas"
    rep.sgd_iters(60)
    strd.sgd_iters(60)               # every mode drawn many times
    for a, b in zip(rep.factors(), strd.factors()):
        assert torch.isfinite(a).all()
        assert torch.equal(a, b)
    _, t_rep = rep.fit()
    _, t_str = strd.fit()
    assert t_str == t_rep            # the same pass over the same mode-1 replica
    # teacher forcing against the oracle on the strided context
    ocfg = orc.Config(dims=dims, R=R, B=B, sampling=sampling, step=step, x_dtype=xdt, alpha=0.01, seed=23)
    forced(strd, orc, ocfg, oracle_xbuf(X), 6, xdt)
    rep.close()
    strd.close()


def test_strided_grad_variance_equals_replicas(cpd):
    dims, R = (30, 25, 20), 4
    _, X, A0 = make_problem(dims, R, noise=0.1, x_dtype="f32")
    kw = dict(dims=dims, R=R, B=16, x_dtype="f32", sampling="euclidean", step="adagrad", seed=3, engine="simt")
    rep = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], **kw)
    strd = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], x_layout="strided", **kw)
    for n in range(3):
        v1, m1 = cpd.cpd_grad_variance(rep.ctx, n)
        v2, m2 = cpd.cpd_grad_variance(strd.ctx, n)
        assert v1 == v2 and m1 == m2
    rep.close()
    strd.close()


def test_strided_layout_rejects_replica_only_paths(cpd):
    dims, R = (40, 30, 20), 16
    _, X, A0 = make_problem(dims, R, x_dtype="bf16")
    with pytest.raises(cpd.CpdError) as e:
        cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=32, x_dtype="bf16",
                          x_layout="strided", engine="cluster")
    assert e.value.status == cpd.EINVAL
    d = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=32, x_dtype="bf16", x_layout="strided")
    assert d.describe()["engine"] == "simt"
    with pytest.raises(cpd.CpdError) as e:
        cpd.cpd_skrp(d.ctx, 0, 0, 1, X=torch.empty(32 * 40, dtype=torch.bfloat16, device="cuda"))
    assert e.value.status == cpd.EINVAL
    d.close()


def test_server_falls_back_to_strided_layout(cpd):
    """With strided_above_mb = 1, a request whose replicas need more than
    1 MiB runs strided on the CUDA-core engine and ends bitwise where the same
    strided configuration ends alone; a small request keeps its replicas."""
    big, small = ((96, 80, 72), 6), ((20, 18, 16), 3)
    srv = cpd.cpd_server_create(max_active=4, fit_every=64, strided_above_mb=1)
    runs = []
    for q, (dims, R) in enumerate((big, small)):
        _, X, A0 = make_problem(dims, R, noise=1e-2, x_dtype="bf16", seed=40 + q)
        cfg = cpd.make_config(dims, R, 64, sampling="euclidean", step="adagrad", x_dtype="bf16", seed=40 + q,
                              engine="tensor" if q == 0 else "simt")
        Xd, A0d = X.cuda(), [a.cuda() for a in A0]
        runs.append((dims, R, Xd, A0d, cpd.cpd_submit(srv, cfg, Xd, A0d, stop_fit=2.0, max_iters=256)))
    assert cpd.cpd_server_wait(srv, 300.0)
    for q, (dims, R, Xd, A0d, tk) in enumerate(runs):
        out = [torch.empty(d, R) for d in dims]
        st, res = cpd.cpd_poll(srv, tk, out)
        assert st == cpd.OK and res["done"] == 1
        assert res["layout"] == (1 if q == 0 else 0)
        solo = cpd.Decomposition(Xd, A0d, dims=dims, R=R, B=64, x_dtype="bf16", sampling="euclidean",
                                 step="adagrad", seed=40 + q, engine="simt",
                                 x_layout="strided" if q == 0 else "replicas")
        solo.sgd_iters(res["iters"])
        for a, b in zip(out, solo.factors()):
            assert torch.equal(a, b)
        solo.close()
    st = cpd.cpd_server_stats(srv)
    assert st["held"] == 0 and st["active"] == 0 and st["queued"] == 0
    cpd.cpd_server_destroy(srv)
