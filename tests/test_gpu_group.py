"""Grouped launches (cpd_group_create / cpd_group_iters): one gradient launch
and one update launch per iteration (plus one Gram and one leverage-row
launch when members sample by leverage) advance many decompositions, and
every member ends bitwise where it ends when run alone."""
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


# dims, R, B, x_dtype, sampling, step, max_ctas, extra
CLASSES = {
    "simt_f32": [
        ((70, 61, 45), 5, 37, "f32", "euclidean", "adagrad", 0, {}),
        ((150, 70, 33), 10, 100, "f32", "uniform", "fixed", 4, dict(alpha=0.002)),
        ((33, 17, 9, 5), 3, 20, "f32", "euclidean", "decay", 2, dict(beta=0.01, gamma=2.0)),
        ((120, 90, 200), 24, 512, "f32", "euclidean", "adagrad", 8, {}),
        ((90, 130, 40), 7, 64, "f32", "leverage", "adagrad", 0, {}),
        ((64, 48, 30), 8, 96, "f32", "euclidean", "adagrad", 0, dict(block=4)),      # sampled blocks
    ],
    "simt_leverage": [
        ((80, 70, 60), 6, 48, "f32", "leverage", "adagrad", 0, {}),
        ((150, 110, 100), 70, 64, "f32", "leverage", "fixed", 8, dict(alpha=0.001)),   # L past shared memory
        ((40, 36, 30, 28), 12, 100, "f32", "leverage", "decay", 2, dict(beta=0.01, gamma=2.0)),
    ],
    "simt_bf16": [
        ((40, 36, 30, 28), 12, 200, "bf16", "euclidean", "adagrad", 0, {}),
        ((90, 50, 64), 7, 300, "bf16", "euclidean", "adagrad", 3, {}),
    ],
    "tensor_bf16": [
        ((200, 150, 100), 50, 300, "bf16", "euclidean", "adagrad", 0, {}),
        ((300, 64, 90), 20, 1024, "bf16", "uniform", "adagrad", 8, {}),
        ((60, 70, 55, 40), 16, 512, "bf16", "euclidean", "adagrad", 4, {}),
        ((129, 257, 70), 64, 256, "bf16", "euclidean", "fixed", 2, dict(alpha=0.0005)),
        ((150, 120, 90), 24, 256, "bf16", "leverage", "adagrad", 4, {}),
        ((128, 96, 60), 24, 256, "bf16", "euclidean", "adagrad", 4, dict(block=8)),
    ],
}


def _pair(C, q, case, engine):
    dims, R, B, xdt, sampling, step, mc, kw = case
    _, X, A0 = make_problem(dims, R, x_dtype=xdt, seed=40 + q, init_seed=140 + q, lognormal_rows=True)
    X, A0 = X.cuda(), [a.cuda() for a in A0]
    mk = lambda: C.Decomposition(X, A0, dims=dims, R=R, B=B, x_dtype=xdt, sampling=sampling, step=step,
                                 seed=7 + q, engine=engine, max_ctas=mc, **kw)
    return mk(), mk()


@pytest.mark.parametrize("cls", list(CLASSES))
def test_group_matches_solo_runs_bitwise(cpd, cls):
    engine = "tensor" if cls.startswith("tensor") else "simt"
    pairs = [_pair(cpd, q, case, engine) for q, case in enumerate(CLASSES[cls])]
    solo, grouped = [p[0] for p in pairs], [p[1] for p in pairs]
    for d in grouped:
        assert d.describe()["engine"] == engine
    grp = cpd.cpd_group_create([d.ctx for d in grouped])
    iters = 3 * 32 + 5                       # graph-replayed chunks and a plain remainder
    cpd.cpd_group_iters(grp, iters)
    cpd.cpd_group_iters(grp, 40)
    torch.cuda.synchronize()
    for s in solo:
        s.sgd_iters(iters + 40)
    torch.cuda.synchronize()
    for s, g in zip(solo, grouped):
        assert s.t == g.t == iters + 40
        for a, b in zip(s.factors(), g.factors()):
            assert torch.isfinite(a).all()
            assert torch.equal(a, b)
        if s.cfg.step == 1:                  # AdaGrad state
            for a, b in zip(s.adagrad(), g.adagrad()):
                assert torch.equal(a, b)
        n1, idx1, p1 = s.last_sample()
        n2, idx2, p2 = g.last_sample()
        assert n1 == n2 and torch.equal(idx1, idx2) and torch.equal(p1, p2)
        assert s.fit() == g.fit()
    cpd.cpd_group_destroy(grp)
    for d in solo + grouped:
        d.close()


def test_group_rejects_incompatible_members(cpd):
    a = _pair(cpd, 0, CLASSES["simt_f32"][0], "simt")[0]
    b = _pair(cpd, 1, CLASSES["simt_bf16"][0], "simt")[0]
    c = _pair(cpd, 2, CLASSES["tensor_bf16"][0], "cluster")[0]
    for members in ([a.ctx, b.ctx], [c.ctx], [a.ctx, a.ctx]):
        with pytest.raises(cpd.CpdError) as e:
            cpd.cpd_group_create(members)
        assert e.value.status == cpd.EINVAL
    for d in (a, b, c):
        d.close()
