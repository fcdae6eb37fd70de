"""The serving loop (cpd_server_create / cpd_submit / cpd_poll): requests of
uneven shape and rank admitted by a memory budget run concurrently, and each
one's factors are exactly those of the same request run alone."""
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


REQS = [
    # dims, R, x_dtype, B, sampling, max_ctas
    ((60, 70, 80), 5, "bf16", 96, "euclidean", 0),
    ((90, 50, 40, 30), 8, "bf16", 128, "euclidean", 4),
    ((120, 110, 100), 16, "bf16", 256, "euclidean", 0),
    ((64, 64, 64), 10, "f32", 64, "leverage", 0),
    ((200, 150, 30), 32, "bf16", 512, "euclidean", 8),
    ((45, 55, 65, 35), 12, "f32", 100, "uniform", 2),
]


def _make(C, dims, R, xdt, B, sampling, seed, max_ctas=0):
    _, X, A0 = make_problem(dims, R, noise=1e-2, x_dtype=xdt, seed=seed, init_seed=seed + 100)
    cfg = C.make_config(dims, R, B, sampling=sampling, step="adagrad", x_dtype=xdt, seed=seed,
                        max_ctas=max_ctas)
    fdt = torch.float32 if xdt != "f64" else torch.float64
    return cfg, X.cuda(), [a.to(fdt).cuda() for a in A0]


def test_concurrent_requests_match_solo_runs(cpd):
    srv = cpd.cpd_server_create(max_active=8, fit_every=100)
    inputs, tickets = [], []
    for q, (dims, R, xdt, B, sampling, mc) in enumerate(REQS):
        cfg, X, A0 = _make(cpd, dims, R, xdt, B, sampling, 10 + q, mc)
        inputs.append((dims, R, xdt, B, sampling, mc, cfg, X, A0))
        tickets.append(cpd.cpd_submit(srv, cfg, X, A0, stop_fit=2.0, max_iters=300 + 50 * q))
    assert cpd.cpd_server_wait(srv, 300.0)
    for (dims, R, xdt, B, sampling, mc, cfg, X, A0), tk in zip(inputs, tickets):
        fdt = torch.float32 if xdt != "f64" else torch.float64
        out = [torch.empty(d, R, dtype=fdt) for d in dims]
        st, res = cpd.cpd_poll(srv, tk, out)
        assert st == cpd.OK and res["done"] == 1, res
        assert res["reached"] == 0 and res["iters"] > 0
        solo = cpd.Decomposition(X, A0, dims=dims, R=R, B=B, x_dtype=xdt, sampling=sampling,
                                 step="adagrad", seed=cfg.seed, max_ctas=mc)
        solo.sgd_iters(res["iters"])
        for a, b in zip(out, solo.factors()):
            assert torch.equal(a, b)
        fit, tol = solo.fit()
        assert tol == pytest.approx(res["tol"], rel=1e-12)
        solo.close()
    cpd.cpd_server_destroy(srv)


def test_budget_admits_one_at_a_time(cpd):
    reqs = [_make(cpd, (80, 70, 60), 6, "bf16", 64, "euclidean", 30 + q) for q in range(4)]
    srv = cpd.cpd_server_create(hbm_budget=16 << 20, max_active=8, fit_every=50)   # ~11 MB each
    tks = [cpd.cpd_submit(srv, cfg, X, A0, stop_fit=2.0, max_iters=200) for cfg, X, A0 in reqs]
    assert cpd.cpd_server_wait(srv, 300.0)
    res = [cpd.cpd_poll(srv, tk)[1] for tk in tks]
    assert all(r["done"] == 1 and r["status"] == cpd.OK for r in res)
    spans = sorted((r["t_start"], r["t_done"]) for r in res)
    for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
        assert s1 >= e0 - 1e-3      # the budget holds one request at a time
    with pytest.raises(cpd.CpdError) as e:
        cfg, X, A0 = _make(cpd, (300, 300, 300), 10, "f32", 64, "euclidean", 99)
        cpd.cpd_submit(srv, cfg, X, A0, stop_fit=2.0, max_iters=10)
    assert e.value.status == cpd.ENOMEM
    cpd.cpd_server_destroy(srv)


def test_fit_target_stops_a_request(cpd):
    dims, R = (40, 50, 60), 3
    A, X, _ = make_problem(dims, R, noise=0.0, x_dtype="f32", seed=5)
    g = torch.Generator().manual_seed(1)
    A0 = [(a + 0.02 * torch.randn(a.shape, generator=g, dtype=torch.float64)).float().cuda() for a in A]
    cfg = cpd.make_config(dims, R, 64, sampling="euclidean", step="fixed", alpha=0.1, x_dtype="f32", seed=5)
    srv = cpd.cpd_server_create(fit_every=100)
    tk = cpd.cpd_submit(srv, cfg, X.cuda(), A0, stop_fit=0.999, max_iters=50000)
    assert cpd.cpd_server_wait(srv, 300.0)
    st, res = cpd.cpd_poll(srv, tk)
    assert st == cpd.OK and res["reached"] == 1 and res["fit"] >= 0.999
    assert res["iters"] < 50000 and res["iters"] % 100 == 0
    cpd.cpd_server_destroy(srv)


def test_grouped_and_per_stream_serving_agree(cpd):
    """The same requests served with grouped launches and with a stream per
    request end bitwise alike (and like a solo run)."""
    reqs = [
        ((70, 60, 50), 6, "bf16", 128, "simt", 4),
        ((80, 40, 30, 20), 9, "bf16", 200, "simt", 0),
        ((150, 120, 90), 24, "bf16", 512, "tensor", 8),
        ((100, 90, 80), 16, "bf16", 256, "tensor", 2),
        ((60, 50, 40), 5, "f32", 64, "simt", 0),
        ((90, 80, 70), 20, "bf16", 300, "tensor", 0),
    ]
    made = []
    for q, (dims, R, xdt, B, engine, mc) in enumerate(reqs):
        _, X, A0 = make_problem(dims, R, noise=1e-2, x_dtype=xdt, seed=60 + q, init_seed=160 + q)
        cfg = cpd.make_config(dims, R, B, step="adagrad", x_dtype=xdt, seed=60 + q, engine=engine,
                              max_ctas=mc)
        made.append((dims, R, xdt, B, engine, mc, cfg, X.cuda(), [a.cuda() for a in A0]))
    outs = {}
    for grouping in (True, False):
        srv = cpd.cpd_server_create(max_active=8, fit_every=64, grouping=grouping)
        tks = [cpd.cpd_submit(srv, m[6], m[7], m[8], stop_fit=2.0, max_iters=200 + 30 * q)
               for q, m in enumerate(made)]
        assert cpd.cpd_server_wait(srv, 300.0)
        res = []
        for m, tk in zip(made, tks):
            out = [torch.empty(d, m[1], dtype=torch.float32) for d in m[0]]
            st, r = cpd.cpd_poll(srv, tk, out)
            assert st == cpd.OK, r
            res.append((r["iters"], r["tol"], out))
        cpd.cpd_server_destroy(srv)
        outs[grouping] = res
    for (it1, tol1, o1), (it2, tol2, o2), m in zip(outs[True], outs[False], made):
        assert it1 == it2
        assert tol1 == tol2
        for a, b in zip(o1, o2):
            assert torch.equal(a, b)
        dims, R, xdt, B, engine, mc, cfg, X, A0 = m
        solo = cpd.Decomposition(X, A0, dims=dims, R=R, B=B, x_dtype=xdt, step="adagrad",
                                 seed=cfg.seed, engine=engine, max_ctas=mc)
        solo.sgd_iters(it1)
        for a, b in zip(o1, solo.factors()):
            assert torch.equal(a, b)
        solo.close()
