"""GPU path against the FP64 CPU oracle, through the C-ABI.

Teacher forcing: before each checked iteration the oracle starts from the
GPU's factors and AdaGrad state at the same t. The mode n, the sampled
indices and the fiber probabilities p_f must agree bit for bit; the
gradient and the updated factor within the dtype's tolerance, both as a
whole (relative Frobenius norm: FP64 1e-11, FP32 1e-5, BF16 tensors on the
CUDA-core engine 1e-5, BF16 on the tensor-core engines 2e-2, the ceilings
stated for the method's precisions) and row by row against the arithmetic's
own error bound (tests/helpers.py states both).
"""
import numpy as np
import pytest
import torch

from helpers import TOL, forced, make_problem, oracle_xbuf, rel
from paper_2103_04081_gb300 import inputs as IN

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cpd():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2103_04081_gb300 import build
    build.build()
    from paper_2103_04081_gb300 import cpd as C
    return C


def _ocfg(orc, dims, R, B, x_dtype, sampling, step, seed, **kw):
    return orc.Config(dims=tuple(dims), R=R, B=B, sampling=sampling, step=step,
                      x_dtype=x_dtype, seed=seed, alpha=kw.get("alpha", 0.1),
                      eta=kw.get("eta", 0.1), b=kw.get("b", 1e-12), beta=kw.get("beta", 1.0),
                      gamma=kw.get("gamma", 1.0), constraint=kw.get("constraint", "none"))


SMALL = [
    # dims, R, B, x_dtype, sampling, step, extra
    ((70, 61, 45), 5, 37, "f64", "euclidean", "fixed", {}),
    ((150, 70, 33), 10, 100, "f32", "euclidean", "adagrad", {}),
    ((90, 130, 40), 7, 64, "f32", "leverage", "adagrad", {}),
    ((50, 60, 70), 4, 50, "f32", "uniform", "decay", dict(beta=0.01, gamma=2.0)),
    ((40, 36, 30, 28), 12, 200, "bf16", "euclidean", "adagrad", {}),
    ((33, 17, 9, 5, 3), 3, 20, "f32", "euclidean", "fixed", dict(alpha=0.05)),
    ((65, 66, 67), 9, 1, "f32", "leverage", "fixed", dict(alpha=0.01)),
]


@pytest.mark.parametrize("dims,R,B,xdt,sampling,step,kw", SMALL)
def test_teacher_forced_small(cpd, orc, dims, R, B, xdt, sampling, step, kw):
    A, X, A0 = make_problem(dims, R, x_dtype=xdt, lognormal_rows=True)
    seed = 1234
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype=xdt,
                            sampling=sampling, step=step, seed=seed, engine="simt", **kw)
    ocfg = _ocfg(orc, dims, R, B, xdt, sampling, step, seed, **kw)
    worst = forced(dec, orc, ocfg, oracle_xbuf(X), 12, xdt)
    print(dims, xdt, sampling, step, worst, dec.describe())
    dec.close()


TENSOR = [
    # dims, R, B, sampling: ragged row tiles and fiber groups, R below and at 64
    ((200, 150, 100), 50, 300, "euclidean"),
    ((40, 36, 130, 28), 12, 77, "euclidean"),
    ((129, 257, 70), 64, 2048, "leverage"),
    ((300, 64, 90), 20, 1024, "uniform"),
]


@pytest.mark.parametrize("engine", ["tensor", "cluster"])
@pytest.mark.parametrize("dims,R,B,sampling", TENSOR)
def test_teacher_forced_tensor_engine(cpd, orc, dims, R, B, sampling, engine):
    A, X, A0 = make_problem(dims, R, x_dtype="bf16", lognormal_rows=True)
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype="bf16",
                            sampling=sampling, step="adagrad", seed=77, engine=engine)
    assert dec.describe()["engine"] == engine
    ocfg = _ocfg(orc, dims, R, B, "bf16", sampling, "adagrad", 77)
    worst = forced(dec, orc, ocfg, oracle_xbuf(X), 10, "bf16_tensor")
    print(dims, R, B, sampling, engine, worst, dec.describe())
    dec.close()


@pytest.mark.parametrize("engine,xdt,dims,R,B", [
    ("simt", "f32", (150, 70, 33), 10, 512),
    ("simt", "bf16", (60, 70, 55, 40), 8, 300),
    ("tensor", "bf16", (300, 200, 100), 24, 512),
    ("cluster", "bf16", (400, 250, 130), 32, 512),
])
@pytest.mark.parametrize("max_ctas", [1, 8])
def test_max_ctas_bounds_grid_and_keeps_parity(cpd, orc, engine, xdt, dims, R, B, max_ctas):
    """A CTA cap regroups the batch into fewer, larger fiber groups; the result
    still follows the oracle (same draws bit-exact, gradient within tolerance)."""
    A, X, A0 = make_problem(dims, R, x_dtype=xdt, lognormal_rows=True)
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype=xdt,
                            sampling="euclidean", step="adagrad", seed=5, engine=engine,
                            max_ctas=max_ctas)
    d = dec.describe()
    assert d["engine"] == engine
    assert d["fiber_groups"] == -(-B // d["fibers_per_cta"])
    full = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype=xdt,
                             sampling="euclidean", step="adagrad", seed=5, engine=engine)
    d0 = full.describe()
    full.close()
    # fewer, larger fiber groups than the whole-GPU tiling (the per-CTA fiber
    # limits of each engine still apply)
    assert d["fiber_groups"] < d0["fiber_groups"] and d["grad_grid"] < d0["grad_grid"]
    ocfg = _ocfg(orc, dims, R, B, xdt, "euclidean", "adagrad", 5)
    worst = forced(dec, orc, ocfg, oracle_xbuf(X), 6, "bf16_tensor" if engine != "simt" else xdt)
    print(engine, dims, max_ctas, worst, d)
    dec.close()


@pytest.mark.parametrize("engine,xdt,dims,R,B,sampling,step,kw", [
    ("simt", "f64", (50, 40, 30), 6, 40, "euclidean", "fixed", dict(alpha=0.1)),
    ("simt", "f32", (150, 70, 33), 10, 100, "euclidean", "adagrad", {}),
    ("simt", "f32", (90, 130, 40), 7, 64, "leverage", "adagrad", {}),
    ("simt", "bf16", (40, 36, 30, 28), 12, 200, "uniform", "decay", dict(beta=0.05, gamma=2.0)),
    ("tensor", "bf16", (200, 150, 100), 50, 300, "euclidean", "adagrad", {}),
    ("cluster", "bf16", (300, 64, 90), 20, 1024, "euclidean", "adagrad", {}),
])
def test_teacher_forced_nonnegative(cpd, orc, engine, xdt, dims, R, B, sampling, step, kw):
    """The nonnegative variant (projected step, Table 5 / Fig. 2) against the
    oracle; the factors stay nonnegative on a free run."""
    A, X, A0 = make_problem(dims, R, x_dtype=xdt, nonneg=True, noise=5e-2)
    kw = dict(kw, constraint="nonneg")
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype=xdt,
                            sampling=sampling, step=step, seed=99, engine=engine, **kw)
    assert dec.describe()["engine"] == engine
    ocfg = _ocfg(orc, dims, R, B, xdt, sampling, step, 99, **kw)
    worst = forced(dec, orc, ocfg, oracle_xbuf(X), 8, "bf16_tensor" if engine != "simt" else xdt)
    dec.sgd_iters(500)
    assert all(bool((a >= 0).all()) for a in dec.factors())
    fit, _ = dec.fit()
    assert np.isfinite(fit)
    print(engine, dims, worst, fit)
    dec.close()


def test_free_run_fp64_matches_oracle_c1(cpd, orc):
    """The 60^3 FP64 workload, 300 fixed-step iterations free-running on both sides."""
    w = IN.WORKLOADS["c1_60cube_f64"]
    A, X, A0 = make_problem(w["dims"], w["R"], noise=w["noise"], x_dtype="f64")
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=w["dims"], R=w["R"], B=w["B"],
                            x_dtype="f64", sampling="euclidean", step="fixed", alpha=0.1, seed=0)
    dec.sgd_iters(w["iters"])
    fit, tol_gpu = dec.fit()
    ocfg = _ocfg(orc, w["dims"], w["R"], w["B"], "f64", "euclidean", "fixed", 0)
    Ao = [a.double().numpy().copy() for a in A0]
    xb = oracle_xbuf(X)
    assert orc.run(ocfg, 0, w["iters"], None, Ao, xbuf=xb) == orc.OK
    tol_orc, _ = orc.tol(xb, Ao, "f64", dims=w["dims"])
    Ag = dec.factors()
    for a, b in zip(Ag, Ao):
        assert rel(a.numpy(), b) < 1e-9
    assert abs(tol_gpu - tol_orc) < 1e-9 * max(1.0, tol_orc)
    dec.close()


@pytest.mark.parametrize("xdt,dims,R", [("f64", (30, 20, 25), 4), ("f32", (64, 50, 40), 6),
                                        ("bf16", (48, 40, 36, 20), 5)])
def test_fit_matches_oracle(cpd, orc, xdt, dims, R):
    A, X, A0 = make_problem(dims, R, noise=0.1, x_dtype=xdt)
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=16, x_dtype=xdt,
                            sampling="euclidean", step="adagrad", seed=3, engine="simt")
    dec.sgd_iters(40)
    fit, tol = dec.fit()
    xb = oracle_xbuf(X)
    tol_o, _ = orc.tol(xb, [a.double().numpy() for a in dec.factors()], xdt, dims=dims)
    assert tol == pytest.approx(tol_o, rel=1e-9 if xdt == "f64" else 1e-5)
    assert fit == pytest.approx(1 - np.sqrt(tol_o), rel=1e-5, abs=1e-6)
    # exact factors of noiseless data: Tol is ~0
    A2, X2, _ = make_problem(dims, R, noise=0.0, x_dtype=xdt)
    dec2 = cpd.Decomposition(X2.cuda(), [a.cuda() for a in A2], dims=dims, R=R, B=16, x_dtype=xdt,
                             sampling="euclidean", step="adagrad", seed=3)
    _, tol2 = dec2.fit()
    tol2_o, _ = orc.tol(oracle_xbuf(X2), [a.double().numpy() for a in dec2.factors()], xdt, dims=dims)
    assert tol2 == pytest.approx(tol2_o, rel=1e-3, abs=1e-12)
    dec.close()
    dec2.close()


def test_chunking_and_graph_replay_are_bitwise(cpd):
    dims, R, B = (80, 70, 60), 6, 48
    _, X, A0 = make_problem(dims, R, x_dtype="f32")
    kw = dict(dims=dims, R=R, B=B, x_dtype="f32", sampling="leverage", step="adagrad", seed=9)
    d1 = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], **kw)
    d1.sgd_iters(100)                       # 3 replays of 32 iterations, one of 4
    d2 = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], **kw)
    for q in (1, 31, 32, 5, 31):            # mixed chunking
        d2.sgd_iters(q)
    assert d1.t == d2.t == 100
    for a, b in zip(d1.factors(), d2.factors()):
        assert torch.equal(a, b)
    # checkpoint at 60, resume in a fresh context, continue to 100
    d3 = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], **kw)
    d3.sgd_iters(60)
    A60, S60 = d3.factors(), d3.adagrad()
    d4 = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], **kw)
    d4.set_factors([a.cuda() for a in A60])
    d4.set_adagrad(S60)
    d4.t = 60
    d4.sgd_iters(40)
    for a, b in zip(d1.factors(), d4.factors()):
        assert torch.equal(a, b)
    for d in (d1, d2, d3, d4):
        d.close()


def test_exact_recovery_gpu(cpd):
    """Noiseless rank-R data from a perturbed start: fixed-step SGD drives Tol to ~0."""
    dims, R = (12, 14, 16), 2
    A, X, _ = make_problem(dims, R, noise=0.0, x_dtype="f64")
    g = torch.Generator().manual_seed(5)
    A0 = [a + 0.05 * torch.randn(a.shape, generator=g, dtype=torch.float64) for a in A]
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=16, x_dtype="f64",
                            sampling="euclidean", step="fixed", alpha=0.2, seed=5)
    _, tol0 = dec.fit()
    dec.sgd_iters(6000)
    _, tol1 = dec.fit()
    assert tol0 > 1e-4 and tol1 < 1e-20, (tol0, tol1)
    dec.close()


def test_degenerate_and_nonfinite_are_reported(cpd):
    dims, R = (20, 21, 22), 3
    _, X, A0 = make_problem(dims, R, x_dtype="f32")
    A0z = [a.clone() for a in A0]
    A0z[1].zero_()
    with pytest.raises(cpd.CpdError) as e:
        cpd.Decomposition(X.cuda(), [a.cuda() for a in A0z], dims=dims, R=R, B=8, x_dtype="f32",
                          sampling="euclidean", step="fixed")
    assert e.value.status == cpd.EDEGENERATE
    A0r = [a.clone() for a in A0]
    A0r[2][:, 1] = A0r[2][:, 0]
    with pytest.raises(cpd.CpdError) as e:
        cpd.Decomposition(X.cuda(), [a.cuda() for a in A0r], dims=dims, R=R, B=8, x_dtype="f32",
                          sampling="leverage", step="fixed")
    assert e.value.status == cpd.EDEGENERATE
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=8, x_dtype="f32",
                            sampling="uniform", step="fixed", alpha=1e30)
    dec.sgd_iters(3)
    with pytest.raises(cpd.CpdError) as e:
        dec.sync()
    assert e.value.status == cpd.ENONFINITE
    dec.close()


def test_profile_events(cpd):
    dims, R = (64, 64, 64), 8
    _, X, A0 = make_problem(dims, R, x_dtype="f32")
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=64, x_dtype="f32",
                            sampling="euclidean", step="adagrad")
    cpd.cpd_profile(dec.ctx, True)
    dec.sgd_iters(10)
    n, ms, ums = cpd.cpd_profile_read(dec.ctx)
    assert n == 10 and 0 < ms < 10 and 0 < ums < 10
    cpd.cpd_profile(dec.ctx, False)
    dec.close()


# --------------------------------------------------------------------------
# Full-size workloads, in the launch configuration the bench times: sampled
# teacher-forced steps (the oracle gathers only the B sampled fibers).
# --------------------------------------------------------------------------

def _full(cpd, orc, name, sampling, steps, warm, engine="auto", max_ctas=0, autotune=False):
    w = IN.WORKLOADS[name]
    dims, R, B, xdt = w["dims"], w["R"], w["B"], w["x_dtype"]
    A = IN.factors(dims, R, w["data_seed"], congruence=w["congruence"],
                   lognormal_rows=w["lognormal_rows"], device="cuda")
    X = IN.cp_tensor(A, w["noise"], w["data_seed"], xdt)
    A0 = IN.init_factors(dims, R, w["init_seed"])
    kw = dict(dims=dims, R=R, B=B, x_dtype=xdt, sampling=sampling, step=w["step"], eta=w.get("eta", 0.1),
              b=w.get("b", 1e-12), seed=w["sample_seed"], engine=engine, max_ctas=max_ctas)
    if autotune:   # the launch the bench times on this GPU
        best, _ = cpd.cpd_autotune(cpd.make_config(**kw), X, [a.cuda() for a in A0], iters=200)
        dec = cpd.Decomposition(X, [a.cuda() for a in A0], config=best)
    else:
        dec = cpd.Decomposition(X, [a.cuda() for a in A0], **kw)
    xb = oracle_xbuf(X)
    del X
    desc = dec.describe()
    dec.sgd_iters(warm)
    key = "bf16_tensor" if desc["engine"] in ("tensor", "cluster", "persistent", "fused") else xdt
    ocfg = _ocfg(orc, dims, R, B, xdt, sampling, w["step"], w["sample_seed"],
                 eta=w.get("eta", 0.1), b=w.get("b", 1e-12))
    worst = forced(dec, orc, ocfg, xb, steps, key)
    print(name, sampling, desc, worst)
    dec.close()


@pytest.mark.parametrize("sampling", ["euclidean", "leverage"])
def test_full_c2_300cube_f32(cpd, orc, sampling):
    _full(cpd, orc, "c2_300cube_f32", sampling, steps=4, warm=200)


def test_full_c3_120pow4_bf16(cpd, orc):
    _full(cpd, orc, "c3_120pow4_bf16", "euclidean", steps=4, warm=100)


@pytest.mark.parametrize("max_ctas", [0, 96])     # heuristic tiling; the autotuned one (12 groups)
def test_full_c4_1000cube_bf16(cpd, orc, max_ctas):
    _full(cpd, orc, "c4_1000cube_bf16", "euclidean", steps=3, warm=50, max_ctas=max_ctas)


def test_full_c4_autotuned_launch(cpd, orc):
    """Whatever engine and CTA cap cpd_autotune picks here (the bench's
    launch), teacher-forced against the oracle at full size."""
    _full(cpd, orc, "c4_1000cube_bf16", "euclidean", steps=2, warm=20, autotune=True)


EDGE = [
    # dims, R, B, x_dtype, sampling: the extremes cpd_init accepts
    ((3, 2, 4, 2, 3, 2, 2, 3), 2, 5, "f32", "euclidean"),     # N = 8 modes
    ((300, 40, 30), 256, 32, "f32", "euclidean"),              # R = 256
    ((1, 40, 30), 3, 16, "f32", "euclidean"),                  # a mode of size 1
    ((50, 40, 30), 4, 65536, "f32", "uniform"),                # B = 65536
    ((2, 3, 2), 1, 1, "f64", "euclidean"),                     # R = 1, B = 1
    ((150, 120, 110), 100, 64, "f32", "leverage"),             # leverage with L past shared memory (R > 64)
    ((260, 258, 257), 256, 32, "f32", "leverage"),             # leverage at R = 256: every lane slot in use
]


@pytest.mark.parametrize("dims,R,B,xdt,sampling", EDGE)
def test_teacher_forced_edge_cases(cpd, orc, dims, R, B, xdt, sampling):
    A, X, A0 = make_problem(dims, R, x_dtype=xdt, lognormal_rows=True)
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype=xdt,
                            sampling=sampling, step="adagrad", seed=21, engine="simt")
    ocfg = _ocfg(orc, dims, R, B, xdt, sampling, "adagrad", 21)
    worst = forced(dec, orc, ocfg, oracle_xbuf(X), 6, xdt)
    fit, t = dec.fit()
    otol, _ = orc.tol(oracle_xbuf(X), [a.double().numpy() for a in dec.factors()], x_dtype=xdt, dims=dims)
    assert t == pytest.approx(otol, rel=1e-9 if xdt == "f64" else 1e-4)
    print(dims, R, B, worst, dec.describe())
    dec.close()


# --------------------------------------------------------------------------
# Persistent cluster engine (engine 4): whole calls of cpd_sgd_iters in one
# launch of one thread-block cluster. max_ctas is its cluster size.
# --------------------------------------------------------------------------
PERSISTENT = [
    # dims, R, B, sampling, cluster size: ragged row tiles (200 = 128 + 72,
    # 129 = 128 + 1), a ragged last chunk of fibers, R below 16, at 64 and
    # between, one CTA without fibers (B = 77 over 8 CTAs of 16)
    ((200, 150, 100), 50, 300, "euclidean", 4),
    ((40, 36, 130, 28), 12, 77, "euclidean", 8),
    ((129, 257, 70), 64, 512, "euclidean", 2),
    ((300, 64, 90), 20, 1024, "uniform", 8),
    ((90, 70, 60), 8, 100, "euclidean", 1),
]


@pytest.mark.parametrize("dims,R,B,sampling,cs", PERSISTENT)
def test_teacher_forced_persistent(cpd, orc, dims, R, B, sampling, cs):
    A, X, A0 = make_problem(dims, R, x_dtype="bf16", lognormal_rows=True)
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype="bf16",
                            sampling=sampling, step="adagrad", seed=77, engine="persistent", max_ctas=cs)
    d = dec.describe()
    assert d["engine"] == "persistent" and d["cluster"] == cs, d
    ocfg = _ocfg(orc, dims, R, B, "bf16", sampling, "adagrad", 77)
    worst = forced(dec, orc, ocfg, oracle_xbuf(X), 8, "bf16_tensor")
    print(dims, R, B, sampling, cs, worst, d)
    dec.close()


@pytest.mark.parametrize("step,kw", [("fixed", dict(alpha=0.05)), ("decay", dict(beta=0.05, gamma=2.0))])
def test_persistent_other_steps_and_nonneg(cpd, orc, step, kw):
    dims, R, B = (150, 120, 90), 24, 256
    A, X, A0 = make_problem(dims, R, x_dtype="bf16", nonneg=True, noise=5e-2)
    kw = dict(kw, constraint="nonneg")
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype="bf16",
                            sampling="euclidean", step=step, seed=5, engine="persistent", max_ctas=4, **kw)
    ocfg = _ocfg(orc, dims, R, B, "bf16", "euclidean", step, 5, **kw)
    forced(dec, orc, ocfg, oracle_xbuf(X), 6, "bf16_tensor")
    dec.sgd_iters(300)
    assert all(bool((a >= 0).all()) for a in dec.factors())
    dec.close()


def test_persistent_chunking_is_bitwise(cpd):
    """One launch of 100 iterations and launches of 1, 31, 32, 5, 31 give the same bits."""
    dims, R, B = (120, 100, 80), 16, 256
    _, X, A0 = make_problem(dims, R, x_dtype="bf16")
    kw = dict(dims=dims, R=R, B=B, x_dtype="bf16", sampling="euclidean", step="adagrad", seed=9,
              engine="persistent", max_ctas=4)
    d1 = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], **kw)
    d1.sgd_iters(100)
    d2 = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], **kw)
    for q in (1, 31, 32, 5, 31):
        d2.sgd_iters(q)
    assert d1.t == d2.t == 100
    for a, b in zip(d1.factors(), d2.factors()):
        assert torch.equal(a, b)
    for a, b in zip(d1.adagrad(), d2.adagrad()):
        assert torch.equal(a, b)
    f1, t1 = d1.fit()
    assert np.isfinite(f1) and np.isfinite(t1)
    d1.close()
    d2.close()


@pytest.mark.parametrize("cs", [8, 16])
def test_full_c4_persistent(cpd, orc, cs):
    """The 1000^3 workload on the persistent engine, teacher-forced at full size."""
    try:   # a 16-CTA cluster is a non-portable size: only where the device can schedule it
        _full(cpd, orc, "c4_1000cube_bf16", "euclidean", steps=3, warm=50, engine="persistent", max_ctas=cs)
    except cpd.CpdError as e:
        if cs == 16 and e.status == cpd.ECUDA and "cannot be scheduled" in str(e):
            pytest.skip("this device does not co-schedule 16-CTA clusters with this layout")
        raise


def test_full_c4_fused(cpd, orc):
    """The 1000^3 workload on the fused engine (a cluster of 16 CTAs per
    128-row tile, 128 fibers each), teacher-forced at full size."""
    _full(cpd, orc, "c4_1000cube_bf16", "euclidean", steps=3, warm=50, engine="fused", max_ctas=16)


def _krp_mode1(A: list) -> np.ndarray:
    """Rows z_j of the mode-1 unfolding's Khatri-Rao product, j = i_2 + I_2 i_3 + ...
    (Eq. (2)): the second factor varies fastest."""
    Z = A[1]
    for a in A[2:]:
        Z = (a[:, None, :] * Z[None, :, :]).reshape(-1, a.shape[1])
    return Z


@pytest.mark.parametrize("dims,R", [
    ((300, 70, 50), 50),          # 2 resident chunks of A^(1) (256 + 44 rows), 28 tiles, ragged last tile
    ((600, 40, 30), 33),          # 3 chunks through the two-slot ring, K = 48
    ((1000, 60, 40), 64),         # 4 chunks, K = 64, the largest operand
    ((20, 30, 40, 5), 16),        # 4-way, one 32-column chunk for 20 rows
    ((100, 50, 40), 1),           # rank 1, K = 16
])
def test_tensor_core_fit_within_split_bound(cpd, orc, dims, R):
    """The tensor-core stop check (BF16 tensors) against the oracle's direct
    residual sum. x_hat is formed from bf16 hi/lo pairs (hi*hi + hi*lo +
    lo*hi), so each entry of x_hat is off by at most
    eps sum_r |a_ir z_jr|, eps = 2^-15 + R 2^-23 (the dropped lo*lo term, the
    two splitting errors, FP32 accumulation over K). With ||delta|| <= eps
    || |A1| |Z|^T ||_F, Cauchy-Schwarz bounds the residual sum's error by
    2 ||r|| ||delta|| + ||delta||^2."""
    _, X, A0 = make_problem(dims, R, noise=0.05, x_dtype="bf16", lognormal_rows=True)
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=64, x_dtype="bf16",
                            sampling="euclidean", step="adagrad", seed=12)
    assert dec.describe()["fit_pass"] == "tensor"
    dec.sgd_iters(30)
    _, tol = dec.fit()
    A = [a.double().numpy() for a in dec.factors()]
    xb = oracle_xbuf(X)
    tol_o, xx = orc.tol(xb, A, "bf16", dims=dims)
    eps = 2.0 ** -15 + R * 2.0 ** -23
    E = eps * np.linalg.norm(np.abs(A[0]) @ np.abs(_krp_mode1(A)).T)
    bound = (2.0 * np.sqrt(tol_o * xx) * E + E * E) / xx
    assert abs(tol - tol_o) <= bound + 1e-6 * tol_o, (tol, tol_o, bound)
    # a second pass over unchanged factors gives the same bits (fixed order)
    _, tol_again = dec.fit()
    assert tol_again == tol
    dec.close()
