"""cpd_skrp (Alg. 3 + Alg. 1 materialised) against the oracle's batch draw.

The GPU draws K batches of one mode from the context's current per-factor
distributions; the oracle draws the same batches (same Philox words, the
same exact fixed-point CDFs) from the GPU's factors. Multi-indices and p_f
must agree bit for bit, the fibers are the stored tensor values (exact), and
the sampled Khatri-Rao rows -- products of at most N-1 FP32 factor entries
on the GPU, in FP64 in the oracle -- within 1e-6 relative.
"""
import numpy as np
import pytest
import torch

from helpers import make_problem, oracle_xbuf
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


def check_batches(cpd, orc, dec, xb, x_dtype, dims, R, B, sampling, modes, K=3, t0=1000, x_offset=0):
    N = len(dims)
    A = [a.double().numpy() for a in dec.factors()]
    ocfg = orc.Config(dims=tuple(dims), R=R, B=B, sampling=sampling, step="adagrad", x_dtype=x_dtype,
                      seed=int(dec.cfg.seed))
    tdt = {"bf16": torch.bfloat16, "f32": torch.float32}[x_dtype]
    for n in modes:
        ld = (dims[n] + 7) // 8 * 8
        idx = torch.empty(K * B, N, dtype=torch.int32, device="cuda")
        p = torch.empty(K * B, dtype=torch.float64, device="cuda")
        Z = torch.empty(K * B, R, dtype=torch.float32, device="cuda")
        # x_offset elements into the allocation: the copy falls back to a
        # narrower unit when X is not 16-byte aligned
        X = torch.empty(K * B * ld + x_offset, dtype=tdt, device="cuda")[x_offset:]
        cpd.cpd_skrp(dec.ctx, n, t0, K, idx, p, Z, X)
        torch.cuda.synchronize()
        idx, p, Z = idx.cpu().numpy(), p.cpu().numpy(), Z.cpu().double().numpy()
        Xg = oracle_xbuf(X).reshape(K * B, ld)
        for b in range(K):
            o = orc.sample_batch(ocfg, n, t0 + b, A, xbuf=xb)
            sl = slice(b * B, (b + 1) * B)
            np.testing.assert_array_equal(idx[sl].astype(np.int64), o["idx"])
            np.testing.assert_array_equal(p[sl], o["p"])
            np.testing.assert_allclose(Z[sl], o["Z"], rtol=1e-6, atol=1e-30)
            got = orc.stored_values(Xg[sl].ravel(), x_dtype).reshape(B, ld)
            np.testing.assert_array_equal(got[:, :dims[n]], o["X"])
            assert not got[:, dims[n]:].any()


@pytest.mark.parametrize("dims,R,B,xdt,sampling,engine", [
    ((200, 150, 100), 12, 300, "bf16", "euclidean", "auto"),       # deferred CDF flushed first
    ((90, 80, 70), 6, 100, "f32", "leverage", "simt"),
    ((40, 36, 30, 28), 8, 77, "bf16", "uniform", "auto"),
    ((120, 100, 80), 16, 256, "bf16", "euclidean", "persistent"),
])
def test_skrp_matches_oracle(cpd, orc, dims, R, B, xdt, sampling, engine):
    _, X, A0 = make_problem(dims, R, x_dtype=xdt, lognormal_rows=True)
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype=xdt,
                            sampling=sampling, step="adagrad", seed=31, engine=engine)
    dec.sgd_iters(20)
    check_batches(cpd, orc, dec, oracle_xbuf(X), xdt, dims, R, B, sampling, range(len(dims)))
    dec.close()


@pytest.mark.parametrize("xdt,x_offset", [("bf16", 1), ("bf16", 2), ("bf16", 4), ("f32", 1), ("f32", 2)])
def test_skrp_unaligned_output(cpd, orc, xdt, x_offset):
    """X at 2, 4 or 8 bytes past a 16-byte boundary: 2-, 4- and 8-byte units."""
    dims, R, B = (50, 43, 37), 5, 70
    _, X, A0 = make_problem(dims, R, x_dtype=xdt, lognormal_rows=True)
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype=xdt,
                            sampling="euclidean", step="adagrad", seed=5)
    dec.sgd_iters(7)
    check_batches(cpd, orc, dec, oracle_xbuf(X), xdt, dims, R, B, "euclidean", range(3), K=2,
                  x_offset=x_offset)
    dec.close()


def test_skrp_long_modes_global_cdf(cpd, orc):
    """Modes whose CDFs exceed the 4096-entry shared-memory stage: mode 0's
    draws search the CDFs of modes 1 and 2 (4500 entries) in global memory."""
    dims, R, B = (20, 2500, 2000), 4, 500
    _, X, A0 = make_problem(dims, R, x_dtype="bf16", lognormal_rows=True, device="cuda")
    dec = cpd.Decomposition(X, [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype="bf16",
                            sampling="euclidean", step="adagrad", seed=9)
    xb = oracle_xbuf(X)
    del X
    dec.sgd_iters(5)
    check_batches(cpd, orc, dec, xb, "bf16", dims, R, B, "euclidean", (0, 1), K=2)
    dec.close()


def test_skrp_full_size_c4(cpd, orc):
    """The 1000^3 workload, one sampled batch per mode at full size."""
    w = IN.WORKLOADS["c4_1000cube_bf16"]
    A = IN.factors(w["dims"], w["R"], w["data_seed"], lognormal_rows=True, device="cuda")
    X = IN.cp_tensor(A, w["noise"], w["data_seed"], "bf16")
    A0 = IN.init_factors(w["dims"], w["R"], w["init_seed"])
    dec = cpd.Decomposition(X, [a.cuda() for a in A0], dims=w["dims"], R=w["R"], B=w["B"], x_dtype="bf16",
                            sampling="euclidean", step="adagrad", eta=w["eta"], seed=0)
    xb = oracle_xbuf(X)
    del X
    dec.sgd_iters(30)
    check_batches(cpd, orc, dec, xb, "bf16", w["dims"], w["R"], w["B"], "euclidean", range(3), K=1)
    dec.close()


@pytest.mark.parametrize("dims,R,B", [((200, 150, 100), 24, 256), ((64, 50, 40, 30), 16, 96)])
def test_gradients_match_oracle_per_batch(cpd, orc, dims, R, B):
    """cpd_gradients: K mini-batch gradients of mode n at the current factors
    (persistent engine, batches on concurrent clusters), each against the
    oracle's Eq. (11) for the same draws: whole-matrix and row-scaled errors
    within the tensor-core tolerances of the teacher-forced tests. The
    context's state does not move."""
    from helpers import TOL, grad_row_scale
    _, X, A0 = make_problem(dims, R, x_dtype="bf16", lognormal_rows=True)
    dec = cpd.Decomposition(X.cuda(), [a.cuda() for a in A0], dims=dims, R=R, B=B, x_dtype="bf16",
                            sampling="euclidean", step="adagrad", seed=17, engine="persistent")
    dec.sgd_iters(12)
    t_before = dec.t
    A = [a.double().numpy() for a in dec.factors()]
    xb = oracle_xbuf(X)
    ocfg = orc.Config(dims=tuple(dims), R=R, B=B, sampling="euclidean", step="adagrad", x_dtype="bf16", seed=17)
    tol = TOL["bf16_tensor"]
    K, t0 = 3, 500
    for n in range(len(dims)):
        G = torch.empty(K, dims[n], R, dtype=torch.float32, device="cuda")
        cpd.cpd_gradients(dec.ctx, n, t0, K, G)
        torch.cuda.synchronize()
        G = G.cpu().double().numpy()
        for b in range(K):
            s = orc.sample_batch(ocfg, n, t0 + b, A, xbuf=xb, want_fibers=False)
            st, p, Go = orc.gradient_for_batch(ocfg, n, s["idx"], xb, A)
            assert st == orc.OK
            np.testing.assert_array_equal(p, s["p"])
            eg = np.linalg.norm(G[b] - Go) / np.linalg.norm(Go)
            sc = grad_row_scale(dims, n, s["idx"], s["p"], A, xb, "bf16", B)
            er = float(np.max(np.linalg.norm(G[b] - Go, axis=1) / sc))
            assert eg < tol["G"] and er < tol["G_row"], (n, b, eg, er)
    assert dec.t == t_before
    assert all(np.array_equal(a, b.double().numpy()) for a, b in zip(A, dec.factors()))
    dec.close()
