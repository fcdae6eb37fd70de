"""The seeded input recipes: deterministic, and with the shapes, ranges and
structure the measurement plan states."""
import numpy as np
import torch

from paper_2103_04081_gb300 import inputs as IN


def test_serve_requests_recipe():
    a = IN.serve_requests(512, rate=200.0, seed=0)
    b = IN.serve_requests(512, rate=200.0, seed=0)
    assert a == b                                           # deterministic
    assert a[0]["arrival"] == 0.0
    arr = np.array([q["arrival"] for q in a])
    assert (np.diff(arr) >= 0).all()
    gaps = np.diff(arr)
    assert abs(gaps.mean() - 1 / 200.0) < 0.15 / 200.0      # Poisson process at 200/s
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.15        # exponential gaps: CV ~ 1
    n3 = sum(q["N"] == 3 for q in a)
    assert 200 < n3 < 312                                   # 3- or 4-way with equal odds
    for q in a:
        assert len(q["dims"]) == q["N"] and all(50 <= d <= 400 for d in q["dims"])
        assert 5 <= q["R"] <= 32
        assert q["data_seed"] == q["init_seed"] == q["sample_seed"] == q["i"]
    assert {q["R"] for q in a} == set(range(5, 33))          # every rank occurs


def test_variance_study_factors():
    d2 = IN.variance_study_factors("data2", I=30, R=4, seed=1)
    d3 = IN.variance_study_factors("data3", I=30, R=4, seed=1)
    for a, b in zip(d2, d3):
        diff = (a != b)
        assert int(diff.sum()) <= 1                          # Data III: one entry per factor ...
        assert (b == 20.0).sum() == 1                        # ... set to 20
    assert all(a.shape == (30, 4) for a in d2)


def test_cp_tensor_matches_explicit_outer_products():
    A = IN.factors((5, 4, 3), 2, seed=3)
    X = IN.cp_tensor(A, 0.0, seed=3, x_dtype="f64").reshape(3, 4, 5).permute(2, 1, 0)
    ref = torch.einsum("ir,jr,kr->ijk", *A)
    assert torch.allclose(X, ref, rtol=0, atol=1e-12)       # column-major, first index fastest


def test_noise_level_and_nonnegative_factors():
    A = IN.factors((20, 18, 16), 3, seed=5, nonneg=True)
    assert all((a >= 0).all() for a in A)
    X0 = IN.cp_tensor(A, 0.0, seed=5, x_dtype="f64")
    X = IN.cp_tensor(A, 0.1, seed=5, x_dtype="f64")
    rel = float((X - X0).norm() / X0.norm())
    assert abs(rel - 0.1) < 1e-9                             # noise scaled to nu ||X_true||
    A0 = IN.init_factors((20, 18, 16), 3, seed=5, nonneg=True)
    assert all((a >= 0).all() for a in A0)


def test_streamed_tensor_follows_the_model():
    """cp_tensor_streamed: the CP part exactly (noise off) equals cp_tensor's,
    and with noise the residual's norm is close to noise * ||[[A]]||
    (the expected-norm scaling, within a few sqrt(2 / #entries))."""
    A = IN.factors((13, 11, 9, 7), 3, seed=5)
    a = IN.cp_tensor_streamed(A, 0.0, 5, "f32", chunk_entries=64)
    b = IN.cp_tensor(A, 0.0, 5, "f32")
    assert torch.allclose(a, b, rtol=1e-5, atol=1e-6)
    x = IN.cp_tensor_streamed(A, 0.1, 5, "f32", chunk_entries=100)
    n = x.numel()
    rel = float((x - a).norm() / a.norm())
    assert abs(rel - 0.1) < 0.1 * 5 * (2.0 / n) ** 0.5
    y = IN.cp_tensor_streamed(A, 0.1, 5, "f32", chunk_entries=100)
    assert torch.equal(x, y)                                 # seeded


def test_correlated_columns_and_lognormal_rows():
    """The factor recipe of the 300^3 and 1000^3 workloads: rows of
    A = G chol(C)^T are N(0, C) with C = (1 - c) I + c 11^T (every pair of
    columns correlated c), and lognormal row scaling multiplies each row by
    one exp(N(0, 1)) factor (the first mode, whose entries are drawn before
    its row scales, compared with the unscaled draw of the same seed)."""
    I, R, c = 40000, 4, 0.8
    A = IN.factors((I,), R, seed=9, congruence=c)[0].numpy()
    corr = np.corrcoef(A.T)
    off = corr[~np.eye(R, dtype=bool)]
    assert np.all(np.abs(off - c) < 0.01), corr
    assert np.all(np.abs(A.std(axis=0) - 1.0) < 0.02)        # unit variances: C has ones on its diagonal
    plain = IN.factors((I, 30), R, seed=11)[0].numpy()
    logn = IN.factors((I, 30), R, seed=11, lognormal_rows=True)[0].numpy()
    ratio = logn / plain
    np.testing.assert_allclose(ratio, ratio[:, :1] * np.ones((1, R)), rtol=1e-12)   # one scale per row
    z = np.log(ratio[:, 0])
    assert abs(z.mean()) < 0.03 and abs(z.std() - 1.0) < 0.03                        # exp(N(0, 1))
