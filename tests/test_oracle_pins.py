"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test compares the oracle with an independent route: numpy's Philox
bit generator, library QR / Khatri-Rao / reshapes, exhaustive enumeration of
every mini-batch on tiny tensors (Thm 5, Thm 10, Table 1), closed forms of
the updates and a hand-worked example under tests/golden/. None of them
re-types the oracle's own formula.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
from scipy.linalg import khatri_rao

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def explicit_Z(A, n):
    """Z^(n) = A^(N) kr ... kr A^(n+1) kr A^(n-1) kr ... kr A^(1) (Eq. (1))."""
    order = [k for k in reversed(range(len(A))) if k != n]
    Z = A[order[0]]
    for k in order[1:]:
        Z = khatri_rao(Z, A[k])
    return Z


def unfold(X, n):
    """Mode-n unfolding by a library reshape (Kolda & Bader ordering)."""
    return np.moveaxis(X, n, 0).reshape(X.shape[n], -1, order="F")


def rand_problem(dims, R, seed, noise=0.3):
    rng = np.random.default_rng(seed)
    A = [rng.standard_normal((d, R)) for d in dims]
    X = np.einsum(",".join(f"{chr(105 + k)}r" for k in range(len(dims))) + "->"
                  + "".join(chr(105 + k) for k in range(len(dims))), *A)
    X = np.asfortranarray(X + noise * rng.standard_normal(dims))
    return A, X


# ------------------------------------------------------------------ #
# Philox4x64-10 against numpy's implementation of the same generator   #
# ------------------------------------------------------------------ #

@pytest.mark.parametrize("ctr,key", [
    ((1, 0, 0, 0), (0, 0)),
    ((5, 7, 9, 11), (123, 456)),
    ((2**64 - 1, 3, 0, 1), (2**63 + 5, 17)),
    ((12345, 2**64 - 1, 2**32, 7), (0xDEADBEEF, 2**64 - 2)),
])
def test_philox_matches_numpy(orc, ctr, key):
    # numpy's Philox increments its 256-bit counter before each block.
    c = list(ctr)
    c[0] -= 1
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array(c, dtype=np.uint64))
    assert orc.philox(ctr, key) == [int(v) for v in bg.random_raw(4)]


def test_mode_draw_uniform(orc):
    """Alg. 4/5 draw n uniformly: chi-square over 30000 iterations."""
    for N in (3, 4, 5):
        counts = np.bincount([orc.mode_draw(11, t, N) for t in range(30000)], minlength=N)
        assert counts.size == N
        exp = 30000 / N
        chi2 = ((counts - exp) ** 2 / exp).sum()
        assert chi2 < 30.0, (N, counts)


# ------------------------------------------------------------------ #
# Eq. (2) / Eq. (3): unfolding and KRP rows                      #
# ------------------------------------------------------------------ #

@pytest.mark.parametrize("dims", [(3, 4, 5), (2, 3, 4, 5)])
def test_index_map_and_fiber_gather(orc, dims):
    X = np.asfortranarray(np.arange(math.prod(dims), dtype=np.float64).reshape(dims, order="F"))
    for n in range(len(dims)):
        Xn = unfold(X, n)
        others = [range(d) if k != n else [0] for k, d in enumerate(dims)]
        for tup in itertools.product(*others):
            j = orc.unfold_col(dims, n, tup)
            fib = orc.gather_fiber(X, n, tup)
            np.testing.assert_array_equal(fib, Xn[:, j])
            # the column holds exactly the fiber X(i_1..:..i_N)
            sl = list(tup)
            sl[n] = slice(None)
            np.testing.assert_array_equal(Xn[:, j], X[tuple(sl)])


@pytest.mark.parametrize("dims", [(3, 4, 5), (2, 3, 4, 5)])
def test_krp_row_and_cp_unfolding(orc, dims):
    R = 3
    A, _ = rand_problem(dims, R, 1, noise=0.0)
    Xexact = np.einsum(",".join(f"{chr(105 + k)}r" for k in range(len(dims))) + "->"
                       + "".join(chr(105 + k) for k in range(len(dims))), *A)
    for n in range(len(dims)):
        Z = explicit_Z(A, n)
        # Kolda & Bader: X_(n) = A^(n) Z^(n)T for an exact CP tensor.
        np.testing.assert_allclose(unfold(Xexact, n), A[n] @ Z.T, rtol=1e-12, atol=1e-12)
        others = [range(d) if k != n else [0] for k, d in enumerate(dims)]
        for tup in itertools.product(*others):
            j = orc.unfold_col(dims, n, tup)
            np.testing.assert_allclose(orc.krp_row(A, n, tup), Z[j], rtol=1e-15, atol=0)


# ------------------------------------------------------------------ #
# Sampling probabilities (Sec. 3.1)                                    #
# ------------------------------------------------------------------ #

def enumerate_batches(orc, cfg, n, X, A):
    """(p_j, G_j) for every single-fiber batch (B = 1), column j of Eq. (2)."""
    dims = cfg.dims
    others = [range(d) if k != n else [-1] for k, d in enumerate(dims)]
    out = {}
    for tup in itertools.product(*others):
        idx = np.array([tup], dtype=np.int64)
        st, p, G = orc.gradient_for_batch(cfg, n, idx, X, A)
        assert st == orc.OK
        j = orc.unfold_col(dims, n, [max(v, 0) for v in tup])
        out[j] = (p[0], G)
    return out


def test_euclidean_probabilities(orc):
    dims, R = (3, 4, 5), 2
    A, X = rand_problem(dims, R, 2)
    cfg = orc.Config(dims=dims, R=R, B=1, sampling="euclidean")
    for n in range(3):
        Z = explicit_Z(A, n)
        ps = enumerate_batches(orc, cfg, n, X, A)
        assert abs(sum(p for p, _ in ps.values()) - 1.0) < 1e-14
        others = [range(d) if k != n else [0] for k, d in enumerate(dims)]
        for tup in itertools.product(*others):
            j = orc.unfold_col(dims, n, tup)
            rows = [np.linalg.norm(A[k][tup[k]]) ** 2 for k in range(3) if k != n]
            fro = [np.linalg.norm(A[k]) ** 2 for k in range(3) if k != n]
            # Eq. (8) (up to the 2^-50 resolution of the fixed-point weights)
            assert ps[j][0] == pytest.approx(np.prod(rows) / np.prod(fro), rel=1e-12)
            # Lemma 3
            assert np.linalg.norm(Z[j]) ** 2 <= np.prod(rows) * (1 + 1e-14)


def test_leverage_scores_match_qr(orc):
    rng = np.random.default_rng(3)
    for I, R in [(7, 1), (40, 5), (100, 20), (300, 50)]:
        A = rng.standard_normal((I, R)) * np.exp(rng.standard_normal((I, 1)))
        st, w = orc.weights("leverage", A)
        assert st == orc.OK
        Q, _ = np.linalg.qr(A)
        np.testing.assert_allclose(w, (Q ** 2).sum(1), rtol=1e-9, atol=1e-13)
        assert w.sum() == pytest.approx(R, rel=1e-12)       # sum of leverage = rank


def test_leverage_rank_deficient_is_degenerate(orc):
    rng = np.random.default_rng(4)
    A = rng.standard_normal((20, 3))
    A[:, 2] = A[:, 0]
    st, _ = orc.weights("leverage", A)
    assert st == orc.EDEGENERATE


def test_leverage_probabilities_and_lemma1(orc):
    dims, R = (6, 5, 7), 3
    A, X = rand_problem(dims, R, 5)
    cfg = orc.Config(dims=dims, R=R, B=1, sampling="leverage")
    for n in range(3):
        Z = explicit_Z(A, n)
        Qz, _ = np.linalg.qr(Z)
        lev_z = (Qz ** 2).sum(1)
        lev = {k: (np.linalg.qr(A[k])[0] ** 2).sum(1) for k in range(3) if k != n}
        ps = enumerate_batches(orc, cfg, n, X, A)
        assert abs(sum(p for p, _ in ps.values()) - 1.0) < 1e-13
        others = [range(d) if k != n else [0] for k, d in enumerate(dims)]
        for tup in itertools.product(*others):
            j = orc.unfold_col(dims, n, tup)
            prod = np.prod([lev[k][tup[k]] for k in lev])
            # Eq. (7) with K = N-1 factors
            assert ps[j][0] == pytest.approx(prod / R ** 2, rel=1e-9)
            # Lemma 1
            assert lev_z[j] <= prod * (1 + 1e-9)


# ------------------------------------------------------------------ #
# Fixed-point distribution and inverse-CDF draw, against exact        #
# big-integer / rational arithmetic                                   #
# ------------------------------------------------------------------ #

def exact_distribution(w):
    """q_i = floor(w_i 2^s), s = 61 - ceil(log2 I) - floor(log2 max w), in Python integers."""
    from fractions import Fraction
    I = len(w)
    wmax = max(w)
    e = math.frexp(wmax)[1]
    s = 61 - (I - 1).bit_length() - (e - 1)
    q = [math.floor(Fraction(float(x)) * Fraction(2) ** s) for x in w]
    cdf, acc = [], 0
    for v in q:
        acc += v
        cdf.append(acc)
    return q, cdf


@pytest.mark.parametrize("I", [1, 2, 31, 32, 33, 1000, 1025, 40000])
def test_distribution_exact(orc, I):
    rng = np.random.default_rng(I)
    w = np.exp(3 * rng.standard_normal(I)) * (rng.random(I) > 0.1)
    w[rng.integers(0, I)] = 5.0
    if I > 3:
        w[:3] = [1e-300, 5e-324, 0.0]          # tiny, subnormal and zero weights
    st, c = orc.distribution(w)
    assert st == orc.OK
    q, cdf = exact_distribution(list(w))
    assert [int(v) for v in c] == cdf
    assert cdf[-1] < 2**62
    for i in range(min(I, 50)):
        assert orc.prob(c, i) == float(q[i]) / float(cdf[-1])


def test_distribution_degenerate(orc):
    assert orc.distribution(np.zeros(5))[0] == orc.EDEGENERATE
    assert orc.distribution(np.array([1.0, np.nan]))[0] == orc.EDEGENERATE
    assert orc.distribution(np.array([1.0, -2.0]))[0] == orc.EDEGENERATE
    for w in ([np.inf, 1.0, 2.0], [1.0, 2.0, np.inf], [np.nan, 1.0], [-0.5, 1.0]):   # first and last entries
        assert orc.distribution(np.array(w))[0] == orc.EDEGENERATE, w


def test_draw_matches_bigint(orc):
    import bisect
    rng = np.random.default_rng(5)
    w = np.array([0.0, 2.0, 0.0, 0.0, 1.0, 5.0, 0.0, 1e-30, 3.0])
    st, c = orc.distribution(w)
    cdf = [int(v) for v in c]
    for x in list(rng.integers(0, 2**63, 2000, dtype=np.uint64)) + [0, 2**64 - 1, 2**63]:
        x = int(x)
        target = (x * cdf[-1]) >> 64
        assert orc.draw(c, x) == bisect.bisect_right(cdf, target)
    drawn = {orc.draw(c, int(x)) for x in rng.integers(0, 2**63, 20000, dtype=np.uint64) * 2}
    assert drawn <= {1, 4, 5, 8} and {1, 4, 5} <= drawn      # zero-weight rows never drawn


def test_uniform_weights_draw_is_multiply_high(orc):
    for I in (1, 7, 1000, 12345):
        st, c = orc.distribution(np.ones(I))
        rng = np.random.default_rng(I)
        for x in rng.integers(0, 2**63, 200, dtype=np.uint64):
            x = int(x) * 2 + 1
            assert orc.draw(c, x) == (x * I) >> 64
            assert orc.prob(c, 0) == 1.0 / I


def test_euclidean_weights_exact_on_integers(orc):
    rng = np.random.default_rng(6)
    A = rng.integers(-50, 50, (40, 77)).astype(np.float64)
    st, w = orc.weights("euclidean", A)
    np.testing.assert_array_equal(w, (A.astype(np.int64) ** 2).sum(1).astype(np.float64))


def test_sampler_frequencies_chi2(orc):
    """Lemma 4: per-factor draws follow p_k(i) = ||A(i,:)||^2/||A||_F^2."""
    rng = np.random.default_rng(6)
    A = rng.standard_normal((50, 4)) * np.exp(rng.standard_normal((50, 1)))
    st, w = orc.weights("euclidean", A)
    np.testing.assert_allclose(w, (A ** 2).sum(1), rtol=1e-15)
    st, c = orc.distribution(w)
    p = (A ** 2).sum(1) / (A ** 2).sum()
    n = 100000
    draws = [orc.draw(c, orc.fiber_word(99, 3, f, 1)) for f in range(n)]
    counts = np.bincount(draws, minlength=50)
    exp = n * p
    keep = exp > 5
    chi2 = ((counts[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    dof = keep.sum() - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof), (chi2, dof)


# ------------------------------------------------------------------ #
# Thm 5 (unbiased gradient) and Thm 10 / Table 1 (variance)             #
# ------------------------------------------------------------------ #

def full_gradient(A, X, n):
    """Full LS gradient R Z with R = A Z^T - X_(n) (Sec. 2), by library ops."""
    Z = explicit_Z(A, n)
    Res = A[n] @ Z.T - unfold(X, n)
    return Res, Z, Res @ Z


CASES = [((3, 4, 5), 2, "euclidean"), ((3, 4, 5), 2, "leverage"),
         ((3, 4, 5), 2, "uniform"), ((2, 3, 2, 3), 2, "euclidean"),
         ((4, 3, 5), 1, "leverage")]


@pytest.mark.parametrize("dims,R,sampling", CASES)
def test_unbiased_gradient_thm5(orc, dims, R, sampling):
    A, X = rand_problem(dims, R, 7)
    cfg = orc.Config(dims=dims, R=R, B=1, sampling=sampling)
    for n in range(len(dims)):
        _, Z, grad = full_gradient(A, X, n)
        Jn = Z.shape[0]
        ps = enumerate_batches(orc, cfg, n, X, A)
        EG = sum(p * G for p, G in ps.values())
        # Eq. (11) taken literally: E[G] = (A Z^T Z - X_(n) Z) / J_n.
        np.testing.assert_allclose(EG, grad / Jn, rtol=1e-11, atol=1e-13 * np.abs(grad).max())


@pytest.mark.parametrize("dims,R,sampling", CASES[:3])
def test_variance_thm10_table1(orc, dims, R, sampling):
    A, X = rand_problem(dims, R, 8)
    for n in range(len(dims)):
        Res, Z, grad = full_gradient(A, X, n)
        Jn = Z.shape[0]
        cfg1 = orc.Config(dims=dims, R=R, B=1, sampling=sampling)
        ps = enumerate_batches(orc, cfg1, n, X, A)
        EG = grad / Jn
        var1 = sum(p * np.sum((G - EG) ** 2) for p, G in ps.values())
        rz = (Res ** 2).sum(0) * (Z ** 2).sum(1)         # ||R(:,j)||^2 ||Z(j,:)||^2
        pj = np.array([ps[j][0] for j in range(Jn)])
        # Thm 10, rescaled by 1/J_n^2 for the literal Eq. (11).
        thm10 = (np.sum(rz / pj) - np.sum(grad ** 2)) / Jn ** 2
        assert var1 == pytest.approx(thm10, rel=1e-10)
        # Table 1, per distribution, in closed form (B = 1).
        if sampling == "uniform":
            tab = Jn * rz.sum() - np.sum(grad ** 2)
        else:
            if sampling == "leverage":
                fac = {k: (np.linalg.qr(A[k])[0] ** 2).sum(1) for k in range(len(dims)) if k != n}
                tot = R ** (len(dims) - 1)
            else:
                fac = {k: (A[k] ** 2).sum(1) for k in range(len(dims)) if k != n}
                tot = np.prod([(A[k] ** 2).sum() for k in fac])
            den = np.empty(Jn)
            others = [range(d) if k != n else [0] for k, d in enumerate(dims)]
            for tup in itertools.product(*others):
                den[orc.unfold_col(dims, n, tup)] = np.prod([fac[k][tup[k]] for k in fac])
            tab = tot * np.sum(rz / den) - np.sum(grad ** 2)
        assert var1 == pytest.approx(tab / Jn ** 2, rel=1e-8)

        # B = 2: independent draws halve the variance (Thm 10's 1/|F_n|).
        if Jn <= 30:
            cfg2 = orc.Config(dims=dims, R=R, B=2, sampling=sampling)
            others = [range(d) if k != n else [-1] for k, d in enumerate(dims)]
            tuples = list(itertools.product(*others))
            E2 = np.zeros_like(EG)
            V2 = 0.0
            for t1 in tuples:
                for t2 in tuples:
                    st, p, G = orc.gradient_for_batch(cfg2, n, np.array([t1, t2]), X, A)
                    w = p[0] * p[1]
                    E2 += w * G
                    V2 += w * np.sum((G - EG) ** 2)
            np.testing.assert_allclose(E2, EG, rtol=1e-10, atol=1e-12 * np.abs(EG).max())
            assert V2 == pytest.approx(thm10 / 2, rel=1e-9)


def test_uniform_reduces_to_brascpd(orc):
    """p = 1/J_n turns Eq. (11) into Alg. 2's (1/B)(A Zs^T Zs - Xs Zs)."""
    dims, R, B = (4, 5, 6), 3, 7
    A, X = rand_problem(dims, R, 9)
    rng = np.random.default_rng(10)
    cfg = orc.Config(dims=dims, R=R, B=B, sampling="uniform")
    for n in range(3):
        idx = np.stack([rng.integers(0, d, B) if k != n else -np.ones(B, int)
                        for k, d in enumerate(dims)], 1)
        st, p, G = orc.gradient_for_batch(cfg, n, idx, X, A)
        Z = explicit_Z(A, n)
        Xn = unfold(X, n)
        cols = [orc.unfold_col(dims, n, np.maximum(row, 0)) for row in idx]
        Zs, Xs = Z[cols], Xn[:, cols]
        np.testing.assert_allclose(G, (A[n] @ Zs.T @ Zs - Xs @ Zs) / B, rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------------ #
# Updates, the hand-worked example and Tol                             #
# ------------------------------------------------------------------ #

def test_hand_worked_2x2x2(orc):
    g = json.load(open(os.path.join(GOLDEN, "hand_2x2x2.json")))
    dims = tuple(g["dims"])
    A = [np.array(a, dtype=np.float64) for a in g["A"]]
    X = np.full(dims, g["X_all_entries"], order="F")
    cfg = orc.Config(dims=dims, R=1, B=1, sampling="euclidean", step="fixed", alpha=0.01)
    st, p, G = orc.gradient_for_batch(cfg, g["n"], np.array(g["idx"]), X, A)
    assert p[0] == pytest.approx(g["p_f"], rel=1e-15)
    np.testing.assert_allclose(G, g["G"], rtol=1e-15)
    An = A[0].copy()
    orc.update(cfg, 0, An, None, G)
    np.testing.assert_allclose(An, g["A_fixed_alpha_0.01"], rtol=1e-15)
    cfg_ada = orc.Config(dims=dims, R=1, B=1, step="adagrad", eta=0.5, b=0.0)
    An, Sn = A[0].copy(), np.zeros_like(A[0])
    orc.update(cfg_ada, 0, An, Sn, G)
    np.testing.assert_allclose(An, g["A_adagrad_eta_0.5_b_0"], rtol=1e-15)


def test_adagrad_closed_form(orc):
    """Eq. (13a) with b=0: step 1 moves by eta*sign(G); step 2 by eta*G2/sqrt(G1^2+G2^2)."""
    rng = np.random.default_rng(12)
    A0 = rng.standard_normal((6, 3))
    G1, G2 = rng.standard_normal((6, 3)), rng.standard_normal((6, 3))
    cfg = orc.Config(dims=(6, 2, 2), R=3, B=1, step="adagrad", eta=0.3, b=0.0)
    A, S = A0.copy(), np.zeros_like(A0)
    orc.update(cfg, 0, A, S, G1)
    np.testing.assert_allclose(A, A0 - 0.3 * np.sign(G1), rtol=1e-15)
    orc.update(cfg, 1, A, S, G2)
    np.testing.assert_allclose(A, A0 - 0.3 * np.sign(G1) - 0.3 * G2 / np.sqrt(G1 ** 2 + G2 ** 2),
                               rtol=1e-14)
    np.testing.assert_allclose(S, G1 ** 2 + G2 ** 2, rtol=1e-15)


def test_decreasing_step(orc):
    rng = np.random.default_rng(13)
    A0, G = rng.standard_normal((5, 2)), rng.standard_normal((5, 2))
    cfg = orc.Config(dims=(5, 2, 2), R=2, B=1, step="decay", beta=2.0, gamma=3.0)
    A = A0.copy()
    orc.update(cfg, 7, A, None, G)
    np.testing.assert_allclose(A, A0 - (2.0 / 10.0) * G, rtol=1e-15)


def test_tol_against_planted_residual(orc):
    dims, R = (5, 6, 7), 3
    A, _ = rand_problem(dims, R, 14, noise=0.0)
    Xhat = np.einsum("ir,jr,kr->ijk", *A)
    E = np.random.default_rng(15).standard_normal(dims) * 0.1
    X = np.asfortranarray(Xhat + E)
    tol, xx = orc.tol(X, A)
    assert xx == pytest.approx(np.sum(X ** 2), rel=1e-13)
    assert tol == pytest.approx(np.sum(E ** 2) / np.sum(X ** 2), rel=1e-10)
    tol0, _ = orc.tol(np.asfortranarray(Xhat), A)
    assert tol0 < 1e-28


def test_zero_gradient_at_exact_solution(orc):
    """Interpolation: with X = [[A]] every sampled gradient vanishes (Eq. (11))."""
    dims, R = (6, 7, 8), 3
    A, _ = rand_problem(dims, R, 16, noise=0.0)
    X = np.asfortranarray(np.einsum("ir,jr,kr->ijk", *A))
    for sampling in ("euclidean", "leverage", "uniform"):
        cfg = orc.Config(dims=dims, R=R, B=5, sampling=sampling, step="fixed", alpha=0.1, seed=3)
        Ac = [a.copy() for a in A]
        for t in range(20):
            out = orc.step(cfg, t, X, Ac)
            assert out["status"] == orc.OK
            assert np.abs(out["G"]).max() < 1e-12
        for a, b in zip(Ac, A):
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)


@pytest.mark.parametrize("sampling", ["euclidean", "leverage"])
def test_exact_recovery_from_perturbed_start(orc, sampling):
    """Noiseless rank-R data, R_fit = R_true: fixed-step SGD recovers X (Tol -> 0)."""
    dims, R = (8, 9, 10), 2
    A, _ = rand_problem(dims, R, 17, noise=0.0)
    X = np.asfortranarray(np.einsum("ir,jr,kr->ijk", *A))
    rng = np.random.default_rng(18)
    A0 = [a + 0.05 * rng.standard_normal(a.shape) for a in A]
    cfg = orc.Config(dims=dims, R=R, B=16, sampling=sampling, step="fixed", alpha=0.2, seed=5)
    tol0, _ = orc.tol(X, A0)
    assert orc.run(cfg, 0, 6000, X, A0) == orc.OK
    tol1, _ = orc.tol(X, A0)
    assert tol0 > 1e-4
    assert tol1 < 1e-20, tol1


def test_step_records_batch_consistently(orc):
    """orc_step's recorded (n, idx, p, G) are those of gradient_for_batch on the same state."""
    dims, R, B = (7, 8, 9), 3, 11
    A, X = rand_problem(dims, R, 19)
    for sampling in ("euclidean", "leverage", "uniform"):
        cfg = orc.Config(dims=dims, R=R, B=B, sampling=sampling, step="adagrad", seed=21)
        Ac = [a.copy() for a in A]
        S = [np.zeros_like(a) for a in A]
        for t in range(5):
            before = [a.copy() for a in Ac]
            out = orc.step(cfg, t, X, Ac, S)
            n = out["n"]
            assert n == orc.mode_draw(21, t, 3)
            assert np.all(out["idx"][:, n] == -1)
            st, p, G = orc.gradient_for_batch(cfg, n, out["idx"], X, before)
            np.testing.assert_array_equal(p, out["p"])
            np.testing.assert_array_equal(G, out["G"])
            for k in range(3):
                if k != n:
                    np.testing.assert_array_equal(Ac[k], before[k])


# ------------------------------------------------------------------ #
# Nonnegative variant (Table 5 / Fig. 2): projected steps             #
# ------------------------------------------------------------------ #

def test_nonneg_projected_steps_reach_nnls(orc):
    """With the exact mode-n gradient (formed here from a library Khatri-Rao
    product), repeated projected fixed steps through the oracle's update
    converge to the row-wise nonnegative least-squares solution that
    scipy.optimize.nnls computes: min_{A >= 0} ||X_(n) - A Z^T||."""
    from scipy.optimize import nnls
    rng = np.random.default_rng(31)
    dims, R, n = (6, 5, 4), 3, 0
    A = [np.abs(rng.standard_normal((d, R))) for d in dims]
    X = np.asfortranarray(rng.standard_normal(dims))      # mixed signs: constraints bind
    Z = explicit_Z(A, n)
    Xn = unfold(X, n)
    Jn = Z.shape[0]
    L = np.linalg.eigvalsh(Z.T @ Z).max() / Jn            # Lipschitz constant of the gradient
    cfg = orc.Config(dims=dims, R=R, B=1, step="fixed", alpha=1.0 / L, constraint="nonneg")
    An = np.ascontiguousarray(A[n].copy())
    for t in range(4000):
        G = np.ascontiguousarray((An @ (Z.T @ Z) - Xn @ Z) / Jn)
        orc.update(cfg, t, An, None, G)
    ref = np.stack([nnls(Z, Xn[i])[0] for i in range(dims[n])])
    assert (ref == 0).any()                               # some constraints are active
    assert (An >= 0).all()
    np.testing.assert_allclose(An, ref, rtol=0, atol=1e-9)


def test_nonneg_adagrad_step_projects_each_entry(orc):
    """Projected AdaGrad step on hand-picked values: entries that the step
    drives below zero land on 0; the others move as without the constraint;
    the accumulator is the same either way."""
    cfg = orc.Config(dims=(2, 2, 2), R=2, B=1, step="adagrad", eta=0.5, b=0.0, constraint="nonneg")
    An = np.array([[1.0, 0.1], [0.2, 3.0]])
    G = np.array([[1.0, 2.0], [-4.0, 8.0]])
    S = np.zeros((2, 2))
    orc.update(cfg, 0, An, S, G)
    # S = G^2; step = 0.5 * G / |G| = 0.5 * sign(G)
    np.testing.assert_array_equal(S, G * G)
    np.testing.assert_array_equal(An, [[0.5, 0.0], [0.7, 2.5]])


def test_nonneg_recovery_keeps_factors_nonnegative(orc):
    """Noiseless nonnegative rank-R data from a nonnegative perturbed start:
    the projected run keeps every factor entry >= 0 and recovers X."""
    dims, R = (8, 9, 10), 2
    rng = np.random.default_rng(41)
    A = [np.abs(rng.standard_normal((d, R))) + 0.1 for d in dims]
    X = np.asfortranarray(np.einsum("ir,jr,kr->ijk", *A))
    A0 = [np.maximum(a + 0.05 * rng.standard_normal(a.shape), 0.0) for a in A]
    cfg = orc.Config(dims=dims, R=R, B=16, sampling="euclidean", step="fixed", alpha=0.2, seed=6,
                     constraint="nonneg")
    tol0, _ = orc.tol(X, A0)
    for chunk in range(30):
        assert orc.run(cfg, 200 * chunk, 200, X, A0) == orc.OK
        assert all((a >= 0).all() for a in A0)
    tol1, _ = orc.tol(X, A0)
    assert tol0 > 1e-4
    assert tol1 < 1e-20, tol1


# ------------------------------------------------------------------ #
# Decoding of stored tensor entries (the oracle reads BF16 / FP32 X)   #
# ------------------------------------------------------------------ #

def _bf16_ieee(bits: int) -> float:
    """Value of a bf16 bit pattern from the IEEE field definitions (1 sign, 8
    exponent bits with bias 127, 7 fraction bits)."""
    s = -1.0 if bits >> 15 else 1.0
    e, m = (bits >> 7) & 0xFF, bits & 0x7F
    if e == 0xFF:
        return s * math.inf if m == 0 else math.nan
    if e == 0:
        return s * math.ldexp(m, -133)            # subnormal: m * 2^(1 - 127 - 7)
    return s * math.ldexp(128 + m, e - 134)       # (1 + m/128) * 2^(e - 127)


def test_bf16_decode_matches_ieee_fields(orc):
    """x_at on bf16 bit patterns: printed values, both signs of zero, the
    subnormal range, the largest finite value, infinities and NaN."""
    golden = {0x3F80: 1.0, 0xC000: -2.0, 0x3F00: 0.5, 0x4049: 3.140625, 0x0001: 2.0 ** -133,
              0x8001: -(2.0 ** -133), 0x007F: 127 * 2.0 ** -133, 0x0080: 2.0 ** -126,
              0x7F7F: (2 - 2 ** -7) * 2.0 ** 127, 0x0000: 0.0, 0x8000: -0.0}
    rng = np.random.default_rng(3)
    pats = list(golden) + [0x7F80, 0xFF80, 0x7FC0, 0xFFC1] + [int(v) for v in rng.integers(0, 2**16, 4000)]
    X = np.array(pats, dtype=np.uint16).reshape(len(pats), 1, 1, order="F")
    got = orc.gather_fiber(X, 0, (0, 0, 0), "bf16")
    for b, v in zip(pats, got):
        want = golden.get(b, _bf16_ieee(b))
        if math.isnan(want):
            assert math.isnan(v), hex(b)
        else:
            assert v == want and math.copysign(1.0, v) == math.copysign(1.0, want), (hex(b), v, want)
    # every pattern decodes to exactly one value: the map is injective on non-NaN
    fin = [b for b in range(0, 2**16, 7) if not math.isnan(_bf16_ieee(b))]
    Xf = np.array(fin, dtype=np.uint16).reshape(len(fin), 1, 1, order="F")
    vals = orc.gather_fiber(Xf, 0, (0, 0, 0), "bf16")
    np.testing.assert_array_equal(vals, [_bf16_ieee(b) for b in fin])


def test_f32_decode_matches_numpy(orc):
    """x_at on FP32 entries widens exactly: against numpy's conversion, with
    subnormals, extremes and signed zero, along every mode."""
    rng = np.random.default_rng(4)
    dims = (7, 5, 6)
    X = rng.standard_normal(dims).astype(np.float32) * np.float32(3.0)
    X.flat[:6] = np.array([np.finfo(np.float32).tiny / 8, -np.finfo(np.float32).max, 0.0, -0.0,
                           np.finfo(np.float32).eps, 1e-45], dtype=np.float32)
    X = np.asfortranarray(X)
    for n in range(3):
        others = [range(d) if k != n else [0] for k, d in enumerate(dims)]
        for tup in itertools.product(*others):
            sl = list(tup)
            sl[n] = slice(None)
            got = orc.gather_fiber(X, n, tup, "f32")
            want = X[tuple(sl)].astype(np.float64)
            np.testing.assert_array_equal(got, want)
            np.testing.assert_array_equal(np.signbit(got), np.signbit(want))


@pytest.mark.parametrize("x_dtype,dims,R", [("f64", (9, 7, 8), 3), ("f32", (6, 5, 4, 3), 2),
                                            ("bf16", (11, 4, 13), 4)])
def test_tol_blas_equals_direct_sum(orc, x_dtype, dims, R):
    """The chunked, matrix-multiply form of Tol equals the entry-by-entry sum."""
    A, X = rand_problem(dims, R, 22, noise=0.4)
    if x_dtype == "bf16":
        xb = (np.asfortranarray(X).ravel(order="F").astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
    else:
        xb = np.asfortranarray(X).ravel(order="F").astype(np.float64 if x_dtype == "f64" else np.float32)
    t_direct, xx_direct = orc.tol(xb, A, x_dtype, dims=dims)
    t_blas, xx_blas = orc.tol_blas(xb, dims, A, x_dtype, chunk_cols=5)
    assert t_blas == pytest.approx(t_direct, rel=1e-12)
    assert xx_blas == pytest.approx(xx_direct, rel=1e-13)


def test_all_cores_build_gives_the_same_bits(orc):
    """The timing-only OpenMP build runs the same arithmetic in the same order."""
    dims, R, B = (23, 17, 19), 4, 64
    A, X = rand_problem(dims, R, 31, noise=0.2)
    for sampling in ("euclidean", "leverage"):
        cfg = orc.Config(dims=dims, R=R, B=B, sampling=sampling, step="adagrad", seed=8)
        A1 = [a.copy() for a in A]
        A2 = [a.copy() for a in A]
        S1 = [np.zeros_like(a) for a in A]
        S2 = [np.zeros_like(a) for a in A]
        assert orc.run(cfg, 0, 40, X, A1, S1) == orc.OK
        assert orc.run(cfg, 0, 40, X, A2, S2, omp=True) == orc.OK
        for a, b in zip(A1, A2):
            np.testing.assert_array_equal(a, b)


def test_grad_row_scale_bounds_every_row(orc):
    """|G_i| <= scale_i for every row (triangle inequality on Eq. (11)), with
    equality-order size: the scale is not vacuous."""
    dims, R, B = (9, 8, 7), 3, 25
    A, X = rand_problem(dims, R, 33, noise=0.5)
    xb = np.asfortranarray(X).ravel(order="F")
    cfg = orc.Config(dims=dims, R=R, B=B, sampling="euclidean", step="fixed", seed=2)
    out = orc.step(cfg, 0, X, [a.copy() for a in A])
    n = out["n"]
    scale = orc.grad_row_scale(dims, n, out["idx"], out["p"], A, xb, "f64", B)
    g = np.linalg.norm(out["G"], axis=1)
    assert np.all(g <= scale * (1 + 1e-12))
    assert np.all(scale <= 100 * g.max() + 1e-300) and scale.min() > 0


@pytest.mark.parametrize("zero,bs", [("X", 1), ("An", 1), ("X", 4), ("An", 4)])
def test_grad_row_scale_is_tight_on_nonnegative_data(orc, zero, bs):
    """With nonnegative factors and tensor, |A^(n)| |H| = A^(n) H and the
    second term is the size of M_i, so when one of the two products of
    Eq. (11) vanishes -- X = 0 (M = 0), or A^(n) = 0 for the mode the step
    draws (A H = 0) -- the scale of every row is |G_i| itself (to rounding):
    an inflated scale would loosen every parity test that uses it. With
    blocks of bs fibers, Eq. (11)'s 1/B counts B / bs terms."""
    dims, R, B = ((8, 8, 7), 3, 24) if bs > 1 else ((9, 8, 7), 3, 25)
    A, X = rand_problem(dims, R, 35, noise=0.0)
    A = [np.abs(a) + 0.1 for a in A]
    X = np.abs(X) + 0.2
    seed, t = 4, 0
    n = orc.mode_draw(seed, t, 3)
    if zero == "X":
        X = np.zeros(dims)
    else:
        A[n] = np.zeros_like(A[n])
    xb = np.asfortranarray(X).ravel(order="F")
    cfg = orc.Config(dims=dims, R=R, B=B, sampling="euclidean", step="fixed", seed=seed, block=bs)
    out = orc.step(cfg, t, X, [a.copy() for a in A])
    assert out["status"] == orc.OK and out["n"] == n
    scale = orc.grad_row_scale(dims, n, out["idx"], out["p"], A, xb, "f64", B, terms=B // bs)
    g = np.linalg.norm(out["G"], axis=1)
    np.testing.assert_allclose(scale, g, rtol=1e-12)


def test_grad_row_scale_ignores_signs(orc):
    """The scale is built from absolute values only: flipping the signs of
    random entries of every factor and of X (which leaves the Euclidean
    distributions, hence the batch, unchanged) leaves it bit for bit."""
    dims, R, B = (9, 8, 7), 3, 25
    A, X = rand_problem(dims, R, 37, noise=0.5)
    cfg = orc.Config(dims=dims, R=R, B=B, sampling="euclidean", step="fixed", seed=6)
    out = orc.step(cfg, 0, X, [a.copy() for a in A])
    n = out["n"]
    rng = np.random.default_rng(8)
    Af = [a * rng.choice([-1.0, 1.0], size=a.shape) for a in A]
    Xf = X * rng.choice([-1.0, 1.0], size=X.shape)
    out_f = orc.step(cfg, 0, Xf, [a.copy() for a in Af])
    np.testing.assert_array_equal(out_f["idx"], out["idx"])
    np.testing.assert_array_equal(out_f["p"], out["p"])
    s0 = orc.grad_row_scale(dims, n, out["idx"], out["p"], A, np.asfortranarray(X).ravel(order="F"), "f64", B)
    s1 = orc.grad_row_scale(dims, n, out["idx"], out["p"], Af, np.asfortranarray(Xf).ravel(order="F"), "f64", B)
    np.testing.assert_array_equal(s0, s1)


def test_sample_batch_is_the_step_batch(orc):
    """orc_sample_batch with the mode of iteration t draws exactly the batch
    orc_step records, and its Z and X rows are the KRP rows and fibers of
    that batch (Eq. (3), Eq. (2) through the explicit unfolding)."""
    dims, R, B = (7, 6, 5), 3, 9
    A, X = rand_problem(dims, R, 41, noise=0.2)
    cfg = orc.Config(dims=dims, R=R, B=B, sampling="euclidean", step="fixed", seed=4)
    for t in range(5):
        out = orc.step(cfg, t, X, [a.copy() for a in A])
        n = out["n"]
        sb = orc.sample_batch(cfg, n, t, A, X=X)
        np.testing.assert_array_equal(sb["idx"], out["idx"])
        np.testing.assert_array_equal(sb["p"], out["p"])
        Z = explicit_Z(A, n)
        Xn = unfold(X, n)
        for f in range(B):
            tup = [int(v) for v in sb["idx"][f]]
            j = orc.unfold_col(dims, n, tup)
            np.testing.assert_allclose(sb["Z"][f], Z[j], rtol=1e-15)
            np.testing.assert_array_equal(sb["X"][f], Xn[:, j])


# ------------------------------------------------------------------ #
# Remark 1: blocks of rows first, then sampling blocks                #
# ------------------------------------------------------------------ #

def _fiber_probs(orc, A, n, sampling):
    """p_j of every mode-n fiber j (Eq. (2) order), from the per-factor
    probabilities computed here by numpy from the oracle's exact CDFs."""
    N = len(A)
    per = []
    for k in range(N):
        if k == n:
            continue
        _, w = orc.weights(sampling, A[k])
        _, cdf = orc.distribution(w)
        q = np.diff(np.concatenate([[0], cdf.astype(object)])).astype(np.float64)
        per.append(q / float(cdf[-1]))
    # Eq. (2): the first other mode varies fastest
    P = per[0]
    for pk in per[1:]:
        P = np.outer(pk, P).reshape(-1)
    return P


@pytest.mark.parametrize("dims,R,bs,sampling", [((4, 6, 3), 2, 2, "euclidean"), ((4, 4, 5), 2, 4, "leverage"),
                                                 ((6, 3, 2, 3), 2, 3, "euclidean"), ((4, 6, 3), 2, 2, "uniform")])
def test_block_sampling_unbiased_and_block_probabilities(orc, dims, R, bs, sampling):
    """Every block of `bs` consecutive mode-n fibers (an aligned range of the
    first other mode's rows, other indices fixed) as the whole batch: the
    recorded probability of each of its fibers is the sum of its fibers'
    per-fiber probabilities (brute force over the explicit Eq. (10) products),
    the block probabilities sum to 1, and the expectation of Eq. (11) over all
    blocks is the full gradient / J_n (Thm 5 for blocks)."""
    A, X = rand_problem(dims, R, 29)
    N = len(dims)
    for n in range(N):
        k0 = 1 if n == 0 else 0
        others = [k for k in range(N) if k != n]
        cfg = orc.Config(dims=dims, R=R, B=bs, sampling=sampling, block=bs)
        Pj = _fiber_probs(orc, A, n, sampling)
        _, Z, grad = full_gradient(A, X, n)
        Jn = Z.shape[0]
        EG = np.zeros_like(grad)
        total = 0.0
        ranges = [range(dims[k] // bs) if k == k0 else range(dims[k]) for k in others]
        for combo in itertools.product(*ranges):
            idx = np.full((bs, N), -1, dtype=np.int64)
            for u in range(bs):
                for k, v in zip(others, combo):
                    idx[u, k] = v * bs + u if k == k0 else v
            st, p, G = orc.gradient_for_batch(cfg, n, idx, X, A)
            assert st == orc.OK
            assert np.all(p == p[0])
            # columns of the block's fibers by Eq. (2), their p_j summed
            cols = []
            for u in range(bs):
                j, Jp = 0, 1
                for k in others:
                    j += idx[u, k] * Jp
                    Jp *= dims[k]
                cols.append(j)
            assert cols == list(range(cols[0], cols[0] + bs))   # consecutive columns
            np.testing.assert_allclose(p[0], Pj[cols].sum(), rtol=1e-13)
            total += p[0]
            EG += p[0] * G
        assert abs(total - 1.0) < 1e-12
        np.testing.assert_allclose(EG, grad / Jn, rtol=1e-11, atol=1e-13 * np.abs(grad).max())


def test_block_sampling_draws_and_reduces_to_per_fiber(orc):
    """block = 1 is the per-fiber method bit for bit; with blocks, the fibers of
    each sampled block share every other index, run through one aligned block
    of rows of the first other mode, and the block's rows are drawn with the
    word of (t, block) -- so the first fiber of block beta repeats the per-fiber
    draw of slot beta, moved to its block's first row."""
    dims, R, B, bs = (8, 12, 6), 3, 24, 4
    A, X = rand_problem(dims, R, 31)
    base = orc.Config(dims=dims, R=R, B=B, sampling="euclidean", seed=5)
    one = orc.Config(dims=dims, R=R, B=B, sampling="euclidean", seed=5, block=1)
    blk = orc.Config(dims=dims, R=R, B=B, sampling="euclidean", seed=5, block=bs)
    for t in range(6):
        n = orc.mode_draw(5, t, 3)
        k0 = 1 if n == 0 else 0
        s0 = orc.sample_batch(base, n, t, A, X=X)
        s1 = orc.sample_batch(one, n, t, A, X=X)
        np.testing.assert_array_equal(s0["idx"], s1["idx"])
        np.testing.assert_array_equal(s0["p"], s1["p"])
        sb = orc.sample_batch(blk, n, t, A, X=X)
        assert sb["status"] == orc.OK
        idx = sb["idx"]
        for beta in range(B // bs):
            rows = idx[beta * bs:(beta + 1) * bs]
            for k in range(3):
                if k in (n, k0):
                    continue
                assert np.all(rows[:, k] == rows[0, k])
                assert rows[0, k] == s0["idx"][beta, k]
            assert rows[0, k0] % bs == 0
            np.testing.assert_array_equal(rows[:, k0], rows[0, k0] + np.arange(bs))
            assert rows[0, k0] == s0["idx"][beta, k0] // bs * bs
            assert np.all(sb["p"][beta * bs:(beta + 1) * bs] == sb["p"][beta * bs])


def test_block_sampling_rejects_blocks_that_do_not_tile(orc):
    A, X = rand_problem((6, 8, 5), 2, 3)
    for dims_ok, B, bs in (((6, 8, 5), 8, 4), ((6, 8, 5), 6, 2)):
        cfg = orc.Config(dims=(6, 8, 5), R=2, B=B, sampling="euclidean", block=bs)
        st = orc.sample_batch(cfg, 2, 0, A, X=X)["status"]
        assert st == (orc.EINVAL if bs == 4 else orc.OK)   # 4 does not divide I_1 = 6


# ------------------------------------------------------------------ #
# Edges: the degeneracy threshold, exact block masses, the step's own  #
# Eq. (11) with blocks, the limits of the configuration, T iterations  #
# ------------------------------------------------------------------ #

def test_leverage_degeneracy_threshold(orc):
    """Def. 3 assumes full column rank; a Cholesky pivot at or below 2^-40 of
    its Gram diagonal entry reads as rank-deficient. A = [[1, c], [0, c s]]
    with powers of two makes every Gram entry and pivot exact: g_00 = 1,
    g_01 = c, g_11 = c^2 (1 + s^2) and the last pivot d = c^2 s^2. With
    c = 2^10 and s = 2^-21 the pivot 2^-22 lies below 2^-40 g_11 (about 2^-20)
    but above 2^-40 g_01 and 2^-40 / g_11: only the threshold on the pivot's
    own diagonal entry calls it degenerate. s = 2^-19 (pivot 2^-18) is full
    rank, and a zero first column (pivot 0 against threshold 0) is not."""
    c = 2.0 ** 10
    for s, want in ((2.0 ** -21, orc.EDEGENERATE), (2.0 ** -19, orc.OK)):
        A = np.array([[1.0, c], [0.0, c * s]])
        st, w = orc.weights("leverage", A)
        assert st == want, (s, st)
        if want == orc.OK:
            np.testing.assert_allclose(w, [1.0, 1.0], rtol=1e-12)   # square A: Q is orthogonal
    A = np.array([[0.0, 1.0], [0.0, 2.0], [0.0, 3.0]])
    assert orc.weights("leverage", A)[0] == orc.EDEGENERATE
    # a pivot exactly at the threshold: four unit columns, then a column of
    # integers whose squares sum to 2^40, so g_44 = 2^40 and the last pivot is
    # 1 = 2^-40 g_44 exactly (every sum below 2^53)
    A = np.eye(5)
    A[:, 4] = [1048575.0, 1447.0, 50.0, 29.0, 1.0]
    assert orc.weights("leverage", A)[0] == orc.EDEGENERATE
    A[4, 4] = 2.0        # g_44 = 2^40 + 3, pivot 4, above its threshold 2^-40 (2^40 + 3)
    assert orc.weights("leverage", A)[0] == orc.OK


def test_block_probability_is_the_exact_block_mass(orc):
    """Remark 1 with Eq. (10): a fiber's recorded probability is its block's
    mass over the total, (cdf[(b+1) bs - 1] - cdf[b bs - 1]) / Q (cdf[-1] = 0),
    times the other modes' q_i / Q, in ascending mode order and compared bit
    for bit. The first block of each factor that can form blocks carries
    weights 1e-12 times the others, so its mass is a small integer that a
    wrong lower bound would change."""
    dims, R, bs = (8, 12, 6), 3, 4
    A, X = rand_problem(dims, R, 41)
    A[0][:bs] *= 1e-6
    A[1][:bs] *= 1e-6
    cdf = {}
    for k in range(3):
        _, w = orc.weights("euclidean", A[k])
        st, ck = orc.distribution(w)
        assert st == orc.OK
        cdf[k] = [0] + [int(v) for v in ck]          # cdf[k][i + 1] = q_0 + ... + q_i
    small = False
    for n in range(3):
        k0 = 1 if n == 0 else 0
        other = [k for k in range(3) if k not in (n, k0)][0]
        cfg = orc.Config(dims=dims, R=R, B=bs, sampling="euclidean", block=bs)
        for b in range(dims[k0] // bs):
            for v in range(dims[other]):
                idx = np.full((bs, 3), -1, dtype=np.int64)
                idx[:, k0] = b * bs + np.arange(bs)
                idx[:, other] = v
                st, p, _ = orc.gradient_for_batch(cfg, n, idx, X, A)
                assert st == orc.OK
                want = 1.0
                for k in sorted((k0, other)):
                    Q = float(cdf[k][-1])
                    if k == k0:
                        mass = cdf[k][(b + 1) * bs] - cdf[k][b * bs]
                        small |= b == 0 and mass < 2 ** 40
                    else:
                        mass = cdf[k][v + 1] - cdf[k][v]
                    want = want * (float(mass) / Q)
                assert np.all(p == want), (n, b, v, p[0], want)
    assert small


def test_block_step_is_its_batch_gradient(orc):
    """orc_step with blocks: the batch is sample_batch's, G is Eq. (11) on it
    with 1/B read as 1/(B / bs) -- equal to gradient_for_batch on the same
    batch, and, Eq. (11) being linear in its terms, to the mean of the
    gradients of its blocks taken one at a time (B = bs, the case the
    enumeration above pins)."""
    dims, R, B, bs = (8, 12, 6), 3, 12, 4
    A, X = rand_problem(dims, R, 43)
    cfg = orc.Config(dims=dims, R=R, B=B, sampling="euclidean", step="fixed", alpha=0.05, block=bs, seed=3)
    one = orc.Config(dims=dims, R=R, B=bs, sampling="euclidean", block=bs)
    for t in range(6):
        A0 = [a.copy() for a in A]
        out = orc.step(cfg, t, X, A)
        assert out["status"] == orc.OK
        n = out["n"]
        sb = orc.sample_batch(cfg, n, t, A0, X=X)
        np.testing.assert_array_equal(sb["idx"], out["idx"])
        st, p, G = orc.gradient_for_batch(cfg, n, out["idx"], X, A0)
        assert st == orc.OK
        np.testing.assert_array_equal(p, out["p"])
        np.testing.assert_array_equal(G, out["G"])
        blocks = [orc.gradient_for_batch(one, n, out["idx"][q * bs:(q + 1) * bs], X, A0)[2]
                  for q in range(B // bs)]
        np.testing.assert_allclose(out["G"], np.mean(blocks, axis=0), rtol=1e-12,
                                   atol=1e-14 * np.abs(out["G"]).max())


@pytest.mark.parametrize("dims,R,B", [((5, 4), 2, 1), ((2,) * 8, 1, 1), ((3, 4, 2), 1, 2)])
def test_configuration_limits_accepted(orc, dims, R, B):
    """N = 2 (a matrix), N = 8 (the largest order), R = 1 and B = 1 are in the
    method's domain: step and sample_batch accept them and draw the same batch,
    the step's G is Eq. (11) on it, and with B = 1 the expectation over every
    fiber is the full gradient / J_n with probabilities summing to 1 (Thm 5)."""
    A, X = rand_problem(dims, R, 47)
    N = len(dims)
    cfg = orc.Config(dims=dims, R=R, B=B, sampling="euclidean", step="fixed", alpha=0.01, seed=2)
    for t in range(3):
        A0 = [a.copy() for a in A]
        out = orc.step(cfg, t, X, A)
        assert out["status"] == orc.OK
        sb = orc.sample_batch(cfg, out["n"], t, A0, X=X)
        assert sb["status"] == orc.OK
        np.testing.assert_array_equal(sb["idx"], out["idx"])
        st, _, G = orc.gradient_for_batch(cfg, out["n"], out["idx"], X, A0)
        np.testing.assert_array_equal(G, out["G"])
    if B != 1:
        return
    for n in range(N):
        _, Z, grad = full_gradient(A, X, n)
        Jn = Z.shape[0]
        others = [k for k in range(N) if k != n]
        EG, total = np.zeros_like(grad), 0.0
        for combo in itertools.product(*[range(dims[k]) for k in others]):
            idx = np.full((1, N), -1, dtype=np.int64)
            idx[0, others] = combo
            st, p, G = orc.gradient_for_batch(cfg, n, idx, X, A)
            assert st == orc.OK
            total += p[0]
            EG += p[0] * G
        assert abs(total - 1.0) < 1e-12
        np.testing.assert_allclose(EG, grad / Jn, rtol=1e-11, atol=1e-13 * np.abs(grad).max())


def test_configuration_out_of_range_rejected(orc):
    """N outside [2, 8], R < 1, B < 1, a mode outside [0, N), a negative or
    non-tiling block and an AdaGrad step without its accumulators are
    rejected; block = 0 means per-fiber sampling, like 1."""
    from dataclasses import replace
    import ctypes
    dims = (3, 4, 2)
    A, X = rand_problem(dims, 2, 5)
    ok = orc.Config(dims=dims, R=2, B=2, step="fixed")
    assert orc.step(ok, 0, X, [a.copy() for a in A])["status"] == orc.OK
    assert orc.step(replace(ok, step="adagrad"), 0, X, [a.copy() for a in A])["status"] == orc.EINVAL  # no S
    for kw in (dict(R=0), dict(B=0), dict(block=-1), dict(block=3)):     # 3 does not divide I_2 = 4
        cfg = replace(ok, **kw)
        assert orc.step(cfg, 0, X, [a.copy() for a in A])["status"] == orc.EINVAL, kw
        assert orc.sample_batch(cfg, 0, 0, A, X=X, want_fibers=False)["status"] == orc.EINVAL, kw
    for n in (-1, 3):
        assert orc.sample_batch(ok, n, 0, A, X=X, want_fibers=False)["status"] == orc.EINVAL, n
    A1, X1 = rand_problem((5,), 2, 6)
    c1 = orc.Config(dims=(5,), R=2, B=2, step="fixed")
    assert orc.step(c1, 0, X1, [a.copy() for a in A1])["status"] == orc.EINVAL
    assert orc.sample_batch(c1, 0, 0, A1, X=X1, want_fibers=False)["status"] == orc.EINVAL
    A8, X8 = rand_problem((2,) * 8, 1, 7)
    c = orc.Config(dims=(2,) * 8, R=1, B=1, step="fixed").c()
    c.N = 9
    buf = orc.x_buffer(X8, "f64")
    idx = np.zeros((1, 9), dtype=np.int64)
    p, G = np.zeros(1), np.zeros((2, 1))
    st = orc.lib().orc_step(ctypes.byref(c), 0, orc._ptr(buf), orc._ptr_array(A8), None, None,
                            orc._ptr(idx), orc._ptr(p), orc._ptr(G))
    assert st == orc.EINVAL
    for t in range(3):
        s0 = orc.sample_batch(replace(ok, block=0), 1, t, A, X=X)
        s1 = orc.sample_batch(ok, 1, t, A, X=X)
        assert s0["status"] == s1["status"] == orc.OK
        np.testing.assert_array_equal(s0["idx"], s1["idx"])
        np.testing.assert_array_equal(s0["p"], s1["p"])


def test_run_is_T_iterations(orc):
    """orc_run(t0, T) performs the iterations t0, ..., t0 + T - 1: the same
    factors and AdaGrad state, bit for bit, as T calls of the step."""
    dims, R, B = (5, 4, 3), 2, 4
    A, X = rand_problem(dims, R, 7)
    cfg = orc.Config(dims=dims, R=R, B=B, step="adagrad", eta=0.1, seed=11)
    A1, S1 = [a.copy() for a in A], [np.zeros_like(a) for a in A]
    A2, S2 = [a.copy() for a in A], [np.zeros_like(a) for a in A]
    assert orc.run(cfg, 3, 5, X, A1, S1) == orc.OK
    for t in range(3, 8):
        assert orc.step(cfg, t, X, A2, S2)["status"] == orc.OK
    for a, b in zip(A1 + S1, A2 + S2):
        np.testing.assert_array_equal(a, b)
