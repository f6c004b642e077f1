"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test ties one oracle function to the paper's definitions or to mathematics that a
plausible mistake (a dropped term, a wrong exponent, a swapped pre-factor, a transposed
index) would violate:
  * hand-derived closed forms of d_beta and a hand-worked KL sweep (tests/golden/);
  * continuity of d_beta at beta -> 1 and beta -> 0, homogeneity d(cx|cy) = c^beta d(x|y);
  * N = 2 CP block updates equal the textbook matrix beta-NMF multiplicative updates;
  * exact fixed points (data equal to the model leave the blocks unchanged);
  * brute-force joint surrogate G(Theta | Theta~) of Appendices A/B: tightness at the
    reference, majorization elsewhere, and every block update being the block argmin;
  * monotone decrease per block (B-CoMM) and per outer iteration (J-CoMM);
  * first J-CoMM block == first B-CoMM block; KL closed-form denominator;
  * Tucker with a superdiagonal core reduces to CP; Tucker with identity factors maps the
    core to the data; Tucker N = 2 core update equals the tri-factor matrix update;
  * the COO oracle equals the dense oracle on the densified tensor; the stable permutation
    equals a brute-force stable sort.
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BETAS = [0.0, 0.5, 1.0, 1.5]


def textbook_gamma(beta):
    # Fevotte & Idier (2011) MM exponent for beta-NMF
    return 1.0 / (2.0 - beta) if beta < 1 else 1.0


# ----------------------------------------------------------------------------- d_beta

def test_dbeta_golden_closed_forms():
    rows = [l.split("#")[0].split() for l in open(os.path.join(GOLDEN, "dbeta_closed_forms.txt"))]
    rows = [r for r in rows if r]
    assert len(rows) >= 8
    for b, x, y, want in rows:
        got = oracle.dbeta(float(x), float(y), float(b))
        assert got == pytest.approx(float(want), rel=1e-13, abs=1e-14), (b, x, y)


def test_dbeta_continuity_and_homogeneity():
    g = np.random.default_rng(3)
    for _ in range(20):
        x, y = g.uniform(0.2, 5.0, size=2)
        kl = oracle.dbeta(x, y, 1.0)
        assert oracle.dbeta(x, y, 1.0 + 1e-7) == pytest.approx(kl, rel=1e-5)
        assert oracle.dbeta(x, y, 1.0 - 1e-7) == pytest.approx(kl, rel=1e-5)
        is_ = oracle.dbeta(x, y, 0.0)
        assert oracle.dbeta(x, y, 1e-7) == pytest.approx(is_, rel=1e-5)
        for b in [0.0, 0.5, 1.0, 1.5, 2.0]:
            c = 3.7
            assert oracle.dbeta(c * x, c * y, b) == pytest.approx(c ** b * oracle.dbeta(x, y, b), rel=1e-12)
            assert oracle.dbeta(x, y, b) >= 0.0
            assert abs(oracle.dbeta(x, x, b)) < 1e-14


def test_gamma_values():
    assert oracle.gamma(0.0) == 0.5
    assert oracle.gamma(0.5) == pytest.approx(2.0 / 3.0)
    assert oracle.gamma(1.0) == 1.0
    assert oracle.gamma(1.5) == 1.0


# ------------------------------------------------------------------- hand-worked sweep

def test_hand_worked_kl_sweep():
    want = {}
    for line in open(os.path.join(GOLDEN, "cp_2x2_kl_hand.txt")):
        if line.startswith("#") or line.startswith("key"):
            continue
        k, v = line.split()
        want[k] = float(v)
    X = np.array([[1.0, 2.0], [3.0, 4.0]])
    A = [np.ones((2, 1)), np.ones((2, 1))]
    new, F = oracle.cp_mu_sweep(X, A, beta=1.0)
    assert new[0][:, 0] == pytest.approx([want["A1_0"], want["A1_1"]], rel=1e-14)
    assert new[1][:, 0] == pytest.approx([want["A2_0"], want["A2_1"]], rel=1e-14)
    assert F == pytest.approx(want["F_in"], rel=1e-13)


# ------------------------------------------------------------- N = 2: textbook beta-NMF

@pytest.mark.parametrize("beta", BETAS)
def test_cp_n2_is_textbook_beta_nmf(beta):
    g = np.random.default_rng(11)
    X = g.gamma(2.0, 1.0, size=(9, 7))
    W = g.uniform(0.2, 1.0, size=(9, 3))
    H = g.uniform(0.2, 1.0, size=(7, 3))
    gm = textbook_gamma(beta)
    V = W @ H.T
    W_tb = W * (((X * V ** (beta - 2)) @ H) / ((V ** (beta - 1)) @ H)) ** gm
    V = W_tb @ H.T
    H_tb = H * (((X * V ** (beta - 2)).T @ W_tb) / ((V ** (beta - 1)).T @ W_tb)) ** gm
    new, _ = oracle.cp_mu_sweep(X, [W, H], beta)
    np.testing.assert_allclose(new[0], W_tb, rtol=1e-12)
    np.testing.assert_allclose(new[1], H_tb, rtol=1e-12)


# -------------------------------------------------------------------- fixed points

@pytest.mark.parametrize("beta", BETAS)
@pytest.mark.parametrize("dims", [(5, 4, 3), (4, 3, 3, 2)])
def test_cp_fixed_point(beta, dims):
    X, A = synth.cp_dense(dims, 3, seed=5, kind="exact")
    X = oracle.cp_full(dims, A)  # exact model in FP64
    new, _ = oracle.cp_mu_sweep(X, A, beta)
    for a, b in zip(new, A):
        np.testing.assert_allclose(a, b, rtol=1e-11)
    new, _ = oracle.cp_jcomm_outer(X, A, beta, L=2)
    for a, b in zip(new, A):
        np.testing.assert_allclose(a, b, rtol=1e-11)


@pytest.mark.parametrize("beta", BETAS)
def test_tucker_fixed_point(beta):
    dims, J = (5, 4, 3), (2, 3, 2)
    _, G, A = synth.tucker_dense(dims, J, seed=2, kind="exact")
    X = oracle.tucker_full(dims, G, A)
    G1, A1, _ = oracle.tucker_mu_sweep(X, G, A, beta)
    np.testing.assert_allclose(G1, G, rtol=1e-11)
    for a, b in zip(A1, A):
        np.testing.assert_allclose(a, b, rtol=1e-11)
    G2, A2, _ = oracle.tucker_jcomm_outer(X, G, A, beta, L=2)
    np.testing.assert_allclose(G2, G, rtol=1e-11)
    for a, b in zip(A2, A):
        np.testing.assert_allclose(a, b, rtol=1e-11)


# --------------------------------------------- brute-force joint surrogate (App. A, B)

def _d_beta_np(x, y, beta):
    if beta == 1.0:
        with np.errstate(divide="ignore", invalid="ignore"):
            xl = np.where(x > 0, x * np.log(np.where(x > 0, x, 1.0) / y), 0.0)
        return xl - x + y
    if beta == 0.0:
        return x / y - np.log(x / y) - 1.0
    return (x ** beta + (beta - 1) * y ** beta - beta * x * y ** (beta - 1)) / (beta * (beta - 1))


def _cp_contribs(A):
    """z_{i,r} = prod_n A^(n)_{i_n r} by broadcasting; shape dims + (R,)."""
    N = len(A)
    z = 1.0
    for n, a in enumerate(A):
        shape = [1] * N + [a.shape[1]]
        shape[n] = a.shape[0]
        z = z * a.reshape(shape)
    return z


def _tucker_contribs(G, A):
    """z_{i,j} = G_j prod_n A^(n)_{i_n j_n}; shape dims + core dims."""
    N = len(A)
    z = G.reshape((1,) * N + G.shape)
    for n, a in enumerate(A):
        shape = [1] * (2 * N)
        shape[n] = a.shape[0]
        shape[N + n] = a.shape[1]
        z = z * a.reshape(shape)
    return z


def _surrogate(X, z, zt, beta):
    """G(Theta | Theta~) = sum_i G_i, z / zt: contributions at Theta / Theta~ with the
    component axes trailing X's axes."""
    ax = tuple(range(X.ndim, z.ndim))
    Xt = zt.sum(axis=ax)
    lam = zt / Xt.reshape(Xt.shape + (1,) * len(ax))
    xe = X.reshape(X.shape + (1,) * len(ax))
    if beta >= 1.0:
        return float((lam * _d_beta_np(xe, z / lam, beta)).sum())
    Xh = z.sum(axis=ax)
    convex = (lam * xe / (1.0 - beta) * (z / lam) ** (beta - 1.0)).sum(axis=ax)
    if beta == 0.0:
        concave = np.log(Xt) + (Xh - Xt) / Xt
        const = -np.log(X) - 1.0
    else:
        concave = Xt ** beta / beta + Xt ** (beta - 1.0) * (Xh - Xt)
        const = X ** beta / (beta * (beta - 1.0))
    return float((convex + concave + const).sum())


def _assert_block_argmin(Gfun, block, rel=1e-12, deltas=(1e-2, 1e-3)):
    base = Gfun(block)
    flat = block.reshape(-1)
    for t in range(flat.size):
        for d in deltas:
            for s in (1 + d, 1 - d):
                pert = flat.copy()
                pert[t] *= s
                val = Gfun(pert.reshape(block.shape))
                assert val >= base - rel * abs(base), (t, d, s, val - base)


@pytest.mark.parametrize("beta", BETAS)
def test_cp_surrogate_tight_and_majorizes(beta):
    g = np.random.default_rng(21)
    dims, R = (4, 3, 5), 3
    X = g.gamma(3.0, 1.0, size=dims) + 0.05
    At = [g.uniform(0.2, 1.0, size=(d, R)) for d in dims]
    zt = _cp_contribs(At)
    F_t = oracle.cp_objective(X, At, beta)
    assert _surrogate(X, zt, zt, beta) == pytest.approx(F_t, rel=1e-12)
    for _ in range(10):
        A = [a * g.uniform(0.3, 3.0, size=a.shape) for a in At]
        assert _surrogate(X, _cp_contribs(A), zt, beta) >= oracle.cp_objective(X, A, beta) * (1 - 1e-12)


@pytest.mark.parametrize("beta", BETAS)
def test_cp_jcomm_blocks_are_surrogate_argmins(beta):
    g = np.random.default_rng(22)
    dims, R, L = (4, 3, 5), 2, 2
    X = g.gamma(3.0, 1.0, size=dims) + 0.05
    At = [g.uniform(0.2, 1.0, size=(d, R)) for d in dims]
    zt = _cp_contribs(At)
    for k in range(L * len(dims)):
        A, _ = oracle.cp_jcomm_outer(X, At, beta, L=L, max_blocks=k + 1)
        n = k % len(dims)

        def Gfun(blk, A=A, n=n):
            B = list(A)
            B[n] = blk
            return _surrogate(X, _cp_contribs(B), zt, beta)

        _assert_block_argmin(Gfun, A[n])
    # outer monotonicity (Theorem "Monotonic decrease across outer iterations")
    A = At
    F_prev = math.inf
    for _ in range(6):
        A, F = oracle.cp_jcomm_outer(X, A, beta, L=L)
        assert F <= F_prev * (1 + 1e-13)
        F_prev = F


@pytest.mark.parametrize("beta", BETAS)
def test_cp_block_updates_are_block_argmins_and_monotone(beta):
    g = np.random.default_rng(23)
    dims, R = (4, 5, 3), 3
    X = g.gamma(3.0, 1.0, size=dims) + 0.05
    A = [g.uniform(0.2, 1.0, size=(d, R)) for d in dims]
    F = oracle.cp_objective(X, A, beta)
    for sweep in range(2):
        for n in range(len(dims)):
            zt = _cp_contribs(A)
            new, _, _ = oracle.cp_block_update(X, A, n, beta)

            def Gfun(blk, A=A, n=n, zt=zt):
                B = list(A)
                B[n] = blk
                return _surrogate(X, _cp_contribs(B), zt, beta)

            _assert_block_argmin(Gfun, new[n])
            F_new = oracle.cp_objective(X, new, beta)
            assert F_new <= F * (1 + 1e-13)
            A, F = new, F_new


@pytest.mark.parametrize("beta", BETAS)
def test_tucker_jcomm_blocks_are_surrogate_argmins(beta):
    g = np.random.default_rng(24)
    dims, J, L = (4, 3, 3), (2, 2, 2), 2
    X = g.gamma(3.0, 1.0, size=dims) + 0.05
    Gt = g.uniform(0.2, 1.0, size=J)
    At = [g.uniform(0.2, 1.0, size=(d, j)) for d, j in zip(dims, J)]
    zt = _tucker_contribs(Gt, At)
    assert _surrogate(X, zt, zt, beta) == pytest.approx(oracle.tucker_objective(X, Gt, At, beta), rel=1e-12)
    nb = len(dims) + 1
    for k in range(L * nb):
        G, A, _ = oracle.tucker_jcomm_outer(X, Gt, At, beta, L=L, max_blocks=k + 1)
        b = k % nb
        if b == 0:
            def Gfun(blk, A=A):
                return _surrogate(X, _tucker_contribs(blk, A), zt, beta)
            _assert_block_argmin(Gfun, G)
        else:
            n = b - 1

            def Gfun(blk, A=A, G=G, n=n):
                B = list(A)
                B[n] = blk
                return _surrogate(X, _tucker_contribs(G, B), zt, beta)

            _assert_block_argmin(Gfun, A[n])


@pytest.mark.parametrize("beta", BETAS)
def test_tucker_block_updates_are_block_argmins_and_monotone(beta):
    g = np.random.default_rng(25)
    dims, J = (4, 3, 3), (2, 2, 2)
    X = g.gamma(3.0, 1.0, size=dims) + 0.05
    G0 = g.uniform(0.2, 1.0, size=J)
    A0 = [g.uniform(0.2, 1.0, size=(d, j)) for d, j in zip(dims, J)]
    nb = len(dims) + 1
    prevG, prevA = G0, A0
    F_prev = oracle.tucker_objective(X, G0, A0, beta)
    for k in range(nb):
        G, A, _ = oracle.tucker_mu_sweep(X, G0, A0, beta, max_blocks=k + 1)
        zt = _tucker_contribs(prevG, prevA)
        if k == 0:
            _assert_block_argmin(lambda blk: _surrogate(X, _tucker_contribs(blk, A), zt, beta), G)
        else:
            n = k - 1

            def Gfun(blk, A=A, G=G, n=n):
                B = list(A)
                B[n] = blk
                return _surrogate(X, _tucker_contribs(G, B), zt, beta)

            _assert_block_argmin(Gfun, A[n])
        F = oracle.tucker_objective(X, G, A, beta)
        assert F <= F_prev * (1 + 1e-13)
        prevG, prevA, F_prev = G, A, F


# ------------------------------------------------------------------ structural pins

@pytest.mark.parametrize("beta", BETAS)
def test_first_jcomm_block_equals_first_bcomm_block(beta):
    X, _ = synth.cp_dense((6, 5, 4), 3, seed=7, kind="gamma_noise")
    A = synth.init_factors((6, 5, 4), 3, seed=8)
    j, _ = oracle.cp_jcomm_outer(X, A, beta, L=1, max_blocks=1)
    b, _, _ = oracle.cp_block_update(X, A, 0, beta)
    np.testing.assert_allclose(j[0], b[0], rtol=1e-13)
    _, G, At = synth.tucker_dense((5, 4, 3), (2, 2, 2), seed=3)
    G0, A0 = synth.init_tucker((5, 4, 3), (2, 2, 2), seed=4)
    Xt = synth.tucker_dense((5, 4, 3), (2, 2, 2), seed=3)[0]
    Gj, _, _ = oracle.tucker_jcomm_outer(Xt, G0, A0, beta, L=1, max_blocks=1)
    Gb, _, _ = oracle.tucker_mu_sweep(Xt, G0, A0, beta, max_blocks=1)
    np.testing.assert_allclose(Gj, Gb, rtol=1e-13)


def test_kl_denominator_is_product_of_colsums():
    X, _ = synth.cp_dense((6, 5, 4), 3, seed=9)
    A = synth.init_factors((6, 5, 4), 3, seed=10)
    for n in range(3):
        _, _, den = oracle.cp_block_update(X, A, n, 1.0)
        cs = np.prod([A[m].sum(axis=0) for m in range(3) if m != n], axis=0)
        np.testing.assert_allclose(den, np.broadcast_to(cs, den.shape), rtol=1e-13)


@pytest.mark.parametrize("beta", BETAS)
def test_scaling_commutes_with_sweep(beta):
    X, _ = synth.cp_dense((6, 5, 4), 3, seed=12, kind="gamma_noise")
    A = synth.init_factors((6, 5, 4), 3, seed=13)
    c = 2.5
    ref, _ = oracle.cp_mu_sweep(X, A, beta)
    sc, _ = oracle.cp_mu_sweep(c * X, [c * A[0], A[1], A[2]], beta)
    np.testing.assert_allclose(sc[0], c * ref[0], rtol=1e-12)
    np.testing.assert_allclose(sc[1], ref[1], rtol=1e-12)
    np.testing.assert_allclose(sc[2], ref[2], rtol=1e-12)


@pytest.mark.parametrize("beta", [0.5, 1.5])
def test_mode_permutation_permutes_numden(beta):
    X, _ = synth.cp_dense((6, 5, 4), 3, seed=14, kind="gamma_noise")
    A = synth.init_factors((6, 5, 4), 3, seed=15)
    perm = (2, 0, 1)
    Xp = np.transpose(X, perm)
    Ap = [A[p] for p in perm]
    for n in range(3):
        _, num, den = oracle.cp_block_update(X, A, n, beta)
        q = perm.index(n)
        _, nump, denp = oracle.cp_block_update(Xp, Ap, q, beta)
        np.testing.assert_allclose(nump, num, rtol=1e-12)
        np.testing.assert_allclose(denp, den, rtol=1e-12)


def test_tucker_superdiagonal_core_reduces_to_cp():
    g = np.random.default_rng(31)
    dims, R = (5, 4, 3), 3
    A = [g.uniform(0.2, 1.0, size=(d, R)) for d in dims]
    gvec = g.uniform(0.5, 2.0, size=R)
    G = np.zeros((R, R, R))
    for r in range(R):
        G[r, r, r] = gvec[r]
    A_cp = [A[0] * gvec, A[1], A[2]]
    np.testing.assert_allclose(oracle.tucker_full(dims, G, A), oracle.cp_full(dims, A_cp), rtol=1e-13)
    T = g.gamma(2.0, 1.0, size=dims)
    for n in range(3):
        tk = oracle.tucker_factor_contr(T, G, A, n)
        cp = oracle.cp_contr(T, A, n) * gvec
        np.testing.assert_allclose(tk, cp, rtol=1e-13)
    core = oracle.tucker_core_contr(T, A, (R, R, R))
    c1 = oracle.cp_contr(T, A, 0)
    for r in range(R):
        assert core[r, r, r] == pytest.approx((c1[:, r] * A[0][:, r]).sum(), rel=1e-13)


@pytest.mark.parametrize("beta", BETAS)
def test_tucker_identity_factors_core_block(beta):
    g = np.random.default_rng(32)
    dims = (3, 4, 2)
    X = g.gamma(2.0, 1.0, size=dims) + 0.1
    G = g.uniform(0.5, 2.0, size=dims)
    A = [np.eye(d) for d in dims]
    G1, _, _ = oracle.tucker_mu_sweep(X, G, A, beta, max_blocks=1)
    gm = textbook_gamma(beta)
    np.testing.assert_allclose(G1, G ** (1 - gm) * X ** gm, rtol=1e-12)


@pytest.mark.parametrize("beta", BETAS)
def test_tucker_n2_core_update_is_trifactor_update(beta):
    g = np.random.default_rng(33)
    X = g.gamma(2.0, 1.0, size=(6, 5)) + 0.1
    G = g.uniform(0.3, 1.0, size=(2, 3))
    A1 = g.uniform(0.3, 1.0, size=(6, 2))
    A2 = g.uniform(0.3, 1.0, size=(5, 3))
    V = A1 @ G @ A2.T
    gm = textbook_gamma(beta)
    G_tb = G * ((A1.T @ (X * V ** (beta - 2)) @ A2) / (A1.T @ (V ** (beta - 1)) @ A2)) ** gm
    G1, _, _ = oracle.tucker_mu_sweep(X, G, [A1, A2], beta, max_blocks=1)
    np.testing.assert_allclose(G1, G_tb, rtol=1e-12)
    # and the next block (factor 1) is the matrix MU with basis G A2^T
    G2, A, _ = oracle.tucker_mu_sweep(X, G, [A1, A2], beta, max_blocks=2)
    H = (G_tb @ A2.T).T
    V = A1 @ H.T
    A1_tb = A1 * (((X * V ** (beta - 2)) @ H) / ((V ** (beta - 1)) @ H)) ** gm
    np.testing.assert_allclose(A[0], A1_tb, rtol=1e-12)


def test_tucker_partial_tensor_definition():
    g = np.random.default_rng(34)
    dims, J = (3, 4, 2), (2, 3, 2)
    G = g.uniform(0.2, 1.0, size=J)
    A = [g.uniform(0.2, 1.0, size=(d, j)) for d, j in zip(dims, J)]
    full = oracle.tucker_full(dims, G, A)
    for n in range(3):
        Bn = oracle.tucker_partial(dims, G, A, n)  # J_n x prod_{m!=n} I_m
        rest = [dims[m] for m in range(3) if m != n]
        rec = np.tensordot(A[n], Bn.reshape((J[n],) + tuple(rest)), axes=(1, 0))
        rec = np.moveaxis(rec, 0, n)
        np.testing.assert_allclose(rec, full, rtol=1e-13)


# ------------------------------------------------------------------------------ COO

def test_coo_oracle_equals_dense_oracle():
    g = np.random.default_rng(41)
    dims, R = (5, 4, 6, 3), 3
    X = np.where(g.uniform(size=dims) < 0.3, 1.0 + g.geometric(0.3, size=dims) - 1.0, 0.0)
    idx, vals = synth.coo_from_dense(X)
    A = [g.uniform(0.2, 1.0, size=(d, R)) for d in dims]
    assert oracle.coo_kl_objective(dims, idx, vals, A) == pytest.approx(oracle.cp_objective(X, A, 1.0), rel=1e-12)
    s1, F1 = oracle.coo_kl_jcomm_outer(dims, idx, vals, A, L=2)
    d1, G1 = oracle.cp_jcomm_outer(X, A, 1.0, L=2)
    assert F1 == pytest.approx(G1, rel=1e-12)
    for a, b in zip(s1, d1):
        np.testing.assert_allclose(a, b, rtol=1e-11)
    s2, F2 = oracle.coo_kl_mu_sweep(dims, idx, vals, A)
    d2, G2 = oracle.cp_mu_sweep(X, A, 1.0)
    assert F2 == pytest.approx(G2, rel=1e-12)
    for a, b in zip(s2, d2):
        np.testing.assert_allclose(a, b, rtol=1e-11)


def test_stable_perm_is_stable_sort():
    g = np.random.default_rng(42)
    keys = g.integers(0, 17, size=500).astype(np.int32)
    perm = oracle.stable_perm(keys, 17)
    brute = sorted(range(len(keys)), key=lambda e: keys[e])  # Python's sort is stable
    assert perm.tolist() == brute


def test_objective_beta0_floor():
    X = np.array([[0.0, 2.0], [1.0, 3.0]])
    A = [np.ones((2, 1)), np.ones((2, 1))]
    f = oracle.cp_objective(X, A, 0.0, eps_x=1e-3)
    want = sum(oracle.dbeta(max(x, 1e-3), 1.0, 0.0) for x in X.ravel())
    assert f == pytest.approx(want, rel=1e-14)


# ----------------------------------------- extrapolated B-CoMM (BMMe-style, Section "Going beyond")

def test_extrap_reduces_to_bcomm_without_extrapolation():
    """alpha = 0, or a previous iterate equal to the current one, is plain B-CoMM (exactly)."""
    g = np.random.default_rng(31)
    dims, R = (4, 5, 3), 3
    X = g.gamma(3.0, 1.0, size=dims) + 0.05
    A = [g.uniform(0.2, 1.0, size=(d, R)) for d in dims]
    Ap = [g.uniform(0.2, 1.0, size=(d, R)) for d in dims]
    want, Fw = oracle.cp_mu_sweep(X, A, 1.5)
    got, prev, F = oracle.cp_mu_sweep_extrap(X, A, Ap, 1.5, alpha=0.0)
    for n in range(3):
        assert np.array_equal(got[n], want[n]) and np.array_equal(prev[n], A[n])
    assert F == Fw
    got, _, _ = oracle.cp_mu_sweep_extrap(X, A, A, 1.5, alpha=0.9)
    for n in range(3):
        assert np.array_equal(got[n], want[n])


@pytest.mark.parametrize("beta", BETAS)
def test_extrap_blocks_are_surrogate_argmins_at_the_extrapolated_point(beta):
    """Each block of the extrapolated sweep minimises the block surrogate built at the
    extrapolated point (Ahat in mode n, current other blocks); alpha and the cap are
    recomputed here from their definitions."""
    g = np.random.default_rng(32)
    dims, R = (4, 3, 5), 2
    X = g.gamma(3.0, 1.0, size=dims) + 0.05
    A = [g.uniform(0.2, 1.0, size=(d, R)) for d in dims]
    Ap = [a * g.uniform(0.5, 1.2, size=a.shape) for a in A]
    alpha, cap, delta, eps = 0.6, 0.05, 1e-12, 1e-12
    got, prev, _ = oracle.cp_mu_sweep_extrap(X, A, Ap, beta, alpha=alpha, cap=cap, delta=delta)
    cur = [a.copy() for a in A]
    for n in range(3):
        D = np.maximum(A[n] - Ap[n], 0.0)
        a_n = min(alpha, cap / (np.linalg.norm(D) + delta))
        hat = np.maximum(A[n] + a_n * D, eps)
        ref = list(cur)
        ref[n] = hat
        zt = _cp_contribs(ref)

        def Gfun(blk, ref=ref, n=n, zt=zt):
            B = list(ref)
            B[n] = blk
            return _surrogate(X, _cp_contribs(B), zt, beta)

        _assert_block_argmin(Gfun, got[n])
        cur[n] = got[n]
    for n in range(3):
        assert np.array_equal(prev[n], A[n])


def test_extrap_cap_limits_the_step():
    """With a tiny cap the extrapolated point stays within cap of the current block."""
    g = np.random.default_rng(33)
    dims, R = (3, 4, 5), 2
    X = g.gamma(3.0, 1.0, size=dims) + 0.05
    A = [g.uniform(0.2, 1.0, size=(d, R)) for d in dims]
    # a non-uniform displacement (a pure rescaling of a block leaves the KL update unchanged)
    Ap = [a * g.uniform(0.3, 0.9, size=a.shape) for a in A]
    # alpha -> 0 through the cap: the sweep approaches plain B-CoMM
    got, _, _ = oracle.cp_mu_sweep_extrap(X, A, Ap, 1.0, alpha=1.0, cap=1e-14)
    want, _ = oracle.cp_mu_sweep(X, A, 1.0)
    for n in range(3):
        assert np.linalg.norm(got[n] - want[n]) / np.linalg.norm(want[n]) < 1e-10
    # a large cap leaves alpha = alpha_nes: the first block differs from plain B-CoMM
    got2, _, _ = oracle.cp_mu_sweep_extrap(X, A, Ap, 1.0, alpha=1.0, cap=1e9)
    assert np.linalg.norm(got2[0] - want[0]) / np.linalg.norm(want[0]) > 1e-3


def test_jcomm_extrap_is_jcomm_from_the_extrapolated_reference():
    """Outer-reference extrapolation = J-CoMM started from max(A + alpha_n [A - Aprev]_+, eps),
    alpha_n recomputed here from its definition; alpha = 0 is plain J-CoMM exactly."""
    g = np.random.default_rng(34)
    dims, R = (4, 5, 3), 3
    X = g.gamma(3.0, 1.0, size=dims) + 0.05
    A = [g.uniform(0.2, 1.0, size=(d, R)) for d in dims]
    Ap = [a * g.uniform(0.4, 1.2, size=a.shape) for a in A]
    for beta in (0.5, 1.0, 1.5):
        want, Fw = oracle.cp_jcomm_outer(X, A, beta, L=2)
        got, prev, F = oracle.cp_jcomm_outer_extrap(X, A, Ap, beta, alpha=0.0, L=2)
        assert all(np.array_equal(x, y) for x, y in zip(got, want)) and F == Fw
        alpha, cap = 0.8, 0.2
        ref = []
        for a, p in zip(A, Ap):
            D = np.maximum(a - p, 0.0)
            ref.append(np.maximum(a + min(alpha, cap / (np.linalg.norm(D) + 1e-12)) * D, 1e-12))
        want2, _ = oracle.cp_jcomm_outer(X, ref, beta, L=2)
        got2, prev2, F2 = oracle.cp_jcomm_outer_extrap(X, A, Ap, beta, alpha=alpha, cap=cap, L=2)
        for n in range(3):
            assert np.allclose(got2[n], want2[n], rtol=1e-13, atol=0.0)
            assert np.array_equal(prev2[n], A[n])
        assert F2 == Fw


def test_tucker_extrap_reduces_to_block_mm_and_blocks_are_argmins():
    """Extrapolated Tucker sweep: alpha = 0 is the plain sweep exactly; otherwise every block
    (core, then factors) minimises the block surrogate built at its extrapolated point."""
    g = np.random.default_rng(35)
    dims, J = (4, 3, 5), (2, 3, 2)
    X = g.gamma(3.0, 1.0, size=dims) + 0.05
    G = g.uniform(0.2, 1.0, size=J)
    A = [g.uniform(0.2, 1.0, size=(d, j)) for d, j in zip(dims, J)]
    Gp = G * g.uniform(0.5, 1.2, size=G.shape)
    Ap = [a * g.uniform(0.5, 1.2, size=a.shape) for a in A]
    Gw, Aw, Fw = oracle.tucker_mu_sweep(X, G, A, 1.5)
    G0, A0, Gp0, Ap0, F0 = oracle.tucker_mu_sweep_extrap(X, G, A, Gp, Ap, 1.5, alpha=0.0)
    assert np.array_equal(G0, Gw) and all(np.array_equal(x, y) for x, y in zip(A0, Aw)) and F0 == Fw
    assert np.array_equal(Gp0, G) and all(np.array_equal(x, y) for x, y in zip(Ap0, A))
    for beta in (0.5, 1.0, 1.5):
        alpha, cap = 0.7, 0.3
        Gn, An, _, _, _ = oracle.tucker_mu_sweep_extrap(X, G, A, Gp, Ap, beta, alpha=alpha, cap=cap)

        def hat(z, zp):
            D = np.maximum(z - zp, 0.0)
            return np.maximum(z + min(alpha, cap / (np.linalg.norm(D) + 1e-12)) * D, 1e-12)
        Gh = hat(G, Gp)
        zt = _tucker_contribs(Gh, A)
        _assert_block_argmin(lambda blk: _surrogate(X, _tucker_contribs(blk, A), zt, beta), Gn)
        cur = list(A)
        for n in range(3):
            ref = list(cur)
            ref[n] = hat(A[n], Ap[n])
            zt = _tucker_contribs(Gn, ref)

            def Gfun(blk, ref=ref, n=n, zt=zt):
                B = list(ref)
                B[n] = blk
                return _surrogate(X, _tucker_contribs(Gn, B), zt, beta)

            _assert_block_argmin(Gfun, An[n])
            cur[n] = An[n]


def test_tucker_jcomm_extrap_is_jcomm_from_the_extrapolated_reference():
    g = np.random.default_rng(36)
    dims, J = (4, 3, 5), (2, 3, 2)
    X = g.gamma(3.0, 1.0, size=dims) + 0.05
    G = g.uniform(0.2, 1.0, size=J)
    A = [g.uniform(0.2, 1.0, size=(d, j)) for d, j in zip(dims, J)]
    Gp = G * g.uniform(0.5, 1.2, size=G.shape)
    Ap = [a * g.uniform(0.5, 1.2, size=a.shape) for a in A]

    def hat(z, zp, alpha, cap):
        D = np.maximum(z - zp, 0.0)
        return np.maximum(z + min(alpha, cap / (np.linalg.norm(D) + 1e-12)) * D, 1e-12)
    for beta in (0.5, 1.0, 1.5):
        Gw, Aw, Fw = oracle.tucker_jcomm_outer(X, G, A, beta, L=2)
        G0, A0, Gp0, Ap0, F0 = oracle.tucker_jcomm_outer_extrap(X, G, A, Gp, Ap, beta, alpha=0.0, L=2)
        assert np.array_equal(G0, Gw) and all(np.array_equal(x, y) for x, y in zip(A0, Aw)) and F0 == Fw
        want_G, want_A, _ = oracle.tucker_jcomm_outer(X, hat(G, Gp, 0.7, 0.3), [hat(a, p, 0.7, 0.3) for a, p in zip(A, Ap)],
                                                      beta, L=2)
        G1, A1, Gp1, Ap1, F1 = oracle.tucker_jcomm_outer_extrap(X, G, A, Gp, Ap, beta, alpha=0.7, cap=0.3, L=2)
        assert np.allclose(G1, want_G, rtol=1e-13, atol=0.0) and F1 == Fw
        for n in range(3):
            assert np.allclose(A1[n], want_A[n], rtol=1e-13, atol=0.0)
            assert np.array_equal(Ap1[n], A[n])
        assert np.array_equal(Gp1, G)


@pytest.mark.parametrize("beta", BETAS)
def test_cp_order4_matches_brute_force_and_permutations(beta):
    """Order 4: Num/Den of every block equal brute-force sums over all entries (written here
    with einsum from the definitions of P, Q and CPContr), mode permutations permute them, and
    exact data is a fixed point of both B-CoMM and J-CoMM."""
    g = np.random.default_rng(37)
    dims, R = (3, 4, 2, 5), 2
    X = g.gamma(3.0, 1.0, size=dims) + 0.05
    A = [g.uniform(0.2, 1.0, size=(d, R)) for d in dims]
    Xh = np.einsum("ir,jr,kr,lr->ijkl", *A)
    y = np.maximum(Xh, 1e-12)
    Xs = np.maximum(X, 1e-12) if beta == 0.0 else X
    P, Q = Xs * y ** (beta - 2.0), y ** (beta - 1.0)
    subs = "ijkl"
    for n in range(4):
        others = [m for m in range(4) if m != n]
        spec = "ijkl," + ",".join(subs[m] + "r" for m in others) + "->" + subs[n] + "r"
        num_bf = np.einsum(spec, P, *[A[m] for m in others])
        den_bf = np.einsum(spec, Q, *[A[m] for m in others])
        _, num, den = oracle.cp_block_update(X, A, n, beta)
        np.testing.assert_allclose(num, num_bf, rtol=1e-12)
        np.testing.assert_allclose(den, den_bf, rtol=1e-12)
    perm = (2, 0, 3, 1)
    Xp, Ap = np.transpose(X, perm), [A[p] for p in perm]
    for n in range(4):
        _, num, den = oracle.cp_block_update(X, A, n, beta)
        _, nump, denp = oracle.cp_block_update(Xp, Ap, perm.index(n), beta)
        np.testing.assert_allclose(nump, num, rtol=1e-12)
        np.testing.assert_allclose(denp, den, rtol=1e-12)
    Xe = oracle.cp_full(dims, A)
    for fn in (lambda: oracle.cp_mu_sweep(Xe, A, beta)[0], lambda: oracle.cp_jcomm_outer(Xe, A, beta, L=2)[0]):
        for a, b in zip(fn(), A):
            np.testing.assert_allclose(a, b, rtol=1e-11)


@pytest.mark.parametrize("beta", BETAS)
def test_tucker_order4_matches_brute_force_and_fixed_points(beta):
    """Order 4 Tucker: the core and factor contractions of P and Q equal brute-force sums over
    all entries (einsum of the definitions of Xhat, P, Q and the Tucker contractions), a
    superdiagonal core gives the CP contractions, and exact data is a fixed point of the block
    sweep and of J-CoMM."""
    g = np.random.default_rng(41)
    dims, J = (4, 3, 5, 2), (2, 3, 2, 2)
    X = g.gamma(3.0, 1.0, size=dims) + 0.05
    G = g.uniform(0.3, 1.0, size=J)
    A = [g.uniform(0.2, 1.0, size=(d, j)) for d, j in zip(dims, J)]
    Xh = np.einsum("abcd,ia,jb,kc,ld->ijkl", G, *A)
    np.testing.assert_allclose(oracle.tucker_full(dims, G, A), Xh, rtol=1e-13)
    y = np.maximum(Xh, 1e-12)
    Xs = np.maximum(X, 1e-12) if beta == 0.0 else X
    P, Q = Xs * y ** (beta - 2.0), y ** (beta - 1.0)
    for T in (P, Q):
        np.testing.assert_allclose(oracle.tucker_core_contr(T, A, J),
                                   np.einsum("ijkl,ia,jb,kc,ld->abcd", T, *A), rtol=1e-12)
        subs, csubs = "ijkl", "abcd"
        for n in range(4):
            spec = ("ijkl," + csubs + "," + ",".join(subs[m] + csubs[m] for m in range(4) if m != n)
                    + "->" + subs[n] + csubs[n])
            want = np.einsum(spec, T, G, *[A[m] for m in range(4) if m != n])
            np.testing.assert_allclose(oracle.tucker_factor_contr(T, G, A, n), want, rtol=1e-12)
    R = 2
    Ac = [g.uniform(0.2, 1.0, size=(d, R)) for d in dims]
    Gd = np.zeros((R,) * 4)
    for r in range(R):
        Gd[r, r, r, r] = 1.0
    for n in range(4):
        np.testing.assert_allclose(oracle.tucker_factor_contr(P, Gd, Ac, n), oracle.cp_contr(P, Ac, n), rtol=1e-12)
    Xe = oracle.tucker_full(dims, G, A)
    for fn in (lambda: oracle.tucker_mu_sweep(Xe, G, A, beta), lambda: oracle.tucker_jcomm_outer(Xe, G, A, beta, L=2)):
        G1, A1, _ = fn()
        np.testing.assert_allclose(G1, G, rtol=1e-10)
        for a, b in zip(A1, A):
            np.testing.assert_allclose(a, b, rtol=1e-10)


@pytest.mark.parametrize("beta", [0.5, 1.0, 1.5])
def test_order5_cp_and_tucker_contractions_brute_force(beta):
    """Order 5 (the highest order the parity tests use with several merged runs): the CP and
    Tucker Num/Den of a middle and the last mode equal brute-force einsum sums of the definitions,
    and a J-CoMM outer iteration keeps exact data fixed."""
    g = np.random.default_rng(43)
    dims = (3, 2, 4, 2, 3)
    subs = "ijklm"
    X = g.gamma(3.0, 1.0, size=dims) + 0.05
    R = 2
    A = [g.uniform(0.2, 1.0, size=(d, R)) for d in dims]
    Xh = np.einsum("ir,jr,kr,lr,mr->ijklm", *A)
    P, Q = X * Xh ** (beta - 2.0), Xh ** (beta - 1.0)
    for n in (2, 4):
        others = [m for m in range(5) if m != n]
        spec = subs + "," + ",".join(subs[m] + "r" for m in others) + "->" + subs[n] + "r"
        _, num, den = oracle.cp_block_update(X, A, n, beta)
        np.testing.assert_allclose(num, np.einsum(spec, P, *[A[m] for m in others]), rtol=1e-12)
        np.testing.assert_allclose(den, np.einsum(spec, Q, *[A[m] for m in others]), rtol=1e-12)
    J = (2, 2, 2, 2, 2)
    G = g.uniform(0.3, 1.0, size=J)
    B = [g.uniform(0.2, 1.0, size=(d, j)) for d, j in zip(dims, J)]
    Th = np.einsum("abcde,ia,jb,kc,ld,me->ijklm", G, *B)
    PT = X * Th ** (beta - 2.0)
    csubs = "abcde"
    for n in (1, 3):
        spec = (subs + "," + csubs + "," + ",".join(subs[m] + csubs[m] for m in range(5) if m != n)
                + "->" + subs[n] + csubs[n])
        want = np.einsum(spec, PT, G, *[B[m] for m in range(5) if m != n])
        np.testing.assert_allclose(oracle.tucker_factor_contr(PT, G, B, n), want, rtol=1e-12)
    Xe = oracle.cp_full(dims, A)
    for a, b in zip(oracle.cp_jcomm_outer(Xe, A, beta, L=2)[0], A):
        np.testing.assert_allclose(a, b, rtol=1e-10)
    Te = oracle.tucker_full(dims, G, B)
    G1, B1, _ = oracle.tucker_jcomm_outer(Te, G, B, beta, L=2)
    np.testing.assert_allclose(G1, G, rtol=1e-10)
    for a, b in zip(B1, B):
        np.testing.assert_allclose(a, b, rtol=1e-10)


# ------------------------------------------------------- sampled Num/Den rows (large-problem checker)

def _chi1_def(z, zt, beta):
    # Section 5.3, "Two transforms": chi_1(Z, Z~) = Z~^(2 - beta) Z^(beta - 1)
    return zt ** (2.0 - beta) * z ** (beta - 1.0)


def _chi2_def(z, zt, beta):
    # Section 5.3, "Two transforms": chi_2 = Z for beta < 1, Z^beta Z~^(1 - beta) otherwise
    return z.copy() if beta < 1.0 else z ** beta * zt ** (1.0 - beta)


@pytest.mark.parametrize("beta", BETAS)
@pytest.mark.parametrize("dims", [(5, 4, 3), (3, 4, 2, 3)])
def test_numden_rows_matches_block_update_and_jcomm_definition(beta, dims):
    """ntfo_cp_numden_rows (the row-sampled checker of the full-size parity tests and of the CPU
    baseline) against two things outside it, on every row of every mode:
      * with one factor set for the reconstruction and both contractions, the Num/Den of
        ntfo_cp_block_update (Algorithm 1's block, whose contractions are pinned by brute force);
      * with three distinct factor sets -- the reference A~ for the reconstruction, chi_1(A, A~)
        for the numerator and chi_2(A, A~) for the denominator -- the J-CoMM Num_J / Den_J of
        Section 5.3 ("CP inner update"), written here as einsum sums of their definitions.
    A swapped numerator / denominator factor set, a wrong mode index or a wrong row mapping
    fails the second check, since all three factor sets differ."""
    g = np.random.default_rng(53 + len(dims))
    N, R = len(dims), 3
    X = g.gamma(3.0, 1.0, size=dims) + 0.05
    if beta == 0.0:
        X.flat[::7] = 0.0  # exercises the eps_x floor of the IS case
    A = [g.uniform(0.2, 1.0, size=(d, R)) for d in dims]
    At = [g.uniform(0.2, 1.0, size=(d, R)) for d in dims]
    subs = "ijkl"[:N]
    # block update: one factor set
    for n in range(N):
        rows = np.arange(dims[n])
        num, den = oracle.cp_numden_rows(X, A, A, A, n, rows, beta)
        _, num_b, den_b = oracle.cp_block_update(X, A, n, beta)
        np.testing.assert_allclose(num, num_b, rtol=1e-12)
        np.testing.assert_allclose(den, den_b, rtol=1e-12)
    # J-CoMM: reference reconstruction, chi_1 / chi_2 contraction factors
    B1 = [_chi1_def(a, at, beta) for a, at in zip(A, At)]
    B2 = [_chi2_def(a, at, beta) for a, at in zip(A, At)]
    Xt = np.einsum(",".join(s + "r" for s in subs) + "->" + subs, *At)
    y = np.maximum(Xt, 1e-12)
    Xs = np.maximum(X, 1e-12) if beta == 0.0 else X
    Pt, Qt = Xs * y ** (beta - 2.0), y ** (beta - 1.0)
    for n in range(N):
        others = [m for m in range(N) if m != n]
        spec = subs + "," + ",".join(subs[m] + "r" for m in others) + "->" + subs[n] + "r"
        num_j = np.einsum(spec, Pt, *[B1[m] for m in others])
        den_j = np.einsum(spec, Qt, *[B2[m] for m in others])
        rows = np.arange(dims[n])[::-1].copy()  # reversed: output q belongs to rows[q]
        num, den = oracle.cp_numden_rows(X, At, B1, B2, n, rows, beta)
        np.testing.assert_allclose(num, num_j[rows], rtol=1e-12)
        np.testing.assert_allclose(den, den_j[rows], rtol=1e-12)


# ------------------------------------------------ FP64 Tucker sweep through mode-n products

@pytest.mark.parametrize("beta", BETAS + [1.2])
@pytest.mark.parametrize("dims,J", [((7, 6, 5), (3, 2, 4)), ((5, 4, 3, 4), (2, 3, 2, 2))])
def test_tucker_modeprod_sweep_equals_entrywise_oracle(beta, dims, J):
    """The mode-n-product form of the Tucker block-MM sweep and objective (used for the
    400^3 checks, where the entry-by-entry oracle is too slow) equals the C oracle's literal
    sweep (core, then modes 1..N; Appendix C.2) and objective, block by block."""
    from oracle import tucker_modeprod as tm
    g = np.random.default_rng(61 + len(dims))
    X = g.gamma(3.0, 1.0, size=dims) + 0.05
    if beta == 0.0:
        X.flat[::5] = 0.0
    G = g.uniform(0.3, 1.0, size=J)
    A = [g.uniform(0.2, 1.0, size=(d, j)) for d, j in zip(dims, J)]
    np.testing.assert_allclose(tm.tucker_objective(X, G, A, beta), oracle.tucker_objective(X, G, A, beta), rtol=1e-12)
    Gw, Aw, Fw = oracle.tucker_mu_sweep(X, G, A, beta)
    Gm, Am, Fm = tm.tucker_mu_sweep(X, G, A, beta)
    assert abs(Fm - Fw) <= 1e-12 * abs(Fw)
    np.testing.assert_allclose(Gm, Gw, rtol=1e-11)
    for a, b in zip(Am, Aw):
        np.testing.assert_allclose(a, b, rtol=1e-11)
