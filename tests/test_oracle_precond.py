"""Pins for the C-form preconditioner (eq. 5.11-5.20) against Table 5.1."""
import os

import numpy as np
import pytest

from oracle.precond import apply_Cinv_block, dense_C, eigenbasis, kappa_C_B, one_d_forms

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table5_1_kappa.txt")


def table5_1():
    rows = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        W, k = line.split()
        rows[int(W)] = float(k)
    return rows


@pytest.mark.parametrize("W", [2, 4, 6, 8, 10])
def test_table_5_1(W):
    kappa = kappa_C_B(W)
    ref = table5_1()[W]
    # the table prints 15 significant digits; W=2 is printed as 3.69999999999999
    assert abs(kappa - ref) < 1e-9 * ref, (W, kappa, ref)


@pytest.mark.slow
@pytest.mark.parametrize("W", [12])
def test_table_5_1_large(W):
    kappa = kappa_C_B(W)
    ref = table5_1()[W]
    assert abs(kappa - ref) < 1e-9 * ref, (W, kappa, ref)


@pytest.mark.parametrize("W", [2, 5, 8])
def test_eigen_identities(W):
    E, F, *_ = one_d_forms(W)
    mu, S = eigenbasis(W)
    assert np.allclose(S.T @ F @ S, np.eye(W + 1), atol=1e-11)
    assert np.allclose(S.T @ E @ S, np.diag(mu), atol=1e-9 * mu.max())
    assert mu.min() > -1e-10 and abs(mu[0]) < 1e-9 * mu.max()  # constants: E(1) = 0


@pytest.mark.parametrize("W", [2, 3, 6])
def test_fast_diagonalisation_inverts_C(W):
    rng = np.random.default_rng(W)
    P = W + 1
    r = rng.standard_normal((P, P, P))
    z = apply_Cinv_block(r, W)
    C = dense_C(W)
    assert np.allclose(C @ z.ravel(), r.ravel(), atol=1e-10 * np.abs(r).max())
    # eq. (5.20): C has eigenvalues mu_i + mu_j + mu_k + 1 relative to F x F x F
    mu, _ = eigenbasis(W)
    E, F, *_ = one_d_forms(W)
    FFF = np.kron(F, np.kron(F, F))
    ev = np.sort(np.linalg.eigvals(np.linalg.solve(FFF, C)).real)
    sig = np.sort((mu[:, None, None] + mu[None, :, None] + mu[None, None, :] + 1).ravel())
    assert np.allclose(ev, sig, rtol=1e-8)


# ---- element-block preconditioner (block Jacobi on the blocks of A) ----------
def _tiny(n, W):
    import workloads as wl
    from oracle.functional import Discretisation
    return Discretisation(wl.varcoef_manufactured(n=n, W=W))


def test_block_on_one_element_is_the_exact_inverse():
    from oracle.precond import apply_block_inverse
    d = _tiny((1, 1, 1), 3)  # one element: A = A_ee
    x = np.random.default_rng(3).standard_normal(d.ndof)
    z = apply_block_inverse(d, d.apply_A(x))
    assert np.linalg.norm(z - x) <= 1e-9 * np.linalg.norm(x)


def test_blocks_are_the_diagonal_blocks_of_A_and_spd():
    from oracle.precond import element_block
    d = _tiny((2, 1, 1), 2)
    A = d.dense_A()
    for e in range(d.E):
        s = slice(d.off[e], d.off[e + 1])
        B = element_block(d, e)
        assert np.abs(B - A[s, s]).max() <= 1e-13 * np.abs(A).max()
        assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
        assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0


def test_block_pcg_reaches_the_cholesky_solution():
    from oracle.pcg import cholesky_solve, pcg
    from oracle.precond import apply_block_inverse, block_factors
    d = _tiny((2, 2, 1), 2)
    b = d.rhs_b()
    fac = block_factors(d)
    x, it, rel = pcg(d.apply_A, lambda r: apply_block_inverse(d, r, fac), b, tol=1e-12)
    xc = cholesky_solve(d.dense_A(), b)
    assert rel <= 1e-12
    assert np.linalg.norm(x - xc) <= 1e-8 * np.linalg.norm(xc)


# ---- C* form of edge elements (eq. 5.29-5.30) -----------------------------
def test_cstar_reduces_to_C_at_eta_one():
    from oracle.precond import dense_Cstar
    for W in (2, 5):
        assert np.abs(dense_Cstar(W, 1.0) - dense_C(W)).max() == 0.0


@pytest.mark.parametrize("eta", [1.0, 0.2, 1e-3])
def test_cstar_fast_diagonalisation_inverts_dense(eta):
    from oracle.precond import apply_Cstar_inv_block, dense_Cstar
    W = 4
    r = np.random.default_rng(2).standard_normal((W + 1,) * 3)
    z = apply_Cstar_inv_block(r, W, eta)
    back = (dense_Cstar(W, eta) @ z.ravel()).reshape(r.shape)
    assert np.abs(back - r).max() <= 1e-10 * np.abs(r).max()


def test_cstar_spectrally_equivalent_uniformly_in_eta():
    # the thesis: C* and B* are spectrally equivalent with constants independent
    # of eta (which tends to 0 towards the edge): kappa(C*^-1 B*) stays bounded
    import scipy.linalg as sla
    from oracle.precond import dense_Bstar, dense_Cstar
    for W in (2, 4):
        ks = []
        for eta in (1.0, 0.3, 0.1, 1e-2, 1e-4):
            ev = sla.eigh(dense_Bstar(W, eta), dense_Cstar(W, eta), eigvals_only=True)
            assert ev.min() > 0
            ks.append(ev.max() / ev.min())
        assert max(ks) <= ks[0] * 1.0001 and min(ks) >= 1.0, ks
