"""Pins of the exact algebra the CUDA kernels are built on, computed on the CPU
from the oracle's GLL tables (no GPU, no library):

* reflection parities on the symmetric GLL grids: with R the reversal of a
  grid, R_Q B0 R_P = B0, R_Q B2 R_P = B2, R_Q B1 R_P = -B1, R D R = -D, and the
  P x P face matrices MP = B0^T W B0, KP = B0^T K B0 (Section 5.3), MP + KP,
  D^T MP D and D^T (MP + KP) D are even -- the even-odd folding of every
  contraction rests on these;
* the folded product: B u from the halves FE, FO of B and the mirrored sums
  and differences of u equals the plain product, for the forward (P -> Q) and
  the transposed (Q -> P) direction;
* the nodal face space: the discrete L^2 and H^{1/2} face norms of eq. (5.49)
  on the (2W+1)-point face grid, pulled back to the nodes, are the Kronecker
  forms MP x MP and MP x MP + MP x KP + KP x MP;
* the two-stage face phase of box meshes: the tangential derivative D, the
  Kronecker factors and the transposed derivative D^T fold into
  U = MP (c D^T (MP + KP) D v) + KP (c D^T MP D v) with the inner products
  along the derivative's axis, for both tangential axes.
"""
import numpy as np
import pytest

from oracle.functional import face_mats, half_norm_1d, h12_face_literal, l2_face_literal, tables
from oracle.gll import diff_matrix, gll, lagrange_eval

WS = list(range(1, 11))


def _rev(n):
    return np.eye(n)[::-1]


def _face_1d(W):
    """MP, KP (P x P) and D on the (W+1)-point grid."""
    t = tables(W)
    B0 = t["B"][0]
    wq = t["wq"]
    K = half_norm_1d(t["Q"])
    MP = B0.T @ np.diag(wq) @ B0
    KP = B0.T @ K @ B0
    D = diff_matrix(t["xp"])
    return MP, KP, D


@pytest.mark.parametrize("W", WS)
def test_reflection_parities(W):
    t = tables(W)
    P, Q = t["P"], t["Q"]
    RP, RQ = _rev(P), _rev(Q)
    B0, B1, B2 = t["B"]
    scale = max(1.0, np.abs(B2).max())
    assert np.abs(RQ @ B0 @ RP - B0).max() <= 1e-13
    assert np.abs(RQ @ B2 @ RP - B2).max() <= 1e-12 * scale
    assert np.abs(RQ @ B1 @ RP + B1).max() <= 1e-12 * scale
    MP, KP, D = _face_1d(W)
    assert np.abs(RP @ D @ RP + D).max() <= 1e-12 * max(1.0, np.abs(D).max())
    for X in (MP, KP, MP + KP, D.T @ MP @ D, D.T @ (MP + KP) @ D):
        assert np.abs(RP @ X @ RP - X).max() <= 1e-12 * max(1.0, np.abs(X).max())


def _halves(B):
    """FE, FO ((HQ+1) x HPE): (B[q][j] +- B[q][P-1-j]) / 2, the middle column
    (P odd) whole in FE and 0 in FO; rows q = 0 .. HQ."""
    Q, P = B.shape
    HP, HPE, HQ = P // 2, (P + 1) // 2, Q // 2
    FE = np.zeros((HQ + 1, HPE))
    FO = np.zeros((HQ + 1, HPE))
    for q in range(HQ + 1):
        for j in range(HPE):
            if P % 2 and j == HP:
                FE[q, j] = B[q, j]
            else:
                FE[q, j] = 0.5 * (B[q, j] + B[q, P - 1 - j])
                FO[q, j] = 0.5 * (B[q, j] - B[q, P - 1 - j])
    return FE, FO


def _fold_forward(B, odd, u):
    """B u by output pairs (q, Q-1-q) from the folded line (the kernel's order)."""
    Q, P = B.shape
    HP, HPE, HQ = P // 2, (P + 1) // 2, Q // 2
    FE, FO = _halves(B)
    e = np.array([u[j] + u[P - 1 - j] if j < HP else u[HP] for j in range(HPE)])
    o = np.array([u[j] - u[P - 1 - j] if j < HP else 0.0 for j in range(HPE)])
    y = np.zeros(Q)
    for q in range(HQ + 1):
        pl = (FO[q, :HP] @ o[:HP]) if odd else (FE[q] @ e)
        mi = 0.0
        if q < HQ:
            mi = (FE[q] @ e) if odd else (FO[q, :HP] @ o[:HP])
        y[q] = pl + mi
        if q < HQ:
            y[Q - 1 - q] = pl - mi
    return y


def _fold_transpose(B, odd, v):
    """B^T v by output pairs (k, P-1-k) from the folded input pairs."""
    Q, P = B.shape
    HP, HPE, HQ = P // 2, (P + 1) // 2, Q // 2
    FE, FO = _halves(B)
    ve = v[:HQ] + v[::-1][:HQ]
    vo = v[:HQ] - v[::-1][:HQ]
    vm = v[HQ]
    r = np.zeros(P)
    for k in range(HPE):
        pl = (FE[:HQ, k] @ (vo if odd else ve))
        mi = (FO[:HQ, k] @ (ve if odd else vo)) if k < HP else 0.0
        if not odd:
            pl += FE[HQ, k] * vm
        elif k < HP:
            mi += FO[HQ, k] * vm
        r[k] = pl + mi
        if k < HP:
            r[P - 1 - k] = pl - mi
    return r


@pytest.mark.parametrize("W", WS)
def test_folded_products_equal_the_plain_ones(W):
    rng = np.random.default_rng(W)
    t = tables(W)
    for m, B in enumerate(t["B"]):
        odd = m == 1
        u = rng.standard_normal(t["P"])
        v = rng.standard_normal(t["Q"])
        ref_f, ref_t = B @ u, B.T @ v
        assert np.abs(_fold_forward(B, odd, u) - ref_f).max() <= 1e-12 * max(1.0, np.abs(ref_f).max())
        assert np.abs(_fold_transpose(B, odd, v) - ref_t).max() <= 1e-12 * max(1.0, np.abs(ref_t).max())


@pytest.mark.parametrize("W", [1, 2, 3, 5])
def test_face_norms_in_the_nodal_face_space(W):
    """Same-degree faces: the face norms of the nodal trace l (P x P, [t2][t1])
    on the (2W+1)^2 grid equal l^T (MP x MP) l and l^T (MP x MP + MP x KP +
    KP x MP) l; the grid forms themselves against the literal sums."""
    rng = np.random.default_rng(100 + W)
    t = tables(W)
    P, Q = t["P"], t["Q"]
    B0 = t["B"][0]
    MP, KP, _ = _face_1d(W)
    W2, H = face_mats(Q)
    for _ in range(3):
        lnod = rng.standard_normal((P, P))
        lq = B0 @ lnod @ B0.T  # values on the Q x Q face grid, [t2][t1]
        vec = lq.ravel()
        l2 = vec @ W2 @ vec
        h12 = vec @ H @ vec
        assert abs(l2 - l2_face_literal(lq, Q)) <= 1e-12 * l2
        assert abs(h12 - h12_face_literal(lq, Q)) <= 1e-11 * h12
        n = lnod.ravel()
        assert abs(n @ np.kron(MP, MP) @ n - l2) <= 1e-12 * l2
        assert abs(n @ (np.kron(MP, MP) + np.kron(MP, KP) + np.kron(KP, MP)) @ n - h12) <= 1e-11 * h12


def _along1(X, V):
    """X applied along p1 (the second index) of V[p2][p1]."""
    return V @ X.T


def _along2(X, V):
    """X applied along p2 (the first index) of V[p2][p1]."""
    return X @ V


@pytest.mark.parametrize("W", WS)
def test_two_stage_face_phase(W):
    """Four line stages (D, the inner and outer Kronecker factors, c D^T) and
    the fused two stages give the same face outputs, for all four fields."""
    rng = np.random.default_rng(200 + W)
    MP, KP, D = _face_1d(W)
    P = MP.shape[0]
    M1 = D.T @ MP @ D
    M12 = D.T @ (MP + KP) @ D
    v = rng.standard_normal((P, P))
    c = 1.7
    # field 1: derivative along p1; inner factor along p1, outer along p2
    J1 = _along1(D, v)
    a, b = _along1(MP, J1), _along1(KP, J1)
    G1 = _along2(MP, a + b) + _along2(KP, a)
    U1 = c * _along1(D.T, G1)
    U1f = _along2(MP, c * _along1(M12, v)) + _along2(KP, c * _along1(M1, v))
    # field 2: derivative along p2; the four-stage form applies the inner factor along p1
    J2 = _along2(D, v)
    a, b = _along1(MP, J2), _along1(KP, J2)
    G2 = _along2(MP, a + b) + _along2(KP, a)
    U2 = c * _along2(D.T, G2)
    U2f = _along1(MP, c * _along2(M12, v)) + _along1(KP, c * _along2(M1, v))
    # fields 0 and 3 (no tangential derivative)
    J = rng.standard_normal((P, P))
    G0 = _along2(MP, _along1(MP, J))
    a, b = _along1(MP, J), _along1(KP, J)
    G3 = _along2(MP, a + b) + _along2(KP, a)
    G3f = _along2(MP, _along1(MP + KP, J)) + _along2(KP, _along1(MP, J))
    for ref, got in ((U1, U1f), (U2, U2f), (G3, G3f), (G0, _along2(MP, _along1(MP, J)))):
        assert np.abs(ref - got).max() <= 1e-11 * max(1.0, np.abs(ref).max())
    # and both equal the Kronecker forms of the face norms (field 1 as the
    # gradient of the H^{1/2} form: U1 = c D^T-side of H applied to D v)
    Hk = np.kron(MP, MP) + np.kron(MP, KP) + np.kron(KP, MP)
    Dx = np.kron(np.eye(P), D)  # D along p1 of the flattened [p2][p1] field
    ref = c * (Dx.T @ Hk @ Dx @ v.ravel()).reshape(P, P)
    assert np.abs(ref - U1).max() <= 1e-11 * max(1.0, np.abs(ref).max())
