"""Pins of the edge oracle's Neumann faces (the last sum of eq. 2.38 / 4.7:
|||(du/dnu^e)_{A^e} - h^e|||^2 with A^e = diag(1, 1, e^{2 tau})).

* A solution inside the discrete space with Neumann faces of all three kinds
  (tau, theta and x3 = const) makes R vanish: the conormal factors (1, 1,
  e^{2 tau}), the outward signs and the data scalings (r q_r, r q_theta,
  r^2 q_x3) agree on every face; the normal equations return it.
* Variation identity with Neumann data; A symmetric positive definite.
* The crack problem of Table 6.19 (Neumann on r = 1 and x3 = 0, 1): the H^1
  error within (1/10, 5) of the table at W = 2 (and W = 4, where it is
  0.388 % against 0.395 %), falling with W (slow-marked).
"""
import numpy as np
import pytest

import workloads as wl
from oracle.edge import EdgeDiscretisation


def _poly_neumann(N, W):
    pb = wl.edge_polynomial(N, W)
    tau1 = pb.meta["tau1"]
    bc = np.zeros((pb.mesh.n_elem, 6), dtype=np.int32)
    for e in range(pb.mesh.n_elem):
        for fi in (1, 3, 5):
            if pb.mesh.elem_nbr[e, fi] == -1:
                bc[e, fi] = 1
    pb.mesh.elem_bc = bc

    def q(rs, ts, zs):
        r, t, z = wl._cyl_grid(rs, ts, zs)
        a = np.log(r) - tau1
        return 2.0 * a * t * z / r, a * a * z / r, 2.0 * z + a * a * t

    pb.flux = [q]
    return pb


def test_edge_neumann_polynomial_reproduction():
    pb = _poly_neumann(2, 3)
    d = EdgeDiscretisation(pb)
    assert d.mesh.elem_bc.sum() >= 3
    U = d.nodal_interpolant(pb.u_exact)
    assert d.functional(U) <= 1e-22 * d.functional(np.zeros(d.ndof))
    x = np.linalg.solve(d.dense_A(), d.rhs_b())
    assert np.linalg.norm(x - U) <= 1e-8 * np.linalg.norm(U)


def test_edge_neumann_variation_identity_and_spd():
    pb = _poly_neumann(2, 2)
    d = EdgeDiscretisation(pb)
    rng = np.random.default_rng(41)
    U, V = rng.standard_normal(d.ndof), rng.standard_normal(d.ndof)
    A, b = d.dense_A(), d.rhs_b()
    assert np.abs(A - A.T).max() <= 1e-11 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0
    for eps in (0.6, -1.4):
        lhs = d.functional(U + eps * V)
        rhs = d.functional(U) + 2 * eps * V @ (A @ U - b) + eps ** 2 * V @ A @ V
        assert lhs == pytest.approx(rhs, rel=1e-10)


def _crack_error(W, N):
    import scipy.linalg as sla
    from oracle.pcg import pcg
    from oracle.precond import element_block
    d = EdgeDiscretisation(wl.edge_crack(N=N, W=W))
    fac = [sla.cho_factor(element_block(d, e)) for e in range(d.E)]
    cinv = []
    for c in range(d.C):
        n = d.Wc[c] + 1
        A = np.zeros((n, n))
        for k in range(n):
            U = np.zeros(d.ndof)
            U[d.coff[c] + k] = 1.0
            A[:, k] = d.corner_apply(U, c)
        cinv.append(np.linalg.inv(A))

    def M(r):
        z = np.zeros_like(r)
        for e in range(d.E):
            z[d.off[e]:d.off[e + 1]] = sla.cho_solve(fac[e], r[d.off[e]:d.off[e + 1]])
        for c in range(d.C):
            sl = slice(d.coff[c], d.coff[c] + d.Wc[c] + 1)
            z[sl] = cinv[c] @ r[sl]
        return z
    x, _, rel = pcg(d.apply_A, M, d.rhs_b(), tol=1e-11, maxit=5000)
    assert rel <= 1e-11
    err, nrm = d.h1_error_exact(x)
    return np.sqrt(err / nrm)


def test_crack_table_6_19_w2():
    # four theta sectors, N = W + 2 layers (the thesis's mesh is drawn, not
    # tabulated); Table 6.19: 12.1 % at W = 2, measured 5.40 %
    from golden_tables import rel_error
    ref = rel_error("table6_19_crack.txt", 2)
    err = _crack_error(2, 4)
    assert ref / 10 < err < ref * 5, err


@pytest.mark.slow
def test_crack_h1_error_falls():
    # measured 5.40 %, 1.10 %, 0.388 % at W = 2, 3, 4 (Table 6.19: 12.1 %,
    # 9.79 %, 0.395 %)
    errs = {W: _crack_error(W, W + 2) for W in (2, 3, 4)}
    assert errs[3] < 0.7 * errs[2] and errs[4] < 0.7 * errs[3], errs
    from golden_tables import rel_error
    ref = rel_error("table6_19_crack.txt", 4)
    assert ref / 10 < errs[4] < ref * 5, errs
