"""Pins of the vertex oracle's Neumann faces (the last sum of eq. 4.3:
||sqrt(R) ((du/dnu^v)_{A^v} - h^v)||_{1/2}^2, A^v = diag(1, 1/sin^2 phi, 1)).

* A solution inside the discrete space with Neumann faces phi, theta and
  rho = const makes R vanish: the conormal factors (1, 1/sin^2 phi, 1), the
  outward signs and the data scalings (rho q_phi, rho q_theta / sin phi,
  rho q_rho) agree on every kind of face; the normal equations return it.
* Variation identity with Neumann data; A symmetric positive definite.
* Table 6.17 (Neumann face rho = 1): within 5x of the table at W = 2
  (measured 13.0 % against 9.63 %), W = 3 on request (2.70 % against 2.52 %).
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle.pcg import pcg
from oracle.precond import element_block
from oracle.vertex import VertexDiscretisation


def _poly_neumann(N, W):
    pb = wl.vertex_polynomial(N, W)
    chi1 = pb.meta["chi1"]
    bc = np.zeros((pb.mesh.n_elem, 6), dtype=np.int32)
    for e in range(pb.mesh.n_elem):
        for fi in (1, 3, 5):
            if pb.mesh.elem_nbr[e, fi] == -1:
                bc[e, fi] = 1
    pb.mesh.elem_bc = bc

    def q(ps, ts, rs):
        # (w_rho, w_phi / rho, w_theta / (rho sin phi)) of 2 + (chi - chi1)^2 phi theta
        p, t, r = wl._sph_grid(ps, ts, rs)
        a = np.log(r) - chi1
        return 2 * a * p * t / r, a * a * t / r, a * a * p / (r * np.sin(p))

    pb.flux = [q]
    return pb


def test_vertex_neumann_polynomial_reproduction():
    pb = _poly_neumann(2, 2)
    d = VertexDiscretisation(pb)
    assert d.mesh.elem_bc.sum() >= 3
    U = d.nodal_interpolant(pb.u_exact)
    assert d.functional(U) <= 1e-22 * d.functional(np.zeros(d.ndof))
    x = np.linalg.solve(d.dense_A(), d.rhs_b())
    assert np.linalg.norm(x - U) <= 1e-8 * np.linalg.norm(U)


def test_vertex_neumann_variation_identity_and_spd():
    d = VertexDiscretisation(_poly_neumann(2, 2))
    rng = np.random.default_rng(43)
    U, V = rng.standard_normal(d.ndof), rng.standard_normal(d.ndof)
    A, b = d.dense_A(), d.rhs_b()
    assert np.abs(A - A.T).max() <= 1e-11 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0
    for eps in (0.5, -1.2):
        lhs = d.functional(U + eps * V)
        rhs = d.functional(U) + 2 * eps * V @ (A @ U - b) + eps ** 2 * V @ A @ V
        assert lhs == pytest.approx(rhs, rel=1e-10)


def _table_6_17_error(W):
    d = VertexDiscretisation(wl.vertex_mixed(2 * W + 4, W))
    fac = [sla.cho_factor(element_block(d, e)) for e in range(d.E)]
    Ucb = np.zeros(d.ndof)
    Ucb[d.coff[0]] = 1.0
    acc = float(d.corner_apply(Ucb, 0)[0])

    def M(r):
        z = np.zeros_like(r)
        for e in range(d.E):
            z[d.off[e]:d.off[e + 1]] = sla.cho_solve(fac[e], r[d.off[e]:d.off[e + 1]])
        z[d.coff[0]] = r[d.coff[0]] / acc
        return z
    x, _, rel = pcg(d.apply_A, M, d.rhs_b(), tol=1e-10, maxit=20000)
    assert rel <= 1e-10
    err, nrm = d.h1_error_exact(x)
    return np.sqrt(err / nrm)


def test_table_6_17_w2():
    from golden_tables import rel_error
    ref = rel_error("table6_17_vertex_mixed.txt", 2)
    err = _table_6_17_error(2)
    assert ref / 5 < err < ref * 5, err


@pytest.mark.slow
def test_table_6_17_w3():
    from golden_tables import rel_error
    ref = rel_error("table6_17_vertex_mixed.txt", 3)
    err = _table_6_17_error(3)
    assert ref / 5 < err < ref * 5, err
