"""Pins of the L-shaped-prism oracle: the edge neighbourhood (modified
coordinates) next to curved regular elements, joined on the circle r = Z by
the interface terms of the singular side (the regular side's gradient
converted into the edge's modified derivatives).

* u = 1 + x3 lies in both regions' spaces and in the corner's: R vanishes and
  block-Jacobi PCG returns it (the interface passes a field with u_x3 != 0).
* A symmetric (random vectors) and the variation identity of the literal
  functional against the matrix-free operator, interface terms included.
* Interface consistency: for a smooth harmonic function interpolated in both
  regions every interface jump falls with W (the conversion of the regular
  side's gradient to u_tau, u_theta, u_x3 is the right one).
* The H^1 error of the re-entrant-edge solution r^(2/3) sin(2 theta'/3) falls
  from W = 2 to W = 3 (N = W + 2 layers).
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle.curved import CurvedMesh, CurvedProblem
from oracle.lprism import LPrismDiscretisation
from oracle.pcg import pcg
from oracle.precond import element_block


def _build(N, W):
    edge, (maps, Ws, nbr, u, gu, f), pairs = wl.lprism_problem(N, W)
    return LPrismDiscretisation(edge, CurvedProblem(CurvedMesh(maps, Ws, nbr), f, u, u, gu), pairs)


def _block_pcg(d, tol):
    """PCG with the two regions' element blocks (interface self terms left
    out: any SPD preconditioner reaches the same solution) and exact corner
    blocks."""
    fe = [sla.cho_factor(element_block(d.ed, e)) for e in range(d.ed.E)]
    fr = [sla.cho_factor(element_block(d.cu, j)) for j in range(d.cu.E)]
    cinv = []
    for c in range(d.ed.C):
        n = d.ed.Wc[c] + 1
        A = np.zeros((n, n))
        for k in range(n):
            U = np.zeros(d.ed.ndof)
            U[d.ed.coff[c] + k] = 1.0
            A[:, k] = d.ed.corner_apply(U, c)
        cinv.append(np.linalg.inv(A))

    def M(r):
        re, rr = d.split(r)
        ze, zr = np.zeros_like(re), np.zeros_like(rr)
        for e in range(d.ed.E):
            s = slice(d.ed.off[e], d.ed.off[e + 1])
            ze[s] = sla.cho_solve(fe[e], re[s])
        for c in range(d.ed.C):
            s = slice(d.ed.coff[c], d.ed.coff[c] + d.ed.Wc[c] + 1)
            ze[s] = cinv[c] @ re[s]
        for j in range(d.cu.E):
            s = slice(d.cu.off[j], d.cu.off[j + 1])
            zr[s] = sla.cho_solve(fr[j], rr[s])
        return d.merge(ze, zr)
    x, _, rel = pcg(d.apply_A, M, d.rhs_b(), tol=tol, maxit=5000)
    assert rel <= tol
    return x


def test_lprism_reproduces_a_function_of_x3():
    d = _build(2, 2)

    def ue(rs, ts, zs):
        r, t, z = wl._cyl_grid(rs, ts, zs)
        return 1.0 + z + 0 * r

    def ur(x, y, z):
        return 1.0 + z + 0 * x

    d.ed.problem.g = [ue]
    d.cu.problem.g = ur
    U = d.merge(d.ed.nodal_interpolant(ue), d.cu.nodal_interpolant(ur))
    assert d.functional(U) <= 1e-22 * d.functional(np.zeros(d.ndof))
    x = _block_pcg(d, 1e-13)
    assert np.linalg.norm(x - U) <= 1e-9 * np.linalg.norm(U)


def test_lprism_symmetry_and_variation_identity():
    d = _build(2, 2)
    rng = np.random.default_rng(31)
    U, V = rng.standard_normal(d.ndof), rng.standard_normal(d.ndof)
    AU, AV, b = d.apply_A(U), d.apply_A(V), d.rhs_b()
    assert abs(V @ AU - U @ AV) <= 1e-12 * abs(V @ AU)
    assert U @ AU > 0 and V @ AV > 0
    for eps in (0.9, -0.4):
        lhs = d.functional(U + eps * V)
        rhs = d.functional(U) + 2 * eps * V @ (AU - b) + eps ** 2 * V @ AV
        assert lhs == pytest.approx(rhs, rel=1e-10)


def test_lprism_interface_jumps_fall_with_w():
    # w = (x - c)^2 - (y - c)^2 + x3: harmonic, the same function on both sides
    def wr(x, y, z):
        return (x - 0.5) ** 2 - (y - 0.5) ** 2 + z

    def we(rs, ts, zs):
        r, t, z = wl._cyl_grid(rs, ts, zs)
        return r * r * np.cos(2 * (t + np.pi / 2)) + z

    # the traces of u, u_theta and u_x3 on the circle are interpolants of the
    # same function on the same GLL nodes on both sides: equal to rounding;
    # u_tau differs by the interpolation error across the face (measured
    # 1.5e-2, 1.2e-4 at W = 3, 6)
    worst = {}
    for W in (3, 6, 9):
        d = _build(2, W)
        Ue, Ur = d.ed.nodal_interpolant(we), d.cu.nodal_interpolant(wr)
        m = 0.0
        for e, j in d.pairs:
            J = d._jumps(Ue, Ur, e, j, d._Qf(e, j))
            for k in (0, 2, 3):
                assert float(np.abs(J[k]).max()) <= 1e-12, (W, k)
            m = max(m, float(np.abs(J[1]).max()))
        worst[W] = m
    assert worst[6] < 0.05 * worst[3] and worst[9] < 0.05 * worst[6], worst


@pytest.mark.slow
def test_lprism_h1_error_falls():
    # measured 15.1 % (W = 2, N = 4, 813 DOF) and 3.09 % (W = 3, N = 5, 2,308 DOF)
    errs = {}
    for W in (2, 3):
        d = _build(W + 2, W)
        errs[W] = d.h1_error_exact(_block_pcg(d, 1e-11))
    assert errs[3] < 0.6 * errs[2], errs


def _build_layers(layer_W, W):
    N = len(layer_W)
    edge, (maps, Ws, nbr, u, gu, f), pairs = wl.lprism_problem(N, W, layer_W=layer_W)
    return LPrismDiscretisation(edge, CurvedProblem(CurvedMesh(maps, Ws, nbr), f, u, u, gu), pairs)


def test_lprism_degrees_rising_across_layers():
    # degrees 1, 2, 3 from the edge outward (config 3 rises 2..8 over six
    # layers): faces between layers of unequal degree take the (2 W_f + 1)-point
    # grid of the larger one; the corner polynomial and the regular sectors
    # have degree 3
    d = _build_layers((1, 2, 3), 3)
    assert sorted(set(d.ed.W)) == [1, 2, 3]
    rng = np.random.default_rng(37)
    U, V = rng.standard_normal(d.ndof), rng.standard_normal(d.ndof)
    AU, AV, b = d.apply_A(U), d.apply_A(V), d.rhs_b()
    assert abs(V @ AU - U @ AV) <= 1e-12 * abs(V @ AU)
    for eps in (0.7, -0.3):
        lhs = d.functional(U + eps * V)
        rhs = d.functional(U) + 2 * eps * V @ (AU - b) + eps ** 2 * V @ AV
        assert lhs == pytest.approx(rhs, rel=1e-10)

    def ue(rs, ts, zs):
        r, t, z = wl._cyl_grid(rs, ts, zs)
        return 1.0 + z + 0 * r

    def ur(x, y, z):
        return 1.0 + z + 0 * x

    d.ed.problem.g = [ue]
    d.cu.problem.g = ur
    U = d.merge(d.ed.nodal_interpolant(ue), d.cu.nodal_interpolant(ur))
    assert d.functional(U) <= 1e-22 * d.functional(np.zeros(d.ndof))
