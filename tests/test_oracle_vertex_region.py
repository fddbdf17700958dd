"""Pins of the composite oracle of a vertex neighbourhood with one re-entrant
edge: the vertex part and the vertex-edge cone joined on phi = pi/6 (the
vertex-edge side's interface terms, the vertex side's derivatives converted by
the chain rule), one constant shared by both regions' corner elements.

* A constant lies in every space (the shared corner constant included): R
  vanishes and block-Jacobi PCG returns it.
* A symmetric and the variation identity with the interface terms.
* Interface consistency: for a smooth function interpolated on both sides the
  traces of u, u_theta and u_zeta on the cone agree to rounding (the two face
  grids are the same points) and the u_psi jump falls with W.
* Table 6.20's solution on the union domain: the H^1 error falls from W = 2
  to W = 3 (slow-marked).
"""
import numpy as np
import pytest

import workloads as wl
from oracle.vertex_region import VertexRegionDiscretisation


def _build(N, W, J=1):
    v, ve, pairs = wl.vertex_with_edge(N, W, J=J)
    return VertexRegionDiscretisation(v, ve, pairs)


def _pcg(d, tol):
    import scipy.linalg as sla
    from oracle.pcg import pcg
    from oracle.precond import element_block
    fv = [sla.cho_factor(element_block(d.vd, e)) for e in range(d.vd.E)]
    fe = [sla.cho_factor(element_block(d.ed, e)) for e in range(d.ed.E)]

    def M(r):
        rv, re = d.split(r)
        zv, ze = np.zeros_like(rv), np.zeros_like(re)
        for e in range(d.vd.E):
            s = slice(d.vd.off[e], d.vd.off[e + 1])
            zv[s] = sla.cho_solve(fv[e], rv[s])
        for e in range(d.ed.E):
            s = slice(d.ed.off[e], d.ed.off[e + 1])
            ze[s] = sla.cho_solve(fe[e], re[s])
        z = d.merge(zv, ze)
        z[d.nV + d.nE:] = r[d.nV + d.nE:]      # corner values: unpreconditioned
        return z
    x, _, rel = pcg(d.apply_A, M, d.rhs_b(), tol=tol, maxit=20000)
    assert rel <= tol
    return x


def test_constant_is_reproduced():
    d = _build(2, 2)

    def c_sph(ps, ts, rs):
        p, t, r = wl._sph_grid(ps, ts, rs)
        return 2.0 + 0 * (p + t + r)

    def c_ve(ps, ts, zs):
        p, t, z = wl._ve_grid(ps, ts, zs)
        return 2.0 + 0 * (p + t + z)

    def zero_sph(ps, ts, rs):
        return 0 * c_sph(ps, ts, rs)

    def zero_ve(ps, ts, zs):
        return 0 * c_ve(ps, ts, zs)

    d.vd.problem.f, d.vd.problem.g = [zero_sph], [c_sph]
    d.ed.problem.f, d.ed.problem.g = [zero_ve], [c_ve]
    U = np.full(d.ndof, 2.0)
    assert d.functional(U) <= 1e-24
    x = _pcg(d, 1e-13)
    assert np.abs(x - 2.0).max() <= 1e-9


def test_symmetry_and_variation_identity():
    d = _build(2, 2)
    rng = np.random.default_rng(47)
    U, V = rng.standard_normal(d.ndof), rng.standard_normal(d.ndof)
    AU, AV, b = d.apply_A(U), d.apply_A(V), d.rhs_b()
    assert abs(V @ AU - U @ AV) <= 1e-12 * abs(V @ AU)
    assert U @ AU > 0 and V @ AV > 0
    for eps in (0.5, -1.0):
        lhs = d.functional(U + eps * V)
        rhs = d.functional(U) + 2 * eps * V @ (AU - b) + eps ** 2 * V @ AV
        assert lhs == pytest.approx(rhs, rel=1e-10)


def test_interface_traces():
    # measured u_psi jumps 5.0e-2, 4.2e-4 at W = 3, 6
    def w_sph(ps, ts, rs):
        p, t, r = wl._sph_grid(ps, ts, rs)
        rr, x3 = r * np.sin(p), r * np.cos(p)
        return rr * rr * np.cos(2 * t) + x3

    def w_ve(ps, ts, zs):
        p, t, z = wl._ve_grid(ps, ts, zs)
        rr, x3 = np.exp(p + z), np.exp(z)
        return rr * rr * np.cos(2 * t) + x3

    worst = {}
    for W in (3, 6):
        d = _build(2, W)
        Uv, Ue = d.vd.nodal_interpolant(w_sph), d.ed.nodal_interpolant(w_ve)
        m = 0.0
        for a, b in d.pairs:
            J = d._jumps(Uv, Ue, a, b, d._Qf(a, b))
            for k in (0, 2, 3):
                assert float(np.abs(J[k]).max()) <= 1e-12, (W, k)
            m = max(m, float(np.abs(J[1]).max()))
        worst[W] = m
    assert worst[6] < 0.05 * worst[3], worst


@pytest.mark.slow
def test_table_6_20_solution_error_falls():
    errs = {}
    for W in (2, 3):
        d = _build(W + 1, W)
        errs[W] = d.h1_error_exact(_pcg(d, 1e-10))
    assert errs[3] < 0.7 * errs[2], errs
