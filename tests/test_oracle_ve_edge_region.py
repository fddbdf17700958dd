"""Pins of the composite oracle of the vertex-edge cone and the edge
neighbourhood above it, joined on the plane x3 = delta (the vertex-edge side's
interface terms, the edge side's derivatives converted by the chain rule of
tau = psi + zeta, x3 = e^zeta).

* A symmetric and the variation identity with the interface terms.
* Interface consistency: for a smooth function interpolated on both sides the
  traces of u, u_psi (= u_tau) and u_theta on the plane agree to rounding
  (the two face grids are the same points) and the u_zeta jump falls with W
  (measured 0.22, 1.9e-3 at W = 3, 6).
* A constant is reproduced across the plane.
"""
import numpy as np
import pytest

import workloads as wl
from oracle.ve_edge_region import VertexEdgeEdgeDiscretisation

DELTA = float(np.cos(np.pi / 6))


def _build(N, W, J=1):
    ve, edge, pairs = wl.vertex_edge_with_edge(N, W, J=J)
    return VertexEdgeEdgeDiscretisation(ve, edge, pairs, DELTA)


def test_symmetry_and_variation_identity():
    d = _build(2, 2)
    rng = np.random.default_rng(53)
    U, V = rng.standard_normal(d.ndof), rng.standard_normal(d.ndof)
    AU, AV, b = d.apply_A(U), d.apply_A(V), d.rhs_b()
    assert abs(V @ AU - U @ AV) <= 1e-12 * abs(V @ AU)
    assert U @ AU > 0 and V @ AV > 0
    for eps in (0.5, -1.0):
        lhs = d.functional(U + eps * V)
        rhs = d.functional(U) + 2 * eps * V @ (AU - b) + eps ** 2 * V @ AV
        assert lhs == pytest.approx(rhs, rel=1e-10)


def test_interface_traces():
    def w_ve(ps, ts, zs):
        p, t, z = wl._ve_grid(ps, ts, zs)
        rr, x3 = np.exp(p + z), np.exp(z)
        return rr * rr * np.cos(2 * t) + x3 * x3 - rr * rr / 2 + x3

    def w_cyl(rs, ts, zs):
        r, t, z = wl._cyl_grid(rs, ts, zs)
        return r * r * np.cos(2 * t) + z * z - r * r / 2 + z

    worst = {}
    for W in (3, 6):
        d = _build(2, W)
        Uv, Ue = d.vd.nodal_interpolant(w_ve), d.ed.nodal_interpolant(w_cyl)
        m = 0.0
        for a, b in d.pairs:
            J = d._jumps(Uv, Ue, a, b, d._Qf(a, b))
            for k in (0, 1, 2):
                assert float(np.abs(J[k]).max()) <= 1e-12, (W, k)
            m = max(m, float(np.abs(J[3]).max()))
        worst[W] = m
    assert worst[6] < 0.05 * worst[3], worst


def test_constant_is_reproduced():
    d = _build(2, 2)

    def c_ve(ps, ts, zs):
        p, t, z = wl._ve_grid(ps, ts, zs)
        return 3.0 + 0 * (p + t + z)

    def c_cyl(rs, ts, zs):
        r, t, z = wl._cyl_grid(rs, ts, zs)
        return 3.0 + 0 * (r + t + z)

    d.vd.problem.f, d.vd.problem.g = [lambda *a: 0 * c_ve(*a)], [c_ve]
    d.ed.problem.f, d.ed.problem.g = [lambda *a: 0 * c_cyl(*a)], [c_cyl]
    U = np.full(d.ndof, 3.0)
    assert d.functional(U) <= 1e-22
    AU, b = d.apply_A(U), d.rhs_b()
    assert np.abs(AU - b).max() <= 1e-11 * np.abs(b).max()
