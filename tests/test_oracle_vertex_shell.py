"""Pins of the composite oracle of a vertex neighbourhood inside a spherical
shell of curved regular elements (joined on the sphere rho = rho_v by the
vertex side's interface terms, the regular side's gradient converted to the
vertex's modified derivatives).

* The spherical shell map's derivatives against central differences.
* A symmetric and the variation identity with the interface terms.
* Interface consistency: for a smooth function interpolated on both sides the
  traces of u, u_phi and u_theta on the sphere agree to rounding and the u_chi
  jump falls with W (measured 5.2e-2, 3.8e-4 at W = 3, 6).
* Table 6.16's solution on the whole wedge (vertex neighbourhood rho < 1/2 and
  the shell): the H^1 error within 5x of the table at W = 2 (measured 1.25 %
  against 1.01 %).
"""
import numpy as np
import pytest

import workloads as wl
from oracle.curved import CurvedMesh, CurvedProblem
from oracle.vertex_shell import VertexShellDiscretisation


def _build(N, W, J=1):
    v, (maps, Ws, nbr, u, gu, f), pairs = wl.vertex_with_shell(N, W, J=J)
    return VertexShellDiscretisation(v, CurvedProblem(CurvedMesh(maps, Ws, nbr), f, u, u, gu), pairs)


def test_shell_map_derivatives():
    m = wl.spherical_shell_map(0.5, 1.0, 0.2, 1.1, 0.5, 1.0)
    rng = np.random.default_rng(59)
    lam = [rng.uniform(-1, 1, 6) for _ in range(3)]
    x, Dx, D2x = m(*lam)
    h = 1e-5
    for a in range(3):
        lp = [v.copy() for v in lam]
        lm = [v.copy() for v in lam]
        lp[a] += h
        lm[a] -= h
        xp, Dp, _ = m(*lp)
        xm, Dm, _ = m(*lm)
        assert np.abs((xp - xm) / (2 * h) - Dx[:, a]).max() <= 1e-8
        assert np.abs((Dp - Dm) / (2 * h) - D2x[:, :, a]).max() <= 1e-8


def test_symmetry_and_variation_identity():
    d = _build(2, 2)
    rng = np.random.default_rng(61)
    U, V = rng.standard_normal(d.ndof), rng.standard_normal(d.ndof)
    AU, AV, b = d.apply_A(U), d.apply_A(V), d.rhs_b()
    assert abs(V @ AU - U @ AV) <= 1e-12 * abs(V @ AU)
    assert U @ AU > 0 and V @ AV > 0
    for eps in (0.5, -1.0):
        lhs = d.functional(U + eps * V)
        rhs = d.functional(U) + 2 * eps * V @ (AU - b) + eps ** 2 * V @ AV
        assert lhs == pytest.approx(rhs, rel=1e-10)


def test_interface_traces():
    def w_sph(ps, ts, rs):
        p, t, r = wl._sph_grid(ps, ts, rs)
        return r * r * np.sin(p) ** 2 * np.cos(2 * t) + r * np.cos(p)

    def w_x(x, y, z):
        return x * x - y * y + z

    worst = {}
    for W in (3, 6):
        d = _build(2, W)
        Uv, Ur = d.vd.nodal_interpolant(w_sph), d.cu.nodal_interpolant(w_x)
        m = 0.0
        for e, j in d.pairs:
            J = d._jumps(Uv, Ur, e, j, d._Qf(e, j))
            for k in (0, 1, 2):
                assert float(np.abs(J[k]).max()) <= 1e-12, (W, k)
            m = max(m, float(np.abs(J[3]).max()))
        worst[W] = m
    assert worst[6] < 0.05 * worst[3], worst


def test_table_6_16_on_vertex_and_shell():
    import scipy.linalg as sla
    from golden_tables import rel_error
    from oracle.pcg import pcg
    from oracle.precond import element_block
    d = _build(2 * 2 + 4, 2, J=3)
    fv = [sla.cho_factor(element_block(d.vd, e)) for e in range(d.vd.E)]
    fr = [sla.cho_factor(element_block(d.cu, j)) for j in range(d.cu.E)]

    def M(r):
        rv, rr = d.split(r)
        zv, zr = np.zeros_like(rv), np.zeros_like(rr)
        for e in range(d.vd.E):
            s = slice(d.vd.off[e], d.vd.off[e + 1])
            zv[s] = sla.cho_solve(fv[e], rv[s])
        zv[d.vd.off[-1]:] = rv[d.vd.off[-1]:]
        for j in range(d.cu.E):
            s = slice(d.cu.off[j], d.cu.off[j + 1])
            zr[s] = sla.cho_solve(fr[j], rr[s])
        return d.merge(zv, zr)
    x, _, rel = pcg(d.apply_A, M, d.rhs_b(), tol=1e-10, maxit=20000)
    assert rel <= 1e-10
    err = d.h1_error_exact(x)
    ref = rel_error("table6_16_vertex.txt", 2)
    assert ref / 5 < err < ref * 5, err
