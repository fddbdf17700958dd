"""Pins of the oracle's H^1 norm of discrete functions on vertex and
vertex-edge neighbourhoods (Section 6.1, physical coordinates), which the
library's hpse_h1_error is checked against.

A discrete function whose element blocks are a coordinate of the modified
system (1, the first, second or third variable) has a closed-form physical H^1
norm over each element box: the integrand is a product of exponentials,
sines and low powers of the variables (vertex: dx = e^{3 chi} sin(phi),
|grad v|^2 = e^{-2 chi}(v_chi^2 + v_phi^2 + v_theta^2 / sin^2 phi);
vertex-edge: dx = e^{2 psi + 3 zeta}, grad v = (v_psi / r, v_theta / r,
(v_zeta - v_psi) / x3)).  A dropped factor, a wrong exponent or a swapped
derivative fails one of the four functions.  The corner sets are pinned by a
constant (the volume of the corner region in closed form) and, on vertex-edge
meshes, by the polynomial zeta on the zeta-layer of its set.  The element rule
is the (2W+1)-point GLL rule, W = 6 here, exact to 1e-11 for these integrands.
"""
import numpy as np
import pytest

import workloads as wl
from oracle.gll import gll
from oracle.vertex import VertexDiscretisation
from oracle.vertex import h1_diff as vertex_h1
from oracle.vertex_edge import VertexEdgeDiscretisation
from oracle.vertex_edge import h1_diff as ve_h1

W = 6


def _blocks(d, g):
    U = np.zeros(d.ndof)
    for e in range(d.E):
        xp, _ = gll(d.P[e])
        lo, hi = d.mesh.elem_lo[e], d.mesh.elem_hi[e]
        xs, ys, zs = (lo[a] + (xp + 1.0) * (hi[a] - lo[a]) / 2.0 for a in range(3))
        G = g(xs[None, None, :], ys[None, :, None], zs[:, None, None]) * np.ones((d.P[e],) * 3)
        U[d.off[e]:d.off[e + 1]] = G.ravel()
    return U


def _vertex():
    base = wl.vertex_poisson_singular(N=3, W=W)
    return VertexDiscretisation(wl.EdgeProblem(wl.vertex_mesh(3, W, I=1, J=2), base.f, base.g, base.u_exact,
                                               base.grad_exact))


def _ve():
    base = wl.vertex_edge_singular(N=2, W=W)
    return VertexEdgeDiscretisation(wl.EdgeProblem(wl.vertex_edge_mesh(2, W, J=2), base.f, base.g, base.u_exact,
                                                   base.grad_exact))


def _vertex_closed(d, which):
    tot = 0.0
    for e in range(d.E):
        (p0, t0, c0), (p1, t1, c1) = d.mesh.elem_lo[e], d.mesh.elem_hi[e]
        dcos = np.cos(p0) - np.cos(p1)
        e3 = (np.exp(3 * c1) - np.exp(3 * c0)) / 3.0
        e1 = np.exp(c1) - np.exp(c0)
        if which == "one":
            tot += dcos * (t1 - t0) * e3
        elif which == "chi":
            F = lambda c: np.exp(3 * c) * (c * c / 3 - 2 * c / 9 + 2 / 27.0) + np.exp(c)
            tot += dcos * (t1 - t0) * (F(c1) - F(c0))
        elif which == "phi":
            G = lambda p: -p * p * np.cos(p) + 2 * p * np.sin(p) + 2 * np.cos(p)
            tot += (t1 - t0) * ((G(p1) - G(p0)) * e3 + dcos * e1)
        else:  # theta
            lt = lambda p: np.log(np.tan(p / 2.0))
            tot += (t1 ** 3 - t0 ** 3) / 3.0 * dcos * e3 + (t1 - t0) * e1 * (lt(p1) - lt(p0))
    return tot


@pytest.mark.parametrize("which,g", [("one", lambda x, y, z: 1.0 + 0 * x), ("chi", lambda x, y, z: z + 0 * x),
                                     ("phi", lambda x, y, z: x + 0 * z), ("theta", lambda x, y, z: y + 0 * x)])
def test_vertex_h1_of_coordinate_functions(which, g):
    d = _vertex()
    U = _blocks(d, g)
    got, _ = vertex_h1(d, U, np.zeros(d.ndof))
    assert got == pytest.approx(_vertex_closed(d, which), rel=1e-11)


def test_vertex_h1_corner_constant():
    d = _vertex()
    U = np.zeros(d.ndof)
    U[d.coff[0]] = 1.7
    got, _ = vertex_h1(d, U, np.zeros(d.ndof))
    want = 0.0
    for e in range(d.E):
        if int(d.mesh.elem_nbr[e, 4]) == -2:
            (p0, t0, c0), (p1, t1, _) = d.mesh.elem_lo[e], d.mesh.elem_hi[e]
            want += 1.7 ** 2 * np.exp(3 * c0) / 3.0 * (np.cos(p0) - np.cos(p1)) * (t1 - t0)
    assert want > 0 and got == pytest.approx(want, rel=1e-13)
    # the second output is the reference's norm, and the difference is taken
    e_uv, n_v = vertex_h1(d, U, U)
    assert e_uv == 0.0 and n_v == pytest.approx(got, rel=1e-15)


def _ve_closed(d, which):
    tot = 0.0
    for e in range(d.E):
        (s0, t0, z0), (s1, t1, z1) = d.mesh.elem_lo[e], d.mesh.elem_hi[e]
        e2 = (np.exp(2 * s1) - np.exp(2 * s0)) / 2.0
        z3 = (np.exp(3 * z1) - np.exp(3 * z0)) / 3.0
        z1e = np.exp(z1) - np.exp(z0)
        th = t1 - t0
        if which == "one":
            tot += th * e2 * z3
        elif which == "psi":
            F = lambda s: np.exp(2 * s) * (s * s / 2 - s / 2 + 0.25)
            tot += th * ((F(s1) - F(s0)) * z3 + (s1 - s0) * z1e + e2 * z1e)
        elif which == "zeta":
            F = lambda z: np.exp(3 * z) * (z * z / 3 - 2 * z / 9 + 2 / 27.0)
            tot += th * (e2 * (F(z1) - F(z0)) + e2 * z1e)
        else:  # theta
            tot += (t1 ** 3 - t0 ** 3) / 3.0 * e2 * z3 + th * (s1 - s0) * z1e
    return tot


@pytest.mark.parametrize("which,g", [("one", lambda x, y, z: 1.0 + 0 * x), ("psi", lambda x, y, z: x + 0 * z),
                                     ("zeta", lambda x, y, z: z + 0 * x), ("theta", lambda x, y, z: y + 0 * x)])
def test_vertex_edge_h1_of_coordinate_functions(which, g):
    d = _ve()
    U = _blocks(d, g)
    got, _ = ve_h1(d, U, np.zeros(d.ndof))
    assert got == pytest.approx(_ve_closed(d, which), rel=1e-11)


def test_vertex_edge_h1_corner_sets():
    d = _ve()
    for c in range(d.C):
        U = np.zeros(d.ndof)
        want = 0.0
        if d.cface[c] == 0:
            # the polynomial zeta on the set's zeta layer:
            # (e^{2 psi_1} / 2) theta-span int (e^{3 zeta} zeta^2 + e^zeta) dzeta
            e = next(e for e in range(d.E) if int(d.mesh.elem_nbr[e, 0]) == -2 - c)
            z0, z1 = d.mesh.elem_lo[e, 2], d.mesh.elem_hi[e, 2]
            xp, _ = gll(d.Wc[c] + 1)
            U[d.coff[c]:d.coff[c] + d.Wc[c] + 1] = z0 + (xp + 1.0) * (z1 - z0) / 2.0
            F = lambda z: np.exp(3 * z) * (z * z / 3 - 2 * z / 9 + 2 / 27.0) + np.exp(z)
            for e in range(d.E):
                if int(d.mesh.elem_nbr[e, 0]) == -2 - c:
                    want += 0.5 * np.exp(2 * d.mesh.elem_lo[e, 0]) * (d.mesh.elem_hi[e, 1] - d.mesh.elem_lo[e, 1]) * (
                        F(z1) - F(z0))
        else:
            # a constant on x3 < x3_1 inside the cone psi < psi_top of every theta sector
            U[d.coff[c]] = 0.9
            sectors = {}
            for e in range(d.E):
                if int(d.mesh.elem_nbr[e, 4]) == -2 - c:
                    k = round(float(d.mesh.elem_lo[e, 1]), 12)
                    th = d.mesh.elem_hi[e, 1] - d.mesh.elem_lo[e, 1]
                    pt = max(sectors.get(k, (0, -np.inf, 0))[1], d.mesh.elem_hi[e, 0])
                    sectors[k] = (th, pt, d.mesh.elem_lo[e, 2])
            for th, pt, z1 in sectors.values():
                want += 0.81 * th * np.exp(2 * pt) / 2.0 * np.exp(3 * z1) / 3.0
        got, _ = ve_h1(d, U, np.zeros(d.ndof))
        assert want > 0 and got == pytest.approx(want, rel=1e-11), c
