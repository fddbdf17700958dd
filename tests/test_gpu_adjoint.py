"""GPU parity of the residual map, its hand-written transpose, point fields
and the adjoint data gradient; autograd gradients of a solution functional
against the oracle's adjoint gradient and against finite differences.

Tolerances: kernels vs oracle 1e-12 relative (FP64 sums in a different
order); end-to-end gradients 1e-7 relative (both sides solve to a relative
residual of 1e-13 / exactly); finite differences: Richardson-extrapolated
central differences, |g - fd| <= 1e-6 max(|fd|, 1e-3 |g|_inf).
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle.adjoint import data_gradient, element_fields, l2_misfit_gradient
from oracle.functional import Discretisation
from oracle.gll import gll
from oracle.pcg import cholesky_solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1110_2316_gb300.build import build
    build()
    from paper_1110_2316_gb300 import api as A
    return A


def _mesh(api, pb):
    kind = api.COEF_SCALAR if pb.a is not None else api.COEF_LAPLACE
    m = api.Mesh(pb.mesh, n_rhs=pb.n_rhs, coef_kind=kind)
    m.set_data(**api.problem_data_arrays(m, pb))
    return m


def _flat(disc, per_elem):
    return np.concatenate([np.asarray(x).ravel() for x in per_elem])


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def u_target(xs, ys, zs):
    x, y, z = wl._grid(xs, ys, zs)
    return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


@pytest.mark.parametrize("n,W", [((2, 2, 1), 4), ((2, 1, 1), 7), ((1, 1, 2), 10)])
def test_fields_residual_transpose_match_oracle(api, n, W):
    pb = wl.varcoef_manufactured(n=n, W=W)
    m = _mesh(api, pb)
    disc = Discretisation(pb)
    U = wl.random_dofs(m.ndof, seed=4)
    u = torch.tensor(U, device="cuda")
    F = torch.empty(1, 5, m.nquad, dtype=torch.float64, device="cuda")
    m.eval_fields(u, F)
    F = F.cpu().numpy()[0]
    ref = [element_fields(disc, U, e) for e in range(disc.E)]
    for k in range(5):
        assert _rel(F[k], _flat(disc, [r[k] for r in ref])) <= 1e-12, k
    z = torch.empty(1, m.nquad, dtype=torch.float64, device="cuda")
    m.apply_residual(u, z)
    zref = _flat(disc, [np.sqrt(disc.vol_weight(e)) * (disc.L_apply(disc.block(U, e), e) - disc.f_at(e, 0))
                        for e in range(disc.E)])
    assert _rel(z.cpu().numpy()[0], zref) <= 1e-12
    Z = np.random.default_rng(1).standard_normal(m.nquad)
    y = torch.empty_like(u)
    m.apply_transpose(torch.tensor(Z, device="cuda"), y)
    Q = [2 * w + 1 for w in disc.W]
    o, yref = 0, []
    for e in range(disc.E):
        n = Q[e] ** 3
        zb = Z[o:o + n].reshape(Q[e], Q[e], Q[e])
        yref.append(disc.L_apply_T(np.sqrt(disc.vol_weight(e)) * zb, e))
        o += n
    assert _rel(y.cpu().numpy(), _flat(disc, yref)) <= 1e-12


@pytest.mark.parametrize("W", [3, 9])
def test_adjoint_identities(api, W):
    pb = wl.varcoef_manufactured(n=(2, 1, 2), W=W)
    m = _mesh(api, pb)
    rng = np.random.default_rng(5)
    u = torch.tensor(rng.standard_normal(m.ndof), device="cuda")
    zz = torch.tensor(rng.standard_normal(m.nquad), device="cuda")
    z0 = torch.empty(1, m.nquad, dtype=torch.float64, device="cuda")
    z1 = torch.empty_like(z0)
    m.apply_residual(torch.zeros_like(u), z0)
    m.apply_residual(u, z1)
    Su = (z1 - z0)[0]  # linear part of the residual map
    y = torch.empty_like(u)
    m.apply_transpose(zz, y)
    lhs, rhs = float((Su * zz).sum()), float((u * y).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)
    F = torch.empty(1, 5, m.nquad, dtype=torch.float64, device="cuda")
    m.eval_fields(u, F)
    m.apply_eval_transpose(zz, y)
    lhs, rhs = float((F[0, 0] * zz).sum()), float((u * y).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("W", [3, 6, 10])
def test_data_gradient_matches_oracle(api, W):
    pb = wl.varcoef_manufactured(n=(2, 1, 1), W=W)
    m = _mesh(api, pb)
    disc = Discretisation(pb)
    rng = np.random.default_rng(8)
    U, L = rng.standard_normal(m.ndof), rng.standard_normal(m.ndof)
    uf = torch.empty(1, 5, m.nquad, dtype=torch.float64, device="cuda")
    lf = torch.empty_like(uf)
    m.eval_fields(torch.tensor(U, device="cuda"), uf)
    m.eval_fields(torch.tensor(L, device="cuda"), lf)
    g = torch.empty_like(uf)
    m.data_gradient(uf, lf, g)
    g = g.cpu().numpy()[0]
    ref = data_gradient(disc, U, L)
    for k in range(5):
        assert _rel(g[k], _flat(disc, [r[k] for r in ref])) <= 1e-12, k


def test_autograd_solve_gradient_matches_oracle(api):
    from paper_1110_2316_gb300.autograd import PointValues, Solve
    pb = wl.varcoef_manufactured(n=(2, 1, 1), W=2)
    m = api.Mesh(pb.mesh, n_rhs=1, coef_kind=api.COEF_SCALAR)
    d = api.problem_data_arrays(m, pb)
    f = torch.tensor(d["f"], device="cuda", requires_grad=True)
    a = torch.tensor(d["a"], device="cuda", requires_grad=True)
    ga = torch.tensor(d["grad_a"], device="cuda", requires_grad=True)
    u = Solve.apply(f, a, ga, m, d["g"], 1e-12)
    v = PointValues.apply(u, m)[0]
    w = torch.empty(m.nquad, dtype=torch.float64, device="cuda")
    m.quad_weights(w)
    disc = Discretisation(pb)
    ut = torch.tensor(_flat(disc, [u_target(*disc.qpoints(e)) for e in range(disc.E)]), device="cuda")
    J = (w * (v - ut) ** 2).sum()
    J.backward()
    # oracle: exact solve, adjoint by Cholesky
    A = disc.dense_A()
    Uo = cholesky_solve(A, disc.rhs_b())
    lam = cholesky_solve(A, l2_misfit_gradient(disc, Uo, u_target))
    ref = data_gradient(disc, Uo, lam)
    assert _rel(f.grad.cpu().numpy()[0], _flat(disc, [r[0] for r in ref])) <= 1e-7
    assert _rel(a.grad.cpu().numpy(), _flat(disc, [r[1] for r in ref])) <= 1e-7
    for k in range(3):
        assert _rel(ga.grad.cpu().numpy()[k], _flat(disc, [r[2 + k] for r in ref])) <= 1e-7


# ---- coefficient parameters theta of a = exp(g), g = sum theta_ijk L_i L_j L_k ----
def _legendre(K, t):
    L = [torch.ones_like(t), t]
    dL = [torch.zeros_like(t), torch.ones_like(t)]
    for m in range(1, K):
        L.append(((2 * m + 1) * t * L[m] - m * L[m - 1]) / (m + 1))
        dL.append(dL[m - 1] + (2 * m + 1) * L[m])
    return torch.stack(L[:K + 1]), torch.stack(dL[:K + 1])


def coef_from_theta(theta, mesh, ax, elem_prob):
    """a and grad a at the volume points from theta [n_problem, 4, 4, 4] (torch, differentiable)."""
    a_parts, g_parts = [], [[], [], []]
    o = 0
    for e, W in enumerate(mesh.elem_W):
        Q = 2 * int(W) + 1
        t = [2 * torch.tensor(ax[o + k * Q:o + (k + 1) * Q], device=theta.device) - 1 for k in range(3)]
        o += 3 * Q
        (Lx, dLx), (Ly, dLy), (Lz, dLz) = (_legendre(3, tt) for tt in t)
        th = theta[int(elem_prob[e])]
        g = torch.einsum("ijk,ia,jb,kc->cba", th, Lx, Ly, Lz)
        gx = 2 * torch.einsum("ijk,ia,jb,kc->cba", th, dLx, Ly, Lz)
        gy = 2 * torch.einsum("ijk,ia,jb,kc->cba", th, Lx, dLy, Lz)
        gz = 2 * torch.einsum("ijk,ia,jb,kc->cba", th, Lx, Ly, dLz)
        aa = torch.exp(g)
        a_parts.append(aa.reshape(-1))
        for k, gk in enumerate((gx, gy, gz)):
            g_parts[k].append((aa * gk).reshape(-1))
    return torch.cat(a_parts), torch.stack([torch.cat(p) for p in g_parts])


def test_theta_gradient_finite_differences(api):
    from paper_1110_2316_gb300.autograd import PointValues, Solve
    parts = [wl.lognormal_coef_problem(W, p, n=2) for p, W in enumerate((3, 4, 2))]
    pb = wl.batch_problems(parts)
    m = api.Mesh(pb.mesh, n_rhs=1, coef_kind=api.COEF_SCALAR)
    d = api.problem_data_arrays(m, pb)
    ax, _ = m.query_points()
    eprob = pb.mesh.elem_problem
    disc = Discretisation(pb)
    ut = torch.tensor(_flat(disc, [u_target(*disc.qpoints(e)) for e in range(disc.E)]), device="cuda")
    f = torch.tensor(d["f"], device="cuda")
    qprob = torch.tensor(np.concatenate([np.full((2 * int(W) + 1) ** 3, int(eprob[e]))
                                         for e, W in enumerate(m.elem_W)]), device="cuda")
    theta0 = torch.tensor(np.stack([p.meta["theta"] for p in parts]), device="cuda")

    def J_per_problem(theta, grad=False):
        a, ga = coef_from_theta(theta, m, ax, eprob)
        u = Solve.apply(f, a, ga, m, None, 1e-11)
        v = PointValues.apply(u, m)[0]
        w = torch.empty(m.nquad, dtype=torch.float64, device="cuda")
        m.quad_weights(w)
        contrib = w * (v - ut) ** 2
        return torch.zeros(len(parts), dtype=torch.float64, device="cuda").index_add(0, qprob, contrib)

    theta = theta0.clone().requires_grad_(True)
    Jp = J_per_problem(theta)
    Jp.sum().backward()
    g = theta.grad.cpu().numpy()
    h = 1e-3
    for idx in [(1, 0, 0), (0, 2, 1), (3, 3, 3)]:
        def central(step):
            tp, tm = theta0.clone(), theta0.clone()
            tp[(slice(None),) + idx] += step
            tm[(slice(None),) + idx] -= step
            with torch.no_grad():
                return ((J_per_problem(tp) - J_per_problem(tm)) / (2 * step)).cpu().numpy()
        fd = (4 * central(h / 2) - central(h)) / 3
        for p in range(len(parts)):
            scale = max(abs(fd[p]), 1e-3 * np.abs(g[p]).max())
            assert abs(g[(p,) + idx] - fd[p]) <= 1e-6 * scale, (p, idx, g[(p,) + idx], fd[p])


def test_theta_gradient_high_degree_difference_form_fd(api):
    # the adjoint batch's problems at W = 8 and 10 (4^3 elements each,
    # lognormal coefficient): the adjoint gradient (forward FP64 to 1e-11,
    # adjoint FP64 to 1e-8) against central differences at h = 1e-4 whose
    # J(+) - J(-) is one quadrature of pointwise differences of the corrected
    # solutions (truncation ~1e-8, rounding noise ~3e-7 of the gradient:
    # measured by a sweep of h on this batch); bound 1e-6 of the scale
    import math
    from paper_1110_2316_gb300.autograd import PointValues, Solve
    from paper_1110_2316_gb300.fields import LegendreLogField
    Ws = wl.adjoint_batch_degrees(256)
    pick = [int(np.flatnonzero(Ws == W)[0]) for W in (8, 10)]
    parts = [wl.lognormal_coef_problem(int(Ws[p]), p, n=4) for p in pick]
    pb = wl.batch_problems(parts)
    m = api.Mesh(pb.mesh, n_rhs=1, coef_kind=api.COEF_SCALAR)
    dev = torch.device("cuda")
    fld = LegendreLogField.from_mesh(m, pb.mesh.elem_problem, device=dev)
    pi = math.pi
    ut = fld.separable(lambda x: torch.sin(pi * x), lambda y: torch.sin(pi * y), lambda z: torch.sin(pi * z))
    f = torch.ones(1, m.nquad, dtype=torch.float64, device=dev)
    th0 = torch.tensor(np.stack([p.meta["theta"] for p in parts]), device=dev)
    a0, ga0 = fld(th0)
    m.set_data(f=f, a=a0, grad_a=ga0)
    m.setup_block_preconditioner()
    w = torch.empty(m.nquad, dtype=torch.float64, device=dev)
    m.quad_weights(w)
    qprob = torch.tensor(np.repeat(pb.mesh.elem_problem.astype(np.int64),
                                   [(2 * int(W) + 1) ** 3 for W in pb.mesh.elem_W]), device=dev)
    th = th0.clone().requires_grad_(True)
    a, ga = fld(th)
    u = Solve.apply(f, a, ga, m, None, 1e-11, api.FP64, api.FP64, 1e-8)
    J = torch.zeros(2, dtype=torch.float64, device=dev).index_add(0, qprob, w * (PointValues.apply(u, m)[0] - ut) ** 2)
    J.sum().backward()
    g = th.grad.detach()
    u0 = u.detach()
    fl = torch.empty(1, 5, m.nquad, dtype=torch.float64, device=dev)
    m.eval_fields(u0, fl)
    v0 = fl[0, 0].clone()

    def correction(theta):
        aa, gg = fld(theta)
        m.set_data(f=f, a=aa, grad_a=gg)
        b = torch.empty_like(u0)
        m.get_rhs(b)
        r = torch.empty_like(u0)
        m.apply_operator(u0, r)
        m.set_rhs(b - r)
        d = torch.zeros_like(u0)
        assert m.pcg_solve(d, tol=1e-11, prec=api.FP64, max_iter=60000)["status"] == 0
        return d

    h = 1e-4
    for idx in [(1, 0, 0), (0, 2, 1), (3, 1, 2)]:
        tp, tm = th0.clone(), th0.clone()
        tp[(slice(None),) + idx] += h
        tm[(slice(None),) + idx] -= h
        dp, dm = correction(tp), correction(tm)
        fa, fb = torch.empty_like(fl), torch.empty_like(fl)
        m.eval_fields(dp - dm, fa)
        m.eval_fields(dp + dm, fb)
        dJ = torch.zeros(2, dtype=torch.float64, device=dev).index_add(
            0, qprob, w * fa[0, 0] * (2 * (v0 - ut) + fb[0, 0]))
        fd = (dJ / (2 * h)).cpu().numpy()
        gi = g[(slice(None),) + idx].cpu().numpy()
        for p in range(2):
            scale = max(abs(fd[p]), 1e-3 * float(g[p].abs().max()))
            assert abs(gi[p] - fd[p]) <= 1e-6 * scale, (idx, p, gi[p], fd[p])
    m.close()
