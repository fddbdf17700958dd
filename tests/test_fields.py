"""The differentiable Legendre-log coefficient field (torch, CPU) against
the seeded host sampling of the same field (workloads), and its autograd
derivative against the closed form of d a / d theta."""
import numpy as np
import torch

import workloads as wl
from oracle.functional import Discretisation
from paper_1110_2316_gb300.fields import LegendreLogField


def _axes(disc):
    return np.concatenate([np.concatenate(disc.qpoints(e)) for e in range(disc.E)])


def test_field_matches_host_sampling():
    parts = [wl.lognormal_coef_problem(W, p, n=2) for p, W in enumerate((2, 3, 2))]
    pb = wl.batch_problems(parts)
    disc = Discretisation(pb)
    fld = LegendreLogField(_axes(disc), pb.mesh.elem_W, pb.mesh.elem_problem, device="cpu")
    theta = torch.tensor(np.stack([p.meta["theta"] for p in parts]))
    a, ga = fld(theta)
    o = 0
    for e in range(disc.E):
        xs, ys, zs = disc.qpoints(e)
        pe = parts[int(pb.mesh.elem_problem[e])]
        n = len(xs) ** 3
        want_a = np.broadcast_to(pe.a(xs, ys, zs), (len(zs), len(ys), len(xs))).ravel()
        np.testing.assert_allclose(a[o:o + n].numpy(), want_a, rtol=1e-13)
        for k, gk in enumerate(pe.grad_a(xs, ys, zs)):
            np.testing.assert_allclose(ga[k, o:o + n].numpy(), np.broadcast_to(gk, (len(zs), len(ys), len(xs))).ravel(),
                                       rtol=1e-12, atol=1e-12)
        o += n


def test_field_theta_derivative():
    # d a_q / d theta_ijk = a_q L_i(x) L_j(y) L_k(z): check one entry through autograd
    parts = [wl.lognormal_coef_problem(2, 0, n=1)]
    pb = wl.batch_problems(parts)
    disc = Discretisation(pb)
    fld = LegendreLogField(_axes(disc), pb.mesh.elem_W, pb.mesh.elem_problem, device="cpu")
    theta = torch.tensor(parts[0].meta["theta"][None]).requires_grad_(True)
    a, _ = fld(theta)
    q = 7
    a[q].backward()
    xs, ys, zs = disc.qpoints(0)
    Q = len(xs)
    x, y, z = xs[q % Q], ys[(q // Q) % Q], zs[q // (Q * Q)]
    from numpy.polynomial import legendre as npl
    Lv = [[npl.legval(2 * c - 1, np.eye(4)[i]) for i in range(4)] for c in (x, y, z)]
    want = float(a[q]) * np.einsum("i,j,k->ijk", *Lv)
    np.testing.assert_allclose(theta.grad[0].numpy(), want, rtol=1e-12, atol=1e-15)
