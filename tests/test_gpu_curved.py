"""Curved regular elements on the GPU (HPSE_COORD_CURVED: the volume term
through the maps' first and second derivatives in k_apply_gen, the face terms
on each face's (2 max(W, W') + 1)-point grid in k_face_curved), against the
oracle's CurvedDiscretisation.

* Affine maps of a box mesh (the curved path must give the box operator) and
  the L-shaped prism's regular region (six polar-blend sectors around the
  re-entrant edge, Dirichlet data w = r^(2/3) sin(2 theta'/3)) with uniform
  degree and with degrees alternating 2 | 3 from sector to sector: operator
  apply (FP64 within 1e-12, FP32 within 2e-5 of max|y|), right-hand side
  (1e-12).
* Solves (element-block preconditioner, FP32 applies with FP64 refinement) on
  the L-prism sectors against the oracle's dense solution: the oracle's own
  residual of the GPU solution; the relative H^1 error of the GPU solution (by
  the oracle) decays from W = 2 to W = 3 and stays within 1e-6 of the error of
  the oracle's own solution.
* The library's H^1 norm on curved elements (through K and |J| per point):
  against the exact solution and between two discrete solutions, within 1e-10
  of the oracle's (the same (2W+1)^3 GLL rule, CurvedDiscretisation.h1_parts_gll).
* A map with a negative Jacobian is refused (HPSE_ERR_INVALID_ARG).
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle.curved import CurvedDiscretisation, CurvedMesh, CurvedProblem

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -53


@pytest.fixture(scope="module")
def api():
    from paper_1110_2316_gb300.build import build
    build()
    from paper_1110_2316_gb300 import api as A
    return A


def _sine(x, y, z):
    return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


def _box_case():
    desc = wl.box_mesh((2, 1, 1), lo=(0.0, 0.0, 0.0), hi=(1.0, 0.5, 0.7), W=3)
    maps, Ws, nbr = wl.curved_mesh_of_boxes(desc)
    f = lambda x, y, z: 3 * np.pi ** 2 * _sine(x, y, z)  # noqa: E731
    return maps, np.asarray(Ws), np.asarray(nbr), f, _sine, None, None


def _lprism_case(Ws):
    maps, W0, nbr, u, gu, f = wl.lprism_regular(2)
    return maps, np.asarray(Ws, dtype=np.int32), nbr, f, u, u, gu


CASES = {
    "affine_box_W3": _box_case,
    "lprism_W2": lambda: _lprism_case([2] * 6),
    "lprism_W3": lambda: _lprism_case([3] * 6),
    "lprism_2_3": lambda: _lprism_case([2, 3, 2, 3, 2, 3]),
}


def _setup(api, case, n_rhs=1):
    maps, Ws, nbr, f, g, u, gu = case
    desc = wl.CurvedMeshDesc(maps, Ws, nbr)
    m = api.Mesh(desc, n_rhs=n_rhs, coef_kind=api.COEF_LAPLACE)
    vol, face, xv, xf = api.curved_geometry_arrays(m, maps)
    m.set_geometry(vol, face)
    m.set_data(**api.curved_data_arrays(m, xv, xf, [f] * n_rhs, [g] * n_rhs))
    d = CurvedDiscretisation(CurvedProblem(CurvedMesh(maps, Ws, nbr), f, g, u, gu))
    return m, d


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_curved_apply_matches_oracle(api, name, prec, tol):
    m, d = _setup(api, CASES[name]())
    U = np.random.default_rng(4).standard_normal(d.ndof)
    dt = torch.float64 if prec == "fp64" else torch.float32
    u = torch.tensor(U, dtype=dt, device="cuda")
    y = torch.empty_like(u)
    m.apply_operator(u, y)
    ref = d.apply_A(U)
    err = np.abs(y.double().cpu().numpy() - ref).max() / np.abs(ref).max()
    print(name, prec, "apply rel err", err)
    assert err <= tol, (name, err)
    m.close()


@pytest.mark.parametrize("name", list(CASES))
def test_curved_rhs_matches_oracle(api, name):
    m, d = _setup(api, CASES[name](), n_rhs=2)
    b = torch.empty(2 * m.ndof, dtype=torch.float64, device="cuda")
    m.get_rhs(b)
    B = b.cpu().numpy().reshape(2, m.ndof)
    ref = d.rhs_b()
    for r in range(2):
        err = np.abs(B[r] - ref).max() / np.abs(ref).max()
        assert err <= 1e-12, (name, r, err)
    m.close()


def test_curved_solve_and_h1_error(api):
    errs = {}
    for W in (2, 3):
        m, d = _setup(api, _lprism_case([W] * 6))
        A = d.dense_A()
        b = d.rhs_b()
        xo = np.linalg.solve(A, b)
        m.setup_block_preconditioner()
        x = torch.zeros(m.ndof, dtype=torch.float64, device="cuda")
        rep = m.pcg_solve(x, tol=1e-11, prec=api.FP32, max_iter=200000)
        assert rep["status"] == 0 and rep["rel_residual"] <= 1e-11, rep
        X = x.cpu().numpy()
        res = np.linalg.norm(b - A @ X) / np.linalg.norm(b)
        assert res <= 1.5e-11 + 32 * EPS64 * np.linalg.norm(A, 2) * np.linalg.norm(X) / np.linalg.norm(b), res
        errs[W] = d.h1_error_exact(X, nq=12)
        assert abs(errs[W] - d.h1_error_exact(xo, nq=12)) <= 1e-6 * errs[W], W
        m.close()
    print("H1 errors", errs)
    assert errs[3] < 0.5 * errs[2], errs


def test_curved_h1_norm_matches_oracle(api):
    maps, Ws, nbr, f, g, u, gu = _lprism_case([2, 3, 2, 3, 2, 3])
    desc = wl.CurvedMeshDesc(maps, Ws, nbr)
    m = api.Mesh(desc, n_rhs=1, coef_kind=api.COEF_LAPLACE)
    vol, face, xv, xf = api.curved_geometry_arrays(m, maps)
    m.set_geometry(vol, face)
    m.set_data(**api.curved_data_arrays(m, xv, xf, [f], [g]))
    d = CurvedDiscretisation(CurvedProblem(CurvedMesh(maps, Ws, nbr), f, g, u, gu))
    rng = np.random.default_rng(12)
    U = d.nodal_interpolant(u) + 1e-3 * rng.standard_normal(d.ndof)
    vq = torch.tensor(u(xv[:, 0], xv[:, 1], xv[:, 2]), device="cuda")
    gq = torch.tensor(np.concatenate([np.asarray(c) * np.ones(len(xv)) for c in gu(xv[:, 0], xv[:, 1], xv[:, 2])]),
                      device="cuda")
    h = m.h1_error(torch.tensor(U, device="cuda"), vq=vq, gq=gq)
    ref = d.h1_parts_gll(U)
    assert h[0, 0] == pytest.approx(ref[0], rel=1e-10) and h[0, 1] == pytest.approx(ref[1], rel=1e-10)
    # two discrete solutions: the oracle's exact data replaced by the second one
    V = d.nodal_interpolant(u)
    h2 = m.h1_error(torch.tensor(U, device="cuda"), ref=torch.tensor(V, device="cuda"))
    err, nrm = 0.0, 0.0
    for e in range(d.E):
        from oracle.functional import eval_tensor, tables
        B0, B1 = tables(d.W[e])["B"][:2]
        wq = tables(d.W[e])["wq"]
        _, K, det, _, _ = d.vol_geom(e)
        wt = wq[:, None, None] * wq[None, :, None] * wq[None, None, :] * det
        for blk, acc in ((d.block(U, e) - d.block(V, e), "err"), (d.block(V, e), "nrm")):
            v = eval_tensor(blk, B0, B0, B0)
            va = [eval_tensor(blk, *[B1 if b == a else B0 for b in range(3)]) for a in range(3)]
            val = v * v + sum(sum(K[..., a, i] * va[a] for a in range(3)) ** 2 for i in range(3))
            if acc == "err":
                err += float(np.sum(wt * val))
            else:
                nrm += float(np.sum(wt * val))
    assert h2[0, 0] == pytest.approx(err, rel=1e-10) and h2[0, 1] == pytest.approx(nrm, rel=1e-10)
    m.close()


def test_negative_jacobian_is_refused(api):
    from paper_1110_2316_gb300._lib import HpseError
    maps, Ws, nbr, f, g, _, _ = _box_case()
    flip = maps[0]

    def mirrored(l1, l2, l3):
        x, Dx, D2x = flip(-l1, l2, l3)
        Dx = Dx.copy()
        Dx[:, 0] = -Dx[:, 0]
        return x, Dx, D2x
    maps = [mirrored] + list(maps[1:])
    desc = wl.CurvedMeshDesc(maps, Ws, nbr)
    m = api.Mesh(desc, n_rhs=1, coef_kind=api.COEF_LAPLACE)
    vol, face, _, _ = api.curved_geometry_arrays(m, maps)
    with pytest.raises(HpseError) as ei:
        m.set_geometry(vol, face)
    assert ei.value.status == 1
    m.close()
