"""Element-block preconditioner (hpse_setup_block_preconditioner) against the
oracle's definition z_e = A_ee^{-1} r_e, and PCG with it against the oracle's
Cholesky solution.

Bounds.  FP64: the blocks are probed from the FP64 operator (entrywise error
O(eps |A|)) and factored by Cholesky (backward stable), so the forward error is
bounded by n eps64 kappa(A_ee) (n = (W+1)^3).  FP32: the FP64 factor inverse
X = L^{-1} is rounded to FP32 and z = X^T (X r) is formed in FP32, so
|z32 - z| <= c n eps32 |X|^T |X| |r| componentwise (rounding of X plus the two
length-n products), checked in the 2-norm with c = 2.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle.functional import Discretisation
from oracle.pcg import cholesky_solve
from oracle.precond import apply_block_inverse, block_factors, element_block

pytestmark = pytest.mark.gpu

EPS64, EPS32 = 2.0 ** -53, 2.0 ** -24


@pytest.fixture(scope="module")
def api():
    from paper_1110_2316_gb300.build import build
    build()
    from paper_1110_2316_gb300 import api as A
    return A


def _mesh(api, pb, n_rhs):
    m = api.Mesh(pb.mesh, n_rhs=n_rhs, coef_kind=api.COEF_SCALAR if pb.a is not None else api.COEF_LAPLACE)
    m.set_data(**api.problem_data_arrays(m, pb))
    return m


def _problems():
    return {
        "varcoef": wl.varcoef_manufactured(n=(2, 2, 1), W=3),
        "batch": wl.batch_problems([wl.lognormal_coef_problem(W, p, n=2) for p, W in enumerate((2, 3))]),
    }


@pytest.mark.parametrize("name", ["varcoef", "batch"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_block_apply_matches_oracle(api, name, prec):
    pb = _problems()[name]
    disc = Discretisation(pb)
    m = _mesh(api, pb, 1)
    m.setup_block_preconditioner()
    r = wl.random_dofs(disc.ndof, 5)
    z_o = apply_block_inverse(disc, r)
    dt = torch.float64 if prec == "fp64" else torch.float32
    rt = torch.tensor(r, dtype=dt, device="cuda")
    z = torch.empty_like(rt)
    m.apply_preconditioner(rt, z)
    z = z.double().cpu().numpy()
    for e in range(disc.E):
        s = slice(disc.off[e], disc.off[e + 1])
        B = element_block(disc, e)
        n = B.shape[0]
        if prec == "fp64":
            bound = n * EPS64 * np.linalg.cond(B) * np.linalg.norm(z_o[s])
        else:
            X = np.linalg.inv(np.linalg.cholesky(B))
            bound = 2 * n * EPS32 * np.linalg.norm(np.abs(X).T @ (np.abs(X) @ np.abs(r[s])))
        err = np.linalg.norm(z[s] - z_o[s])
        assert err <= bound, (name, prec, e, err, bound)
    m.close()


def test_one_element_block_inverts_the_operator(api):
    pb = wl.varcoef_manufactured(n=(1, 1, 1), W=4)
    disc = Discretisation(pb)
    m = _mesh(api, pb, 1)
    m.setup_block_preconditioner()
    x = torch.tensor(wl.random_dofs(disc.ndof, 2), device="cuda")
    y, z = torch.empty_like(x), torch.empty_like(x)
    m.apply_operator(x, y)
    m.apply_preconditioner(y, z)
    kappa = np.linalg.cond(element_block(disc, 0))
    n = disc.ndof
    assert float(torch.linalg.norm(z - x)) <= 4 * n * EPS64 * kappa * float(torch.linalg.norm(x))
    m.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_block_pcg_matches_oracle_solution(api, prec):
    pb = wl.varcoef_manufactured(n=(2, 2, 1), W=3)
    disc = Discretisation(pb)
    xo = cholesky_solve(disc.dense_A(), disc.rhs_b())
    m = _mesh(api, pb, 1)
    P = api.FP64 if prec == "fp64" else api.FP32
    x0 = torch.zeros(m.ndof, dtype=torch.float64, device="cuda")
    rep0 = m.pcg_solve(x0, tol=1e-11, prec=P)
    m.setup_block_preconditioner()
    x = torch.zeros_like(x0)
    rep = m.pcg_solve(x, tol=1e-11, prec=P)
    assert rep["status"] == 0 and rep["rel_residual"] <= 1e-11
    assert rep["iterations"] < rep0["iterations"], (rep, rep0)
    # ||x - xo|| <= kappa(A) * 2e-11 ||xo|| is the residual bound, checked with
    # kappa from the dense operator (measured 5.3e4: the bound is 1.1e-6); and
    # the oracle's own FP64 residual of the GPU solution
    A = disc.dense_A()
    kA = np.linalg.cond(A)
    assert kA * 2e-11 <= 2e-6, kA
    X = x.cpu().numpy()
    bo = disc.rhs_b()
    res = np.linalg.norm(bo - A @ X) / np.linalg.norm(bo)
    assert res <= 1.5e-11 + 32 * 2.0 ** -53 * np.linalg.norm(A, 2) * np.linalg.norm(X) / np.linalg.norm(bo), res
    err = np.linalg.norm(X - xo)
    assert err <= kA * 2e-11 * np.linalg.norm(xo), (err, kA)
    # and it agrees with the separable-preconditioner solve
    assert float(torch.linalg.norm(x - x0)) <= kA * 4e-11 * float(torch.linalg.norm(x0))
    m.close()


def test_block_preconditioner_errors(api):
    pb = wl.varcoef_manufactured(n=(1, 1, 1), W=2)
    m = api.Mesh(pb.mesh, n_rhs=1, coef_kind=api.COEF_SCALAR)
    from paper_1110_2316_gb300._lib import HpseError
    with pytest.raises(HpseError):
        m.setup_block_preconditioner()          # no data yet
    m.set_data(**api.problem_data_arrays(m, pb))
    with pytest.raises(HpseError):
        m.select_preconditioner(api.PRECOND_BLOCK)  # not set up
    with pytest.raises(HpseError):
        m.select_preconditioner(7)
    m.setup_block_preconditioner()
    m.select_preconditioner(api.PRECOND_SEPARABLE)
    m.select_preconditioner(api.PRECOND_BLOCK)
    m.close()


@pytest.mark.parametrize("n_rhs", [5, 33, 70])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_block_apply_many_rhs(api, n_rhs, prec):
    # the three tile shapes of the triangular products (1, 2..31 and >= 32
    # right-hand sides), with ragged right-hand-side tiles
    base = wl.varcoef_manufactured(n=(2, 1, 1), W=3)
    pb = wl.Problem(base.mesh, base.f * n_rhs, base.g * n_rhs, base.a, base.grad_a)
    disc = Discretisation(base)
    m = _mesh(api, pb, n_rhs)
    m.setup_block_preconditioner()
    R = wl.random_dofs(n_rhs * disc.ndof, 11).reshape(n_rhs, disc.ndof)
    dt = torch.float64 if prec == "fp64" else torch.float32
    rt = torch.tensor(R.ravel(), dtype=dt, device="cuda")
    z = torch.empty_like(rt)
    m.apply_preconditioner(rt, z)
    z = z.double().cpu().numpy().reshape(n_rhs, disc.ndof)
    blocks = [element_block(disc, e) for e in range(disc.E)]
    Xs = [np.linalg.inv(np.linalg.cholesky(B)) for B in blocks]
    fac = block_factors(disc)
    for k in range(n_rhs):
        zo = apply_block_inverse(disc, R[k], fac)
        for e in range(disc.E):
            s = slice(disc.off[e], disc.off[e + 1])
            n = blocks[e].shape[0]
            if prec == "fp64":
                bound = n * EPS64 * np.linalg.cond(blocks[e]) * np.linalg.norm(zo[s])
            else:
                X = Xs[e]
                bound = 2 * n * EPS32 * np.linalg.norm(np.abs(X).T @ (np.abs(X) @ np.abs(R[k][s])))
            assert np.linalg.norm(z[k][s] - zo[s]) <= bound, (n_rhs, prec, k, e)
    m.close()


@pytest.mark.parametrize("n_rhs", [1, 5, 40])
def test_block_tile_autotuner(api, n_rhs):
    # every tile variant gives the same products (to the FP32 / FP64 rounding of
    # a length-n sum), the autotuner picks a candidate of the rhs count, and
    # the forced variants are honoured
    base = wl.varcoef_manufactured(n=(2, 1, 1), W=3)
    pb = wl.Problem(base.mesh, base.f * n_rhs, base.g * n_rhs, base.a, base.grad_a)
    m = _mesh(api, pb, n_rhs)
    m.setup_block_preconditioner()
    cand = {1: (5, 6, 7), 5: (3, 4), 40: (0, 1, 2, 8)}[n_rhs]
    for prec, dt, tol in ((api.FP64, torch.float64, 1e-13), (api.FP32, torch.float32, 1e-5)):
        v, tile, ms = m.block_tile(3, prec)
        ok = [c for c in cand if prec == api.FP32 or c not in (2, 4, 6, 8)]
        assert v in ok and all(ms[c] > 0 for c in ok), (v, ms)
        r = torch.tensor(wl.random_dofs(n_rhs * m.ndof, 3), dtype=dt, device="cuda")
        outs = []
        for c in ok:
            m.set_block_tile(3, prec, c)
            z = torch.empty_like(r)
            m.apply_preconditioner(r, z)
            outs.append(z.double())
        for z in outs[1:]:
            assert float((z - outs[0]).abs().max()) <= tol * float(outs[0].abs().max())
    from paper_1110_2316_gb300._lib import HpseError
    with pytest.raises(HpseError):
        m.set_block_tile(3, api.FP64, 2)  # FP32-only shape
    with pytest.raises(HpseError):
        m.set_block_tile(3, api.FP64, 8)  # the tensor-core form is FP32 only
    if n_rhs < 32:
        with pytest.raises(HpseError):
            m.set_block_tile(3, api.FP32, 8)  # no tiles built below 32 right-hand sides
    m.close()


@pytest.mark.parametrize("W", [3, 5, 6])
@pytest.mark.parametrize("n_rhs", [33, 70])
def test_block_tensor_core_products(api, W, n_rhs):
    # variant 8: both triangular products on the tensor cores (3xTF32, FP32
    # accumulation); blocks of n = 64, 216, 343 (one to three 128-row tiles, the
    # last one ragged), one or two 64-rhs tiles (70: the second holds 6).  Bound:
    # the FP32 bound of the CUDA-core products (2 n eps32 |X|^T |X| |r| per
    # element) against the exact block solve, and agreement with variant 0.
    base = wl.varcoef_manufactured(n=(2, 1, 1), W=W)
    pb = wl.Problem(base.mesh, base.f * n_rhs, base.g * n_rhs, base.a, base.grad_a)
    disc = Discretisation(base)
    m = _mesh(api, pb, n_rhs)
    m.setup_block_preconditioner()
    R = wl.random_dofs(n_rhs * disc.ndof, 17).reshape(n_rhs, disc.ndof)
    rt = torch.tensor(R.ravel(), dtype=torch.float32, device="cuda")
    outs = {}
    for v in (8, 0):
        m.set_block_tile(W, api.FP32, v)
        z = torch.full_like(rt, float("nan"))
        m.apply_preconditioner(rt, z)
        torch.cuda.synchronize()
        outs[v] = z.double().cpu().numpy().reshape(n_rhs, disc.ndof)
    assert np.isfinite(outs[8]).all()
    blocks = [element_block(disc, e) for e in range(disc.E)]
    Xs = [np.linalg.inv(np.linalg.cholesky(B)) for B in blocks]
    for e in range(disc.E):
        s = slice(disc.off[e], disc.off[e + 1])
        n = blocks[e].shape[0]
        for k in range(n_rhs):
            zo = np.linalg.solve(blocks[e], R[k][s])
            X = Xs[e]
            bound = 2 * n * EPS32 * np.linalg.norm(np.abs(X).T @ (np.abs(X) @ np.abs(R[k][s])))
            assert np.linalg.norm(outs[8][k][s] - zo) <= bound, (W, n_rhs, k, e)
            assert np.linalg.norm(outs[8][k][s] - outs[0][k][s]) <= bound, (W, n_rhs, k, e)
    m.close()
