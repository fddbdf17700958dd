"""GPU parity of batched, uneven-degree launches: many independent problems of
different degree W in one handle (per-degree groups launched concurrently).

* the batched operator equals the oracle's on every element (1e-12);
* the batched solve of each problem equals the solve of that problem alone
  (relative H1 difference 1e-8) and the oracle's solution for a small one.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle.functional import Discretisation
from oracle.h1 import h1_rel_diff
from oracle.pcg import pcg
from oracle.precond import apply_Cinv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1110_2316_gb300.build import build
    build()
    from paper_1110_2316_gb300 import api as A
    return A


def _batch():
    parts = [wl.lognormal_coef_problem(W, p, n=(2, 1, 1) if W > 4 else (2, 2, 1))
             for p, W in enumerate((3, 6, 4, 2))]
    return parts, wl.batch_problems(parts)


def _mesh(api, pb):
    m = api.Mesh(pb.mesh, n_rhs=pb.n_rhs, coef_kind=api.COEF_SCALAR)
    m.set_data(**api.problem_data_arrays(m, pb))
    return m


def test_batched_apply_matches_oracle(api):
    parts, pb = _batch()
    m = _mesh(api, pb)
    disc = Discretisation(pb)
    U = wl.random_dofs(m.ndof, seed=21)
    u = torch.tensor(U, device="cuda")
    y = torch.empty_like(u)
    m.apply_operator(u, y)
    ref = disc.apply_A(U)
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_solve_equals_individual_solves(api, prec):
    parts, pb = _batch()
    m = _mesh(api, pb)
    p = api.FP64 if prec == "fp64" else api.FP32
    x = torch.zeros(m.ndof, dtype=torch.float64, device="cuda")
    rep = m.pcg_solve(x, tol=1e-10, prec=p)
    assert rep["status"] == 0 and rep["rel_residual"] <= 1e-10
    X = x.cpu().numpy()
    off = 0
    for k, part in enumerate(parts):
        mk = _mesh(api, part)
        xk = torch.zeros(mk.ndof, dtype=torch.float64, device="cuda")
        mk.pcg_solve(xk, tol=1e-10, prec=api.FP64)
        dk = Discretisation(part)
        blk = X[off:off + mk.ndof]
        assert h1_rel_diff(dk, blk, xk.cpu().numpy()) <= 1e-8, k
        if k == 0:
            xo, _, _ = pcg(dk.apply_A, lambda r: apply_Cinv(dk, r), dk.rhs_b(), tol=1e-10)
            assert h1_rel_diff(dk, blk, xo) <= 1e-8
        off += mk.ndof
