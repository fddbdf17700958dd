"""GPU vs oracle at the full size of the variable-coefficient benchmark:
-div(a grad u) = f on [0,1]^3, 8 x 8 x 8 elements, W = 8, 64 right-hand sides
in one launch (the launch configuration the benchmark times: 32,768 CTAs per
operator apply, element offsets into 64 right-hand-side slabs).

* Operator apply, FP64 and FP32, every element of right-hand sides 0 and 63
  taken out of the 64-RHS launch, element by element against the oracle's
  apply: 1e-12 x max|y| (FP64) and 2e-5 x max|y| (FP32: unit roundoff 6e-8
  times the cancellation of the O(W^4) second-derivative matrix entries).
* Right-hand side b = S^T M d of right-hand sides 0 and 63: 1e-12 x max|b|.
* The mixed-precision solve of the whole batch (FP32 applies, FP64 refinement,
  block preconditioner) to ||b - A x|| <= 1e-10 ||b||: for right-hand sides
  0-3 the oracle recomputes b and A x in FP64 and the relative residual must
  be <= 1.1e-10 (the stopping rule of Section 6.1 plus the 1e-12 apply and
  right-hand-side parity); the relative H^1 difference to an FP64 GPU solve
  of the same four right-hand sides, measured by the oracle's H^1 norm, must be
  <= 1e-8.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle.functional import Discretisation
from oracle.h1 import h1_rel_diff

pytestmark = pytest.mark.gpu

N_EL, W, N_RHS = 8, 8, 64
SAMPLE_RHS = (0, 63)


@pytest.fixture(scope="module")
def api():
    from paper_1110_2316_gb300.build import build
    build()
    from paper_1110_2316_gb300 import api as A
    return A


@pytest.fixture(scope="module")
def full(api):
    pb = wl.varcoef_random_rhs(n=N_EL, W=W, n_rhs=N_RHS, seed0=20260)
    m = api.Mesh(pb.mesh, n_rhs=N_RHS, coef_kind=api.COEF_SCALAR)
    data = api.problem_data_arrays(m, pb)
    m.set_data(**data)
    disc = Discretisation(pb)
    yield pb, m, data, disc
    m.close()


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_fullsize_apply_matches_oracle(api, full, prec, tol):
    _, m, _, disc = full
    n = m.ndof
    U = wl.random_dofs(N_RHS * n, seed=2026).reshape(N_RHS, n)
    dt = torch.float64 if prec == "fp64" else torch.float32
    u = torch.tensor(U, dtype=dt, device="cuda")
    y = torch.full_like(u, float("nan"))
    m.apply_operator(u.reshape(-1), y.reshape(-1))
    torch.cuda.synchronize()
    assert torch.isfinite(y).all()
    y = y.double().cpu().numpy()
    for r in SAMPLE_RHS:
        Ur = U[r].astype(np.float32).astype(np.float64) if prec == "fp32" else U[r]
        ref = disc.apply_A(Ur)
        scale = np.abs(ref).max()
        err = [np.abs(y[r, disc.off[e]:disc.off[e + 1]] - ref[disc.off[e]:disc.off[e + 1]]).max() / scale
               for e in range(disc.E)]
        assert max(err) <= tol, (r, int(np.argmax(err)), max(err))


def test_fullsize_rhs_matches_oracle(api, full):
    _, m, _, disc = full
    b = torch.empty(N_RHS * m.ndof, dtype=torch.float64, device="cuda")
    m.get_rhs(b)
    b = b.cpu().numpy().reshape(N_RHS, m.ndof)
    for r in SAMPLE_RHS:
        ref = disc.rhs_b(r)
        assert _rel(b[r], ref) <= 1e-12, r


def test_fullsize_mixed_solve_oracle_residual(api, full):
    pb, m, data, disc = full
    n = m.ndof
    m.setup_block_preconditioner()
    x = torch.zeros(N_RHS * n, dtype=torch.float64, device="cuda")
    rep = m.pcg_solve(x, tol=1e-10, prec=api.FP32, max_iter=60000)
    assert rep["status"] == 0 and rep["rel_residual"] <= 1e-10
    X = x.cpu().numpy().reshape(N_RHS, n)
    k = 4
    sub = wl.Problem(pb.mesh, pb.f[:k], pb.g[:k], pb.a, pb.grad_a)
    m4 = api.Mesh(sub.mesh, n_rhs=k, coef_kind=api.COEF_SCALAR)
    m4.set_data(f=data["f"][:k], a=data["a"], grad_a=data["grad_a"])
    m4.setup_block_preconditioner()
    x64 = torch.zeros(k * n, dtype=torch.float64, device="cuda")
    rep64 = m4.pcg_solve(x64, tol=1e-10, prec=api.FP64, max_iter=60000)
    assert rep64["status"] == 0
    X64 = x64.cpu().numpy().reshape(k, n)
    m4.close()
    for r in range(k):
        bo = disc.rhs_b(r)
        res = np.linalg.norm(bo - disc.apply_A(X[r])) / np.linalg.norm(bo)
        assert res <= 1.1e-10, (r, res)
        d = h1_rel_diff(disc, X[r], X64[r])
        assert d <= 1e-8, (r, d)
