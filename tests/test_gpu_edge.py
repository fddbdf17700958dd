"""Edge-neighbourhood elements on the GPU (eq. 4.7 in modified coordinates)
against the oracle: operator, right-hand side, element-block preconditioner
with the corner blocks, PCG solutions; and the H^1 error of Table 6.18's
problem computed from GPU solutions.

Tolerances: FP64 applies 1e-12 of max|y| (as for box meshes); FP32 applies
2e-5 of max|y| (W <= 5: the FP32 unit roundoff times the cancellation of the
second-derivative matrices); solutions: relative difference <= kappa(A) x
the stopping residual, with kappa(A) from the dense oracle operator.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle.edge import EdgeDiscretisation

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -53


@pytest.fixture(scope="module")
def api():
    from paper_1110_2316_gb300.build import build
    build()
    from paper_1110_2316_gb300 import api as A
    return A


def _problem(N, W, I=1, J=1):
    base = wl.edge_laplace_singular(N=N, W=W)
    return wl.EdgeProblem(wl.edge_mesh(N, W, I=I, J=J), base.f, base.g, base.u_exact, base.grad_exact)


def _mesh(api, pb, n_rhs=1):
    m = api.Mesh(pb.mesh, n_rhs=n_rhs, coef_kind=api.COEF_LAPLACE)
    m.set_data(**api.problem_data_arrays(m, pb))
    return m


@pytest.mark.parametrize("N,W,I,J", [(3, 3, 1, 1), (2, 4, 2, 2), (3, 2, 2, 1)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_edge_apply_matches_oracle(api, N, W, I, J, prec):
    pb = _problem(N, W, I, J)
    d = EdgeDiscretisation(pb)
    m = _mesh(api, pb)
    assert m.ndof == d.ndof
    U = wl.random_dofs(d.ndof, seed=3)
    yo = d.apply_A(U)
    dt = torch.float64 if prec == "fp64" else torch.float32
    u = torch.tensor(U, dtype=dt, device="cuda")
    y = torch.empty_like(u)
    m.apply_operator(u, y)
    err = np.abs(y.double().cpu().numpy() - yo).max() / np.abs(yo).max()
    assert err <= (1e-12 if prec == "fp64" else 2e-5), err
    m.close()


def test_edge_rhs_matches_oracle(api):
    pb = _problem(2, 3, 2, 2)
    d = EdgeDiscretisation(pb)
    m = _mesh(api, pb)
    b = torch.empty(m.ndof, dtype=torch.float64, device="cuda")
    m.get_rhs(b)
    bo = d.rhs_b()
    assert np.abs(b.cpu().numpy() - bo).max() <= 1e-12 * np.abs(bo).max()
    m.close()


def test_edge_block_preconditioner_matches_oracle(api):
    pb = _problem(2, 3, 2, 1)
    d = EdgeDiscretisation(pb)
    A = d.dense_A()
    m = _mesh(api, pb)
    m.setup_block_preconditioner()
    r = wl.random_dofs(d.ndof, seed=9)
    z = torch.empty(d.ndof, dtype=torch.float64, device="cuda")
    m.apply_preconditioner(torch.tensor(r, device="cuda"), z)
    z = z.cpu().numpy()
    blocks = [slice(d.off[e], d.off[e + 1]) for e in range(d.E)]
    blocks += [slice(d.coff[c], d.coff[c] + d.Wc[c] + 1) for c in range(d.C)]
    for sl in blocks:
        B = A[sl, sl]
        zo = np.linalg.solve(B, r[sl])
        n = B.shape[0]
        # n eps kappa for the factorisation, plus the fixed roundings of z = X^T (X r)
        assert np.linalg.norm(z[sl] - zo) <= (n + 4) * EPS64 * np.linalg.cond(B) * np.linalg.norm(zo)
    m.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("precond", ["separable", "block"])
def test_edge_solve_matches_oracle(api, prec, precond):
    pb = _problem(3, 3)
    d = EdgeDiscretisation(pb)
    A = d.dense_A()
    b = d.rhs_b()
    xo = np.linalg.solve(A, b)
    m = _mesh(api, pb)
    if precond == "block":
        m.setup_block_preconditioner()
    x = torch.zeros(m.ndof, dtype=torch.float64, device="cuda")
    rep = m.pcg_solve(x, tol=1e-11, prec=api.FP64 if prec == "fp64" else api.FP32, max_iter=200000)
    assert rep["status"] == 0 and rep["rel_residual"] <= 1e-11
    kA = np.linalg.cond(A)
    # measured kappa(A) of this case is 1e3..1e5: the bound below stays under 2e-6
    assert kA * 2e-11 <= 2e-6, kA
    X = x.cpu().numpy()
    bo = b
    # the oracle's FP64 residual of the GPU solution: the stopping rule 1e-11 plus
    # the rounding of b - A x (32 eps ||A|| ||x||)
    res = np.linalg.norm(bo - A @ X) / np.linalg.norm(bo)
    assert res <= 1.5e-11 + 32 * 2.0 ** -53 * np.linalg.norm(A, 2) * np.linalg.norm(X) / np.linalg.norm(bo), (res, kA)
    assert np.linalg.norm(X - xo) <= kA * 2e-11 * np.linalg.norm(xo), kA
    m.close()


def test_table_6_18_h1_error_from_gpu_solutions(api):
    # relative H^1 error (%) of Table 6.18 at W = 2..5: 0.4645, 0.1314, 0.0402, 0.0124;
    # layers N = 2W + 4
    table = {2: 0.464542e-2, 3: 0.131359e-2, 4: 0.402204e-3, 5: 0.123974e-3}
    errs = {}
    for W in (2, 3, 4, 5):
        pb = wl.edge_laplace_singular(N=2 * W + 4, W=W)
        d = EdgeDiscretisation(pb)
        m = _mesh(api, pb)
        m.setup_block_preconditioner()
        x = torch.zeros(m.ndof, dtype=torch.float64, device="cuda")
        rep = m.pcg_solve(x, tol=1e-10, prec=api.FP32, max_iter=200000)
        assert rep["status"] == 0
        err, nrm = d.h1_error_exact(x.cpu().numpy())
        errs[W] = np.sqrt(err / nrm)
        m.close()
    for W in (2, 3, 4, 5):
        assert table[W] / 5 < errs[W] < table[W] * 5, (W, errs[W], table[W])
    for W in (3, 4, 5):
        assert errs[W] < 0.5 * errs[W - 1], errs


def test_edge_separable_preconditioner_matches_oracle(api):
    # C* form (eq. 5.30) on the finite elements, exact blocks on the corner sets;
    # two independent eigen-decompositions (scipy, the library's Jacobi) agree
    # to O(eps kappa) with kappa = max sigma / min sigma of each element
    from oracle.edge import apply_separable_preconditioner
    from oracle.precond import cstar_eigen_z, eigenbasis
    pb = _problem(3, 4, 2, 1)
    d = EdgeDiscretisation(pb)
    m = _mesh(api, pb)
    r = wl.random_dofs(d.ndof, seed=4)
    zo = apply_separable_preconditioner(d, r)
    z = torch.empty(d.ndof, dtype=torch.float64, device="cuda")
    m.apply_preconditioner(torch.tensor(r, device="cuda"), z)
    z = z.cpu().numpy()
    mu, _ = eigenbasis(4)
    for e in range(d.E):
        nu, _ = cstar_eigen_z(4, float(np.exp(d.mesh.elem_hi[e, 0])))
        kappa = (2 * mu.max() + nu.max() + 1) / (2 * mu.min() + nu.min() + 1)
        sl = slice(d.off[e], d.off[e + 1])
        assert np.abs(z[sl] - zo[sl]).max() <= max(1e-12, 8 * EPS64 * 2 * kappa) * np.abs(zo[sl]).max(), e
    sl = slice(int(d.coff[0]), d.ndof)
    assert np.abs(z[sl] - zo[sl]).max() <= 1e-10 * np.abs(zo[sl]).max()
    m.close()


def test_edge_h1_norm_matches_oracle(api):
    # difference of two discrete solutions: element terms with the (2W+1)^3 GLL
    # rule in modified coordinates, corner sets in physical coordinates; both
    # sides sum the same terms in FP64 (1e-12 relative)
    from oracle.edge import h1_diff
    pb = _problem(3, 3, 2, 2)
    d = EdgeDiscretisation(pb)
    m = _mesh(api, pb)
    rng = np.random.default_rng(5)
    U, V = rng.standard_normal(d.ndof), rng.standard_normal(d.ndof)
    h = m.h1_error(torch.tensor(U, device="cuda"), ref=torch.tensor(V, device="cuda"))
    e, n = h1_diff(d, U, V)
    assert h[0, 0] == pytest.approx(e, rel=1e-12) and h[0, 1] == pytest.approx(n, rel=1e-12)
    m.close()


def test_edge_batch_equals_individual_solves(api):
    # uneven degrees in one launch: the batched solution of each problem equals
    # its own solve (per-problem PCG scalars; same iteration path)
    Ws = (2, 4, 3)
    pb = wl.edge_batch(Ws)
    m = _mesh(api, pb)
    m.setup_block_preconditioner()
    x = torch.zeros(m.ndof, dtype=torch.float64, device="cuda")
    assert m.pcg_solve(x, tol=1e-11, prec=api.FP64, max_iter=200000)["status"] == 0
    parts = []
    for W in Ws:
        one = wl.edge_batch([W])
        mi = _mesh(api, one)
        mi.setup_block_preconditioner()
        xi = torch.zeros(mi.ndof, dtype=torch.float64, device="cuda")
        assert mi.pcg_solve(xi, tol=1e-11, prec=api.FP64, max_iter=200000)["status"] == 0
        parts.append((one, xi.cpu().numpy()))
        mi.close()
    # reassemble: elements of the problems in order, then the corner sets in order
    xb = x.cpu().numpy()
    el, co = [], []
    for one, xi in parts:
        d = EdgeDiscretisation(one)
        el.append(xi[:d.off[-1]])
        co.append(xi[d.off[-1]:])
    ref = np.concatenate(el + co)
    assert np.linalg.norm(xb - ref) <= 1e-8 * np.linalg.norm(ref)
    m.close()
