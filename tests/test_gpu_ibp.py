"""The volume transpose in integration-by-parts form on the GPU
(hpse_apply_transpose_ibp, eq. 5.45-5.48), against the oracle and the direct
transpose.

* FP64 against the oracle's transpose of the residual map (the Discretisation's
  L_apply_T of sqrt(w J) z, element by element) on Laplacian and
  -div(a grad u) box meshes, two right-hand sides, a two-degree batch, and the
  Laplacian at W = 10: within 1e-12 of max|y|, the bound of the direct
  transpose (measured 3e-15 to 2e-14 for both forms: the D_Q^2 entries grow
  like W^4, but the integration-by-parts form's volume and face terms are of
  the result's size, so no cancellation amplifies the rounding).
* FP64 against the direct transpose at W = 8 and W = 10 (Laplacian).
* FP32 against the FP64 direct transpose within 1e-4 of max|y|: FP32 unit
  roundoff 6e-8 times the (2W+1)-term sums of three stages and the D_Q^2
  contraction (measured 3e-6 at W = 8 in the bench).
* Refusals: the general operator (HPSE_ERR_INVALID_ARG) and -div(a grad u)
  in FP64 at W = 10 (its shared-memory layout, three (2W+1)^3 arrays, does
  not fit; HPSE_ERR_DEGREE).
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle.functional import Discretisation

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


def _two(pb):
    return wl.Problem(pb.mesh, pb.f * 2, pb.g * 2, pb.a, pb.grad_a)


def _oracle_T(disc, Z):
    Q = [2 * w + 1 for w in disc.W]
    o, out = 0, []
    for e in range(disc.E):
        n = Q[e] ** 3
        zb = Z[o:o + n].reshape(Q[e], Q[e], Q[e])
        out.append(disc.L_apply_T(np.sqrt(disc.vol_weight(e)) * zb, e).ravel())
        o += n
    return np.concatenate(out)


CASES = {
    "laplace_aniso_W5": lambda: wl.poisson_sine(n=(2, 1, 2), W=5),
    "varcoef_W4": lambda: wl.varcoef_manufactured(n=(2, 2, 1), W=4),
    "varcoef_batch_W3_W7": lambda: wl.batch_problems([wl.varcoef_manufactured(n=(2, 1, 1), W=3),
                                                      wl.varcoef_manufactured(n=(1, 1, 2), W=7)]),
    "laplace_W10": lambda: wl.poisson_sine(n=(1, 1, 2), W=10),
}


@pytest.mark.parametrize("name", list(CASES))
def test_ibp_transpose_matches_oracle(api, name):
    pb = _two(CASES[name]())
    disc = Discretisation(pb)
    m = _mesh(api, pb)
    rng = np.random.default_rng(3)
    Z = rng.standard_normal((2, m.nquad))
    y = torch.empty(2 * m.ndof, dtype=torch.float64, device="cuda")
    m.apply_transpose_ibp(torch.tensor(Z, device="cuda"), y)
    Y = y.cpu().numpy().reshape(2, m.ndof)
    yd = torch.empty_like(y)
    m.apply_transpose(torch.tensor(Z, device="cuda"), yd)
    Yd = yd.cpu().numpy().reshape(2, m.ndof)
    for r in range(2):
        ref = _oracle_T(disc, Z[r])
        err = np.abs(Y[r] - ref).max() / np.abs(ref).max()
        print(name, r, "ibp vs oracle", err, "direct vs oracle", np.abs(Yd[r] - ref).max() / np.abs(ref).max())
        assert err <= 1e-12, (name, r, err)
    m.close()


@pytest.mark.parametrize("W", [8, 10])
def test_ibp_equals_direct_transpose_fp64(api, W):
    pb = wl.poisson_sine(n=(2, 2, 2), W=W)
    m = _mesh(api, pb)
    z = torch.tensor(np.random.default_rng(W).standard_normal(m.nquad), device="cuda")
    y1 = torch.empty(m.ndof, dtype=torch.float64, device="cuda")
    y2 = torch.empty_like(y1)
    m.apply_transpose(z, y1)
    m.apply_transpose_ibp(z, y2)
    err = float((y1 - y2).abs().max() / y1.abs().max())
    print("W", W, "ibp vs direct", err)
    assert err <= 1e-12
    m.close()


@pytest.mark.parametrize("name", ["laplace_aniso_W5", "varcoef_W4"])
def test_ibp_fp32(api, name):
    pb = CASES[name]()
    m = _mesh(api, pb)
    Z = np.random.default_rng(9).standard_normal(m.nquad)
    y64 = torch.empty(m.ndof, dtype=torch.float64, device="cuda")
    m.apply_transpose(torch.tensor(Z, device="cuda"), y64)
    y32 = torch.empty(m.ndof, dtype=torch.float32, device="cuda")
    m.apply_transpose_ibp(torch.tensor(Z, dtype=torch.float32, device="cuda"), y32)
    err = float((y32.double() - y64).abs().max() / y64.abs().max())
    print(name, "fp32 ibp vs fp64 direct", err)
    assert err <= 1e-4
    m.close()


def test_ibp_refusals(api):
    from paper_1110_2316_gb300._lib import HpseError
    pb = wl.nonsym_mixed(n=2, W=2)
    m = api.Mesh(pb.mesh, coef_kind=api.COEF_GENERAL)
    m.set_data(**api.problem_data_arrays(m, pb))
    z = torch.zeros(m.nquad, dtype=torch.float64, device="cuda")
    y = torch.empty(m.ndof, dtype=torch.float64, device="cuda")
    with pytest.raises(HpseError) as ei:
        m.apply_transpose_ibp(z, y)
    assert ei.value.status == 1
    m.close()
    pb = wl.varcoef_manufactured(n=(1, 1, 1), W=10)
    m = _mesh(api, pb)
    z = torch.zeros(m.nquad, dtype=torch.float64, device="cuda")
    y = torch.empty(m.ndof, dtype=torch.float64, device="cuda")
    with pytest.raises(HpseError) as ei:
        m.apply_transpose_ibp(z, y)
    assert ei.value.status == 3
    m.close()
