"""Pins for the H^1 error metric (Section 6.1) and whole-method behaviour.

* ||sin(pi x) sin(pi y) sin(pi z)||_{H^1((0,1)^3)}^2 = (1 + 3 pi^2) / 8 (closed form);
* the error of an interpolant of a degree-<=W polynomial is zero;
* exponential decay of the error in W (Theorem 4.3.1) on the Poisson problem;
* loose comparison with Table 6.2 (iteration counts / errors depend on the basis
  and on face-norm conventions the thesis leaves open).
"""
import math
import os

import numpy as np
import pytest

import workloads as wl
from oracle.functional import Discretisation
from oracle.h1 import h1_error_exact, h1_norm_sq, h1_rel_diff
from oracle.pcg import pcg
from oracle.precond import apply_Cinv

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table6_2_poisson.txt")


def test_h1_norm_closed_form():
    pb = wl.poisson_sine(n=2, W=10)
    d = Discretisation(pb)
    U = d.nodal_interpolant(pb.u_exact[0])
    exact = (1 + 3 * math.pi ** 2) / 8
    assert abs(h1_norm_sq(d, U) - exact) < 1e-7 * exact


def test_h1_error_of_polynomial_interpolant_is_zero():
    pb = wl.polynomial_exact(n=2, W=3)
    d = Discretisation(pb)
    U = d.nodal_interpolant(pb.u_exact[0])
    assert h1_error_exact(d, U) < 1e-13
    assert h1_rel_diff(d, U, U) == 0.0


def _solve(W, lo, hi):
    pb = wl.poisson_sine(n=2, W=W, lo=lo, hi=hi)
    d = Discretisation(pb)
    x, it, rel = pcg(d.apply_A, lambda r: apply_Cinv(d, r), d.rhs_b(), tol=1e-10)
    return it, h1_error_exact(d, x)


def test_exponential_decay_in_W():
    errs = [_solve(W, 0.0, 1.0)[1] for W in (2, 3, 4, 5)]
    for a, b in zip(errs, errs[1:]):
        assert b < a / 3.0, errs
    # log-linear: a straight-line fit explains the data well (Figs. 6.3-6.4)
    Ws = np.array([2, 3, 4, 5.0])
    c = np.polyfit(Ws, np.log(errs), 1)
    resid = np.log(errs) - np.polyval(c, Ws)
    assert np.abs(resid).max() < 1.0 and c[0] < -1.0


def test_table_6_2_loose():
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    ref = {int(r[0]): (int(r[2]), float(r[3]) / 100.0) for r in rows}
    for W in (2, 4):
        it, err = _solve(W, -1.0, 1.0)
        it_ref, err_ref = ref[W]
        assert err_ref / 10 < err < err_ref * 10, (W, err, err_ref)
        assert it_ref / 3 < it < it_ref * 3, (W, it, it_ref)


def _table_6_1_error(W):
    from oracle.pcg import pcg
    from oracle.precond import apply_block_inverse, block_factors
    d = Discretisation(wl.laplace_sinh(n=2, W=W))
    fac = block_factors(d)
    x, _, rel = pcg(d.apply_A, lambda r: apply_block_inverse(d, r, fac), d.rhs_b(), tol=1e-12, maxit=5000)
    assert rel <= 1e-12
    return h1_error_exact(d, x)


def test_table_6_1_w2_w4():
    # relative H^1 error (%) of Table 6.1 (Laplace, Dirichlet data, (0,1)^3 in
    # 2x2x2 elements): 38.0 at W = 2, 2.05 at W = 4; measured 23.6 and 0.430 --
    # the oracle's error falls faster with W than the table's (0.62, 0.21, 0.15
    # of it at W = 2, 4, 6), so the window is (1/10, 5) of the table
    from golden_tables import rel_error
    for W in (2, 4):
        ref = rel_error("table6_1_laplace.txt", W)
        err = _table_6_1_error(W)
        assert ref / 10 < err < ref * 5, (W, err, ref)


@pytest.mark.slow
def test_table_6_1_w6():
    from golden_tables import rel_error
    ref = rel_error("table6_1_laplace.txt", 6)   # 0.0270 %, measured 4.06E-03 %
    err = _table_6_1_error(6)
    assert ref / 10 < err < ref * 5, err
