"""The seeded synthetic inputs are the stated recipes (CPU, no GPU):

* the bench's right-hand sides f_r = sum_{i,j,k<=8} c_ijk 2^-(i+j+k)
  L_i(2x-1) L_j(2y-1) L_k(2z-1) with c ~ N(0,1) from PCG64(20260 + r),
  evaluated here with numpy's own Legendre series; the coefficient
  a = 1 + 1/2 sin 2 pi x sin 2 pi y sin 2 pi z lies in [1/2, 3/2] and its
  closed-form gradient matches central differences; rank p of a multi-GPU run
  starts at seed 20260 + 64 p;
* the adjoint batch: degrees W_p in {4..10} from PCG64(7), every degree
  present among 256 problems; g = log a has theta_000 = 0 and L2 standard
  deviation 1/2 on [0,1]^3 (Gauss-Legendre quadrature exact for the
  polynomial g^2), and grad a = a grad g (central differences).
"""
import numpy as np
from numpy.polynomial import legendre as npleg

import workloads as wl


def _series(c, x, y, z):
    """sum_ijk c[i,j,k] L_i(x) L_j(y) L_k(z) at one point (numpy's Legendre series)."""
    return float(npleg.legval3d(x, y, z, c))


def test_bench_rhs_recipe():
    pb = wl.varcoef_random_rhs(n=2, W=2, n_rhs=4)
    K = 8
    i = np.arange(K + 1)
    decay = 2.0 ** -(i[:, None, None] + i[None, :, None] + i[None, None, :])
    pts = np.random.default_rng(3).uniform(0.0, 1.0, size=(5, 3))
    for r in (0, 3):
        c = np.random.Generator(np.random.PCG64(20260 + r)).standard_normal((K + 1,) * 3) * decay
        for x, y, z in pts:
            got = float(pb.f[r](np.array([x]), np.array([y]), np.array([z])).ravel()[0])
            ref = _series(c, 2 * x - 1, 2 * y - 1, 2 * z - 1)
            assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (r, got, ref)


def test_bench_coefficient_and_gradient():
    pb = wl.varcoef_random_rhs(n=2, W=2, n_rhs=1)
    xs = np.linspace(0.0, 1.0, 13)
    a = pb.a(xs, xs, xs)
    assert a.min() >= 0.5 - 1e-15 and a.max() <= 1.5 + 1e-15
    x0 = np.array([0.13]), np.array([0.71]), np.array([0.42])
    g = [float(v.ravel()[0]) for v in pb.grad_a(*x0)]
    h = 1e-6
    for d in range(3):
        p = [v.copy() for v in x0]
        m = [v.copy() for v in x0]
        p[d] = p[d] + h
        m[d] = m[d] - h
        fd = (float(pb.a(*p).ravel()[0]) - float(pb.a(*m).ravel()[0])) / (2 * h)
        assert abs(fd - g[d]) <= 1e-7 * max(1.0, abs(g[d])), d


def test_rank_seed_ranges_are_disjoint():
    import bench
    assert bench.shard_seed0(0, 64) == 20260
    assert bench.shard_seed0(3, 64) == 20260 + 3 * 64


def test_adjoint_batch_degrees():
    Ws = wl.adjoint_batch_degrees()
    assert Ws.shape == (256,) and Ws.min() >= 4 and Ws.max() <= 10
    assert set(Ws.tolist()) == set(range(4, 11))
    assert np.array_equal(Ws, wl.adjoint_batch_degrees())
    ref = np.random.Generator(np.random.PCG64(7)).integers(4, 11, size=256)
    assert np.array_equal(Ws, ref)


def test_lognormal_coefficient_statistics():
    xg, wg = npleg.leggauss(6)  # exact for g^2 (degree 6 per axis)
    x01, w01 = 0.5 * (xg + 1.0), 0.5 * wg
    for p in (0, 5):
        pb = wl.lognormal_coef_problem(W=4, p=p, n=1)
        th = pb.meta["theta"]
        assert th[0, 0, 0] == 0.0
        a = pb.a(x01, x01, x01)  # [z][y][x]
        gq = np.log(a)
        wt = w01[:, None, None] * w01[None, :, None] * w01[None, None, :]
        mean = float(np.sum(wt * gq))
        var = float(np.sum(wt * gq * gq)) - mean ** 2
        assert abs(mean) <= 1e-13
        assert abs(np.sqrt(var) - 0.5) <= 1e-12, np.sqrt(var)
        # grad a = a grad g, against central differences of a
        x0 = np.array([0.3]), np.array([0.6]), np.array([0.8])
        g = [float(v.ravel()[0]) for v in pb.grad_a(*x0)]
        h = 1e-6
        for d in range(3):
            pp = [v.copy() for v in x0]
            mm = [v.copy() for v in x0]
            pp[d] = pp[d] + h
            mm[d] = mm[d] - h
            fd = (float(pb.a(*pp).ravel()[0]) - float(pb.a(*mm).ravel()[0])) / (2 * h)
            assert abs(fd - g[d]) <= 1e-7 * max(1.0, abs(g[d])), (p, d)
