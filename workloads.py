"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module holds problem *data* only: meshes of axis-aligned box elements
(element boxes, degrees, face adjacency) and the closed-form coefficient,
source, boundary and exact-solution functions of the manufactured problems.
It contains none of the method's arithmetic (no quadrature, no norms, no
operators), so both sides can take their inputs from here and still share no
code.

Data functions are evaluated on tensor grids: ``fun(xs, ys, zs)`` takes three
1-D coordinate arrays and returns an array of shape
``(len(zs), len(ys), len(xs))`` (x fastest in C order, the lexicographic
ordering of Section 5.3).  Face data use a length-1 array for the normal
coordinate.

Face numbering of a box element: face ``2*axis + side`` with axis 0/1/2 = x/y/z
and side 0 = the low face (lambda = -1), side 1 = the high face (lambda = +1).
A neighbour id of -1 marks a Dirichlet boundary face.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

PI = math.pi


# --------------------------------------------------------------------------
# Meshes
# --------------------------------------------------------------------------
@dataclass
class MeshDesc:
    """A batch of box-element meshes (one or more independent problems)."""

    elem_lo: np.ndarray        # [E, 3] float64, box lower corner
    elem_hi: np.ndarray        # [E, 3] float64, box upper corner
    elem_W: np.ndarray         # [E] int32, polynomial degree per variable
    elem_nbr: np.ndarray       # [E, 6] int32, neighbour element id or -1
    elem_problem: np.ndarray   # [E] int32, problem index of each element
    n_problem: int = 1
    # [E, 6] boundary condition of each outer face (elem_nbr = -1): 0 Dirichlet,
    # 1 Neumann; None = every outer face Dirichlet
    elem_bc: Optional[np.ndarray] = None

    @property
    def n_elem(self) -> int:
        return int(self.elem_W.shape[0])


def box_mesh(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), W=4) -> MeshDesc:
    """Uniform n[0] x n[1] x n[2] grid of boxes on [lo, hi]; all outer faces Dirichlet.

    Elements are numbered x fastest, then y, then z.
    """
    if isinstance(n, int):
        n = (n, n, n)
    nx, ny, nz = (int(v) for v in n)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    E = nx * ny * nz
    elem_lo = np.zeros((E, 3))
    elem_hi = np.zeros((E, 3))
    nbr = -np.ones((E, 6), dtype=np.int32)
    cuts = [np.linspace(lo[a], hi[a], m + 1) for a, m in enumerate((nx, ny, nz))]

    def eid(i, j, k):
        return (k * ny + j) * nx + i

    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                e = eid(i, j, k)
                idx = (i, j, k)
                for a in range(3):
                    elem_lo[e, a] = cuts[a][idx[a]]
                    elem_hi[e, a] = cuts[a][idx[a] + 1]
                if i > 0:
                    nbr[e, 0] = eid(i - 1, j, k)
                if i < nx - 1:
                    nbr[e, 1] = eid(i + 1, j, k)
                if j > 0:
                    nbr[e, 2] = eid(i, j - 1, k)
                if j < ny - 1:
                    nbr[e, 3] = eid(i, j + 1, k)
                if k > 0:
                    nbr[e, 4] = eid(i, j, k - 1)
                if k < nz - 1:
                    nbr[e, 5] = eid(i, j, k + 1)
    return MeshDesc(elem_lo, elem_hi, np.full(E, W, dtype=np.int32), nbr,
                    np.zeros(E, dtype=np.int32), 1)


def concat_meshes(meshes: List[MeshDesc]) -> MeshDesc:
    """Batch independent problems into one description (ids are offset)."""
    los, his, Ws, nbrs, probs = [], [], [], [], []
    off = 0
    poff = 0
    for m in meshes:
        los.append(m.elem_lo)
        his.append(m.elem_hi)
        Ws.append(m.elem_W)
        nb = m.elem_nbr.copy()
        nb[nb >= 0] += off
        nbrs.append(nb)
        probs.append(m.elem_problem + poff)
        off += m.n_elem
        poff += m.n_problem
    bc = None
    if any(getattr(m, "elem_bc", None) is not None for m in meshes):
        bc = np.concatenate([m.elem_bc if getattr(m, "elem_bc", None) is not None
                             else np.zeros((m.n_elem, 6), dtype=np.int32) for m in meshes]).astype(np.int32)
    return MeshDesc(np.concatenate(los), np.concatenate(his),
                    np.concatenate(Ws).astype(np.int32),
                    np.concatenate(nbrs).astype(np.int32),
                    np.concatenate(probs).astype(np.int32), poff, elem_bc=bc)


# --------------------------------------------------------------------------
# Problems: closed-form data on tensor grids
# --------------------------------------------------------------------------
Fun = Callable[[np.ndarray, np.ndarray, np.ndarray], np.ndarray]


def _grid(xs, ys, zs):
    xs = np.asarray(xs, dtype=np.float64)
    ys = np.asarray(ys, dtype=np.float64)
    zs = np.asarray(zs, dtype=np.float64)
    return xs[None, None, :], ys[None, :, None], zs[:, None, None]


def _full(val, xs, ys, zs):
    return np.full((len(zs), len(ys), len(xs)), float(val))


@dataclass
class Problem:
    """Data of -div(a grad u) = f in the problem's box mesh, u = g on the boundary.

    ``f`` and ``g`` are lists with one function per right-hand side.
    ``a`` / ``grad_a`` are None for the Laplacian (a = 1).
    ``u_exact`` / ``grad_u_exact`` (per right-hand side) are optional.
    """

    mesh: MeshDesc
    f: List[Fun]
    g: List[Fun]
    a: Optional[Fun] = None
    grad_a: Optional[Callable] = None  # returns (ax, ay, az)
    u_exact: Optional[List[Fun]] = None
    grad_u_exact: Optional[List[Callable]] = None
    name: str = ""
    meta: dict = field(default_factory=dict)
    # Neumann data (eq. 2.1): per right-hand side the conormal field a grad u,
    # (qx, qy, qz) on tensor grids; a Neumann face takes h = nu . q, a Robin
    # face (bc 2) h = nu . q + robin_gamma g
    flux: Optional[List[Callable]] = None
    robin_gamma: float = 1.0
    # general operator sum A_ij u_ij + sum b_i u_i + c u (oracle, and the
    # library's COEF_GENERAL meshes):
    # op(xs, ys, zs) -> (A 3x3, b 3, c) on tensor grids; None: -div(a grad u)
    op: Optional[Callable] = None

    @property
    def n_rhs(self) -> int:
        return len(self.f)


def _zero(xs, ys, zs):
    return _full(0.0, xs, ys, zs)


def poisson_sine(n=2, W=4, lo=0.0, hi=1.0) -> Problem:
    """-Lap u = f with u = sin(pi x) sin(pi y) sin(pi z), u = 0 on the boundary.

    On [0,1]^3 this is the 2x2x2, W=4 configuration; on (-1,1)^3 it is the
    problem of Table 6.2.
    """
    mesh = box_mesh(n, (lo,) * 3, (hi,) * 3, W)

    def u(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        return np.sin(PI * x) * np.sin(PI * y) * np.sin(PI * z)

    def f(xs, ys, zs):
        return 3.0 * PI * PI * u(xs, ys, zs)

    def gu(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        sx, sy, sz = np.sin(PI * x), np.sin(PI * y), np.sin(PI * z)
        cx, cy, cz = np.cos(PI * x), np.cos(PI * y), np.cos(PI * z)
        return (PI * cx * sy * sz, PI * sx * cy * sz, PI * sx * sy * cz)

    return Problem(mesh, [f], [_zero], None, None, [u], [gu], name="poisson_sine")


def poisson_mixed(n=2, W=4) -> Problem:
    """Table 6.3: -Lap u = f on (-1,1)^3, Dirichlet on x = -1, x = 1, y = -1,
    Neumann on y = 1, z = -1, z = 1, exact
    u = (2 / pi^2) sin(pi x / 2) (cos(pi y / 2) - sin(pi z / 2)), so that
    -Lap u = (pi^2 / 2) u."""
    mesh = box_mesh(n, (-1.0,) * 3, (1.0,) * 3, W)
    bc = np.zeros((mesh.n_elem, 6), dtype=np.int32)
    for e in range(mesh.n_elem):
        for fi in (3, 4, 5):
            if mesh.elem_nbr[e, fi] == -1:
                bc[e, fi] = 1
    mesh.elem_bc = bc
    c = 2.0 / (PI * PI)

    def u(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        return c * np.sin(PI * x / 2) * (np.cos(PI * y / 2) - np.sin(PI * z / 2))

    def f(xs, ys, zs):
        return 0.5 * PI * PI * u(xs, ys, zs)

    def gu(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        sx, cx = np.sin(PI * x / 2), np.cos(PI * x / 2)
        return (c * PI / 2 * cx * (np.cos(PI * y / 2) - np.sin(PI * z / 2)),
                -c * PI / 2 * sx * np.sin(PI * y / 2),
                -c * PI / 2 * sx * np.cos(PI * z / 2))

    return Problem(mesh, [f], [u], None, None, [u], [gu], name="poisson_mixed", flux=[gu])


def _mixed_bc(mesh, neumann_faces=(3, 4, 5), code=1):
    """Face codes of the outer faces: `code` on the listed faces (fi = 2 axis + side), 0 elsewhere."""
    bc = np.zeros((mesh.n_elem, 6), dtype=np.int32)
    for e in range(mesh.n_elem):
        for fi in neumann_faces:
            if mesh.elem_nbr[e, fi] == -1:
                bc[e, fi] = code
    mesh.elem_bc = bc
    return mesh


def helmholtz_mixed(n=2, W=4) -> Problem:
    """Tables 6.6-6.7: -Lap u + u = f on (-1,1)^3, Dirichlet on x = +-1 and
    y = -1, du/dnu = h on y = 1 and z = +-1, exact u = e^x cos(y) sin(z)
    (so f = 2u).  General-operator form: A = -I, b = 0, c = 1."""
    mesh = _mixed_bc(box_mesh(n, (-1.0,) * 3, (1.0,) * 3, W))

    def u(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        return np.exp(x) * np.cos(y) * np.sin(z)

    def f(xs, ys, zs):
        return 2.0 * u(xs, ys, zs)

    def gu(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        ex = np.exp(x)
        return ex * np.cos(y) * np.sin(z), -ex * np.sin(y) * np.sin(z), ex * np.cos(y) * np.cos(z)

    def op(xs, ys, zs):
        return ([[-1.0, 0.0, 0.0], [0.0, -1.0, 0.0], [0.0, 0.0, -1.0]], [0.0, 0.0, 0.0], 1.0)

    return Problem(mesh, [f], [u], None, None, [u], [gu], name="helmholtz_mixed", flux=[gu], op=op)


def varcoef_robin(n=3, W=2) -> Problem:
    """Table 6.12: a u_xx + b u_yy + c u_zz + d u = f on (-1,1)^3 with
    du/dnu + u = g on every face, a = -(1 + 0.01 y sin x),
    b = -(2.5 + 0.02 cos(x^2 + z)), c = -(3 + 0.03 y e^z),
    d = 0.15 sin(2 pi (y + z)), exact u = cos(pi (x + y)) e^z."""
    mesh = _mixed_bc(box_mesh(n, (-1.0,) * 3, (1.0,) * 3, W), neumann_faces=range(6), code=2)

    def coefs(x, y, z):
        return (-(1.0 + 0.01 * y * np.sin(x)), -(2.5 + 0.02 * np.cos(x * x + z)), -(3.0 + 0.03 * y * np.exp(z)),
                0.15 * np.sin(2 * PI * (y + z)))

    def u(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        return np.cos(PI * (x + y)) * np.exp(z)

    def f(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        a, b, c, d = coefs(x, y, z)
        w = np.cos(PI * (x + y)) * np.exp(z)
        return (-PI * PI * (a + b) + c + d) * w

    def gu(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        s_, ez = np.sin(PI * (x + y)), np.exp(z)
        return -PI * s_ * ez, -PI * s_ * ez, np.cos(PI * (x + y)) * ez

    def op(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        a, b, c, d = coefs(x, y, z)
        zero = 0.0 * x
        return ([[a, zero, zero], [zero, b, zero], [zero, zero, c]], [zero, zero, zero], d)

    return Problem(mesh, [f], [u], None, None, [u], [gu], name="varcoef_robin", flux=[gu], op=op)


def nonsym_mixed(n=2, W=4) -> Problem:
    """Table 6.14: a u_xx + b u_yy + c u_zz + d (u_xy + u_yz + u_zx) + e u = f
    on (-1,1)^3 with the boundary conditions of Table 6.3,
    a = -(0.5 + 0.05 exp(xyz)), b = -(1 + 0.015 cos(x + y)),
    c = -(2.5 + 0.02 exp(y + z)), d = -0.001 sin(pi (x + y + z)),
    e = 4.05 + 0.045 cos(pi (x + y + z) / 2), exact
    u = (sin(pi x) + sin(pi y / 2)) cos(pi z)."""
    mesh = _mixed_bc(box_mesh(n, (-1.0,) * 3, (1.0,) * 3, W))

    def coefs(x, y, z):
        t = PI * (x + y + z)
        return (-(0.5 + 0.05 * np.exp(x * y * z)), -(1.0 + 0.015 * np.cos(x + y)), -(2.5 + 0.02 * np.exp(y + z)),
                -0.001 * np.sin(t), 4.05 + 0.045 * np.cos(t / 2))

    def u(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        return (np.sin(PI * x) + np.sin(PI * y / 2)) * np.cos(PI * z)

    def f(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        a, b, c, d, e = coefs(x, y, z)
        sx, cx, sy, cy = np.sin(PI * x), np.cos(PI * x), np.sin(PI * y / 2), np.cos(PI * y / 2)
        sz, cz = np.sin(PI * z), np.cos(PI * z)
        uxx = -PI * PI * sx * cz
        uyy = -PI * PI / 4 * sy * cz
        uzz = -PI * PI * (sx + sy) * cz
        uxy = 0.0 * x
        uyz = -PI * PI / 2 * cy * sz
        uzx = -PI * PI * cx * sz
        return a * uxx + b * uyy + c * uzz + d * (uxy + uyz + uzx) + e * (sx + sy) * cz

    def gu(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        return (PI * np.cos(PI * x) * np.cos(PI * z), PI / 2 * np.cos(PI * y / 2) * np.cos(PI * z),
                -PI * (np.sin(PI * x) + np.sin(PI * y / 2)) * np.sin(PI * z))

    def op(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        a, b, c, d, e = coefs(x, y, z)
        h = 0.5 * d
        zero = 0.0 * x
        return ([[a, h, h], [h, b, h], [h, h, c]], [zero, zero, zero], e)

    return Problem(mesh, [f], [u], None, None, [u], [gu], name="nonsym_mixed", flux=[gu], op=op)


def polynomial_exact(n=2, W=3, lo=-1.0, hi=1.0) -> Problem:
    """Exact solution inside the discrete space (degree 3 per variable).

    u = (1-x^2)(1-y^2)(1-z^2)(1+xy) on (-1,1)^3 vanishes on the boundary; for
    W >= 3 the least-squares minimiser reproduces it exactly.
    """
    mesh = box_mesh(n, (lo,) * 3, (hi,) * 3, W)

    def u(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        return (1 - x * x) * (1 - y * y) * (1 - z * z) * (1 + x * y)

    def grad(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        X, Y, Z = 1 - x * x, 1 - y * y, 1 - z * z
        ux = (-2 * x * (1 + x * y) + X * y) * Y * Z
        uy = (-2 * y * (1 + x * y) + Y * x) * X * Z
        uz = -2 * z * X * Y * (1 + x * y)
        return ux, uy, uz

    def f(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        X, Y, Z = 1 - x * x, 1 - y * y, 1 - z * z
        # second derivatives of (1-x^2)(1+xy) in x: d2/dx2 = -2(1+xy) - 4xy
        uxx = (-2 * (1 + x * y) - 4 * x * y) * Y * Z
        uyy = (-2 * (1 + x * y) - 4 * x * y) * X * Z
        uzz = -2 * X * Y * (1 + x * y)
        return -(uxx + uyy + uzz)

    return Problem(mesh, [f], [_zero], None, None, [u], [grad], name="polynomial_exact")


def _legendre_table(kmax, t):
    """Legendre values L_0..L_kmax at t (three-term recurrence; input data only)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros((kmax + 1,) + t.shape)
    out[0] = 1.0
    if kmax >= 1:
        out[1] = t
    for m in range(1, kmax):
        out[m + 1] = ((2 * m + 1) * t * out[m] - m * out[m - 1]) / (m + 1)
    return out


def _legendre_deriv_table(kmax, t):
    """Derivatives L'_0..L'_kmax at t, from (1-t^2) L'_m = m (L_{m-1} - t L_m)."""
    t = np.asarray(t, dtype=np.float64)
    Lt = _legendre_table(kmax + 1, t)
    d = np.zeros((kmax + 1,) + t.shape)
    # recurrence L'_{m+1} = L'_{m-1} + (2m+1) L_m  (valid at the endpoints too)
    if kmax >= 1:
        d[1] = 1.0
    for m in range(1, kmax):
        d[m + 1] = d[m - 1] + (2 * m + 1) * Lt[m]
    return d


def legendre_field(coef, box_lo, box_hi):
    """Return (F, dF) for F(x) = sum c_ijk L_i(s x) L_j(s y) L_k(s z) on a box.

    ``coef`` has shape [K+1, K+1, K+1] indexed [i, j, k] (x, y, z degrees);
    s maps the box affinely onto (-1,1)^3.  ``dF`` returns the gradient.
    """
    coef = np.asarray(coef, dtype=np.float64)
    K = coef.shape[0] - 1
    lo = np.asarray(box_lo, dtype=np.float64)
    hi = np.asarray(box_hi, dtype=np.float64)
    sc = 2.0 / (hi - lo)

    def tabs(xs, ys, zs):
        tx = sc[0] * (np.asarray(xs) - lo[0]) - 1
        ty = sc[1] * (np.asarray(ys) - lo[1]) - 1
        tz = sc[2] * (np.asarray(zs) - lo[2]) - 1
        return tx, ty, tz

    def F(xs, ys, zs):
        tx, ty, tz = tabs(xs, ys, zs)
        Lx, Ly, Lz = (_legendre_table(K, t) for t in (tx, ty, tz))
        return np.einsum("ijk,ia,jb,kc->cba", coef, Lx, Ly, Lz, optimize=True)

    def dF(xs, ys, zs):
        tx, ty, tz = tabs(xs, ys, zs)
        Lx, Ly, Lz = (_legendre_table(K, t) for t in (tx, ty, tz))
        dx, dy, dz = (_legendre_deriv_table(K, t) for t in (tx, ty, tz))
        gx = sc[0] * np.einsum("ijk,ia,jb,kc->cba", coef, dx, Ly, Lz, optimize=True)
        gy = sc[1] * np.einsum("ijk,ia,jb,kc->cba", coef, Lx, dy, Lz, optimize=True)
        gz = sc[2] * np.einsum("ijk,ia,jb,kc->cba", coef, Lx, Ly, dz, optimize=True)
        return gx, gy, gz

    return F, dF


def varcoef_random_rhs(n=8, W=8, n_rhs=64, seed0=20260, kmax=8) -> Problem:
    """-div(a grad u) = f on [0,1]^3, a = 1 + 0.5 sin(2pi x) sin(2pi y) sin(2pi z).

    f_r = sum_{i,j,k<=kmax} c_ijk 2^-(i+j+k) L_i(2x-1) L_j(2y-1) L_k(2z-1),
    c ~ N(0,1) i.i.d. from numpy PCG64 with seed seed0 + r; u = 0 on the boundary.
    """
    mesh = box_mesh(n, (0.0,) * 3, (1.0,) * 3, W)
    tp = 2 * PI

    def a(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        return 1.0 + 0.5 * np.sin(tp * x) * np.sin(tp * y) * np.sin(tp * z)

    def grad_a(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        sx, sy, sz = np.sin(tp * x), np.sin(tp * y), np.sin(tp * z)
        cx, cy, cz = np.cos(tp * x), np.cos(tp * y), np.cos(tp * z)
        return (0.5 * tp * cx * sy * sz, 0.5 * tp * sx * cy * sz, 0.5 * tp * sx * sy * cz)

    fs = []
    decay = 2.0 ** -np.add.outer(np.add.outer(np.arange(kmax + 1), np.arange(kmax + 1)),
                                 np.arange(kmax + 1))
    for r in range(n_rhs):
        rng = np.random.Generator(np.random.PCG64(seed0 + r))
        c = rng.standard_normal((kmax + 1,) * 3) * decay
        F, _ = legendre_field(c, (0.0,) * 3, (1.0,) * 3)
        fs.append(F)
    return Problem(mesh, fs, [_zero] * n_rhs, a, grad_a, None, None,
                   name="varcoef_random_rhs", meta={"seed0": seed0})


def lognormal_coef_problem(W, p, n=4, seed=100, target_std=0.5, kmax=3) -> Problem:
    """One problem of the adjoint batch: a = exp(g) on [0,1]^3, f = 1, u = 0.

    g = sum_{i,j,k<=kmax} theta_ijk L_i L_j L_k (on [0,1]^3 mapped to (-1,1)^3),
    theta ~ N(0,1) from PCG64(seed + p), theta_000 = 0, rescaled so that the
    L2(Omega)-standard deviation of g is target_std.  With Legendre orthogonality
    on (-1,1) (|L_i|^2 = 2/(2i+1)) and |Omega| = 1 the variance of g is
    sum theta_ijk^2 / ((2i+1)(2j+1)(2k+1)).
    """
    rng = np.random.Generator(np.random.PCG64(seed + p))
    th = rng.standard_normal((kmax + 1,) * 3)
    th[0, 0, 0] = 0.0
    m = np.arange(kmax + 1)
    norm = 1.0 / np.multiply.outer(np.multiply.outer(2 * m + 1, 2 * m + 1), 2 * m + 1)
    var = float(np.sum(th * th * norm))
    th *= target_std / math.sqrt(var)
    mesh = box_mesh(n, (0.0,) * 3, (1.0,) * 3, W)
    G, dG = legendre_field(th, (0.0,) * 3, (1.0,) * 3)

    def a(xs, ys, zs):
        return np.exp(G(xs, ys, zs))

    def grad_a(xs, ys, zs):
        e = np.exp(G(xs, ys, zs))
        gx, gy, gz = dG(xs, ys, zs)
        return e * gx, e * gy, e * gz

    def one(xs, ys, zs):
        return _full(1.0, xs, ys, zs)

    return Problem(mesh, [one], [_zero], a, grad_a, None, None,
                   name="lognormal_coef", meta={"theta": th, "W": W, "p": p})


def adjoint_batch_degrees(n_problem=256, seed=7, wmin=4, wmax=10) -> np.ndarray:
    """Per-problem degrees W_p ~ U{wmin..wmax} from PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(wmin, wmax + 1, size=n_problem).astype(np.int32)


def random_dofs(n, seed, dtype=np.float64) -> np.ndarray:
    """Seeded N(0,1) vector (test input for operator applies)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(n).astype(dtype)


def laplace_sinh(n=2, W=4) -> Problem:
    """Table 6.1: Lap u = 0 on (0,1)^3, u = g on the boundary, with
    u = sin(pi x) sin(pi y) sinh(sqrt2 pi z) / (pi^2 sinh(sqrt2 pi))."""
    mesh = box_mesh(n, (0.0,) * 3, (1.0,) * 3, W)
    r2 = math.sqrt(2.0) * PI
    c = 1.0 / (PI * PI * math.sinh(r2))

    def u(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        return c * np.sin(PI * x) * np.sin(PI * y) * np.sinh(r2 * z)

    def grad(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        sx, sy, shz = np.sin(PI * x), np.sin(PI * y), np.sinh(r2 * z)
        return (c * PI * np.cos(PI * x) * sy * shz, c * PI * sx * np.cos(PI * y) * shz,
                c * r2 * sx * sy * np.cosh(r2 * z))

    return Problem(mesh, [_zero], [u], None, None, [u], [grad], name="laplace_sinh")


def varcoef_manufactured(n=(2, 2, 1), W=4) -> Problem:
    """-div(a grad u) = f on (0,1)^3 with a = 1 + 0.5 sin(2pi x) sin(2pi y) sin(2pi z),
    exact u = exp(x) sin(pi y) (1 + z^2), Dirichlet data g = u (test problem)."""
    mesh = box_mesh(n, (0.0,) * 3, (1.0,) * 3, W)
    tp = 2 * PI

    def a(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        return 1.0 + 0.5 * np.sin(tp * x) * np.sin(tp * y) * np.sin(tp * z)

    def grad_a(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        sx, sy, sz = np.sin(tp * x), np.sin(tp * y), np.sin(tp * z)
        cx, cy, cz = np.cos(tp * x), np.cos(tp * y), np.cos(tp * z)
        return (0.5 * tp * cx * sy * sz, 0.5 * tp * sx * cy * sz, 0.5 * tp * sx * sy * cz)

    def u(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        return np.exp(x) * np.sin(PI * y) * (1 + z * z)

    def grad(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        ex, sy, cy = np.exp(x), np.sin(PI * y), np.cos(PI * y)
        return (ex * sy * (1 + z * z), ex * PI * cy * (1 + z * z), ex * sy * 2 * z)

    def f(xs, ys, zs):
        x, y, z = _grid(xs, ys, zs)
        ex, sy = np.exp(x), np.sin(PI * y)
        lap = ex * sy * (1 + z * z) - PI * PI * ex * sy * (1 + z * z) + ex * sy * 2.0
        ux, uy, uz = grad(xs, ys, zs)
        ax, ay, az = grad_a(xs, ys, zs)
        return -(a(xs, ys, zs) * lap + ax * ux + ay * uy + az * uz)

    return Problem(mesh, [f], [u], a, grad_a, [u], [grad], name="varcoef_manufactured")


def batch_problems(problems: List[Problem]) -> Problem:
    """Independent problems in one batch (one mesh, per-problem data).

    The returned Problem carries ``parts``: element e takes its data from
    ``parts[mesh.elem_problem[e]]``.  All parts must have the same number of
    right-hand sides and the same coefficient kind.
    """
    nr = problems[0].n_rhs
    if any(p.n_rhs != nr for p in problems):
        raise ValueError("all problems of a batch need the same number of right-hand sides")
    if any((p.a is None) != (problems[0].a is None) for p in problems):
        raise ValueError("all problems of a batch need the same coefficient kind")
    mesh = concat_meshes([p.mesh for p in problems])
    out = Problem(mesh, list(problems[0].f), list(problems[0].g), problems[0].a, problems[0].grad_a,
                  name="batch", meta={"n": len(problems)})
    out.parts = list(problems)
    return out


def adjoint_batch(n_problem=256, n=4, seed_w=7, seed_theta=100, wmin=4, wmax=10) -> Problem:
    """The adjoint batch: n_problem independent lognormal-coefficient problems,
    degrees W_p ~ U{wmin..wmax} (PCG64(seed_w)), theta from PCG64(seed_theta + p)."""
    Ws = adjoint_batch_degrees(n_problem, seed_w, wmin, wmax)
    return batch_problems([lognormal_coef_problem(int(W), p, n=n, seed=seed_theta) for p, W in enumerate(Ws)])


# ---------------------------------------------------------------------------
# Edge neighbourhood (Section 2.3 / eq. 4.7): elements are boxes in the modified
# coordinates (tau, theta, x3) = (ln r, theta, x3) around an edge on the x3 axis
# ---------------------------------------------------------------------------
@dataclass
class EdgeMeshDesc:
    """Geometric mesh of an edge neighbourhood {0 < r < Z, th0 < theta < th1, z0 < x3 < z1}.

    Finite elements are boxes [ln r_i, ln r_{i+1}] x [theta_j, theta_{j+1}] x
    [x3_n, x3_{n+1}] in modified coordinates with r_i = Z mu^(N+1-i),
    i = 1..N+1 (layer i = 1 is next to the edge).  The corner elements
    r < r_1 hold one polynomial in x3 per x3-slab n, shared by every theta
    sector (corner set n).  Face codes in elem_nbr: >= 0 neighbour element,
    -1 Dirichlet face, -2 - n the corner set n (the r = r_1 face of layer 1).
    """
    elem_lo: np.ndarray        # [E, 3] (tau, theta, x3) lower corner
    elem_hi: np.ndarray        # [E, 3]
    elem_W: np.ndarray         # [E] int32
    elem_nbr: np.ndarray       # [E, 6] int32
    elem_problem: np.ndarray   # [E] int32
    corner_W: np.ndarray       # [C] int32, degree of each corner polynomial in x3
    corner_lo: np.ndarray      # [C] x3 lower end of the slab
    corner_hi: np.ndarray      # [C] x3 upper end
    corner_problem: np.ndarray  # [C] int32
    n_problem: int = 1
    kind: str = "edge"         # "edge", "vertex" (phi, theta, ln rho) or "vertex-edge" (ln tan phi, theta, ln x3)

    @property
    def n_elem(self) -> int:
        return int(self.elem_W.shape[0])

    @property
    def n_corner(self) -> int:
        return int(self.corner_W.shape[0])


def edge_mesh(N, W, mu=0.15, Z=1.0, theta=(0.0, PI / 2), x3=(0.0, 1.0), I=1, J=1,
              layer_W=None) -> EdgeMeshDesc:
    """N finite layers x I theta-sectors x J x3-slabs (degree W in every
    modified coordinate, or layer_W[i] in layer i) plus J corner sets of
    degree W; every outer face of the finite elements (r = Z,
    theta = theta_0 / theta_1, x3 = x3_0 / x3_1) is Dirichlet.  Elements are
    numbered layer fastest, then sector, then slab."""
    r = [Z * mu ** (N + 1 - i) for i in range(1, N + 2)]
    taus = np.log(np.array(r))
    ths = np.linspace(theta[0], theta[1], I + 1)
    zs = np.linspace(x3[0], x3[1], J + 1)
    E = N * I * J
    lo = np.zeros((E, 3))
    hi = np.zeros((E, 3))
    nbr = -np.ones((E, 6), dtype=np.int32)

    def eid(i, j, n):
        return (n * I + j) * N + i

    for n in range(J):
        for j in range(I):
            for i in range(N):
                e = eid(i, j, n)
                lo[e] = (taus[i], ths[j], zs[n])
                hi[e] = (taus[i + 1], ths[j + 1], zs[n + 1])
                nbr[e, 0] = eid(i - 1, j, n) if i > 0 else -2 - n
                nbr[e, 1] = eid(i + 1, j, n) if i < N - 1 else -1
                nbr[e, 2] = eid(i, j - 1, n) if j > 0 else -1
                nbr[e, 3] = eid(i, j + 1, n) if j < I - 1 else -1
                nbr[e, 4] = eid(i, j, n - 1) if n > 0 else -1
                nbr[e, 5] = eid(i, j, n + 1) if n < J - 1 else -1
    Ws = np.full(E, W, dtype=np.int32)
    if layer_W is not None:
        Ws = np.array([int(layer_W[e % N]) for e in range(E)], dtype=np.int32)
    return EdgeMeshDesc(lo, hi, Ws, nbr, np.zeros(E, dtype=np.int32),
                        np.full(J, W, dtype=np.int32), zs[:-1].copy(), zs[1:].copy(), np.zeros(J, dtype=np.int32))


@dataclass
class EdgeProblem:
    """-Lap u = f in the edge neighbourhood, u = g on its Dirichlet faces.

    Data are functions of cylindrical coordinates on tensor grids:
    fun(rs, thetas, x3s) -> array [len x3s, len thetas, len rs] (r fastest).
    """
    mesh: EdgeMeshDesc
    f: List[Callable]
    g: List[Callable]
    u_exact: Optional[Callable] = None
    grad_exact: Optional[Callable] = None  # (u_r, u_theta / r, u_x3) on tensor grids
    name: str = ""
    meta: dict = field(default_factory=dict)
    # Neumann data (edge meshes with elem_bc): per right-hand side the
    # physical gradient field (q_r, q_theta = u_theta / r, q_x3) on tensor grids
    flux: Optional[List[Callable]] = None


def _cyl_grid(rs, ts, zs):
    z, t, r = np.meshgrid(np.asarray(zs, dtype=np.float64), np.asarray(ts, dtype=np.float64),
                          np.asarray(rs, dtype=np.float64), indexing="ij")
    return r, t, z


def edge_laplace_singular(N, W, mu=0.15, alpha=1.0 / 3.0) -> EdgeProblem:
    """Table 6.18: Lap u = 0 on {0 < r < 1, 0 < theta < pi/2, 0 < x3 < 1},
    u = g on the boundary with the exact solution w = r^alpha sin(alpha theta) x3
    (alpha = 1/3, an edge singularity along the x3 axis)."""
    mesh = edge_mesh(N, W, mu=mu)

    def w(rs, ts, zs):
        r, t, z = _cyl_grid(rs, ts, zs)
        return r ** alpha * np.sin(alpha * t) * z

    def grad(rs, ts, zs):
        r, t, z = _cyl_grid(rs, ts, zs)
        return (alpha * r ** (alpha - 1) * np.sin(alpha * t) * z,
                alpha * r ** (alpha - 1) * np.cos(alpha * t) * z,
                r ** alpha * np.sin(alpha * t))

    def zero(rs, ts, zs):
        return np.zeros((len(zs), len(ts), len(rs)))

    return EdgeProblem(mesh, [zero], [w], w, grad, name="edge_laplace_singular", meta=dict(alpha=alpha))


def edge_polynomial(N, W, mu=0.15) -> EdgeProblem:
    """A solution inside the discrete space: u = 1 + x3^2 + (tau - tau_1)^2 theta x3
    (tau = ln r, tau_1 = ln r_1 the corner face), whose trace on the corner face
    is 1 + x3^2 with no tau or theta derivative, so the corner polynomial
    reproduces it; f = -Lap u = -(u_tautau + u_thetatheta) / r^2 - u_x3x3."""
    mesh = edge_mesh(N, W, mu=mu)
    tau1 = float(mesh.elem_lo[0, 0])

    def u(rs, ts, zs):
        r, t, z = _cyl_grid(rs, ts, zs)
        return 1.0 + z * z + (np.log(r) - tau1) ** 2 * t * z

    def f(rs, ts, zs):
        r, t, z = _cyl_grid(rs, ts, zs)
        return -(2.0 * t * z) / (r * r) - 2.0

    return EdgeProblem(mesh, [f], [u], u, None, name="edge_polynomial", meta=dict(tau1=tau1))


def concat_edge_meshes(meshes: List[EdgeMeshDesc]) -> EdgeMeshDesc:
    """Batch independent edge neighbourhoods (element ids and corner codes offset)."""
    los, his, Ws, nbrs, probs, cW, clo, chi, cprob = [], [], [], [], [], [], [], [], []
    off = coff = poff = 0
    for m in meshes:
        los.append(m.elem_lo)
        his.append(m.elem_hi)
        Ws.append(m.elem_W)
        nb = m.elem_nbr.copy()
        nb[nb >= 0] += off
        nb[nb <= -2] -= coff
        nbrs.append(nb)
        probs.append(m.elem_problem + poff)
        cW.append(m.corner_W)
        clo.append(m.corner_lo)
        chi.append(m.corner_hi)
        cprob.append(m.corner_problem + poff)
        off += m.n_elem
        coff += m.n_corner
        poff += m.n_problem
    cat = np.concatenate
    return EdgeMeshDesc(cat(los), cat(his), cat(Ws).astype(np.int32), cat(nbrs).astype(np.int32),
                        cat(probs).astype(np.int32), cat(cW).astype(np.int32), cat(clo), cat(chi),
                        cat(cprob).astype(np.int32), poff, kind=meshes[0].kind)


def edge_batch(Ws, mu=0.15) -> EdgeProblem:
    """Independent copies of Table 6.18's problem with uneven degrees W_p
    (N_p = 2 W_p + 4 layers each) in one batch; every problem has the same
    data functions."""
    base = edge_laplace_singular(N=2, W=2, mu=mu)
    mesh = concat_edge_meshes([edge_mesh(2 * int(W) + 4, int(W), mu=mu) for W in Ws])
    return EdgeProblem(mesh, base.f, base.g, base.u_exact, base.grad_exact, name="edge_batch",
                       meta=dict(Ws=[int(w) for w in Ws]))


# ---------------------------------------------------------------------------
# Vertex neighbourhood (Section 2.3 / eq. 4.3): elements are boxes in the
# modified coordinates (phi, theta, chi) = (phi, theta, ln rho) around a vertex
# ---------------------------------------------------------------------------
def vertex_mesh(N, W, mu=0.15, phi=(PI / 6, PI / 3), theta=(0.0, 1.5 * PI), I=1, J=3) -> EdgeMeshDesc:
    """N finite layers in chi = ln rho (rho_i = mu^(N+1-i), layer 1 next to the
    vertex) x I phi-sectors x J theta-sectors, degree W in every modified
    coordinate; one corner set rho < rho_1 holding a constant (degree 0) shared
    by every sector.  Axes (x, y, z) = (phi, theta, chi); the corner set is the
    neighbour of face 4 (chi = lo) of layer 1, code -2.  Every other outer face
    is Dirichlet.  Elements are numbered layer fastest, then phi, then theta."""
    rho = [mu ** (N + 1 - i) for i in range(1, N + 2)]
    chis = np.log(np.array(rho))
    phs = np.linspace(phi[0], phi[1], I + 1)
    ths = np.linspace(theta[0], theta[1], J + 1)
    E = N * I * J
    lo = np.zeros((E, 3))
    hi = np.zeros((E, 3))
    nbr = -np.ones((E, 6), dtype=np.int32)

    def eid(i, a, b):
        return (b * I + a) * N + i

    for b in range(J):
        for a in range(I):
            for i in range(N):
                e = eid(i, a, b)
                lo[e] = (phs[a], ths[b], chis[i])
                hi[e] = (phs[a + 1], ths[b + 1], chis[i + 1])
                nbr[e, 0] = eid(i, a - 1, b) if a > 0 else -1
                nbr[e, 1] = eid(i, a + 1, b) if a < I - 1 else -1
                nbr[e, 2] = eid(i, a, b - 1) if b > 0 else -1
                nbr[e, 3] = eid(i, a, b + 1) if b < J - 1 else -1
                nbr[e, 4] = eid(i - 1, a, b) if i > 0 else -2
                nbr[e, 5] = eid(i + 1, a, b) if i < N - 1 else -1
    return EdgeMeshDesc(lo, hi, np.full(E, W, dtype=np.int32), nbr, np.zeros(E, dtype=np.int32),
                        np.zeros(1, dtype=np.int32), np.zeros(1), np.zeros(1), np.zeros(1, dtype=np.int32),
                        kind="vertex")


def _sph_grid(phs, ths, rhos):
    r, t, p = np.meshgrid(np.asarray(rhos, dtype=np.float64), np.asarray(ths, dtype=np.float64),
                          np.asarray(phs, dtype=np.float64), indexing="ij")
    return p, t, r


def vertex_poisson_singular(N, W, mu=0.15) -> EdgeProblem:
    """Table 6.16: -Lap u = f on {pi/6 < phi < pi/3, 0 < theta < 3 pi/2, rho < 1},
    u = g on the boundary, exact w = rho^(1/2) sin(phi/2) (a vertex singularity);
    f = -Lap w = -rho^(-3/2) (sin(phi/2) + cot(phi) cos(phi/2)) / 2.
    Data are functions of spherical coordinates on tensor grids
    fun(phis, thetas, rhos) -> [len rhos, len thetas, len phis]."""
    mesh = vertex_mesh(N, W, mu=mu)

    def w(ps, ts, rs):
        p, t, r = _sph_grid(ps, ts, rs)
        return np.sqrt(r) * np.sin(p / 2)

    def grad(ps, ts, rs):
        # (w_rho, w_phi / rho, w_theta / (rho sin phi))
        p, t, r = _sph_grid(ps, ts, rs)
        return 0.5 / np.sqrt(r) * np.sin(p / 2), 0.5 / np.sqrt(r) * np.cos(p / 2), 0.0 * r

    def f(ps, ts, rs):
        p, t, r = _sph_grid(ps, ts, rs)
        return -0.5 * r ** -1.5 * (np.sin(p / 2) + np.cos(p / 2) / np.tan(p))

    return EdgeProblem(mesh, [f], [w], w, grad, name="vertex_poisson_singular")


def vertex_polynomial(N, W, mu=0.15) -> EdgeProblem:
    """A solution inside the discrete space with the corner constant 2:
    u = 2 + (chi - chi_1)^2 phi theta (chi = ln rho); -Lap u = f with
    rho^2 Lap u = u_chichi + u_chi + u_phiphi + cot(phi) u_phi + u_thetatheta / sin^2(phi)."""
    mesh = vertex_mesh(N, W, mu=mu)
    chi1 = float(mesh.elem_lo[0, 2])

    def u(ps, ts, rs):
        p, t, r = _sph_grid(ps, ts, rs)
        return 2.0 + (np.log(r) - chi1) ** 2 * p * t

    def f(ps, ts, rs):
        p, t, r = _sph_grid(ps, ts, rs)
        c = np.log(r) - chi1
        lap = 2 * p * t + 2 * c * p * t + c * c * t / np.tan(p)
        return -lap / (r * r)

    return EdgeProblem(mesh, [f], [u], u, None, name="vertex_polynomial", meta=dict(chi1=chi1))


def vertex_batch(Ws, mu=0.15) -> EdgeProblem:
    """Independent copies of Table 6.16's problem with uneven degrees W_p
    (N_p = 2 W_p + 4 layers each) in one batch."""
    base = vertex_poisson_singular(N=2, W=2, mu=mu)
    mesh = concat_edge_meshes([vertex_mesh(2 * int(W) + 4, int(W), mu=mu) for W in Ws])
    return EdgeProblem(mesh, base.f, base.g, base.u_exact, base.grad_exact, name="vertex_batch",
                       meta=dict(Ws=[int(w) for w in Ws]))


# ---------------------------------------------------------------------------
# Vertex-edge neighbourhood (Section 2.3 / eq. 2.28-2.29, 4.5): around the
# edge x3 > 0 leaving a vertex at the origin, the modified coordinates are
# (psi, theta, zeta) = (ln tan phi, theta, ln x3), so r = e^{psi + zeta}
# and x3 = e^zeta; every element is a box in these coordinates
# ---------------------------------------------------------------------------
def vertex_edge_mesh(N, W, mu=0.15, phi_v=PI / 4, delta=1.0, theta=(0.0, 1.5 * PI), J=3) -> EdgeMeshDesc:
    """{0 < x3 < delta, 0 < phi < phi_v, theta_0 < theta < theta_1}: N finite
    layers in psi (tan phi_i = mu^(N+1-i) tan phi_v, i = 1..N+1) x J theta
    sectors x N layers in zeta (x3_k = delta mu^(N+1-k)), degree W in every
    modified coordinate.  Corner sets: for each zeta layer k a polynomial in
    zeta of degree W on psi < psi_1, shared by the theta sectors (code -2 - k,
    the neighbour of face 0 of psi layer 1); and one constant on x3 < x3_1
    (code -2 - N, the neighbour of face 4 of zeta layer 1).  Every other outer
    face is Dirichlet.  Elements are numbered psi layer fastest, then zeta
    layer, then theta sector."""
    psis = np.log(np.tan(phi_v)) + np.log(mu) * np.arange(N, -1, -1, dtype=np.float64)
    zets = np.log(delta) + np.log(mu) * np.arange(N, -1, -1, dtype=np.float64)
    ths = np.linspace(theta[0], theta[1], J + 1)
    E = N * N * J
    lo = np.zeros((E, 3))
    hi = np.zeros((E, 3))
    nbr = -np.ones((E, 6), dtype=np.int32)

    def eid(i, k, j):
        return (j * N + k) * N + i

    for j in range(J):
        for k in range(N):
            for i in range(N):
                e = eid(i, k, j)
                lo[e] = (psis[i], ths[j], zets[k])
                hi[e] = (psis[i + 1], ths[j + 1], zets[k + 1])
                nbr[e, 0] = eid(i - 1, k, j) if i > 0 else -2 - k
                nbr[e, 1] = eid(i + 1, k, j) if i < N - 1 else -1
                nbr[e, 2] = eid(i, k, j - 1) if j > 0 else -1
                nbr[e, 3] = eid(i, k, j + 1) if j < J - 1 else -1
                nbr[e, 4] = eid(i, k - 1, j) if k > 0 else -2 - N
                nbr[e, 5] = eid(i, k + 1, j) if k < N - 1 else -1
    cW = np.array([W] * N + [0], dtype=np.int32)
    clo = np.concatenate([zets[:-1], [zets[0]]])   # the constant: its face zeta = zeta_1
    chi = np.concatenate([zets[1:], [zets[0]]])
    return EdgeMeshDesc(lo, hi, np.full(E, W, dtype=np.int32), nbr, np.zeros(E, dtype=np.int32),
                        cW, clo, chi, np.zeros(N + 1, dtype=np.int32), kind="vertex-edge")


def _ve_grid(ps, ts, zs):
    z, t, p = np.meshgrid(np.asarray(zs, dtype=np.float64), np.asarray(ts, dtype=np.float64),
                          np.asarray(ps, dtype=np.float64), indexing="ij")
    return p, t, z


def vertex_edge_singular(N, W, mu=0.15, alpha=2.0 / 3.0) -> EdgeProblem:
    """Laplace problem with the edge singularity of a re-entrant edge of
    opening 3 pi/2: w = r^alpha sin(alpha theta), alpha = 2/3, harmonic,
    w = 0 on theta = 0 and theta = 3 pi/2, w = g on the other outer faces.
    Data are functions of the modified coordinates on tensor grids
    fun(psis, thetas, zetas) -> [len zetas, len thetas, len psis]; the
    gradient is (w_r, w_theta / r, w_x3)."""
    mesh = vertex_edge_mesh(N, W, mu=mu)

    def w(ps, ts, zs):
        p, t, z = _ve_grid(ps, ts, zs)
        return np.exp(alpha * (p + z)) * np.sin(alpha * t)

    def grad(ps, ts, zs):
        p, t, z = _ve_grid(ps, ts, zs)
        rp = alpha * np.exp((alpha - 1.0) * (p + z))
        return rp * np.sin(alpha * t), rp * np.cos(alpha * t), 0.0 * p

    def f(ps, ts, zs):
        return 0.0 * _ve_grid(ps, ts, zs)[0]

    return EdgeProblem(mesh, [f], [w], w, grad, name="vertex_edge_singular", meta=dict(alpha=alpha))


def vertex_edge_polynomial(N, W, mu=0.15) -> EdgeProblem:
    """A solution inside the discrete space, consistent with both corner kinds:
    u = 2 + (zeta - zeta_1)^2 (zeta + (psi - psi_1)^2 theta): on psi = psi_1 it
    is the polynomial 2 + (zeta - zeta_1)^2 zeta with vanishing psi and theta
    derivatives, on zeta = zeta_1 the constant 2 with vanishing derivatives.
    -Lap u = f with r^2 Lap u = u_psipsi + u_thetatheta
    + e^{2 psi} (u_psipsi - 2 u_psizeta + u_zetazeta + u_psi - u_zeta)."""
    mesh = vertex_edge_mesh(N, W, mu=mu)
    psi1, zet1 = float(mesh.elem_lo[0, 0]), float(mesh.elem_lo[0, 2])

    def u(ps, ts, zs):
        p, t, z = _ve_grid(ps, ts, zs)
        return 2.0 + (z - zet1) ** 2 * (z + (p - psi1) ** 2 * t)

    def f(ps, ts, zs):
        p, t, z = _ve_grid(ps, ts, zs)
        a, b = z - zet1, p - psi1
        u_p = 2.0 * a * a * b * t
        u_pp = 2.0 * a * a * t
        u_tt = 0.0 * p
        u_z = 2.0 * a * (z + b * b * t) + a * a
        u_zz = 2.0 * (z + b * b * t) + 4.0 * a
        u_pz = 4.0 * a * b * t
        k = np.exp(2.0 * p)
        r2lap = u_pp + u_tt + k * (u_pp - 2.0 * u_pz + u_zz + u_p - u_z)
        return -r2lap / np.exp(2.0 * (p + z))

    return EdgeProblem(mesh, [f], [u], u, None, name="vertex_edge_polynomial", meta=dict(psi1=psi1, zeta1=zet1))


def vertex_edge_batch(Ws, mu=0.15) -> EdgeProblem:
    """Independent copies of the vertex-edge Laplace problem with uneven
    degrees W_p (N_p = W_p + 2 layers in psi and in zeta) in one batch."""
    base = vertex_edge_singular(N=2, W=2, mu=mu)
    mesh = concat_edge_meshes([vertex_edge_mesh(int(W) + 2, int(W), mu=mu) for W in Ws])
    return EdgeProblem(mesh, base.f, base.g, base.u_exact, base.grad_exact, name="vertex_edge_batch",
                       meta=dict(Ws=[int(w) for w in Ws]))


# ---------------------------------------------------------------------------
# Curved regular elements: maps from the reference cube (-1,1)^3, each
# returning (x [3, ...], dx/dlambda [3, 3, ...], d^2x/dlambda^2 [3, 3, 3, ...])
# on broadcast arrays of reference coordinates
# ---------------------------------------------------------------------------
def affine_box_map(lo, hi):
    """x = lo + (lambda + 1) (hi - lo) / 2."""
    lo = np.asarray(lo, dtype=np.float64)
    hh = (np.asarray(hi, dtype=np.float64) - lo) / 2.0

    def m(l1, l2, l3):
        l1, l2, l3 = np.broadcast_arrays(l1, l2, l3)
        lam = (l1, l2, l3)
        x = np.stack([lo[k] + (lam[k] + 1.0) * hh[k] for k in range(3)])
        Dx = np.zeros((3, 3) + l1.shape)
        for k in range(3):
            Dx[k, k] = hh[k]
        return x, Dx, np.zeros((3, 3, 3) + l1.shape)
    return m


@dataclass
class CurvedMeshDesc:
    """Elements as reference cubes through maps (x, Dx, D2x) = maps[e](l1, l2, l3);
    face f of e and face f^1 of elem_nbr[e, f] share the face's parametrisation."""
    maps: list
    elem_W: np.ndarray
    elem_nbr: np.ndarray
    n_problem: int = 1

    @property
    def n_elem(self) -> int:
        return len(self.maps)

    @property
    def elem_problem(self) -> np.ndarray:
        return np.zeros(self.n_elem, dtype=np.int32)

    @property
    def elem_lo(self) -> np.ndarray:
        return -np.ones((self.n_elem, 3))

    @property
    def elem_hi(self) -> np.ndarray:
        return np.ones((self.n_elem, 3))


def curved_mesh_of_boxes(desc):
    """The affine maps of a box mesh, its degrees and neighbours."""
    maps = [affine_box_map(desc.elem_lo[e], desc.elem_hi[e]) for e in range(desc.n_elem)]
    return maps, np.asarray(desc.elem_W), np.asarray(desc.elem_nbr)


LPRISM_C = 0.5


def _lprism_side(theta_mid):
    """(s, s') with r_max = 0.5 / s(theta): the side of the L-shaped section
    seen from the re-entrant corner (0.5, 0.5) in direction theta."""
    t = theta_mid % (2 * PI)
    if PI / 2 <= t < 3 * PI / 4:
        return (lambda th: np.sin(th)), (lambda th: np.cos(th))          # y = 1
    if 3 * PI / 4 <= t < 5 * PI / 4:
        return (lambda th: -np.cos(th)), (lambda th: np.sin(th))         # x = 0
    if 5 * PI / 4 <= t < 7 * PI / 4:
        return (lambda th: -np.sin(th)), (lambda th: -np.cos(th))        # y = 0
    return (lambda th: np.cos(th)), (lambda th: -np.sin(th))             # x = 1


def lprism_blend_map(th0, th1, Z=0.25, z0=0.0, z1=1.0):
    """Polar blend of a sector of the L-shaped section ((0,1)^2 minus
    (0.5,1)^2) x (z0, z1) around the re-entrant corner c = (0.5, 0.5):
    x = c + [(1 - t) Z + t r_max(theta)] (cos theta, sin theta), x3 = z, with
    t = (l1 + 1)/2, theta = th0 + (l2 + 1)(th1 - th0)/2, z = z0 + (l3 + 1)(z1 - z0)/2.
    The sector must lie on one side of the square (r_max analytic in it)."""
    s, sp = _lprism_side(0.5 * (th0 + th1))
    dth, dz = th1 - th0, z1 - z0
    fac = (0.5, 0.5 * dth, 0.5 * dz)

    def m(l1, l2, l3):
        l1, l2, l3 = np.broadcast_arrays(l1, l2, l3)
        t = (l1 + 1.0) / 2.0
        th = th0 + (l2 + 1.0) * dth / 2.0
        zz = z0 + (l3 + 1.0) * dz / 2.0
        sv, spv = s(th), sp(th)
        R = 0.5 / sv
        R1 = -0.5 * spv / sv ** 2
        R2 = 0.5 * (2 * spv * spv + sv * sv) / sv ** 3
        rho = (1.0 - t) * Z + t * R
        r1, r2 = t * R1, t * R2
        c, sn = np.cos(th), np.sin(th)
        x = np.stack([LPRISM_C + rho * c, LPRISM_C + rho * sn, zz])
        zero = np.zeros_like(t)
        d = [[(R - Z) * c, r1 * c - rho * sn, zero],
             [(R - Z) * sn, r1 * sn + rho * c, zero],
             [zero, zero, zero + 1.0]]
        Dx = np.stack([np.stack([d[k][a] * fac[a] for a in range(3)]) for k in range(3)])
        h = [[[zero, R1 * c - (R - Z) * sn, zero], [R1 * c - (R - Z) * sn, r2 * c - 2 * r1 * sn - rho * c, zero],
              [zero, zero, zero]],
             [[zero, R1 * sn + (R - Z) * c, zero], [R1 * sn + (R - Z) * c, r2 * sn + 2 * r1 * c - rho * sn, zero],
              [zero, zero, zero]],
             [[zero] * 3, [zero] * 3, [zero] * 3]]
        D2x = np.stack([np.stack([np.stack([h[k][a][b] * fac[a] * fac[b] for b in range(3)]) for a in range(3)])
                        for k in range(3)])
        return x, Dx, D2x
    return m


def lprism_regular(W, Z=0.25, J=6):
    """The regular region of the L-shaped prism around its edge neighbourhood
    of radius Z: J sectors of pi/4 from theta = pi/2 to 2 pi, one element each,
    Laplace with w = r^(2/3) sin(2 theta'/3), theta' = theta - pi/2 measured from
    the re-entrant face (w = 0 on both re-entrant faces).  Every outer face is
    Dirichlet, the circle r = Z (the interface with the edge neighbourhood)
    included.  Returns (maps, elem_W, elem_nbr, u, grad u, f) with pointwise
    data functions of physical coordinates."""
    ths = PI / 2 + np.arange(J + 1) * (1.5 * PI / J)
    maps = [lprism_blend_map(ths[j], ths[j + 1], Z=Z) for j in range(J)]
    nbr = -np.ones((J, 6), dtype=np.int32)
    for j in range(J):
        if j > 0:
            nbr[j, 2] = j - 1
        if j < J - 1:
            nbr[j, 3] = j + 1

    def polar(x, y):
        dx, dy = x - LPRISM_C, y - LPRISM_C
        r = np.hypot(dx, dy)
        th = np.mod(np.arctan2(dy, dx) - PI / 2, 2 * PI)   # theta' in [0, 2 pi)
        return r, th

    def u(x, y, z):
        r, th = polar(x, y)
        return r ** (2.0 / 3.0) * np.sin(2.0 * th / 3.0) + 0 * z

    def grad(x, y, z):
        r, th = polar(x, y)
        ur = 2.0 / 3.0 * r ** (-1.0 / 3.0) * np.sin(2.0 * th / 3.0)
        ut = 2.0 / 3.0 * r ** (-1.0 / 3.0) * np.cos(2.0 * th / 3.0)
        phi = th + PI / 2
        return (ur * np.cos(phi) - ut * np.sin(phi), ur * np.sin(phi) + ut * np.cos(phi), 0 * z)

    def f(x, y, z):
        return 0.0 * (x + y + z)

    return maps, np.full(J, W, dtype=np.int32), nbr, u, grad, f


def lprism_problem(N, W, Z=0.25, mu=0.15, J=6, layer_W=None):
    """The L-shaped prism with the re-entrant-edge solution
    w = r^(2/3) sin(2 theta'/3): the edge neighbourhood r < Z (N layers,
    J sectors of pi/4 in theta' in (0, 3 pi/2), one x3 slab, degree W or
    layer_W[i] in layer i from the edge outward, corner polynomial of degree
    W) and the regular region (J polar-blend sectors, degree W), Dirichlet
    data w on the outer faces.  Config 3 takes N = 6, layer_W =
    (2, 3, 4, 6, 7, 8), W = 8.  Returns (edge problem, regular-region pieces
    of lprism_regular, interface pairs (edge element of the outer layer,
    regular element) sharing the circle r = Z)."""
    mesh = edge_mesh(N, W, mu=mu, Z=Z, theta=(0.0, 1.5 * PI), x3=(0.0, 1.0), I=J, J=1, layer_W=layer_W)

    def w(rs, ts, zs):
        r, t, z = _cyl_grid(rs, ts, zs)
        return r ** (2.0 / 3.0) * np.sin(2.0 * t / 3.0) + 0 * z

    def grad(rs, ts, zs):
        r, t, z = _cyl_grid(rs, ts, zs)
        return (2.0 / 3.0 * r ** (-1.0 / 3.0) * np.sin(2.0 * t / 3.0),
                2.0 / 3.0 * r ** (-1.0 / 3.0) * np.cos(2.0 * t / 3.0), 0 * z)

    def zero(rs, ts, zs):
        return np.zeros((len(zs), len(ts), len(rs)))

    edge = EdgeProblem(mesh, [zero], [w], w, grad, name="lprism_edge")
    regular = lprism_regular(W, Z=Z, J=J)
    pairs = [(j * N + N - 1, j) for j in range(J)]
    return edge, regular, pairs


def edge_crack(N, W, mu=0.15, I=4):
    """Table 6.19's crack problem: Lap u = 0 in the unit cylinder slit along
    theta = 0 (0 < theta < 2 pi, 0 < x3 < 1), u = 0 on both crack faces,
    du/dnu = h on r = 1 and on x3 = 0, 1 (Neumann faces, elem_bc = 1), exact
    w = r^(1/2) sin(theta / 2)."""
    mesh = edge_mesh(N, W, mu=mu, Z=1.0, theta=(0.0, 2 * PI), x3=(0.0, 1.0), I=I, J=1)
    bc = np.zeros((mesh.n_elem, 6), dtype=np.int32)
    for e in range(mesh.n_elem):
        for fi in (1, 4, 5):
            if mesh.elem_nbr[e, fi] == -1:
                bc[e, fi] = 1
    mesh.elem_bc = bc

    def w(rs, ts, zs):
        r, t, z = _cyl_grid(rs, ts, zs)
        return np.sqrt(r) * np.sin(t / 2) + 0 * z

    def grad(rs, ts, zs):
        r, t, z = _cyl_grid(rs, ts, zs)
        return 0.5 / np.sqrt(r) * np.sin(t / 2) + 0 * z, 0.5 / np.sqrt(r) * np.cos(t / 2) + 0 * z, 0 * r * t * z

    def zero(rs, ts, zs):
        return np.zeros((len(zs), len(ts), len(rs)))

    return EdgeProblem(mesh, [zero], [w], w, grad, name="edge_crack", flux=[grad])


def vertex_mixed(N, W, mu=0.15):
    """Table 6.17: -Lap u = f on the spherical wedge of Table 6.16 with
    Dirichlet faces phi = pi/6, pi/3 and theta = 0, 3 pi/2 and the Neumann face
    rho = 1 (elem_bc = 1), exact w = rho^0.1 (1 - rho) sin(2 phi).  The
    gradient (w_rho, w_phi / rho, w_theta / (rho sin phi)) is also the Neumann
    data field."""
    mesh = vertex_mesh(N, W, mu=mu)
    bc = np.zeros((mesh.n_elem, 6), dtype=np.int32)
    for e in range(mesh.n_elem):
        if mesh.elem_nbr[e, 5] == -1:
            bc[e, 5] = 1
    mesh.elem_bc = bc

    def g_(r):
        return r ** 0.1 - r ** 1.1

    def w(ps, ts, rs):
        p, t, r = _sph_grid(ps, ts, rs)
        return g_(r) * np.sin(2 * p) + 0 * t

    def grad(ps, ts, rs):
        p, t, r = _sph_grid(ps, ts, rs)
        gp = 0.1 * r ** -0.9 - 1.1 * r ** 0.1
        return gp * np.sin(2 * p) + 0 * t, g_(r) / r * 2 * np.cos(2 * p) + 0 * t, 0 * p * t * r

    def f(ps, ts, rs):
        p, t, r = _sph_grid(ps, ts, rs)
        radial = 0.11 * r ** -1.9 - 2.31 * r ** -0.9
        ang = 2 * np.cos(p) / np.sin(p) * np.cos(2 * p) - 4 * np.sin(2 * p)
        return -(radial * np.sin(2 * p) + g_(r) / (r * r) * ang) + 0 * t

    return EdgeProblem(mesh, [f], [w], w, grad, name="vertex_mixed", flux=[grad])


def vertex_edge_table_6_20(N, W, mu=0.15, J=3):
    """Table 6.20's solution w = rho^(3/4) (sin phi)^(1/2) sin(theta / 2)
    (vertex, edge and vertex-edge singularities) with f = -Lap w
    = -(9/16) rho^(-5/4) (sin phi)^(1/2) sin(theta / 2), on the vertex-edge
    neighbourhood phi < pi/6, 0 < theta < 3 pi/2, x3 < cos(pi/6) (the cone of
    Table 6.20 truncated by the plane inscribed in its unit sphere: the
    elements here are boxes in (ln tan phi, theta, ln x3)).  Data in modified
    coordinates; gradient (w_r, w_theta / r, w_x3)."""
    mesh = vertex_edge_mesh(N, W, mu=mu, phi_v=PI / 6, delta=np.cos(PI / 6), J=J)

    def parts(ps, ts, zs):
        p, t, z = _ve_grid(ps, ts, zs)
        r, x3 = np.exp(p + z), np.exp(z)
        rho = np.hypot(r, x3)
        return r, t, x3, rho, r / rho

    def w(ps, ts, zs):
        r, t, x3, rho, sphi = parts(ps, ts, zs)
        return rho ** 0.75 * np.sqrt(sphi) * np.sin(t / 2)

    def f(ps, ts, zs):
        r, t, x3, rho, sphi = parts(ps, ts, zs)
        return -9.0 / 16.0 * rho ** -1.25 * np.sqrt(sphi) * np.sin(t / 2)

    def grad(ps, ts, zs):
        # w = r^(1/2) rho^(1/4) sin(theta / 2) in cylindrical coordinates
        r, t, x3, rho, sphi = parts(ps, ts, zs)
        s2, c2 = np.sin(t / 2), np.cos(t / 2)
        w_r = (0.5 * r ** -0.5 * rho ** 0.25 + r ** 0.5 * 0.25 * rho ** -0.75 * r / rho) * s2
        w_t = r ** 0.5 * rho ** 0.25 * 0.5 * c2 / r
        w_z = r ** 0.5 * 0.25 * rho ** -0.75 * x3 / rho * s2
        return w_r, w_t, w_z

    return EdgeProblem(mesh, [f], [w], w, grad, name="vertex_edge_table_6_20")


def vertex_with_edge(N, W, mu=0.15, J=3):
    """A vertex neighbourhood with one re-entrant edge (the thesis's splitting
    of Omega^v into the vertex-edge cone and the rest): the vertex part
    pi/6 < phi < pi/3, rho < 1 and the vertex-edge part phi < pi/6,
    x3 < cos(pi/6) (they meet on the circle phi = pi/6, rho = 1), both with
    0 < theta < 3 pi/2 in J sectors and N layers of ratio mu, degree W;
    Table 6.20's w = rho^(3/4) (sin phi)^(1/2) sin(theta / 2) as the exact
    solution, Dirichlet data w on the outer faces.  Returns (vertex problem
    (data in (phi, theta, rho)), vertex-edge problem (data in
    (ln tan phi, theta, ln x3)), interface pairs (vertex-edge element of the
    outer psi layer, vertex element) sharing the cone phi = pi/6)."""
    vmesh = vertex_mesh(N, W, mu=mu, phi=(PI / 6, PI / 3), theta=(0.0, 1.5 * PI), I=1, J=J)

    def w(ps, ts, rs):
        p, t, r = _sph_grid(ps, ts, rs)
        return r ** 0.75 * np.sqrt(np.sin(p)) * np.sin(t / 2)

    def grad(ps, ts, rs):
        # (w_rho, w_phi / rho, w_theta / (rho sin phi))
        p, t, r = _sph_grid(ps, ts, rs)
        s = np.sin(p)
        return (0.75 * r ** -0.25 * np.sqrt(s) * np.sin(t / 2), r ** -0.25 * 0.5 / np.sqrt(s) * np.cos(p) * np.sin(t / 2),
                r ** -0.25 / np.sqrt(s) * 0.5 * np.cos(t / 2))

    def f(ps, ts, rs):
        p, t, r = _sph_grid(ps, ts, rs)
        return -9.0 / 16.0 * r ** -1.25 * np.sqrt(np.sin(p)) * np.sin(t / 2)

    vertex = EdgeProblem(vmesh, [f], [w], w, grad, name="vertex_with_edge")
    ve = vertex_edge_table_6_20(N, W, mu=mu, J=J)
    pairs = [((j * N + k) * N + (N - 1), j * N + k) for j in range(J) for k in range(N)]
    return vertex, ve, pairs


def vertex_edge_with_edge(N, W, mu=0.15, J=3, phi_v=PI / 6, delta=None):
    """The vertex-edge cone phi < phi_v, x3 < delta and the edge neighbourhood
    above it, r < delta tan(phi_v), delta < x3 < 1 (the thesis's splitting
    along an edge leaving a vertex), both 0 < theta < 3 pi/2 in J sectors,
    N layers of ratio mu, degree W: the edge layers r_i = delta tan(phi_i)
    continue the cone's psi layers across the plane x3 = delta.  Exact
    solution Table 6.20's w = rho^(3/4) (sin phi)^(1/2) sin(theta / 2).
    Returns (vertex-edge problem, edge problem (data in (r, theta, x3)),
    interface pairs (vertex-edge element of the top zeta layer, edge element
    of the first x3 slab))."""
    if delta is None:
        delta = float(np.cos(phi_v))
    ve = vertex_edge_table_6_20(N, W, mu=mu, J=J)
    Z = delta * np.tan(phi_v)
    emesh = edge_mesh(N, W, mu=mu, Z=Z, theta=(0.0, 1.5 * PI), x3=(delta, 1.0), I=J, J=1)

    def w(rs, ts, zs):
        r, t, z = _cyl_grid(rs, ts, zs)
        rho = np.hypot(r, z)
        return np.sqrt(r) * rho ** 0.25 * np.sin(t / 2)

    def grad(rs, ts, zs):
        r, t, z = _cyl_grid(rs, ts, zs)
        rho = np.hypot(r, z)
        s2, c2 = np.sin(t / 2), np.cos(t / 2)
        return ((0.5 / np.sqrt(r) * rho ** 0.25 + np.sqrt(r) * 0.25 * rho ** -0.75 * r / rho) * s2,
                np.sqrt(r) * rho ** 0.25 * 0.5 * c2 / r, np.sqrt(r) * 0.25 * rho ** -0.75 * z / rho * s2)

    def f(rs, ts, zs):
        r, t, z = _cyl_grid(rs, ts, zs)
        rho = np.hypot(r, z)
        return -9.0 / 16.0 * rho ** -1.25 * np.sqrt(r / rho) * np.sin(t / 2)

    edge = EdgeProblem(emesh, [f], [w], w, grad, name="edge_above_cone")
    pairs = [((j * N + (N - 1)) * N + i, j * N + i) for j in range(J) for i in range(N)]
    return ve, edge, pairs


def spherical_shell_map(ph0, ph1, th0, th1, r0, r1):
    """x = rho (sin phi cos theta, sin phi sin theta, cos phi) on the box
    (phi, theta, rho) in [ph0, ph1] x [th0, th1] x [r0, r1] (a curved regular
    element of a spherical shell), from the reference cube."""
    fac = (0.5 * (ph1 - ph0), 0.5 * (th1 - th0), 0.5 * (r1 - r0))

    def m(l1, l2, l3):
        l1, l2, l3 = np.broadcast_arrays(l1, l2, l3)
        p = ph0 + (l1 + 1.0) * fac[0]
        t = th0 + (l2 + 1.0) * fac[1]
        r = r0 + (l3 + 1.0) * fac[2]
        sp, cp, st, ct = np.sin(p), np.cos(p), np.sin(t), np.cos(t)
        x = np.stack([r * sp * ct, r * sp * st, r * cp])
        # d/dphi, d/dtheta, d/drho of each component
        d = [[r * cp * ct, -r * sp * st, sp * ct],
             [r * cp * st, r * sp * ct, sp * st],
             [-r * sp, 0 * r, cp]]
        # second derivatives [k][a][b] in (phi, theta, rho)
        h = [[[-r * sp * ct, -r * cp * st, cp * ct], [-r * cp * st, -r * sp * ct, -sp * st], [cp * ct, -sp * st, 0 * r]],
             [[-r * sp * st, r * cp * ct, cp * st], [r * cp * ct, -r * sp * st, sp * ct], [cp * st, sp * ct, 0 * r]],
             [[-r * cp, 0 * r, -sp], [0 * r, 0 * r, 0 * r], [-sp, 0 * r, 0 * r]]]
        Dx = np.stack([np.stack([d[k][a] * fac[a] for a in range(3)]) for k in range(3)])
        D2x = np.stack([np.stack([np.stack([h[k][a][b] * fac[a] * fac[b] for b in range(3)]) for a in range(3)])
                        for k in range(3)])
        return x, Dx, D2x
    return m


def vertex_with_shell(N, W, mu=0.15, rho_v=0.5, J=3):
    """Table 6.16's wedge pi/6 < phi < pi/3, 0 < theta < 3 pi/2, rho < 1 split
    into the vertex neighbourhood rho < rho_v (N layers of ratio mu, J theta
    sectors, the corner constant) and the spherical shell rho_v < rho < 1 of J
    curved regular elements; exact w = rho^(1/2) sin(phi / 2) (Dirichlet data
    w on the outer faces).  Returns (vertex problem, regular-region pieces
    (maps, degrees, neighbours, w, grad w, f) with pointwise data, interface
    pairs (vertex element of the outer layer, shell element) sharing the
    sphere rho = rho_v)."""
    base = vertex_poisson_singular(N, W, mu=mu)
    rho = [rho_v * mu ** (N + 1 - i) for i in range(1, N + 2)]
    vm = vertex_mesh(N, W, mu=mu, J=J)
    chis = np.log(np.array(rho))
    for e in range(vm.n_elem):
        i = e % N
        vm.elem_lo[e, 2], vm.elem_hi[e, 2] = chis[i], chis[i + 1]
    vertex = EdgeProblem(vm, base.f, base.g, base.u_exact, base.grad_exact, name="vertex_with_shell")
    ths = np.linspace(0.0, 1.5 * PI, J + 1)
    maps = [spherical_shell_map(PI / 6, PI / 3, ths[j], ths[j + 1], rho_v, 1.0) for j in range(J)]
    nbr = -np.ones((J, 6), dtype=np.int32)
    for j in range(J):
        if j > 0:
            nbr[j, 2] = j - 1
        if j < J - 1:
            nbr[j, 3] = j + 1

    def sph(x, y, z):
        r = np.sqrt(x * x + y * y + z * z)
        return r, np.arccos(np.clip(z / r, -1.0, 1.0)), np.mod(np.arctan2(y, x), 2 * PI)

    def u(x, y, z):
        r, p, t = sph(x, y, z)
        return np.sqrt(r) * np.sin(p / 2)

    def grad(x, y, z):
        r, p, t = sph(x, y, z)
        wr, wp = 0.5 / np.sqrt(r) * np.sin(p / 2), 0.5 / np.sqrt(r) * np.cos(p / 2)
        er = (np.sin(p) * np.cos(t), np.sin(p) * np.sin(t), np.cos(p))
        ep = (np.cos(p) * np.cos(t), np.cos(p) * np.sin(t), -np.sin(p))
        return tuple(wr * er[k] + wp * ep[k] for k in range(3))

    def f(x, y, z):
        r, p, t = sph(x, y, z)
        return -0.5 * r ** -1.5 * (np.sin(p / 2) + np.cos(p / 2) / np.tan(p))

    pairs = [(j * N + (N - 1), j) for j in range(J)]
    return vertex, (maps, np.full(J, W, dtype=np.int32), nbr, u, grad, f), pairs
