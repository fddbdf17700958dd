"""Python binding of the hpse C ABI (include/hpse.h): argument marshalling only.

Every numerical step runs in the CUDA library; this module converts numpy /
torch arguments to pointers and sizes and checks the returned status.
Device vectors are torch CUDA tensors (float64 or float32, contiguous) of
n_rhs * ndof entries in the layout of include/hpse.h; the current torch CUDA
stream is passed to the library.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import COEF_GENERAL, COEF_LAPLACE, COEF_SCALAR, FP32, FP64, PRECOND_BLOCK, PRECOND_SEPARABLE, check

__all__ = ["Mesh", "problem_data_arrays", "FP64", "FP32", "COEF_LAPLACE", "COEF_SCALAR", "COEF_GENERAL", "PRECOND_SEPARABLE",
           "PRECOND_BLOCK"]


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p)
    return C.c_void_p(a.data_ptr())  # torch tensor


def _stream(stream=None):
    if stream is not None:
        return C.c_void_p(stream)
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _prec_of(t):
    import torch
    if t.dtype == torch.float64:
        return FP64
    if t.dtype == torch.float32:
        return FP32
    raise TypeError("device vectors must be float64 or float32, got %s" % t.dtype)


class Mesh:
    """Handle of hpse_setup_mesh for a batch of box-element problems.

    ``desc`` provides elem_lo [E,3], elem_hi [E,3], elem_W [E], elem_nbr [E,6],
    elem_problem [E] and n_problem (e.g. workloads.MeshDesc).
    """

    def __init__(self, desc, n_rhs=1, coef_kind=COEF_LAPLACE, device=0, robin_gamma=None):
        """``desc.elem_bc`` (optional, [E,6]): 0 Dirichlet, 1 Neumann, 2 Robin
        on outer faces; ``robin_gamma``: the Robin gamma, one per problem or a
        scalar (default 1)."""
        self._lib = _lib.load()
        self._keep = [np.ascontiguousarray(desc.elem_W, dtype=np.int32),
                      np.ascontiguousarray(desc.elem_problem, dtype=np.int32),
                      np.ascontiguousarray(desc.elem_lo, dtype=np.float64),
                      np.ascontiguousarray(desc.elem_hi, dtype=np.float64),
                      np.ascontiguousarray(desc.elem_nbr, dtype=np.int32)]
        d = _lib.MeshDesc()
        d.n_elem = int(self._keep[0].shape[0])
        d.n_problem = int(desc.n_problem)
        d.n_rhs = int(n_rhs)
        d.coef_kind = int(coef_kind)
        d.elem_W, d.elem_problem, d.elem_lo, d.elem_hi, d.elem_nbr = (
            k.ctypes.data_as(C.c_void_p) for k in self._keep)
        # curved elements (workloads.CurvedMeshDesc): reference cubes through the caller's maps
        self.is_curved = hasattr(desc, "maps")
        # edge neighbourhood (workloads.EdgeMeshDesc): modified coordinates + corner sets
        self.is_edge = hasattr(desc, "corner_W")
        if self.is_edge:
            self._keep += [np.ascontiguousarray(desc.corner_W, dtype=np.int32),
                           np.ascontiguousarray(desc.corner_problem, dtype=np.int32)]
            d.coord = {"edge": _lib.COORD_EDGE, "vertex": _lib.COORD_VERTEX,
                       "vertex-edge": _lib.COORD_VERTEX_EDGE}[getattr(desc, "kind", "edge")]
            self.nbhd_kind = getattr(desc, "kind", "edge")
            d.n_corner = int(self._keep[5].shape[0])
            d.corner_W = self._keep[5].ctypes.data_as(C.c_void_p)
            d.corner_problem = self._keep[6].ctypes.data_as(C.c_void_p)
        else:
            d.coord = _lib.COORD_CURVED if self.is_curved else _lib.COORD_CARTESIAN
            d.n_corner = 0
        bc = getattr(desc, "elem_bc", None)
        self.face_bc = None
        if bc is not None and np.any(np.asarray(bc) != 0):
            self.face_bc = np.ascontiguousarray(bc, dtype=np.int32).reshape(-1, 6)
            gam = np.broadcast_to(np.asarray(1.0 if robin_gamma is None else robin_gamma, dtype=np.float64),
                                  (int(desc.n_problem),))
            self.robin_gamma = np.ascontiguousarray(gam)
            self._keep += [self.face_bc, self.robin_gamma]
            d.face_bc = self._keep[-2].ctypes.data_as(C.c_void_p)
            d.robin_gamma = self._keep[-1].ctypes.data_as(C.c_void_p)
        h = C.c_void_p()
        check(self._lib.hpse_setup_mesh(C.byref(d), int(device), C.byref(h)), "hpse_setup_mesh")
        self._h = h
        self.n_elem = d.n_elem
        self.n_rhs = int(n_rhs)
        self.n_problem = int(desc.n_problem)
        self.coef_kind = int(coef_kind)
        self.elem_W = self._keep[0]
        self.device = device
        # bumped by every set_data (the operator's coefficients and f): the
        # autograd functions check it; set_rhs changes only b
        self.data_version = 0

    # -- sizes ------------------------------------------------------------
    @property
    def ndof(self) -> int:
        return int(self._lib.hpse_ndof(self._h))

    @property
    def nquad(self) -> int:
        return int(self._lib.hpse_nquad(self._h))

    @property
    def nface_points(self) -> int:
        return int(self._lib.hpse_nface_points(self._h))

    @property
    def n_boundary_faces(self) -> int:
        return int(self._lib.hpse_n_boundary_faces(self._h))

    def query_points(self):
        """(vol_axes [sum 3Q], face_norm [n_boundary_faces]) of hpse_query_points."""
        nax = int(sum(3 * (2 * int(w) + 1) for w in self.elem_W))
        ax = np.zeros(nax)
        fn = np.zeros(max(1, self.n_boundary_faces))
        check(self._lib.hpse_query_points(self._h, _ptr(ax), _ptr(fn)), "hpse_query_points")
        return ax, fn[: self.n_boundary_faces]

    # -- curved elements -----------------------------------------------------
    def curved_points(self):
        """(vol_ref [nquad, 3], face_ref [n, 3]) reference coordinates of the
        volume points and of every element face's points."""
        nf = int(self._lib.hpse_curved_n_face_points(self._h))
        vol = np.zeros((max(self.nquad, 1), 3))
        face = np.zeros((max(nf, 1), 3))
        check(self._lib.hpse_curved_points(self._h, _ptr(vol), _ptr(face)), "hpse_curved_points")
        return vol[: self.nquad], face[:nf]

    def set_geometry(self, vol, face, stream=None):
        """The maps' derivatives at curved_points (host arrays or CUDA tensors):
        vol [nquad, 27], face [n, 9]."""
        if not isinstance(vol, np.ndarray) and getattr(vol, "is_cuda", False):
            vol, face = vol.detach().double().contiguous(), face.detach().double().contiguous()
        else:
            vol, face = np.ascontiguousarray(vol, dtype=np.float64), np.ascontiguousarray(face, dtype=np.float64)
        self.data_version += 1
        check(self._lib.hpse_set_geometry(self._h, _ptr(vol), _ptr(face), _stream(stream)), "hpse_set_geometry")

    # -- data ---------------------------------------------------------------
    def set_data(self, f, a=None, grad_a=None, g=None, op=None, stream=None):
        """Data at the query points: numpy arrays (host) or CUDA float64 torch
        tensors (device, read on the current torch stream); not mixed.  ``op``
        [10, nquad]: the general operator's A_11, A_22, A_33, A_12, A_23,
        A_13, b_1, b_2, b_3, c (COEF_GENERAL)."""
        vals = (f, a, grad_a, g, op)
        on_dev = [v is not None and not isinstance(v, np.ndarray) and getattr(v, "is_cuda", False) for v in vals]
        if any(on_dev):
            import torch
            if not all(d for v, d in zip(vals, on_dev) if v is not None):
                raise TypeError("set_data: give all data as host arrays or all as CUDA tensors")
            arrs = [None if v is None else v.detach().to(torch.float64).contiguous() for v in vals]
        else:
            arrs = [None if v is None else np.ascontiguousarray(v, dtype=np.float64) for v in vals]
        d = _lib.Data(*[_ptr(v) for v in arrs])
        self.data_version += 1
        check(self._lib.hpse_set_data(self._h, C.byref(d), _stream(stream)), "hpse_set_data")

    # -- preconditioner choice ------------------------------------------------
    def setup_block_preconditioner(self):
        """Build and select the element-block preconditioner from the current data."""
        check(self._lib.hpse_setup_block_preconditioner(self._h), "hpse_setup_block_preconditioner")

    def block_tile(self, W, prec):
        """(variant, (tile rows, tile rhs), ms per variant) chosen by the autotuner."""
        v, tr, tc = C.c_int32(), C.c_int32(), C.c_int32()
        ms = np.zeros(9, dtype=np.float32)
        check(self._lib.hpse_block_tile(self._h, int(W), int(prec), C.byref(v), C.byref(tr), C.byref(tc),
                                        ms.ctypes.data_as(C.c_void_p)), "hpse_block_tile")
        return int(v.value), (int(tr.value), int(tc.value)), ms

    def set_block_tile(self, W, prec, variant):
        check(self._lib.hpse_set_block_tile(self._h, int(W), int(prec), int(variant)), "hpse_set_block_tile")

    def select_preconditioner(self, kind):
        check(self._lib.hpse_select_preconditioner(self._h, int(kind)), "hpse_select_preconditioner")

    def get_rhs(self, b, stream=None):
        check(self._lib.hpse_get_rhs(self._h, _ptr(b), _stream(stream)), "hpse_get_rhs")

    # -- operators -----------------------------------------------------------
    def apply_operator(self, u, y, stream=None):
        check(self._lib.hpse_apply_operator(self._h, _prec_of(u), _ptr(u), _ptr(y), _stream(stream)),
              "hpse_apply_operator")

    def apply_preconditioner(self, r, z, stream=None):
        check(self._lib.hpse_apply_preconditioner(self._h, _prec_of(r), _ptr(r), _ptr(z), _stream(stream)),
              "hpse_apply_preconditioner")

    def pcg_solve(self, x, tol=1e-10, prec=FP64, max_iter=20000, inner_tol=0.0, max_sweeps=200,
                  check_every=16, zero_init=True, time_limit_s=0.0, refine_mode=0, stream=None,
                  raise_on_error=True):
        # inner_tol 0 selects the library default of the refinement mode
        o = _lib.SolveOpts(float(tol), int(max_iter), int(prec), float(inner_tol), int(max_sweeps),
                           int(check_every), 1 if zero_init else 0, float(time_limit_s), int(refine_mode))
        rep = _lib.SolveReport()
        st = self._lib.hpse_pcg_solve(self._h, C.byref(o), _ptr(x), C.byref(rep), _stream(stream))
        out = dict(status=int(rep.status), iterations=int(rep.iterations), sweeps=int(rep.sweeps),
                   applies=int(rep.applies), rel_residual=float(rep.rel_residual))
        if raise_on_error:
            check(st, "hpse_pcg_solve")
        return out

    def h1_error(self, u, ref=None, vq=None, gq=None, stream=None):
        """[n_rhs, 2] array of (||u - v||_{H1}^2, ||v||_{H1}^2)."""
        out = np.zeros(2 * self.n_rhs)
        check(self._lib.hpse_h1_error(self._h, _ptr(u), _ptr(ref), _ptr(vq), _ptr(gq), _ptr(out),
                                      _stream(stream)), "hpse_h1_error")
        return out.reshape(self.n_rhs, 2)

    def conforming_correction(self, u, p, stream=None):
        """p = the conforming correction of the FP64 solution u (box meshes)."""
        check(self._lib.hpse_conforming_correction(self._h, _ptr(u), _ptr(p), _stream(stream)),
              "hpse_conforming_correction")

    # -- residual map, point fields and adjoint data gradients (FP64) -------
    def apply_residual(self, u, z, stream=None):
        check(self._lib.hpse_apply_residual(self._h, _prec_of(u), _ptr(u), _ptr(z), _stream(stream)),
              "hpse_apply_residual")

    def apply_transpose(self, z, y, stream=None):
        check(self._lib.hpse_apply_transpose(self._h, _prec_of(z), _ptr(z), _ptr(y), _stream(stream)),
              "hpse_apply_transpose")

    def apply_transpose_ibp(self, z, y, stream=None):
        """y = S^T z in the integration-by-parts form of eq. (5.45)-(5.48)."""
        check(self._lib.hpse_apply_transpose_ibp(self._h, _prec_of(z), _ptr(z), _ptr(y), _stream(stream)),
              "hpse_apply_transpose_ibp")

    def eval_fields(self, u, out, stream=None):
        check(self._lib.hpse_eval_fields(self._h, _ptr(u), _ptr(out), _stream(stream)), "hpse_eval_fields")

    def apply_eval_transpose(self, rho, y, stream=None):
        check(self._lib.hpse_apply_eval_transpose(self._h, _ptr(rho), _ptr(y), _stream(stream)),
              "hpse_apply_eval_transpose")

    def quad_weights(self, out, stream=None):
        check(self._lib.hpse_quad_weights(self._h, _ptr(out), _stream(stream)), "hpse_quad_weights")

    def set_rhs(self, b, stream=None):
        check(self._lib.hpse_set_rhs(self._h, _ptr(b), _stream(stream)), "hpse_set_rhs")

    def data_gradient(self, ufields, lfields, out, stream=None):
        check(self._lib.hpse_data_gradient(self._h, _ptr(ufields), _ptr(lfields), _ptr(out), _stream(stream)),
              "hpse_data_gradient")

    def data_gradient_bilinear(self, ufields, lfields, out, stream=None):
        check(self._lib.hpse_data_gradient_bilinear(self._h, _ptr(ufields), _ptr(lfields), _ptr(out),
                                                    _stream(stream)), "hpse_data_gradient_bilinear")

    def data_gradient_vjp(self, with_f, ufields, lfields, obar, ubar, lbar, dbar, stream=None):
        check(self._lib.hpse_data_gradient_vjp(self._h, 1 if with_f else 0, _ptr(ufields), _ptr(lfields),
                                               _ptr(obar), _ptr(ubar), _ptr(lbar), _ptr(dbar), _stream(stream)),
              "hpse_data_gradient_vjp")

    def apply_fields_transpose(self, wf, y, stream=None):
        check(self._lib.hpse_apply_fields_transpose(self._h, _ptr(wf), _ptr(y), _stream(stream)),
              "hpse_apply_fields_transpose")

    def work_counts(self):
        v, f = C.c_double(), C.c_double()
        check(self._lib.hpse_work_counts(self._h, C.byref(v), C.byref(f)), "hpse_work_counts")
        return v.value, f.value

    def set_block_threads(self, kind, prec, W, threads):
        check(self._lib.hpse_set_block_threads(self._h, kind, prec, W, threads), "hpse_set_block_threads")

    def get_block_threads(self, kind, prec, W):
        return int(self._lib.hpse_get_block_threads(self._h, kind, prec, W))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hpse_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_launch_count(reset=False) -> int:
    return int(_lib.load().hpse_kernel_launch_count(1 if reset else 0))


_PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def curved_geometry_arrays(mesh: Mesh, maps):
    """Sample the elements' maps at the library's reference points.

    ``maps[e](l1, l2, l3) -> (x [3, ...], Dx [3, 3, ...], D2x [3, 3, 3, ...])``
    (Dx[k, a] = d x_k / d lambda_a).  Returns (vol [nquad, 27], face [n, 9],
    x_vol [nquad, 3], x_face [n, 3]) for Mesh.set_geometry and the data."""
    vref, fref = mesh.curved_points()
    Ws = [int(w) for w in mesh.elem_W]
    nbr = mesh._keep[4]
    vol = np.zeros((len(vref), 27))
    xv = np.zeros((len(vref), 3))
    o = 0
    for e, W in enumerate(Ws):
        n = (2 * W + 1) ** 3
        r = vref[o:o + n]
        x, Dx, D2x = maps[e](r[:, 0], r[:, 1], r[:, 2])
        xv[o:o + n] = np.asarray(x).T
        vol[o:o + n, :9] = np.asarray(Dx).reshape(9, n).T
        for k in range(3):
            for p, (a, b) in enumerate(_PAIRS):
                vol[o:o + n, 9 + 6 * k + p] = D2x[k, a, b]
        o += n
    face = np.zeros((len(fref), 9))
    xf = np.zeros((len(fref), 3))
    o = 0
    for e, W in enumerate(Ws):
        for f in range(6):
            nb = int(nbr[e, f])
            Qf = 2 * (max(W, Ws[nb]) if nb >= 0 else W) + 1
            n = Qf * Qf
            r = fref[o:o + n]
            x, Dx, _ = maps[e](r[:, 0], r[:, 1], r[:, 2])
            xf[o:o + n] = np.asarray(x).T
            face[o:o + n] = np.asarray(Dx).reshape(9, n).T
            o += n
    return vol, face, xv, xf


def curved_data_arrays(mesh: Mesh, x_vol, x_face, f, g):
    """Data of a curved mesh: f[r](x, y, z), g[r](x, y, z) pointwise functions
    of physical coordinates (one per rhs), sampled at the volume points and at
    the Dirichlet faces' points (element, face order)."""
    Ws = [int(w) for w in mesh.elem_W]
    nbr = mesh._keep[4]
    R = mesh.n_rhs
    F = np.stack([np.asarray(f[r](x_vol[:, 0], x_vol[:, 1], x_vol[:, 2]), dtype=np.float64) * np.ones(len(x_vol))
                  for r in range(R)])
    rows = []
    o = 0
    for e, W in enumerate(Ws):
        for fi in range(6):
            nb = int(nbr[e, fi])
            Qf = 2 * (max(W, Ws[nb]) if nb >= 0 else W) + 1
            if nb == -1:
                rows.append(np.arange(o, o + Qf * Qf))
            o += Qf * Qf
    idx = np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64)
    xb = x_face[idx]
    G = np.stack([np.asarray(g[r](xb[:, 0], xb[:, 1], xb[:, 2]), dtype=np.float64) * np.ones(len(xb))
                  for r in range(R)]) if len(idx) else None
    return dict(f=F, g=G)


def problem_data_arrays(mesh: Mesh, problem):
    """Sample a problem's data functions on the mesh's query grids.

    ``problem`` provides f (list per rhs), g (list per rhs), a / grad_a (or
    None) as callables on tensor grids (see workloads), or op (the general
    operator of eq. 2.2: (A, b, c) on tensor grids, for a COEF_GENERAL mesh).
    Returns the dict of host arrays expected by Mesh.set_data.  For an edge neighbourhood the
    query grids are modified coordinates (tau, theta, x3) and the data
    functions take cylindrical coordinates: they are sampled at r = e^tau;
    for a vertex neighbourhood at rho = e^chi; a vertex-edge neighbourhood's
    data functions take its modified coordinates themselves.
    """
    general = getattr(problem, "op", None) is not None or any(
        getattr(p, "op", None) is not None for p in (getattr(problem, "parts", None) or []))
    if general and mesh.coef_kind != COEF_GENERAL:
        raise ValueError("a problem with the general operator of eq. (2.2) needs a COEF_GENERAL mesh")
    if mesh.coef_kind == COEF_GENERAL and not general:
        raise ValueError("a COEF_GENERAL mesh needs the problem's general operator (op)")
    if getattr(mesh, "is_edge", False):
        if mesh.nbhd_kind == "vertex":   # (phi, theta, ln rho): sample at rho = e^chi
            def cyl(fun):
                return lambda ps, hs, cs: fun(ps, hs, np.exp(cs))
        elif mesh.nbhd_kind == "vertex-edge":  # data given in (ln tan phi, theta, ln x3)
            def cyl(fun):
                return fun
        else:                            # (ln r, theta, x3): sample at r = e^tau
            def cyl(fun):
                return lambda ts, hs, zs: fun(np.exp(ts), hs, zs)
        from types import SimpleNamespace
        problem = SimpleNamespace(f=[cyl(v) for v in problem.f], g=[cyl(v) for v in problem.g], a=None,
                                  grad_a=None)
    ax, fnorm = mesh.query_points()
    Ws = [int(w) for w in mesh.elem_W]
    R = mesh.n_rhs
    nq = mesh.nquad
    parts = getattr(problem, "parts", None)
    eprob = mesh._keep[1]

    def part(e):
        return parts[int(eprob[e])] if parts is not None else problem

    f = np.zeros((R, nq))
    a = grad = op = None
    if general:
        op = np.zeros((10, nq))
    elif problem.a is not None:
        a = np.zeros(nq)
        grad = np.zeros((3, nq))
    axes = []
    o = oq = 0
    for e, W in enumerate(Ws):
        Q = 2 * W + 1
        xs, ys, zs = ax[o:o + Q], ax[o + Q:o + 2 * Q], ax[o + 2 * Q:o + 3 * Q]
        axes.append((xs, ys, zs))
        o += 3 * Q
        n = Q ** 3
        pe = part(e)
        for r in range(R):
            f[r, oq:oq + n] = np.broadcast_to(pe.f[r](xs, ys, zs), (Q, Q, Q)).ravel()
        if op is not None:
            A_, b_, c_ = pe.op(xs, ys, zs)
            vals = [A_[0][0], A_[1][1], A_[2][2], A_[0][1], A_[1][2], A_[0][2], b_[0], b_[1], b_[2], c_]
            for k, v in enumerate(vals):
                op[k, oq:oq + n] = np.broadcast_to(np.asarray(v, dtype=np.float64), (Q, Q, Q)).ravel()
        if a is not None:
            a[oq:oq + n] = np.broadcast_to(pe.a(xs, ys, zs), (Q, Q, Q)).ravel()
            gx, gy, gz = pe.grad_a(xs, ys, zs)
            grad[0, oq:oq + n] = np.broadcast_to(gx, (Q, Q, Q)).ravel()
            grad[1, oq:oq + n] = np.broadcast_to(gy, (Q, Q, Q)).ravel()
            grad[2, oq:oq + n] = np.broadcast_to(gz, (Q, Q, Q)).ravel()
        oq += n
    g = None
    nfp = mesh.nface_points
    if nfp > 0:
        g = np.zeros((R, nfp))
        nbr = mesh._keep[4]
        fo = 0
        k = 0
        for e, W in enumerate(Ws):
            Q = 2 * W + 1
            for fi in range(6):
                if nbr[e, fi] != -1:
                    continue
                axis = fi // 2
                grid = list(axes[e])
                grid[axis] = np.array([fnorm[k]])
                bc = 0 if getattr(mesh, "face_bc", None) is None else int(mesh.face_bc[e, fi])
                for r in range(R):
                    if bc == 0:
                        g[r, fo:fo + Q * Q] = part(e).g[r](*grid).ravel()
                    else:
                        # Neumann / Robin data h = nu . q (+ gamma g) from the conormal field q
                        q = part(e).flux[r](*grid)[axis]
                        shape = (len(grid[2]), len(grid[1]), len(grid[0]))
                        h = (1.0 if fi % 2 else -1.0) * np.broadcast_to(q, shape)
                        if bc == 2:
                            gam = float(mesh.robin_gamma[int(eprob[e])])
                            h = h + gam * np.broadcast_to(part(e).g[r](*grid), shape)
                        g[r, fo:fo + Q * Q] = h.ravel()
                fo += Q * Q
                k += 1
    out = dict(f=f, a=a, grad_a=grad, g=g)
    if op is not None:
        out["op"] = op
    return out
