"""Host-side validation of hpse_setup_mesh: failures are reported as status
codes before any device call (runs without a GPU)."""
import numpy as np
import pytest

import workloads as wl


@pytest.fixture(scope="module")
def api():
    from paper_1110_2316_gb300.build import build
    build()
    from paper_1110_2316_gb300 import api as A
    return A


def _status(api, desc, **kw):
    from paper_1110_2316_gb300._lib import HpseError
    try:
        api.Mesh(desc, **kw)
    except HpseError as e:
        return e.status
    return 0


def test_nonmatching_face(api):
    m = wl.box_mesh((2, 1, 1), W=3)
    m.elem_hi[1, 1] = 0.9  # neighbour face is smaller
    assert _status(api, m) == 2


def test_asymmetric_adjacency(api):
    m = wl.box_mesh((2, 1, 1), W=3)
    m.elem_nbr[1, 0] = -1
    assert _status(api, m) == 2


def test_degree_out_of_range(api):
    m = wl.box_mesh((1, 1, 1), W=3)
    m.elem_W[0] = 11
    assert _status(api, m) == 3
    m.elem_W[0] = 0
    assert _status(api, m) == 3


def test_unequal_degree_across_face(api):
    # box meshes take it (the face terms on the higher degree's grid); the
    # neighbourhood meshes do not
    m = wl.box_mesh((2, 1, 1), W=3)
    m.elem_W[1] = 4
    assert _status(api, m) in (0, 7)  # 7: no device here
    e = wl.edge_mesh(2, 3)
    k = int(np.nonzero((np.asarray(e.elem_nbr) >= -1).all(axis=1))[0][0])
    e.elem_W[k] = 4
    assert _status(api, e) == 3


def test_degenerate_box_and_bad_counts(api):
    m = wl.box_mesh((1, 1, 1), W=3)
    m.elem_hi[0, 2] = m.elem_lo[0, 2]
    assert _status(api, m) == 1
    m = wl.box_mesh((1, 1, 1), W=3)
    assert _status(api, m, n_rhs=0) == 1
    m.elem_problem[0] = 5
    assert _status(api, m) == 1


def test_neighbourhood_corner_sets(api):
    # vertex-edge: zeta polynomials through face 0 (degree W), the constant
    # through face 4 (degree 0); any other combination is refused
    assert _status(api, wl.vertex_edge_mesh(2, 3, J=2)) in (0, 7)  # 7: no device here
    m = wl.vertex_edge_mesh(2, 3, J=2)
    m.corner_W[0] = 2                     # polynomial degree differs from its elements'
    assert _status(api, m) == 3
    m = wl.vertex_edge_mesh(2, 3, J=2)
    m.corner_W[-1] = 1                    # the constant must have degree 0
    assert _status(api, m) == 3
    m = wl.vertex_edge_mesh(2, 3, J=2)
    e = int(np.nonzero(m.elem_nbr[:, 4] == -2 - 2)[0][0])
    m.elem_nbr[e, 4] = -2                 # a zeta polynomial entered through face 4
    assert _status(api, m) == 3
    m = wl.vertex_edge_mesh(2, 3, J=2)
    e = int(np.nonzero(m.elem_nbr[:, 0] == -2 - 1)[0][0])
    m.elem_nbr[e, 0] = -2                 # the same polynomial in two zeta layers
    assert _status(api, m) == 2
    # edge meshes take corner sets through face 0 only, vertex meshes through face 4 only
    m = wl.edge_mesh(2, 3)
    m.elem_nbr[0, 4], m.elem_nbr[0, 0] = m.elem_nbr[0, 0], -1
    assert _status(api, m) == 1
    m = wl.vertex_mesh(2, 2)
    m.elem_nbr[0, 0], m.elem_nbr[0, 4] = m.elem_nbr[0, 4], -1
    assert _status(api, m) == 1


def test_neumann_faces_outside_the_built_cases_are_refused(api):
    # Neumann and Robin faces: box meshes of the Laplacian or the general
    # operator only (a variable coefficient's conormal derivative is not
    # built), outer faces only, codes 0-2
    pb = wl.varcoef_robin(n=2, W=2)
    assert _status(api, pb.mesh, coef_kind=api.COEF_SCALAR) == 1
    m = wl.poisson_mixed(n=2, W=3).mesh
    m.elem_bc = m.elem_bc.copy()
    m.elem_bc[0, 1] = 1            # an interior face
    assert _status(api, m) == 1
    m = wl.poisson_mixed(n=2, W=3).mesh
    m.elem_bc = m.elem_bc.copy()
    m.elem_bc[m.elem_bc == 1] = 3  # no such condition
    assert _status(api, m) == 1
    e = wl.edge_mesh(2, 3)
    e.elem_bc = np.zeros((e.n_elem, 6), dtype=np.int32)
    e.elem_bc[np.asarray(e.elem_nbr) == -1] = 1
    assert _status(api, e) == 1


def test_general_operator_outside_the_built_cases_is_refused(api):
    from types import SimpleNamespace
    # a problem with the general operator needs a COEF_GENERAL mesh, and back
    with pytest.raises(ValueError):
        api.problem_data_arrays(SimpleNamespace(coef_kind=api.COEF_LAPLACE), wl.helmholtz_mixed(n=2, W=2))
    with pytest.raises(ValueError):
        api.problem_data_arrays(SimpleNamespace(coef_kind=api.COEF_GENERAL), wl.poisson_mixed(n=2, W=2))
    # box elements only (the neighbourhoods' modified operators are the Laplacian's)
    assert _status(api, wl.edge_mesh(2, 3), coef_kind=api.COEF_GENERAL) == 1
    # W = 10: the FP64 kernel's shared-memory layout does not fit (HPSE_ERR_DEGREE)
    assert _status(api, wl.box_mesh(1, W=10), coef_kind=api.COEF_GENERAL) == 3
    # an unknown kind
    assert _status(api, wl.box_mesh(1, W=2), coef_kind=7) == 1
