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
    m = wl.box_mesh((2, 1, 1), W=3)
    m.elem_W[1] = 4
    assert _status(api, m) == 3


def test_degenerate_box_and_bad_counts(api):
    m = wl.box_mesh((1, 1, 1), W=3)
    m.elem_hi[0, 2] = m.elem_lo[0, 2]
    assert _status(api, m) == 1
    m = wl.box_mesh((1, 1, 1), W=3)
    assert _status(api, m, n_rhs=0) == 1
    m.elem_problem[0] = 5
    assert _status(api, m) == 1
