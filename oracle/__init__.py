"""CPU oracle for the least-squares h-p spectral element hot path (FP64, numpy).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything from this package.  The
product library never calls it; it shares no code, tables or helpers with the
CUDA path (both take their inputs from ``workloads``, which holds no method
arithmetic).

What it computes, following the thesis (A. Husain, h-p spectral element
methods for three dimensional elliptic problems on non-smooth domains using
parallel computers, 2010):

* ``gll``        -- Gauss-Lobatto-Legendre rules, Lagrange evaluation matrices,
                    the differentiation matrix of eq. (5.47).
* ``functional`` -- the regular-region least-squares functional of eq. (4.2):
                    weighted PDE residual at the (2W+1)^3 GLL points
                    (Section 5.3), jump terms in the L2 and H^{1/2} face norms
                    (eq. 2.17b, discretised as in Section 5.3, eq. 5.49) and
                    Dirichlet terms in the H^{3/2} norm (eq. 2.18); its normal
                    operator A = S^T M S and right-hand side b = S^T M d.
* ``precond``    -- the separable C-form preconditioner (eq. 5.11-5.20) and the
                    H^2 form B of eq. (5.7)/(5.9) (Table 5.1 pin).
* ``pcg``        -- preconditioned conjugate gradients (Section 5.1, Section 6.1
                    stopping rule) and dense Cholesky for tiny meshes.
* ``h1``         -- the relative H^1 error of Section 6.1.
* ``edge``, ``vertex``, ``vertex_edge``
                 -- the functional of the edge (eq. 4.7), vertex (eq. 4.3) and
                    vertex-edge (eq. 2.28-2.29, 4.5) neighbourhoods in their
                    modified coordinates, with their corner sets.
* ``curved``     -- regular elements with a curved (non-affine) map: the chain
                    rule through the map's first and second derivatives.
* ``lprism``     -- the L-shaped prism: the edge neighbourhood next to curved
                    regular elements, joined by the interface terms of the
                    singular side.
* ``vertex_region`` -- a vertex neighbourhood with one re-entrant edge: the
                    vertex part and the vertex-edge cone joined on their cone,
                    one shared corner constant.
* ``ve_edge_region`` -- the vertex-edge cone and the edge neighbourhood above
                    it, joined on the plane x3 = delta.
* ``vertex_shell`` -- a vertex neighbourhood inside a spherical shell of curved
                    regular elements, joined on the sphere.
* ``adjoint``    -- gradients of a solution functional by an adjoint solve.
* ``conforming`` -- the conforming correction of a box-element solution
                    (Remark 4.3.0, Appendix C.1).
* ``ibp``        -- the volume variation in integration-by-parts form
                    (eq. 5.45-5.48), the alternative to the direct transpose.

Every function is written for clarity, not speed.  Where the thesis is silent
or ambiguous, the reading taken is stated in the docstring of the function
that depends on it.
Parity status: every function here is pinned by tests under ``tests/``
(``test_oracle_*.py``) against values the paper prints (Table 5.1),
closed forms, polynomial reproduction and brute-force identities.
"""
