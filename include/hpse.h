/*
 * hpse.h -- C ABI of the GB300 (sm_103a) library for the hot path of the
 * nonconforming h-p least-squares spectral element method for 3-D elliptic
 * problems (A. Husain, "h-p spectral element methods for three dimensional
 * elliptic problems on non-smooth domains using parallel computers", 2010).
 *
 * The library applies, matrix-free, the normal operator A = S^T M S of the
 * least-squares functional of eq. (4.2), the block-diagonal separable
 * preconditioner of eq. (5.19)-(5.20), and solves A U = b by preconditioned
 * conjugate gradients (Section 5.1, stopping rule of Section 6.1), in FP64 or
 * with FP32 operator applies wrapped in FP64 iterative refinement.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Elements.  Axis-aligned boxes mapped affinely onto the master cube
 *   Q = (-1,1)^3 (the regular region of Section 2.3); degree W per variable,
 *   1 <= W <= HPSE_MAX_W; unknowns are the nodal values on the (W+1)^3
 *   Gauss-Lobatto-Legendre grid, lexicographic with x fastest (Section 5.3:
 *   U_{(W+1)^2 k + (W+1) j + i} = u(x_i, y_j, z_k)).
 * Faces.  Face f = 2*axis + side of an element (axis 0/1/2 = x/y/z, side 0 =
 *   the face lambda_axis = -1, side 1 = lambda_axis = +1).  elem_nbr[6e+f] is
 *   the element across that face, or -1 for a Dirichlet boundary face.
 * Vectors.  A "DOF vector" holds n_rhs right-hand sides back to back:
 *   value of rhs r, element e, node n at  r*ndof + elem_offset(e) + n, where
 *   elem_offset(e) = sum_{e'<e} (W_e'+1)^3 and ndof = hpse_ndof().
 *   Device DOF vectors are caller-owned; FP64 entry points take double*,
 *   precision-selectable ones take double* (HPSE_FP64) or float* (HPSE_FP32).
 * Quadrature points.  Volume data are sampled on each element's (2W+1)^3 GLL
 *   grid, laid out per element as [c][b][a] (x fastest), elements back to
 *   back (hpse_nquad() values per right-hand side).  Dirichlet data are
 *   sampled on each boundary face's (2W+1)^2 GLL grid, [t2][t1] with t1 < t2
 *   the two tangential axes, faces in (element, face) order
 *   (hpse_nface_points() values per right-hand side).  hpse_query_points()
 *   returns the 1-D coordinates that span these grids.
 * Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).  Entry
 *   points that only launch kernels are asynchronous with respect to the host.
 * Errors.  Every entry point returns an hpse_status; nothing aborts or traps
 *   on the device.  Invalid arguments are detected on the host before any
 *   launch.  After HPSE_ERR_CUDA the handle should be destroyed.
 * Ownership.  The library owns the mesh handle, its tables, coefficient
 *   arrays, right-hand side and solver workspaces (all device memory it
 *   allocates at set-up); callers own every vector they pass.
 * Threads.  A handle may be used from one host thread at a time.
 */
#ifndef HPSE_H
#define HPSE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HPSE_MAX_W 10

typedef struct hpse_mesh hpse_mesh;

typedef enum {
  HPSE_OK = 0,
  HPSE_ERR_INVALID_ARG = 1,     /* bad pointer, size, enum or state */
  HPSE_ERR_NONMATCHING_FACE = 2,/* neighbour faces do not coincide (one-to-one matching faces required) */
  HPSE_ERR_DEGREE = 3,          /* W outside [1, HPSE_MAX_W], or unequal W across an interior face */
  HPSE_ERR_BREAKDOWN = 4,       /* PCG breakdown: p^T A p <= 0 or a non-finite scalar */
  HPSE_ERR_NO_CONVERGENCE = 5,  /* iteration cap reached before the tolerance */
  HPSE_ERR_TIMEOUT = 6,         /* wall-clock limit of the solve reached */
  HPSE_ERR_CUDA = 7,            /* a CUDA runtime call failed */
  HPSE_ERR_OOM = 8,             /* device allocation failed */
  HPSE_ERR_NO_DATA = 9,         /* hpse_set_data has not been called */
  HPSE_ERR_CAPACITY = 10        /* sizes beyond the fixed scratch of hpse_h1_error_noalloc */
} hpse_status;

typedef enum { HPSE_FP64 = 0, HPSE_FP32 = 1 } hpse_prec;

/* Preconditioner used by hpse_apply_preconditioner and hpse_pcg_solve. */
typedef enum {
  HPSE_PRECOND_SEPARABLE = 0, /* the C-form of eq. (5.19)-(5.20) (default)          */
  HPSE_PRECOND_BLOCK = 1      /* exact element blocks A_ee of A (set up explicitly) */
} hpse_precond_kind;

typedef enum {
  HPSE_COEF_LAPLACE = 0,  /* L u = -Lap u                       */
  HPSE_COEF_SCALAR = 1,   /* L u = -div(a grad u), a(x) > 0 given with grad a */
  HPSE_COEF_GENERAL = 2   /* L u = sum_ij A_ij u_{x_i x_j} + sum_i b_i u_{x_i} + c u
                             (eq. 2.2 written out, A symmetric; the ten-term form of
                             eq. 5.45 per element), A, b, c given per volume point in
                             hpse_data.op; box elements (HPSE_COORD_CARTESIAN) with
                             W <= 9 (the FP64 instance of W = 10 exceeds shared memory,
                             HPSE_ERR_DEGREE) */
} hpse_coef_kind;

/* Mesh of one or more independent problems (eq. 2.1-2.2: the operator, the
 * Dirichlet face set Gamma^[0]; Section 2.3: elements and faces).  All
 * arrays are host memory, read during hpse_setup_mesh only. */
typedef struct {
  int32_t n_elem;              /* number of box elements (all problems)        */
  int32_t n_problem;           /* independent problems (PCG scalars per (problem, rhs)) */
  int32_t n_rhs;               /* right-hand sides per problem                 */
  int32_t coef_kind;           /* hpse_coef_kind                               */
  const int32_t *elem_W;       /* [n_elem] degree per variable                 */
  const int32_t *elem_problem; /* [n_elem] problem index in [0, n_problem)     */
  const double *elem_lo;       /* [n_elem*3] box lower corner (x, y, z)        */
  const double *elem_hi;       /* [n_elem*3] box upper corner                  */
  const int32_t *elem_nbr;     /* [n_elem*6] neighbour id or -1 (Dirichlet);
                                  HPSE_COORD_EDGE: -2-c on face 0 (tau = lo)
                                  for the corner set c                          */
  /* Edge neighbourhood (Section 2.3; eq. 4.7, 2.34, 2.35).  With
   * HPSE_COORD_EDGE the boxes are given in the modified coordinates
   * (tau, theta, x3) = (ln r, theta, x3) of an edge on the x3 axis, the
   * operator is L^e u = -(u_tautau + u_thetatheta + e^{2 tau} u_x3x3) (r^2 times
   * -Lap; coef_kind must be HPSE_COEF_LAPLACE), the face terms are the
   * anisotropic norms of eq. (2.34) with H and G = sup e^tau, and the corner
   * sets r < r_1 hold one polynomial in x3 each (nodal values on the (W+1)
   * GLL points of the slab of their layer-1 elements), shared by every theta
   * sector; they enter only through the faces r = r_1 (their volumes and other
   * faces have infinite measure).  Unknowns: the elements' (W+1)^3 blocks in
   * element order, then the corner sets' W+1 values.  hpse_query_points
   * returns modified coordinates; the caller samples f and g at
   * r = e^tau, theta, x3 (physical data), the library forms F^e = e^{2 tau} f.
   * hpse_h1_error on a neighbourhood mesh takes the difference of two
   * discrete solutions only (ref given; see hpse_h1_error).  Not supported
   * with a neighbourhood coordinate kind (HPSE_ERR_INVALID_ARG): the adjoint
   * entry points, hpse_h1_error against pointwise data,
   * hpse_h1_error_noalloc. */
  int32_t coord;               /* HPSE_COORD_CARTESIAN (0), _EDGE (1), _VERTEX (2) or _VERTEX_EDGE (3) */
  int32_t n_corner;            /* corner sets (HPSE_COORD_EDGE), else 0            */
  const int32_t *corner_W;     /* [n_corner] degree in x3 (= that of its elements) */
  const int32_t *corner_problem; /* [n_corner] problem index                       */
  /* Outer-face conditions (eq. 2.1, the last sum of eq. 4.2).  face_bc
   * [n_elem*6], on faces with elem_nbr == -1: 0 Dirichlet (u = g), 1 Neumann
   * (du/dnu = h), 2 Robin (du/dnu + gamma u = h); NULL: every outer face
   * Dirichlet.  A Neumann / Robin face measures the outward normal derivative
   * (+ gamma u) minus h in the H^{1/2} norm of the other face terms; its data
   * h replaces g in hpse_set_data at that face's points.  robin_gamma
   * [n_problem] (NULL: 1).  Neumann and Robin faces need box elements and
   * HPSE_COEF_LAPLACE or HPSE_COEF_GENERAL (else HPSE_ERR_INVALID_ARG; with
   * the general operator the face measures the plain normal derivative): the
   * conormal derivative of a variable coefficient is not built. */
  const int32_t *face_bc;
  const double *robin_gamma;
} hpse_mesh_desc;

/* HPSE_COORD_VERTEX (eq. 4.3): boxes in (phi, theta, chi) = (phi, theta, ln rho)
 * of a vertex at the origin, L^v u = -e^{chi/2} sqrt(sin phi) (u_chichi + u_chi +
 * u_phiphi + cot(phi) u_phi + u_thetatheta / sin^2 phi), F^v = e^{5 chi/2}
 * sqrt(sin phi) f, face norms L2 + H^{1/2} in modified coordinates times
 * R = sup e^chi, Dirichlet ||sqrt(R)(u - g)||_{3/2}; the corner sets rho < rho_1
 * hold one constant each (corner_W = 0), neighbour code -2-c on face 4
 * (chi = lo); data sampled at (phi, theta, rho = e^chi).  Same restrictions as
 * HPSE_COORD_EDGE, and no H^1 norm. */
/* HPSE_COORD_VERTEX_EDGE (eq. 2.27-2.29; eq. 4.5): boxes in
 * (psi, theta, zeta) = (ln tan phi, theta, ln x3) where an edge on the x3 axis
 * leaves a vertex at the origin (r = e^{psi + zeta}, x3 = e^zeta).
 * L^{v-e} u = -e^{zeta/2} (u_psipsi + u_thetatheta + e^{2 psi} (u_psipsi
 * - 2 u_psizeta + u_zetazeta + u_psi - u_zeta)) = -e^{zeta/2} r^2 Lap u,
 * F^{v-e} = e^{zeta/2} r^2 f; face norms of eq. (2.27) with E = sup sin phi and
 * F = sup e^zeta ([u] in L2 times F G, G = E on faces zeta = const; the zeta
 * derivative times E); Dirichlet faces: F (u - g) in L2 and the two
 * tangential derivatives of u - g in the norm of eq. (2.27).  Two kinds of
 * corner set: a polynomial in zeta (corner_W = the element degree, nodal on
 * the W+1 GLL points of the zeta layer) on psi < psi_1 of one zeta layer,
 * shared by the theta sectors, code -2-c on face 0 (psi = lo); and the vertex
 * constant (corner_W = 0) on zeta < zeta_1, code -2-c on face 4 (zeta = lo).
 * Data are sampled at the modified coordinates themselves (the caller
 * converts).  Same restrictions as HPSE_COORD_VERTEX. */
/* HPSE_COORD_CURVED (eq. 4.2 on elements M_e(Q) with an analytic map that
 * need not be affine; Section 2.3's regular region next to a neighbourhood):
 * every element is the reference cube Q = (-1,1)^3 mapped by the caller's
 * map (elem_lo, elem_hi are ignored and may be NULL); coef_kind must be
 * HPSE_COEF_LAPLACE (L u = -Lap u in physical coordinates), every outer face
 * Dirichlet (face_bc NULL or all 0), no corner sets.  Face f of e and face
 * f^1 of its neighbour must share the face's parametrisation (the same
 * tangential axes and directions); degrees may differ across faces.  The
 * geometry comes from hpse_set_geometry (before hpse_set_data): the map's
 * first and second derivatives at the volume points and its first
 * derivatives at every face point, sampled by the caller at the reference
 * coordinates of hpse_curved_points.  Volume term: the ten-term form of
 * eq. (5.45) with C_ab = -(1 or 2) g^{ab}, C_a = -Lap lambda_a (g^{ab} =
 * sum_i K_ai K_bi, K = (dx/dlambda)^{-1}, Lap lambda_a from the second
 * derivatives) and weight w |J|.  Face terms on the reference face's
 * (2 max(W, W') + 1)-point grid: the jumps of u and of the physical gradient
 * (each side through its own K) in the L2 and H^{1/2} forms of eq. (5.49);
 * Dirichlet faces: u - g in L2, its reference-tangential derivatives in
 * H^{1/2} (eq. 2.18).  f is sampled at the physical volume points, g at the
 * physical points of the Dirichlet faces (hpse_nface_points, in element,
 * face order, (2W+1)^2 per face).  Not built for curved meshes
 * (HPSE_ERR_INVALID_ARG): the H^1 norm, the adjoint entry points, the
 * conforming correction. */
enum { HPSE_COORD_CARTESIAN = 0, HPSE_COORD_EDGE = 1, HPSE_COORD_VERTEX = 2, HPSE_COORD_VERTEX_EDGE = 3,
       HPSE_COORD_CURVED = 4 };

/* Problem data (Section 4.2: F, g of eq. 4.2).  Host FP64 arrays, copied.
 *   f      [n_rhs][hpse_nquad()]        source at the volume points (required)
 *   a      [hpse_nquad()]               coefficient (HPSE_COEF_SCALAR only)
 *   grad_a [3][hpse_nquad()]            its gradient d a / d x_k (idem)
 *   g      [n_rhs][hpse_nface_points()] Dirichlet data, or NULL for g = 0
 *   op     [10][hpse_nquad()]           the general operator's coefficients at
 *                                       the volume points, in the order A_11,
 *                                       A_22, A_33, A_12, A_23, A_13, b_1, b_2,
 *                                       b_3, c (HPSE_COEF_GENERAL only; finite,
 *                                       else HPSE_ERR_INVALID_ARG)            */
typedef struct {
  const double *f;
  const double *a;
  const double *grad_a;
  const double *g;
  const double *op;
} hpse_data;

typedef struct {
  double tol;          /* relative residual target ||b - A x||_2 <= tol ||b||_2 (Section 6.1) */
  int32_t max_iter;    /* cap on PCG iterations (all sweeps together)              */
  int32_t prec;        /* hpse_prec of the operator applies inside PCG:
                          HPSE_FP64 = plain FP64 PCG;
                          HPSE_FP32 = FP32 applies + FP64 iterative refinement     */
  double inner_tol;    /* HPSE_FP32: refine_mode 0: residual reduction factor of the
                          FP32 iteration between FP64 residual refreshes (delta,
                          in (0,1); otherwise 0.1);
                          refine_mode 1: relative tolerance of each inner solve
                          (> 0; otherwise 1e-4)                                   */
  int32_t max_sweeps;  /* cap on refinement sweeps (HPSE_FP32)                     */
  int32_t check_every; /* PCG iterations per host convergence check (CUDA graph)   */
  int32_t zero_init;   /* 1: start from x = 0 (the input x is ignored)             */
  double time_limit_s; /* wall-clock limit, <= 0 for none                          */
  int32_t refine_mode; /* HPSE_FP32 only.  0: one FP32 PCG whose residual is replaced
                          by the FP64 residual b - A x (x accumulated in FP64) each
                          time it has dropped by inner_tol, search direction kept
                          ("reliable updates"); 1: restarted refinement, a fresh
                          FP32 PCG per FP64 residual                               */
} hpse_solve_opts;

typedef struct {
  int32_t status;        /* hpse_status of the whole solve                         */
  int32_t iterations;    /* PCG iterations performed (max over right-hand sides)   */
  int32_t sweeps;        /* FP64 refinement sweeps (1 for plain FP64)              */
  int32_t applies;       /* operator applies performed (per right-hand side)      */
  double rel_residual;   /* max over rhs of ||b - A x||_2 / ||b||_2, FP64          */
} hpse_solve_report;

/* Build the mesh on `device`: validates the description (matching faces,
 * degrees), builds the GLL / Lagrange / face-norm / preconditioner tables in
 * FP64 on the host, uploads geometry and tables.  Section 2.3 (mesh),
 * Section 5.3 (tables), eq. (5.15)-(5.17) (preconditioner eigenbases).
 * desc and its arrays are read during the call only.  On success *out is a
 * handle owned by the caller until hpse_destroy; on failure *out is NULL and
 * the status says why: HPSE_ERR_INVALID_ARG (pointers, counts, enums, corner
 * codes), HPSE_ERR_NONMATCHING_FACE, HPSE_ERR_DEGREE (W outside [1, 10], or
 * unequal across a face of a neighbourhood mesh), HPSE_ERR_OOM, HPSE_ERR_CUDA.
 * Validation runs before any device call.  Synchronous.  Box meshes may have
 * unequal degrees W, W' across an interior face: its terms are taken on the
 * (2 max(W, W') + 1)-point grid of the face (eq. 4.2), as the nodal forms of
 * the higher degree with both traces interpolated onto its nodes. */
hpse_status hpse_setup_mesh(const hpse_mesh_desc *desc, int device, hpse_mesh **out);

/* Sizes: DOFs per right-hand side; volume points; Dirichlet face points. */
int64_t hpse_ndof(const hpse_mesh *m);
int64_t hpse_nquad(const hpse_mesh *m);
int64_t hpse_nface_points(const hpse_mesh *m);
int32_t hpse_nrhs(const hpse_mesh *m);

/* 1-D coordinates spanning the data grids (host output, caller-allocated):
 *   vol_axes  [sum_e 3*(2W_e+1)]: per element the x, y, z coordinates of its
 *             (2W_e+1)-point GLL rule mapped to the box;
 *   face_norm [n_boundary_faces]: per Dirichlet face (element, face order)
 *             the fixed normal coordinate; its tangential coordinates are the
 *             element's vol_axes along t1 and t2.
 * Either pointer may be NULL. */
hpse_status hpse_query_points(const hpse_mesh *m, double *vol_axes, double *face_norm);
int64_t hpse_n_boundary_faces(const hpse_mesh *m);

/* Curved meshes: the number of face points (every face of every element,
 * (2 max(W, W') + 1)^2 each; -1 for other meshes) and the reference
 * coordinates (lambda_1, lambda_2, lambda_3) of the volume points
 * (vol_ref [nquad][3], element by element, x fastest) and of the face points
 * (face_ref [n][3], element by element, faces 0..5, [t2][t1] with t1 < t2
 * the two tangential axes).  Either pointer may be NULL. */
int64_t hpse_curved_n_face_points(const hpse_mesh *m);
hpse_status hpse_curved_points(const hpse_mesh *m, double *vol_ref, double *face_ref);

/* Curved meshes: the map's derivatives at the points of hpse_curved_points,
 * FP64, both host or both device memory: vol [nquad][27] = dx_k/dlambda_a
 * (row-major [k][a]) then d^2 x_k / dlambda_a dlambda_b ([k][pair], pairs
 * 00, 11, 22, 01, 02, 12); face [n][9] = dx_k/dlambda_a.  Computes the
 * volume coefficients and the face points' K on the device.
 * HPSE_ERR_INVALID_ARG for other meshes, missing arrays, or a point where
 * det(dx/dlambda) <= 0 or a value is not finite (then no data until valid
 * geometry and data are set).  Drops captured solver graphs and the data:
 * hpse_set_data must follow.  Synchronous on `stream`. */
hpse_status hpse_set_geometry(hpse_mesh *m, const double *vol, const double *face, void *stream);

/* Upload data and build b = S^T M d in FP64 on the device (Section 5.3: the
 * right-hand side of the normal equations from the sampled data, eq. 2.1-2.2).
 * The arrays of data are FP64 and either all host or all device (CUDA device
 * or managed) memory; the kind is read from the pointers.  Device data is
 * read on `stream` (ordered after the caller's earlier work there) and the
 * coefficient transform runs in a kernel, so no data crosses to the host.
 * data and its arrays are copied during the call; the call returns after
 * `stream` has finished its work (NULL: the legacy default stream).
 * HPSE_ERR_INVALID_ARG for missing arrays, arrays in different memory kinds,
 * or a coefficient a <= 0 or not finite (ellipticity; with device data the
 * handle then has no data until a valid set is given).  Drops captured solver
 * graphs (they refer to the previous data). */
hpse_status hpse_set_data(hpse_mesh *m, const hpse_data *data, void *stream);

/* y = A u, the normal operator of eq. (4.2) (Section 5.3), for all n_rhs
 * right-hand sides.  u, y: caller-owned device DOF vectors of n_rhs*ndof
 * scalars of the given precision (HPSE_FP64 or HPSE_FP32); u and y must not
 * overlap.  Asynchronous on `stream` (NULL: the legacy default stream).
 * HPSE_ERR_INVALID_ARG (pointers, prec, u == y), HPSE_ERR_NO_DATA before
 * hpse_set_data, HPSE_ERR_CUDA. */
hpse_status hpse_apply_operator(hpse_mesh *m, int32_t prec, const void *u, void *y, void *stream);

/* z = C^{-1} r for all right-hand sides with the selected preconditioner:
 * the separable C-form of eq. (5.19)-(5.20) (C* of eq. 5.30 on edge
 * elements; the exact block on corner sets), or the element blocks after
 * hpse_setup_block_preconditioner / hpse_select_preconditioner.  r, z:
 * caller-owned device DOF vectors (must not overlap).  Asynchronous on
 * `stream`; errors as hpse_apply_operator. */
hpse_status hpse_apply_preconditioner(hpse_mesh *m, int32_t prec, const void *r, void *z, void *stream);

/* Element-block preconditioner (no counterpart in the thesis, which uses the
 * separable C-form of Section 5.2; this is block Jacobi on the same element
 * blocks).  Builds, from the data of the last hpse_set_data, the diagonal
 * block A_ee of the normal operator of eq. (4.2) for every element (volume
 * term and the element's own side of each face term), factors it
 * A_ee = L L^T in FP64 and stores X = L^{-1} (packed lower triangle, FP64 and
 * an FP32 copy); the preconditioner is then z_e = X^T X r_e.  Device memory:
 * 12 n(n+1)/2 bytes per element with n = (W+1)^3 (3.3 GB for 512 elements of
 * W = 8), plus two vectors of n_rhs*ndof and, during the call, one FP64 copy
 * of the blocks and 2 x 64 probe vectors (capped at 2 GB each); from 32
 * right-hand sides on also the FP32 factor as 128 x 128 tiles of X and of X^T
 * for the tensor-core products (8 ceil(n/128)(ceil(n/128)+1) x 16384 bytes per
 * element: 1.38 GB for 512 elements of W = 8).  Selects
 * HPSE_PRECOND_BLOCK on success.  hpse_set_data does not rebuild it (a
 * preconditioner from older data stays symmetric positive definite, only
 * less effective).  Synchronous.  Errors: HPSE_ERR_NO_DATA before
 * hpse_set_data, HPSE_ERR_OOM, HPSE_ERR_BREAKDOWN if a block is not positive
 * definite to FP64 working accuracy (the separable form stays selected). */
hpse_status hpse_setup_block_preconditioner(hpse_mesh *m);

/* Tile shape of the element-block preconditioner's two triangular products,
 * per degree W and precision: hpse_setup_block_preconditioner times every
 * candidate shape for the mesh's right-hand-side count on the factors it has
 * just built (variants 0-2 and 8 for >= 32 right-hand sides, 3-4 for 2..31,
 * 5-7 for one; 2, 4, 6 and 8 in FP32 only) and keeps the fastest.  Variants
 * 0-7 are FP32/FP64 CUDA-core tiles; variant 8 runs both products on the
 * tensor cores (tcgen05, 128 rows x 64 right-hand sides per CTA, each FP32
 * operand split into two TF32 parts, three MMAs per product, FP32
 * accumulation in tensor memory).  hpse_block_tile returns the chosen
 * variant, its tile (rows x right-hand sides per CTA) and, if ms is not NULL,
 * the measured milliseconds of each of the 9 variants (0 for those not tried);
 * HPSE_ERR_NO_DATA before the set-up.  hpse_set_block_tile overrides the
 * choice (HPSE_ERR_INVALID_ARG for a variant that does not exist in that
 * precision, or variant 8 when its tiles were not built).  No counterpart in
 * the thesis. */
hpse_status hpse_block_tile(const hpse_mesh *m, int32_t W, int32_t prec, int32_t *variant, int32_t *tile_rows,
                            int32_t *tile_rhs, float *ms);
hpse_status hpse_set_block_tile(hpse_mesh *m, int32_t W, int32_t prec, int32_t variant);

/* Choose the preconditioner (hpse_precond_kind).  HPSE_PRECOND_BLOCK needs a
 * successful hpse_setup_block_preconditioner (else HPSE_ERR_NO_DATA). */
hpse_status hpse_select_preconditioner(hpse_mesh *m, int32_t kind);

/* Copy the FP64 right-hand side b = S^T M d (device, n_rhs*ndof doubles). */
hpse_status hpse_get_rhs(hpse_mesh *m, double *b, void *stream);

/* Solve A x = b for every right-hand side by PCG (FP64) or by FP32-apply PCG
 * inside FP64 iterative refinement.  x: device FP64 DOF vector (input initial
 * guess unless opts->zero_init, output solution).  Synchronous; the report
 * holds iterations, sweeps and the final FP64 relative residual. */
hpse_status hpse_pcg_solve(hpse_mesh *m, const hpse_solve_opts *opts, double *x,
                           hpse_solve_report *rep, void *stream);

/* Squared H^1 norms in physical coordinates (Section 6.1), per right-hand
 * side, with the (2W+1)^3 GLL rule of each element:
 *   out[2r]   = || u_r - v_r ||_{H^1}^2
 *   out[2r+1] = || v_r ||_{H^1}^2
 * where u is a device FP64 DOF vector and v is either
 *   (ref != NULL) another device FP64 DOF vector, or
 *   (ref == NULL) the function sampled at the volume points: vq (device,
 *   n_rhs*nquad doubles, the values) and gq (device, n_rhs*3*nquad doubles,
 *   d/dx, d/dy, d/dz blocks per rhs).  out: host, 2*n_rhs doubles.  Synchronous.
 * Neighbourhood meshes take ref only (the difference of two discrete
 * solutions) and integrate in physical coordinates through the modified ones:
 *   edge (tau, theta, x3):     e^{2tau} v^2 + v_tau^2 + v_theta^2 + e^{2tau} v_x3^2
 *   vertex (phi, theta, chi):  sin(phi) e^{3chi} v^2 + sin(phi) e^chi (v_chi^2 + v_phi^2)
 *                              + e^chi v_theta^2 / sin(phi)
 *   vertex-edge (psi, theta, zeta): e^{2psi+3zeta} v^2 + e^zeta (v_psi^2 + v_theta^2)
 *                              + e^{2psi+zeta} (v_zeta - v_psi)^2
 * over each element's (2W+1)^3 GLL rule; corner sets exactly in the radial
 * variable (r or rho) and, for a polynomial set, with its own (2W+1)-point GLL
 * rule along the slab (edge: x3, vertex-edge: zeta); constant sets over their
 * whole region (vertex: rho < rho_1; vertex-edge: x3 < x3_1 inside the cone
 * of each theta sector). */
hpse_status hpse_h1_error(hpse_mesh *m, const double *u, const double *ref,
                          const double *vq, const double *gq, double *out, void *stream);

/* Conforming correction (Remark 4.3.0; the construction in the proof of
 * Lemma 3.3.1, Appendix C.1): p = u + delta + epsilon + nu, the nodal
 * solution u corrected to a conforming function in H^1 that vanishes on the
 * Dirichlet faces: delta trilinear to the average of u at every element
 * vertex, epsilon per element edge to the average of u + delta along it
 * (blended bilinearly in the other variables), nu per face to the average of
 * the two traces (blended linearly in the normal variable); target 0 on the
 * Dirichlet boundary.  p stays in the (W+1)^3 nodal space of every element.
 * HPSE_ERR_DEGREE for meshes with unequal degrees across a face.
 * u, p: device FP64 DOF vectors of n_rhs*ndof (p may be u).  Box meshes
 * (HPSE_ERR_INVALID_ARG for neighbourhood kinds).  The first call builds the
 * vertex and edge tables and two scratch vectors on the handle (synchronous);
 * later calls are asynchronous on `stream`. */
hpse_status hpse_conforming_correction(hpse_mesh *m, const double *u, double *p, void *stream);

/* Residual map and its transpose (Section 5.3: the weighted PDE residual of
 * eq. (4.2) collocated on the (2W+1)^3 GLL points), box meshes.
 *   hpse_apply_residual:  z[r][q] = sqrt(w_q J) (L u_r - f_r)(x_q), with
 *                         L u = -a Lap u - grad a . grad u and the data of
 *                         hpse_set_data; u a device DOF vector, z device
 *                         [n_rhs][nquad], both of precision prec.
 *   hpse_apply_transpose: y = S^T z, the exact transpose of u -> z without the
 *                         data term (the backward of the residual map); z and
 *                         y device, of precision prec.
 * prec: HPSE_FP64, or HPSE_FP32 (the sum factorisations in FP32 with the FP64
 * tables and data rounded to FP32).  Asynchronous on `stream`.  Both use a
 * scratch buffer the handle allocates on first use.  HPSE_ERR_INVALID_ARG for
 * neighbourhood meshes, bad pointers or prec; HPSE_ERR_NO_DATA before
 * hpse_set_data. */
hpse_status hpse_apply_residual(hpse_mesh *m, int32_t prec, const void *u, void *z, void *stream);
hpse_status hpse_apply_transpose(hpse_mesh *m, int32_t prec, const void *z, void *y, void *stream);

/* The same volume transpose as hpse_apply_transpose (y = S^T z of the
 * residual map, faces excluded), computed in the integration-by-parts form of
 * eq. (5.45)-(5.48): the point values are interpolated on the (2W+1)-point
 * grid, differentiated there with its differentiation matrix (eq. 5.47) after
 * each term's coefficient is applied, projected onto the nodal basis, and the
 * six faces' boundary terms added.  Equal to hpse_apply_transpose up to
 * rounding (the rule integrates every integrand exactly).  Same arguments,
 * layouts and restrictions as hpse_apply_transpose; HPSE_ERR_DEGREE where the
 * kernel's shared-memory layout does not fit (FP64 with -div(a grad u) at
 * W = 10). */
hpse_status hpse_apply_transpose_ibp(hpse_mesh *m, int32_t prec, const void *z, void *y, void *stream);

/* Point values of a DOF vector (FP64): out[r][0..4][q] = v, dv/dx, dv/dy,
 * dv/dz, Lap v at the volume points (physical coordinates). */
hpse_status hpse_eval_fields(hpse_mesh *m, const double *u, double *out, void *stream);

/* Transpose of point evaluation (FP64): y = sum_q rho[r][q] dv_r(x_q)/dV,
 * rho device [n_rhs][nquad], y a device DOF vector (overwritten). */
hpse_status hpse_apply_eval_transpose(hpse_mesh *m, const double *rho, double *y, void *stream);

/* Transpose of hpse_eval_fields (FP64): y = sum_q sum_k wf[r][k][q]
 * d(field_k v_r)(x_q)/dV over the five fields (v, v_x, v_y, v_z, Lap v); wf
 * device [n_rhs][5][nquad], y a device DOF vector (overwritten).  The backward
 * of the point fields, for second-order adjoints. */
hpse_status hpse_apply_fields_transpose(hpse_mesh *m, const double *wf, double *y, void *stream);

/* w_q J_e at the volume points (device FP64 [nquad]). */
hpse_status hpse_quad_weights(hpse_mesh *m, double *out, void *stream);

/* Replace the right-hand side b by a device FP64 vector (e.g. dJ/du for an
 * adjoint solve A lambda = dJ/du, A being symmetric).  Synchronous. */
hpse_status hpse_set_rhs(hpse_mesh *m, const double *b, void *stream);

/* Gradient of a solution functional J with respect to the data at the volume
 * points, given the point fields (hpse_eval_fields) of the solution u and of
 * the adjoint state lambda (A lambda = dJ/du): out[r][0..4][q] =
 *   dJ/df = wJ L lambda,  dJ/da = wJ (Lap u L lambda + (L u - f) Lap lambda),
 *   dJ/d(d_k a) = wJ (d_k u L lambda + (L u - f) d_k lambda), k = x, y, z.
 * Derivative of -lambda^T (A u - b) with respect to each datum (the volume
 * term of eq. 4.2 is the only one that depends on f and a). */
hpse_status hpse_data_gradient(hpse_mesh *m, const double *ufields, const double *lfields, double *out,
                               void *stream);

/* The same with f taken as 0 (L u in place of L u - f): out = -d/dtheta of
 * lambda^T A(theta) u for fixed u and lambda (symmetric in the two), the
 * derivative of an adjoint solve lambda = A^{-1} g with respect to a, grad a. */
hpse_status hpse_data_gradient_bilinear(hpse_mesh *m, const double *ufields, const double *lfields, double *out,
                                        void *stream);

/* Vector-Jacobian product of hpse_data_gradient (with_f = 1) or of
 * hpse_data_gradient_bilinear (with_f = 0) at every point: given the
 * cotangent obar [n_rhs][5][nquad] of its output, the cotangents of its
 * inputs: ubar, lbar [n_rhs][5][nquad] (the fields of u and of lambda) and
 * dbar [n_rhs][5][nquad] (f, a, d_x a, d_y a, d_z a per rhs; a and grad a
 * are shared by the rhs, so their cotangent is the sum over r; dbar[.][0] is
 * 0 when with_f = 0).  Device FP64 arrays, overwritten.  The pointwise
 * derivatives of the formulas of hpse_data_gradient; with the fields'
 * transpose and two more solves they give Hessian-vector products of a
 * solution functional (second-order adjoint). */
hpse_status hpse_data_gradient_vjp(hpse_mesh *m, int32_t with_f, const double *ufields, const double *lfields,
                                   const double *obar, double *ubar, double *lbar, double *dbar, void *stream);

/* Allocation-free variant of hpse_h1_error (same arguments, same results up
 * to the order of the final per-rhs sums).  The thesis has no counterpart: it
 * exists for callers that cannot call cudaMalloc -- applications whose device
 * memory is owned entirely by another allocator (a framework caching
 * allocator, a fixed arena reserved at start-up) and latency-critical loops
 * that must not incur the device-wide synchronisation of cudaFree.
 * It allocates nothing: its scratch (per-(element, rhs) partial sums, per-rhs
 * results, a table-pointer array) is one file-scope device array of about
 * 2.1 MB that every GPU loading the library holds until process exit.
 * Limits: n_elem * n_rhs <= 131072 and n_rhs <= 4096, else HPSE_ERR_CAPACITY
 * before any device work.  The first call on a device looks up the array's
 * device address on that device.  Every call shares the one array and keeps
 * the previous call's contents; all of it is overwritten before it is read,
 * but calls that overlap on the GPU (other streams, other host threads on the
 * same device) race and must be ordered by the caller.  The call is
 * synchronous (it copies its pointer table in, waits on `stream` and copies
 * the results to `out`, host memory): it must not be made while a stream is
 * being captured into a CUDA graph. */
hpse_status hpse_h1_error_noalloc(hpse_mesh *m, const double *u, const double *ref,
                                  const double *vq, const double *gq, double *out, void *stream);

/* Operator work counters for the loaded mesh: multiply-adds of one apply of A
 * per right-hand side, split into volume and face parts, as implemented. */
hpse_status hpse_work_counts(const hpse_mesh *m, double *vol_macs, double *face_macs);

/* ---- One problem over several GPUs (Section 5.3: each processor evaluates the
 * residuals of its own elements after exchanging element-boundary values with
 * its neighbours, and the PCG scalars are summed over all processors) ----
 *
 * hpse_partition assigns every element of a box mesh (coord
 * HPSE_COORD_CARTESIAN) to one of n_parts parts: within each problem the
 * elements are ordered along the Morton (Z-order) curve of their box centres,
 * the problems follow one another, and the sequence is cut into n_parts
 * contiguous pieces of nearly equal weight (W+1)^3.  owner: host array of
 * n_elem entries, written.  Host only (no device call); deterministic.
 * HPSE_ERR_INVALID_ARG for n_parts < 1, a neighbourhood mesh or bad pointers.
 *
 * A part runs as its own mesh: its elements followed by ghost copies of the
 * elements of other parts that share a face with them (every other face of a
 * ghost is marked Dirichlet); the rows of its own elements in A u are then
 * those of the whole mesh once the ghosts hold the current values.
 * hpse_pack_blocks / hpse_unpack_blocks move whole element blocks between a
 * vector of `m` (n_rhs x ndof, FP64 or FP32 as `prec`) and a contiguous
 * buffer (n_rhs x buf_len): buf[r][buf_off[i] + t] <-> vec[r][block of
 * element items[i]][t], t < (W+1)^3.  items [n] and buf_off [n] are device
 * int32 / int64 arrays (buf_off[i] + the block size of items[i] <= buf_len),
 * vec and buf device memory of the caller.  One launch, asynchronous on
 * `stream` (graph-capturable); no check of the device arrays' contents. */
hpse_status hpse_partition(const hpse_mesh_desc *d, int32_t n_parts, int32_t *owner);
hpse_status hpse_pack_blocks(const hpse_mesh *m, int32_t prec, const int32_t *items, const int64_t *buf_off,
                             int32_t n, int64_t buf_len, const void *vec, void *buf, void *stream);
hpse_status hpse_unpack_blocks(const hpse_mesh *m, int32_t prec, const int32_t *items, const int64_t *buf_off,
                               int32_t n, int64_t buf_len, const void *buf, void *vec, void *stream);

/* Kernel launch parameters: threads per CTA for degree W, precision prec,
 * kernel kind (0 = operator apply, 1 = preconditioner); 0 restores the
 * default.  The operator and separable-preconditioner kernels of this build
 * fix their CTA shapes at compile time, so the setting is recorded and
 * reported but does not change those launches. */
hpse_status hpse_set_block_threads(hpse_mesh *m, int32_t kind, int32_t prec, int32_t W, int32_t threads);
int32_t hpse_get_block_threads(const hpse_mesh *m, int32_t kind, int32_t prec, int32_t W);

/* Kernels launched by this library since the last call (and reset). */
int64_t hpse_kernel_launch_count(int32_t reset);

const char *hpse_status_string(hpse_status s);
void hpse_destroy(hpse_mesh *m);

#ifdef __cplusplus
}
#endif
#endif /* HPSE_H */
