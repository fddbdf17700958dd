// registry.h -- interface between the host library and the per-(precision,
// degree) kernel translation units.  Each unit compiles kernels.cuh for one
// (REAL, WDEG) pair and fills a KernelSet with launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hpse {

// COEF_EDGE: -(u_11 + u_22 + kappa(x_1) u_33) in the edge neighbourhood's
// modified coordinates, kappa = e^{2 tau} per x-point of the element
// COEF_VERTEX: the variable-coefficient form with per-point weights and
// first-order terms, u_22 scaled by 1/sin^2(x_1) per x-point (vertex
// neighbourhood, modified coordinates (phi, theta, ln rho))
// COEF_VERTEX_EDGE: the variable-coefficient form with the mixed term u_13 in
// place of u_2 (vertex-edge neighbourhood, (ln tan phi, theta, ln x3)):
// per-point m and coefficients of (u_1, u_13, u_3), u_11 scaled by 1 + kappa
// and u_33 by kappa per x-point, kappa = e^{2 psi}
// COEF_GENERAL: the ten-term operator of eq. (5.45) with per-point
// coefficients (weight and C's, GEN_NC = 12 per point; general.cuh)
enum { COEF_LAPLACE = 0, COEF_SCALAR = 1, COEF_EDGE = 2, COEF_VERTEX = 3, COEF_VERTEX_EDGE = 4, COEF_GENERAL = 5 };
// KAPPA_STRIDE = 2 * HPSE_MAX_W + 1, CSCR_STRIDE = HPSE_MAX_W + 1 (checked in the host library)
enum { KAPPA_STRIDE = 21, CSCR_STRIDE = 11, FACE_W = 10, ZEIG_STRIDE = 132 };
enum { MODE_PLAIN = 0, MODE_PCG = 1, MODE_TRANSPOSE = 2 };

template <typename T>
struct ApplyArgsT {
  const T *u;
  T *y;
  const int32_t *elems;
  int32_t n_group;
  int32_t n_rhs;
  int64_t ndof;
  const int64_t *dof_off;
  const int32_t *nbr;
  const T *geo;
  const int32_t *prob;
  const T *coef;            // [nquad][4]: m, d_x, d_y (COEF_VERTEX_EDGE: d_xz), d_z per volume point;
                            // COEF_GENERAL: [nquad][12] (w |J|, C_11 .. C_0, 0)
  const int64_t *coef_off;
  int64_t nquad;
  const T *z;
  const double *beta;
  T *pnew;
  double *partial;
  const double *rho;
  int32_t skip_faces;
  int32_t self_only;        // 1: neighbour traces taken as zero (diagonal blocks of A)
  // edge neighbourhood (COEF_EDGE); null / 0 for box meshes
  int32_t n_elem;           // corner set c's values start at dof_off[n_elem + c]
  const T *kappa;           // [E][KAPPA_STRIDE]: per x-point factor (e^{2 tau}, 1/sin^2 phi, e^{2 psi})
  const T *fw;              // [E][6][10] face-norm weights (null: all 1)
  const int32_t *cslot;     // [E][2] slot of the element's corner face 0 / face 4, or -1
  T *cscr;                  // [slots][n_rhs][CSCR_STRIDE] corner-side face contributions
  // outer-face conditions of box meshes of the Laplacian; null: every outer face Dirichlet
  const int32_t *fbc;       // [E][6]: 0 Dirichlet, 1 Neumann, 2 Robin
  const T *fgam;            // [E][6]: the Robin gamma (0 elsewhere)
};

template <typename T>
struct PrecArgsT {
  const int32_t *elems;
  int32_t n_group;
  int32_t n_rhs;
  int64_t ndof;
  const int64_t *dof_off;
  const int32_t *prob;
  const T *rin;
  T *zout;
  T *x;
  T *r;
  const T *p;
  const T *q;
  const double *alpha;
  double *part_rr;
  double *part_rz;
  // edge neighbourhood, C* form (eq. 5.30): per element the x3 eigenbasis
  // S_z (P x P, node-major) then its eigenvalues nu (P), ZEIG_STRIDE apart;
  // null for box meshes (the master C-form in every direction)
  const T *zeig;
};

// Packed FP64 tables for one degree, in the order of the device struct:
// B0, B1, B2 (Q*P each), D (P*P), S (P*P), MP (P*P), KP (P*P), WQ (Q), MU (P),
// then DQ (Q*Q, the differentiation matrix of the Q-point grid).
inline int packed_table_size(int W) {
  const int P = W + 1, Q = 2 * W + 1;
  return 3 * Q * P + 4 * P * P + Q + P + Q * Q;
}

struct KernelSet {
  int W;
  int is_double;
  cudaError_t (*upload)(const double *packed);
  // coef: COEF_*, mode: MODE_*; args points to ApplyArgsT<T>
  cudaError_t (*apply)(int coef, int mode, const void *args, int n_items, int threads, cudaStream_t s);
  size_t (*apply_smem)(int coef);
  int (*apply_max_threads)(int coef);
  // mode: MODE_PLAIN or MODE_PCG; args points to PrecArgsT<T>
  cudaError_t (*precond)(int mode, const void *args, int n_items, int threads, cudaStream_t s);
  // volume transpose in integration-by-parts form (COEF_LAPLACE, COEF_SCALAR;
  // args as for MODE_TRANSPOSE); ibp_smem: its shared memory, 0 where the
  // instance is not built
  cudaError_t (*transpose_ibp)(int coef, const void *args, int n_items, cudaStream_t s);
  size_t (*ibp_smem)(int coef);
};

}  // namespace hpse
