// Corner sets of the edge neighbourhood (Section 2.3, eq. 4.7): on the
// corner elements r < r_1 of an x3-slab the function is one polynomial in x3,
// shared by every theta sector.  Their volumes and their other faces have
// infinite measure, so they enter the functional only through the faces
// r = r_1 with the layer-1 elements.  The operator kernel of each such element
// writes the corner side of its face terms into a slot (k_apply, face phase);
// these kernels sum the slots of each corner set, do the PCG bookkeeping of
// its values, and apply its exact block A_cc^{-1} = X^T X (X = L^{-1},
// A_cc = L L^T assembled and factored in FP64 on the host).
#pragma once

template <typename T>
struct CornerArgsT {
  int32_t n_corner, n_rhs, n_elem;
  int64_t ndof;
  const int64_t *dof_off;       // [n_elem + n_corner]
  const int32_t *cW;            // [n_corner] degree
  const int32_t *cprob;         // [n_corner] problem
  const int32_t *slot_ptr;      // [n_corner + 1] CSR of face slots per corner set
  const int32_t *slot_list;
  const T *cscr;                // [slots][n_rhs][CSCR_STRIDE]
  const T *cinv;                // [n_corner][CSCR_STRIDE^2] X = L^{-1}, row-major
  // apply: y (out), u; PCG mode: z, p (read), pnew (write), beta, partial
  // preconditioner: rin / zout; PCG mode: x, r, p, q, alpha, part_rr, part_rz
  const T *u;
  T *y;
  const T *z;
  const T *p;
  T *pnew;
  const double *beta;
  double *partial;
  const T *rin;
  T *zout;
  T *x;
  T *r;
  const T *q;
  const double *alpha;
  double *part_rr, *part_rz;
};

// grid: n_corner * n_rhs, 32 threads
template <typename T, int MODE>
__global__ void k_corner_apply(CornerArgsT<T> A) {
  const int item = blockIdx.x;
  const int c = item / A.n_rhs, rr = item - c * A.n_rhs;
  const int P = A.cW[c] + 1;
  const int64_t base = (int64_t)rr * A.ndof + A.dof_off[A.n_elem + c];
  double part = 0.0;
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    T v = (T)0;
    if (MODE != hpse::MODE_TRANSPOSE)
      for (int i = A.slot_ptr[c]; i < A.slot_ptr[c + 1]; ++i)
        v += A.cscr[((int64_t)A.slot_list[i] * A.n_rhs + rr) * hpse::CSCR_STRIDE + k];
    A.y[base + k] = v;
    if (MODE == hpse::MODE_PCG) {
      const T pv = A.z[base + k] + (T)A.beta[A.cprob[c] * A.n_rhs + rr] * A.p[base + k];
      A.pnew[base + k] = pv;
      part += (double)pv * (double)v;
    }
  }
  if (MODE == hpse::MODE_PCG) {
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (threadIdx.x == 0) A.partial[(int64_t)(A.n_elem + c) * A.n_rhs + rr] = part;
  }
}

// grid: n_corner * n_rhs, 32 threads (P <= 11 values per item)
template <typename T, int MODE>
__global__ void k_corner_prec(CornerArgsT<T> A) {
  __shared__ T sr[hpse::CSCR_STRIDE], st[hpse::CSCR_STRIDE];
  const int item = blockIdx.x;
  const int c = item / A.n_rhs, rr = item - c * A.n_rhs;
  const int P = A.cW[c] + 1, k = threadIdx.x;
  const int64_t base = (int64_t)rr * A.ndof + A.dof_off[A.n_elem + c];
  double prr = 0.0, prz = 0.0;
  if (k < P) {
    T rv;
    if (MODE == hpse::MODE_PCG) {
      const T al = (T)A.alpha[A.cprob[c] * A.n_rhs + rr];
      if (A.x) A.x[base + k] += al * A.p[base + k];
      rv = A.r[base + k] - al * A.q[base + k];
      A.r[base + k] = rv;
      prr = (double)rv * (double)rv;
    } else {
      rv = A.rin[base + k];
    }
    sr[k] = rv;
  }
  __syncwarp();
  const T *X = A.cinv + (int64_t)c * hpse::CSCR_STRIDE * hpse::CSCR_STRIDE;
  if (k < P) {  // t = X r (X lower triangular)
    T s = 0;
    for (int j = 0; j <= k; ++j) s += X[k * hpse::CSCR_STRIDE + j] * sr[j];
    st[k] = s;
  }
  __syncwarp();
  if (k < P) {  // z = X^T t
    T s = 0;
    for (int j = k; j < P; ++j) s += X[j * hpse::CSCR_STRIDE + k] * st[j];
    A.zout[base + k] = s;
    prz = (double)s * (double)sr[k];
  }
  if (MODE == hpse::MODE_PCG) {
    for (int o = 16; o > 0; o >>= 1) {
      prr += __shfl_xor_sync(0xffffffffu, prr, o);
      prz += __shfl_xor_sync(0xffffffffu, prz, o);
    }
    if (k == 0) {
      A.part_rr[(int64_t)(A.n_elem + c) * A.n_rhs + rr] = prr;
      A.part_rz[(int64_t)(A.n_elem + c) * A.n_rhs + rr] = prz;
    }
  }
}
