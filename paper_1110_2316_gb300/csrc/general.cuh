// general.cuh -- operator apply for a general second-order operator with
// per-point coefficients, one (REAL, WDEG) instantiation (included after
// kernels.cuh by inst_template.cuh).
//
// On a box element the operator of eq. (2.2), written out as
//   L u = sum_ij A_ij u_{x_i x_j} + sum_i b_i u_{x_i} + c u   (A symmetric),
// is, in the reference coordinates lambda of the element, the ten-term form
// of eq. (5.45):
//   L u = C_11 u_11 + C_22 u_22 + C_33 u_33 + C_12 u_12 + C_23 u_23
//       + C_13 u_13 + C_1 u_1 + C_2 u_2 + C_3 u_3 + C_0 u
// (u_a = du/dlambda_a), with C_aa = A_aa s_a^2, C_ab = 2 A_ab s_a s_b,
// C_a = b_a s_a, C_0 = c, s_a = dlambda_a / dx_a.  The host library stores,
// per volume point, the quadrature weight w_a w_b w_c |J| and the ten C's
// (GEN_NC values per point, the last one padding).
//
// Sum factorisation (Section 5.3) of the ten fields:
//   x-stage:  X_m = B_m along x,              m = 0, 1, 2
//   y-stage:  T_mn = B_n along y of X_m,      (m, n) = 00 01 02 10 11 20
//   z-stage:  u = B0 T00, u_3 = B1 T00, u_33 = B2 T00, u_2 = B0 T01,
//             u_23 = B1 T01, u_22 = B0 T02, u_1 = B0 T10, u_13 = B1 T10,
//             u_12 = B0 T11, u_11 = B0 T20,
// then rho = w |J| (L u) per point and the transposed stages in reverse
// order; the face terms of box meshes (jumps of u and of the physical
// gradient, Dirichlet and Neumann / Robin faces) are those of the Laplacian
// (face_phase of kernels.cuh), since they do not involve the operator.
//
// Design: one CTA per (element, rhs) item like k_apply; every stage is a
// whole-CTA loop over line jobs, the contractions unrolled loops with
// constant-bank matrix entries (B of c_tab), those of the z-stage (most of
// the multiply-adds) folded into even-odd halves like k_apply's.  The z-stage reads the point
// coefficients twice per apply (forward, then transpose), from L1 / L2 the
// second time.  Shared memory: su | X[3] | T[6] | D copy + face scales | reduction;
// the T region later holds sy and the face scratch.  Instances whose layout
// exceeds 227 KB (FP64 at W = 10) are not built; the host library refuses
// such meshes.
#pragma once

namespace {

constexpr int GEN_NC = 12;

struct GenLayout {
  static constexpr int T_REGION0 = 6 * Q2P;
  static constexpr int T_NEED = P3 + 6 * FACE_ARR * P2;
  static constexpr int T_REGION = T_REGION0 > T_NEED ? T_REGION0 : T_NEED;
  static constexpr int TABS = P2 + FACE_META_REALS;
  static constexpr int TOTAL = P3 + 3 * QP2 + T_REGION + TABS;
  static constexpr size_t RED_OFF = (((size_t)TOTAL * sizeof(real) + 15) / 16) * 16;
  static constexpr size_t BYTES = RED_OFF + 64 * sizeof(double);
  static constexpr bool FITS = BYTES <= 232448;
};

constexpr int GEN_MINB = sizeof(real) == 8 ? 1 : 2;
// coefficient stride between consecutive z-points of a column
constexpr int GEN_CQ = GEN_NC * Q2;

// z-stage helpers of one column (cp: the column's first point coefficients).
// The contractions are folded like k_apply's (even-odd halves of B_n on the
// symmetric grids): a T line is loaded as its folded halves (e, o), and the
// transposed contractions of a line accumulate folded (pl, mi) pairs that
// are unfolded when the line is stored.
__device__ __forceinline__ void gen_load(const real *col, real *e, real *o) {
  real v[P];
#pragma unroll
  for (int k = 0; k < P; ++k) v[k] = col[k * Q2];
  fold_p(v, e, o);
}
__device__ __forceinline__ void gen_store(const real *pl, const real *mi, real *col, bool ok) {
  if (!ok) return;
#pragma unroll
  for (int k = 0; k < HPE; ++k) put_p(col, Q2, k, pl[k], mi[k]);
}
__device__ __forceinline__ void gen_zero(real *pl, real *mi) {
#pragma unroll
  for (int k = 0; k < HPE; ++k) pl[k] = mi[k] = (real)0;
}
// rho[q] += C_CS[q] (B_NN t)[q], output pairs (q, Q-1-q) from the folded line
template <int NN, int CS>
__device__ __forceinline__ void gen_zf(const real *e, const real *o, real *rho, const real *cp) {
#pragma unroll
  for (int qc = 0; qc <= HQ; ++qc) {
    real pl = 0, mi = 0;
    fwd_pm<NN>(e, o, qc, pl, mi);
    rho[qc] += cp[qc * GEN_CQ + CS] * (pl + mi);
    if (qc < HQ) rho[Q - 1 - qc] += cp[(Q - 1 - qc) * GEN_CQ + CS] * (pl - mi);
  }
  __syncwarp();  // scheduling fence (register pressure); reached by all 32 lanes
}
// (pl, mi)[k] += the folded halves of sum_q B_NN[q][k] C_CS[q] rho[q]
template <int NN, int CS>
__device__ __forceinline__ void gen_zr(const real *rho, const real *cp, real *pl, real *mi) {
#pragma unroll
  for (int qc = 0; qc < HQ; ++qc) {
    const real g0 = cp[qc * GEN_CQ + CS] * rho[qc], g1 = cp[(Q - 1 - qc) * GEN_CQ + CS] * rho[Q - 1 - qc];
    rev_pair<NN>(g0 + g1, g0 - g1, qc, pl, mi);
  }
  rev_mid<NN>(cp[HQ * GEN_CQ + CS] * rho[HQ], pl, mi);
  __syncwarp();  // scheduling fence (register pressure); reached by all 32 lanes
}

template <int MODE>
__global__ void __launch_bounds__(NT, GEN_MINB) k_apply_gen(const ApplyArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real *su = reinterpret_cast<real *>(smem_raw);
  real *sX = su + P3;                 // X0 | X1 | X2, later X0' | X1' | X2'
  real *sT = sX + 3 * QP2;            // T00 T01 T02 T10 T11 T20 (in place -> T')
  real *stab = sT + GenLayout::T_REGION;
  double *red = reinterpret_cast<double *>(smem_raw + GenLayout::RED_OFF);

  const int item = blockIdx.x;
  const int ge = item / A.n_rhs;
  const int r = item - ge * A.n_rhs;
  const int e = A.elems[ge];
  const int64_t base = (int64_t)r * A.ndof + A.dof_off[e];
  const real *geo_e = A.geo + (int64_t)e * 4;
  const int tid = threadIdx.x;
  constexpr int nt = NT;

  for (int t = tid; t < P2; t += nt) stab[t] = c_tab.D[t];
  FaceMeta *fm = face_meta(stab);
  if (MODE != MODE_TRANSPOSE && tid < 6) face_meta_fill<COEF_LAPLACE, MODE>(A, e, r, geo_e, fm, tid);
  if (MODE != MODE_TRANSPOSE) {
    if (MODE == MODE_PCG) {
      const double bt = A.beta[A.prob[e] * A.n_rhs + r];
      for (int t = tid; t < P3; t += nt) {
        const real v = A.z[base + t] + (real)bt * A.u[base + t];
        su[t] = v;
        A.pnew[base + t] = v;
      }
    } else {
      for (int t = tid; t < P3; t += nt) su[t] = A.u[base + t];
    }
    __syncthreads();
    // x-stage: jobs (line (j, k), m); X_m[(k P + j) Q + qa]
    for (int t = tid; t < 3 * P2; t += nt) {
      const int m = t / P2, l = t - m * P2;
      real v[P];
#pragma unroll
      for (int i = 0; i < P; ++i) v[i] = su[l * P + i];
      real *X = sX + m * QP2 + l * Q;
#define GEN_XF(MM)                                                   \
  _Pragma("unroll") for (int q = 0; q < Q; ++q) {                    \
    real acc = 0;                                                    \
    _Pragma("unroll") for (int i = 0; i < P; ++i) acc += c_tab.B[MM][q * P + i] * v[i]; \
    X[q] = acc;                                                      \
  }
      if (m == 0) {
        GEN_XF(0)
      } else if (m == 1) {
        GEN_XF(1)
      } else {
        GEN_XF(2)
      }
#undef GEN_XF
    }
    __syncthreads();
    // y-stage: jobs (line (qa, k), output field); T[f][k Q^2 + qb Q + qa]
    for (int t = tid; t < 6 * QP; t += nt) {
      const int f = t / QP, l = t - f * QP;
      const int qa = l % Q, k = l / Q;
      const int m = f < 3 ? 0 : (f < 5 ? 1 : 2);
      const int n = f < 3 ? f : (f == 3 ? 0 : (f == 4 ? 1 : 0));
      const real *X = sX + m * QP2;
      real v[P];
#pragma unroll
      for (int j = 0; j < P; ++j) v[j] = X[(k * P + j) * Q + qa];
      real *T = sT + f * Q2P + k * Q2 + qa;
#define GEN_YF(NN)                                                   \
  _Pragma("unroll") for (int qb = 0; qb < Q; ++qb) {                 \
    real acc = 0;                                                    \
    _Pragma("unroll") for (int j = 0; j < P; ++j) acc += c_tab.B[NN][qb * P + j] * v[j]; \
    T[qb * Q] = acc;                                                 \
  }
      if (n == 0) {
        GEN_YF(0)
      } else if (n == 1) {
        GEN_YF(1)
      } else {
        GEN_YF(2)
      }
#undef GEN_YF
    }
    __syncthreads();
  }

  // z-stage per column (qa, qb): forward + pointwise weight into rho[Q], then
  // the transposed contractions, written in place over the column's T
  // entries.  Both run field by field (one T line and rho[Q] live at a time)
  // to bound the registers; field k of a T line: line m of T, matrix n, and
  // its coefficient slot c (the ten-term order of the header).
  // (the loop runs to whole warps: lanes past the last column repeat it
  // without storing, so that every lane reaches the __syncwarp fences)
  for (int lp = tid; lp < PAD32(Q2); lp += nt) {
    const bool ok = lp < Q2;
    const int l = ok ? lp : Q2 - 1;
    const int64_t cbase = A.coef_off[e] + l;
    const real *cp = A.coef + GEN_NC * cbase;
    real rho[Q];
    if (MODE == MODE_TRANSPOSE) {
#pragma unroll
      for (int qc = 0; qc < Q; ++qc) rho[qc] = (real)A.rho[(int64_t)r * A.nquad + cbase + (int64_t)qc * Q2];
    } else {
#pragma unroll
      for (int q = 0; q < Q; ++q) rho[q] = (real)0;
      real te[HPE], to[HPE];
      gen_load(sT + 0 * Q2P + l, te, to);
      gen_zf<0, 10>(te, to, rho, cp);  // u
      gen_zf<1, 9>(te, to, rho, cp);   // u_3
      gen_zf<2, 3>(te, to, rho, cp);   // u_33
      gen_load(sT + 1 * Q2P + l, te, to);
      gen_zf<0, 8>(te, to, rho, cp);   // u_2
      gen_zf<1, 5>(te, to, rho, cp);   // u_23
      gen_load(sT + 2 * Q2P + l, te, to);
      gen_zf<0, 2>(te, to, rho, cp);   // u_22
      gen_load(sT + 3 * Q2P + l, te, to);
      gen_zf<0, 7>(te, to, rho, cp);   // u_1
      gen_zf<1, 6>(te, to, rho, cp);   // u_13
      gen_load(sT + 4 * Q2P + l, te, to);
      gen_zf<0, 4>(te, to, rho, cp);   // u_12
      gen_load(sT + 5 * Q2P + l, te, to);
      gen_zf<0, 1>(te, to, rho, cp);   // u_11
#pragma unroll
      for (int q = 0; q < Q; ++q) rho[q] *= cp[q * GEN_CQ];
    }
    // T'_line[k] = sum over its fields of sum_q B_n[q][k] C_c[q] rho[q]
    {
      real pl[HPE], mi[HPE];
      gen_zero(pl, mi);
      gen_zr<0, 10>(rho, cp, pl, mi);
      gen_zr<1, 9>(rho, cp, pl, mi);
      gen_zr<2, 3>(rho, cp, pl, mi);
      gen_store(pl, mi, sT + 0 * Q2P + l, ok);
      gen_zero(pl, mi);
      gen_zr<0, 8>(rho, cp, pl, mi);
      gen_zr<1, 5>(rho, cp, pl, mi);
      gen_store(pl, mi, sT + 1 * Q2P + l, ok);
      gen_zero(pl, mi);
      gen_zr<0, 2>(rho, cp, pl, mi);
      gen_store(pl, mi, sT + 2 * Q2P + l, ok);
      gen_zero(pl, mi);
      gen_zr<0, 7>(rho, cp, pl, mi);
      gen_zr<1, 6>(rho, cp, pl, mi);
      gen_store(pl, mi, sT + 3 * Q2P + l, ok);
      gen_zero(pl, mi);
      gen_zr<0, 4>(rho, cp, pl, mi);
      gen_store(pl, mi, sT + 4 * Q2P + l, ok);
      gen_zero(pl, mi);
      gen_zr<0, 1>(rho, cp, pl, mi);
      gen_store(pl, mi, sT + 5 * Q2P + l, ok);
    }
  }
  __syncthreads();

  // y-stage transpose: jobs (line (qa, k), m); X_m'[(k P + j) Q + qa]
  //   X0' = B0^T T00' + B1^T T01' + B2^T T02', X1' = B0^T T10' + B1^T T11', X2' = B0^T T20'
  for (int t = tid; t < 3 * QP; t += nt) {
    const int m = t / QP, l = t - m * QP;
    const int qa = l % Q, k = l / Q;
    const real *T = sT + k * Q2 + qa;
    real acc[P];
#pragma unroll
    for (int j = 0; j < P; ++j) acc[j] = (real)0;
    if (m == 0) {
#pragma unroll
      for (int qb = 0; qb < Q; ++qb) {
        const real v0 = T[0 * Q2P + qb * Q], v1 = T[1 * Q2P + qb * Q], v2 = T[2 * Q2P + qb * Q];
#pragma unroll
        for (int j = 0; j < P; ++j)
          acc[j] += c_tab.B[0][qb * P + j] * v0 + c_tab.B[1][qb * P + j] * v1 + c_tab.B[2][qb * P + j] * v2;
      }
    } else if (m == 1) {
#pragma unroll
      for (int qb = 0; qb < Q; ++qb) {
        const real v0 = T[3 * Q2P + qb * Q], v1 = T[4 * Q2P + qb * Q];
#pragma unroll
        for (int j = 0; j < P; ++j) acc[j] += c_tab.B[0][qb * P + j] * v0 + c_tab.B[1][qb * P + j] * v1;
      }
    } else {
#pragma unroll
      for (int qb = 0; qb < Q; ++qb) {
        const real v0 = T[5 * Q2P + qb * Q];
#pragma unroll
        for (int j = 0; j < P; ++j) acc[j] += c_tab.B[0][qb * P + j] * v0;
      }
    }
    real *X = sX + m * QP2;
#pragma unroll
    for (int j = 0; j < P; ++j) X[(k * P + j) * Q + qa] = acc[j];
  }
  __syncthreads();

  // x-stage transpose: jobs (line (j, k)); y[i] = sum_m B_m^T X_m'
  real *sy = sT;  // the T region is free now
  for (int l = tid; l < P2; l += nt) {
    real acc[P];
#pragma unroll
    for (int i = 0; i < P; ++i) acc[i] = (real)0;
#pragma unroll
    for (int qa = 0; qa < Q; ++qa) {
      const real v0 = sX[l * Q + qa], v1 = sX[QP2 + l * Q + qa], v2 = sX[2 * QP2 + l * Q + qa];
#pragma unroll
      for (int i = 0; i < P; ++i)
        acc[i] += c_tab.B[0][qa * P + i] * v0 + c_tab.B[1][qa * P + i] * v1 + c_tab.B[2][qa * P + i] * v2;
    }
#pragma unroll
    for (int i = 0; i < P; ++i) sy[l * P + i] = acc[i];
  }
  __syncthreads();

  // faces: those of the Laplacian on box meshes (the operator does not enter)
  if (MODE != MODE_TRANSPOSE && !A.skip_faces)
    face_phase<COEF_LAPLACE, MODE>(A, e, r, su, sy, sT + P3, stab, geo_e, fm);

  double part = 0.0;
  for (int t = tid; t < P3; t += nt) {
    const real v = sy[t];
    A.y[base + t] = v;
    if (MODE == MODE_PCG) part += (double)v * (double)su[t];
  }
  if (MODE == MODE_PCG) {
    const double s = block_sum(part, red);
    if (tid == 0) A.partial[(int64_t)e * A.n_rhs + r] = s;
  }
}

template <int MODE>
cudaError_t launch_apply_gen(const void *args, int n_items, cudaStream_t s) {
  if constexpr (GenLayout::FITS) {
    k_apply_gen<MODE><<<n_items, NT, GenLayout::BYTES, s>>>(*static_cast<const ApplyArgs *>(args));
    return cudaGetLastError();
  } else {
    (void)args;
    (void)n_items;
    (void)s;
    return cudaErrorInvalidConfiguration;
  }
}

template <int MODE>
cudaError_t set_smem_attr_gen() {
  if constexpr (GenLayout::FITS) {
    cudaError_t e = cudaFuncSetAttribute(k_apply_gen<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)GenLayout::BYTES);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_apply_gen<MODE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
  } else {
    return cudaSuccess;
  }
}

}  // namespace
