// ibp.cuh -- the volume transpose in integration-by-parts form (eq. 5.45-5.48),
// one (REAL, WDEG) instantiation (included after kernels.cuh).
//
// The transpose of the volume residual, y_k = sum_q rho_q (L phi_k)(xi_q) over
// the (2W+1)^3 GLL points of an element (rho_q = w_q |J| times the residual,
// as the direct transpose of k_apply<.., MODE_TRANSPOSE> takes it), is the
// integral of (L phi_k) I(zeta) with zeta_q = rho_q / w_q and I the
// degree-2W interpolant; integrating by parts moves the derivatives onto
// I(c zeta) (c the coefficient of each term, applied pointwise first), taken
// with the (2W+1)-point differentiation matrix D_Q (eq. 5.47), and adds the
// six faces' boundary terms.  Every integrand is a polynomial the GLL rule
// integrates exactly, so the result equals the direct transpose up to
// rounding.  Operators (the kernels' reference-coordinate forms):
//   COEF_LAPLACE: L v = sum_a s_a^2 v_aa
//   COEF_SCALAR:  L v = sum_a s_a^2 v_aa + sum_a d_a v_a  (d_a per point, the
//                 coefficient array's entries 1..3)
// y_k = int phi_k (sum_a s_a^2 D_Q,a^2 zeta - sum_a D_Q,a (d_a zeta))
//     + sum_a [s_a^2 (phi_k,a zeta - phi_k D_Q,a zeta) + phi_k d_a zeta]_a
// ([g]_a: g at xi_a = 1 minus g at xi_a = -1, integrated over the face by
// the GLL rule).  Shared memory: zeta | V | (d_a zeta) | face values F0, F1
// (then their projections G0, G1) | the first projection H | copies of D_Q,
// D_Q^2, B0, D.
// Instances whose layout exceeds 227 KB are not built (the host refuses).
#pragma once

namespace {

constexpr int Q3 = Q * Q2;

template <int COEF>
struct IbpLayout {
  static constexpr int NB = COEF == COEF_SCALAR ? 3 : 2;
  static constexpr int FACE = 12 * Q2;    // F0, F1 of the six faces, later G0, G1 (12 P^2)
  static constexpr int HBUF = 12 * QP;    // their projection along p1
  static constexpr int TABS = 2 * Q2 + QP + P2;
  static constexpr int TOTAL = NB * Q3 + FACE + HBUF + TABS;
  static constexpr size_t BYTES = (size_t)TOTAL * sizeof(real);
  static constexpr bool FITS = BYTES <= 232448;
};

// Q x Q differentiation matrix of the (2W+1)-point grid and its square
struct IbpTables {
  real DQ[Q2];
  real DQ2[Q2];
};
__constant__ IbpTables c_ibp;

template <int COEF>
__global__ void __launch_bounds__(NT, 1) k_transpose_ibp(const ApplyArgs A) {
  typedef IbpLayout<COEF> L;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real *Zs = reinterpret_cast<real *>(smem_raw);
  real *Vs = Zs + Q3;
  real *Ts = Vs + Q3;                     // d_a zeta (COEF_SCALAR)
  real *Fs = Zs + L::NB * Q3;
  real *Hs = Fs + L::FACE;
  real *Gs = Fs;                          // F is dead once H is formed
  real *dq = Hs + L::HBUF;
  real *dq2 = dq + Q2;
  real *b0 = dq2 + Q2;
  real *dp = b0 + QP;

  const int item = blockIdx.x;
  const int ge = item / A.n_rhs;
  const int r = item - ge * A.n_rhs;
  const int e = A.elems[ge];
  const int64_t base = (int64_t)r * A.ndof + A.dof_off[e];
  const int64_t qbase = A.coef_off[e];
  const real *geo_e = A.geo + (int64_t)e * 4;
  real s2[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) s2[a] = geo_e[a] * geo_e[a];
  const int tid = threadIdx.x;
  constexpr int nt = NT;

  for (int t = tid; t < Q2; t += nt) {
    dq[t] = c_ibp.DQ[t];
    dq2[t] = c_ibp.DQ2[t];
  }
  for (int t = tid; t < QP; t += nt) b0[t] = c_tab.B[0][t];
  for (int t = tid; t < P2; t += nt) dp[t] = c_tab.D[t];
  // zeta = rho / w at every point ([qc][qb][qa], x fastest)
  for (int t = tid; t < Q3; t += nt) {
    const int qa = t % Q, qb = (t / Q) % Q, qc = t / Q2;
    Zs[t] = (real)A.rho[(int64_t)r * A.nquad + qbase + t] / (c_tab.WQ[qa] * c_tab.WQ[qb] * c_tab.WQ[qc]);
  }
  __syncthreads();
  // V = sum_a s_a^2 (D_Q^2 along a) zeta
  for (int t = tid; t < Q3; t += nt) {
    const int qa = t % Q, qb = (t / Q) % Q, qc = t / Q2;
    const real *zx = Zs + qc * Q2 + qb * Q, *zy = Zs + qc * Q2 + qa, *zz = Zs + qb * Q + qa;
    real vx = 0, vy = 0, vz = 0;
#pragma unroll
    for (int m = 0; m < Q; ++m) {
      vx += dq2[qa * Q + m] * zx[m];
      vy += dq2[qb * Q + m] * zy[m * Q];
      vz += dq2[qc * Q + m] * zz[m * Q2];
    }
    Vs[t] = s2[0] * vx + s2[1] * vy + s2[2] * vz;
  }
  // faces: F0 = w2 s_a^2 zeta, F1 = -w2 s_a^2 (D_Q,a zeta) on the layer xi_a = +-1;
  // face f = 2a + side, point (p1, p2) over the two tangential axes in order
  for (int t = tid; t < 6 * Q2; t += nt) {
    const int f = t / Q2, sp = t - f * Q2;
    const int p1 = sp % Q, p2 = sp / Q;
    const int a = f >> 1, n = (f & 1) ? Q - 1 : 0;
    // (qa, qb, qc) of the layer point and the stride along a
    const int qa = a == 0 ? n : p1, qb = a == 1 ? n : (a == 0 ? p1 : p2), qc = a == 2 ? n : p2;
    const int st = a == 0 ? 1 : (a == 1 ? Q : Q2);
    const int t0 = qc * Q2 + qb * Q + qa - n * st;  // the line through the point along a
    real dz = 0;
#pragma unroll
    for (int m = 0; m < Q; ++m) dz += dq[n * Q + m] * Zs[t0 + m * st];
    const real w2 = c_tab.WQ[p1] * c_tab.WQ[p2];
    Fs[f * Q2 + sp] = w2 * s2[a] * Zs[t0 + n * st];
    Fs[6 * Q2 + f * Q2 + sp] = -w2 * s2[a] * dz;
  }
  __syncthreads();
  if (COEF == COEF_SCALAR) {
    // first-order terms, axis by axis: T = d_a zeta; V -= D_Q,a T; F1 += w2 T on the layer
#pragma unroll 1
    for (int a = 0; a < 3; ++a) {
      for (int t = tid; t < Q3; t += nt) Ts[t] = A.coef[4 * (qbase + t) + 1 + a] * Zs[t];
      __syncthreads();
      for (int t = tid; t < Q3; t += nt) {
        const int qa = t % Q, qb = (t / Q) % Q, qc = t / Q2;
        const int qi = a == 0 ? qa : (a == 1 ? qb : qc);
        const int st = a == 0 ? 1 : (a == 1 ? Q : Q2);
        const real *tl = Ts + t - qi * st;
        real v = 0;
#pragma unroll
        for (int m = 0; m < Q; ++m) v += dq[qi * Q + m] * tl[m * st];
        Vs[t] -= v;
      }
      for (int t = tid; t < 2 * Q2; t += nt) {
        const int side = t / Q2, sp = t - side * Q2;
        const int p1 = sp % Q, p2 = sp / Q;
        const int f = 2 * a + side, n = side ? Q - 1 : 0;
        const int qa = a == 0 ? n : p1, qb = a == 1 ? n : (a == 0 ? p1 : p2), qc = a == 2 ? n : p2;
        Fs[6 * Q2 + f * Q2 + sp] += c_tab.WQ[p1] * c_tab.WQ[p2] * Ts[qc * Q2 + qb * Q + qa];
      }
      __syncthreads();
    }
  }
  // face projections, first along p1: H[g][p2][j1] (g = the 12 face fields)
  for (int t = tid; t < 12 * Q; t += nt) {
    const int g = t / Q, p2 = t - g * Q;
    const real *F = Fs + g * Q2 + p2 * Q;
    real acc[P];
#pragma unroll
    for (int j = 0; j < P; ++j) acc[j] = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const real v = F[q];
#pragma unroll
      for (int j = 0; j < P; ++j) acc[j] += b0[q * P + j] * v;
    }
#pragma unroll
    for (int j = 0; j < P; ++j) Hs[g * QP + p2 * P + j] = acc[j];
  }
  // volume projection along x: Zs <- T1[qc][qb][i] = sum_qa B0[qa][i] w3 V (zeta is no longer needed)
  for (int l = tid; l < Q2; l += nt) {
    const int qb = l % Q, qc = l / Q;
    const real wbc = c_tab.WQ[qb] * c_tab.WQ[qc];
    real acc[P];
#pragma unroll
    for (int i = 0; i < P; ++i) acc[i] = 0;
#pragma unroll
    for (int qa = 0; qa < Q; ++qa) {
      const real v = wbc * c_tab.WQ[qa] * Vs[l * Q + qa];
#pragma unroll
      for (int i = 0; i < P; ++i) acc[i] += b0[qa * P + i] * v;
    }
#pragma unroll
    for (int i = 0; i < P; ++i) Zs[l * P + i] = acc[i];
  }
  __syncthreads();
  // second face projection along p2: G[g][j2][j1]
  for (int t = tid; t < 12 * P; t += nt) {
    const int g = t / P, j1 = t - g * P;
    real acc[P];
#pragma unroll
    for (int j = 0; j < P; ++j) acc[j] = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const real v = Hs[g * QP + q * P + j1];
#pragma unroll
      for (int j = 0; j < P; ++j) acc[j] += b0[q * P + j] * v;
    }
#pragma unroll
    for (int j = 0; j < P; ++j) Gs[g * P2 + j * P + j1] = acc[j];
  }
  // volume projection along y: Vs <- T2[qc][j][i] = sum_qb B0[qb][j] T1[qc][qb][i]
  for (int l = tid; l < QP; l += nt) {
    const int i = l % P, qc = l / P;
    real acc[P];
#pragma unroll
    for (int j = 0; j < P; ++j) acc[j] = 0;
#pragma unroll
    for (int qb = 0; qb < Q; ++qb) {
      const real v = Zs[(qc * Q + qb) * P + i];
#pragma unroll
      for (int j = 0; j < P; ++j) acc[j] += b0[qb * P + j] * v;
    }
#pragma unroll
    for (int j = 0; j < P; ++j) Vs[(qc * P + j) * P + i] = acc[j];
  }
  __syncthreads();
  // along z, plus the face terms, per node
  for (int t = tid; t < P3; t += nt) {
    const int i = t % P, j = (t / P) % P, k = t / P2;
    real acc = 0;
#pragma unroll
    for (int qc = 0; qc < Q; ++qc) acc += b0[qc * P + k] * Vs[qc * P2 + j * P + i];
    const int nd[3] = {i, j, k};
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int a = f >> 1, side = f & 1, en = side ? P - 1 : 0;
      const int j1 = a == 0 ? j : i, j2 = a == 2 ? j : k;
      const real sg = side ? (real)1 : (real)-1;
      const real g0 = Gs[f * P2 + j2 * P + j1], g1 = Gs[(6 + f) * P2 + j2 * P + j1];
      acc += sg * (dp[en * P + nd[a]] * g0 + (nd[a] == en ? g1 : (real)0));
    }
    A.y[base + t] = acc;
  }
}

template <int COEF>
cudaError_t launch_transpose_ibp_t(const void *args, int n_items, cudaStream_t s) {
  if constexpr (IbpLayout<COEF>::FITS) {
    k_transpose_ibp<COEF><<<n_items, NT, IbpLayout<COEF>::BYTES, s>>>(*static_cast<const ApplyArgs *>(args));
    return cudaGetLastError();
  } else {
    (void)args;
    (void)n_items;
    (void)s;
    return cudaErrorInvalidConfiguration;
  }
}

template <int COEF>
cudaError_t set_smem_attr_ibp() {
  if constexpr (IbpLayout<COEF>::FITS)
    return cudaFuncSetAttribute(k_transpose_ibp<COEF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)IbpLayout<COEF>::BYTES);
  else
    return cudaSuccess;
}

}  // namespace
