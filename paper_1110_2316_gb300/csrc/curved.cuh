// curved.cuh -- regular elements with a curved map (included by hpse.cu).
//
// Eq. (4.2) on elements Omega_e = M_e(Q) with an analytic map M_e that need not
// be affine.  With K = (dx/dlambda)^{-1} (K_ai = d lambda_a / d x_i) the chain
// rule gives u_{x_i} = sum_a K_ai u_a and
//   Lap u = sum_ab g^{ab} u_ab + sum_a (Lap lambda_a) u_a,  g^{ab} = sum_i K_ai K_bi,
//   Lap lambda_a = - sum_k K_ak sum_bc (d^2 x_k / d lambda_b d lambda_c) g^{bc},
// so the volume term is the ten-term form of eq. (5.45) with per-point
// coefficients C_aa = -g^{aa}, C_ab = -2 g^{ab}, C_a = -Lap lambda_a, C_0 = 0
// and weight w |J| (k_apply_gen runs it).  The face terms (k_face_curved) are
// those of the reference face: on the (2 max(W, W') + 1)-point grid of every
// face, the jumps of u and of the physical gradient, each side through its
// own K, in the L2 form (w x w) and the H^{1/2} form of eq. (5.49)
// (w x w + w x K1 + K1 x w, K1 the 1-D quotient form); Dirichlet faces: u - g
// in L2 and its two reference-tangential derivatives in H^{1/2} (eq. 2.18).
// The two sides of an interior face share its parametrisation (face f of e and
// face f^1 of the neighbour, the same tangential axes and directions).
#pragma once

namespace curved {

// per volume point: vol [27] = Dx (Dx[k][a] = d x_k / d lambda_a, row-major),
// D2x [k][pair] with pairs (00, 11, 22, 01, 02, 12).  Writes the general
// coefficient layout (w |J|, C_11, C_22, C_33, C_12, C_23, C_13, C_1, C_2, C_3,
// C_0, 0) in FP64 and FP32, wja = -w |J|, K (9 per point, K[a][i]) and |J|
// (for the H^1 norm); bad[0] = 1 where |J| <= 0 or a value is not finite.  One
// block per element.
__global__ void k_geom_vol(int64_t nq, const int32_t *elem_W, const int64_t *coef_off, const double *const *qtab,
                           const double *vol, double *coef64, float *coef32, double *wja, double *Kv, double *detv,
                           int32_t *bad) {
  const int e = blockIdx.x;
  const int W = elem_W[e], P = W + 1, Q = 2 * W + 1;
  const double *wq = qtab[W] + 2 * Q * P + 2 * Q * Q;
  for (int t = threadIdx.x; t < Q * Q * Q; t += blockDim.x) {
    const int qa = t % Q, qb = (t / Q) % Q, qc = t / (Q * Q);
    const int64_t i = coef_off[e] + t;
    const double *g = vol + 27 * i;
    double J[3][3], H[3][3][3];
    for (int k = 0; k < 3; ++k)
      for (int a = 0; a < 3; ++a) J[k][a] = g[3 * k + a];
    const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
    for (int k = 0; k < 3; ++k)
      for (int p = 0; p < 6; ++p) H[k][pa[p]][pb[p]] = H[k][pb[p]][pa[p]] = g[9 + 6 * k + p];
    // K = J^{-1} by the adjugate
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    bool ok = det > 0.0 && isfinite(det);
    for (int m = 0; m < 27; ++m) ok = ok && isfinite(g[m]);
    if (!ok) {
      bad[0] = 1;
      for (int m = 0; m < 12; ++m) {
        coef64[12 * i + m] = 0.0;
        coef32[12 * i + m] = 0.0f;
      }
      wja[i] = 0.0;
      for (int m = 0; m < 9; ++m) Kv[9 * i + m] = 0.0;
      detv[i] = 0.0;
      continue;
    }
    double K[3][3];
    K[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    K[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    K[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    K[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    K[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    K[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    K[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    K[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    K[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < 3; ++k) Kv[9 * i + 3 * a + k] = K[a][k];
    detv[i] = det;
    double G[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) G[a][b] = K[a][0] * K[b][0] + K[a][1] * K[b][1] + K[a][2] * K[b][2];
    double lap[3];
    for (int a = 0; a < 3; ++a) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) {
        double hk = 0.0;
        for (int b = 0; b < 3; ++b)
          for (int c = 0; c < 3; ++c) hk += H[k][b][c] * G[b][c];
        s += K[a][k] * hk;
      }
      lap[a] = -s;
    }
    double c[12];
    c[0] = wq[qa] * wq[qb] * wq[qc] * det;
    c[1] = -G[0][0];
    c[2] = -G[1][1];
    c[3] = -G[2][2];
    c[4] = -2.0 * G[0][1];
    c[5] = -2.0 * G[1][2];
    c[6] = -2.0 * G[0][2];
    c[7] = -lap[0];
    c[8] = -lap[1];
    c[9] = -lap[2];
    c[10] = 0.0;
    c[11] = 0.0;
    for (int m = 0; m < 12; ++m) {
      coef64[12 * i + m] = c[m];
      coef32[12 * i + m] = (float)c[m];
    }
    wja[i] = -c[0];
  }
}

// per face point: face [9] = Dx; writes K (9, row-major K[a][i]) in FP64 and
// FP32; bad[0] = 1 where det <= 0 or not finite
__global__ void k_geom_face(int64_t nfp, const double *face, double *K64, float *K32, int32_t *bad) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nfp; p += (int64_t)gridDim.x * blockDim.x) {
    const double *g = face + 9 * p;
    double J[3][3];
    for (int k = 0; k < 3; ++k)
      for (int a = 0; a < 3; ++a) J[k][a] = g[3 * k + a];
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double K[9];
    K[0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    K[1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    K[2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    K[3] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    K[4] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    K[5] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    K[6] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    K[7] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    K[8] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    bool ok = det > 0.0 && isfinite(det);
    for (int m = 0; m < 9; ++m) ok = ok && isfinite(g[m]) && isfinite(K[m]);
    if (!ok) bad[0] = 1;
    for (int m = 0; m < 9; ++m) {
      K64[9 * p + m] = ok ? K[m] : 0.0;
      K32[9 * p + m] = ok ? (float)K[m] : 0.0f;
    }
  }
}

struct FaceArgs {
  int n_rhs;
  int64_t ndof;
  const int64_t *dof_off;
  const int32_t *nbr, *elem_W;
  const int64_t *cf_off;       // [6 E + 1] first point of element-face (e, f)
  const int32_t *cf_q;         // [6 E] its grid size Qf
  const double *const *dtab;   // [W]: D (P x P)
  const double *const *btab;   // [W * 22 + Qf]: B0 | B1 (Qf x P each)
  const double *const *qtab;   // [Qf]: w (Qf) | K1 (Qf x Qf) | DQ (Qf x Qf)
  int self_only;
  int only_W;
  const int64_t *bf_off;       // Dirichlet data: [6 E] offset of (e, f)'s samples, -1 if not a Dirichlet face
  int64_t nface_pts;           // per rhs
};

constexpr int QM = 2 * HPSE_MAX_W + 1, QM2 = QM * QM, PMC = HPSE_MAX_W + 1;

// out = M_p2 in M_p1^T-style products on [p2][p1] arrays: out[r][c] = sum_k
// A[r][k] B[c][l] in[k][l] with A (n2 x m2), B (n1 x m1) row-major; either may
// be transposed (tA / tB: A^T, B^T).  Two passes through tmp.
template <typename T>
__device__ void c_kron(const double *A, int n2, int m2, bool tA, const double *B, int n1, int m1, bool tB,
                       const T *in, T *tmp, T *out) {
  // in: (tA ? n2 : m2) rows x (tB ? n1 : m1) columns
  const int ir = tA ? n2 : m2, ic = tB ? n1 : m1;
  const int orr = tA ? m2 : n2, oc = tB ? m1 : n1;
  for (int t = threadIdx.x; t < ir * oc; t += blockDim.x) {
    const int r = t / oc, c = t - r * oc;
    T acc = 0;
    for (int l = 0; l < ic; ++l) acc += (T)(tB ? B[l * m1 + c] : B[c * m1 + l]) * in[r * ic + l];
    tmp[t] = acc;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < orr * oc; t += blockDim.x) {
    const int r = t / oc, c = t - r * oc;
    T acc = 0;
    for (int k = 0; k < ir; ++k) acc += (T)(tA ? A[k * m2 + r] : A[r * m2 + k]) * tmp[k * oc + c];
    out[t] = acc;
  }
  __syncthreads();
}

// the fields (u, u_0, u_1, u_2) (reference derivatives) of a P^3 block on face
// f's Qf x Qf grid [p2][p1]: the layer and the normal derivative by D, then
// B0 / B1 along the tangential axes
template <typename T>
__device__ void face_fields(const T *blk, int P, int f, int Qf, const double *D, const double *B0, const double *B1,
                            T *lay, T *nrm, T *tmp, T *F[4]) {
  const int a = f >> 1, end = (f & 1) ? P - 1 : 0;
  for (int t = threadIdx.x; t < P * P; t += blockDim.x) {
    const int p1 = t % P, p2 = t / P;
    T nv = 0;
    for (int k = 0; k < P; ++k) {
      const int i = a == 0 ? k : p1, j = a == 1 ? k : (a == 0 ? p1 : p2), kk = a == 2 ? k : p2;
      nv += (T)D[end * P + k] * blk[(kk * P + j) * P + i];
    }
    const int i = a == 0 ? end : p1, j = a == 1 ? end : (a == 0 ? p1 : p2), kk = a == 2 ? end : p2;
    lay[t] = blk[(kk * P + j) * P + i];
    nrm[t] = nv;
  }
  __syncthreads();
  const int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
  c_kron<T>(B0, Qf, P, false, B0, Qf, P, false, lay, tmp, F[0]);   // u
  c_kron<T>(B0, Qf, P, false, B1, Qf, P, false, lay, tmp, F[1 + t1]);  // d/d lambda_t1
  c_kron<T>(B1, Qf, P, false, B0, Qf, P, false, lay, tmp, F[1 + t2]);  // d/d lambda_t2
  c_kron<T>(B0, Qf, P, false, B0, Qf, P, false, nrm, tmp, F[1 + a]);  // d/d lambda_a
}

// H^{1/2} form of eq. (5.49) on a Qf x Qf grid: out = (w x w + w x K1 + K1 x w) in
template <typename T>
__device__ void h12(const double *w, const double *K1, int Qf, const T *in, T *tmp, T *out) {
  const int n = Qf * Qf;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int r = t / Qf, c = t - r * Qf;
    T acc = (T)w[c] * in[t];
    for (int l = 0; l < Qf; ++l) acc += (T)K1[c * Qf + l] * in[r * Qf + l];
    tmp[t] = acc;  // (w + K1) along p1
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int r = t / Qf, c = t - r * Qf;
    T acc = (T)w[r] * tmp[t];
    for (int k = 0; k < Qf; ++k) acc += (T)K1[r * Qf + k] * (T)w[c] * in[k * Qf + c];
    out[t] = acc;
  }
  __syncthreads();
}

// Face terms of curved elements, y += (and, PCG mode, partial += p . terms);
// one block per (element, rhs), its six faces one after the other.
// MODE 0 plain, 1 PCG; DATA: the Dirichlet data part of b instead (u unused,
// g the samples, y = b).
template <typename T, int MODE, bool DATA>
__global__ void k_face_curved(FaceArgs A, const T *u, const T *K, const double *g, T *y, double *partial) {
  extern __shared__ __align__(16) unsigned char cur_raw[];
  T *sm = reinterpret_cast<T *>(cur_raw);
  const int e = blockIdx.x / A.n_rhs, r = blockIdx.x - e * A.n_rhs;
  const int We = A.elem_W[e], Pe = We + 1, Pe3 = Pe * Pe * Pe;
  if (A.only_W && We != A.only_W) return;
  T *ue = sm, *ye = ue + PMC * PMC * PMC;
  T *lay = ye + PMC * PMC * PMC, *nrm = lay + PMC * PMC;
  T *buf = nrm + PMC * PMC;  // 16 Qf^2 arrays
  T *Fe[4] = {buf, buf + QM2, buf + 2 * QM2, buf + 3 * QM2};
  T *Fn[4] = {buf + 4 * QM2, buf + 5 * QM2, buf + 6 * QM2, buf + 7 * QM2};
  T *G[4] = {buf + 8 * QM2, buf + 9 * QM2, buf + 10 * QM2, buf + 11 * QM2};
  T *tmp = buf + 12 * QM2, *tmp2 = buf + 13 * QM2, *R = buf + 14 * QM2;
  const int64_t base = (int64_t)r * A.ndof + A.dof_off[e];
  for (int t = threadIdx.x; t < Pe3; t += blockDim.x) {
    ue[t] = DATA ? (T)0 : u[base + t];
    ye[t] = 0;
  }
  __syncthreads();
  const double *De = A.dtab[We];
  for (int f = 0; f < 6; ++f) {
    const int nb = A.nbr[6 * (int64_t)e + f];
    if (DATA && (nb != -1 || A.bf_off[6 * (int64_t)e + f] < 0)) continue;
    const int Qf = A.cf_q[6 * (int64_t)e + f], Q2f = Qf * Qf;
    const double *qt = A.qtab[Qf], *w = qt, *K1 = qt + Qf, *DQ = K1 + Qf * Qf;
    const double *B0e = A.btab[We * 22 + Qf], *B1e = B0e + Qf * Pe;
    const int a = f >> 1, end = (f & 1) ? Pe - 1 : 0;
    const int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
    if (nb == -1) {
      // Dirichlet face: G0 = W2 s0, G_t1 = H s1, G_t2 = H s2 with the samples of
      // u (or, DATA, of g and its Qf-grid derivatives)
      if (DATA) {
        const double *gs = g + (int64_t)r * A.nface_pts + A.bf_off[6 * (int64_t)e + f];
        for (int t = threadIdx.x; t < Q2f; t += blockDim.x) {
          const int rr = t / Qf, c = t - rr * Qf;
          T d1 = 0, d2 = 0;
          for (int l = 0; l < Qf; ++l) {
            d1 += (T)DQ[c * Qf + l] * (T)gs[rr * Qf + l];
            d2 += (T)DQ[rr * Qf + l] * (T)gs[l * Qf + c];
          }
          Fe[0][t] = (T)gs[t];
          Fe[1 + t1][t] = d1;
          Fe[1 + t2][t] = d2;
        }
        __syncthreads();
      } else {
        face_fields<T>(ue, Pe, f, Qf, De, B0e, B1e, lay, nrm, tmp, Fe);
      }
      for (int t = threadIdx.x; t < Q2f; t += blockDim.x) G[0][t] = (T)(w[t / Qf] * w[t % Qf]) * Fe[0][t];
      __syncthreads();
      h12<T>(w, K1, Qf, Fe[1 + t1], tmp, G[1 + t1]);
      h12<T>(w, K1, Qf, Fe[1 + t2], tmp, G[1 + t2]);
      // layer: (B0 x B0)^T G0 + (B0 x B1)^T G_t1 + (B1 x B0)^T G_t2
      c_kron<T>(B0e, Qf, Pe, true, B0e, Qf, Pe, true, G[0], tmp, lay);
      c_kron<T>(B0e, Qf, Pe, true, B1e, Qf, Pe, true, G[1 + t1], tmp, tmp2);
      for (int t = threadIdx.x; t < Pe * Pe; t += blockDim.x) lay[t] += tmp2[t];
      __syncthreads();
      c_kron<T>(B1e, Qf, Pe, true, B0e, Qf, Pe, true, G[1 + t2], tmp, tmp2);
      for (int t = threadIdx.x; t < Pe * Pe; t += blockDim.x) {
        lay[t] += tmp2[t];
        nrm[t] = 0;
      }
      __syncthreads();
    } else {
      // interior face: own and neighbour fields, physical gradients, jumps
      face_fields<T>(ue, Pe, f, Qf, De, B0e, B1e, lay, nrm, tmp, Fe);
      const T *Ke = K + 9 * A.cf_off[6 * (int64_t)e + f];
      const int Wn = A.elem_W[nb], Pn = Wn + 1;
      const T *Kn = K + 9 * A.cf_off[6 * (int64_t)nb + (f ^ 1)];
      if (A.self_only) {
        for (int t = threadIdx.x; t < Q2f; t += blockDim.x)
          for (int k = 0; k < 4; ++k) Fn[k][t] = 0;
        __syncthreads();
      } else {
        // the neighbour's block, into ye's unused tail? no: into tmp2 region
        // chain (Pn^3 <= 1331 <= 3 Qf-grid arrays of QM2 = 441)
        T *un = G[0];
        const int64_t nbase = (int64_t)r * A.ndof + A.dof_off[nb];
        for (int t = threadIdx.x; t < Pn * Pn * Pn; t += blockDim.x) un[t] = u[nbase + t];
        __syncthreads();
        face_fields<T>(un, Pn, f ^ 1, Qf, A.dtab[Wn], A.btab[Wn * 22 + Qf], A.btab[Wn * 22 + Qf] + Qf * Pn, tmp2,
                       R, tmp, Fn);
      }
      // jumps: J0 (G0) = u - u_n (W2 applied), J_i = g_i - g_i,n (into Fn[1..3] slots
      // reused), then H; R_a = sum_i Ke[a][i] G_i
      for (int t = threadIdx.x; t < Q2f; t += blockDim.x) {
        T ge[3], gn[3];
        for (int i = 0; i < 3; ++i) {
          ge[i] = Ke[9 * t + 0 * 3 + i] * Fe[1][t] + Ke[9 * t + 1 * 3 + i] * Fe[2][t] + Ke[9 * t + 2 * 3 + i] * Fe[3][t];
          gn[i] = Kn[9 * t + 0 * 3 + i] * Fn[1][t] + Kn[9 * t + 1 * 3 + i] * Fn[2][t] + Kn[9 * t + 2 * 3 + i] * Fn[3][t];
        }
        G[0][t] = (T)(w[t / Qf] * w[t % Qf]) * (Fe[0][t] - Fn[0][t]);
        for (int i = 0; i < 3; ++i) Fn[1 + i][t] = ge[i] - gn[i];
      }
      __syncthreads();
      for (int i = 0; i < 3; ++i) h12<T>(w, K1, Qf, Fn[1 + i], tmp, G[1 + i]);
      // reference cotangents R_a (a = 0, 1, 2) into Fe[1 + a]
      for (int t = threadIdx.x; t < Q2f; t += blockDim.x)
        for (int b = 0; b < 3; ++b)
          Fe[1 + b][t] = Ke[9 * t + 3 * b + 0] * G[1][t] + Ke[9 * t + 3 * b + 1] * G[2][t] + Ke[9 * t + 3 * b + 2] * G[3][t];
      __syncthreads();
      c_kron<T>(B0e, Qf, Pe, true, B0e, Qf, Pe, true, G[0], tmp, lay);
      c_kron<T>(B0e, Qf, Pe, true, B1e, Qf, Pe, true, Fe[1 + t1], tmp, tmp2);
      for (int t = threadIdx.x; t < Pe * Pe; t += blockDim.x) lay[t] += tmp2[t];
      __syncthreads();
      c_kron<T>(B1e, Qf, Pe, true, B0e, Qf, Pe, true, Fe[1 + t2], tmp, tmp2);
      for (int t = threadIdx.x; t < Pe * Pe; t += blockDim.x) lay[t] += tmp2[t];
      __syncthreads();
      c_kron<T>(B0e, Qf, Pe, true, B0e, Qf, Pe, true, Fe[1 + a], tmp, nrm);
    }
    // gather: the face layer takes lay, every node of a normal line D[end][k] nrm
    for (int t = threadIdx.x; t < Pe3; t += blockDim.x) {
      const int i = t % Pe, j = (t / Pe) % Pe, kk = t / (Pe * Pe);
      const int n = a == 0 ? i : (a == 1 ? j : kk);
      const int p1 = a == 0 ? j : i, p2 = a == 2 ? j : kk;
      const int sp = p2 * Pe + p1;
      T acc = (T)De[end * Pe + n] * nrm[sp];
      if (n == end) acc += lay[sp];
      ye[t] += acc;
    }
    __syncthreads();
  }
  double part = 0.0;
  for (int t = threadIdx.x; t < Pe3; t += blockDim.x) {
    y[base + t] += ye[t];
    if (MODE == 1) part += (double)ye[t] * (double)ue[t];
  }
  if (MODE == 1) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) tot += red[wv];
      partial[(int64_t)e * A.n_rhs + r] += tot;
    }
  }
}

inline size_t face_smem(size_t real_bytes) {
  return (size_t)(2 * PMC * PMC * PMC + 2 * PMC * PMC + 15 * QM2) * real_bytes;
}

}  // namespace curved
