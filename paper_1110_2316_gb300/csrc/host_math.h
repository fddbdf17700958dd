// host_math.h -- FP64 host computation of the 1-D tables of the method:
// Gauss-Lobatto-Legendre rules (Section 5.3), Lagrange interpolation and
// differentiation (eq. 5.47), the discrete H^{1/2} face form (Section 5.3,
// eq. 5.49) and the 1-D generalised eigenproblem of the separable
// preconditioner (eq. 5.11-5.17).  Plain C++, no CUDA.
#pragma once
#include <cmath>
#include <vector>

namespace hpse {
namespace hm {

// Legendre L_n(x) and its derivative by the three-term recurrence.
inline void legendre_and_deriv(int n, double x, double *Ln, double *dLn) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    *Ln = 1.0;
    *dLn = 0.0;
    return;
  }
  double d0 = 0.0, d1 = 1.0;
  for (int m = 1; m < n; ++m) {
    const double p2 = ((2.0 * m + 1.0) * x * p1 - m * p0) / (m + 1.0);
    const double d2 = d0 + (2.0 * m + 1.0) * p1;  // L'_{m+1} = L'_{m-1} + (2m+1) L_m
    p0 = p1;
    p1 = p2;
    d0 = d1;
    d1 = d2;
  }
  *Ln = p1;
  *dLn = d1;
}

// GLL rule with n points: -1, +1 and the zeros of L'_{n-1} found by Newton's
// method on q(x) = L'_N(x) (q' from the Legendre equation
// (1 - x^2) L''_N = 2x L'_N - N(N+1) L_N), started from Chebyshev-Gauss-Lobatto
// points; weights 2 / (N (N+1) L_N(x_i)^2).
inline void gll_rule(int n, std::vector<double> &x, std::vector<double> &w) {
  const int N = n - 1;
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  x[0] = -1.0;
  x[N] = 1.0;
  for (int i = 1; i < N; ++i) {
    double t = -std::cos(M_PI * i / N);
    for (int it = 0; it < 100; ++it) {
      double L, dL;
      legendre_and_deriv(N, t, &L, &dL);
      const double d2L = (2.0 * t * dL - N * (N + 1.0) * L) / (1.0 - t * t);
      const double dt = dL / d2L;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[i] = t;
  }
  // symmetrise (the rule is symmetric about 0)
  for (int i = 0; i < n / 2; ++i) {
    const double s = 0.5 * (x[N - i] - x[i]);
    x[i] = -s;
    x[N - i] = s;
  }
  if (n % 2) x[N / 2] = 0.0;
  for (int i = 0; i < n; ++i) {
    double L, dL;
    legendre_and_deriv(N, x[i], &L, &dL);
    w[i] = 2.0 / (N * (N + 1.0) * L * L);
  }
}

// Barycentric weights of the nodes.
inline std::vector<double> bary_weights(const std::vector<double> &x) {
  const int n = (int)x.size();
  std::vector<double> lam(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int m = 0; m < n; ++m)
      if (m != j) lam[j] /= (x[j] - x[m]);
  return lam;
}

// Differentiation matrix D[i][j] = l_j'(x_i) on the nodes (eq. 5.47), from the
// barycentric weights: D_ij = (lam_j / lam_i) / (x_i - x_j), D_ii = -sum_{j!=i} D_ij.
inline std::vector<double> diff_matrix(const std::vector<double> &x) {
  const int n = (int)x.size();
  const std::vector<double> lam = bary_weights(x);
  std::vector<double> D(n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      D[i * n + j] = (lam[j] / lam[i]) / (x[i] - x[j]);
      s += D[i * n + j];
    }
    D[i * n + i] = -s;
  }
  return D;
}

// Interpolation matrix I[q][j] = l_j(y_q) (barycentric formula of the second kind).
inline std::vector<double> interp_matrix(const std::vector<double> &x, const std::vector<double> &y) {
  const int n = (int)x.size(), m = (int)y.size();
  const std::vector<double> lam = bary_weights(x);
  std::vector<double> I(m * n, 0.0);
  for (int q = 0; q < m; ++q) {
    int hit = -1;
    for (int j = 0; j < n; ++j)
      if (y[q] == x[j]) hit = j;
    if (hit >= 0) {
      I[q * n + hit] = 1.0;
      continue;
    }
    double den = 0.0;
    for (int j = 0; j < n; ++j) den += lam[j] / (y[q] - x[j]);
    for (int j = 0; j < n; ++j) I[q * n + j] = (lam[j] / (y[q] - x[j])) / den;
  }
  return I;
}

inline std::vector<double> matmul(const std::vector<double> &A, const std::vector<double> &B, int m, int k, int n) {
  std::vector<double> C(m * n, 0.0);
  for (int i = 0; i < m; ++i)
    for (int l = 0; l < k; ++l) {
      const double a = A[i * k + l];
      for (int j = 0; j < n; ++j) C[i * n + j] += a * B[l * n + j];
    }
  return C;
}

// 1-D H^{1/2} matrix on an n-point GLL grid: l^T K l = sum_{i!=i'} w_i w_i'
// ((l_i - l_i')/(x_i - x_i'))^2 + sum_i w_i^2 (D l)_i^2  (Section 5.3).
inline std::vector<double> half_norm_matrix(const std::vector<double> &x, const std::vector<double> &w) {
  const int n = (int)x.size();
  const std::vector<double> D = diff_matrix(x);
  std::vector<double> K(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += D[k * n + i] * w[k] * w[k] * D[k * n + j];
      K[i * n + j] = s;
    }
  for (int i = 0; i < n; ++i)
    for (int ip = 0; ip < n; ++ip) {
      if (i == ip) continue;
      const double c = w[i] * w[ip] / ((x[i] - x[ip]) * (x[i] - x[ip]));
      K[i * n + i] += c;
      K[ip * n + ip] += c;
      K[i * n + ip] -= c;
      K[ip * n + i] -= c;
    }
  return K;
}

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix A (row-major):
// A = V diag(ev) V^T, eigenvalues ascending, eigenvectors in the columns of V.
inline void jacobi_eigen(std::vector<double> A, int n, std::vector<double> &ev, std::vector<double> &V) {
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += A[i * n + j] * A[i * n + j];
        if (i != j) off += A[i * n + j] * A[i * n + j];
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = A[p * n + p], aqq = A[q * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  ev.assign(n, 0.0);
  for (int i = 0; i < n; ++i) ev[i] = A[i * n + i];
  // sort ascending
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (ev[idx[j]] < ev[idx[i]]) {
        const int t = idx[i];
        idx[i] = idx[j];
        idx[j] = t;
      }
  std::vector<double> ev2(n), V2(n * n);
  for (int c = 0; c < n; ++c) {
    ev2[c] = ev[idx[c]];
    for (int k = 0; k < n; ++k) V2[k * n + c] = V[k * n + idx[c]];
  }
  ev = ev2;
  V = V2;
}

// All tables of degree W (packed in the order of registry.h) plus the FP64
// Q-grid face tables used when building the right-hand side.
struct DegreeTables {
  int W, P, Q;
  std::vector<double> xp, wp, xq, wq;
  std::vector<double> B0, B1, B2;  // Q x P
  std::vector<double> D;           // P x P
  std::vector<double> S, mu;       // eigenvectors (node, mode), eigenvalues
  std::vector<double> MP, KP;      // P x P face forms
  std::vector<double> DQ, KQ;      // Q x Q differentiation and H^{1/2} matrices
  std::vector<double> packed;
};

inline DegreeTables build_tables(int W) {
  DegreeTables t;
  t.W = W;
  t.P = W + 1;
  t.Q = 2 * W + 1;
  const int P = t.P, Q = t.Q;
  gll_rule(P, t.xp, t.wp);
  gll_rule(Q, t.xq, t.wq);
  t.D = diff_matrix(t.xp);
  t.B0 = interp_matrix(t.xp, t.xq);
  t.B1 = matmul(t.B0, t.D, Q, P, P);         // derivative of the interpolant (exact)
  t.B2 = matmul(t.B1, t.D, Q, P, P);
  t.DQ = diff_matrix(t.xq);
  t.KQ = half_norm_matrix(t.xq, t.wq);
  // face forms in nodal space: MP = B0^T W B0, KP = B0^T K B0
  t.MP.assign(P * P, 0.0);
  t.KP.assign(P * P, 0.0);
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) {
      double m = 0.0, k = 0.0;
      for (int a = 0; a < Q; ++a) {
        m += t.B0[a * P + i] * t.wq[a] * t.B0[a * P + j];
        for (int b = 0; b < Q; ++b) k += t.B0[a * P + i] * t.KQ[a * Q + b] * t.B0[b * P + j];
      }
      t.MP[i * P + j] = m;
      t.KP[i * P + j] = k;
    }
  // preconditioner: E = D2^T Wp D2 + D^T Wp D, F = Wp ((W+1)-point GLL, Table 5.1
  // convention); symmetric form F^{-1/2} E F^{-1/2} = V diag(mu) V^T, S = F^{-1/2} V.
  const std::vector<double> D2 = matmul(t.D, t.D, P, P, P);
  std::vector<double> E(P * P, 0.0);
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) {
      double s = 0.0;
      for (int k = 0; k < P; ++k) s += t.wp[k] * (D2[k * P + i] * D2[k * P + j] + t.D[k * P + i] * t.D[k * P + j]);
      E[i * P + j] = s / std::sqrt(t.wp[i] * t.wp[j]);
    }
  std::vector<double> V;
  jacobi_eigen(E, P, t.mu, V);
  for (int i = 0; i < P; ++i) t.mu[i] = t.mu[i] < 0 ? 0.0 : t.mu[i];
  t.S.assign(P * P, 0.0);
  for (int k = 0; k < P; ++k)
    for (int c = 0; c < P; ++c) t.S[k * P + c] = V[k * P + c] / std::sqrt(t.wp[k]);
  t.packed.clear();
  for (double v : t.B0) t.packed.push_back(v);
  for (double v : t.B1) t.packed.push_back(v);
  for (double v : t.B2) t.packed.push_back(v);
  for (double v : t.D) t.packed.push_back(v);
  for (double v : t.S) t.packed.push_back(v);
  for (double v : t.MP) t.packed.push_back(v);
  for (double v : t.KP) t.packed.push_back(v);
  for (double v : t.wq) t.packed.push_back(v);
  for (double v : t.mu) t.packed.push_back(v);
  for (double v : t.DQ) t.packed.push_back(v);
  return t;
}

}  // namespace hm
}  // namespace hpse
