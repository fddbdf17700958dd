// kernels.cuh -- device kernels of the least-squares h-p spectral element
// operator, instantiated once per (scalar type REAL, degree WDEG) translation
// unit.  The including file defines REAL (double or float) and WDEG (1..10).
//
// Method (A. Husain 2010): the normal operator A = S^T M S of the functional
// of eq. (4.2) on box elements, applied matrix-free (Section 5.3), and the
// separable block preconditioner C^{-1} (eq. 5.19-5.20).
//
// Design (GB300, sm_103a):
//  * one CTA per (element, right-hand side) work item; the element's nodal
//    block, the partially transformed fields and its output live in shared
//    memory; nothing of size (2W+1)^3 ever reaches global memory;
//  * every 1-D contraction is a fully unrolled loop whose matrix entry is a
//    compile-time index into __constant__ memory, so each FMA takes it as an
//    immediate constant-bank operand (warp-uniform, no load instruction);
//  * the z-stage of the forward sum factorisation, the pointwise weighting
//    and the z-stage of the transpose are fused per (x, y) line in registers;
//  * face terms are applied in the nodal face space: the Q-grid face norms
//    of Section 5.3 equal the Kronecker sums (B0^T W B0) x (B0^T W B0) etc. of
//    P x P matrices, which is exact algebra, not an approximation;
//  * reductions for PCG are written per work item in FP64 and summed by a
//    separate deterministic kernel (no atomics, bitwise reproducible).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "registry.h"

#ifndef REAL
#error "define REAL before including kernels.cuh"
#endif
#ifndef WDEG
#error "define WDEG before including kernels.cuh"
#endif

namespace {

constexpr int W = WDEG;
constexpr int P = W + 1;
constexpr int Q = 2 * W + 1;
constexpr int P2 = P * P;
constexpr int P3 = P * P * P;
constexpr int Q2 = Q * Q;
constexpr int QP = Q * P;
constexpr int QP2 = Q * P * P;
constexpr int Q2P = Q * Q * P;

typedef REAL real;

// 1-D tables of this degree (filled by upload_tables):
//   B[m][q*P+k]  = d^m l_k / dlambda^m at the q-th (2W+1)-point GLL node
//   D[i*P+k]     = GLL differentiation matrix on the (W+1)-point grid (eq. 5.47)
//   S[k*P+c]     = preconditioner eigenvectors (node k, mode c), eq. (5.15)-(5.17)
//   MP, KP       = B0^T diag(w) B0 and B0^T K B0 (P x P face-norm matrices)
//   WQ[q]        = (2W+1)-point GLL weights; MU[c] = eigenvalues of eq. (5.15)
struct Tables {
  real B[3][QP];
  real D[P2];
  real S[P2];
  real MP[P2];
  real KP[P2];
  real WQ[Q];
  real MU[P];
};
__constant__ Tables c_tab;

using hpse::COEF_LAPLACE;
using hpse::COEF_SCALAR;
using hpse::MODE_PLAIN;
using hpse::MODE_PCG;
using hpse::MODE_TRANSPOSE;
typedef hpse::ApplyArgsT<real> ApplyArgs;
typedef hpse::PrecArgsT<real> PrecArgs;

// index of u(normal index n, tangential p1 (t1), p2 (t2)) for face axis a
__device__ __forceinline__ int fidx(int a, int n, int p1, int p2) {
  // array u[k][j][i]; t1 < t2 are the axes other than a
  if (a == 0) return (p2 * P + p1) * P + n;   // (i=n, j=p1, k=p2)
  if (a == 1) return (p2 * P + n) * P + p1;   // (i=p1, j=n, k=p2)
  return (n * P + p2) * P + p1;               // (i=p1, j=p2, k=n)
}

template <typename T>
__device__ __forceinline__ double block_sum(T v, double *red) {
  double s = (double)v;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = s;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < nw; ++i) t += red[i];
  }
  return t;  // valid in thread 0
}

// ---------------------------------------------------------------------------
// Face phase: y_e += contributions of the six faces of element e (eq. 4.2).
// su: own block, snb: scratch P3, scr: scratch >= 10*P2, tabs: D, MP, KP copy
// ---------------------------------------------------------------------------
// out = (A (x) B) v with A acting on p2 and B on p1 (face arrays [p2][p1])
__device__ __forceinline__ void kron_apply(const real *Am, const real *Bm, const real *v, real *tmp, real *out,
                                           bool accumulate) {
  for (int t = threadIdx.x; t < P2; t += blockDim.x) {
    const int p1 = t % P, p2 = t / P;
    real s = 0;
#pragma unroll
    for (int m = 0; m < P; ++m) s += Bm[p1 * P + m] * v[p2 * P + m];
    tmp[t] = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < P2; t += blockDim.x) {
    const int p1 = t % P, p2 = t / P;
    real s = 0;
#pragma unroll
    for (int m = 0; m < P; ++m) s += Am[p2 * P + m] * tmp[m * P + p1];
    out[t] = accumulate ? out[t] + s : s;
  }
  __syncthreads();
}

// g = (MP x MP + MP x KP + KP x MP) v  -- the H^{1/2} face form in nodal space
__device__ __forceinline__ void half_norm_apply(const real *MPs, const real *KPs, const real *v, real *ta, real *tb,
                                                real *g) {
  for (int t = threadIdx.x; t < P2; t += blockDim.x) {
    const int p1 = t % P, p2 = t / P;
    real a = 0, b = 0;
#pragma unroll
    for (int m = 0; m < P; ++m) {
      a += MPs[p1 * P + m] * v[p2 * P + m];
      b += KPs[p1 * P + m] * v[p2 * P + m];
    }
    ta[t] = a;
    tb[t] = a + b;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < P2; t += blockDim.x) {
    const int p1 = t % P, p2 = t / P;
    real s = 0;
#pragma unroll
    for (int m = 0; m < P; ++m) s += MPs[p2 * P + m] * tb[m * P + p1] + KPs[p2 * P + m] * ta[m * P + p1];
    g[t] = s;
  }
  __syncthreads();
}

// traces of block blk on face (a, nend): F = u, N = du/dlambda_a, G1, G2 tangential
__device__ __forceinline__ void face_traces(const real *blk, int a, int nend, const real *Ds, real *F, real *N,
                                            real *G1, real *G2) {
  for (int t = threadIdx.x; t < P2; t += blockDim.x) {
    const int p1 = t % P, p2 = t / P;
    F[t] = blk[fidx(a, nend, p1, p2)];
    real s = 0;
#pragma unroll
    for (int k = 0; k < P; ++k) s += Ds[nend * P + k] * blk[fidx(a, k, p1, p2)];
    N[t] = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < P2; t += blockDim.x) {
    const int p1 = t % P, p2 = t / P;
    real s1 = 0, s2 = 0;
#pragma unroll
    for (int m = 0; m < P; ++m) {
      s1 += Ds[p1 * P + m] * F[p2 * P + m];
      s2 += Ds[p2 * P + m] * F[m * P + p1];
    }
    G1[t] = s1;
    G2[t] = s2;
  }
  __syncthreads();
}

template <int MODE>
__device__ void face_phase(const ApplyArgs &A, int e, int r, const real *su, real *sy, real *snb, real *scr,
                           const real *Ds, const real *MPs, const real *KPs, const real *geo_e) {
  real *F = scr, *N = scr + P2, *G1 = scr + 2 * P2, *G2 = scr + 3 * P2;
  real *Fn = scr + 4 * P2, *Nn = scr + 5 * P2, *G1n = scr + 6 * P2, *G2n = scr + 7 * P2;
  real *ta = scr + 8 * P2, *tb = scr + 9 * P2;
  real *g0 = scr + 10 * P2, *g1 = scr + 11 * P2, *g2 = scr + 12 * P2, *g3 = scr + 13 * P2;
  for (int fi = 0; fi < 6; ++fi) {
    const int a = fi >> 1, side = fi & 1;
    const int t1 = (a == 0) ? 1 : 0;
    const int t2 = (a == 2) ? 1 : 2;
    const int nend = side ? P - 1 : 0;
    const int nb = A.nbr[(int64_t)e * 6 + fi];
    face_traces(su, a, nend, Ds, F, N, G1, G2);
    if (nb >= 0) {
      // neighbour block of the same right-hand side
      const int64_t base = (int64_t)r * A.ndof + A.dof_off[nb];
      if (MODE == MODE_PCG) {
        const double bt = A.beta[A.prob[nb] * A.n_rhs + r];
        for (int t = threadIdx.x; t < P3; t += blockDim.x)
          snb[t] = A.z[base + t] + (real)bt * A.u[base + t];
      } else {
        for (int t = threadIdx.x; t < P3; t += blockDim.x) snb[t] = A.u[base + t];
      }
      __syncthreads();
      face_traces(snb, a, P - 1 - nend, Ds, Fn, Nn, G1n, G2n);
      const real sa = geo_e[a], s1 = geo_e[t1], s2 = geo_e[t2];
      const real *gn = A.geo + (int64_t)nb * 4;
      const real na = gn[a], n1 = gn[t1], n2 = gn[t2];
      // jumps of u and of the physical derivatives u_{x_k}
      for (int t = threadIdx.x; t < P2; t += blockDim.x) {
        Fn[t] = F[t] - Fn[t];                 // [u]
        G1n[t] = s1 * G1[t] - n1 * G1n[t];    // [u_{x_t1}]
        G2n[t] = s2 * G2[t] - n2 * G2n[t];    // [u_{x_t2}]
        Nn[t] = sa * N[t] - na * Nn[t];       // [u_{x_a}]
      }
      __syncthreads();
      kron_apply(MPs, MPs, Fn, ta, g0, false);
      half_norm_apply(MPs, KPs, G1n, ta, tb, g1);
      half_norm_apply(MPs, KPs, G2n, ta, tb, g2);
      half_norm_apply(MPs, KPs, Nn, ta, tb, g3);
      // transpose of the traces: face layer gets g0 + s1 D^T g1 + s2 D^T g2,
      // every layer k along a gets sa * D[nend][k] * g3
      for (int t = threadIdx.x; t < P2; t += blockDim.x) {
        const int p1 = t % P, p2 = t / P;
        real s = g0[t];
        real u1 = 0, u2 = 0;
#pragma unroll
        for (int m = 0; m < P; ++m) {
          u1 += Ds[m * P + p1] * g1[p2 * P + m];
          u2 += Ds[m * P + p2] * g2[m * P + p1];
        }
        s += s1 * u1 + s2 * u2;
        const real gz = sa * g3[t];
#pragma unroll
        for (int k = 0; k < P; ++k) {
          real add = Ds[nend * P + k] * gz;
          if (k == nend) add += s;
          sy[fidx(a, k, p1, p2)] += add;
        }
      }
      __syncthreads();
    } else {
      // Dirichlet face: ||u||_0^2 + sum_i ||du/dlambda_i||_{1/2}^2 (eq. 2.18)
      kron_apply(MPs, MPs, F, ta, g0, false);
      half_norm_apply(MPs, KPs, G1, ta, tb, g1);
      half_norm_apply(MPs, KPs, G2, ta, tb, g2);
      for (int t = threadIdx.x; t < P2; t += blockDim.x) {
        const int p1 = t % P, p2 = t / P;
        real s = g0[t];
#pragma unroll
        for (int m = 0; m < P; ++m) s += Ds[m * P + p1] * g1[p2 * P + m] + Ds[m * P + p2] * g2[m * P + p1];
        sy[fidx(a, nend, p1, p2)] += s;
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// Operator apply: y = A u  (volume + faces), one CTA per (element, rhs).
// Shared memory: su[P3] | X[NX][QP2] | T[NTF][Q2P] (later reused for sy, snb,
// face scratch) | small tables.
// ---------------------------------------------------------------------------
template <int COEF>
struct ApplyLayout {
  static constexpr int NX = (COEF == COEF_SCALAR) ? 3 : 2;
  static constexpr int NTF = (COEF == COEF_SCALAR) ? 4 : 2;
  static constexpr int T_REGION0 = NTF * Q2P;
  static constexpr int T_NEED = 2 * P3 + 14 * P2;
  static constexpr int T_REGION = T_REGION0 > T_NEED ? T_REGION0 : T_NEED;
  static constexpr int TABS = 3 * P2;
  static constexpr int TOTAL = P3 + NX * QP2 + T_REGION + TABS;
  // the FP64 reduction buffer starts on a 16-byte boundary whatever REAL is
  static constexpr size_t RED_OFF = (((size_t)TOTAL * sizeof(real) + 15) / 16) * 16;
  static constexpr size_t BYTES = RED_OFF + 64 * sizeof(double);
};

#if defined(HPSE_DOUBLE)
#define HPSE_APPLY_MAXT 256
#else
#define HPSE_APPLY_MAXT 384
#endif

template <int COEF, int MODE>
__global__ void __launch_bounds__(HPSE_APPLY_MAXT) k_apply(const ApplyArgs A) {
  typedef ApplyLayout<COEF> L;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real *su = reinterpret_cast<real *>(smem_raw);
  real *sX = su + P3;               // X0 | X2 | (X1)
  real *sT = sX + L::NX * QP2;      // T00 | TL | (T10 | T01)
  real *stab = sT + L::T_REGION;    // D | MP | KP (runtime-indexed copies)
  double *red = reinterpret_cast<double *>(smem_raw + L::RED_OFF);
  static_assert(L::RED_OFF % 16 == 0, "reduction buffer must be 16-byte aligned");
  real *X0 = sX, *X2 = sX + QP2, *X1 = sX + 2 * QP2;
  real *T00 = sT, *TL = sT + Q2P, *T10 = sT + 2 * Q2P, *T01 = sT + 3 * Q2P;

  const int item = blockIdx.x;
  const int ge = item / A.n_rhs;
  const int r = item - ge * A.n_rhs;
  const int e = A.elems[ge];
  const int64_t base = (int64_t)r * A.ndof + A.dof_off[e];
  const real *geo_e = A.geo + (int64_t)e * 4;
  const real sx = geo_e[0], sy_ = geo_e[1], sz = geo_e[2], Jac = geo_e[3];
  const real sx2 = sx * sx, sy2 = sy_ * sy_, sz2 = sz * sz;
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int t = tid; t < P2; t += nt) {
    stab[t] = c_tab.D[t];
    stab[P2 + t] = c_tab.MP[t];
    stab[2 * P2 + t] = c_tab.KP[t];
  }
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

    // ---- x-stage (lines along x: (j, k)) -------------------------------
    for (int l = tid; l < P2; l += nt) {
      real v[P];
#pragma unroll
      for (int i = 0; i < P; ++i) v[i] = su[l * P + i];
      real *o0 = X0 + l * Q, *o2 = X2 + l * Q, *o1 = X1 + l * Q;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        real a0 = 0, a2 = 0, a1 = 0;
#pragma unroll
        for (int i = 0; i < P; ++i) {
          a0 += c_tab.B[0][q * P + i] * v[i];
          a2 += c_tab.B[2][q * P + i] * v[i];
          if (COEF == COEF_SCALAR) a1 += c_tab.B[1][q * P + i] * v[i];
        }
        o0[q] = a0;
        o2[q] = a2;
        if (COEF == COEF_SCALAR) o1[q] = a1;
      }
    }
    __syncthreads();

    // ---- y-stage (lines along y: (qa, k)) -------------------------------
    for (int l = tid; l < QP; l += nt) {
      const int qa = l % Q, k = l / Q;
      real v0[P], v2[P], v1[P];
#pragma unroll
      for (int j = 0; j < P; ++j) {
        v0[j] = X0[(k * P + j) * Q + qa];
        v2[j] = X2[(k * P + j) * Q + qa];
        if (COEF == COEF_SCALAR) v1[j] = X1[(k * P + j) * Q + qa];
      }
#pragma unroll
      for (int qb = 0; qb < Q; ++qb) {
        real t00 = 0, tl0 = 0, tl2 = 0, t10 = 0, t01 = 0;
#pragma unroll
        for (int j = 0; j < P; ++j) {
          t00 += c_tab.B[0][qb * P + j] * v0[j];
          tl0 += c_tab.B[2][qb * P + j] * v0[j];
          tl2 += c_tab.B[0][qb * P + j] * v2[j];
          if (COEF == COEF_SCALAR) {
            t10 += c_tab.B[0][qb * P + j] * v1[j];
            t01 += c_tab.B[1][qb * P + j] * v0[j];
          }
        }
        const int o = (k * Q + qb) * Q + qa;
        T00[o] = t00;
        TL[o] = sx2 * tl2 + sy2 * tl0;
        if (COEF == COEF_SCALAR) {
          T10[o] = t10;
          T01[o] = t01;
        }
      }
    }
    __syncthreads();
  }

  // ---- fused z-stage: forward, pointwise weight, transpose ----------------
  for (int l = tid; l < Q2; l += nt) {
    const int qa = l % Q, qb = l / Q;
    real a00[P], aL[P], a10[P], a01[P];
    real rz[P], r0[P], rx[P], ry[P];
    if (MODE != MODE_TRANSPOSE) {
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const int o = (k * Q + qb) * Q + qa;
        a00[k] = T00[o];
        aL[k] = TL[o];
        if (COEF == COEF_SCALAR) {
          a10[k] = T10[o];
          a01[k] = T01[o];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
      rz[k] = 0;
      r0[k] = 0;
      rx[k] = 0;
      ry[k] = 0;
    }
    const real wab = c_tab.WQ[qa] * c_tab.WQ[qb] * Jac;
    const int64_t cbase = A.coef_off[e] + (int64_t)qb * Q + qa;
#pragma unroll
    for (int qc = 0; qc < Q; ++qc) {
      real rho, dx = 0, dy = 0, dz = 0;
      if (COEF == COEF_SCALAR) {
        const int64_t ci = cbase + (int64_t)qc * Q2;
        dx = A.coef[A.nquad + ci];
        dy = A.coef[2 * A.nquad + ci];
        dz = A.coef[3 * A.nquad + ci];
      }
      if (MODE == MODE_TRANSPOSE) {
        rho = (real)A.rho[(int64_t)r * A.nquad + cbase + (int64_t)qc * Q2];
      } else {
        real s2 = 0, s0 = 0, s1z = 0, sxx = 0, syy = 0;
#pragma unroll
        for (int k = 0; k < P; ++k) {
          s2 += c_tab.B[2][qc * P + k] * a00[k];
          s0 += c_tab.B[0][qc * P + k] * aL[k];
          if (COEF == COEF_SCALAR) {
            s1z += c_tab.B[1][qc * P + k] * a00[k];
            sxx += c_tab.B[0][qc * P + k] * a10[k];
            syy += c_tab.B[0][qc * P + k] * a01[k];
          }
        }
        real sigma = sz2 * s2 + s0;
        if (COEF == COEF_SCALAR) {
          sigma += dz * s1z + dx * sxx + dy * syy;
          rho = A.coef[cbase + (int64_t)qc * Q2] * sigma;
        } else {
          rho = wab * c_tab.WQ[qc] * sigma;
        }
      }
      const real rz2 = sz2 * rho;
      const real rzd = dz * rho, rxd = dx * rho, ryd = dy * rho;
#pragma unroll
      for (int k = 0; k < P; ++k) {
        rz[k] += c_tab.B[2][qc * P + k] * rz2;
        r0[k] += c_tab.B[0][qc * P + k] * rho;
        if (COEF == COEF_SCALAR) {
          rz[k] += c_tab.B[1][qc * P + k] * rzd;
          rx[k] += c_tab.B[0][qc * P + k] * rxd;
          ry[k] += c_tab.B[0][qc * P + k] * ryd;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
      const int o = (k * Q + qb) * Q + qa;
      T00[o] = rz[k];
      TL[o] = r0[k];
      if (COEF == COEF_SCALAR) {
        T10[o] = rx[k];
        T01[o] = ry[k];
      }
    }
  }
  __syncthreads();

  // ---- y-stage transpose (lines (qa, k)) ---------------------------------
  for (int l = tid; l < QP; l += nt) {
    const int qa = l % Q, k = l / Q;
    real vz[Q], v0[Q], vx[Q], vy[Q];
#pragma unroll
    for (int qb = 0; qb < Q; ++qb) {
      const int o = (k * Q + qb) * Q + qa;
      vz[qb] = T00[o];
      v0[qb] = TL[o];
      if (COEF == COEF_SCALAR) {
        vx[qb] = T10[o];
        vy[qb] = T01[o];
      }
    }
#pragma unroll
    for (int j = 0; j < P; ++j) {
      real x0 = 0, x0b = 0, x2 = 0, x1 = 0, x0c = 0;
#pragma unroll
      for (int qb = 0; qb < Q; ++qb) {
        x0 += c_tab.B[0][qb * P + j] * vz[qb];
        x0b += c_tab.B[2][qb * P + j] * v0[qb];
        x2 += c_tab.B[0][qb * P + j] * v0[qb];
        if (COEF == COEF_SCALAR) {
          x1 += c_tab.B[0][qb * P + j] * vx[qb];
          x0c += c_tab.B[1][qb * P + j] * vy[qb];
        }
      }
      const int o = (k * P + j) * Q + qa;
      X0[o] = x0 + sy2 * x0b + x0c;
      X2[o] = sx2 * x2;
      if (COEF == COEF_SCALAR) X1[o] = x1;
    }
  }
  __syncthreads();

  // ---- x-stage transpose (lines (j, k)) -> sy ----------------------------
  real *sy = sT;  // T region is free now
  for (int l = tid; l < P2; l += nt) {
    real v0[Q], v2[Q], v1[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      v0[q] = X0[l * Q + q];
      v2[q] = X2[l * Q + q];
      if (COEF == COEF_SCALAR) v1[q] = X1[l * Q + q];
    }
#pragma unroll
    for (int i = 0; i < P; ++i) {
      real s = 0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        s += c_tab.B[0][q * P + i] * v0[q] + c_tab.B[2][q * P + i] * v2[q];
        if (COEF == COEF_SCALAR) s += c_tab.B[1][q * P + i] * v1[q];
      }
      sy[l * P + i] = s;
    }
  }
  __syncthreads();

  // ---- faces ---------------------------------------------------------------
  if (MODE != MODE_TRANSPOSE && !A.skip_faces) {
    real *snb = sT + P3;
    real *scr = sT + 2 * P3;
    face_phase<MODE>(A, e, r, su, sy, snb, scr, stab, stab + P2, stab + 2 * P2, geo_e);
  }

  // ---- store (and the p.q partial of PCG) --------------------------------
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

// ---------------------------------------------------------------------------
// Preconditioner z = C^{-1} r by fast diagonalisation (eq. 5.19-5.20).
// MODE_PCG also performs the PCG update x += alpha p, r -= alpha q first and
// writes the partial sums r.r and r.z.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tensor_stage(const real *in, real *out, int axis, bool transpose) {
  // out = (S^T or S) applied along `axis` of a P x P x P block (x fastest)
  const int stride = axis == 0 ? 1 : (axis == 1 ? P : P2);
  for (int l = threadIdx.x; l < P2; l += blockDim.x) {
    int b;
    if (axis == 0) b = l * P;
    else if (axis == 1) b = (l / P) * P2 + (l % P);
    else b = l;
    real v[P];
#pragma unroll
    for (int k = 0; k < P; ++k) v[k] = in[b + k * stride];
#pragma unroll
    for (int c = 0; c < P; ++c) {
      real s = 0;
#pragma unroll
      for (int k = 0; k < P; ++k) s += (transpose ? c_tab.S[k * P + c] : c_tab.S[c * P + k]) * v[k];
      out[b + c * stride] = s;
    }
  }
  __syncthreads();
}

template <int MODE>
__global__ void __launch_bounds__(256) k_precond(const PrecArgs A) {
  __shared__ __align__(16) real s0[P3];
  __shared__ __align__(16) real s1[P3];
  __shared__ real smu[P];
  __shared__ double red[32];
  const int item = blockIdx.x;
  const int ge = item / A.n_rhs;
  const int rr = item - ge * A.n_rhs;
  const int e = A.elems[ge];
  const int64_t base = (int64_t)rr * A.ndof + A.dof_off[e];
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid < P) smu[tid] = c_tab.MU[tid];
  double prr = 0.0;
  if (MODE == MODE_PCG) {
    const real al = (real)A.alpha[A.prob[e] * A.n_rhs + rr];
    for (int t = tid; t < P3; t += nt) {
      const real pv = A.p[base + t];
      if (A.x) A.x[base + t] += al * pv;
      const real rv = A.r[base + t] - al * A.q[base + t];
      A.r[base + t] = rv;
      s0[t] = rv;
      prr += (double)rv * (double)rv;
    }
  } else {
    for (int t = tid; t < P3; t += nt) s0[t] = A.rin[base + t];
  }
  __syncthreads();
  tensor_stage(s0, s1, 0, true);
  tensor_stage(s1, s0, 1, true);
  tensor_stage(s0, s1, 2, true);
  for (int t = tid; t < P3; t += nt) {
    const int a = t % P, b = (t / P) % P, c = t / P2;
    s1[t] = s1[t] / (smu[a] + smu[b] + smu[c] + (real)1);
  }
  __syncthreads();
  tensor_stage(s1, s0, 2, false);
  tensor_stage(s0, s1, 1, false);
  tensor_stage(s1, s0, 0, false);
  double prz = 0.0;
  for (int t = tid; t < P3; t += nt) {
    const real zv = s0[t];
    A.zout[base + t] = zv;
    if (MODE == MODE_PCG) prz += (double)zv * (double)A.r[base + t];
  }
  if (MODE == MODE_PCG) {
    const double a = block_sum(prr, red);
    const double b = block_sum(prz, red);
    if (tid == 0) {
      A.part_rr[(int64_t)e * A.n_rhs + rr] = a;
      A.part_rz[(int64_t)e * A.n_rhs + rr] = b;
    }
  }
}

}  // namespace
