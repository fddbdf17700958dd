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

#include <type_traits>

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

// even-odd folding of the symmetric GLL grids: HP mirrored node pairs of the
// P-grid (plus its middle node when P is odd: HPE = ceil(P / 2) folded
// entries) and HQ = W mirrored point pairs of the Q-grid around its middle
// point q = W
constexpr int HP = P / 2;
constexpr int HPE = (P + 1) / 2;
constexpr int HQ = W;
// B1 is odd under the reflection of both grids, B0 and B2 even
__host__ __device__ constexpr bool odd_mat(int m) { return m == 1; }
// P x P matrices of the face phase: D and D^T are odd, MP and KP even
__host__ __device__ constexpr bool odd_pp(int t) { return t < 2; }

// Threads per apply CTA: one thread per z-line (Q^2 lines) rounded up to
// whole warps, capped; every stage then runs at most once per thread when
// Q^2 <= NT, so no constant-table read is loop-invariant across line
// iterations and every FMA keeps its constant-bank operand.
#if defined(HPSE_DOUBLE)
#define HPSE_APPLY_MAXT 256
#else
#define HPSE_APPLY_MAXT 448
#endif
#define PAD32(n) ((((n) + 31) / 32) * 32)
constexpr int NT_RAW = PAD32(Q2);
#if defined(HPSE_APPLY_NT)
constexpr int NT = HPSE_APPLY_NT;  // set at build time (launch-shape experiments)
#else
constexpr int NT = NT_RAW < 64 ? 64 : (NT_RAW > HPSE_APPLY_MAXT ? HPSE_APPLY_MAXT : NT_RAW);
#endif
static_assert(NT % 32 == 0, "warp-uniform line loops need a whole number of warps per CTA");
// FP32: enough resident CTAs for ~30 warps per SM (measured best on GB300 for
// W = 8: 3 CTAs of 320 threads); FP64 is bound by the FP64 pipe at any occupancy
constexpr int APPLY_MINB_RAW = 960 / NT;
#if defined(HPSE_APPLY_MINB)
constexpr int APPLY_MINB = HPSE_APPLY_MINB;  // set at build time (launch-shape experiments)
#else
constexpr int APPLY_MINB = sizeof(real) == 8 ? 1 : (APPLY_MINB_RAW < 1 ? 1 : (APPLY_MINB_RAW > 4 ? 4 : APPLY_MINB_RAW));
#endif


// 1-D tables of this degree (filled by upload_tables):
//   B[m][q*P+k]  = d^m l_k / dlambda^m at the q-th (2W+1)-point GLL node
//   FE[m][q*HPE+j], FO[m][q*HPE+j] (q = 0..W) = the folded halves of B[m]:
//                  (B[m][q][j] +- B[m][q][P-1-j]) / 2 for j < HP; the middle
//                  column (P odd) is B[m][q][HP] in FE and 0 in FO
//   PF[t][0|1][i*HPE+j] (i, j < HPE) = the same halves of the P x P matrices
//                  t = 0: D, 1: D^T, 2: MP, 3: KP, 4: MP + KP, 5: D^T MP D,
//                  6: D^T (MP + KP) D
//   D[i*P+k]     = GLL differentiation matrix on the (W+1)-point grid (eq. 5.47)
//   S[k*P+c]     = preconditioner eigenvectors (node k, mode c), eq. (5.15)-(5.17)
//   MP, KP       = B0^T diag(w) B0 and B0^T K B0 (P x P face-norm matrices)
//   WQ[q]        = (2W+1)-point GLL weights; MU[c] = eigenvalues of eq. (5.15)
struct Tables {
  real B[3][QP];
  real FE[3][P * HPE];
  real FO[3][P * HPE];
  real PF[7][2][HPE * HPE];
  real D[P2];
  real S[P2];
  real MP[P2];
  real KP[P2];
  real WQ[Q];
  real MU[P];
  // pairs of folded entries for the packed FP32 contractions (two matrices
  // applied at once, see fwd_pm2): XE[0][i] = (FE[0][i], FE[0][i]),
  // XE[1][i] = (FE[0][i], FE[2][i]); XO likewise from FO
  float2 XE[2][P * HPE];
  float2 XO[2][P * HPE];
};
__constant__ Tables c_tab;

using hpse::COEF_LAPLACE;
using hpse::COEF_SCALAR;
using hpse::COEF_EDGE;
using hpse::COEF_VERTEX;
using hpse::COEF_VERTEX_EDGE;
// variable-coefficient fields (first derivatives, per-point weights)
__host__ __device__ constexpr bool var_coef(int c) {
  return c == hpse::COEF_SCALAR || c == hpse::COEF_VERTEX || c == hpse::COEF_VERTEX_EDGE;
}
// the first derivative along y is a field (its coefficient is zero in the
// vertex and vertex-edge operators, which skip it)
__host__ __device__ constexpr bool y_first(int c) { return c == hpse::COEF_SCALAR; }
// the mixed derivative u_xz is a field (vertex-edge operator)
__host__ __device__ constexpr bool mixed_xz(int c) { return c == hpse::COEF_VERTEX_EDGE; }
// neighbourhood elements: face-norm weights and corner sets
__host__ __device__ constexpr bool nbhd_coef(int c) {
  return c == hpse::COEF_EDGE || c == hpse::COEF_VERTEX || c == hpse::COEF_VERTEX_EDGE;
}
// corner sets through face 0 (a polynomial along z) / face 4 (a constant)
__host__ __device__ constexpr bool corner_f0(int c) { return c == hpse::COEF_EDGE || c == hpse::COEF_VERTEX_EDGE; }
__host__ __device__ constexpr bool corner_f4(int c) { return c == hpse::COEF_VERTEX || c == hpse::COEF_VERTEX_EDGE; }
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

// vector load of the 4 pointwise coefficients (m, d_x, d_y, d_z) of a point
__device__ __forceinline__ void load_coef4(const real *p, real &m, real &dx, real &dy, real &dz) {
#if defined(HPSE_DOUBLE)
  const double2 a = *reinterpret_cast<const double2 *>(p);
  const double2 b = *reinterpret_cast<const double2 *>(p + 2);
  m = a.x;
  dx = a.y;
  dy = b.x;
  dz = b.y;
#else
  const float4 a = *reinterpret_cast<const float4 *>(p);
  m = a.x;
  dx = a.y;
  dy = a.z;
  dz = a.w;
#endif
}

// ---------------------------------------------------------------------------
// Line stages of the sum factorisation, with the even-odd decomposition of
// the 1-D matrices (Solomonoff, "A fast algorithm for spectral
// differentiation", J. Comput. Phys. 98, 1992): on the symmetric GLL grids
// B0 and B2 are even and B1 is odd under the reflection of both grids,
// B_m[Q-1-q][P-1-j] = +-B_m[q][j].  Folding an input line into the sums and
// differences of its mirrored entries and producing each output pair
// (q, Q-1-q) at once halves the multiply-adds of every contraction:
//   forward (P -> Q), output pair q <= W (q = W is the middle point):
//     even M: PLUS = FE_M[q] . e, MINUS = FO_M[q] . o
//     odd M:  PLUS = FO_M[q] . o, MINUS = FE_M[q] . e
//     y[q] = PLUS + MINUS, y[Q-1-q] = PLUS - MINUS
//   transpose (Q -> P), output pair k < HPE, folded input (ve, vo, vm):
//     even M: PLUS += FE_M[.][k] . ve + FE_M[W][k] vm, MINUS += FO_M[.][k] . vo
//     odd M:  PLUS += FE_M[.][k] . vo, MINUS += FO_M[.][k] . ve + FO_M[W][k] vm
//     r[k] = PLUS + MINUS, r[P-1-k] = PLUS - MINUS
// Contributions of several matrices to one output add into one PLUS/MINUS
// pair, whatever their parities.
//
// A stage has L lines of one element; the output pairs of a line are split
// into NC chunks of compile-time range and item = chunk * PAD32(L) + line, so
// the chunk index is warp-uniform, all warps of the CTA get work, and every
// FMA keeps its constant-bank operand.  Padding lanes (line >= L) read a
// clamped valid line and store nothing.
// ---------------------------------------------------------------------------
template <int L>
struct Lines {
  static constexpr int PADL = PAD32(L);
  static constexpr int NC_RAW = NT / PADL;
#if defined(HPSE_LINES_NC)
  static constexpr int NC_MAX = HPSE_LINES_NC;  // set at build time (launch-shape experiments)
#else
  static constexpr int NC_MAX = 2;
#endif
  static constexpr int NC = NC_RAW < 1 ? 1 : (NC_RAW > NC_MAX ? NC_MAX : NC_RAW);
};
template <int CI, int NC, int N>
struct Range {
  static constexpr int B = CI * N / NC;
  static constexpr int E = (CI + 1) * N / NC;
};

// u[P] -> e (mirrored sums, then the middle node), o (mirrored differences, middle 0)
__device__ __forceinline__ void fold_p(const real *u, real *e, real *o) {
#pragma unroll
  for (int j = 0; j < HP; ++j) {
    e[j] = u[j] + u[P - 1 - j];
    o[j] = u[j] - u[P - 1 - j];
  }
  if (P & 1) {
    e[HP] = u[HP];
    o[HP] = (real)0;
  }
}

// v[Q] -> ve[HQ], vo[HQ] (mirrored sums / differences), vm (the middle point)
__device__ __forceinline__ void fold_q(const real *v, real *ve, real *vo, real &vm) {
#pragma unroll
  for (int q = 0; q < HQ; ++q) {
    ve[q] = v[q] + v[Q - 1 - q];
    vo[q] = v[q] - v[Q - 1 - q];
  }
  vm = v[HQ];
}

// forward, output pair q: PLUS / MINUS of matrix M applied to the folded line
template <int M>
__device__ __forceinline__ void fwd_pm(const real *e, const real *o, int q, real &pl, real &mi) {
#pragma unroll
  for (int j = 0; j < HPE; ++j) {
    if (!odd_mat(M)) pl += c_tab.FE[M][q * HPE + j] * e[j];
    else if (q < HQ) mi += c_tab.FE[M][q * HPE + j] * e[j];
  }
#pragma unroll
  for (int j = 0; j < HP; ++j) {
    if (odd_mat(M)) pl += c_tab.FO[M][q * HPE + j] * o[j];
    else if (q < HQ) mi += c_tab.FO[M][q * HPE + j] * o[j];
  }
}

// transpose, one folded input pair q < HQ (ve, vo) into the PLUS / MINUS of
// every output pair k
template <int M>
__device__ __forceinline__ void rev_pair(real ve, real vo, int q, real *pl, real *mi) {
#pragma unroll
  for (int k = 0; k < HPE; ++k) {
    pl[k] += c_tab.FE[M][q * HPE + k] * (odd_mat(M) ? vo : ve);
    if (k < HP) mi[k] += c_tab.FO[M][q * HPE + k] * (odd_mat(M) ? ve : vo);
  }
}
// transpose, the middle input point vm
template <int M>
__device__ __forceinline__ void rev_mid(real vm, real *pl, real *mi) {
#pragma unroll
  for (int k = 0; k < HPE; ++k) {
    if (!odd_mat(M)) pl[k] += c_tab.FE[M][HQ * HPE + k] * vm;
    else if (k < HP) mi[k] += c_tab.FO[M][HQ * HPE + k] * vm;
  }
}
// transpose of a whole folded line into output pair k
template <int M>
__device__ __forceinline__ void rev_line(const real *ve, const real *vo, real vm, int k, real &pl, real &mi) {
#pragma unroll
  for (int q = 0; q < HQ; ++q) {
    pl += c_tab.FE[M][q * HPE + k] * (odd_mat(M) ? vo[q] : ve[q]);
    if (k < HP) mi += c_tab.FO[M][q * HPE + k] * (odd_mat(M) ? ve[q] : vo[q]);
  }
  if (!odd_mat(M)) pl += c_tab.FE[M][HQ * HPE + k] * vm;
  else if (k < HP) mi += c_tab.FO[M][HQ * HPE + k] * vm;
}

// store the pair (q, Q-1-q) of a forward output from PLUS / MINUS
__device__ __forceinline__ void put_q(real *dst, int stride, int q, real pl, real mi) {
  dst[q * stride] = pl + mi;
  if (q < HQ) dst[(Q - 1 - q) * stride] = pl - mi;
}
// store the pair (k, P-1-k) of a transposed output from PLUS / MINUS
__device__ __forceinline__ void put_p(real *dst, int stride, int k, real pl, real mi) {
  dst[k * stride] = pl + mi;
  if (k < HP) dst[(P - 1 - k) * stride] = pl - mi;
}

// ---------------------------------------------------------------------------
// Packed FP32 contractions.  Blackwell issues two FP32 FMAs in one
// instruction (__ffma2_rn: each half is an fmaf, rounded once), so two folded
// contractions with the same (q, j) pattern run at half the issue cost of the
// scalar form.  A pair applies two EVEN matrices, each half to its own folded
// line: half .x takes B0, half .y takes B0 (pair K = 0) or B2 (K = 1), with
// the entries from c_tab.XE / XO.  Each half accumulates in the same order as
// the scalar helpers above, so a pair gives bit for bit the two scalar
// results.  Used by the FP32 instances of the Laplacian and -div(a grad u);
// the odd matrix B1 stays scalar, reading one half of a packed line.
// ---------------------------------------------------------------------------
// k_apply's FP32 stages of these operators take the packed forms; stage bits
// (x, y, z forward, z, y, x transpose = 1, 2, 4, 8, 16, 32) select which
#if defined(HPSE_PACK_STAGES)
constexpr int PACK_STAGES = HPSE_PACK_STAGES;  // set at build time (register-pressure experiments)
#else
constexpr int PACK_STAGES = 63;
#endif
__host__ __device__ constexpr bool packed_coef(int c, int stage) {
#if defined(HPSE_DOUBLE)
  return false && c && stage;
#else
  return (c == hpse::COEF_LAPLACE || c == hpse::COEF_SCALAR) && (PACK_STAGES & stage);
#endif
}

// -div(a grad u) in the transpose mode (rho read from global memory) keeps
// the scalar stages and rho in registers: the packed form measured slower there
__host__ __device__ constexpr bool packed_mode(int c, int mode) {
  return mode != hpse::MODE_TRANSPOSE || c != hpse::COEF_SCALAR;
}

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b, exactly rounded (a + (-1) b in one FMA)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 zero2() { return make_float2(0.f, 0.f); }
template <int H>
__device__ __forceinline__ float half2_of(float2 v) { return H ? v.y : v.x; }

// u[P] (pairs) -> e, o as fold_p, both halves at once
__device__ __forceinline__ void fold_p2(const float2 *u, float2 *e, float2 *o) {
#pragma unroll
  for (int j = 0; j < HP; ++j) {
    e[j] = add2(u[j], u[P - 1 - j]);
    o[j] = sub2(u[j], u[P - 1 - j]);
  }
  if (P & 1) {
    e[HP] = u[HP];
    o[HP] = zero2();
  }
}
// v[Q] (pairs) -> ve, vo, vm as fold_q
__device__ __forceinline__ void fold_q2(const float2 *v, float2 *ve, float2 *vo, float2 &vm) {
#pragma unroll
  for (int q = 0; q < HQ; ++q) {
    ve[q] = add2(v[q], v[Q - 1 - q]);
    vo[q] = sub2(v[q], v[Q - 1 - q]);
  }
  vm = v[HQ];
}

// forward pair, output pair q: as fwd_pm for two even matrices
template <int K>
__device__ __forceinline__ void fwd_pm2(const float2 *e, const float2 *o, int q, float2 &pl, float2 &mi) {
#pragma unroll
  for (int j = 0; j < HPE; ++j) pl = __ffma2_rn(c_tab.XE[K][q * HPE + j], e[j], pl);
  if (q < HQ) {
#pragma unroll
    for (int j = 0; j < HP; ++j) mi = __ffma2_rn(c_tab.XO[K][q * HPE + j], o[j], mi);
  }
}
// fwd_pm of matrix M on half H of a packed line
template <int M, int H>
__device__ __forceinline__ void fwd_pm_h(const float2 *e, const float2 *o, int q, real &pl, real &mi) {
#pragma unroll
  for (int j = 0; j < HPE; ++j) {
    if (!odd_mat(M)) pl += c_tab.FE[M][q * HPE + j] * half2_of<H>(e[j]);
    else if (q < HQ) mi += c_tab.FE[M][q * HPE + j] * half2_of<H>(e[j]);
  }
#pragma unroll
  for (int j = 0; j < HP; ++j) {
    if (odd_mat(M)) pl += c_tab.FO[M][q * HPE + j] * half2_of<H>(o[j]);
    else if (q < HQ) mi += c_tab.FO[M][q * HPE + j] * half2_of<H>(o[j]);
  }
}
// transpose pair: as rev_pair / rev_mid for two even matrices
template <int K>
__device__ __forceinline__ void rev_pair2(float2 ve, float2 vo, int q, float2 *pl, float2 *mi) {
#pragma unroll
  for (int k = 0; k < HPE; ++k) {
    pl[k] = __ffma2_rn(c_tab.XE[K][q * HPE + k], ve, pl[k]);
    if (k < HP) mi[k] = __ffma2_rn(c_tab.XO[K][q * HPE + k], vo, mi[k]);
  }
}
template <int K>
__device__ __forceinline__ void rev_mid2(float2 vm, float2 *pl) {
#pragma unroll
  for (int k = 0; k < HPE; ++k) pl[k] = __ffma2_rn(c_tab.XE[K][HQ * HPE + k], vm, pl[k]);
}
// transpose of a whole folded pair of lines into output pair k: as rev_line
template <int K>
__device__ __forceinline__ void rev_line2(const float2 *ve, const float2 *vo, float2 vm, int k, float2 &pl,
                                          float2 &mi) {
#pragma unroll
  for (int q = 0; q < HQ; ++q) {
    pl = __ffma2_rn(c_tab.XE[K][q * HPE + k], ve[q], pl);
    if (k < HP) mi = __ffma2_rn(c_tab.XO[K][q * HPE + k], vo[q], mi);
  }
  pl = __ffma2_rn(c_tab.XE[K][HQ * HPE + k], vm, pl);
}
// rev_line of matrix M on half H of a packed folded line
template <int M, int H>
__device__ __forceinline__ void rev_line_h(const float2 *ve, const float2 *vo, float2 vm, int k, real &pl,
                                           real &mi) {
#pragma unroll
  for (int q = 0; q < HQ; ++q) {
    pl += c_tab.FE[M][q * HPE + k] * half2_of<H>(odd_mat(M) ? vo[q] : ve[q]);
    if (k < HP) mi += c_tab.FO[M][q * HPE + k] * half2_of<H>(odd_mat(M) ? ve[q] : vo[q]);
  }
  if (!odd_mat(M)) pl += c_tab.FE[M][HQ * HPE + k] * half2_of<H>(vm);
  else if (k < HP) mi += c_tab.FO[M][HQ * HPE + k] * half2_of<H>(vm);
}
// store the pairs (q, Q-1-q) of two forward outputs: half .x to dx, .y to dy
__device__ __forceinline__ void put_q2(real *dx, real *dy, int stride, int q, float2 pl, float2 mi) {
  const float2 a = add2(pl, mi);
  dx[q * stride] = a.x;
  dy[q * stride] = a.y;
  if (q < HQ) {
    const float2 b = sub2(pl, mi);
    dx[(Q - 1 - q) * stride] = b.x;
    dy[(Q - 1 - q) * stride] = b.y;
  }
}
// store the pairs (k, P-1-k) of two transposed outputs
__device__ __forceinline__ void put_p2(real *dx, real *dy, int stride, int k, float2 pl, float2 mi) {
  const float2 a = add2(pl, mi);
  dx[k * stride] = a.x;
  dy[k * stride] = a.y;
  if (k < HP) {
    const float2 b = sub2(pl, mi);
    dx[(P - 1 - k) * stride] = b.x;
    dy[(P - 1 - k) * stride] = b.y;
  }
}

// x-stage: X0 = B0 u, X2 = B2 u (X1 = B1 u) along x for line l = (j, k)
template <int COEF, int CI, int NC>
__device__ __forceinline__ void x_fwd_chunk(const real *e, const real *o, real *X0, real *X1, real *X2, int l,
                                            bool ok) {
  typedef Range<CI, NC, HQ + 1> R;
#pragma unroll
  for (int q = R::B; q < R::E; ++q) {
    real p0 = 0, m0 = 0, p2 = 0, m2 = 0, p1 = 0, m1 = 0;
    fwd_pm<0>(e, o, q, p0, m0);
    fwd_pm<2>(e, o, q, p2, m2);
    if (var_coef(COEF)) fwd_pm<1>(e, o, q, p1, m1);
    if (ok) {
      put_q(X0 + l * Q, 1, q, p0, m0);
      put_q(X2 + l * Q, 1, q, p2, m2);
      if (var_coef(COEF)) put_q(X1 + l * Q, 1, q, p1, m1);
    }
    __syncwarp();  // scheduling fence (register pressure); reached by all 32 lanes
  }
}

// y-stage: T00 = B0 X0, TL = sx2 B0 X2 + sy2 B2 X0 (T10 = B0 X1, T01 = B1 X0) along y
template <int COEF, int CI, int NC>
__device__ __forceinline__ void y_fwd_chunk(const real *e0, const real *o0, const real *e1, const real *o1,
                                            const real *e2, const real *o2, real *T00, real *TL, real *T10,
                                            real *T01, int qa, int k, bool ok, real sx2, real sy2) {
  typedef Range<CI, NC, HQ + 1> R;
#pragma unroll
  for (int qb = R::B; qb < R::E; ++qb) {
    real p00 = 0, m00 = 0, pl0 = 0, ml0 = 0, pl2 = 0, ml2 = 0, p10 = 0, m10 = 0, p01 = 0, m01 = 0;
    fwd_pm<0>(e0, o0, qb, p00, m00);
    fwd_pm<2>(e0, o0, qb, pl0, ml0);
    fwd_pm<0>(e2, o2, qb, pl2, ml2);
    if (var_coef(COEF)) fwd_pm<0>(e1, o1, qb, p10, m10);
    if (y_first(COEF)) fwd_pm<1>(e0, o0, qb, p01, m01);
    const int o = k * Q2 + qa;  // + qb * Q
    if (ok) {
      put_q(T00 + o, Q, qb, p00, m00);
      put_q(TL + o, Q, qb, sx2 * pl2 + sy2 * pl0, sx2 * ml2 + sy2 * ml0);
      if (var_coef(COEF)) put_q(T10 + o, Q, qb, p10, m10);
      if (y_first(COEF)) put_q(T01 + o, Q, qb, p01, m01);
    }
    __syncwarp();  // scheduling fence (register pressure); reached by all 32 lanes
  }
}

// y-stage transpose: X0 = B0^T RZ + sy2 B2^T R0 + B1^T RY, X2 = sx2 B0^T R0 (X1 = B0^T RX)
template <int COEF, int CI, int NC>
__device__ __forceinline__ void y_rev_chunk(const real *RZ, const real *R0, const real *RX, const real *RY,
                                            real *X0, real *X1, real *X2, int qa, int k, bool ok, real sx2,
                                            real sy2) {
  typedef Range<CI, NC, HPE> R;
  const int o = k * Q2 + qa;  // + qb * Q
  {
    real ze[HQ], zo[HQ], zm, re[HQ], ro[HQ], rm, ye[HQ], yo[HQ], ym;
    {
      real v[Q];
#pragma unroll
      for (int qb = 0; qb < Q; ++qb) v[qb] = RZ[o + qb * Q];
      fold_q(v, ze, zo, zm);
#pragma unroll
      for (int qb = 0; qb < Q; ++qb) v[qb] = R0[o + qb * Q];
      fold_q(v, re, ro, rm);
      if (y_first(COEF)) {
#pragma unroll
        for (int qb = 0; qb < Q; ++qb) v[qb] = RY[o + qb * Q];
        fold_q(v, ye, yo, ym);
      }
    }
#pragma unroll
    for (int j = R::B; j < R::E; ++j) {
      real pz = 0, mz = 0, p2 = 0, m2 = 0, py = 0, my = 0, p0 = 0, m0 = 0;
      rev_line<0>(ze, zo, zm, j, pz, mz);
      rev_line<2>(re, ro, rm, j, p2, m2);
      rev_line<0>(re, ro, rm, j, p0, m0);
      if (y_first(COEF)) rev_line<1>(ye, yo, ym, j, py, my);
      if (ok) {
        const int ox = k * P * Q + qa;  // + j * Q
        put_p(X0 + ox, Q, j, pz + sy2 * p2 + py, mz + sy2 * m2 + my);
        put_p(X2 + ox, Q, j, sx2 * p0, sx2 * m0);
      }
    }
  }
  if (var_coef(COEF)) {
    real xe[HQ], xo[HQ], xm;
    {
      real v[Q];
#pragma unroll
      for (int qb = 0; qb < Q; ++qb) v[qb] = RX[o + qb * Q];
      fold_q(v, xe, xo, xm);
    }
#pragma unroll
    for (int j = R::B; j < R::E; ++j) {
      real p1 = 0, m1 = 0;
      rev_line<0>(xe, xo, xm, j, p1, m1);
      if (ok) put_p(X1 + k * P * Q + qa, Q, j, p1, m1);
    }
  }
}

// x-stage transpose: y = B0^T X0 + B2^T X2 (+ B1^T X1) along x for line l
template <int COEF, int CI, int NC>
__device__ __forceinline__ void x_rev_chunk(const real *X0, const real *X1, const real *X2, real *sy, int l,
                                            bool ok) {
  typedef Range<CI, NC, HPE> R;
  real e0[HQ], o0[HQ], m0v, e2[HQ], o2[HQ], m2v, e1[HQ], o1[HQ], m1v;
  {
    real v[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) v[q] = X0[l * Q + q];
    fold_q(v, e0, o0, m0v);
#pragma unroll
    for (int q = 0; q < Q; ++q) v[q] = X2[l * Q + q];
    fold_q(v, e2, o2, m2v);
    if (var_coef(COEF)) {
#pragma unroll
      for (int q = 0; q < Q; ++q) v[q] = X1[l * Q + q];
      fold_q(v, e1, o1, m1v);
    }
  }
#pragma unroll
  for (int i = R::B; i < R::E; ++i) {
    real pl = 0, mi = 0;
    rev_line<0>(e0, o0, m0v, i, pl, mi);
    rev_line<2>(e2, o2, m2v, i, pl, mi);
    if (var_coef(COEF)) rev_line<1>(e1, o1, m1v, i, pl, mi);
    if (ok) put_p(sy + l * P, 1, i, pl, mi);
  }
}

// ---- packed stages (FP32 Laplacian and -div(a grad u), see packed_coef) ----
// x-stage: e, o hold the folded line u in both halves: (B0 u, B2 u) packed,
// B1 u (variable coefficient) scalar on the .x half
template <int COEF, int CI, int NC>
__device__ __forceinline__ void x_fwd_chunk2(const float2 *e, const float2 *o, real *X0, real *X1, real *X2, int l,
                                             bool ok) {
  typedef Range<CI, NC, HQ + 1> R;
#pragma unroll
  for (int q = R::B; q < R::E; ++q) {
    float2 pl = zero2(), mi = zero2();
    real p1 = 0, m1 = 0;
    fwd_pm2<1>(e, o, q, pl, mi);
    if (var_coef(COEF)) fwd_pm_h<1, 0>(e, o, q, p1, m1);
    if (ok) {
      put_q2(X0 + l * Q, X2 + l * Q, 1, q, pl, mi);
      if (var_coef(COEF)) put_q(X1 + l * Q, 1, q, p1, m1);
    }
    __syncwarp();  // scheduling fence (register pressure); reached by all 32 lanes
  }
}

// y-stage.  -div(a grad u): d = X0 in both halves -> (B0 X0, B2 X0),
// w = (X2, X1) -> (B0 X2, B0 X1), B1 X0 scalar on d.x.  Laplacian:
// w = (X0, X2) -> (B0 X0, B0 X2), B2 X0 scalar on w.x (d unused).
template <int COEF, int CI, int NC>
__device__ __forceinline__ void y_fwd_chunk2(const float2 *de, const float2 *dd, const float2 *we, const float2 *wo,
                                             real *T00, real *TL, real *T10, real *T01, int qa, int k, bool ok,
                                             real sx2, real sy2) {
  typedef Range<CI, NC, HQ + 1> R;
#pragma unroll
  for (int qb = R::B; qb < R::E; ++qb) {
    const int o = k * Q2 + qa;  // + qb * Q
    if (COEF == COEF_SCALAR) {
      float2 ap = zero2(), am = zero2(), bp = zero2(), bm = zero2();
      real p01 = 0, m01 = 0;
      fwd_pm2<1>(de, dd, qb, ap, am);
      fwd_pm2<0>(we, wo, qb, bp, bm);
      fwd_pm_h<1, 0>(de, dd, qb, p01, m01);
      if (ok) {
        put_q(T00 + o, Q, qb, ap.x, am.x);
        put_q(TL + o, Q, qb, sx2 * bp.x + sy2 * ap.y, sx2 * bm.x + sy2 * am.y);
        put_q(T10 + o, Q, qb, bp.y, bm.y);
        put_q(T01 + o, Q, qb, p01, m01);
      }
    } else {
      float2 bp = zero2(), bm = zero2();
      real pl0 = 0, ml0 = 0;
      fwd_pm2<0>(we, wo, qb, bp, bm);
      fwd_pm_h<2, 0>(we, wo, qb, pl0, ml0);
      if (ok) {
        put_q(T00 + o, Q, qb, bp.x, bm.x);
        put_q(TL + o, Q, qb, sx2 * bp.y + sy2 * pl0, sx2 * bm.y + sy2 * ml0);
      }
    }
    __syncwarp();  // scheduling fence (register pressure); reached by all 32 lanes
  }
}

// y-stage transpose: (RZ, R0) packed -> (B0^T RZ, B0^T R0), B2^T R0 scalar on
// the .y half, B1^T RY and B0^T RX (variable coefficient) scalar
template <int COEF, int CI, int NC>
__device__ __forceinline__ void y_rev_chunk2(const real *RZ, const real *R0, const real *RX, const real *RY,
                                             real *X0, real *X1, real *X2, int qa, int k, bool ok, real sx2,
                                             real sy2) {
  typedef Range<CI, NC, HPE> R;
  const int o = k * Q2 + qa;  // + qb * Q
  {
    float2 ze[HQ], zo[HQ], zm;
    real ye[HQ], yo[HQ], ym;
    {
      float2 v[Q];
#pragma unroll
      for (int qb = 0; qb < Q; ++qb) v[qb] = make_float2(RZ[o + qb * Q], R0[o + qb * Q]);
      fold_q2(v, ze, zo, zm);
    }
    if (y_first(COEF)) {
      real v[Q];
#pragma unroll
      for (int qb = 0; qb < Q; ++qb) v[qb] = RY[o + qb * Q];
      fold_q(v, ye, yo, ym);
    }
#pragma unroll
    for (int j = R::B; j < R::E; ++j) {
      float2 pl = zero2(), mi = zero2();
      real p2 = 0, m2 = 0, py = 0, my = 0;
      rev_line2<0>(ze, zo, zm, j, pl, mi);
      rev_line_h<2, 1>(ze, zo, zm, j, p2, m2);
      if (y_first(COEF)) rev_line<1>(ye, yo, ym, j, py, my);
      if (ok) {
        const int ox = k * P * Q + qa;  // + j * Q
        put_p(X0 + ox, Q, j, pl.x + sy2 * p2 + py, mi.x + sy2 * m2 + my);
        put_p(X2 + ox, Q, j, sx2 * pl.y, sx2 * mi.y);
      }
    }
  }
  if (var_coef(COEF)) {
    real xe[HQ], xo[HQ], xm;
    {
      real v[Q];
#pragma unroll
      for (int qb = 0; qb < Q; ++qb) v[qb] = RX[o + qb * Q];
      fold_q(v, xe, xo, xm);
    }
#pragma unroll
    for (int j = R::B; j < R::E; ++j) {
      real p1 = 0, m1 = 0;
      rev_line<0>(xe, xo, xm, j, p1, m1);
      if (ok) put_p(X1 + k * P * Q + qa, Q, j, p1, m1);
    }
  }
}

// x-stage transpose: (X0, X2) packed -> (B0^T X0, B2^T X2), B1^T X1 scalar;
// y = the sum of the three
template <int COEF, int CI, int NC>
__device__ __forceinline__ void x_rev_chunk2(const real *X0, const real *X1, const real *X2, real *sy, int l,
                                             bool ok) {
  typedef Range<CI, NC, HPE> R;
  float2 e[HQ], o[HQ], m;
  real e1[HQ], o1[HQ], m1v;
  {
    float2 v[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) v[q] = make_float2(X0[l * Q + q], X2[l * Q + q]);
    fold_q2(v, e, o, m);
  }
  if (var_coef(COEF)) {
    real v[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) v[q] = X1[l * Q + q];
    fold_q(v, e1, o1, m1v);
  }
#pragma unroll
  for (int i = R::B; i < R::E; ++i) {
    float2 pl = zero2(), mi = zero2();
    real p1 = 0, q1 = 0;
    rev_line2<1>(e, o, m, i, pl, mi);
    if (var_coef(COEF)) rev_line<1>(e1, o1, m1v, i, p1, q1);
    if (ok) put_p(sy + l * P, 1, i, pl.x + pl.y + p1, mi.x + mi.y + q1);
  }
}

// ---------------------------------------------------------------------------
// Face phase: y_e += contributions of the six faces of element e (eq. 4.2),
// all six faces processed at once, then gathered node by node (no two
// threads ever add into the same node: deterministic, no atomics).
//
// Per face f (axis a, side s, tangential axes t1 < t2, nodal face grid P x P,
// p1 along t1, p2 along t2):
//   own traces  F = u|face, N = du/dlambda_a|face, tangential derivatives D F
//   interior:   J0 = [u], J1 = [u_{x_t1}], J2 = [u_{x_t2}], J3 = [u_{x_a}]
//               g0 = (MP x MP) J0, gk = (MP x MP + MP x KP + KP x MP) Jk
//   Dirichlet:  J0 = u, J1 = du/dlambda_t1, J2 = du/dlambda_t2 (eq. 2.18)
// MP = B0^T W B0 and KP = B0^T K B0 are the Section 5.3 face forms on the
// (2W+1)-point grid pulled back to the nodal grid (exact algebra).
//
// Every 1-D product runs as a line job: one thread takes one line of P face
// values, folds it (even-odd) and applies D, D^T (odd), MP or KP (even) with
// compile-time constant-bank operands.  The normal derivative at the face
// takes the first row of D only: D[P-1][P-1-k] = -D[0][k] on the symmetric
// grid, so both sides walk their normal line from the face inward.
// Scratch per face: 14 arrays of P x P (the G_k of the norm products reuse
// the J slots, the transposed tangential derivatives the A slots).
// ---------------------------------------------------------------------------
constexpr int FACE_ARR = 15;

template <int MODE>
__device__ __forceinline__ real nb_value(const ApplyArgs &A, int64_t idx, real bt) {
  if (MODE == MODE_PCG) return A.z[idx] + bt * A.u[idx];
  return A.u[idx];
}

// y[0..P-1] = X v for one folded line (e, o) of the P x P matrix t:
// 0 = D, 1 = D^T (odd), 2 = MP, 3 = KP, 4 = MP + KP, 5 = D^T MP D,
// 6 = D^T (MP + KP) D (even)
template <int T>
__device__ __forceinline__ void pp_line(const real *e, const real *o, real *y) {
#pragma unroll
  for (int i = 0; i < HPE; ++i) {
    real pl = 0, mi = 0;
#pragma unroll
    for (int j = 0; j < HPE; ++j) {
      if (!odd_pp(T)) {
        pl += c_tab.PF[T][0][i * HPE + j] * e[j];
        if (i < HP && j < HP) mi += c_tab.PF[T][1][i * HPE + j] * o[j];
      } else {
        if (j < HP) pl += c_tab.PF[T][1][i * HPE + j] * o[j];
        if (i < HP) mi += c_tab.PF[T][0][i * HPE + j] * e[j];
      }
    }
    y[i] = pl + mi;
    if (i < HP) y[P - 1 - i] = pl - mi;
  }
}

// load a line of P values with stride st and fold it
__device__ __forceinline__ void load_fold(const real *p, int st, real *e, real *o) {
  real v[P];
#pragma unroll
  for (int m = 0; m < P; ++m) v[m] = p[m * st];
  fold_p(v, e, o);
}

// Per-face data of the face phase, gathered once per CTA by six threads at
// the start of the kernel, so that the face phase's line jobs read shared
// memory instead of chains of dependent loads from the mesh arrays:
//   nb, bc  the neighbour (-1 boundary, < -1 corner set) and the face code
//   nbase   the neighbour's (corner set's) block in the vectors, rhs included
//   bt      PCG mode: beta of the neighbour's problem (the search direction
//           there is z + beta p)
//   s1      the neighbour's scales s_a (the element's own on boundary faces
//           and towards corner sets, which share the scales of their layer)
//   fsc     the gather's scales: the normal term (s_a on interior faces,
//           +-s_a on Neumann / Robin faces, 0 on Dirichlet faces and faces
//           left to k_face_mixed) and the Robin gamma
struct FaceMeta {
  int64_t nbase[6];
  real s1[6][3];
  real bt[6];
  real fsc[12];
  int nb[6];
  int bc[6];
};
// reals reserved for it after the D copy (8-byte alignment included)
constexpr int FACE_META_REALS = (int)((sizeof(FaceMeta) + 8 + sizeof(real) - 1) / sizeof(real));
__device__ __forceinline__ FaceMeta *face_meta(real *stab) {
  const uintptr_t p = reinterpret_cast<uintptr_t>(stab + P2);
  return reinterpret_cast<FaceMeta *>((p + 7) & ~(uintptr_t)7);
}
template <int COEF, int MODE>
__device__ __forceinline__ void face_meta_fill(const ApplyArgs &A, int e, int r, const real *geo_e, FaceMeta *M,
                                               int f) {
  const int nb = A.nbr[(int64_t)e * 6 + f];
  const int bc = A.fbc ? A.fbc[(int64_t)e * 6 + f] : 0;
  M->nb[f] = nb;
  M->bc[f] = bc;
  M->fsc[f] = bc == 3 ? (real)0
                      : (nb != -1 ? geo_e[f >> 1] : (bc ? ((f & 1) ? geo_e[f >> 1] : -geo_e[f >> 1]) : (real)0));
  M->fsc[6 + f] = bc == 2 ? A.fgam[(int64_t)e * 6 + f] : (real)0;
  int64_t nbase = 0;
  real bt = 0;
  const real *gn = geo_e;
  if (nbhd_coef(COEF) && nb < -1) {
    nbase = (int64_t)r * A.ndof + A.dof_off[A.n_elem + (-2 - nb)];
    if (MODE == MODE_PCG) bt = (real)A.beta[A.prob[e] * A.n_rhs + r];
  } else if (nb >= 0) {
    nbase = (int64_t)r * A.ndof + A.dof_off[nb];
    if (MODE == MODE_PCG) bt = (real)A.beta[A.prob[nb] * A.n_rhs + r];
    gn = A.geo + (int64_t)nb * 4;
  }
  M->nbase[f] = nbase;
  M->bt[f] = bt;
#pragma unroll
  for (int a = 0; a < 3; ++a) M->s1[f][a] = gn[a];
}

template <int COEF, int MODE>
__device__ void face_phase(const ApplyArgs &A, int e, int r, const real *su, real *sy, real *scr, const real *Ds,
                           const real *geo_e, const FaceMeta *fm) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const real *fsc = fm->fsc;
  // slot s of face f: scr + (f * FACE_ARR + s) * P2; G_k reuse J_k, U1 / U2 reuse A1 / A2
#define FSLOT(f, s) (scr + ((f)*FACE_ARR + (s)) * P2)
  enum { sF = 0, sFn, sJ0, sJ1, sJ2, sJ3, sA0, sA1, sA2, sA3, sB0, sB1, sB2, sB3 };
  // per face: the scale of the normal term in the gather (s_a on interior
  // faces, +-s_a on Neumann / Robin faces, 0 on Dirichlet faces) and of the
  // face-layer term of a Robin face (gamma)
  // (an interior face between unequal degrees, code 3, is left to k_face_mixed:
  // zero scales and zero slots here)
  // 1: traces at every face point: F, J0 = [u] (u), J3 = [u_{x_a}] (0), the neighbour's trace Fn
  for (int t = tid; t < 6 * P2; t += nt) {
    const int f = t / P2, sp = t - f * P2;
    const int p1 = sp % P, p2 = sp / P;
    const int a = f >> 1, side = f & 1;
    const int stride = a == 0 ? 1 : (a == 1 ? P : P2);
    const int b0 = a == 0 ? (p2 * P + p1) * P : (a == 1 ? p2 * P2 + p1 : p2 * P + p1);
    // own normal line from the face inward
    const int o0 = side ? b0 + (P - 1) * stride : b0, os = side ? -stride : stride;
    const real Fv = su[o0];
    real Nv = 0;
#pragma unroll
    for (int k = 0; k < P; ++k) Nv += c_tab.D[k] * su[o0 + k * os];
    if (side) Nv = -Nv;
    const int nb = fm->nb[f];
    const int bc = fm->bc[f];
    real Fn = 0, Nn = 0;
    if (bc == 3 || (nb != -1 && A.self_only)) {
      // diagonal block: the neighbour's trace is zero
    } else if (nbhd_coef(COEF) && nb < -1) {
      // corner set: through face 0 a polynomial along z (the p2 direction of
      // this face), constant in the other two variables (edge: x3; vertex-edge:
      // zeta); through face 4 one constant (vertex, vertex-edge)
      Fn = nb_value<MODE>(A, fm->nbase[f] + (corner_f0(COEF) && f == 0 ? p2 : 0), fm->bt[f]);
    } else if (nb >= 0) {
      const int64_t nbase = fm->nbase[f];
      const real bt = fm->bt[f];
      // the neighbour's face is its opposite end: its normal line from that face inward
      const int q0 = side ? b0 : b0 + (P - 1) * stride, qs = side ? stride : -stride;
      Fn = nb_value<MODE>(A, nbase + q0, bt);
#pragma unroll
      for (int k = 0; k < P; ++k) Nn += c_tab.D[k] * nb_value<MODE>(A, nbase + q0 + k * qs, bt);
      if (!side) Nn = -Nn;
    }
    FSLOT(f, sF)[sp] = Fv;
    if (bc == 3) {
      FSLOT(f, sJ0)[sp] = (real)0;
      FSLOT(f, sJ3)[sp] = (real)0;
    } else if (bc) {
      // Neumann / Robin face (eq. 2.1): the outward normal derivative (+ gamma u)
      // in the slot of the normal-derivative jump, nothing in the others
      const real gam = fsc[6 + f];
      FSLOT(f, sJ0)[sp] = (real)0;
      FSLOT(f, sJ3)[sp] = (side ? geo_e[a] : -geo_e[a]) * Nv + gam * Fv;
    } else if (nb != -1) {
      // a corner set shares the theta and x3 scales of its layer-1 element
      FSLOT(f, sFn)[sp] = Fn;
      FSLOT(f, sJ0)[sp] = Fv - Fn;
      FSLOT(f, sJ3)[sp] = geo_e[a] * Nv - fm->s1[f][a] * Nn;
    } else {
      FSLOT(f, sJ0)[sp] = Fv;
      FSLOT(f, sJ3)[sp] = (real)0;
    }
  }
  __syncthreads();
  if constexpr (!nbhd_coef(COEF)) {
    // Box meshes (unit face-norm weights): stages 2-5 in two line-job stages.
    // The Kronecker forms of every field k factor as G_k = MP (x) X_k + KP (x) Y_k
    // (inner factor along the field's first axis, outer along the other), and
    // the tangential derivative D and its transpose D^T act along the same
    // axis as the inner factor, so they fold into P x P products:
    //   field 0: X = MP, Y = 0 (along p1)
    //   field 3: X = MP + KP, Y = MP (along p1)
    //   field 1: X = c M12, Y = c M1 on v (along p1), field 2 the same along p2,
    //            M1 = D^T MP D, M12 = D^T (MP + KP) D, v = s0 F - s1 Fn on
    //            interior faces (F on Dirichlet faces, c = 1 there), 0 on
    //            Neumann / Robin faces and faces left to k_face_mixed;
    // the outputs are G0, G3 and U1 = c D^T G1, U2 = c D^T G2 directly.
    // Stage A: alpha = X v -> B slot, beta = Y v -> A slot (inner axis)
    for (int t = tid; t < 24 * P; t += nt) {
      const int f = t / (4 * P), rem = t - f * 4 * P;
      const int fld = rem / P, ln = rem - fld * P;
      const int ob = fld == 2 ? ln : ln * P, os = fld == 2 ? P : 1;
      real ev[HPE], od[HPE], al[P], be[P];
      if (fld == 0 || fld == 3) {
        load_fold(FSLOT(f, fld ? sJ3 : sJ0) + ob, os, ev, od);
        if (fld == 0) {
          pp_line<2>(ev, od, al);
#pragma unroll
          for (int i = 0; i < P; ++i) be[i] = (real)0;
        } else {
          pp_line<4>(ev, od, al);
          pp_line<2>(ev, od, be);
        }
      } else if (fm->bc[f]) {
#pragma unroll
        for (int i = 0; i < P; ++i) al[i] = be[i] = (real)0;
      } else {
        const int a = f >> 1;
        const int tax = fld == 2 ? ((a == 2) ? 1 : 2) : ((a == 0) ? 1 : 0);
        const real *Fp = FSLOT(f, sF) + ob;
        real v[P], c = (real)1;
        if (fm->nb[f] != -1) {
          const real s0 = geo_e[tax], s1 = fm->s1[f][tax];
          const real *Fnp = FSLOT(f, sFn) + ob;
#pragma unroll
          for (int m = 0; m < P; ++m) v[m] = s0 * Fp[m * os] - s1 * Fnp[m * os];
          c = s0;
        } else {
#pragma unroll
          for (int m = 0; m < P; ++m) v[m] = Fp[m * os];
        }
        fold_p(v, ev, od);
        pp_line<6>(ev, od, al);
        pp_line<5>(ev, od, be);
#pragma unroll
        for (int i = 0; i < P; ++i) {
          al[i] *= c;
          be[i] *= c;
        }
      }
      real *Bs = FSLOT(f, sB0 + fld) + ob, *As = FSLOT(f, sA0 + fld) + ob;
#pragma unroll
      for (int i = 0; i < P; ++i) {
        Bs[i * os] = al[i];
        As[i * os] = be[i];
      }
    }
    __syncthreads();
    // Stage B (outer axis): G = MP alpha + KP beta -> the J slot of the field
    // (G0, U1, U2, G3)
    for (int t = tid; t < 24 * P; t += nt) {
      const int f = t / (4 * P), rem = t - f * 4 * P;
      const int fld = rem / P, ln = rem - fld * P;
      const int ob = fld == 2 ? ln * P : ln, os = fld == 2 ? 1 : P;
      real ev[HPE], od[HPE], g[P];
      load_fold(FSLOT(f, sB0 + fld) + ob, os, ev, od);
      pp_line<2>(ev, od, g);
      if (fld) {
        real h[P];
        load_fold(FSLOT(f, sA0 + fld) + ob, os, ev, od);
        pp_line<3>(ev, od, h);
#pragma unroll
        for (int i = 0; i < P; ++i) g[i] += h[i];
      }
      real *G = FSLOT(f, sJ0 + fld) + ob;
#pragma unroll
      for (int i = 0; i < P; ++i) G[i * os] = g[i];
    }
    __syncthreads();
  } else {
    // 2: tangential derivatives (line jobs): J1 along p1 (lines p2), J2 along p2 (lines p1);
    // interior faces: jumps of the physical derivatives, Dirichlet faces: d/dlambda
    for (int t = tid; t < 12 * P; t += nt) {
      const int dir = t / (6 * P), rem = t - dir * 6 * P;
      const int f = rem / P, ln = rem - f * P;
      const int a = f >> 1;
      const int tax = dir ? ((a == 2) ? 1 : 2) : ((a == 0) ? 1 : 0);
      const int ob = dir ? ln : ln * P, os = dir ? P : 1;
      const int nb = fm->nb[f];
      real ev[HPE], od[HPE], g[P];
      load_fold(FSLOT(f, sF) + ob, os, ev, od);
      pp_line<0>(ev, od, g);
      real *J = FSLOT(f, dir ? sJ2 : sJ1) + ob;
      if (fm->bc[f]) {  // Neumann / Robin, or left to k_face_mixed
#pragma unroll
        for (int m = 0; m < P; ++m) J[m * os] = (real)0;
      } else if (nb != -1) {
        const real s0 = geo_e[tax], s1 = fm->s1[f][tax];
        real h[P];
        load_fold(FSLOT(f, sFn) + ob, os, ev, od);
        pp_line<0>(ev, od, h);
#pragma unroll
        for (int m = 0; m < P; ++m) J[m * os] = s0 * g[m] - s1 * h[m];
      } else {
#pragma unroll
        for (int m = 0; m < P; ++m) J[m * os] = g[m];
      }
    }
    __syncthreads();
    // 3: first Kronecker factor along p1 (line jobs per field): a = MP J, b = KP J;
    // face-norm weights: w[0] on the L2 jump of u; (w[3k-2], w[3k-1], w[3k]) =
    // (L2, quotient along t1, quotient along t2) on jump field k (1 on box meshes):
    // A_k = w[3k] a, B_k = w[3k-2] a + w[3k-1] b; field 0: A_0 = 0, B_0 = w[0] a
    for (int t = tid; t < 24 * P; t += nt) {
      const int f = t / (4 * P), rem = t - f * 4 * P;
      const int fld = rem / P, p2 = rem - fld * P;
      real ev[HPE], od[HPE], av[P], bv[P];
      load_fold(FSLOT(f, sJ0 + fld) + p2 * P, 1, ev, od);
      pp_line<2>(ev, od, av);
      real wb = (real)1, wc = (real)1;
      if (nbhd_coef(COEF) && A.fw) {
        const real *wf = A.fw + ((int64_t)e * 6 + f) * hpse::FACE_W;
        wb = fld ? wf[3 * fld - 2] : wf[0];
        wc = fld ? wf[3 * fld - 1] : (real)0;
        if (fld) {
          const real wa = wf[3 * fld];
#pragma unroll
          for (int i = 0; i < P; ++i) FSLOT(f, sA0 + fld)[p2 * P + i] = wa * av[i];
        }
      } else if (fld) {
#pragma unroll
        for (int i = 0; i < P; ++i) FSLOT(f, sA0 + fld)[p2 * P + i] = av[i];
      }
      if (fld) {
        pp_line<3>(ev, od, bv);
#pragma unroll
        for (int i = 0; i < P; ++i) FSLOT(f, sB0 + fld)[p2 * P + i] = wb * av[i] + wc * bv[i];
      } else {
#pragma unroll
        for (int i = 0; i < P; ++i) FSLOT(f, sB0)[p2 * P + i] = wb * av[i];
      }
    }
    __syncthreads();
    // 4: second factor along p2 (line jobs per field): G_k = MP B_k + KP A_k -> J_k slots
    for (int t = tid; t < 24 * P; t += nt) {
      const int f = t / (4 * P), rem = t - f * 4 * P;
      const int fld = rem / P, p1 = rem - fld * P;
      real ev[HPE], od[HPE], g[P];
      load_fold(FSLOT(f, sB0 + fld) + p1, P, ev, od);
      pp_line<2>(ev, od, g);
      if (fld) {
        real h[P];
        load_fold(FSLOT(f, sA0 + fld) + p1, P, ev, od);
        pp_line<3>(ev, od, h);
#pragma unroll
        for (int i = 0; i < P; ++i) g[i] += h[i];
      }
      real *G = FSLOT(f, sJ0 + fld) + p1;
#pragma unroll
      for (int i = 0; i < P; ++i) G[i * P] = g[i];
    }
    __syncthreads();
    // corner side of face 0 (r = r_1 of the edge, psi = psi_1 of the vertex-edge
    // neighbourhood): minus the transposed corner traces of the weighted jumps,
    // y_c[k] = -sum_p1 g0[k][p1] - s_z sum_m D[m][k] sum_p1 g2[m][p1] (the
    // corner's derivatives along x and y vanish), stored per (slot, rhs) for the
    // corner kernel
    if (corner_f0(COEF) && A.cscr && !A.self_only) {
      const int slot = A.cslot[2 * e];
      if (slot >= 0) {
        for (int k = tid; k < P; k += nt) {
          real s0 = 0, s2 = 0;
          for (int p1 = 0; p1 < P; ++p1) s0 += FSLOT(0, sJ0)[k * P + p1];
          for (int m = 0; m < P; ++m) {
            real g2 = 0;
            for (int p1 = 0; p1 < P; ++p1) g2 += FSLOT(0, sJ2)[m * P + p1];
            s2 += Ds[m * P + k] * g2;
          }
          A.cscr[((int64_t)slot * A.n_rhs + r) * hpse::CSCR_STRIDE + k] = -(s0 + geo_e[2] * s2);
        }
      }
    }
    // corner side of face 4 (rho = rho_1 of the vertex, zeta = zeta_1 of the
    // vertex-edge neighbourhood): the corner constant's trace is 1 at every face
    // node, so y_c = -sum of the weighted jump of u over the face
    if (corner_f4(COEF) && A.cscr && !A.self_only && tid == 0) {
      const int slot = A.cslot[2 * e + 1];
      if (slot >= 0) {
        real s0 = 0;
        for (int t = 0; t < P2; ++t) s0 += FSLOT(4, sJ0)[t];
        A.cscr[((int64_t)slot * A.n_rhs + r) * hpse::CSCR_STRIDE] = -s0;
      }
    }
    // 5: transposed tangential derivatives (line jobs): U1 = c1 D^T G1 along p1,
    // U2 = c2 D^T G2 along p2 (c = the tangential scale on interior faces, 1 on
    // Dirichlet faces)
    for (int t = tid; t < 12 * P; t += nt) {
      const int dir = t / (6 * P), rem = t - dir * 6 * P;
      const int f = rem / P, ln = rem - f * P;
      const int a = f >> 1;
      const int tax = dir ? ((a == 2) ? 1 : 2) : ((a == 0) ? 1 : 0);
      const int ob = dir ? ln : ln * P, os = dir ? P : 1;
      const real c = fm->nb[f] != -1 ? geo_e[tax] : (real)1;
      real ev[HPE], od[HPE], u[P];
      load_fold(FSLOT(f, dir ? sJ2 : sJ1) + ob, os, ev, od);
      pp_line<1>(ev, od, u);
      real *U = FSLOT(f, dir ? sA2 : sA1) + ob;
#pragma unroll
      for (int m = 0; m < P; ++m) U[m * os] = c * u[m];
    }
    __syncthreads();
  }
  // 6: gather onto the nodes of the element: per face the face layer takes
  // G0 + U1 + U2, every node of a normal line D[nend][n] s_a G3
  constexpr int sU1 = nbhd_coef(COEF) ? sA1 : sJ1, sU2 = nbhd_coef(COEF) ? sA2 : sJ2;
  for (int t = tid; t < P3; t += nt) {
    const int i = t % P, j = (t / P) % P, k = t / P2;
    real acc = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int a = f >> 1, nend = (f & 1) ? P - 1 : 0;
      const int n = a == 0 ? i : (a == 1 ? j : k);
      const int p1 = a == 0 ? j : i;
      const int p2 = a == 2 ? j : k;
      const int sp = p2 * P + p1;
      acc += Ds[nend * P + n] * (fsc[f] * FSLOT(f, sJ3)[sp]);
      if (n == nend) acc += FSLOT(f, sJ0)[sp] + FSLOT(f, sU1)[sp] + FSLOT(f, sU2)[sp] + fsc[6 + f] * FSLOT(f, sJ3)[sp];
    }
    sy[t] += acc;
  }
  __syncthreads();
#undef FSLOT
}

// rho[q] of one z-column: registers, or shared memory (stride Q2 + 1)
template <bool SMEM>
struct ColumnRho {
  real v[Q];
  __device__ __forceinline__ void bind(real *, int) {}
  __device__ __forceinline__ real &operator[](int q) { return v[q]; }
};
template <>
struct ColumnRho<true> {
  real *p;
  __device__ __forceinline__ void bind(real *base, int col) { p = base + col; }
  __device__ __forceinline__ real &operator[](int q) { return p[q * (Q2 + 1)]; }
};

// rho[q] of one z-column in place, in the column's own slots of the T
// fields (q -> T00 / TL row q mod P; Q <= 2P): the forward holds the
// column's T inputs in registers before it writes rho, the transpose stores
// its outputs there after its last read of rho.  Lanes past the last column
// read the last column's rho and write nothing.
struct ColumnRhoT {
  real *p;
  bool w;
  struct Ref {
    real *a;
    bool w;
    __device__ __forceinline__ operator real() const { return *a; }
    __device__ __forceinline__ Ref &operator=(real v) {
      if (w) *a = v;
      return *this;
    }
  };
  __device__ __forceinline__ void bind(real *T, int col, bool ok) {
    p = T + col;
    w = ok;
  }
  __device__ __forceinline__ Ref operator[](int q) { return Ref{p + (q / P) * Q2P + (q % P) * Q2, w}; }
};

// warp-uniform dispatch of a runtime chunk index to its compile-time instance
#define HPSE_DISPATCH4(NC, c, CALL)            \
  do {                                         \
    if ((c) == 0) CALL(0);                     \
    if constexpr ((NC) > 1) if ((c) == 1) CALL(1); \
    if constexpr ((NC) > 2) if ((c) == 2) CALL(2); \
    if constexpr ((NC) > 3) if ((c) == 3) CALL(3); \
  } while (0)

// ---------------------------------------------------------------------------
// Operator apply: y = A u  (volume + faces), one CTA per (element, rhs).
// Shared memory: su[P3] | X[NX][QP2] | T region (T fields, then sy and the
// face scratch) | D copy, per-face scales | (rho of the z-stage) | FP64
// reduction buffer (16-byte aligned).
// ---------------------------------------------------------------------------
template <int COEF>
struct ApplyLayout {
  static constexpr int NX = (var_coef(COEF)) ? 3 : 2;
  static constexpr int NTF = y_first(COEF) ? 4 : (var_coef(COEF) ? 3 : 2);
  static constexpr int T_REGION0 = NTF * Q2P;
  static constexpr int T_NEED = P3 + 6 * FACE_ARR * P2;
  static constexpr int T_REGION = T_REGION0 > T_NEED ? T_REGION0 : T_NEED;
  static constexpr int TABS = P2 + FACE_META_REALS;  // D copy, then the face phase's per-face data
  static constexpr int TOTAL0 = P3 + NX * QP2 + T_REGION + TABS;
  // the z-stage's pointwise residual rho per column in shared memory (Q
  // entries per column, one spare column for the lanes past the last one)
  // where that keeps APPLY_MINB CTAs per SM; else in registers
  static constexpr int RHO_LEN = Q * (Q2 + 1);
  // packed z-stage: rho in place in the T fields (ColumnRhoT), no buffer
  static constexpr bool RHO_INPLACE = packed_coef(COEF, 4) || packed_coef(COEF, 8);
#if defined(HPSE_APPLY_RHO_REG)
  static constexpr bool RHO_SMEM = false;  // set at build time (layout experiments)
#else
  static constexpr bool RHO_SMEM =
      !RHO_INPLACE &&
      (((size_t)(TOTAL0 + RHO_LEN) * sizeof(real) + 64 * sizeof(double) + 1024) * APPLY_MINB <= 232448);
#endif
  static constexpr int TOTAL = TOTAL0 + (RHO_SMEM ? RHO_LEN : 0);
  // the FP64 reduction buffer starts on a 16-byte boundary whatever REAL is
  static constexpr size_t RED_OFF = (((size_t)TOTAL * sizeof(real) + 15) / 16) * 16;
  static constexpr size_t BYTES = RED_OFF + 64 * sizeof(double);
};

template <int COEF, int MODE>
__global__ void __launch_bounds__(NT, APPLY_MINB) k_apply(const ApplyArgs A) {
  typedef ApplyLayout<COEF> L;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real *su = reinterpret_cast<real *>(smem_raw);
  real *sX = su + P3;               // X0 | X2 | (X1)
  real *sT = sX + L::NX * QP2;      // T00 | TL | (T10) | (T01)
  real *stab = sT + L::T_REGION;    // D (runtime-indexed copy for the face gather) | per-face scales
  real *srho = stab + L::TABS;      // rho of the z-stage (L::RHO_SMEM)
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
  const int tid = threadIdx.x;
  constexpr int nt = NT;

  for (int t = tid; t < P2; t += nt) stab[t] = c_tab.D[t];
  FaceMeta *fm = face_meta(stab);
  if (MODE != MODE_TRANSPOSE && tid < 6) face_meta_fill<COEF, MODE>(A, e, r, geo_e, fm, tid);
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

    // ---- x-stage (lines along x: (j, k)), outputs in chunks -------------
    {
      typedef Lines<P2> LS;
      for (int it = tid; it < LS::NC * LS::PADL; it += nt) {
        const int c = it / LS::PADL, lp = it - c * LS::PADL;
        const bool ok = lp < P2;
        const int l = ok ? lp : P2 - 1;
        real e[HPE], o[HPE];
        {
          real v[P];
#pragma unroll
          for (int i = 0; i < P; ++i) v[i] = su[l * P + i];
          fold_p(v, e, o);
        }
        if constexpr (packed_coef(COEF, 1)) {
          float2 e2[HPE], o2[HPE];
#pragma unroll
          for (int j = 0; j < HPE; ++j) {
            e2[j] = make_float2(e[j], e[j]);
            o2[j] = make_float2(o[j], o[j]);
          }
#define XF_CALL(CI) x_fwd_chunk2<COEF, (CI < LS::NC ? CI : 0), LS::NC>(e2, o2, X0, X1, X2, l, ok)
          HPSE_DISPATCH4(LS::NC, c, XF_CALL);
#undef XF_CALL
        } else {
#define XF_CALL(CI) x_fwd_chunk<COEF, (CI < LS::NC ? CI : 0), LS::NC>(e, o, X0, X1, X2, l, ok)
          HPSE_DISPATCH4(LS::NC, c, XF_CALL);
#undef XF_CALL
        }
      }
    }
    __syncthreads();

    // ---- y-stage (lines along y: (qa, k)), outputs in chunks ------------
    {
      typedef Lines<QP> LS;
      for (int it = tid; it < LS::NC * LS::PADL; it += nt) {
        const int c = it / LS::PADL, lp = it - c * LS::PADL;
        const bool ok = lp < QP;
        const int l = ok ? lp : QP - 1;
        const int qa = l % Q, k = l / Q;
        if constexpr (packed_coef(COEF, 2)) {
          float2 de[HPE], dd[HPE], we[HPE], wo[HPE];
          {
            float2 v[P];
            if (COEF == COEF_SCALAR) {
#pragma unroll
              for (int j = 0; j < P; ++j) {
                const real x0 = X0[(k * P + j) * Q + qa];
                v[j] = make_float2(x0, x0);
              }
              fold_p2(v, de, dd);
#pragma unroll
              for (int j = 0; j < P; ++j) v[j] = make_float2(X2[(k * P + j) * Q + qa], X1[(k * P + j) * Q + qa]);
              fold_p2(v, we, wo);
            } else {
#pragma unroll
              for (int j = 0; j < P; ++j) v[j] = make_float2(X0[(k * P + j) * Q + qa], X2[(k * P + j) * Q + qa]);
              fold_p2(v, we, wo);
            }
          }
#define YF_CALL(CI) \
  y_fwd_chunk2<COEF, (CI < LS::NC ? CI : 0), LS::NC>(de, dd, we, wo, T00, TL, T10, T01, qa, k, ok, sx2, sy2)
          HPSE_DISPATCH4(LS::NC, c, YF_CALL);
#undef YF_CALL
        } else {
          real e0[HPE], o0[HPE], e2[HPE], o2[HPE], e1[HPE], o1[HPE];
          {
            real v[P];
#pragma unroll
            for (int j = 0; j < P; ++j) v[j] = X0[(k * P + j) * Q + qa];
            fold_p(v, e0, o0);
#pragma unroll
            for (int j = 0; j < P; ++j) v[j] = X2[(k * P + j) * Q + qa];
            fold_p(v, e2, o2);
            if (var_coef(COEF)) {
#pragma unroll
              for (int j = 0; j < P; ++j) v[j] = X1[(k * P + j) * Q + qa];
              fold_p(v, e1, o1);
            }
          }
          // per-x-point factors, constant along this y-line: vertex neighbourhood
          // 1/sin^2(x_1) on u_22, vertex-edge 1 + e^{2 x_1} on u_11
          const real sy2q = (COEF == COEF_VERTEX) ? sy2 * A.kappa[(int64_t)e * hpse::KAPPA_STRIDE + qa] : sy2;
          const real sx2q =
              (COEF == COEF_VERTEX_EDGE) ? sx2 * ((real)1 + A.kappa[(int64_t)e * hpse::KAPPA_STRIDE + qa]) : sx2;
#define YF_CALL(CI) \
    y_fwd_chunk<COEF, (CI < LS::NC ? CI : 0), LS::NC>(e0, o0, e1, o1, e2, o2, T00, TL, T10, T01, qa, k, ok, sx2q, \
                                                      sy2q)
          HPSE_DISPATCH4(LS::NC, c, YF_CALL);
#undef YF_CALL
        }
      }
    }
    __syncthreads();
  }

  // ---- z-stage per (qa, qb) column: forward + pointwise weight into rho[Q]
  // (registers), then the transpose from rho; both folded (even-odd) ------
  for (int lp = tid; lp < PAD32(Q2); lp += nt) {
    const bool ok = lp < Q2;
    const int l = ok ? lp : Q2 - 1;
    const int qa = l % Q, qb = l / Q;
    const int64_t cbase = A.coef_off[e] + (int64_t)qb * Q + qa;
    // edge (vertex-edge) neighbourhood: e^{2 tau} (e^{2 psi}) multiplies the
    // z second derivative; x is constant along this z-column
    const real sz2c =
        (COEF == COEF_EDGE || COEF == COEF_VERTEX_EDGE) ? sz2 * A.kappa[(int64_t)e * hpse::KAPPA_STRIDE + qa] : sz2;
    // lanes past the last column keep their rho in the spare column Q2
    constexpr bool inplace = L::RHO_INPLACE && packed_mode(COEF, MODE);
    std::conditional_t<inplace, ColumnRhoT, ColumnRho<L::RHO_SMEM>> rho;
    if constexpr (inplace) rho.bind(sT, l, ok);
    else rho.bind(srho, ok ? l : Q2);
    if (MODE == MODE_TRANSPOSE) {
#pragma unroll
      for (int qc = 0; qc < Q; ++qc) rho[qc] = (real)A.rho[(int64_t)r * A.nquad + cbase + (int64_t)qc * Q2];
    } else if constexpr (packed_coef(COEF, 4)) {
      // -div(a grad u): A = (TL, T10) -> (p0, px) = (B0 TL, B0 T10),
      // B = (T01, T00) -> (py, p2) = (B0 T01, B2 T00), p1 = B1 T00 on B.y;
      // Laplacian: B = (TL, T00) -> (p0, p2)
      float2 eA[HPE], oA[HPE], eB[HPE], oB[HPE];
      {
        float2 v[P];
        if (COEF == COEF_SCALAR) {
#pragma unroll
          for (int k = 0; k < P; ++k) v[k] = make_float2(TL[k * Q2 + l], T10[k * Q2 + l]);
          fold_p2(v, eA, oA);
#pragma unroll
          for (int k = 0; k < P; ++k) v[k] = make_float2(T01[k * Q2 + l], T00[k * Q2 + l]);
          fold_p2(v, eB, oB);
        } else {
#pragma unroll
          for (int k = 0; k < P; ++k) v[k] = make_float2(TL[k * Q2 + l], T00[k * Q2 + l]);
          fold_p2(v, eB, oB);
        }
      }
      const real wab = c_tab.WQ[qa] * c_tab.WQ[qb] * Jac;
#pragma unroll
      for (int qc = 0; qc <= HQ; ++qc) {
        float2 ap = zero2(), am = zero2(), bp = zero2(), bm = zero2();
        real p1 = 0, m1 = 0;
        fwd_pm2<1>(eB, oB, qc, bp, bm);
        if (COEF == COEF_SCALAR) {
          fwd_pm2<0>(eA, oA, qc, ap, am);
          fwd_pm_h<1, 1>(eB, oB, qc, p1, m1);
        }
#pragma unroll
        for (int side = 0; side < (qc < HQ ? 2 : 1); ++side) {
          const int q = side ? Q - 1 - qc : qc;
          const real sg = side ? (real)-1 : (real)1;
          const float2 b = side ? sub2(bp, bm) : add2(bp, bm);
          if (COEF == COEF_SCALAR) {
            const float2 a = side ? sub2(ap, am) : add2(ap, am);
            const real sigma0 = sz2c * b.y + a.x;
            real mq, dx, dy, dz;
            load_coef4(A.coef + 4 * (cbase + (int64_t)q * Q2), mq, dx, dy, dz);
            rho[q] = mq * (sigma0 + dz * (p1 + sg * m1) + dx * a.y + dy * b.x);
          } else {
            rho[q] = wab * c_tab.WQ[q] * (sz2c * b.y + b.x);
          }
        }
        __syncwarp();  // scheduling fence (register pressure); reached by all 32 lanes
      }
    } else {
      real e00[HPE], o00[HPE], eL[HPE], oL[HPE], e10[HPE], o10[HPE], e01[HPE], o01[HPE];
      {
        real v[P];
#pragma unroll
        for (int k = 0; k < P; ++k) v[k] = T00[k * Q2 + l];
        fold_p(v, e00, o00);
#pragma unroll
        for (int k = 0; k < P; ++k) v[k] = TL[k * Q2 + l];
        fold_p(v, eL, oL);
        if (var_coef(COEF)) {
#pragma unroll
          for (int k = 0; k < P; ++k) v[k] = T10[k * Q2 + l];
          fold_p(v, e10, o10);
        }
        if (y_first(COEF)) {
#pragma unroll
          for (int k = 0; k < P; ++k) v[k] = T01[k * Q2 + l];
          fold_p(v, e01, o01);
        }
      }
      const real wab = c_tab.WQ[qa] * c_tab.WQ[qb] * Jac;
#pragma unroll
      for (int qc = 0; qc <= HQ; ++qc) {
        real p2 = 0, m2 = 0, p0 = 0, m0 = 0, p1 = 0, m1 = 0, px = 0, mx = 0, py = 0, my = 0;
        fwd_pm<2>(e00, o00, qc, p2, m2);
        fwd_pm<0>(eL, oL, qc, p0, m0);
        if (var_coef(COEF)) {
          fwd_pm<1>(e00, o00, qc, p1, m1);
          fwd_pm<0>(e10, o10, qc, px, mx);
        }
        // the d_y slot: u_y (variable coefficient) or u_xz (vertex-edge)
        if (y_first(COEF)) fwd_pm<0>(e01, o01, qc, py, my);
        if (mixed_xz(COEF)) fwd_pm<1>(e10, o10, qc, py, my);
#pragma unroll
        for (int side = 0; side < (qc < HQ ? 2 : 1); ++side) {
          const int q = side ? Q - 1 - qc : qc;
          const real sg = side ? (real)-1 : (real)1;
          const real sigma0 = sz2c * (p2 + sg * m2) + (p0 + sg * m0);
          if (var_coef(COEF)) {
            real mq, dx, dy, dz;
            load_coef4(A.coef + 4 * (cbase + (int64_t)q * Q2), mq, dx, dy, dz);
            rho[q] = mq * (sigma0 + dz * (p1 + sg * m1) + dx * (px + sg * mx) + dy * (py + sg * my));
          } else {
            rho[q] = wab * c_tab.WQ[q] * sigma0;
          }
        }
        __syncwarp();  // scheduling fence (register pressure); reached by all 32 lanes
      }
    }
    if constexpr (packed_coef(COEF, 8) && packed_mode(COEF, MODE)) {
      // -div(a grad u): (rho, d_x rho) -> (rp, xp) by (B0, B0), (d_y rho,
      // sz2 rho) -> (yp, zp) by (B0, B2), d_z rho by B1 into zp (scalar);
      // Laplacian: (rho, sz2 rho) -> (rp, zp) by (B0, B2)
      float2 pa[HPE], ma[HPE], pb[HPE], mb[HPE];
#pragma unroll
      for (int k = 0; k < HPE; ++k) pa[k] = ma[k] = pb[k] = mb[k] = zero2();
#pragma unroll
      for (int qc = 0; qc <= HQ; ++qc) {
        float2 va[2], vb[2];
        real sd[2];
#pragma unroll
        for (int side = 0; side < (qc < HQ ? 2 : 1); ++side) {
          const int q = side ? Q - 1 - qc : qc;
          const real rq = rho[q];
          if (COEF == COEF_SCALAR) {
            real mq, dx, dy, dz;
            load_coef4(A.coef + 4 * (cbase + (int64_t)q * Q2), mq, dx, dy, dz);
            va[side] = make_float2(rq, dx * rq);
            vb[side] = make_float2(dy * rq, sz2c * rq);
            sd[side] = dz * rq;
          } else {
            vb[side] = make_float2(rq, sz2c * rq);
          }
        }
        if (qc < HQ) {
          rev_pair2<1>(add2(vb[0], vb[1]), sub2(vb[0], vb[1]), qc, pb, mb);
          if (COEF == COEF_SCALAR) {
            rev_pair2<0>(add2(va[0], va[1]), sub2(va[0], va[1]), qc, pa, ma);
            const real se = sd[0] + sd[1], so = sd[0] - sd[1];
#pragma unroll
            for (int k = 0; k < HPE; ++k) {
              pb[k].y += c_tab.FE[1][qc * HPE + k] * so;
              if (k < HP) mb[k].y += c_tab.FO[1][qc * HPE + k] * se;
            }
          }
        } else {
          rev_mid2<1>(vb[0], pb);
          if (COEF == COEF_SCALAR) {
            rev_mid2<0>(va[0], pa);
#pragma unroll
            for (int k = 0; k < HP; ++k) mb[k].y += c_tab.FO[1][HQ * HPE + k] * sd[0];
          }
        }
      }
      if (ok) {
#pragma unroll
        for (int k = 0; k < HPE; ++k) {
          if (COEF == COEF_SCALAR) {
            put_p2(TL + l, T10 + l, Q2, k, pa[k], ma[k]);
            put_p2(T01 + l, T00 + l, Q2, k, pb[k], mb[k]);
          } else {
            put_p2(TL + l, T00 + l, Q2, k, pb[k], mb[k]);
          }
        }
      }
    } else {
      real zp[HPE], zm[HPE], rp[HPE], rm[HPE], xp[HPE], xm[HPE], yp[HPE], ym[HPE];
#pragma unroll
      for (int k = 0; k < HPE; ++k) {
        zp[k] = zm[k] = rp[k] = rm[k] = xp[k] = xm[k] = yp[k] = ym[k] = (real)0;
      }
#pragma unroll
      for (int qc = 0; qc <= HQ; ++qc) {
        // the streams rz2 = sz2 rho, rzd = d_z rho, rho, rxd = d_x rho, ryd = d_y rho
        // at the pair of points (qc, Q-1-qc), folded
        real s2[2], sd[2], s0[2], sx[2], sy[2];
#pragma unroll
        for (int side = 0; side < (qc < HQ ? 2 : 1); ++side) {
          const int q = side ? Q - 1 - qc : qc;
          const real rq = rho[q];
          real dx = 0, dy = 0, dz = 0;
          if (var_coef(COEF)) {
            real mq;
            load_coef4(A.coef + 4 * (cbase + (int64_t)q * Q2), mq, dx, dy, dz);
          }
          s2[side] = sz2c * rq;
          sd[side] = dz * rq;
          s0[side] = rq;
          sx[side] = dx * rq;
          sy[side] = dy * rq;
        }
        if (qc < HQ) {
          rev_pair<2>(s2[0] + s2[1], s2[0] - s2[1], qc, zp, zm);
          rev_pair<0>(s0[0] + s0[1], s0[0] - s0[1], qc, rp, rm);
          if (var_coef(COEF)) {
            rev_pair<1>(sd[0] + sd[1], sd[0] - sd[1], qc, zp, zm);
            rev_pair<0>(sx[0] + sx[1], sx[0] - sx[1], qc, xp, xm);
          }
          if (y_first(COEF)) rev_pair<0>(sy[0] + sy[1], sy[0] - sy[1], qc, yp, ym);
          if (mixed_xz(COEF)) rev_pair<1>(sy[0] + sy[1], sy[0] - sy[1], qc, xp, xm);
        } else {
          rev_mid<2>(s2[0], zp, zm);
          rev_mid<0>(s0[0], rp, rm);
          if (var_coef(COEF)) {
            rev_mid<1>(sd[0], zp, zm);
            rev_mid<0>(sx[0], xp, xm);
          }
          if (y_first(COEF)) rev_mid<0>(sy[0], yp, ym);
          if (mixed_xz(COEF)) rev_mid<1>(sy[0], xp, xm);
        }
      }
      if (ok) {
#pragma unroll
        for (int k = 0; k < HPE; ++k) {
          put_p(T00 + l, Q2, k, zp[k], zm[k]);
          put_p(TL + l, Q2, k, rp[k], rm[k]);
          if (var_coef(COEF)) put_p(T10 + l, Q2, k, xp[k], xm[k]);
          if (y_first(COEF)) put_p(T01 + l, Q2, k, yp[k], ym[k]);
        }
      }
    }
  }
  __syncthreads();

  // ---- y-stage transpose (lines (qa, k)), outputs j in chunks ------------
  {
    typedef Lines<QP> LS;
    for (int it = tid; it < LS::NC * LS::PADL; it += nt) {
      const int c = it / LS::PADL, lp = it - c * LS::PADL;
      const bool ok = lp < QP;
      const int l = ok ? lp : QP - 1;
      const int qa = l % Q, k = l / Q;
      const real sy2q = (COEF == COEF_VERTEX) ? sy2 * A.kappa[(int64_t)e * hpse::KAPPA_STRIDE + qa] : sy2;
      const real sx2q =
          (COEF == COEF_VERTEX_EDGE) ? sx2 * ((real)1 + A.kappa[(int64_t)e * hpse::KAPPA_STRIDE + qa]) : sx2;
      if constexpr (packed_coef(COEF, 16) && packed_mode(COEF, MODE)) {
#define YR_CALL(CI) \
  y_rev_chunk2<COEF, (CI < LS::NC ? CI : 0), LS::NC>(T00, TL, T10, T01, X0, X1, X2, qa, k, ok, sx2q, sy2q)
        HPSE_DISPATCH4(LS::NC, c, YR_CALL);
#undef YR_CALL
      } else {
#define YR_CALL(CI) \
  y_rev_chunk<COEF, (CI < LS::NC ? CI : 0), LS::NC>(T00, TL, T10, T01, X0, X1, X2, qa, k, ok, sx2q, sy2q)
        HPSE_DISPATCH4(LS::NC, c, YR_CALL);
#undef YR_CALL
      }
    }
  }
  __syncthreads();

  // ---- x-stage transpose (lines (j, k)), outputs i in chunks -> sy ---------
  real *sy = sT;  // T region is free now
  {
    typedef Lines<P2> LS;
    for (int it = tid; it < LS::NC * LS::PADL; it += nt) {
      const int c = it / LS::PADL, lp = it - c * LS::PADL;
      const bool ok = lp < P2;
      const int l = ok ? lp : P2 - 1;
      if constexpr (packed_coef(COEF, 32) && packed_mode(COEF, MODE)) {
#define XR_CALL(CI) x_rev_chunk2<COEF, (CI < LS::NC ? CI : 0), LS::NC>(X0, X1, X2, sy, l, ok)
        HPSE_DISPATCH4(LS::NC, c, XR_CALL);
#undef XR_CALL
      } else {
#define XR_CALL(CI) x_rev_chunk<COEF, (CI < LS::NC ? CI : 0), LS::NC>(X0, X1, X2, sy, l, ok)
        HPSE_DISPATCH4(LS::NC, c, XR_CALL);
#undef XR_CALL
      }
    }
  }
  __syncthreads();

  // ---- faces ---------------------------------------------------------------
  if (MODE != MODE_TRANSPOSE && !A.skip_faces)
    face_phase<COEF, MODE>(A, e, r, su, sy, sT + P3, stab, geo_e, fm);

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
// Preconditioner CTAs hold several (element, rhs) items; each item owns
// PC_TPI threads (one per line of P nodes, whole warps).
constexpr int PC_TPI = PAD32(P2);
constexpr int PC_ITEMS_RAW = 384 / PC_TPI;
constexpr int PC_ITEMS = PC_ITEMS_RAW < 1 ? 1 : (PC_ITEMS_RAW > 8 ? 8 : PC_ITEMS_RAW);
constexpr int PC_NT = PC_ITEMS * PC_TPI;
constexpr int PC_WARPS_PER_ITEM = PC_TPI / 32;
// per item: two P^3 blocks; then the reduction buffer; then per item the x3
// eigenbasis and eigenvalues of the C* form (edge neighbourhood)
constexpr size_t PC_RED_OFF = (size_t)PC_ITEMS * 2 * P3 * sizeof(real);
constexpr size_t PC_Z_OFF = PC_RED_OFF + (size_t)(PC_NT / 32) * 2 * sizeof(double);
constexpr size_t PC_BYTES = PC_Z_OFF + (size_t)PC_ITEMS * (P2 + P) * sizeof(real);

// out = (S^T or S) applied along `axis` of one P x P x P block (x fastest);
// thread lt of the item handles line lt (no loop: PC_TPI >= P^2 lines)
__device__ __forceinline__ void tensor_stage(const real *in, real *out, int axis, bool transpose, int lt) {
  const int stride = axis == 0 ? 1 : (axis == 1 ? P : P2);
  if (lt < P2) {
    int b;
    if (axis == 0) b = lt * P;
    else if (axis == 1) b = (lt / P) * P2 + (lt % P);
    else b = lt;
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

// as tensor_stage along x3 (axis 2) with the P x P matrix Sz (node-major) from
// shared memory: the per-element x3 eigenbasis of the C* form (eq. 5.30)
__device__ __forceinline__ void tensor_stage_z(const real *in, real *out, const real *Sz, bool transpose, int lt) {
  if (lt < P2) {
    real v[P];
#pragma unroll
    for (int k = 0; k < P; ++k) v[k] = in[lt + k * P2];
#pragma unroll
    for (int c = 0; c < P; ++c) {
      real s = 0;
#pragma unroll
      for (int k = 0; k < P; ++k) s += (transpose ? Sz[k * P + c] : Sz[c * P + k]) * v[k];
      out[lt + c * P2] = s;
    }
  }
  __syncthreads();
}

// per-thread sum of products: FP64 for double, compensated (Kahan) FP32 for float
struct DotAcc {
  real s = 0, c = 0;
  __device__ __forceinline__ void add(real a, real b) {
#if defined(HPSE_DOUBLE)
    s += a * b;
#else
    const real y = a * b - c;
    const real t = s + y;
    c = (t - s) - y;
    s = t;
#endif
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// sum of one item's warps (valid in lane 0 of the item's first warp)
__device__ __forceinline__ double item_sum(double v, double *red, int warp_in_cta, int first_warp_of_item) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[warp_in_cta] = v;
  __syncthreads();
  double t = 0.0;
  if (warp_in_cta == first_warp_of_item && (threadIdx.x & 31) == 0)
    for (int w = 0; w < PC_WARPS_PER_ITEM; ++w) t += red[first_warp_of_item + w];
  __syncthreads();
  return t;
}

template <int MODE>
__global__ void __launch_bounds__(PC_NT) k_precond(const PrecArgs A) {
  extern __shared__ __align__(16) unsigned char pc_raw[];
  const int sub = threadIdx.x / PC_TPI;  // item within the CTA (warp-uniform)
  const int lt = threadIdx.x - sub * PC_TPI;
  real *s0 = reinterpret_cast<real *>(pc_raw) + (size_t)sub * 2 * P3;
  real *s1 = s0 + P3;
  double *red = reinterpret_cast<double *>(pc_raw + PC_RED_OFF);
  real *sz = reinterpret_cast<real *>(pc_raw + PC_Z_OFF) + (size_t)sub * (P2 + P);
  const bool cstar = A.zeig != nullptr;
  __shared__ real smu[P];
  const int item = blockIdx.x * PC_ITEMS + sub;
  const bool valid = item < A.n_group * A.n_rhs;
  const int ge = valid ? item / A.n_rhs : 0;
  const int rr = valid ? item - ge * A.n_rhs : 0;
  const int e = A.elems[ge];
  const int64_t base = (int64_t)rr * A.ndof + A.dof_off[e];
  if (threadIdx.x < P) smu[threadIdx.x] = c_tab.MU[threadIdx.x];
  if (cstar)
    for (int t = lt; t < P2 + P; t += PC_TPI) sz[t] = A.zeig[(int64_t)e * hpse::ZEIG_STRIDE + t];
  DotAcc arr, arz;
  if (valid) {
    if (MODE == MODE_PCG) {
      const real al = (real)A.alpha[A.prob[e] * A.n_rhs + rr];
      for (int t = lt; t < P3; t += PC_TPI) {
        const real pv = A.p[base + t];
        if (A.x) A.x[base + t] += al * pv;
        const real rv = A.r[base + t] - al * A.q[base + t];
        A.r[base + t] = rv;
        s0[t] = rv;
        arr.add(rv, rv);
      }
    } else {
      for (int t = lt; t < P3; t += PC_TPI) s0[t] = A.rin[base + t];
    }
  }
  __syncthreads();
  tensor_stage(s0, s1, 0, true, lt);
  tensor_stage(s1, s0, 1, true, lt);
  if (cstar) tensor_stage_z(s0, s1, sz, true, lt);
  else tensor_stage(s0, s1, 2, true, lt);
  for (int t = lt; t < P3; t += PC_TPI) {
    const int a = t % P, b = (t / P) % P, c = t / P2;
    s1[t] = s1[t] / (smu[a] + smu[b] + (cstar ? sz[P2 + c] : smu[c]) + (real)1);
  }
  __syncthreads();
  if (cstar) tensor_stage_z(s1, s0, sz, false, lt);
  else tensor_stage(s1, s0, 2, false, lt);
  tensor_stage(s0, s1, 1, false, lt);
  tensor_stage(s1, s0, 0, false, lt);
  if (valid) {
    for (int t = lt; t < P3; t += PC_TPI) {
      const real zv = s0[t];
      A.zout[base + t] = zv;
      if (MODE == MODE_PCG) arz.add(zv, A.r[base + t]);
    }
  }
  if (MODE == MODE_PCG) {
    const int w = threadIdx.x >> 5, w0 = sub * PC_WARPS_PER_ITEM;
    const double a = item_sum(arr.value(), red, w, w0);
    const double b = item_sum(arz.value(), red, w, w0);
    if (valid && lt == 0) {
      A.part_rr[(int64_t)e * A.n_rhs + rr] = a;
      A.part_rz[(int64_t)e * A.n_rhs + rr] = b;
    }
  }
}

}  // namespace
