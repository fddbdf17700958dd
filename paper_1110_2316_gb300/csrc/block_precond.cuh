// Element-block preconditioner: z_e = A_ee^{-1} r_e with A_ee the diagonal
// block of the normal operator A = S^T M S of eq. (4.2) for element e (its
// volume term and its own side of every face term).  Not the thesis's
// preconditioner (Section 5.2, eq. 5.19-5.20, which is kept as the default);
// a block-Jacobi alternative on the same element blocks.
//
// Set-up (FP64): A_ee is probed column by column with the operator kernel in
// self-only mode (neighbour traces taken as zero), gathered into packed
// lower-triangular storage (row i holds columns 0..i at offset i(i+1)/2),
// factored A_ee = L L^T (right-looking Cholesky, one CTA per block) and
// X = L^{-1} is formed row by row.  The preconditioner is z = X^T (X r): two
// triangular products, kept in FP64 and rounded to FP32.  Storing the factor
// rather than A_ee^{-1} keeps the FP32 operator X~^T X~ symmetric positive
// definite whatever the rounding of X (A_ee^{-1} itself rounded to FP32 loses
// definiteness once eps32 * kappa(A_ee) approaches 1).
#pragma once

struct BjArgs {
  const int32_t *elems;    // element ids of one degree group
  int32_t n_group;         // elements in the group
  int32_t n;               // block size (W+1)^3
  int32_t n_rhs;
  int64_t ndof;            // stride between right-hand sides of a vector
  const int64_t *dof_off;  // per element
  const int64_t *blk_off;  // per element: offset of its packed block
};

// offset of (i, j), j <= i, inside one packed block (n <= 1331: fits 32 bits)
__device__ __forceinline__ int pk(int i, int j) { return i * (i + 1) / 2 + j; }

// u[c][off_e + i] = (i == j0 + c) for the group's elements, c < nc
__global__ void k_bj_probe(BjArgs A, int j0, int nc, double *u) {
  const int item = blockIdx.x;
  const int ge = item / nc, c = item - ge * nc;
  const int e = A.elems[ge];
  const int64_t base = (int64_t)c * A.ndof + A.dof_off[e];
  for (int i = threadIdx.x; i < A.n; i += blockDim.x) u[base + i] = (i == j0 + c) ? 1.0 : 0.0;
}

// column j = j0 + c of every block: rows i >= j into packed storage
__global__ void k_bj_gather(BjArgs A, int j0, int nc, const double *y, double *blk) {
  const int item = blockIdx.x;
  const int ge = item / nc, c = item - ge * nc;
  const int e = A.elems[ge], j = j0 + c;
  const int64_t base = (int64_t)c * A.ndof + A.dof_off[e];
  double *B = blk + A.blk_off[e];
  for (int i = j + threadIdx.x; i < A.n; i += blockDim.x) B[pk(i, j)] = y[base + i];
}

// in-place Cholesky A = L L^T of each packed block; fail[0] set (block index
// + 1) on a non-positive pivot, the block is then left partly factored.
// Dynamic shared memory: n doubles.
__global__ void __launch_bounds__(256) k_bj_chol(BjArgs A, double *blk, int32_t *fail) {
  extern __shared__ double colk[];
  __shared__ double s_inv;
  __shared__ int s_bad;
  const int e = A.elems[blockIdx.x], n = A.n;
  double *L = blk + A.blk_off[e];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, w = tid >> 5, nw = nt >> 5;
  if (tid == 0) s_bad = 0;
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      double d = L[pk(k, k)];
      if (!(d > 0.0) || !isfinite(d)) {
        s_bad = 1;
        d = 1.0;
      }
      d = sqrt(d);
      L[pk(k, k)] = d;
      s_inv = 1.0 / d;
    }
    __syncthreads();
    if (s_bad) break;
    for (int i = k + 1 + tid; i < n; i += nt) {
      const double v = L[pk(i, k)] * s_inv;
      L[pk(i, k)] = v;
      colk[i] = v;
    }
    __syncthreads();
    // trailing update of rows i > k, columns k < j <= i: one warp per row
    for (int i = k + 1 + w; i < n; i += nw) {
      const double li = colk[i];
      double *Li = L + pk(i, 0);
      for (int j = k + 1 + lane; j <= i; j += 32) Li[j] -= li * colk[j];
    }
    __syncthreads();
  }
  if (tid == 0 && s_bad) atomicCAS(fail, 0, blockIdx.x + 1);
}

// X = L^{-1} (packed lower), row by row: X_ii = 1 / L_ii and, for j < i,
// X_ij = -(sum_{j <= m < i} L_im X_mj) / L_ii.  Dynamic shared memory: n doubles.
__global__ void __launch_bounds__(256) k_bj_trinv(BjArgs A, const double *blk, double *xout) {
  extern __shared__ double lrow[];
  const int e = A.elems[blockIdx.x], n = A.n;
  const double *L = blk + A.blk_off[e];
  double *X = xout + A.blk_off[e];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = 0; i < n; ++i) {
    for (int m = tid; m <= i; m += nt) lrow[m] = L[pk(i, m)];
    __syncthreads();
    const double inv = 1.0 / lrow[i];
    // columns in chunks of nt; rows m of X are read in order, so at each m
    // the active threads read consecutive addresses of row m
    for (int j0 = 0; j0 <= i; j0 += nt) {
      const int j = j0 + tid;
      double s = 0.0;
      for (int m = j0; m < i; ++m)
        if (m >= j) s += lrow[m] * X[pk(m, j)];
      if (j < i) X[pk(i, j)] = -s * inv;
      else if (j == i) X[pk(i, i)] = inv;
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void k_bj_convert(const double *in, T *out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (T)in[i];
}

// out_e = X_e in_e (TRANS = false, lower) or X_e^T in_e (TRANS = true) for
// every element of the group and every right-hand side.  CTA tile: TM rows
// of one element x RT right-hand sides, k in chunks of 32; thread tile MR x MC
// with rows tr + TR m and right-hand sides tc + TC c (tr = tid % TR fastest, so
// the shared reads are conflict-free and the stores coalesced; FP32 4 x 4
// tiles instead take 4 consecutive rows / right-hand sides per thread and read
// them with one 16-byte shared load each).  The next
// chunk is fetched into registers while the current one is used.
// grid: n_group * ceil(n / TM) row tiles (row tile fastest, so the tiles of an
// element run together and share its vector segment in L2), ceil(n_rhs / RT).
template <typename T, bool TRANS, int TM, int RT, int TR, int TC>
__global__ void __launch_bounds__(TR *TC) k_bj_tri(BjArgs A, const T *X, const T *in, T *out) {
  constexpr int KC = 32, MR = TM / TR, MC = RT / TC, NT = TR * TC;
  constexpr int NA = (TM * KC + NT - 1) / NT, NB = (KC * RT + NT - 1) / NT;
  // FP32 4 x 4 thread tiles read their operands as float4: rows 4 tr + m and
  // right-hand sides 4 tc + c, rows of the tiles padded to 16 bytes
  constexpr bool VEC = sizeof(T) == 4 && MR == 4 && MC == 4;
  constexpr int PADA = VEC ? 4 : 1, PADB = VEC ? 4 : 1;
  __shared__ __align__(16) T As[KC][TM + PADA];
  __shared__ __align__(16) T Bs[KC][RT + PADB];
  const int n = A.n, nrt = (n + TM - 1) / TM;
  const int ge = blockIdx.x / nrt, rt = blockIdx.x - ge * nrt;
  const int e = A.elems[ge];
  const int i0 = rt * TM, r0 = blockIdx.y * RT;
  const T *Xe = X + A.blk_off[e];
  const int64_t vb = A.dof_off[e];
  const int tid = threadIdx.x, tr = tid % TR, tc = tid / TR;
  T acc[MR][MC];
#pragma unroll
  for (int a = 0; a < MR; ++a)
#pragma unroll
    for (int b = 0; b < MC; ++b) acc[a][b] = (T)0;
  const int kbeg = TRANS ? (i0 / KC) * KC : 0;
  const int kend = TRANS ? n : min(n, i0 + TM);
  T ra[NA], rb[NB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const int idx = tid + q * NT;
      int row, kk;
      if (!TRANS) {
        row = idx / KC;
        kk = idx - row * KC;
      } else {
        kk = idx / TM;
        row = idx - kk * TM;
      }
      const int i = i0 + row, k = k0 + kk;
      T v = (T)0;
      if (idx < TM * KC && i < n && k < n) {
        if (!TRANS) {
          if (k <= i) v = Xe[pk(i, k)];
        } else {
          if (i <= k) v = Xe[pk(k, i)];
        }
      }
      ra[q] = v;
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int idx = tid + q * NT;
      const int rr = idx / KC, kk = idx - rr * KC;
      const int k = k0 + kk, rhs = r0 + rr;
      rb[q] = (idx < KC * RT && k < n && rhs < A.n_rhs) ? in[(int64_t)rhs * A.ndof + vb + k] : (T)0;
    }
  };
  if (kbeg < kend) fetch(kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += KC) {
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const int idx = tid + q * NT;
      if (idx < TM * KC) {
        if (!TRANS) As[idx % KC][idx / KC] = ra[q];
        else As[idx / TM][idx % TM] = ra[q];
      }
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int idx = tid + q * NT;
      if (idx < KC * RT) Bs[idx % KC][idx / KC] = rb[q];
    }
    __syncthreads();
    if (k0 + KC < kend) fetch(k0 + KC);
#pragma unroll 8
    for (int kk = 0; kk < KC; ++kk) {
      T a[MR], b[MC];
      if constexpr (VEC) {
        const float4 av = *reinterpret_cast<const float4 *>(&As[kk][4 * tr]);
        const float4 bv = *reinterpret_cast<const float4 *>(&Bs[kk][4 * tc]);
        a[0] = av.x; a[1] = av.y; a[2] = av.z; a[3] = av.w;
        b[0] = bv.x; b[1] = bv.y; b[2] = bv.z; b[3] = bv.w;
      } else {
#pragma unroll
        for (int m = 0; m < MR; ++m) a[m] = As[kk][tr + TR * m];
#pragma unroll
        for (int c = 0; c < MC; ++c) b[c] = Bs[kk][tc + TC * c];
      }
#pragma unroll
      for (int m = 0; m < MR; ++m)
#pragma unroll
        for (int c = 0; c < MC; ++c) acc[m][c] += a[m] * b[c];
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < MR; ++m) {
    const int i = i0 + (VEC ? 4 * tr + m : tr + TR * m);
    if (i >= n) continue;
#pragma unroll
    for (int c = 0; c < MC; ++c) {
      const int rhs = r0 + (VEC ? 4 * tc + c : tc + TC * c);
      if (rhs < A.n_rhs) out[(int64_t)rhs * A.ndof + vb + i] = acc[m][c];
    }
  }
}

// PCG update x += alpha p, r -= alpha q on the group's blocks, partial r.r per
// (element, rhs).  grid: n_group * n_rhs.
template <typename T>
__global__ void k_bj_update(BjArgs A, const int32_t *prob, const double *alpha, T *x, T *r, const T *p, const T *q,
                            double *part_rr) {
  const int item = blockIdx.x;
  const int ge = item / A.n_rhs, rr = item - ge * A.n_rhs;
  const int e = A.elems[ge];
  const int64_t base = (int64_t)rr * A.ndof + A.dof_off[e];
  const T al = (T)alpha[prob[e] * A.n_rhs + rr];
  double s = 0.0;
  for (int t = threadIdx.x; t < A.n; t += blockDim.x) {
    if (x) x[base + t] += al * p[base + t];
    const T v = r[base + t] - al * q[base + t];
    r[base + t] = v;
    s += (double)v * (double)v;
  }
  s = block_sum_d(s);
  if (threadIdx.x == 0) part_rr[(int64_t)e * A.n_rhs + rr] = s;
}

// partial z.r per (element, rhs) on the group's blocks.  grid: n_group * n_rhs.
template <typename T>
__global__ void k_bj_dot(BjArgs A, const T *z, const T *r, double *part) {
  const int item = blockIdx.x;
  const int ge = item / A.n_rhs, rr = item - ge * A.n_rhs;
  const int e = A.elems[ge];
  const int64_t base = (int64_t)rr * A.ndof + A.dof_off[e];
  double s = 0.0;
  for (int t = threadIdx.x; t < A.n; t += blockDim.x) s += (double)z[base + t] * (double)r[base + t];
  s = block_sum_d(s);
  if (threadIdx.x == 0) part[(int64_t)e * A.n_rhs + rr] = s;
}

// Tile shapes of the two triangular products (rows x right-hand sides per
// CTA), picked per degree group and precision by timing the candidates of
// the right-hand-side count on the actual factors (bj_candidates); variants
// 2, 4 and 6 exceed 48 KB of static shared memory in FP64 and exist in FP32
// only; variant 8 is the tensor-core form (bj_tc.cuh: 128 rows x 64
// right-hand sides, 3xTF32), FP32 only, offered from 32 right-hand sides on.
constexpr int BJ_NVAR = 9;
constexpr int BJ_TC = 8;
constexpr int BJ_TILE[BJ_NVAR][2] = {{64, 64}, {128, 32}, {256, 16}, {128, 8}, {256, 8},
                                     {128, 1}, {256, 1},  {64, 1},   {128, 64}};
inline bool bj_variant_ok(int v, bool fp32) {
  return v >= 0 && v < BJ_NVAR && (fp32 || (v != 2 && v != 4 && v != 6 && v != BJ_TC));
}
inline int bj_candidates(int n_rhs, bool fp32, int *v) {
  int n = 0;
  const int all[3][4] = {{0, 1, 2, BJ_TC}, {3, 4, -1, -1}, {5, 6, 7, -1}};
  const int *c = all[n_rhs >= 32 ? 0 : (n_rhs >= 2 ? 1 : 2)];
  for (int i = 0; i < 4; ++i)
    if (c[i] >= 0 && bj_variant_ok(c[i], fp32)) v[n++] = c[i];
  return n;
}

template <typename T, int TM, int RT, int TR, int TC>
static void bj_pair(const BjArgs &a, const T *X, const T *r, T *t, T *z, cudaStream_t s) {
  dim3 g(a.n_group * ((a.n + TM - 1) / TM), (a.n_rhs + RT - 1) / RT);
  k_bj_tri<T, false, TM, RT, TR, TC><<<g, TR * TC, 0, s>>>(a, X, r, t);
  k_bj_tri<T, true, TM, RT, TR, TC><<<g, TR * TC, 0, s>>>(a, X, t, z);
}

// z = X^T (X r) for the group with tile variant v; t: scratch vector of the same layout.
template <typename T>
static cudaError_t bj_apply_group(const BjArgs &a, const T *X, const T *r, T *t, T *z, cudaStream_t s, int v) {
  if (a.n_group == 0) return cudaSuccess;
  if (v == 0) bj_pair<T, 64, 64, 16, 16>(a, X, r, t, z, s);
  else if (v == 1) bj_pair<T, 128, 32, 32, 8>(a, X, r, t, z, s);
  else if (v == 3) bj_pair<T, 128, 8, 64, 4>(a, X, r, t, z, s);
  else if (v == 5) bj_pair<T, 128, 1, 128, 1>(a, X, r, t, z, s);
  else if (v == 7) bj_pair<T, 64, 1, 64, 1>(a, X, r, t, z, s);
  else if constexpr (sizeof(T) == 4) {
    if (v == 2) bj_pair<T, 256, 16, 64, 4>(a, X, r, t, z, s);
    else if (v == 4) bj_pair<T, 256, 8, 128, 2>(a, X, r, t, z, s);
    else if (v == 6) bj_pair<T, 256, 1, 256, 1>(a, X, r, t, z, s);
    else return cudaErrorInvalidValue;
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
