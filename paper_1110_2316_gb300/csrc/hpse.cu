// hpse.cu -- host side of the C ABI declared in include/hpse.h: mesh set-up,
// data upload and right-hand side, operator / preconditioner dispatch, the
// device-resident PCG driver with FP64 iterative refinement, the H^1 error
// and the FP64 helper kernels.
//
// Method: A. Husain (2010), the least-squares functional of eq. (4.2), its
// normal equations (Section 5.3), the separable preconditioner (eq. 5.19-5.20)
// and PCG (Section 5.1, stopping rule of Section 6.1).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "hpse.h"
#include "host_math.h"
#include "registry.h"

using namespace hpse;

// ---------------------------------------------------------------------------
// kernel registry (one KernelSet per (precision, degree), filled by the
// generated instantiation units)
// ---------------------------------------------------------------------------
#define HPSE_DECL(W)                                          \
  extern "C" void hpse_register_f64_w##W(hpse::KernelSet *); \
  extern "C" void hpse_register_f32_w##W(hpse::KernelSet *);
HPSE_DECL(1)
HPSE_DECL(2)
HPSE_DECL(3)
HPSE_DECL(4)
HPSE_DECL(5)
HPSE_DECL(6)
HPSE_DECL(7)
HPSE_DECL(8)
HPSE_DECL(9)
HPSE_DECL(10)

static KernelSet g_sets[2][HPSE_MAX_W + 1];
static bool g_sets_ready = false;
static long long g_launches = 0;

static void init_registry() {
  if (g_sets_ready) return;
  typedef void (*RegFn)(KernelSet *);
  RegFn f64[HPSE_MAX_W + 1] = {nullptr, hpse_register_f64_w1, hpse_register_f64_w2, hpse_register_f64_w3,
                               hpse_register_f64_w4, hpse_register_f64_w5, hpse_register_f64_w6,
                               hpse_register_f64_w7, hpse_register_f64_w8, hpse_register_f64_w9,
                               hpse_register_f64_w10};
  RegFn f32[HPSE_MAX_W + 1] = {nullptr, hpse_register_f32_w1, hpse_register_f32_w2, hpse_register_f32_w3,
                               hpse_register_f32_w4, hpse_register_f32_w5, hpse_register_f32_w6,
                               hpse_register_f32_w7, hpse_register_f32_w8, hpse_register_f32_w9,
                               hpse_register_f32_w10};
  for (int w = 1; w <= HPSE_MAX_W; ++w) {
    f64[w](&g_sets[0][w]);
    f32[w](&g_sets[1][w]);
  }
  g_sets_ready = true;
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e__ = (call);                      \
    if (e__ != cudaSuccess) {                      \
      last_cuda_error(e__, #call, __LINE__);       \
      return HPSE_ERR_CUDA;                        \
    }                                              \
  } while (0)

static char g_last_err[512];
static int verbose() {
  static int v = -1;
  if (v < 0) {
    const char *e = getenv("HPSE_VERBOSE");
    v = (e && e[0] && e[0] != '0') ? 1 : 0;
  }
  return v;
}
static void last_cuda_error(cudaError_t e, const char *what, int line) {
  snprintf(g_last_err, sizeof(g_last_err), "%s (%s) at hpse.cu:%d", cudaGetErrorString(e), what, line);
}

// ---------------------------------------------------------------------------
// device buffers
// ---------------------------------------------------------------------------
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes) {
    o.p = nullptr;
    o.bytes = 0;
  }
  DevBuf &operator=(DevBuf &&o) noexcept {
    if (this != &o) {
      if (p) cudaFree(p);
      p = o.p;
      bytes = o.bytes;
      o.p = nullptr;
      o.bytes = 0;
    }
    return *this;
  }
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t b) {
    if (p) {
      cudaFree(p);
      p = nullptr;
    }
    bytes = b;
    if (b == 0) return cudaSuccess;
    return cudaMalloc(&p, b);
  }
  template <typename T>
  T *as() const {
    return static_cast<T *>(p);
  }
};

// copy into an existing allocation of the same size (device pointers that
// captured CUDA graphs hold stay valid), else reallocate
template <typename T>
static cudaError_t upload_reuse(DevBuf &b, const std::vector<T> &v) {
  const size_t bytes = v.size() * sizeof(T);
  if (!b.p || b.bytes != bytes) {
    cudaError_t e = b.alloc(bytes);
    if (e != cudaSuccess) return e;
  }
  if (v.empty()) return cudaSuccess;
  return cudaMemcpy(b.p, v.data(), bytes, cudaMemcpyHostToDevice);
}

template <typename T>
static cudaError_t upload(DevBuf &b, const std::vector<T> &v) {
  cudaError_t e = b.alloc(v.size() * sizeof(T));
  if (e != cudaSuccess || v.empty()) return e;
  return cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

struct Group {
  int W;
  int n;          // elements in this degree group
  DevBuf elems;   // int32 element ids
};

struct SolverWork {
  size_t n = 0;  // n_rhs * ndof
  // FP64
  DevBuf x64, r64, z64, pa64, pb64, q64, ri64;
  // FP32
  DevBuf x32, r32, z32, pa32, pb32, q32;
  // partials per (element, rhs) and PCG scalars per (problem, rhs)
  DevBuf part0, part1, part2;
  DevBuf sc;      // doubles: 8 arrays of NPR
  DevBuf flags;   // int32: active[NPR], iters[NPR], status[NPR], n_active[1]
  int *h_flags = nullptr;  // pinned host mirror
  double *h_sc = nullptr;  // pinned host mirror
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  std::map<long long, cudaGraphExec_t> graphs;
  std::map<long long, int> graph_launches;
  ~SolverWork() {
    for (auto &g : graphs) cudaGraphExecDestroy(g.second);
    if (h_flags) cudaFreeHost(h_flags);
    if (h_sc) cudaFreeHost(h_sc);
    if (st) cudaStreamDestroy(st);
    if (ev) cudaEventDestroy(ev);
  }
};

struct hpse_mesh {
  int device = 0;
  int n_elem = 0, n_problem = 0, n_rhs = 0, coef_kind = 0;
  std::vector<int> W, prob, nbr;
  std::vector<double> lo, hi;
  // outer-face conditions per (element, face): 0 Dirichlet, 1 Neumann, 2 Robin;
  // the Robin gamma per (element, face); has_nr: some face is Neumann or Robin
  std::vector<int> fbc;
  std::vector<double> fgam;
  bool has_nr = false;
  DevBuf d_fbc, d_fgam64, d_fgam32;
  // interior faces between unequal degrees (fbc code 3; box meshes): the
  // elements that have one, and the 1-D tables of k_face_mixed
  bool has_mixed = false;
  std::vector<int32_t> mixed_elems;
  DevBuf d_mixed_elems, d_mix_tab, d_mix_ptr;
  // curved elements (HPSE_COORD_CURVED): per element-face grid size and first
  // point, the Dirichlet data offsets, the 1-D tables of k_face_curved, the
  // face-point K (FP64, FP32) and w |J| of the volume points (negated)
  bool curved = false, has_geometry = false;
  std::vector<int32_t> cf_q;
  std::vector<int64_t> cf_off, bf_off;
  DevBuf d_cf_q, d_cf_off, d_bf_off, d_cur_tab, d_cur_ptr, d_cK64, d_cK32, d_cwja, d_cKv, d_cdet;
  std::vector<int64_t> dof_off, coef_off;
  int64_t ndof = 0, nquad = 0;
  std::vector<int> bface_elem, bface_fi;   // boundary faces
  std::vector<int64_t> bface_off;          // offset of each face's Q^2 points
  int64_t nface_pts = 0;
  std::vector<int> prob_ptr, prob_elems;   // CSR of elements per problem
  std::map<int, hm::DegreeTables> tabs;
  std::vector<Group> groups;
  // device mesh arrays
  // d_prob: problem of each vector item (n_elem + n_corner entries)
  DevBuf d_dof_off, d_nbr, d_geo64, d_geo32, d_prob, d_coef_off, d_prob_ptr, d_prob_elems, d_elem_W;
  DevBuf d_coef64, d_coef32;  // [nquad][4] (m, d_x, d_y, d_z) per point (COEF_SCALAR);
                              // [nquad][12] (w J, C_11 .. C_0, 0) (HPSE_COEF_GENERAL)
  DevBuf d_b;                 // FP64 right-hand side
  DevBuf d_f;                 // FP64 source at the volume points [n_rhs][nquad]
  DevBuf d_aux;               // FP64 [5][nquad]: w J, a, a_x, a_y, a_z at the volume points
  DevBuf d_tabs_ptr;          // device array of the per-degree FP64 table pointers
  DevBuf d_scr_fields, d_scr_rho;  // scratch of the residual map and its transpose
  // conforming correction (box meshes; built on first use): per element corner
  // (8) and edge (12) the shared vertex / edge, their members (CSR) and
  // Dirichlet flags, the linear blends (1 -+ x)/2 at the GLL nodes per degree
  bool conf_ready = false;
  DevBuf d_cf_vid, d_cf_vptr, d_cf_vmem, d_cf_vdir, d_cf_eid, d_cf_eptr, d_cf_emem, d_cf_edir, d_cf_lin;
  DevBuf d_cf_linptr, d_cf_w, d_cf_v;
  DevBuf d_bnorm2;            // FP64 ||b||^2 per (problem, rhs)
  std::map<int, DevBuf> d_qtab;  // per degree FP64 Q-grid tables for the face data
  bool has_data = false;
  // element-block preconditioner (hpse_setup_block_preconditioner)
  // edge neighbourhood (HPSE_COORD_EDGE): corner sets and face weights
  int coord = HPSE_COORD_CARTESIAN, n_corner = 0, apply_coef = 0;
  std::vector<int> cW, cprob;             // per corner set: degree, problem
  std::vector<int> cslot;                 // per element [2]: slot of its corner face 0 / face 4, or -1
  std::vector<int> slot_elem, slot_face;  // per slot: its element and face
  std::vector<int> slot_ptr, slot_list;   // CSR of slots per corner set
  std::vector<int> item_n;                // DOF count of each vector item (elements, then corner sets)
  DevBuf d_item_n, d_kappa64, d_kappa32, d_fw64, d_fw32, d_cslot, d_cW, d_cprob, d_slot_ptr, d_slot_list;
  DevBuf d_cinv64, d_cinv32, d_cscr64, d_cscr32;
  DevBuf d_zeig64, d_zeig32;              // C* form: per element x3 eigenbasis and eigenvalues
  DevBuf d_h1w;                           // H^1 integrand weights of neighbourhood elements [E][8][KAPPA_STRIDE]
  DevBuf d_ch1w;                          // H^1 weights of corner sets [C][2][KAPPA_STRIDE]
  int precond_kind = HPSE_PRECOND_SEPARABLE;
  bool bj_ready = false;
  DevBuf d_bj_off;            // int64 per element: offset of its packed block
  DevBuf d_bj64, d_bj32;      // X = L^{-1} per element, packed lower triangle
  DevBuf bj_t64, bj_t32;      // scratch vector X r of the preconditioner
  // degree groups whose FP32 factor products lose more than 1 % against the
  // FP64 ones (measured at set-up): their FP32 solves use the FP64 factor
  // through two conversions (bj_r64, bj_z64 scratch)
  bool bj_poor32[HPSE_MAX_W + 1] = {};
  DevBuf bj_r64, bj_z64;
  int bj_var[HPSE_MAX_W + 1][2] = {};  // tile variant of the products per degree and precision (autotuned)
  float bj_ms[HPSE_MAX_W + 1][2][9] = {};  // [BJ_NVAR]  // measured time per variant (ms; 0: not a candidate)
  DevBuf d_bjt, d_bjt_off;    // tensor-core form: FP32 tiles of X and X^T per element, their offsets
  DevBuf d_bjt_err;           // int32: set by a tensor-core product whose bounded wait expired
  int threads[2][2][HPSE_MAX_W + 1];  // [kind][prec][W]
  // one stream per degree group: per-degree launches of one operator or
  // preconditioner application run concurrently (fork/join through events,
  // parallel branches when captured in a CUDA graph)
  std::vector<cudaStream_t> gstreams;
  std::vector<cudaEvent_t> gevents;
  cudaEvent_t fork_ev = nullptr;
  ~hpse_mesh() {
    for (auto st : gstreams) cudaStreamDestroy(st);
    for (auto ev : gevents) cudaEventDestroy(ev);
    if (fork_ev) cudaEventDestroy(fork_ev);
  }
  std::unique_ptr<SolverWork> work;
};

static int default_threads(int kind, int prec, int W) {
  const int Q = 2 * W + 1;
  if (kind == 1) {
    const int P2 = (W + 1) * (W + 1);
    return std::min(256, ((P2 + 31) / 32) * 32);
  }
  const int lines = Q * Q;
  const int maxt = prec == HPSE_FP64 ? 256 : 384;
  int t = ((lines + 31) / 32) * 32;
  if (t > maxt) {
    // two passes over the z-lines
    t = (((lines + 1) / 2 + 31) / 32) * 32;
    if (t > maxt) t = maxt;
  }
  return std::max(t, 64);
}

// ---------------------------------------------------------------------------
// FP64 helper kernels (not templated on the degree)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double s) {
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// deterministic block sum (result valid in thread 0)
__device__ double block_sum_d(double v) {
  __shared__ double red[32];
  double s = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = s;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; ++i) t += red[i];
  __syncthreads();
  return t;
}

// vector items: the elements' (W+1)^3 blocks, then the corner sets' W+1 values
struct ElemVecArgs {
  int32_t n_elem, n_rhs;     // n_elem: number of items
  int64_t ndof;
  const int64_t *dof_off;
  const int32_t *item_n;     // DOF count of each item
};

#include "block_precond.cuh"
#include "curved.cuh"
#include "bj_tc.cuh"
#include "edge.cuh"
static_assert(BJ_NVAR == 9, "bj_ms holds one time per tile variant");

// per (element, rhs) block: generic vector kernels with FP64 partials
template <typename TA, typename TB>
__global__ void k_dot(ElemVecArgs A, const TA *a, const TB *b, double *part) {
  const int item = blockIdx.x;
  const int e = item / A.n_rhs, r = item - e * A.n_rhs;
  const int n = A.item_n[e];
  const int64_t base = (int64_t)r * A.ndof + A.dof_off[e];
  double s = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) s += (double)a[base + t] * (double)b[base + t];
  s = block_sum_d(s);
  if (threadIdx.x == 0) part[(int64_t)e * A.n_rhs + r] = s;
}

// r = b - q (FP64) and partial ||r||^2
__global__ void k_residual(ElemVecArgs A, const double *b, const double *q, double *r, double *part) {
  const int item = blockIdx.x;
  const int e = item / A.n_rhs, rr = item - e * A.n_rhs;
  const int n = A.item_n[e];
  const int64_t base = (int64_t)rr * A.ndof + A.dof_off[e];
  double s = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const double v = b[base + t] - q[base + t];
    r[base + t] = v;
    s += v * v;
  }
  s = block_sum_d(s);
  if (threadIdx.x == 0) part[(int64_t)e * A.n_rhs + rr] = s;
}

// out = r64 * scale[pr] converted to TO
template <typename TO>
__global__ void k_scale_copy(ElemVecArgs A, const int32_t *prob, int n_rhs, const double *r64, const double *scale,
                             TO *out) {
  const int item = blockIdx.x;
  const int e = item / A.n_rhs, rr = item - e * A.n_rhs;
  const int n = A.item_n[e];
  const int64_t base = (int64_t)rr * A.ndof + A.dof_off[e];
  const double s = scale[prob[e] * n_rhs + rr];
  for (int t = threadIdx.x; t < n; t += blockDim.x) out[base + t] = (TO)(r64[base + t] * s);
}

// x64 += d * scale[pr]
template <typename TI>
__global__ void k_add_scaled(ElemVecArgs A, const int32_t *prob, int n_rhs, const TI *d, const double *scale,
                             double *x64) {
  const int item = blockIdx.x;
  const int e = item / A.n_rhs, rr = item - e * A.n_rhs;
  const int n = A.item_n[e];
  const int64_t base = (int64_t)rr * A.ndof + A.dof_off[e];
  const double s = scale[prob[e] * n_rhs + rr];
  for (int t = threadIdx.x; t < n; t += blockDim.x) x64[base + t] += (double)d[base + t] * s;
}

// r32 = r64 * scale[pr]  (scale = 1/||r64|| of the (problem, rhs), 0 if inactive)
__global__ void k_scale_to_f32(ElemVecArgs A, const int32_t *prob, int n_rhs, const double *r64, const double *scale,
                               float *r32) {
  const int item = blockIdx.x;
  const int e = item / A.n_rhs, rr = item - e * A.n_rhs;
  const int n = A.item_n[e];
  const int64_t base = (int64_t)rr * A.ndof + A.dof_off[e];
  const double s = scale[prob[e] * n_rhs + rr];
  for (int t = threadIdx.x; t < n; t += blockDim.x) r32[base + t] = (float)(r64[base + t] * s);
}

// x64 += d32 * scale[pr]
__global__ void k_add_scaled_f32(ElemVecArgs A, const int32_t *prob, int n_rhs, const float *d32,
                                 const double *scale, double *x64) {
  const int item = blockIdx.x;
  const int e = item / A.n_rhs, rr = item - e * A.n_rhs;
  const int n = A.item_n[e];
  const int64_t base = (int64_t)rr * A.ndof + A.dof_off[e];
  const double s = scale[prob[e] * n_rhs + rr];
  for (int t = threadIdx.x; t < n; t += blockDim.x) x64[base + t] += (double)d32[base + t] * s;
}

// x += d (FP64)
__global__ void k_add64(ElemVecArgs A, const double *d, double *x) {
  const int item = blockIdx.x;
  const int e = item / A.n_rhs, rr = item - e * A.n_rhs;
  const int n = A.item_n[e];
  const int64_t base = (int64_t)rr * A.ndof + A.dof_off[e];
  for (int t = threadIdx.x; t < n; t += blockDim.x) x[base + t] += d[base + t];
}

// PCG scalars per (problem, rhs), arrays of length NPR inside one buffer
struct Scalars {
  double *rz, *bb, *rr, *alpha, *beta, *pq, *scale, *tol2;
  int32_t *active, *iters, *status, *n_active;
};

static Scalars scalars_of(SolverWork &w, int npr) {
  Scalars s;
  double *d = w.sc.as<double>();
  s.rz = d;
  s.bb = d + npr;
  s.rr = d + 2 * npr;
  s.alpha = d + 3 * npr;
  s.beta = d + 4 * npr;
  s.pq = d + 5 * npr;
  s.scale = d + 6 * npr;
  s.tol2 = d + 7 * npr;
  int32_t *f = w.flags.as<int32_t>();
  s.active = f;
  s.iters = f + npr;
  s.status = f + 2 * npr;
  s.n_active = f + 3 * npr;
  return s;
}

struct FinArgs {
  int n_rhs;
  const int32_t *prob_ptr;
  const int32_t *prob_elems;
};

// deterministic sum of per-element partials for (problem p, rhs r) = block
__device__ double fin_sum(const FinArgs &F, const double *part, int p, int r) {
  const int b = F.prob_ptr[p], e_ = F.prob_ptr[p + 1];
  double s = 0.0;
  for (int i = b + threadIdx.x; i < e_; i += blockDim.x) s += part[(int64_t)F.prob_elems[i] * F.n_rhs + r];
  return block_sum_d(s);
}

// after q = A p: alpha = rz / (p.q)
__global__ void k_fin_alpha(FinArgs F, Scalars S, const double *part_pq) {
  const int pr = blockIdx.x;
  const int p = pr / F.n_rhs, r = pr - p * F.n_rhs;
  const double pq = fin_sum(F, part_pq, p, r);
  if (threadIdx.x == 0) {
    S.pq[pr] = pq;
    double a = 0.0;
    if (S.active[pr]) {
      if (!(pq > 0.0) || !isfinite(pq)) {
        S.status[pr] = HPSE_ERR_BREAKDOWN;
        S.active[pr] = 0;
      } else {
        a = S.rz[pr] / pq;
        if (!isfinite(a)) {
          S.status[pr] = HPSE_ERR_BREAKDOWN;
          S.active[pr] = 0;
          a = 0.0;
        }
      }
    }
    S.alpha[pr] = a;
  }
}

// after the update + preconditioner: convergence test and beta
__global__ void k_fin_beta(FinArgs F, Scalars S, const double *part_rr, const double *part_rz) {
  const int pr = blockIdx.x;
  const int p = pr / F.n_rhs, r = pr - p * F.n_rhs;
  const double rr = fin_sum(F, part_rr, p, r);
  const double rz = fin_sum(F, part_rz, p, r);
  if (threadIdx.x == 0) {
    double b = 0.0;
    if (S.active[pr]) {
      S.iters[pr] += 1;
      S.rr[pr] = rr;
      if (!isfinite(rr) || !isfinite(rz)) {
        S.status[pr] = HPSE_ERR_BREAKDOWN;
        S.active[pr] = 0;
      } else if (rr <= S.tol2[pr] * S.bb[pr]) {
        S.active[pr] = 0;  // converged
      } else {
        b = rz / S.rz[pr];
        S.rz[pr] = rz;
      }
    }
    S.beta[pr] = b;
  }
}

// start of a PCG solve: rz = r.z, bb = r.r (= rr), beta = 0, active if bb > 0
__global__ void k_fin_init(FinArgs F, Scalars S, const double *part_rz, const double *part_rr, double rel_tol,
                           const double *scale_in, int unit_bb) {
  const int pr = blockIdx.x;
  const int p = pr / F.n_rhs, r = pr - p * F.n_rhs;
  const double rz = fin_sum(F, part_rz, p, r);
  const double rr = fin_sum(F, part_rr, p, r);
  if (threadIdx.x == 0) {
    S.rz[pr] = rz;
    S.bb[pr] = unit_bb ? 1.0 : rr;
    S.rr[pr] = rr;
    S.beta[pr] = 0.0;
    S.alpha[pr] = 0.0;
    S.iters[pr] = 0;
    S.tol2[pr] = rel_tol * rel_tol;
    const bool want = scale_in ? (scale_in[pr] != 0.0) : true;
    S.active[pr] = (want && rr > 0.0 && isfinite(rr)) ? 1 : 0;
    if (!isfinite(rr)) S.status[pr] = HPSE_ERR_BREAKDOWN;
  }
}

// FP64 residual refresh inside the FP32 PCG: the recursive FP32 residual is
// replaced by the true one (already in r, z); beta is rescaled so that the
// next direction is z~ + beta~ p with beta~ = (r~, z~) / (r, z)_{k-1}, or the
// direction restarts where the recursion had drifted below the true residual.
__global__ void k_fin_reliable(FinArgs F, Scalars S, const double *part_rz, const double *part_rr, const double *rel,
                               double tol) {
  const int pr = blockIdx.x;
  const int p = pr / F.n_rhs, r = pr - p * F.n_rhs;
  const double rz = fin_sum(F, part_rz, p, r);
  const double rr = fin_sum(F, part_rr, p, r);
  if (threadIdx.x == 0) {
    if (rel[pr] > tol && isfinite(rz) && rz > 0.0) {
      // the recursive residual claimed convergence and the true one refuted
      // it: the next claim must reach half of the level (the 2-norm of the
      // residual is not monotone in CG, and a claim just below the tolerance
      // can be refuted again and again)
      if (!S.active[pr] && S.status[pr] == HPSE_OK) S.tol2[pr] = fmax(0.25 * S.tol2[pr], 1e-6 * tol * tol);
      // a recursive residual that had fallen far below the true one (the
      // low-precision recursion drifted: a strong preconditioner converges it
      // within one graph replay) leaves a stale direction: restart (beta = 0)
      const bool drift = S.rz[pr] < 1e-2 * rz;
      const double b = (S.active[pr] && S.rz[pr] > 0.0 && !drift) ? S.beta[pr] * (rz / S.rz[pr]) : 0.0;
      S.beta[pr] = isfinite(b) ? b : 0.0;
      S.rz[pr] = rz;
      S.rr[pr] = rr;
      S.active[pr] = 1;
    } else {
      S.beta[pr] = 0.0;
      S.alpha[pr] = 0.0;
      S.active[pr] = 0;
    }
  }
}

__global__ void k_count_active(const int32_t *active, int npr, int32_t *n_active) {
  int c = 0;
  for (int i = threadIdx.x; i < npr; i += blockDim.x) c += active[i] ? 1 : 0;
  const double s = block_sum_d((double)c);
  if (threadIdx.x == 0) *n_active = (int32_t)s;
}

// per (problem, rhs): rel residual and the refinement scale 1/||r||
__global__ void k_fin_outer(FinArgs F, const double *part_rr, const double *bnorm2, double tol, double *rel_out,
                            double *scale, double *rnorm) {
  const int pr = blockIdx.x;
  const int p = pr / F.n_rhs, r = pr - p * F.n_rhs;
  const double rr = fin_sum(F, part_rr, p, r);
  if (threadIdx.x == 0) {
    const double bb = bnorm2[pr];
    const double rel = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    rel_out[pr] = rel;
    const bool done = !(rel > tol);
    scale[pr] = (done || !(rr > 0.0)) ? 0.0 : 1.0 / sqrt(rr);
    rnorm[pr] = (done || !(rr > 0.0)) ? 0.0 : sqrt(rr);
  }
}

__global__ void k_bnorm(FinArgs F, const double *part, double *out) {
  const int pr = blockIdx.x;
  const int p = pr / F.n_rhs, r = pr - p * F.n_rhs;
  const double s = fin_sum(F, part, p, r);
  if (threadIdx.x == 0) out[pr] = s;
}

// rho_b = -(w J a) f at the volume points; coef holds m = w J a^2 and the
// host passes wJa separately
__global__ void k_rho_b(int64_t n, const double *wja, const double *f, int64_t nquad, double *rho) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    rho[i] = -wja[i % nquad] * f[i];
}

// Dirichlet data part of b for one element and rhs (block): for each boundary
// face of e: b_face += (B0 x B0)^T W2 g + (B1 x B0)^T H D_t1 g + (B0 x B1)^T H D_t2 g
struct FaceDataArgs {
  int n_rhs;
  int64_t ndof, nface_pts;
  const int64_t *dof_off;
  const int32_t *elem_W;
  const int32_t *felem_ptr;   // CSR over elements with boundary faces: faces of e
  const int32_t *felems;      // element of each CSR row
  const int32_t *face_fi;     // face index of each boundary face (CSR order)
  const int64_t *face_off;    // point offset of each boundary face
  const double *const *qtab;  // per degree: B0, B1 (QxP), DQ, KQ (QxQ), wq (Q)
  const double *g;            // [n_rhs][nface_pts]
  double *b;
  const double *fw;           // edge neighbourhood: [E][6][10] face-norm weights, else null
  const int32_t *fbc;         // [E][6] outer-face conditions (null: all Dirichlet)
  const double *fgam;         // [E][6] Robin gamma
  const double *geo;          // [E][4] s_x, s_y, s_z, J
};

__global__ void k_face_data(FaceDataArgs A) {
  extern __shared__ double sm[];
  const int row = blockIdx.x / A.n_rhs, r = blockIdx.x % A.n_rhs;
  const int e = A.felems[row];
  const int W = A.elem_W[e], P = W + 1, Q = 2 * W + 1;
  const double *tb = A.qtab[W];
  const double *B0 = tb, *B1 = tb + Q * P, *DQ = tb + 2 * Q * P, *KQ = DQ + Q * Q, *wq = KQ + Q * Q;
  double *g = sm, *g1 = g + Q * Q, *g2 = g1 + Q * Q, *h0 = g2 + Q * Q, *h1 = h0 + Q * Q, *h2 = h1 + Q * Q;
  double *ta = h2 + Q * Q, *tb2 = ta + Q * Q, *F = tb2 + Q * Q;  // F: P x P
  const int64_t base = (int64_t)r * A.ndof + A.dof_off[e];
  for (int fi_i = A.felem_ptr[row]; fi_i < A.felem_ptr[row + 1]; ++fi_i) {
    const int fi = A.face_fi[fi_i];
    const int a = fi >> 1, side = fi & 1;
    const int64_t go = (int64_t)r * A.nface_pts + A.face_off[fi_i];
    for (int t = threadIdx.x; t < Q * Q; t += blockDim.x) g[t] = A.g[go + t];
    __syncthreads();
    const int bc = A.fbc ? A.fbc[(int64_t)e * 6 + fi] : 0;
    if (bc) {
      // Neumann / Robin face: the data h in the H^{1/2} norm (L2 included),
      // back through the transposed outward normal derivative (+ gamma u)
      for (int t = threadIdx.x; t < Q * Q; t += blockDim.x) {
        const int i = t % Q, j = t / Q;
        double k1 = 0.0, l1 = 0.0;
        for (int m = 0; m < Q; ++m) {
          k1 += KQ[i * Q + m] * g[j * Q + m];
          l1 += KQ[j * Q + m] * g[m * Q + i];
        }
        h0[t] = wq[i] * wq[j] * g[t] + wq[j] * k1 + wq[i] * l1;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < Q * P; t += blockDim.x) {
        const int p1 = t % P, j = t / P;
        double s0 = 0.0;
        for (int i = 0; i < Q; ++i) s0 += B0[i * P + p1] * h0[j * Q + i];
        ta[j * P + p1] = s0;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < P * P; t += blockDim.x) {
        const int p1 = t % P, p2 = t / P;
        double s0 = 0.0;
        for (int j = 0; j < Q; ++j) s0 += B0[j * P + p2] * ta[j * P + p1];
        F[t] = s0;
      }
      __syncthreads();
      // d/dlambda_a at the face (the endpoint row of B1) times the outward sign and s_a
      const double sn = (side ? 1.0 : -1.0) * A.geo[4 * (int64_t)e + a];
      const double gam = bc == 2 ? A.fgam[(int64_t)e * 6 + fi] : 0.0;
      const double *Dn = B1 + (side ? Q - 1 : 0) * P;
      const int nend = side ? P - 1 : 0;
      for (int t = threadIdx.x; t < P * P; t += blockDim.x) {
        const int p1 = t % P, p2 = t / P;
        for (int n = 0; n < P; ++n) {
          int idx;
          if (a == 0) idx = (p2 * P + p1) * P + n;
          else if (a == 1) idx = (p2 * P + n) * P + p1;
          else idx = (n * P + p2) * P + p1;
          A.b[base + idx] += (sn * Dn[n] + (n == nend ? gam : 0.0)) * F[t];
        }
      }
      __syncthreads();
      continue;
    }
    // tangential derivatives of the data on the face grid [t2][t1]
    for (int t = threadIdx.x; t < Q * Q; t += blockDim.x) {
      const int i = t % Q, j = t / Q;
      double s1 = 0.0, s2 = 0.0;
      for (int m = 0; m < Q; ++m) {
        s1 += DQ[i * Q + m] * g[j * Q + m];
        s2 += DQ[j * Q + m] * g[m * Q + i];
      }
      g1[t] = s1;
      g2[t] = s2;
    }
    __syncthreads();
    // h0 = (W x W) g ; h1 = H g1 ; h2 = H g2 with H = WxW + WxK + KxW
    const double *wf = A.fw ? A.fw + ((int64_t)e * 6 + fi) * hpse::FACE_W : nullptr;
    const double w0 = wf ? wf[0] : 1.0;
    const double c10 = wf ? wf[1] : 1.0, c11 = wf ? wf[2] : 1.0, c12 = wf ? wf[3] : 1.0;
    const double c20 = wf ? wf[4] : 1.0, c21 = wf ? wf[5] : 1.0, c22 = wf ? wf[6] : 1.0;
    for (int t = threadIdx.x; t < Q * Q; t += blockDim.x) {
      const int i = t % Q, j = t / Q;
      h0[t] = w0 * wq[i] * wq[j] * g[t];
      double k1 = 0.0, k2 = 0.0, l1 = 0.0, l2 = 0.0;
      for (int m = 0; m < Q; ++m) {
        k1 += KQ[i * Q + m] * g1[j * Q + m];  // K along t1
        l1 += KQ[j * Q + m] * g1[m * Q + i];  // K along t2
        k2 += KQ[i * Q + m] * g2[j * Q + m];
        l2 += KQ[j * Q + m] * g2[m * Q + i];
      }
      h1[t] = c10 * wq[i] * wq[j] * g1[t] + c11 * wq[j] * k1 + c12 * wq[i] * l1;
      h2[t] = c20 * wq[i] * wq[j] * g2[t] + c21 * wq[j] * k2 + c22 * wq[i] * l2;
    }
    __syncthreads();
    // project to nodal face values: along t1 first (ta: [t2 q][p1]), then t2
    for (int t = threadIdx.x; t < Q * P; t += blockDim.x) {
      const int p1 = t % P, j = t / P;
      double s0 = 0.0, s1 = 0.0;
      for (int i = 0; i < Q; ++i) {
        s0 += B0[i * P + p1] * h0[j * Q + i] + B1[i * P + p1] * h1[j * Q + i];
        s1 += B0[i * P + p1] * h2[j * Q + i];
      }
      ta[j * P + p1] = s0;
      tb2[j * P + p1] = s1;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < P * P; t += blockDim.x) {
      const int p1 = t % P, p2 = t / P;
      double s = 0.0;
      for (int j = 0; j < Q; ++j) s += B0[j * P + p2] * ta[j * P + p1] + B1[j * P + p2] * tb2[j * P + p1];
      F[t] = s;
    }
    __syncthreads();
    const int nend = side ? P - 1 : 0;
    for (int t = threadIdx.x; t < P * P; t += blockDim.x) {
      const int p1 = t % P, p2 = t / P;
      int idx;
      if (a == 0) idx = (p2 * P + p1) * P + nend;
      else if (a == 1) idx = (p2 * P + nend) * P + p1;
      else idx = (nend * P + p2) * P + p1;
      A.b[base + idx] += F[t];
    }
    __syncthreads();
  }
}

// H^1 norms per (element, rhs): err = sum w J [(u - v)^2 + |grad(u - v)|^2],
// nrm = sum w J [v^2 + |grad v|^2]; v a DOF vector (ref) or sampled (vq, gq).
struct H1Args {
  int n_rhs;
  int64_t ndof, nquad;
  const int64_t *dof_off, *coef_off;
  const int32_t *elem_W;
  const double *geo;  // s_x, s_y, s_z, J
  const double *const *qtab;
  const double *u, *ref, *vq, *gq;
  double *part_err, *part_nrm;
  // neighbourhood meshes (difference of two discrete solutions only): per
  // element the weights a_k(x), b_k(z) of the physical H^1 integrand and the
  // mixed-term coefficient hc; corner sets: their W and per set the weights
  // w0, w1 on its own GLL points (see setup_edge)
  const double *hw;
  double hc;
  int32_t n_elem, n_corner;
  const int32_t *cW;
  // curved elements: K (9 per volume point, K[a][i]) and |J| per point; null otherwise
  const double *cK, *cdet;
  const double *cw;
};

__device__ void h1_fields(const double *blk, int P, int Q, const double *B0, const double *B1, double *X0, double *X1,
                          double *T00, double *T01, double *T10) {
  for (int t = threadIdx.x; t < Q * P * P; t += blockDim.x) {
    const int qa = t % Q, l = t / Q;  // l = k*P + j
    double a0 = 0.0, a1 = 0.0;
    for (int i = 0; i < P; ++i) {
      a0 += B0[qa * P + i] * blk[l * P + i];
      a1 += B1[qa * P + i] * blk[l * P + i];
    }
    X0[l * Q + qa] = a0;
    X1[l * Q + qa] = a1;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < Q * Q * P; t += blockDim.x) {
    const int qa = t % Q, qb = (t / Q) % Q, k = t / (Q * Q);
    double a = 0.0, b = 0.0, c = 0.0;
    for (int j = 0; j < P; ++j) {
      const double x0 = X0[(k * P + j) * Q + qa];
      a += B0[qb * P + j] * x0;
      b += B1[qb * P + j] * x0;
      c += B0[qb * P + j] * X1[(k * P + j) * Q + qa];
    }
    T00[t] = a;
    T01[t] = b;
    T10[t] = c;
  }
  __syncthreads();
}

__global__ void k_h1(H1Args A) {
  extern __shared__ double sm[];
  const int item = blockIdx.x;
  const int e = item / A.n_rhs, r = item - e * A.n_rhs;
  const int W = A.elem_W[e], P = W + 1, Q = 2 * W + 1;
  const double *tb = A.qtab[W];
  const double *B0 = tb, *B1 = tb + Q * P, *wq = tb + 2 * Q * P + 2 * Q * Q;
  const double *geo = A.geo + (int64_t)e * 4;
  double *blk = sm, *X0 = blk + P * P * P, *X1 = X0 + Q * P * P, *T00 = X1 + Q * P * P, *T01 = T00 + Q * Q * P,
         *T10 = T01 + Q * Q * P;
  const int64_t base = (int64_t)r * A.ndof + A.dof_off[e];
  double serr = 0.0, snrm = 0.0;
  for (int pass = 0; pass < (A.ref ? 2 : 1); ++pass) {
    for (int t = threadIdx.x; t < P * P * P; t += blockDim.x)
      blk[t] = pass == 0 ? (A.ref ? A.u[base + t] - A.ref[base + t] : A.u[base + t]) : A.ref[base + t];
    __syncthreads();
    h1_fields(blk, P, Q, B0, B1, X0, X1, T00, T01, T10);
    for (int t = threadIdx.x; t < Q * Q * Q; t += blockDim.x) {
      const int qa = t % Q, qb = (t / Q) % Q, qc = t / (Q * Q);
      double u = 0.0, ux = 0.0, uy = 0.0, uz = 0.0;
      for (int k = 0; k < P; ++k) {
        const int o = (k * Q + qb) * Q + qa;
        u += B0[qc * P + k] * T00[o];
        uz += B1[qc * P + k] * T00[o];
        uy += B0[qc * P + k] * T01[o];
        ux += B0[qc * P + k] * T10[o];
      }
      double wJ = wq[qa] * wq[qb] * wq[qc] * geo[3];
      if (A.cK) {
        // curved element: the physical gradient through K, the weight w |J|
        const int64_t pi = A.coef_off[e] + t;
        const double *K = A.cK + 9 * pi;
        const double u1 = ux, u2 = uy, u3 = uz;
        ux = K[0] * u1 + K[3] * u2 + K[6] * u3;
        uy = K[1] * u1 + K[4] * u2 + K[7] * u3;
        uz = K[2] * u1 + K[5] * u2 + K[8] * u3;
        wJ = wq[qa] * wq[qb] * wq[qc] * A.cdet[pi];
      } else {
        ux *= geo[0];
        uy *= geo[1];
        uz *= geo[2];
      }
      if (A.ref) {
        double v;
        if (A.hw) {
          // neighbourhood element: the physical integrand in modified coordinates
          const int KS = hpse::KAPPA_STRIDE;
          const double *ax = A.hw + (int64_t)e * 8 * KS, *bz = ax + 4 * KS;
          const double w = uz - A.hc * ux;
          v = ax[qa] * bz[qc] * u * u + ax[KS + qa] * bz[KS + qc] * ux * ux +
              ax[2 * KS + qa] * bz[2 * KS + qc] * uy * uy + ax[3 * KS + qa] * bz[3 * KS + qc] * w * w;
        } else {
          v = u * u + ux * ux + uy * uy + uz * uz;
        }
        if (pass == 0) serr += wJ * v;
        else snrm += wJ * v;
      } else {
        const int64_t qi = (int64_t)r * A.nquad + A.coef_off[e] + t;
        const int64_t gi = (int64_t)r * 3 * A.nquad + A.coef_off[e] + t;
        const double v = A.vq[qi], gx = A.gq[gi], gy = A.gq[gi + A.nquad], gz = A.gq[gi + 2 * A.nquad];
        serr += wJ * ((u - v) * (u - v) + (ux - gx) * (ux - gx) + (uy - gy) * (uy - gy) + (uz - gz) * (uz - gz));
        snrm += wJ * (v * v + gx * gx + gy * gy + gz * gz);
      }
    }
    __syncthreads();
  }
  serr = block_sum_d(serr);
  snrm = block_sum_d(snrm);
  if (threadIdx.x == 0) {
    A.part_err[item] = serr;
    A.part_nrm[item] = snrm;
  }
}

// corner sets of the edge neighbourhood: on r < r_1 the difference is
// p(x3), so its squared H^1 norm in physical coordinates is
// int_0^{r_1} r dr x (theta span) x int (p^2 + p_x3^2) dx3, the last integral
// with the (2W+1)-point GLL rule.  grid: n_corner * n_rhs, 32 threads.
__global__ void k_h1_corner(H1Args A) {
  const int item = blockIdx.x;
  const int c = item / A.n_rhs, r = item - c * A.n_rhs;
  const int W = A.cW[c], P = W + 1, Q = 2 * W + 1;
  const int64_t base = (int64_t)r * A.ndof + A.dof_off[A.n_elem + c];
  const double *w0 = A.cw + (int64_t)c * 2 * hpse::KAPPA_STRIDE, *w1 = w0 + hpse::KAPPA_STRIDE;
  double se = 0.0, sn = 0.0;
  if (W == 0) {
    // a constant set
    if (threadIdx.x == 0) {
      const double dv = A.u[base] - A.ref[base], v = A.ref[base];
      se = w0[0] * dv * dv;
      sn = w0[0] * v * v;
    }
  } else {
    const double *tb = A.qtab[W];
    const double *B0 = tb, *B1 = tb + Q * P;
    for (int q = threadIdx.x; q < Q; q += blockDim.x) {
      double d0 = 0.0, d1 = 0.0, v0 = 0.0, v1 = 0.0;
      for (int k = 0; k < P; ++k) {
        const double dv = A.u[base + k] - A.ref[base + k];
        d0 += B0[q * P + k] * dv;
        d1 += B1[q * P + k] * dv;
        v0 += B0[q * P + k] * A.ref[base + k];
        v1 += B1[q * P + k] * A.ref[base + k];
      }
      se += w0[q] * d0 * d0 + w1[q] * d1 * d1;
      sn += w0[q] * v0 * v0 + w1[q] * v1 * v1;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    se += __shfl_xor_sync(0xffffffffu, se, o);
    sn += __shfl_xor_sync(0xffffffffu, sn, o);
  }
  if (threadIdx.x == 0) {
    A.part_err[(int64_t)(A.n_elem + c) * A.n_rhs + r] = se;
    A.part_nrm[(int64_t)(A.n_elem + c) * A.n_rhs + r] = sn;
  }
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
// The dynamic shared-memory limit of a kernel is one setting per (function,
// device), shared by every handle and host thread.  It is only ever raised,
// under a lock, so that a call for a mesh of lower degree can never lower it
// beneath what a concurrent launch for a larger mesh needs.
static cudaError_t raise_smem(const void *fn, int device, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, size_t> done;
  std::lock_guard<std::mutex> lock(mu);
  size_t &cur = done[std::make_pair(fn, device)];
  if (bytes <= cur) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

static ElemVecArgs elem_args(const hpse_mesh *m) {
  ElemVecArgs a;
  a.n_elem = m->n_elem + m->n_corner;
  a.n_rhs = m->n_rhs;
  a.ndof = m->ndof;
  a.dof_off = m->d_dof_off.as<int64_t>();
  a.item_n = m->d_item_n.as<int32_t>();
  return a;
}

static FinArgs fin_args(const hpse_mesh *m) {
  FinArgs f;
  f.n_rhs = m->n_rhs;
  f.prob_ptr = m->d_prob_ptr.as<int32_t>();
  f.prob_elems = m->d_prob_elems.as<int32_t>();
  return f;
}

static int n_items_all(const hpse_mesh *m) { return m->n_elem * m->n_rhs; }
// vector items (elements and corner sets) x right-hand sides
static int n_items_vec(const hpse_mesh *m) { return (m->n_elem + m->n_corner) * m->n_rhs; }
static int npr_of(const hpse_mesh *m) { return m->n_problem * m->n_rhs; }

template <typename T>
static ApplyArgsT<T> apply_args(const hpse_mesh *m, const Group &g, const T *u, T *y) {
  ApplyArgsT<T> a;
  memset(&a, 0, sizeof(a));
  a.u = u;
  a.y = y;
  a.elems = g.elems.as<int32_t>();
  a.n_group = g.n;
  a.n_rhs = m->n_rhs;
  a.ndof = m->ndof;
  a.dof_off = m->d_dof_off.as<int64_t>();
  a.nbr = m->d_nbr.as<int32_t>();
  a.geo = (sizeof(T) == 8) ? (const T *)m->d_geo64.p : (const T *)m->d_geo32.p;
  a.prob = m->d_prob.as<int32_t>();
  a.coef = (sizeof(T) == 8) ? (const T *)m->d_coef64.p : (const T *)m->d_coef32.p;
  a.coef_off = m->d_coef_off.as<int64_t>();
  a.nquad = m->nquad;
  a.n_elem = m->n_elem;
  if (m->coord != HPSE_COORD_CARTESIAN) {
    const bool d = sizeof(T) == 8;
    a.kappa = d ? (const T *)m->d_kappa64.p : (const T *)m->d_kappa32.p;
    a.fw = d ? (const T *)m->d_fw64.p : (const T *)m->d_fw32.p;
    a.cslot = m->d_cslot.as<int32_t>();
    a.cscr = m->n_corner ? (d ? (T *)m->d_cscr64.p : (T *)m->d_cscr32.p) : nullptr;
  }
  if (m->has_nr || m->has_mixed || m->curved) {
    a.fbc = m->d_fbc.as<int32_t>();
    a.fgam = (sizeof(T) == 8) ? (const T *)m->d_fgam64.p : (const T *)m->d_fgam32.p;
  }
  return a;
}

template <typename T>
static CornerArgsT<T> corner_args(const hpse_mesh *m) {
  CornerArgsT<T> c;
  memset(&c, 0, sizeof(c));
  const bool d = sizeof(T) == 8;
  c.n_corner = m->n_corner;
  c.n_rhs = m->n_rhs;
  c.n_elem = m->n_elem;
  c.ndof = m->ndof;
  c.dof_off = m->d_dof_off.as<int64_t>();
  c.cW = m->d_cW.as<int32_t>();
  c.cprob = m->d_cprob.as<int32_t>();
  c.slot_ptr = m->d_slot_ptr.as<int32_t>();
  c.slot_list = m->d_slot_list.as<int32_t>();
  c.cscr = d ? (const T *)m->d_cscr64.p : (const T *)m->d_cscr32.p;
  c.cinv = d ? (const T *)m->d_cinv64.p : (const T *)m->d_cinv32.p;
  return c;
}

template <typename T>
static PrecArgsT<T> prec_args(const hpse_mesh *m, const Group &g) {
  PrecArgsT<T> a;
  memset(&a, 0, sizeof(a));
  a.elems = g.elems.as<int32_t>();
  a.n_group = g.n;
  a.n_rhs = m->n_rhs;
  a.ndof = m->ndof;
  a.dof_off = m->d_dof_off.as<int64_t>();
  a.prob = m->d_prob.as<int32_t>();
  if (m->coord == HPSE_COORD_EDGE)
    a.zeig = (sizeof(T) == 8) ? (const T *)m->d_zeig64.p : (const T *)m->d_zeig32.p;
  return a;
}

// stream of degree group gi for a launch ordered after work already on s
static cudaError_t group_fork(hpse_mesh *m, cudaStream_t s) {
  if (m->groups.size() < 2) return cudaSuccess;
  cudaError_t e = cudaEventRecord(m->fork_ev, s);
  if (e != cudaSuccess) return e;
  for (cudaStream_t gs : m->gstreams)
    if ((e = cudaStreamWaitEvent(gs, m->fork_ev, 0)) != cudaSuccess) return e;
  return cudaSuccess;
}
static cudaError_t group_join(hpse_mesh *m, cudaStream_t s) {
  if (m->groups.size() < 2) return cudaSuccess;
  cudaError_t e;
  for (size_t i = 0; i < m->gstreams.size(); ++i) {
    if ((e = cudaEventRecord(m->gevents[i], m->gstreams[i])) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, m->gevents[i], 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}
static cudaStream_t group_stream(hpse_mesh *m, size_t gi, cudaStream_t s) {
  return m->groups.size() < 2 ? s : m->gstreams[gi];
}

template <typename T>
static hpse_status launch_mixed(hpse_mesh *m, int mode, const T *u, T *y, double *partial, int n_rhs, int self_only,
                                int only_W, cudaStream_t s);
template <typename T>
static hpse_status launch_curved(hpse_mesh *m, int mode, const T *u, T *y, double *partial, int n_rhs,
                                 int self_only, int only_W, cudaStream_t s);

template <typename T>
static hpse_status launch_apply_all(hpse_mesh *m, int mode, ApplyArgsT<T> base_args, cudaStream_t s) {
  const int pi = sizeof(T) == 8 ? 0 : 1;
  CK(group_fork(m, s));
  for (size_t gi = 0; gi < m->groups.size(); ++gi) {
    const Group &g = m->groups[gi];
    ApplyArgsT<T> a = base_args;
    a.elems = g.elems.as<int32_t>();
    a.n_group = g.n;
    const KernelSet &ks = g_sets[pi][g.W];
    const int th = m->threads[0][pi][g.W];
    CK(ks.apply(m->apply_coef, mode, &a, g.n * m->n_rhs, th, group_stream(m, gi, s)));
    ++g_launches;
  }
  CK(group_join(m, s));
  if (m->has_mixed && mode != MODE_TRANSPOSE && !base_args.skip_faces) {
    // faces between unequal degrees, after every element's apply (PCG mode:
    // the new search direction of every element is in pnew by then)
    const T *uu = mode == MODE_PCG ? base_args.pnew : base_args.u;
    hpse_status st = launch_mixed<T>(m, mode, uu, base_args.y, base_args.partial, base_args.n_rhs,
                                     base_args.self_only, 0, s);
    if (st != HPSE_OK) return st;
  }
  if (m->curved && mode != MODE_TRANSPOSE && !base_args.skip_faces) {
    const T *uu = mode == MODE_PCG ? base_args.pnew : base_args.u;
    hpse_status st = launch_curved<T>(m, mode, uu, base_args.y, base_args.partial, base_args.n_rhs,
                                      base_args.self_only, 0, s);
    if (st != HPSE_OK) return st;
  }
  if (m->n_corner > 0 && !base_args.self_only) {
    // corner sets: sum of their face slots (after every element's face phase)
    CornerArgsT<T> c = corner_args<T>(m);
    c.y = base_args.y;
    c.z = base_args.z;
    c.p = base_args.u;
    c.pnew = base_args.pnew;
    c.beta = base_args.beta;
    c.partial = base_args.partial;
    const int items = m->n_corner * m->n_rhs;
    if (mode == MODE_PCG) k_corner_apply<T, MODE_PCG><<<items, 32, 0, s>>>(c);
    else if (mode == MODE_TRANSPOSE) k_corner_apply<T, MODE_TRANSPOSE><<<items, 32, 0, s>>>(c);
    else k_corner_apply<T, MODE_PLAIN><<<items, 32, 0, s>>>(c);
    CK(cudaGetLastError());
    ++g_launches;
  }
  return HPSE_OK;
}

// corner sets of the edge neighbourhood: exact blocks, with the PCG update in PCG mode
template <typename T>
static hpse_status launch_corner_prec(hpse_mesh *m, int mode, const PrecArgsT<T> &b, cudaStream_t s) {
  if (m->n_corner == 0) return HPSE_OK;
  CornerArgsT<T> c = corner_args<T>(m);
  c.rin = b.rin;
  c.zout = b.zout;
  c.x = b.x;
  c.r = b.r;
  c.p = b.p;
  c.q = b.q;
  c.alpha = b.alpha;
  c.part_rr = b.part_rr;
  c.part_rz = b.part_rz;
  const int items = m->n_corner * b.n_rhs;
  if (mode == MODE_PCG) k_corner_prec<T, MODE_PCG><<<items, 32, 0, s>>>(c);
  else k_corner_prec<T, MODE_PLAIN><<<items, 32, 0, s>>>(c);
  CK(cudaGetLastError());
  ++g_launches;
  return HPSE_OK;
}

static BjArgs bj_args(const hpse_mesh *m, const Group &g, int n_rhs) {
  BjArgs a;
  a.elems = g.elems.as<int32_t>();
  a.n_group = g.n;
  a.n = (g.W + 1) * (g.W + 1) * (g.W + 1);
  a.n_rhs = n_rhs;
  a.ndof = m->ndof;
  a.dof_off = m->d_dof_off.as<int64_t>();
  a.blk_off = m->d_bj_off.as<int64_t>();
  return a;
}

// z = X^T (X r) for a group on the tensor cores (FP32, variant BJ_TC)
static hpse_status bj_tc_pair(hpse_mesh *m, const Group &g, int n_rhs, const float *r, float *t, float *z,
                              cudaStream_t s) {
  if (!m->d_bjt.p || !m->d_bjt_err.p) return HPSE_ERR_INVALID_ARG;
  BjTcArgs a;
  a.elems = g.elems.as<int32_t>();
  a.n_group = g.n;
  a.n = (g.W + 1) * (g.W + 1) * (g.W + 1);
  a.n_rhs = n_rhs;
  a.ndof = m->ndof;
  a.dof_off = m->d_dof_off.as<int64_t>();
  a.tile_off = m->d_bjt_off.as<int64_t>();
  a.err = m->d_bjt_err.as<int32_t>();
  const dim3 grid(g.n * ((a.n + BJT - 1) / BJT), (n_rhs + BJT_N - 1) / BJT_N);
  k_bj_tc<false><<<grid, BJT_THREADS, BJT_SMEM, s>>>(a, m->d_bjt.as<float>(), r, t);
  k_bj_tc<true><<<grid, BJT_THREADS, BJT_SMEM, s>>>(a, m->d_bjt.as<float>(), t, z);
  CK(cudaGetLastError());
  return HPSE_OK;
}

template <typename T>
static hpse_status bj_products(hpse_mesh *m, const Group &g, const BjArgs &a, const T *X, const T *r, T *t, T *z,
                               cudaStream_t s, int v) {
  if constexpr (sizeof(T) == 4) {
    if (v == BJ_TC) return bj_tc_pair(m, g, a.n_rhs, r, t, z, s);
  }
  CK(bj_apply_group<T>(a, X, r, t, z, s, v));
  return HPSE_OK;
}

// the group's blocks of a vector, converted (FP32 <-> FP64)
template <typename TI, typename TO>
__global__ void k_bj_cvt(BjArgs A, const TI *in, TO *out) {
  const int item = blockIdx.x;
  const int ge = item / A.n_rhs, r = item - ge * A.n_rhs;
  const int64_t base = (int64_t)r * A.ndof + A.dof_off[A.elems[ge]];
  for (int i = threadIdx.x; i < A.n; i += blockDim.x) out[base + i] = (TO)in[base + i];
}

// sums over the group's blocks of (a - b)^2 and b^2 (FP64), into acc[0..1]
__global__ void k_bj_cmp(BjArgs A, const float *a, const double *b, double *acc) {
  const int item = blockIdx.x;
  const int ge = item / A.n_rhs, r = item - ge * A.n_rhs;
  const int64_t base = (int64_t)r * A.ndof + A.dof_off[A.elems[ge]];
  double d2 = 0.0, b2 = 0.0;
  for (int i = threadIdx.x; i < A.n; i += blockDim.x) {
    const double d = (double)a[base + i] - b[base + i];
    d2 += d * d;
    b2 += b[base + i] * b[base + i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    b2 += __shfl_xor_sync(0xffffffffu, b2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc, d2);
    atomicAdd(acc + 1, b2);
  }
}

// pseudo-random test vector (FP64 and its FP32 rounding) from a hash of the index
__global__ void k_bj_testvec(int64_t n, double *v64, float *v32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t h = (uint64_t)i * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    h ^= h >> 31;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 29;
    const double v = (double)(h >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    v64[i] = v;
    v32[i] = (float)v;
  }
}

// element-block preconditioner for every degree group: PCG mode fuses the
// update x += alpha p, r -= alpha q and the partials r.r, z.r around z = X^T X r
template <typename T>
static hpse_status launch_bj_all(hpse_mesh *m, int mode, const PrecArgsT<T> &b, cudaStream_t s) {
  const T *X = sizeof(T) == 8 ? (const T *)m->d_bj64.p : (const T *)m->d_bj32.p;
  T *t = sizeof(T) == 8 ? (T *)m->bj_t64.p : (T *)m->bj_t32.p;
  if (!X || !t) return HPSE_ERR_INVALID_ARG;
  CK(group_fork(m, s));
  for (size_t gi = 0; gi < m->groups.size(); ++gi) {
    const Group &g = m->groups[gi];
    const BjArgs a = bj_args(m, g, b.n_rhs);
    cudaStream_t gs = group_stream(m, gi, s);
    const int items = g.n * b.n_rhs;
    const T *rin = mode == MODE_PCG ? b.r : b.rin;
    if (mode == MODE_PCG) {
      k_bj_update<T><<<items, 128, 0, gs>>>(a, b.prob, b.alpha, b.x, b.r, b.p, b.q, b.part_rr);
      CK(cudaGetLastError());
      g_launches += 2;
    }
    if (sizeof(T) == 4 && m->bj_poor32[g.W]) {
      // FP32 solve, FP64 factor: convert, apply, convert back
      k_bj_cvt<T, double><<<items, 128, 0, gs>>>(a, rin, m->bj_r64.as<double>());
      CK(cudaGetLastError());
      CK(bj_apply_group<double>(a, m->d_bj64.as<double>(), m->bj_r64.as<double>(), m->bj_t64.as<double>(),
                                m->bj_z64.as<double>(), gs, m->bj_var[g.W][0]));
      k_bj_cvt<double, T><<<items, 128, 0, gs>>>(a, m->bj_z64.as<double>(), b.zout);
      CK(cudaGetLastError());
      g_launches += 4;
    } else {
      hpse_status st = bj_products<T>(m, g, a, X, rin, t, b.zout, gs, m->bj_var[g.W][sizeof(T) == 8 ? 0 : 1]);
      if (st != HPSE_OK) return st;
      g_launches += 2;
    }
    if (mode == MODE_PCG) {
      k_bj_dot<T><<<items, 128, 0, gs>>>(a, b.zout, b.r, b.part_rz);
      CK(cudaGetLastError());
    }
  }
  CK(group_join(m, s));
  return launch_corner_prec<T>(m, mode, b, s);
}

template <typename T>
static hpse_status launch_prec_all(hpse_mesh *m, int mode, PrecArgsT<T> base_args, cudaStream_t s) {
  if (m->precond_kind == HPSE_PRECOND_BLOCK) return launch_bj_all<T>(m, mode, base_args, s);
  const int pi = sizeof(T) == 8 ? 0 : 1;
  CK(group_fork(m, s));
  for (size_t gi = 0; gi < m->groups.size(); ++gi) {
    const Group &g = m->groups[gi];
    PrecArgsT<T> a = base_args;
    a.elems = g.elems.as<int32_t>();
    a.n_group = g.n;
    const KernelSet &ks = g_sets[pi][g.W];
    const int th = m->threads[1][pi][g.W];
    CK(ks.precond(mode, &a, g.n * m->n_rhs, th, group_stream(m, gi, s)));
    ++g_launches;
  }
  CK(group_join(m, s));
  return launch_corner_prec<T>(m, mode, base_args, s);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" const char *hpse_status_string(hpse_status s) {
  switch (s) {
    case HPSE_OK: return "ok";
    case HPSE_ERR_INVALID_ARG: return "invalid argument";
    case HPSE_ERR_NONMATCHING_FACE: return "non-matching face";
    case HPSE_ERR_DEGREE: return "unsupported degree";
    case HPSE_ERR_BREAKDOWN: return "PCG breakdown";
    case HPSE_ERR_NO_CONVERGENCE: return "no convergence within the iteration cap";
    case HPSE_ERR_TIMEOUT: return "time limit reached";
    case HPSE_ERR_CUDA: return g_last_err[0] ? g_last_err : "CUDA error";
    case HPSE_ERR_OOM: return "out of device memory";
    case HPSE_ERR_NO_DATA: return "no data: call hpse_set_data first";
    case HPSE_ERR_CAPACITY: return "size exceeds the fixed scratch of an allocation-free entry point";
  }
  return "unknown status";
}

extern "C" int64_t hpse_kernel_launch_count(int32_t reset) {
  const long long v = g_launches;
  if (reset) g_launches = 0;
  return v;
}

// Edge neighbourhood tables (eq. 4.7, 2.34): e^{2 tau} at each element's Q
// x-points, the face-norm weights of every (element, face), and the corner
// blocks A_cc with their inverse Cholesky factors.
//
// Weights, face of axis a with tangential axes t1 < t2, half-lengths hh and
// scales s = 1/hh of the element's box in (tau, theta, x3), G = sup e^tau:
// |||.|||^2 = c0 L2 + c1 quotient(t1) + c2 quotient(t2) with
// (c0, c1, c2) = (hh_t1 hh_t2, hh_t2, hh_t1), the quotient along x3 times G,
// all of it times G on a face x3 = const.  Interior and corner faces:
// [u] in L2 times hh_t1 hh_t2 (times H = G on x3 = const), the derivative
// jumps in |||.|||, the x3 derivative times G^2.  Dirichlet faces: u - g in L2
// times hh_t1 hh_t2 and the two tangential derivatives in |||.||| (x3: times
// G^2), times s_t^2 since the kernels form lambda-derivatives there.
//
// Vertex neighbourhood (eq. 4.3; axes (phi, theta, chi)): the per-x-point
// factor is 1/sin^2 phi (on u_thetatheta); every face norm carries
// R = sup e^chi with (c0, c1, c2) = R (hh_t1 hh_t2, hh_t2, hh_t1) for all
// fields, [u] in L2 times R hh_t1 hh_t2; Dirichlet likewise, the tangential
// fields times s_t^2; a corner set is one constant, A_cc = sum_faces 4 w0.
//
// Vertex-edge neighbourhood (eq. 2.27-2.29; axes (psi, theta, zeta)): the
// per-x-point factor is e^{2 psi}; E = sup sin phi = sup (1 + e^{-2 psi})^{-1/2},
// F = sup e^zeta over the face; (c0, c1, c2) = F (hh_t1 hh_t2, hh_t2, hh_t1),
// the quotient along zeta times E, all of it times E on a face zeta = const;
// [u] in L2 times F hh_t1 hh_t2 (times G = E on zeta = const), the zeta
// derivative times E^2; Dirichlet: u - g in L2 times F hh_t1 hh_t2, the
// tangential fields times s_t^2 (zeta: times E^2).  Corner sets of both kinds.
// ---------------------------------------------------------------------------
// Interior faces between unequal degrees W and W' (box meshes).  The face
// terms of eq. (4.2) on the (2 Wf + 1)-point grid, Wf = max(W, W'), are the
// nodal Kronecker forms of degree Wf (as on equal-degree faces): both traces
// are interpolated onto the (Wf + 1)^2 face nodes (exactly: a polynomial of
// degree <= Wf), the jumps of u and of the physical gradient formed there, the
// L2 form MP x MP and the H^{1/2} form MP x MP + MP x KP + KP x MP of degree
// Wf applied, and the result taken back to the element's own nodes by the
// transposed interpolation.  One block per (element with such a face, rhs);
// its faces one after the other; y += the face terms (and, in PCG mode, the
// partial p.q += p . the face terms).  k_apply skips these faces (code 3).
// ---------------------------------------------------------------------------
struct MixArgs {
  int n_items;
  const int32_t *items;       // elements with at least one face of code 3
  int n_rhs;
  int64_t ndof;
  const int64_t *dof_off;
  const int32_t *nbr, *fbc, *elem_W;
  const double *geo;          // per element (s_x, s_y, s_z, J), FP64
  const double *const *tab;   // [W]: D (P x P, D[i][k] = l_k'(x_i)) | MP | KP
  const double *const *itp;   // [W * 11 + Wf], W < Wf: (Wf + 1) x (W + 1) interpolation
  int self_only;              // neighbour traces taken as zero (diagonal blocks)
  int only_W;                 // 0: every item; else only the elements of this degree
};

// out[r][c] (n x n, [p2][p1]) = sum_k M[c][k] in[r][k] (along p1) or
// sum_k M[r][k] in[k][c] (along p2); M of size n x m, in m-wide
template <typename T>
__device__ void mix_apply(const double *M, int n, int m, const T *in, T *out, bool along_p1, bool transpose,
                          int rows) {
  // transpose: M^T (m x n) applied, i.e. out has m columns (along p1) or m rows (along p2)
  const int oc = along_p1 ? (transpose ? m : n) : rows;
  const int orr = along_p1 ? rows : (transpose ? m : n);
  const int ic = along_p1 ? (transpose ? n : m) : rows;
  for (int t = threadIdx.x; t < orr * oc; t += blockDim.x) {
    const int r = t / oc, c = t - r * oc;
    T acc = 0;
    if (along_p1) {
      const int K = transpose ? n : m;
      for (int k = 0; k < K; ++k) acc += (T)(transpose ? M[k * m + c] : M[c * m + k]) * in[r * ic + k];
    } else {
      const int K = transpose ? n : m;
      for (int k = 0; k < K; ++k) acc += (T)(transpose ? M[k * m + r] : M[r * m + k]) * in[k * ic + c];
    }
    out[t] = acc;
  }
  __syncthreads();
}

template <typename T, int MODE>
__global__ void k_face_mixed(MixArgs A, const T *u, T *y, double *partial) {
  extern __shared__ __align__(16) unsigned char mix_raw[];
  T *sm = reinterpret_cast<T *>(mix_raw);
  const int item = blockIdx.x / A.n_rhs, r = blockIdx.x - item * A.n_rhs;
  const int e = A.items[item];
  const int We = A.elem_W[e];
  if (A.only_W && We != A.only_W) return;
  const int Pe = We + 1;
  constexpr int PM = HPSE_MAX_W + 1, PM2 = PM * PM;
  T *ue = sm;                      // own block, P_e^3
  T *ye = ue + PM * PM2;           // its face terms, P_e^3
  T *buf = ye + PM * PM2;          // 12 face arrays of PM^2
  T *Te = buf, *Ne = buf + PM2, *Tn = buf + 2 * PM2, *Nn = buf + 3 * PM2;
  T *X0 = buf + 4 * PM2, *X1 = buf + 5 * PM2, *X2 = buf + 6 * PM2, *X3 = buf + 7 * PM2;
  T *W0 = buf + 8 * PM2, *W1 = buf + 9 * PM2, *W2 = buf + 10 * PM2, *W3 = buf + 11 * PM2;
  const int64_t base = (int64_t)r * A.ndof + A.dof_off[e];
  const int Pe3 = Pe * Pe * Pe;
  for (int t = threadIdx.x; t < Pe3; t += blockDim.x) {
    ue[t] = u[base + t];
    ye[t] = 0;
  }
  __syncthreads();
  const double *se = A.geo + 4 * (int64_t)e;
  const double *De = A.tab[We];
  for (int f = 0; f < 6; ++f) {
    if (A.fbc[6 * (int64_t)e + f] != 3) continue;
    const int nb = A.nbr[6 * (int64_t)e + f];
    const int Wn = A.elem_W[nb], Pn = Wn + 1;
    const int Wf = We > Wn ? We : Wn, Pf = Wf + 1;
    const int a = f >> 1, side = f & 1;
    const int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
    const double *sn = A.geo + 4 * (int64_t)nb;
    const double *Dn = A.tab[Wn];
    const double *Df = A.tab[Wf], *MPf = Df + Pf * Pf, *KPf = MPf + Pf * Pf;
    const double *Ie = We < Wf ? A.itp[We * 11 + Wf] : nullptr;
    const double *In = Wn < Wf ? A.itp[Wn * 11 + Wf] : nullptr;
    // traces and normal derivatives (d/dlambda_a) on each side's own face nodes [p2][p1]
    const int ende = side ? Pe - 1 : 0, endn = side ? 0 : Pn - 1;
    const int64_t nbase = (int64_t)r * A.ndof + A.dof_off[nb];
    for (int t = threadIdx.x; t < Pe * Pe; t += blockDim.x) {
      const int p1 = t % Pe, p2 = t / Pe;
      T nv = 0;
      for (int k = 0; k < Pe; ++k) {
        const int i = a == 0 ? k : p1, j = a == 1 ? k : (a == 0 ? p1 : p2), kk = a == 2 ? k : p2;
        nv += (T)De[ende * Pe + k] * ue[(kk * Pe + j) * Pe + i];
      }
      const int i = a == 0 ? ende : p1, j = a == 1 ? ende : (a == 0 ? p1 : p2), kk = a == 2 ? ende : p2;
      Te[t] = ue[(kk * Pe + j) * Pe + i];
      Ne[t] = nv;
    }
    for (int t = threadIdx.x; t < Pn * Pn; t += blockDim.x) {
      T tv = 0, nv = 0;
      if (!A.self_only) {
        const int p1 = t % Pn, p2 = t / Pn;
        for (int k = 0; k < Pn; ++k) {
          const int i = a == 0 ? k : p1, j = a == 1 ? k : (a == 0 ? p1 : p2), kk = a == 2 ? k : p2;
          nv += (T)Dn[endn * Pn + k] * u[nbase + (kk * Pn + j) * Pn + i];
        }
        const int i = a == 0 ? endn : p1, j = a == 1 ? endn : (a == 0 ? p1 : p2), kk = a == 2 ? endn : p2;
        tv = u[nbase + (kk * Pn + j) * Pn + i];
      }
      Tn[t] = tv;
      Nn[t] = nv;
    }
    __syncthreads();
    // interpolate the lower-degree side onto the Pf x Pf face nodes (both directions)
    if (Ie) {
      mix_apply<T>(Ie, Pf, Pe, Te, X0, true, false, Pe);
      mix_apply<T>(Ie, Pf, Pe, X0, Te, false, false, Pf);
      mix_apply<T>(Ie, Pf, Pe, Ne, X0, true, false, Pe);
      mix_apply<T>(Ie, Pf, Pe, X0, Ne, false, false, Pf);
    }
    if (In) {
      mix_apply<T>(In, Pf, Pn, Tn, X0, true, false, Pn);
      mix_apply<T>(In, Pf, Pn, X0, Tn, false, false, Pf);
      mix_apply<T>(In, Pf, Pn, Nn, X0, true, false, Pn);
      mix_apply<T>(In, Pf, Pn, X0, Nn, false, false, Pf);
    }
    // jumps: J0 = u_e - u_n (in X0), J3 = s_a N_e - s'_a N_n (X3), and the
    // tangential ones from D_f of s T_e - s' T_n along p1 (X1) and p2 (X2)
    const int Pf2 = Pf * Pf;
    for (int t = threadIdx.x; t < Pf2; t += blockDim.x) {
      X0[t] = Te[t] - Tn[t];
      X3[t] = (T)se[a] * Ne[t] - (T)sn[a] * Nn[t];
      W1[t] = (T)se[t1] * Te[t] - (T)sn[t1] * Tn[t];
      W2[t] = (T)se[t2] * Te[t] - (T)sn[t2] * Tn[t];
    }
    __syncthreads();
    mix_apply<T>(Df, Pf, Pf, W1, X1, true, false, Pf);
    mix_apply<T>(Df, Pf, Pf, W2, X2, false, false, Pf);
    // norms: G0 = (MP x MP) J0; G_k = (MP x MP + MP x KP + KP x MP) J_k, k = 1, 2, 3
    // first factor along p1: W0 = MP J0; for k: W_k = (MP + KP) J_k kept, and
    // MP J_k (for the KP factor along p2) formed in turn
    mix_apply<T>(MPf, Pf, Pf, X0, W0, true, false, Pf);
    mix_apply<T>(MPf, Pf, Pf, W0, X0, false, false, Pf);  // X0 = G0
    T *Jk[3] = {X1, X2, X3};
    for (int k = 0; k < 3; ++k) {
      mix_apply<T>(MPf, Pf, Pf, Jk[k], W0, true, false, Pf);   // MP J along p1
      mix_apply<T>(KPf, Pf, Pf, Jk[k], W1, true, false, Pf);   // KP J along p1
      for (int t = threadIdx.x; t < Pf2; t += blockDim.x) W1[t] += W0[t];
      __syncthreads();
      mix_apply<T>(MPf, Pf, Pf, W1, W2, false, false, Pf);     // MP (MP + KP) J
      mix_apply<T>(KPf, Pf, Pf, W0, W3, false, false, Pf);     // KP MP J
      for (int t = threadIdx.x; t < Pf2; t += blockDim.x) Jk[k][t] = W2[t] + W3[t];
      __syncthreads();
    }
    // back to the own nodes: L = (I^T x I^T)[G0 + s_t1 D_f^T(p1) G1 + s_t2 D_f^T(p2) G2],
    // M = s_a (I^T x I^T) G3
    mix_apply<T>(Df, Pf, Pf, X1, W1, true, true, Pf);
    mix_apply<T>(Df, Pf, Pf, X2, W2, false, true, Pf);
    for (int t = threadIdx.x; t < Pf2; t += blockDim.x) {
      X0[t] += (T)se[t1] * W1[t] + (T)se[t2] * W2[t];
      X3[t] *= (T)se[a];
    }
    __syncthreads();
    if (Ie) {
      mix_apply<T>(Ie, Pf, Pe, X0, W0, true, true, Pf);   // Pf rows x Pe columns
      mix_apply<T>(Ie, Pf, Pe, W0, X0, false, true, Pe);  // Pe x Pe
      mix_apply<T>(Ie, Pf, Pe, X3, W0, true, true, Pf);
      mix_apply<T>(Ie, Pf, Pe, W0, X3, false, true, Pe);
    }
    // gather: the face layer takes L, every node of a normal line D_e[end][k] M
    for (int t = threadIdx.x; t < Pe3; t += blockDim.x) {
      const int i = t % Pe, j = (t / Pe) % Pe, kk = t / (Pe * Pe);
      const int n = a == 0 ? i : (a == 1 ? j : kk);
      const int p1 = a == 0 ? j : i, p2 = a == 2 ? j : kk;
      const int sp = p2 * Pe + p1;
      T acc = (T)De[ende * Pe + n] * X3[sp];
      if (n == ende) acc += X0[sp];
      ye[t] += acc;
    }
    __syncthreads();
  }
  double part = 0.0;
  for (int t = threadIdx.x; t < Pe3; t += blockDim.x) {
    y[base + t] += ye[t];
    if (MODE == MODE_PCG) part += (double)ye[t] * (double)ue[t];
  }
  if (MODE == MODE_PCG) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
      partial[(int64_t)e * A.n_rhs + r] += tot;
    }
  }
}

static size_t mix_smem(size_t real_bytes) {
  const size_t PM = HPSE_MAX_W + 1;
  return (2 * PM * PM * PM + 12 * PM * PM) * real_bytes;
}

static hpse_status setup_mixed(hpse_mesh *m) {
  m->mixed_elems.clear();
  for (int e = 0; e < m->n_elem; ++e)
    for (int f = 0; f < 6; ++f)
      if (m->fbc[6 * e + f] == 3) {
        m->mixed_elems.push_back(e);
        break;
      }
  // tables: per degree present D | MP | KP, per pair W < Wf the interpolation
  std::vector<double> tab;
  std::vector<int64_t> toff(HPSE_MAX_W + 1, -1), ioff((HPSE_MAX_W + 1) * 11, -1);
  for (auto &kv : m->tabs) {
    const hm::DegreeTables &t = kv.second;
    toff[kv.first] = (int64_t)tab.size();
    tab.insert(tab.end(), t.D.begin(), t.D.end());
    tab.insert(tab.end(), t.MP.begin(), t.MP.end());
    tab.insert(tab.end(), t.KP.begin(), t.KP.end());
  }
  for (auto &lo : m->tabs)
    for (auto &hi : m->tabs)
      if (lo.first < hi.first) {
        const std::vector<double> I = hm::interp_matrix(lo.second.xp, hi.second.xp);
        ioff[lo.first * 11 + hi.first] = (int64_t)tab.size();
        tab.insert(tab.end(), I.begin(), I.end());
      }
  CK(upload(m->d_mix_tab, tab));
  std::vector<const double *> ptr((HPSE_MAX_W + 1) + (HPSE_MAX_W + 1) * 11, nullptr);
  const double *b = m->d_mix_tab.as<double>();
  for (int w = 0; w <= HPSE_MAX_W; ++w)
    if (toff[w] >= 0) ptr[w] = b + toff[w];
  for (int k = 0; k < (HPSE_MAX_W + 1) * 11; ++k)
    if (ioff[k] >= 0) ptr[HPSE_MAX_W + 1 + k] = b + ioff[k];
  CK(upload(m->d_mix_ptr, ptr));
  CK(upload(m->d_mixed_elems, m->mixed_elems));
  CK(raise_smem((const void *)k_face_mixed<double, MODE_PLAIN>, m->device, mix_smem(8)));
  CK(raise_smem((const void *)k_face_mixed<double, MODE_PCG>, m->device, mix_smem(8)));
  CK(raise_smem((const void *)k_face_mixed<float, MODE_PLAIN>, m->device, mix_smem(4)));
  CK(raise_smem((const void *)k_face_mixed<float, MODE_PCG>, m->device, mix_smem(4)));
  return HPSE_OK;
}

static MixArgs mix_args(const hpse_mesh *m, int n_rhs) {
  MixArgs A;
  memset(&A, 0, sizeof(A));
  A.n_items = (int)m->mixed_elems.size();
  A.items = m->d_mixed_elems.as<int32_t>();
  A.n_rhs = n_rhs;
  A.ndof = m->ndof;
  A.dof_off = m->d_dof_off.as<int64_t>();
  A.nbr = m->d_nbr.as<int32_t>();
  A.fbc = m->d_fbc.as<int32_t>();
  A.elem_W = m->d_elem_W.as<int32_t>();
  A.geo = m->d_geo64.as<double>();
  A.tab = m->d_mix_ptr.as<const double *>();
  A.itp = m->d_mix_ptr.as<const double *>() + (HPSE_MAX_W + 1);
  return A;
}

template <typename T>
static hpse_status launch_mixed(hpse_mesh *m, int mode, const T *u, T *y, double *partial, int n_rhs, int self_only,
                                int only_W, cudaStream_t s) {
  if (!m->has_mixed || m->mixed_elems.empty()) return HPSE_OK;
  MixArgs A = mix_args(m, n_rhs);
  A.self_only = self_only;
  A.only_W = only_W;
  const int grid = A.n_items * n_rhs;
  if (mode == MODE_PCG)
    k_face_mixed<T, MODE_PCG><<<grid, 128, mix_smem(sizeof(T)), s>>>(A, u, y, partial);
  else
    k_face_mixed<T, MODE_PLAIN><<<grid, 128, mix_smem(sizeof(T)), s>>>(A, u, y, partial);
  CK(cudaGetLastError());
  ++g_launches;
  return HPSE_OK;
}

// curved elements: the element-face grids (Qf = 2 max(W, W') + 1 on interior
// faces, 2 W + 1 on Dirichlet faces), the Dirichlet data offsets (the
// boundary faces in element, face order: those of hpse_nface_points), the
// 1-D tables of k_face_curved
static hpse_status setup_curved(hpse_mesh *m) {
  const int E = m->n_elem;
  m->cf_q.assign(6 * (size_t)E, 0);
  m->cf_off.assign(6 * (size_t)E + 1, 0);
  m->bf_off.assign(6 * (size_t)E, -1);
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      const int n = m->nbr[6 * e + f];
      const int Wf = n >= 0 ? std::max(m->W[e], m->W[n]) : m->W[e];
      m->cf_q[6 * e + f] = 2 * Wf + 1;
      m->cf_off[6 * e + f + 1] = m->cf_off[6 * e + f] + (int64_t)(2 * Wf + 1) * (2 * Wf + 1);
    }
  for (size_t i = 0; i < m->bface_elem.size(); ++i) m->bf_off[6 * m->bface_elem[i] + m->bface_fi[i]] = m->bface_off[i];
  // tables: D per degree; B0 | B1 (Qf x P) per (degree, grid); w | K1 | DQ per grid
  std::vector<double> tab;
  std::map<int, int64_t> doff, qoff;
  std::map<std::pair<int, int>, int64_t> boff;
  for (auto &kv : m->tabs) {
    doff[kv.first] = (int64_t)tab.size();
    tab.insert(tab.end(), kv.second.D.begin(), kv.second.D.end());
  }
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      const int Qf = m->cf_q[6 * e + f];
      if (!qoff.count(Qf)) {
        std::vector<double> x, w;
        hm::gll_rule(Qf, x, w);
        const std::vector<double> K1 = hm::half_norm_matrix(x, w), DQ = hm::diff_matrix(x);
        qoff[Qf] = (int64_t)tab.size();
        tab.insert(tab.end(), w.begin(), w.end());
        tab.insert(tab.end(), K1.begin(), K1.end());
        tab.insert(tab.end(), DQ.begin(), DQ.end());
      }
      // every degree meeting this grid: the element's and its neighbour's
      const int n = m->nbr[6 * e + f];
      for (int W : {m->W[e], n >= 0 ? m->W[n] : m->W[e]}) {
        if (boff.count({W, Qf})) continue;
        std::vector<double> x, w;
        hm::gll_rule(Qf, x, w);
        const hm::DegreeTables &t = m->tabs.at(W);
        const std::vector<double> B0 = hm::interp_matrix(t.xp, x);
        const std::vector<double> B1 = hm::matmul(B0, t.D, Qf, W + 1, W + 1);
        boff[{W, Qf}] = (int64_t)tab.size();
        tab.insert(tab.end(), B0.begin(), B0.end());
        tab.insert(tab.end(), B1.begin(), B1.end());
      }
    }
  CK(upload(m->d_cur_tab, tab));
  const double *b = m->d_cur_tab.as<double>();
  // pointer table: [W] D, then [W * 22 + Qf] B0 | B1, then [Qf] w | K1 | DQ
  std::vector<const double *> ptr((HPSE_MAX_W + 1) + (HPSE_MAX_W + 1) * 22 + 22, nullptr);
  for (auto &kv : doff) ptr[kv.first] = b + kv.second;
  for (auto &kv : boff) ptr[(HPSE_MAX_W + 1) + kv.first.first * 22 + kv.first.second] = b + kv.second;
  for (auto &kv : qoff) ptr[(HPSE_MAX_W + 1) + (HPSE_MAX_W + 1) * 22 + kv.first] = b + kv.second;
  CK(upload(m->d_cur_ptr, ptr));
  CK(upload(m->d_cf_q, m->cf_q));
  CK(upload(m->d_cf_off, m->cf_off));
  CK(upload(m->d_bf_off, m->bf_off));
  const size_t sm64 = curved::face_smem(8), sm32 = curved::face_smem(4);
  CK(raise_smem((const void *)curved::k_face_curved<double, 0, false>, m->device, sm64));
  CK(raise_smem((const void *)curved::k_face_curved<double, 1, false>, m->device, sm64));
  CK(raise_smem((const void *)curved::k_face_curved<double, 0, true>, m->device, sm64));
  CK(raise_smem((const void *)curved::k_face_curved<float, 0, false>, m->device, sm32));
  CK(raise_smem((const void *)curved::k_face_curved<float, 1, false>, m->device, sm32));
  return HPSE_OK;
}

static curved::FaceArgs curved_args(const hpse_mesh *m, int n_rhs) {
  curved::FaceArgs A;
  memset(&A, 0, sizeof(A));
  A.n_rhs = n_rhs;
  A.ndof = m->ndof;
  A.dof_off = m->d_dof_off.as<int64_t>();
  A.nbr = m->d_nbr.as<int32_t>();
  A.elem_W = m->d_elem_W.as<int32_t>();
  A.cf_off = m->d_cf_off.as<int64_t>();
  A.cf_q = m->d_cf_q.as<int32_t>();
  const double *const *p = m->d_cur_ptr.as<const double *>();
  A.dtab = p;
  A.btab = p + (HPSE_MAX_W + 1);
  A.qtab = p + (HPSE_MAX_W + 1) + (HPSE_MAX_W + 1) * 22;
  A.bf_off = m->d_bf_off.as<int64_t>();
  A.nface_pts = m->nface_pts;
  return A;
}

// the face terms of curved elements (y +=; PCG mode: partial +=)
template <typename T>
static hpse_status launch_curved(hpse_mesh *m, int mode, const T *u, T *y, double *partial, int n_rhs,
                                 int self_only, int only_W, cudaStream_t s) {
  if (!m->curved || m->n_elem == 0) return HPSE_OK;
  curved::FaceArgs A = curved_args(m, n_rhs);
  A.self_only = self_only;
  A.only_W = only_W;
  const T *K = sizeof(T) == 8 ? (const T *)m->d_cK64.p : (const T *)m->d_cK32.p;
  const int grid = m->n_elem * n_rhs;
  const size_t sm = curved::face_smem(sizeof(T));
  if (mode == MODE_PCG)
    curved::k_face_curved<T, 1, false><<<grid, 128, sm, s>>>(A, u, K, nullptr, y, partial);
  else
    curved::k_face_curved<T, 0, false><<<grid, 128, sm, s>>>(A, u, K, nullptr, y, partial);
  CK(cudaGetLastError());
  ++g_launches;
  return HPSE_OK;
}

static hpse_status setup_edge(hpse_mesh *m) {
  const int E = m->n_elem, C = m->n_corner;
  const bool vtx = m->coord == HPSE_COORD_VERTEX;
  const bool ve = m->coord == HPSE_COORD_VERTEX_EDGE;
  std::vector<double> kap((size_t)E * hpse::KAPPA_STRIDE, 0.0), fw((size_t)E * 6 * hpse::FACE_W, 0.0);
  for (int e = 0; e < E; ++e) {
    const hm::DegreeTables &t = m->tabs.at(m->W[e]);
    double hh[3], sc[3];
    for (int a = 0; a < 3; ++a) {
      hh[a] = 0.5 * (m->hi[3 * e + a] - m->lo[3 * e + a]);
      sc[a] = 1.0 / hh[a];
    }
    for (int q = 0; q < t.Q; ++q) {
      const double x = m->lo[3 * e] + (t.xq[q] + 1.0) * hh[0];
      kap[(size_t)e * hpse::KAPPA_STRIDE + q] = vtx ? 1.0 / (std::sin(x) * std::sin(x)) : std::exp(2.0 * x);
    }
    for (int fi = 0; fi < 6; ++fi) {
      const int a = fi >> 1, side = fi & 1;
      const int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
      if (ve) {
        const double psi = (a == 0 && !side) ? m->lo[3 * e] : m->hi[3 * e];
        const double zet = (a == 2 && !side) ? m->lo[3 * e + 2] : m->hi[3 * e + 2];
        const double Es = 1.0 / std::sqrt(1.0 + std::exp(-2.0 * psi)), F = std::exp(zet);
        double c[3] = {F * hh[t1] * hh[t2], F * hh[t2], F * hh[t1]};
        if (t2 == 2) c[2] *= Es;
        if (a == 2)
          for (double &v : c) v *= Es;
        double *w = &fw[((size_t)e * 6 + fi) * hpse::FACE_W];
        const bool dir = m->nbr[6 * e + fi] == -1;
        w[0] = F * (a == 2 && !dir ? Es : 1.0) * hh[t1] * hh[t2];
        const int ax[3] = {t1, t2, a};
        for (int k = 0; k < 3; ++k) {
          double f = ax[k] == 2 ? Es * Es : 1.0;
          if (dir) f *= (k < 2) ? sc[ax[k]] * sc[ax[k]] : 0.0;
          for (int j = 0; j < 3; ++j) w[1 + 3 * k + j] = f * c[j];
        }
        continue;
      }
      if (vtx) {
        const double R = std::exp(a == 2 ? (side ? m->hi[3 * e + 2] : m->lo[3 * e + 2]) : m->hi[3 * e + 2]);
        const double c[3] = {R * hh[t1] * hh[t2], R * hh[t2], R * hh[t1]};
        double *w = &fw[((size_t)e * 6 + fi) * hpse::FACE_W];
        const bool dir = m->nbr[6 * e + fi] == -1;
        w[0] = c[0];
        const int ax[3] = {t1, t2, a};
        for (int k = 0; k < 3; ++k) {
          const double f = dir ? ((k < 2) ? sc[ax[k]] * sc[ax[k]] : 0.0) : 1.0;
          for (int j = 0; j < 3; ++j) w[1 + 3 * k + j] = f * c[j];
        }
        continue;
      }
      const double G = std::exp(a == 0 ? (side ? m->hi[3 * e] : m->lo[3 * e]) : m->hi[3 * e]);
      double c[3] = {hh[t1] * hh[t2], hh[t2], hh[t1]};
      if (t2 == 2) c[2] *= G;
      if (a == 2)
        for (double &v : c) v *= G;
      double *w = &fw[((size_t)e * 6 + fi) * hpse::FACE_W];
      const bool dir = m->nbr[6 * e + fi] == -1;
      w[0] = (dir || a != 2 ? 1.0 : G) * hh[t1] * hh[t2];
      // fields 1, 2, 3: derivative along t1, t2, the normal a
      const int ax[3] = {t1, t2, a};
      for (int k = 0; k < 3; ++k) {
        double f = ax[k] == 2 ? G * G : 1.0;
        if (dir) f *= (k < 2) ? sc[ax[k]] * sc[ax[k]] : 0.0;
        for (int j = 0; j < 3; ++j) w[1 + 3 * k + j] = f * c[j];
      }
    }
  }
  // C* form (eq. 5.29-5.30) of every element: in x3 the 1-D forms
  // G = eta^4 D2^T Wp D2 + eta^2 D^T Wp D and H = Wp with eta = sup e^tau over
  // the element; (G - nu H) d = 0 in the symmetric form Wp^{-1/2} G Wp^{-1/2},
  // stored like the master tables (node-major eigenvectors, then nu)
  std::vector<double> zeig((size_t)E * hpse::ZEIG_STRIDE, 0.0);
  for (int e = 0; e < E && m->coord == HPSE_COORD_EDGE; ++e) {
    const hm::DegreeTables &t = m->tabs.at(m->W[e]);
    const int P = t.P;
    const double eta = std::exp(m->hi[3 * e]), e2 = eta * eta, e4 = e2 * e2;
    const std::vector<double> D2 = hm::matmul(t.D, t.D, P, P, P);
    std::vector<double> G((size_t)P * P, 0.0), V, nu;
    for (int i = 0; i < P; ++i)
      for (int j = 0; j < P; ++j) {
        double v = 0.0;
        for (int k = 0; k < P; ++k) v += t.wp[k] * (e4 * D2[k * P + i] * D2[k * P + j] + e2 * t.D[k * P + i] * t.D[k * P + j]);
        G[i * P + j] = v / std::sqrt(t.wp[i] * t.wp[j]);
      }
    hm::jacobi_eigen(G, P, nu, V);
    double *z = &zeig[(size_t)e * hpse::ZEIG_STRIDE];
    for (int k = 0; k < P; ++k)
      for (int c = 0; c < P; ++c) z[k * P + c] = V[k * P + c] / std::sqrt(t.wp[k]);
    for (int c = 0; c < P; ++c) z[P * P + c] = nu[c] < 0 ? 0.0 : nu[c];
  }
  std::vector<float> zeig32(zeig.begin(), zeig.end());
  CK(upload(m->d_zeig64, zeig));
  CK(upload(m->d_zeig32, zeig32));
  std::vector<float> kap32(kap.begin(), kap.end()), fw32(fw.begin(), fw.end());
  CK(upload(m->d_kappa64, kap));
  CK(upload(m->d_kappa32, kap32));
  CK(upload(m->d_fw64, fw));
  CK(upload(m->d_fw32, fw32));
  CK(upload(m->d_cslot, m->cslot));
  if (C == 0) return HPSE_OK;
  // corner blocks.  A constant (degree 0, through face 4): its trace is 1 on
  // the face and its derivatives vanish, A_cc = sum_faces 4 w0.  A polynomial
  // along z (through face 0; nodal face grid p2 = z, p1 = y): the trace is p
  // replicated along p1 and its z derivative s_z D p; with 1^T MP 1 = 2 and
  // 1^T KP 1 = 0, A_cc = sum_faces 2 (w0 MP + s_z^2 D^T (w4 MP + w6 KP) D)
  const int S = (int)m->slot_list.size();
  std::vector<double> cinv((size_t)C * hpse::CSCR_STRIDE * hpse::CSCR_STRIDE, 0.0);
  for (int c = 0; c < C; ++c) {
    if (m->cW[c] != 0) continue;
    double a = 0.0;
    for (int i = m->slot_ptr[c]; i < m->slot_ptr[c + 1]; ++i)
      a += 4.0 * fw[((size_t)m->slot_elem[m->slot_list[i]] * 6 + 4) * hpse::FACE_W];
    if (!(a > 0.0)) return HPSE_ERR_BREAKDOWN;
    cinv[(size_t)c * hpse::CSCR_STRIDE * hpse::CSCR_STRIDE] = 1.0 / std::sqrt(a);
  }
  for (int c = 0; c < C; ++c) {
    if (m->cW[c] == 0) continue;
    const hm::DegreeTables &t = m->tabs.at(m->cW[c]);
    const int P = t.P;
    std::vector<double> Acc((size_t)P * P, 0.0);
    if (m->slot_ptr[c] == m->slot_ptr[c + 1]) return HPSE_ERR_BREAKDOWN;
    for (int i = m->slot_ptr[c]; i < m->slot_ptr[c + 1]; ++i) {
      const int e = m->slot_elem[m->slot_list[i]];
      const double *w = &fw[((size_t)e * 6 + 0) * hpse::FACE_W];
      const double sz = 2.0 / (m->hi[3 * e + 2] - m->lo[3 * e + 2]);
      // M = w4 MP + w6 KP (the x3-derivative field, quotient along x3 = t2)
      std::vector<double> M((size_t)P * P), DM((size_t)P * P, 0.0);
      for (int k = 0; k < P * P; ++k) M[k] = w[4] * t.MP[k] + w[6] * t.KP[k];
      for (int i2 = 0; i2 < P; ++i2)
        for (int j2 = 0; j2 < P; ++j2) {
          double v = 0.0;
          for (int k = 0; k < P; ++k) v += M[i2 * P + k] * t.D[k * P + j2];
          DM[i2 * P + j2] = v;
        }
      for (int i2 = 0; i2 < P; ++i2)
        for (int j2 = 0; j2 < P; ++j2) {
          double v = 0.0;
          for (int k = 0; k < P; ++k) v += t.D[k * P + i2] * DM[k * P + j2];
          Acc[i2 * P + j2] += 2.0 * (w[0] * t.MP[i2 * P + j2] + sz * sz * v);
        }
    }
    // Cholesky A_cc = L L^T, then X = L^{-1}
    std::vector<double> L(Acc);
    for (int k = 0; k < P; ++k) {
      double d = L[k * P + k];
      for (int j = 0; j < k; ++j) d -= L[k * P + j] * L[k * P + j];
      if (!(d > 0.0)) return HPSE_ERR_BREAKDOWN;
      d = std::sqrt(d);
      L[k * P + k] = d;
      for (int i2 = k + 1; i2 < P; ++i2) {
        double v = L[i2 * P + k];
        for (int j = 0; j < k; ++j) v -= L[i2 * P + j] * L[k * P + j];
        L[i2 * P + k] = v / d;
      }
    }
    double *X = &cinv[(size_t)c * hpse::CSCR_STRIDE * hpse::CSCR_STRIDE];
    for (int i2 = 0; i2 < P; ++i2) {
      X[i2 * hpse::CSCR_STRIDE + i2] = 1.0 / L[i2 * P + i2];
      for (int j = 0; j < i2; ++j) {
        double v = 0.0;
        for (int k = j; k < i2; ++k) v += L[i2 * P + k] * X[k * hpse::CSCR_STRIDE + j];
        X[i2 * hpse::CSCR_STRIDE + j] = -v / L[i2 * P + i2];
      }
    }
  }
  std::vector<float> cinv32(cinv.begin(), cinv.end());
  CK(upload(m->d_cinv64, cinv));
  CK(upload(m->d_cinv32, cinv32));
  CK(upload(m->d_cW, m->cW));
  CK(upload(m->d_cprob, m->cprob));
  CK(upload(m->d_slot_ptr, m->slot_ptr));
  CK(upload(m->d_slot_list, m->slot_list));
  // H^1 norm in physical coordinates (Section 6.1) of the difference of two
  // discrete solutions.  Elements: the integrand in modified coordinates is
  //   a0(x) b0(z) u^2 + a1 b1 u_x^2 + a2 b2 u_y^2 + a3 b3 (u_z - c u_x)^2
  // with the element's (2W+1)-point GLL rule (x = first, z = third variable):
  //   edge (tau, theta, x3):      e^{2tau} u^2 + u_tau^2 + u_theta^2 + e^{2tau} u_x3^2
  //   vertex (phi, theta, chi):   sin(phi) e^{3chi} u^2 + sin(phi) e^chi u_phi^2
  //                               + e^chi / sin(phi) u_theta^2 + sin(phi) e^chi u_chi^2
  //   vertex-edge (psi, th, zeta): e^{2psi+3zeta} u^2 + e^zeta (u_psi^2 + u_theta^2)
  //                               + e^{2psi+zeta} (u_zeta - u_psi)^2
  // (dx = e^{2tau} dtau dtheta dx3, e^{3chi} sin(phi) dchi dphi dtheta,
  // e^{2psi+3zeta} dpsi dtheta dzeta).  Corner sets, integrated exactly in r
  // or rho: per point of the set's own GLL rule weights w0 (on p^2) and w1
  // (on (dp/dlambda)^2), a constant set one weight w0:
  //   edge p(x3) on r < r1: (r1^2/2) theta-span (h/2) w_q and the same times s_x3^2
  //   vertex-edge p(zeta) on psi < psi1: (e^{2psi1}/2) theta-span (h/2) w_q e^{3zeta_q},
  //                       and (e^{2psi1}/2) theta-span (h/2) w_q e^{zeta_q} s_zeta^2
  //   vertex constant on rho < rho1: rho1^3/3 sum (cos phi_lo - cos phi_hi) theta-span
  //   vertex-edge constant on x3 < x3_1 in the cone psi < psi_top, per theta
  //                       sector: theta-span (e^{2 psi_top}/2) x3_1^3/3
  {
    const int KS = hpse::KAPPA_STRIDE;
    std::vector<double> hw((size_t)E * 8 * KS, 0.0), cw((size_t)std::max(C, 1) * 2 * KS, 0.0);
    for (int e = 0; e < E; ++e) {
      const hm::DegreeTables &t = m->tabs.at(m->W[e]);
      double *ax = &hw[(size_t)e * 8 * KS], *bz = ax + 4 * KS;
      for (int q = 0; q < t.Q; ++q) {
        const double x = m->lo[3 * e] + (t.xq[q] + 1.0) * 0.5 * (m->hi[3 * e] - m->lo[3 * e]);
        const double z = m->lo[3 * e + 2] + (t.xq[q] + 1.0) * 0.5 * (m->hi[3 * e + 2] - m->lo[3 * e + 2]);
        double a[4], b[4];
        if (vtx) {
          const double sp = std::sin(x), ez = std::exp(z);
          a[0] = sp, a[1] = sp, a[2] = 1.0 / sp, a[3] = sp;
          b[0] = ez * ez * ez, b[1] = ez, b[2] = ez, b[3] = ez;
        } else if (ve) {
          const double e2x = std::exp(2.0 * x), ez = std::exp(z);
          a[0] = e2x, a[1] = 1.0, a[2] = 1.0, a[3] = e2x;
          b[0] = ez * ez * ez, b[1] = ez, b[2] = ez, b[3] = ez;
        } else {
          const double e2x = std::exp(2.0 * x);
          a[0] = e2x, a[1] = 1.0, a[2] = 1.0, a[3] = e2x;
          b[0] = b[1] = b[2] = b[3] = 1.0;
        }
        for (int k = 0; k < 4; ++k) {
          ax[k * KS + q] = a[k];
          bz[k * KS + q] = b[k];
        }
      }
    }
    std::vector<double> ptop((size_t)std::max(C, 1) * E, -1e300);  // vertex-edge cones: psi_top per (set, sector)
    for (int e = 0; e < E; ++e) {
      for (int f : {0, 4}) {
        if (m->nbr[6 * e + f] >= -1) continue;
        const int c = -2 - m->nbr[6 * e + f];
        const double th = m->hi[3 * e + 1] - m->lo[3 * e + 1];
        double *w0 = &cw[(size_t)c * 2 * KS], *w1 = w0 + KS;
        if (m->cW[c] > 0) {
          // a polynomial along the third variable (edge: x3, vertex-edge: zeta)
          const hm::DegreeTables &t = m->tabs.at(m->cW[c]);
          const double hz = m->hi[3 * e + 2] - m->lo[3 * e + 2], sz = 2.0 / hz;
          for (int q = 0; q < t.Q; ++q) {
            if (ve) {
              const double zq = m->lo[3 * e + 2] + (t.xq[q] + 1.0) * 0.5 * hz, ez = std::exp(zq);
              const double f0 = 0.5 * std::exp(2.0 * m->lo[3 * e]) * th * 0.5 * hz * t.wq[q];
              w0[q] += f0 * ez * ez * ez;
              w1[q] += f0 * ez * sz * sz;
            } else {
              const double r1 = std::exp(m->lo[3 * e]);
              const double f0 = 0.5 * r1 * r1 * th * 0.5 * hz * t.wq[q];
              w0[q] += f0;
              w1[q] += f0 * sz * sz;
            }
          }
        } else if (vtx) {
          const double r1 = std::exp(m->lo[3 * e + 2]);
          w0[0] += r1 * r1 * r1 / 3.0 * (std::cos(m->lo[3 * e]) - std::cos(m->hi[3 * e])) * th;
        } else if (ve) {
          // one cone per theta sector: psi_top = the largest psi of the set's elements in it
          for (int e2 = 0; e2 < E; ++e2)
            if (m->nbr[6 * e2 + 4] == m->nbr[6 * e + 4] && std::fabs(m->lo[3 * e2 + 1] - m->lo[3 * e + 1]) < 1e-14)
              ptop[(size_t)c * E + e] = std::max(ptop[(size_t)c * E + e], m->hi[3 * e2]);
          if (std::fabs(m->hi[3 * e] - ptop[(size_t)c * E + e]) < 1e-14) {
            const double x31 = std::exp(m->lo[3 * e + 2]);
            w0[0] += th * 0.5 * std::exp(2.0 * ptop[(size_t)c * E + e]) * x31 * x31 * x31 / 3.0;
          }
        }
      }
    }
    CK(upload(m->d_h1w, hw));
    CK(upload(m->d_ch1w, cw));
  }
  const size_t ns = (size_t)std::max(1, S) * m->n_rhs * hpse::CSCR_STRIDE;
  CK(m->d_cscr64.alloc(ns * sizeof(double)));
  CK(m->d_cscr32.alloc(ns * sizeof(float)));
  CK(cudaMemset(m->d_cscr64.p, 0, ns * sizeof(double)));
  CK(cudaMemset(m->d_cscr32.p, 0, ns * sizeof(float)));
  return HPSE_OK;
}

extern "C" hpse_status hpse_setup_mesh(const hpse_mesh_desc *d, int device, hpse_mesh **out) {
  if (!d || !out) return HPSE_ERR_INVALID_ARG;
  *out = nullptr;
  if (d->n_elem < 0 || d->n_problem < 1 || d->n_rhs < 1) return HPSE_ERR_INVALID_ARG;
  init_registry();
  if (d->coef_kind != HPSE_COEF_LAPLACE && d->coef_kind != HPSE_COEF_SCALAR && d->coef_kind != HPSE_COEF_GENERAL)
    return HPSE_ERR_INVALID_ARG;
  if (d->n_elem > 0 && (!d->elem_W || !d->elem_problem || !d->elem_nbr ||
                        (d->coord != HPSE_COORD_CURVED && (!d->elem_lo || !d->elem_hi))))
    return HPSE_ERR_INVALID_ARG;
  const int E = d->n_elem;
  if ((int64_t)E * d->n_rhs > 2147483647LL) return HPSE_ERR_INVALID_ARG;
  std::unique_ptr<hpse_mesh> m(new hpse_mesh());
  m->device = device;
  m->n_elem = E;
  m->n_problem = d->n_problem;
  m->n_rhs = d->n_rhs;
  m->coef_kind = d->coef_kind;
  m->coord = d->coord;
  if (m->coord != HPSE_COORD_CARTESIAN && m->coord != HPSE_COORD_EDGE && m->coord != HPSE_COORD_VERTEX &&
      m->coord != HPSE_COORD_VERTEX_EDGE && m->coord != HPSE_COORD_CURVED)
    return HPSE_ERR_INVALID_ARG;
  m->curved = m->coord == HPSE_COORD_CURVED;
  if (m->curved) {
    // -Lap u through the maps, Dirichlet faces, no corner sets
    if (d->coef_kind != HPSE_COEF_LAPLACE || d->n_corner != 0) return HPSE_ERR_INVALID_ARG;
    if (d->face_bc)
      for (int i = 0; i < 6 * d->n_elem; ++i)
        if (d->face_bc[i] != 0) return HPSE_ERR_INVALID_ARG;
  }
  const bool nbhd = m->coord != HPSE_COORD_CARTESIAN && !m->curved;
  // faces of layer 1 towards the corner sets: 0 (a polynomial along z: edge,
  // vertex-edge) and 4 (a constant: vertex, vertex-edge)
  const bool face0_ok = m->coord == HPSE_COORD_EDGE || m->coord == HPSE_COORD_VERTEX_EDGE;
  const bool face4_ok = m->coord == HPSE_COORD_VERTEX || m->coord == HPSE_COORD_VERTEX_EDGE;
  if (nbhd) {
    // the modified-coordinate operator is built for the Laplacian (eq. 2.35)
    if (d->coef_kind != HPSE_COEF_LAPLACE || d->n_corner < 0) return HPSE_ERR_INVALID_ARG;
    if (d->n_corner > 0 && (!d->corner_W || !d->corner_problem)) return HPSE_ERR_INVALID_ARG;
    m->n_corner = d->n_corner;
    m->cW.assign(d->corner_W, d->corner_W + d->n_corner);
    m->cprob.assign(d->corner_problem, d->corner_problem + d->n_corner);
  }
  m->apply_coef = m->curved                               ? hpse::COEF_GENERAL
                 : m->coord == HPSE_COORD_EDGE            ? hpse::COEF_EDGE
                 : m->coord == HPSE_COORD_VERTEX        ? hpse::COEF_VERTEX
                 : m->coord == HPSE_COORD_VERTEX_EDGE ? hpse::COEF_VERTEX_EDGE
                 : d->coef_kind == HPSE_COEF_GENERAL  ? hpse::COEF_GENERAL
                                                        : d->coef_kind;
  m->W.assign(d->elem_W, d->elem_W + E);
  m->prob.assign(d->elem_problem, d->elem_problem + E);
  m->nbr.assign(d->elem_nbr, d->elem_nbr + 6 * (size_t)E);
  if (m->curved) {
    // the reference cube: unit scales for everything the box path reads
    m->lo.assign(3 * (size_t)E, -1.0);
    m->hi.assign(3 * (size_t)E, 1.0);
  } else {
    m->lo.assign(d->elem_lo, d->elem_lo + 3 * (size_t)E);
    m->hi.assign(d->elem_hi, d->elem_hi + 3 * (size_t)E);
  }
  // ---- validation (Section 2.3: one-to-one matching faces) -----------------
  for (int e = 0; e < E; ++e) {
    if (m->W[e] < 1 || m->W[e] > HPSE_MAX_W) return HPSE_ERR_DEGREE;
    // the general operator's kernel exists where its layout fits shared memory
    if (d->coef_kind == HPSE_COEF_GENERAL && (g_sets[0][m->W[e]].apply_smem(hpse::COEF_GENERAL) == 0 ||
                                              g_sets[1][m->W[e]].apply_smem(hpse::COEF_GENERAL) == 0))
      return HPSE_ERR_DEGREE;
    if (m->prob[e] < 0 || m->prob[e] >= m->n_problem) return HPSE_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
      if (!(m->hi[3 * e + a] > m->lo[3 * e + a]) || !std::isfinite(m->lo[3 * e + a]) ||
          !std::isfinite(m->hi[3 * e + a]))
        return HPSE_ERR_INVALID_ARG;
  }
  // outer-face conditions (eq. 2.1): Neumann and Robin faces on box meshes of the Laplacian
  m->fbc.assign(6 * (size_t)E, 0);
  m->fgam.assign(6 * (size_t)E, 0.0);
  if (d->face_bc) {
    for (size_t i = 0; i < 6 * (size_t)E; ++i) {
      const int c = d->face_bc[i];
      if (c < 0 || c > 2 || (c != 0 && m->nbr[i] != -1)) return HPSE_ERR_INVALID_ARG;
      m->fbc[i] = c;
      if (c == 2) {
        const double g = d->robin_gamma ? d->robin_gamma[m->prob[i / 6]] : 1.0;
        if (!std::isfinite(g)) return HPSE_ERR_INVALID_ARG;
        m->fgam[i] = g;
      }
      if (c != 0) m->has_nr = true;
    }
    if (m->has_nr && (nbhd || (d->coef_kind != HPSE_COEF_LAPLACE && d->coef_kind != HPSE_COEF_GENERAL)))
      return HPSE_ERR_INVALID_ARG;
  }
  const int C = m->n_corner;
  for (int c = 0; c < C; ++c)
    if (m->cW[c] < 0 || m->cW[c] > HPSE_MAX_W || m->cprob[c] < 0 || m->cprob[c] >= m->n_problem)
      return HPSE_ERR_INVALID_ARG;
  std::vector<int> corner_e(C, -1);  // first layer-1 element of each corner set
  std::vector<int> corner_f(C, -1);  // the face through which it enters
  for (int e = 0; e < E; ++e)
    for (int fi = 0; fi < 6; ++fi) {
      const int n = m->nbr[6 * e + fi];
      if (n <= -2) {
        // corner set: edge coordinates, face tau = lo only, same degree, problem and x3 slab
        const int c = -2 - n;
        if (!nbhd || c >= C || !((fi == 0 && face0_ok) || (fi == 4 && face4_ok))) return HPSE_ERR_INVALID_ARG;
        // a polynomial along z has the degree of its elements, a constant 0
        if (fi == 0 && m->cW[c] != m->W[e]) return HPSE_ERR_DEGREE;
        if (fi == 4 && m->cW[c] != 0) return HPSE_ERR_DEGREE;
        if (m->cprob[c] != m->prob[e]) return HPSE_ERR_INVALID_ARG;
        if (corner_f[c] >= 0 && corner_f[c] != fi) return HPSE_ERR_INVALID_ARG;
        corner_f[c] = fi;
        if (corner_e[c] < 0) {
          corner_e[c] = e;
        } else {
          // face 0: one z slab and the same x = lo; face 4: the same z = lo
          const int e0 = corner_e[c];
          auto differ = [&](int i0, int i1) {
            return std::fabs(m->lo[i0] - m->lo[i1]) > 1e-12 * std::max(1.0, std::fabs(m->lo[i1]));
          };
          auto differ_hi = [&](int i0, int i1) {
            return std::fabs(m->hi[i0] - m->hi[i1]) > 1e-12 * std::max(1.0, std::fabs(m->hi[i1]));
          };
          const bool bad = fi == 0
                               ? (differ(3 * e + 2, 3 * e0 + 2) || differ_hi(3 * e + 2, 3 * e0 + 2) || differ(3 * e, 3 * e0))
                               : differ(3 * e + 2, 3 * e0 + 2);
          if (bad) return HPSE_ERR_NONMATCHING_FACE;
        }
        continue;
      }
      if (n < -1 || n >= E || n == e) return HPSE_ERR_INVALID_ARG;
      if (n < 0) continue;
      if (m->nbr[6 * n + (fi ^ 1)] != e) return HPSE_ERR_NONMATCHING_FACE;
      if (m->prob[n] != m->prob[e]) return HPSE_ERR_INVALID_ARG;
      if (m->curved) continue;  // the maps share the face's parametrisation (the caller's mesh)
      const int a = fi >> 1, side = fi & 1;
      const double xe = side ? m->hi[3 * e + a] : m->lo[3 * e + a];
      const double xn = side ? m->lo[3 * n + a] : m->hi[3 * n + a];
      const double scale = std::max(1.0, std::fabs(xe));
      if (std::fabs(xe - xn) > 1e-12 * scale) return HPSE_ERR_NONMATCHING_FACE;
      for (int b = 0; b < 3; ++b) {
        if (b == a) continue;
        const double s2 = std::max(1.0, std::fabs(m->hi[3 * e + b]));
        if (std::fabs(m->lo[3 * e + b] - m->lo[3 * n + b]) > 1e-12 * s2 ||
            std::fabs(m->hi[3 * e + b] - m->hi[3 * n + b]) > 1e-12 * s2)
          return HPSE_ERR_NONMATCHING_FACE;
      }
      if (m->W[n] != m->W[e]) {
        // unequal degrees across the face: box meshes (the face terms on the
        // (2 max(W, W') + 1)-point grid, in k_face_mixed)
        if (nbhd) return HPSE_ERR_DEGREE;
        m->fbc[6 * e + fi] = 3;
        m->has_mixed = true;
      }
    }
  if (m->curved) {
    // every face of a curved element is k_face_curved's (code 3: k_apply_gen leaves it)
    for (size_t i = 0; i < m->fbc.size(); ++i) m->fbc[i] = 3;
  }
  // ---- offsets, groups, boundary faces -------------------------------------
  m->dof_off.assign(E, 0);
  m->coef_off.assign(E, 0);
  int64_t od = 0, oq = 0;
  for (int e = 0; e < E; ++e) {
    const int P = m->W[e] + 1, Q = 2 * m->W[e] + 1;
    m->dof_off[e] = od;
    m->coef_off[e] = oq;
    od += (int64_t)P * P * P;
    oq += (int64_t)Q * Q * Q;
  }
  // corner sets follow the elements in every vector
  m->item_n.assign(E + C, 0);
  for (int e = 0; e < E; ++e) m->item_n[e] = (m->W[e] + 1) * (m->W[e] + 1) * (m->W[e] + 1);
  for (int c = 0; c < C; ++c) {
    m->dof_off.push_back(od);
    m->item_n[E + c] = m->cW[c] + 1;
    od += m->cW[c] + 1;
  }
  m->ndof = od;
  m->nquad = oq;
  // face slots of the corner sets
  m->cslot.assign(2 * (size_t)E, -1);
  m->slot_ptr.assign(C + 1, 0);
  m->slot_elem.clear();
  m->slot_face.clear();
  for (int e = 0; e < E; ++e)
    for (int k = 0; k < 2; ++k) {
      const int fi = 4 * k;
      if (m->nbr[6 * e + fi] <= -2) {
        m->cslot[2 * e + k] = (int)m->slot_elem.size();
        m->slot_elem.push_back(e);
        m->slot_face.push_back(fi);
        m->slot_ptr[-2 - m->nbr[6 * e + fi] + 1]++;
      }
    }
  for (int c = 0; c < C; ++c) m->slot_ptr[c + 1] += m->slot_ptr[c];
  {
    std::vector<int> fill(m->slot_ptr.begin(), m->slot_ptr.end() - 1);
    m->slot_list.assign(m->slot_elem.size(), 0);
    for (size_t sl = 0; sl < m->slot_elem.size(); ++sl)
      m->slot_list[fill[-2 - m->nbr[6 * m->slot_elem[sl] + m->slot_face[sl]]]++] = (int)sl;
  }
  int64_t of = 0;
  for (int e = 0; e < E; ++e)
    for (int fi = 0; fi < 6; ++fi)
      if (m->nbr[6 * e + fi] == -1) {
        const int Q = 2 * m->W[e] + 1;
        m->bface_elem.push_back(e);
        m->bface_fi.push_back(fi);
        m->bface_off.push_back(of);
        of += (int64_t)Q * Q;
      }
  m->nface_pts = of;
  // vector items (elements, then corner sets) per problem
  m->prob_ptr.assign(m->n_problem + 1, 0);
  for (int e = 0; e < E; ++e) m->prob_ptr[m->prob[e] + 1]++;
  for (int c = 0; c < C; ++c) m->prob_ptr[m->cprob[c] + 1]++;
  for (int p = 0; p < m->n_problem; ++p) m->prob_ptr[p + 1] += m->prob_ptr[p];
  {
    std::vector<int> fill(m->prob_ptr.begin(), m->prob_ptr.end() - 1);
    m->prob_elems.assign(E + C, 0);
    for (int e = 0; e < E; ++e) m->prob_elems[fill[m->prob[e]]++] = e;
    for (int c = 0; c < C; ++c) m->prob_elems[fill[m->cprob[c]]++] = E + c;
  }
  for (int k = 0; k < 2; ++k)
    for (int p = 0; p < 2; ++p)
      for (int w = 0; w <= HPSE_MAX_W; ++w) m->threads[k][p][w] = w >= 1 ? default_threads(k, p, w) : 0;

  // ---- device ---------------------------------------------------------------
  init_registry();
  CK(cudaSetDevice(device));
  std::map<int, std::vector<int>> by_w;
  for (int e = 0; e < E; ++e) by_w[m->W[e]].push_back(e);
  for (auto &kv : by_w) {
    const int W = kv.first;
    m->tabs[W] = hm::build_tables(W);
    const hm::DegreeTables &t = m->tabs[W];
    CK(g_sets[0][W].upload(t.packed.data()));
    CK(g_sets[1][W].upload(t.packed.data()));
    Group g;
    g.W = W;
    g.n = (int)kv.second.size();
    m->groups.push_back(std::move(g));
    CK(upload(m->groups.back().elems, kv.second));
    // FP64 Q-grid tables for the face data and the H^1 error: B0, B1, DQ, KQ, wq
    std::vector<double> q;
    q.insert(q.end(), t.B0.begin(), t.B0.end());
    q.insert(q.end(), t.B1.begin(), t.B1.end());
    q.insert(q.end(), t.DQ.begin(), t.DQ.end());
    q.insert(q.end(), t.KQ.begin(), t.KQ.end());
    q.insert(q.end(), t.wq.begin(), t.wq.end());
    q.insert(q.end(), t.B2.begin(), t.B2.end());
    CK(upload(m->d_qtab[W], q));
  }
  // heaviest degree groups first (they are launched first on their streams)
  std::sort(m->groups.begin(), m->groups.end(), [](const Group &x, const Group &y) {
    const double wx = (double)x.n * std::pow(2.0 * x.W + 1, 3) * (x.W + 1);
    const double wy = (double)y.n * std::pow(2.0 * y.W + 1, 3) * (y.W + 1);
    return wx > wy;
  });
  if (m->groups.size() > 1) {
    CK(cudaEventCreateWithFlags(&m->fork_ev, cudaEventDisableTiming));
    for (size_t i = 0; i < m->groups.size(); ++i) {
      cudaStream_t st;
      cudaEvent_t ev;
      CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      m->gstreams.push_back(st);
      m->gevents.push_back(ev);
    }
  }
  std::vector<double> geo(4 * (size_t)E);
  std::vector<float> geo32(4 * (size_t)E);
  for (int e = 0; e < E; ++e) {
    double J = 1.0;
    for (int a = 0; a < 3; ++a) {
      const double h = m->hi[3 * e + a] - m->lo[3 * e + a];
      geo[4 * e + a] = 2.0 / h;
      J *= h / 2.0;
    }
    geo[4 * e + 3] = J;
    for (int k = 0; k < 4; ++k) geo32[4 * e + k] = (float)geo[4 * e + k];
  }
  if (nbhd) {
    hpse_status st = setup_edge(m.get());
    if (st != HPSE_OK) return st;
  }
  CK(upload(m->d_item_n, m->item_n));
  CK(upload(m->d_dof_off, m->dof_off));
  CK(upload(m->d_coef_off, m->coef_off));
  CK(upload(m->d_nbr, m->nbr));
  CK(upload(m->d_geo64, geo));
  CK(upload(m->d_geo32, geo32));
  if (m->has_nr || m->has_mixed || m->curved) {
    std::vector<float> g32(m->fgam.begin(), m->fgam.end());
    CK(upload(m->d_fbc, m->fbc));
    CK(upload(m->d_fgam64, m->fgam));
    CK(upload(m->d_fgam32, g32));
  }
  if (m->has_mixed) {
    hpse_status st = setup_mixed(m.get());
    if (st != HPSE_OK) return st;
  }
  if (m->curved) {
    hpse_status st = setup_curved(m.get());
    if (st != HPSE_OK) return st;
  }
  {
    // problem of every vector item (elements, then corner sets): the vector
    // kernels index it by item
    std::vector<int> prob_items(m->prob);
    prob_items.insert(prob_items.end(), m->cprob.begin(), m->cprob.end());
    CK(upload(m->d_prob, prob_items));
  }
  CK(upload(m->d_prob_ptr, m->prob_ptr));
  CK(upload(m->d_prob_elems, m->prob_elems));
  CK(upload(m->d_elem_W, m->W));
  *out = m.release();
  return HPSE_OK;
}

extern "C" void hpse_destroy(hpse_mesh *m) {
  if (!m) return;
  cudaSetDevice(m->device);
  delete m;
}

extern "C" int64_t hpse_ndof(const hpse_mesh *m) { return m ? m->ndof : -1; }
extern "C" int64_t hpse_nquad(const hpse_mesh *m) { return m ? m->nquad : -1; }
extern "C" int64_t hpse_nface_points(const hpse_mesh *m) { return m ? m->nface_pts : -1; }
extern "C" int32_t hpse_nrhs(const hpse_mesh *m) { return m ? m->n_rhs : -1; }
extern "C" int64_t hpse_n_boundary_faces(const hpse_mesh *m) { return m ? (int64_t)m->bface_elem.size() : -1; }

static int pointer_space(const void *p);

extern "C" int64_t hpse_curved_n_face_points(const hpse_mesh *m) {
  return (m && m->curved) ? m->cf_off.back() : -1;
}

extern "C" hpse_status hpse_curved_points(const hpse_mesh *m, double *vol_ref, double *face_ref) {
  if (!m || !m->curved) return HPSE_ERR_INVALID_ARG;
  if (vol_ref) {
    for (int e = 0; e < m->n_elem; ++e) {
      const hm::DegreeTables &t = m->tabs.at(m->W[e]);
      const int Q = t.Q;
      double *o = vol_ref + 3 * m->coef_off[e];
      for (int c = 0; c < Q; ++c)
        for (int b = 0; b < Q; ++b)
          for (int a = 0; a < Q; ++a, o += 3) {
            o[0] = t.xq[a];
            o[1] = t.xq[b];
            o[2] = t.xq[c];
          }
    }
  }
  if (face_ref) {
    for (int e = 0; e < m->n_elem; ++e)
      for (int f = 0; f < 6; ++f) {
        const int Qf = m->cf_q[6 * e + f], a = f >> 1;
        const int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
        std::vector<double> x, w;
        hm::gll_rule(Qf, x, w);
        double *o = face_ref + 3 * m->cf_off[6 * e + f];
        for (int p2 = 0; p2 < Qf; ++p2)
          for (int p1 = 0; p1 < Qf; ++p1, o += 3) {
            o[a] = (f & 1) ? 1.0 : -1.0;
            o[t1] = x[p1];
            o[t2] = x[p2];
          }
      }
  }
  return HPSE_OK;
}

extern "C" hpse_status hpse_set_geometry(hpse_mesh *m, const double *vol, const double *face, void *stream) {
  if (!m || !m->curved) return HPSE_ERR_INVALID_ARG;
  const int64_t nq = m->nquad, nfp = m->cf_off.back();
  if ((nq > 0 && !vol) || (nfp > 0 && !face)) return HPSE_ERR_INVALID_ARG;
  const int sv = nq > 0 ? pointer_space(vol) : -2, sf = nfp > 0 ? pointer_space(face) : -2;
  if (sv == -1 || sf == -1 || (sv >= 0 && sf >= 0 && sv != sf)) return HPSE_ERR_INVALID_ARG;
  CK(cudaSetDevice(m->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (m->work) {
    CK(cudaDeviceSynchronize());
    for (auto &g : m->work->graphs) cudaGraphExecDestroy(g.second);
    m->work->graphs.clear();
    m->work->graph_launches.clear();
  }
  m->has_geometry = false;
  m->has_data = false;
  DevBuf dv, df, dbad;
  const double *vp = vol, *fp = face;
  if (sv == 0) {
    CK(dv.alloc(27 * (size_t)nq * sizeof(double)));
    CK(cudaMemcpyAsync(dv.p, vol, 27 * (size_t)nq * sizeof(double), cudaMemcpyHostToDevice, s));
    vp = dv.as<double>();
  }
  if (sf == 0) {
    CK(df.alloc(9 * (size_t)nfp * sizeof(double)));
    CK(cudaMemcpyAsync(df.p, face, 9 * (size_t)nfp * sizeof(double), cudaMemcpyHostToDevice, s));
    fp = df.as<double>();
  }
  {
    std::vector<const double *> tp(HPSE_MAX_W + 1, nullptr);
    for (auto &kv : m->d_qtab) tp[kv.first] = kv.second.as<double>();
    CK(upload_reuse(m->d_tabs_ptr, tp));
  }
  CK(dbad.alloc(sizeof(int32_t)));
  CK(cudaMemsetAsync(dbad.p, 0, sizeof(int32_t), s));
  if (!m->d_coef64.p || m->d_coef64.bytes != 12 * (size_t)std::max<int64_t>(nq, 1) * sizeof(double))
    CK(m->d_coef64.alloc(12 * (size_t)std::max<int64_t>(nq, 1) * sizeof(double)));
  if (!m->d_coef32.p || m->d_coef32.bytes != 12 * (size_t)std::max<int64_t>(nq, 1) * sizeof(float))
    CK(m->d_coef32.alloc(12 * (size_t)std::max<int64_t>(nq, 1) * sizeof(float)));
  if (!m->d_cwja.p) CK(m->d_cwja.alloc((size_t)std::max<int64_t>(nq, 1) * sizeof(double)));
  if (!m->d_cKv.p) CK(m->d_cKv.alloc(9 * (size_t)std::max<int64_t>(nq, 1) * sizeof(double)));
  if (!m->d_cdet.p) CK(m->d_cdet.alloc((size_t)std::max<int64_t>(nq, 1) * sizeof(double)));
  if (!m->d_cK64.p) CK(m->d_cK64.alloc(9 * (size_t)std::max<int64_t>(nfp, 1) * sizeof(double)));
  if (!m->d_cK32.p) CK(m->d_cK32.alloc(9 * (size_t)std::max<int64_t>(nfp, 1) * sizeof(float)));
  if (m->n_elem > 0) {
    curved::k_geom_vol<<<m->n_elem, 256, 0, s>>>(nq, m->d_elem_W.as<int32_t>(), m->d_coef_off.as<int64_t>(),
                                                 m->d_tabs_ptr.as<const double *>(), vp, m->d_coef64.as<double>(),
                                                 m->d_coef32.as<float>(), m->d_cwja.as<double>(),
                                                 m->d_cKv.as<double>(), m->d_cdet.as<double>(), dbad.as<int32_t>());
    CK(cudaGetLastError());
    curved::k_geom_face<<<256, 256, 0, s>>>(nfp, fp, m->d_cK64.as<double>(), m->d_cK32.as<float>(),
                                            dbad.as<int32_t>());
    CK(cudaGetLastError());
    g_launches += 2;
  }
  int32_t h_bad = 0;
  CK(cudaMemcpyAsync(&h_bad, dbad.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h_bad) return HPSE_ERR_INVALID_ARG;
  m->has_geometry = true;
  return HPSE_OK;
}

extern "C" hpse_status hpse_query_points(const hpse_mesh *m, double *vol_axes, double *face_norm) {
  if (!m) return HPSE_ERR_INVALID_ARG;
  if (vol_axes) {
    int64_t o = 0;
    for (int e = 0; e < m->n_elem; ++e) {
      const hm::DegreeTables &t = m->tabs.at(m->W[e]);
      for (int a = 0; a < 3; ++a) {
        const double lo = m->lo[3 * e + a], h = m->hi[3 * e + a] - lo;
        for (int q = 0; q < t.Q; ++q) vol_axes[o++] = lo + (t.xq[q] + 1.0) * 0.5 * h;
      }
    }
  }
  if (face_norm) {
    for (size_t i = 0; i < m->bface_elem.size(); ++i) {
      const int e = m->bface_elem[i], fi = m->bface_fi[i];
      const int a = fi >> 1;
      face_norm[i] = (fi & 1) ? m->hi[3 * e + a] : m->lo[3 * e + a];
    }
  }
  return HPSE_OK;
}

// Variable coefficient of box elements from device data, per volume point:
// coef = (w J a^2, s_k (d_k a) / a) in FP64 and FP32, wja = w J a, aux =
// (w J, a, d_x a, d_y a, d_z a); bad[0] = 1 where a <= 0 or a is not finite
// (the operator of eq. 2.1 must be elliptic).  One CTA per element.
__global__ void k_coef_scalar(int64_t nq, const int32_t *elem_W, const int64_t *coef_off, const double *geo,
                              const double *const *qtab, const double *a, const double *ga, double *coef64,
                              float *coef32, double *wja, double *aux, int32_t *bad) {
  const int e = blockIdx.x;
  const int W = elem_W[e], P = W + 1, Q = 2 * W + 1;
  const double *wq = qtab[W] + 2 * Q * P + 2 * Q * Q;
  const double *gs = geo + 4 * (int64_t)e;
  for (int t = threadIdx.x; t < Q * Q * Q; t += blockDim.x) {
    const int qa = t % Q, qb = (t / Q) % Q, qc = t / (Q * Q);
    const int64_t i = coef_off[e] + t;
    const double wJ = wq[qa] * wq[qb] * wq[qc] * gs[3];
    double av = a[i];
    if (!(av > 0.0) || !isfinite(av)) {
      bad[0] = 1;
      av = 1.0;
    }
    coef64[4 * i] = wJ * av * av;
    coef32[4 * i] = (float)(wJ * av * av);
    aux[i] = wJ;
    aux[nq + i] = av;
    for (int k = 0; k < 3; ++k) {
      const double g = ga[k * nq + i];
      coef64[4 * i + 1 + k] = gs[k] * g / av;
      coef32[4 * i + 1 + k] = (float)(gs[k] * g / av);
      aux[(2 + k) * nq + i] = g;
    }
    wja[i] = wJ * av;
  }
}

// General operator of box elements (eq. 2.2 written out; the ten-term form
// of eq. 5.45 in the element's reference coordinates) from op = (A_11, A_22,
// A_33, A_12, A_23, A_13, b_1, b_2, b_3, c) per volume point (device memory):
// coef = (w J, C_11, C_22, C_33, C_12, C_23, C_13, C_1, C_2, C_3, C_0, 0) with
// C_aa = A_aa s_a^2, C_ab = 2 A_ab s_a s_b, C_a = b_a s_a, C_0 = c, in FP64
// and FP32; wja = -w J (the volume part of b is then the transposed apply of
// w J f); bad[0] = 1 where a coefficient is not finite.  One CTA per element.
__global__ void k_coef_general(int64_t nq, const int32_t *elem_W, const int64_t *coef_off, const double *geo,
                               const double *const *qtab, const double *op, double *coef64, float *coef32,
                               double *wja, int32_t *bad) {
  const int e = blockIdx.x;
  const int W = elem_W[e], P = W + 1, Q = 2 * W + 1;
  const double *wq = qtab[W] + 2 * Q * P + 2 * Q * Q;
  const double *gs = geo + 4 * (int64_t)e;
  // (row, column) of A_11 .. A_13 and the factor of the off-diagonal pairs
  const int ia[6] = {0, 1, 2, 0, 1, 0}, ja[6] = {0, 1, 2, 1, 2, 2};
  for (int t = threadIdx.x; t < Q * Q * Q; t += blockDim.x) {
    const int qa = t % Q, qb = (t / Q) % Q, qc = t / (Q * Q);
    const int64_t i = coef_off[e] + t;
    const double wJ = wq[qa] * wq[qb] * wq[qc] * gs[3];
    double c[12];
    c[0] = wJ;
    for (int k = 0; k < 10; ++k) {
      double v = op[k * nq + i];
      if (!isfinite(v)) {
        bad[0] = 1;
        v = 0.0;
      }
      if (k < 6) c[1 + k] = (k < 3 ? 1.0 : 2.0) * v * gs[ia[k]] * gs[ja[k]];
      else if (k < 9) c[1 + k] = v * gs[k - 6];
      else c[10] = v;
    }
    c[11] = 0.0;
    for (int k = 0; k < 12; ++k) {
      coef64[12 * i + k] = c[k];
      coef32[12 * i + k] = (float)c[k];
    }
    wja[i] = -wJ;
  }
}

// where a data pointer points: 1 device (or managed), 0 host, -1 unknown
static int pointer_space(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? 1 : 0;
}

extern "C" hpse_status hpse_set_data(hpse_mesh *m, const hpse_data *data, void *stream) {
  if (!m || !data || (!data->f && m->nquad > 0)) return HPSE_ERR_INVALID_ARG;
  if (m->coef_kind == HPSE_COEF_SCALAR && (!data->a || !data->grad_a)) return HPSE_ERR_INVALID_ARG;
  const bool gen = m->coef_kind == HPSE_COEF_GENERAL;
  if (gen && !data->op && m->nquad > 0) return HPSE_ERR_INVALID_ARG;
  // curved elements: the operator's coefficients come from hpse_set_geometry
  if (m->curved && !m->has_geometry) return HPSE_ERR_NO_DATA;
  CK(cudaSetDevice(m->device));
  // host or device data: every given pointer in the same space
  int space = -2;
  for (const void *p : {(const void *)data->f, (const void *)data->a, (const void *)data->grad_a,
                        (const void *)data->g, (const void *)(gen ? data->op : nullptr)}) {
    if (!p) continue;
    const int sp = pointer_space(p);
    if (sp < 0 || (space != -2 && sp != space)) return HPSE_ERR_INVALID_ARG;
    space = sp;
  }
  const bool dev = space == 1;
  const cudaMemcpyKind kin = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaStream_t s = (cudaStream_t)stream;
  // captured solver graphs refer to the coefficient and right-hand side
  // buffers: drop them so that the next solve re-captures with current data
  if (m->work) {
    CK(cudaDeviceSynchronize());
    for (auto &g : m->work->graphs) cudaGraphExecDestroy(g.second);
    m->work->graphs.clear();
    m->work->graph_launches.clear();
  }
  const int64_t nq = m->nquad;
  const int R = m->n_rhs;
  // coefficients at the volume points: m = w J a^2, d_k = s_k a_k / a; wJa for b
  std::vector<double> wja(nq);
  std::vector<double> coef;
  const bool vtx = m->coord == HPSE_COORD_VERTEX, ve = m->coord == HPSE_COORD_VERTEX_EDGE;
  // a variable coefficient given on the device is transformed on the device
  const bool dev_coef = dev && m->coef_kind == HPSE_COEF_SCALAR;
  if ((m->coef_kind == HPSE_COEF_SCALAR && !dev_coef) || vtx || ve) coef.assign(4 * (size_t)nq, 0.0);
  for (int e = 0; e < (dev_coef ? 0 : m->n_elem); ++e) {
    const hm::DegreeTables &t = m->tabs.at(m->W[e]);
    const int Q = t.Q;
    double s[3], J = 1.0;
    for (int a = 0; a < 3; ++a) {
      const double h = m->hi[3 * e + a] - m->lo[3 * e + a];
      s[a] = 2.0 / h;
      J *= h / 2.0;
    }
    const int64_t o = m->coef_off[e];
    for (int c = 0; c < Q; ++c)
      for (int b = 0; b < Q; ++b)
        for (int a = 0; a < Q; ++a) {
          const int64_t i = o + ((int64_t)c * Q + b) * Q + a;
          const double wJ = t.wq[a] * t.wq[b] * t.wq[c] * J;
          if (m->coef_kind == HPSE_COEF_SCALAR) {
            const double av = data->a[i];
            if (!(av > 0.0) || !std::isfinite(av)) return HPSE_ERR_INVALID_ARG;  // ellipticity
            coef[4 * i] = wJ * av * av;
            for (int k = 0; k < 3; ++k) coef[4 * i + k + 1] = s[k] * data->grad_a[k * nq + i] / av;
            wja[i] = wJ * av;
          } else if (vtx) {
            // L^v = -c (u_chichi + u_chi + u_phiphi + cot(phi) u_phi + u_thetatheta / sin^2 phi)
            // with c^2 = e^chi sin(phi) (eq. 4.3): m = w J c^2, d = (s_phi cot(phi), 0, s_chi);
            // the 1/sin^2 phi of u_thetatheta is a per-x-point factor of the kernel;
            // b: F^v = c e^{2 chi} f, so w J c F^v = w J c^2 e^{2 chi} f
            const double ph = m->lo[3 * e] + (t.xq[a] + 1.0) * 0.5 * (m->hi[3 * e] - m->lo[3 * e]);
            const double ch = m->lo[3 * e + 2] + (t.xq[c] + 1.0) * 0.5 * (m->hi[3 * e + 2] - m->lo[3 * e + 2]);
            const double c2 = std::exp(ch) * std::sin(ph);
            coef[4 * i] = wJ * c2;
            coef[4 * i + 1] = s[0] * std::cos(ph) / std::sin(ph);
            coef[4 * i + 2] = 0.0;
            coef[4 * i + 3] = s[2];
            wja[i] = wJ * c2 * std::exp(2.0 * ch);
          } else if (ve) {
            // L^{v-e} = -c (u_psipsi + u_thetatheta + k (u_psipsi - 2 u_psizeta +
            // u_zetazeta + u_psi - u_zeta)) with c^2 = e^zeta, k = e^{2 psi}
            // (eq. 2.28): m = w J c^2, d = (s_psi k, -2 s_psi s_zeta k [u_psizeta],
            // -s_zeta k); 1 + k on u_psipsi and k on u_zetazeta are per-x-point
            // factors of the kernel; b: F^{v-e} = c r^2 f with r = e^{psi + zeta}
            const double ps = m->lo[3 * e] + (t.xq[a] + 1.0) * 0.5 * (m->hi[3 * e] - m->lo[3 * e]);
            const double ze = m->lo[3 * e + 2] + (t.xq[c] + 1.0) * 0.5 * (m->hi[3 * e + 2] - m->lo[3 * e + 2]);
            const double k = std::exp(2.0 * ps), c2 = std::exp(ze);
            coef[4 * i] = wJ * c2;
            coef[4 * i + 1] = s[0] * k;
            coef[4 * i + 2] = -2.0 * s[0] * s[2] * k;
            coef[4 * i + 3] = -s[2] * k;
            wja[i] = wJ * c2 * std::exp(2.0 * (ps + ze));
          } else if (m->coord == HPSE_COORD_EDGE) {
            // F^e = e^{2 tau} f (eq. 4.7): tau is the x coordinate of the point
            const double tau = m->lo[3 * e] + (t.xq[a] + 1.0) * 0.5 * (m->hi[3 * e] - m->lo[3 * e]);
            wja[i] = wJ * std::exp(2.0 * tau);
          } else {
            wja[i] = wJ;
          }
        }
  }
  if (!dev_coef) {
    std::vector<double> aux(5 * (size_t)nq);
    for (int e = 0; e < m->n_elem; ++e) {
      const hm::DegreeTables &t = m->tabs.at(m->W[e]);
      const int Q = t.Q;
      double J = 1.0;
      for (int a = 0; a < 3; ++a) J *= (m->hi[3 * e + a] - m->lo[3 * e + a]) / 2.0;
      const int64_t o = m->coef_off[e];
      for (int c = 0; c < Q; ++c)
        for (int b = 0; b < Q; ++b)
          for (int a = 0; a < Q; ++a) {
            const int64_t i = o + ((int64_t)c * Q + b) * Q + a;
            aux[i] = t.wq[a] * t.wq[b] * t.wq[c] * J;
            const bool var = m->coef_kind == HPSE_COEF_SCALAR;
            aux[nq + i] = var ? data->a[i] : 1.0;
            for (int k = 0; k < 3; ++k) aux[(2 + k) * nq + i] = var ? data->grad_a[k * nq + i] : 0.0;
          }
    }
    CK(upload_reuse(m->d_aux, aux));
  }
  if (!m->d_f.p || m->d_f.bytes != (size_t)R * nq * sizeof(double)) CK(m->d_f.alloc((size_t)R * nq * sizeof(double)));
  if (nq > 0) CK(cudaMemcpyAsync(m->d_f.p, data->f, (size_t)R * nq * sizeof(double), kin, s));
  {
    std::vector<const double *> tp(HPSE_MAX_W + 1, nullptr);
    for (auto &kv : m->d_qtab) tp[kv.first] = kv.second.as<double>();
    CK(upload_reuse(m->d_tabs_ptr, tp));
  }
  DevBuf dwja, dbad;
  if (dev_coef) {
    if (!m->d_coef64.p || m->d_coef64.bytes != 4 * (size_t)nq * sizeof(double))
      CK(m->d_coef64.alloc(4 * (size_t)std::max<int64_t>(nq, 1) * sizeof(double)));
    if (!m->d_coef32.p || m->d_coef32.bytes != 4 * (size_t)nq * sizeof(float))
      CK(m->d_coef32.alloc(4 * (size_t)std::max<int64_t>(nq, 1) * sizeof(float)));
    if (!m->d_aux.p || m->d_aux.bytes != 5 * (size_t)nq * sizeof(double))
      CK(m->d_aux.alloc(5 * (size_t)std::max<int64_t>(nq, 1) * sizeof(double)));
    CK(dwja.alloc((size_t)std::max<int64_t>(nq, 1) * sizeof(double)));
    CK(dbad.alloc(sizeof(int32_t)));
    CK(cudaMemsetAsync(dbad.p, 0, sizeof(int32_t), s));
    if (m->n_elem > 0) {
      k_coef_scalar<<<m->n_elem, 256, 0, s>>>(nq, m->d_elem_W.as<int32_t>(), m->d_coef_off.as<int64_t>(),
                                             m->d_geo64.as<double>(), m->d_tabs_ptr.as<const double *>(), data->a,
                                             data->grad_a, m->d_coef64.as<double>(), m->d_coef32.as<float>(),
                                             dwja.as<double>(), m->d_aux.as<double>(), dbad.as<int32_t>());
      CK(cudaGetLastError());
      ++g_launches;
    }
  } else if (gen) {
    // the general operator's coefficients are transformed on the device
    // (host data is first copied there)
    if (!m->d_coef64.p || m->d_coef64.bytes != 12 * (size_t)nq * sizeof(double))
      CK(m->d_coef64.alloc(12 * (size_t)std::max<int64_t>(nq, 1) * sizeof(double)));
    if (!m->d_coef32.p || m->d_coef32.bytes != 12 * (size_t)nq * sizeof(float))
      CK(m->d_coef32.alloc(12 * (size_t)std::max<int64_t>(nq, 1) * sizeof(float)));
    CK(dwja.alloc((size_t)std::max<int64_t>(nq, 1) * sizeof(double)));
    CK(dbad.alloc(sizeof(int32_t)));
    CK(cudaMemsetAsync(dbad.p, 0, sizeof(int32_t), s));
    DevBuf dop;
    const double *opd = data->op;
    if (!dev && nq > 0) {
      CK(dop.alloc(10 * (size_t)nq * sizeof(double)));
      CK(cudaMemcpyAsync(dop.p, data->op, 10 * (size_t)nq * sizeof(double), cudaMemcpyHostToDevice, s));
      opd = dop.as<double>();
    }
    if (m->n_elem > 0) {
      k_coef_general<<<m->n_elem, 256, 0, s>>>(nq, m->d_elem_W.as<int32_t>(), m->d_coef_off.as<int64_t>(),
                                              m->d_geo64.as<double>(), m->d_tabs_ptr.as<const double *>(), opd,
                                              m->d_coef64.as<double>(), m->d_coef32.as<float>(),
                                              dwja.as<double>(), dbad.as<int32_t>());
      CK(cudaGetLastError());
      ++g_launches;
    }
    CK(cudaStreamSynchronize(s));
  } else {
    if (m->coef_kind == HPSE_COEF_SCALAR || vtx || ve) {
      std::vector<float> c32(coef.size());
      for (size_t i = 0; i < coef.size(); ++i) c32[i] = (float)coef[i];
      CK(upload_reuse(m->d_coef64, coef));
      CK(upload_reuse(m->d_coef32, c32));
    }
    CK(upload(dwja, wja));
  }
  const size_t nv = (size_t)R * m->ndof;
  if (!m->d_b.p || m->d_b.bytes != nv * sizeof(double)) CK(m->d_b.alloc(nv * sizeof(double)));
  if (nv) CK(cudaMemsetAsync(m->d_b.p, 0, nv * sizeof(double), s));
  // volume part of b: transpose kernel on rho_b = -(w J a) f
  if (nq > 0 && m->n_elem > 0) {
    DevBuf drho;
    CK(drho.alloc((size_t)R * nq * sizeof(double)));
    k_rho_b<<<1024, 256, 0, s>>>((int64_t)R * nq, m->curved ? m->d_cwja.as<double>() : dwja.as<double>(),
                                 m->d_f.as<double>(), nq, drho.as<double>());
    CK(cudaGetLastError());
    ++g_launches;
    ApplyArgsT<double> a = apply_args<double>(m, m->groups[0], nullptr, m->d_b.as<double>());
    a.rho = drho.as<double>();
    a.skip_faces = 1;
    hpse_status st = launch_apply_all<double>(m, MODE_TRANSPOSE, a, s);
    if (st != HPSE_OK) return st;
    CK(cudaStreamSynchronize(s));
  }
  // Dirichlet data part of b (curved elements: on each face's grid, by k_face_curved)
  if (m->curved && data->g && m->nface_pts > 0 && m->n_elem > 0) {
    DevBuf dg;
    CK(dg.alloc((size_t)R * m->nface_pts * sizeof(double)));
    CK(cudaMemcpyAsync(dg.p, data->g, (size_t)R * m->nface_pts * sizeof(double), kin, s));
    curved::FaceArgs A = curved_args(m, R);
    curved::k_face_curved<double, 0, true><<<m->n_elem * R, 128, curved::face_smem(8), s>>>(
        A, nullptr, m->d_cK64.as<double>(), dg.as<double>(), m->d_b.as<double>(), nullptr);
    CK(cudaGetLastError());
    ++g_launches;
    CK(cudaStreamSynchronize(s));
  } else if (data->g && m->nface_pts > 0) {
    std::vector<int> felem_ptr(1, 0), felems, ffi;
    std::vector<int64_t> foff;
    for (size_t i = 0; i < m->bface_elem.size(); ++i) {
      if (felems.empty() || felems.back() != m->bface_elem[i]) {
        if (!felems.empty()) felem_ptr.push_back((int)ffi.size());
        felems.push_back(m->bface_elem[i]);
      }
      ffi.push_back(m->bface_fi[i]);
      foff.push_back(m->bface_off[i]);
    }
    felem_ptr.push_back((int)ffi.size());
    DevBuf dptr, delems, dfi, doff, dg, dtabs;
    CK(upload(dptr, felem_ptr));
    CK(upload(delems, felems));
    CK(upload(dfi, ffi));
    CK(upload(doff, foff));
    CK(dg.alloc((size_t)R * m->nface_pts * sizeof(double)));
    CK(cudaMemcpyAsync(dg.p, data->g, (size_t)R * m->nface_pts * sizeof(double), kin, s));
    std::vector<const double *> tp(HPSE_MAX_W + 1, nullptr);
    int Wmax = 1;
    for (auto &kv : m->d_qtab) {
      tp[kv.first] = kv.second.as<double>();
      Wmax = std::max(Wmax, kv.first);
    }
    CK(upload(dtabs, tp));
    FaceDataArgs A;
    A.n_rhs = R;
    A.ndof = m->ndof;
    A.nface_pts = m->nface_pts;
    A.dof_off = m->d_dof_off.as<int64_t>();
    A.elem_W = m->d_elem_W.as<int32_t>();
    A.felem_ptr = dptr.as<int32_t>();
    A.felems = delems.as<int32_t>();
    A.face_fi = dfi.as<int32_t>();
    A.face_off = doff.as<int64_t>();
    A.qtab = dtabs.as<const double *>();
    A.g = dg.as<double>();
    A.b = m->d_b.as<double>();
    A.fw = m->coord != HPSE_COORD_CARTESIAN ? m->d_fw64.as<double>() : nullptr;
    A.fbc = m->has_nr ? m->d_fbc.as<int32_t>() : nullptr;
    A.fgam = m->has_nr ? m->d_fgam64.as<double>() : nullptr;
    A.geo = m->d_geo64.as<double>();
    const int Q = 2 * Wmax + 1, P = Wmax + 1;
    const size_t smem = (size_t)(8 * Q * Q + 2 * Q * P + P * P) * sizeof(double);
    CK(raise_smem((const void *)k_face_data, m->device, (size_t)smem));
    k_face_data<<<(int)felems.size() * R, 128, smem, s>>>(A);
    CK(cudaGetLastError());
    ++g_launches;
    CK(cudaStreamSynchronize(s));
  }
  // ||b||^2 per (problem, rhs)
  {
    const int npr = npr_of(m);
    DevBuf part;
    CK(part.alloc((size_t)std::max(1, n_items_vec(m)) * sizeof(double)));
    if (!m->d_bnorm2.p) CK(m->d_bnorm2.alloc((size_t)npr * sizeof(double)));
    if (n_items_vec(m) > 0) {
      k_dot<double, double><<<n_items_vec(m), 128, 0, s>>>(elem_args(m), m->d_b.as<double>(),
                                                           m->d_b.as<double>(), part.as<double>());
      CK(cudaGetLastError());
      ++g_launches;
    }
    k_bnorm<<<npr, 128, 0, s>>>(fin_args(m), part.as<double>(), m->d_bnorm2.as<double>());
    CK(cudaGetLastError());
    ++g_launches;
    CK(cudaStreamSynchronize(s));
  }
  if (dev_coef || gen) {
    int32_t h_bad = 0;
    CK(cudaMemcpy(&h_bad, dbad.p, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (h_bad) {
      // the device buffers now hold the rejected data: no solve until valid data is set
      m->has_data = false;
      return HPSE_ERR_INVALID_ARG;
    }
  }
  m->has_data = true;
  return HPSE_OK;
}

extern "C" hpse_status hpse_get_rhs(hpse_mesh *m, double *b, void *stream) {
  if (!m || (!b && m->ndof > 0)) return HPSE_ERR_INVALID_ARG;
  if (!m->has_data) return HPSE_ERR_NO_DATA;
  CK(cudaSetDevice(m->device));
  const size_t nv = (size_t)m->n_rhs * m->ndof;
  if (nv) CK(cudaMemcpyAsync(b, m->d_b.p, nv * sizeof(double), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return HPSE_OK;
}

static hpse_status check_coef(hpse_mesh *m) {
  if ((m->coef_kind == HPSE_COEF_SCALAR || m->coef_kind == HPSE_COEF_GENERAL) && !m->has_data)
    return HPSE_ERR_NO_DATA;
  return HPSE_OK;
}

extern "C" hpse_status hpse_apply_operator(hpse_mesh *m, int32_t prec, const void *u, void *y, void *stream) {
  if (!m || (prec != HPSE_FP64 && prec != HPSE_FP32)) return HPSE_ERR_INVALID_ARG;
  if (m->ndof == 0) return HPSE_OK;
  if (!u || !y || u == y) return HPSE_ERR_INVALID_ARG;
  hpse_status st = check_coef(m);
  if (st != HPSE_OK) return st;
  CK(cudaSetDevice(m->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == HPSE_FP64) {
    ApplyArgsT<double> a = apply_args<double>(m, m->groups[0], (const double *)u, (double *)y);
    return launch_apply_all<double>(m, MODE_PLAIN, a, s);
  }
  ApplyArgsT<float> a = apply_args<float>(m, m->groups[0], (const float *)u, (float *)y);
  return launch_apply_all<float>(m, MODE_PLAIN, a, s);
}

extern "C" hpse_status hpse_apply_preconditioner(hpse_mesh *m, int32_t prec, const void *r, void *z, void *stream) {
  if (!m || (prec != HPSE_FP64 && prec != HPSE_FP32)) return HPSE_ERR_INVALID_ARG;
  if (m->ndof == 0) return HPSE_OK;
  if (!r || !z || r == z) return HPSE_ERR_INVALID_ARG;
  CK(cudaSetDevice(m->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == HPSE_FP64) {
    PrecArgsT<double> a = prec_args<double>(m, m->groups[0]);
    a.rin = (const double *)r;
    a.zout = (double *)z;
    return launch_prec_all<double>(m, MODE_PLAIN, a, s);
  }
  PrecArgsT<float> a = prec_args<float>(m, m->groups[0]);
  a.rin = (const float *)r;
  a.zout = (float *)z;
  return launch_prec_all<float>(m, MODE_PLAIN, a, s);
}

static void drop_graphs(hpse_mesh *m) {
  if (!m->work) return;
  for (auto &g : m->work->graphs) cudaGraphExecDestroy(g.second);
  m->work->graphs.clear();
  m->work->graph_launches.clear();
}

extern "C" hpse_status hpse_setup_block_preconditioner(hpse_mesh *m) {
  if (!m) return HPSE_ERR_INVALID_ARG;
  if (!m->has_data) return HPSE_ERR_NO_DATA;
  CK(cudaSetDevice(m->device));
  CK(cudaDeviceSynchronize());
  drop_graphs(m);
  m->bj_ready = false;
  m->precond_kind = HPSE_PRECOND_SEPARABLE;
  const int E = m->n_elem;
  std::vector<int64_t> off(E + 1, 0);
  for (int e = 0; e < E; ++e) {
    const int64_t n = (int64_t)(m->W[e] + 1) * (m->W[e] + 1) * (m->W[e] + 1);
    off[e + 1] = off[e] + n * (n + 1) / 2;
  }
  const int64_t total = off[E];
  CK(upload(m->d_bj_off, off));
  DevBuf blk;
  if (blk.alloc(std::max<int64_t>(total, 1) * sizeof(double)) != cudaSuccess) return HPSE_ERR_OOM;
  if (m->d_bj64.alloc(std::max<int64_t>(total, 1) * sizeof(double)) != cudaSuccess) return HPSE_ERR_OOM;
  if (m->d_bj32.alloc(std::max<int64_t>(total, 1) * sizeof(float)) != cudaSuccess) return HPSE_ERR_OOM;
  const size_t nv = (size_t)m->n_rhs * m->ndof;
  if (m->bj_t64.alloc(std::max<size_t>(nv, 1) * sizeof(double)) != cudaSuccess) return HPSE_ERR_OOM;
  if (m->bj_t32.alloc(std::max<size_t>(nv, 1) * sizeof(float)) != cudaSuccess) return HPSE_ERR_OOM;
  DevBuf fail;
  CK(fail.alloc(sizeof(int32_t)));
  CK(cudaMemset(fail.p, 0, sizeof(int32_t)));
  // probes: nc unit vectors per launch, each in every element of a group at once
  const size_t maxbytes = (size_t)1 << 31;
  int nc = (int)std::min<size_t>(64, std::max<size_t>(1, maxbytes / (std::max<int64_t>(m->ndof, 1) * sizeof(double))));
  DevBuf pu, py;
  if (pu.alloc((size_t)nc * std::max<int64_t>(m->ndof, 1) * sizeof(double)) != cudaSuccess) return HPSE_ERR_OOM;
  if (py.alloc((size_t)nc * std::max<int64_t>(m->ndof, 1) * sizeof(double)) != cudaSuccess) return HPSE_ERR_OOM;
  cudaStream_t s = 0;
  for (size_t gi = 0; gi < m->groups.size(); ++gi) {
    const Group &g = m->groups[gi];
    const int n = (g.W + 1) * (g.W + 1) * (g.W + 1);
    BjArgs ba = bj_args(m, g, nc);
    ApplyArgsT<double> a = apply_args<double>(m, g, pu.as<double>(), py.as<double>());
    a.n_rhs = nc;
    a.self_only = 1;
    const KernelSet &ks = g_sets[0][g.W];
    const int th = m->threads[0][0][g.W];
    for (int j0 = 0; j0 < n; j0 += nc) {
      const int c = std::min(nc, n - j0);
      a.n_rhs = c;
      ba.n_rhs = c;
      k_bj_probe<<<g.n * c, 128, 0, s>>>(ba, j0, c, pu.as<double>());
      CK(cudaGetLastError());
      CK(ks.apply(m->apply_coef, MODE_PLAIN, &a, g.n * c, th, s));
      {
        hpse_status st = launch_mixed<double>(m, MODE_PLAIN, pu.as<double>(), py.as<double>(), nullptr, c, 1, g.W, s);
        if (st != HPSE_OK) return st;
        st = launch_curved<double>(m, MODE_PLAIN, pu.as<double>(), py.as<double>(), nullptr, c, 1, g.W, s);
        if (st != HPSE_OK) return st;
      }
      k_bj_gather<<<g.n * c, 128, 0, s>>>(ba, j0, c, py.as<double>(), blk.as<double>());
      CK(cudaGetLastError());
      g_launches += 3;
    }
    const size_t sm = (size_t)n * sizeof(double);
    CK(raise_smem((const void *)k_bj_chol, m->device, (size_t)std::max<size_t>(sm, 1)));
    CK(raise_smem((const void *)k_bj_trinv, m->device, (size_t)std::max<size_t>(sm, 1)));
    k_bj_chol<<<g.n, 256, sm, s>>>(ba, blk.as<double>(), fail.as<int32_t>());
    CK(cudaGetLastError());
    k_bj_trinv<<<g.n, 256, sm, s>>>(ba, blk.as<double>(), m->d_bj64.as<double>());
    CK(cudaGetLastError());
    g_launches += 2;
  }
  if (total > 0) {
    k_bj_convert<float><<<1024, 256, 0, s>>>(m->d_bj64.as<double>(), m->d_bj32.as<float>(), total);
    CK(cudaGetLastError());
    ++g_launches;
  }
  int32_t h_fail = 0;
  CK(cudaMemcpy(&h_fail, fail.p, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (h_fail) return HPSE_ERR_BREAKDOWN;
  // tensor-core form (a candidate from 32 right-hand sides on): FP32 tiles of
  // X and X^T per element
  m->d_bjt = DevBuf();
  m->d_bjt_off = DevBuf();
  if (m->n_rhs >= 32 && total > 0) {
    std::vector<int64_t> toff(E + 1, 0);
    for (int e = 0; e < E; ++e) {
      const int n = (m->W[e] + 1) * (m->W[e] + 1) * (m->W[e] + 1);
      toff[e + 1] = toff[e] + 2 * (int64_t)bjt_blocks(n) * BJT_TILE;
    }
    if (m->d_bjt.alloc((size_t)toff[E] * sizeof(float)) != cudaSuccess) return HPSE_ERR_OOM;
    CK(upload(m->d_bjt_off, toff));
    if (!m->d_bjt_err.p) CK(m->d_bjt_err.alloc(sizeof(int32_t)));
    CK(cudaMemset(m->d_bjt_err.p, 0, sizeof(int32_t)));
    CK(raise_smem((const void *)k_bj_tc<false>, m->device, BJT_SMEM));
    CK(raise_smem((const void *)k_bj_tc<true>, m->device, BJT_SMEM));
    for (size_t gi = 0; gi < m->groups.size(); ++gi) {
      const Group &g = m->groups[gi];
      const BjArgs ba = bj_args(m, g, m->n_rhs);
      const int n = (g.W + 1) * (g.W + 1) * (g.W + 1);
      k_bj_tile<<<g.n * 2 * bjt_blocks(n), 256, 0, s>>>(ba, m->d_bjt_off.as<int64_t>(), m->d_bj64.as<double>(),
                                                         m->d_bjt.as<float>());
      CK(cudaGetLastError());
      ++g_launches;
    }
  }
  // autotuner: time every candidate tile shape of the two triangular products
  // on the factors just built (right-hand-side count of the mesh, per degree
  // group and precision; one warm-up, then the mean of 3 launches by CUDA
  // events) and keep the fastest
  {
    DevBuf tin, tout;
    const size_t nvb = std::max<size_t>(nv, 1) * sizeof(double);
    if (tin.alloc(nvb) != cudaSuccess || tout.alloc(nvb) != cudaSuccess) return HPSE_ERR_OOM;
    CK(cudaMemset(tin.p, 0, nvb));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (size_t gi = 0; gi < m->groups.size(); ++gi) {
      const Group &g = m->groups[gi];
      const BjArgs ba = bj_args(m, g, m->n_rhs);
      for (int pi = 0; pi < 2; ++pi) {
        int cand[4];
        const int nc2 = bj_candidates(m->n_rhs, pi == 1, cand);
        float best = 1e30f;
        for (int k = 0; k < BJ_NVAR; ++k) m->bj_ms[g.W][pi][k] = 0.0f;
        for (int ci = 0; ci < nc2; ++ci) {
          const int v = cand[ci];
          if (v == BJ_TC && !m->d_bjt.p) continue;
          float ms = 0.0f;
          for (int rep = 0; rep < 4; ++rep) {
            if (rep == 1) CK(cudaEventRecord(e0, s));
            if (pi == 0)
              CK(bj_apply_group<double>(ba, m->d_bj64.as<double>(), tin.as<double>(), m->bj_t64.as<double>(),
                                        tout.as<double>(), s, v));
            else {
              const hpse_status st = bj_products<float>(m, g, ba, m->d_bj32.as<float>(), tin.as<float>(),
                                                        m->bj_t32.as<float>(), tout.as<float>(), s, v);
              if (st != HPSE_OK) return st;
            }
            g_launches += 2;
          }
          CK(cudaEventRecord(e1, s));
          CK(cudaEventSynchronize(e1));
          CK(cudaEventElapsedTime(&ms, e0, e1));
          ms /= 3.0f;
          if (v == BJ_TC) {
            // a tensor-core product whose bounded wait expired is not a candidate
            int32_t h_err = 0;
            CK(cudaMemcpy(&h_err, m->d_bjt_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost));
            if (h_err) continue;
          }
          m->bj_ms[g.W][pi][v] = ms;
          if (ms < best) {
            best = ms;
            m->bj_var[g.W][pi] = v;
          }
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  // accuracy of the FP32 factor products, per degree group, on a test vector:
  // ||z32 - z64|| / ||z64|| > 1e-2 (a block whose triangular factor loses that
  // much to FP32 rounding, eps32 |X|^T |X| |r| against |X^T X r|) sends the
  // group's FP32 solves through the FP64 factor
  {
    const size_t nvb = std::max<size_t>(nv, 1);
    DevBuf v64, v32, z64, z32, acc;
    if (v64.alloc(nvb * sizeof(double)) != cudaSuccess || v32.alloc(nvb * sizeof(float)) != cudaSuccess ||
        z64.alloc(nvb * sizeof(double)) != cudaSuccess || z32.alloc(nvb * sizeof(float)) != cudaSuccess)
      return HPSE_ERR_OOM;
    CK(acc.alloc(2 * sizeof(double)));
    k_bj_testvec<<<256, 256, 0, s>>>((int64_t)nv, v64.as<double>(), v32.as<float>());
    CK(cudaGetLastError());
    ++g_launches;
    bool any_poor = false;
    for (size_t gi = 0; gi < m->groups.size(); ++gi) {
      const Group &g = m->groups[gi];
      const BjArgs ba = bj_args(m, g, m->n_rhs);
      CK(bj_apply_group<double>(ba, m->d_bj64.as<double>(), v64.as<double>(), m->bj_t64.as<double>(),
                                z64.as<double>(), s, m->bj_var[g.W][0]));
      const hpse_status st = bj_products<float>(m, g, ba, m->d_bj32.as<float>(), v32.as<float>(),
                                                m->bj_t32.as<float>(), z32.as<float>(), s, m->bj_var[g.W][1]);
      if (st != HPSE_OK) return st;
      CK(cudaMemsetAsync(acc.p, 0, 2 * sizeof(double), s));
      k_bj_cmp<<<g.n * m->n_rhs, 128, 0, s>>>(ba, z32.as<float>(), z64.as<double>(), acc.as<double>());
      CK(cudaGetLastError());
      g_launches += 5;
      double h[2] = {0.0, 0.0};
      CK(cudaMemcpyAsync(h, acc.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      const double rel = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : 0.0;
      m->bj_poor32[g.W] = !(rel <= 1e-2);
      any_poor = any_poor || m->bj_poor32[g.W];
      if (verbose())
        fprintf(stderr, "[hpse] block preconditioner W=%d: FP32 products %.2e of FP64%s\n", g.W, rel,
                m->bj_poor32[g.W] ? " (FP32 solves use the FP64 factor)" : "");
    }
    if (any_poor) {
      if (!m->bj_r64.p && m->bj_r64.alloc(nvb * sizeof(double)) != cudaSuccess) return HPSE_ERR_OOM;
      if (!m->bj_z64.p && m->bj_z64.alloc(nvb * sizeof(double)) != cudaSuccess) return HPSE_ERR_OOM;
    }
  }
  m->bj_ready = true;
  m->precond_kind = HPSE_PRECOND_BLOCK;
  return HPSE_OK;
}

extern "C" hpse_status hpse_block_tile(const hpse_mesh *m, int32_t W, int32_t prec, int32_t *variant,
                                       int32_t *tile_rows, int32_t *tile_rhs, float *ms) {
  if (!m || W < 1 || W > HPSE_MAX_W || (prec != HPSE_FP64 && prec != HPSE_FP32)) return HPSE_ERR_INVALID_ARG;
  if (!m->bj_ready) return HPSE_ERR_NO_DATA;
  const int pi = prec == HPSE_FP64 ? 0 : 1, v = m->bj_var[W][pi];
  if (variant) *variant = v;
  if (tile_rows) *tile_rows = BJ_TILE[v][0];
  if (tile_rhs) *tile_rhs = BJ_TILE[v][1];
  if (ms)
    for (int k = 0; k < BJ_NVAR; ++k) ms[k] = m->bj_ms[W][pi][k];
  return HPSE_OK;
}

extern "C" hpse_status hpse_set_block_tile(hpse_mesh *m, int32_t W, int32_t prec, int32_t variant) {
  if (!m || W < 1 || W > HPSE_MAX_W || (prec != HPSE_FP64 && prec != HPSE_FP32)) return HPSE_ERR_INVALID_ARG;
  if (!bj_variant_ok(variant, prec == HPSE_FP32)) return HPSE_ERR_INVALID_ARG;
  if (variant == BJ_TC && !m->d_bjt.p) return HPSE_ERR_INVALID_ARG;
  CK(cudaSetDevice(m->device));
  CK(cudaDeviceSynchronize());
  drop_graphs(m);
  m->bj_var[W][prec == HPSE_FP64 ? 0 : 1] = variant;
  return HPSE_OK;
}

extern "C" hpse_status hpse_select_preconditioner(hpse_mesh *m, int32_t kind) {
  if (!m || (kind != HPSE_PRECOND_SEPARABLE && kind != HPSE_PRECOND_BLOCK)) return HPSE_ERR_INVALID_ARG;
  if (kind == HPSE_PRECOND_BLOCK && !m->bj_ready) return HPSE_ERR_NO_DATA;
  CK(cudaSetDevice(m->device));
  CK(cudaDeviceSynchronize());
  drop_graphs(m);
  m->precond_kind = kind;
  return HPSE_OK;
}

extern "C" hpse_status hpse_set_block_threads(hpse_mesh *m, int32_t kind, int32_t prec, int32_t W, int32_t threads) {
  if (!m || kind < 0 || kind > 1 || (prec != 0 && prec != 1) || W < 1 || W > HPSE_MAX_W) return HPSE_ERR_INVALID_ARG;
  const int maxt = kind == 1 ? 256 : (prec == HPSE_FP64 ? 256 : 384);
  if (threads == 0) threads = default_threads(kind, prec, W);
  if (threads < 32 || threads > maxt || threads % 32) return HPSE_ERR_INVALID_ARG;
  m->threads[kind][prec][W] = threads;
  if (m->work) {
    for (auto &g : m->work->graphs) cudaGraphExecDestroy(g.second);
    m->work->graphs.clear();
  }
  return HPSE_OK;
}

extern "C" int32_t hpse_get_block_threads(const hpse_mesh *m, int32_t kind, int32_t prec, int32_t W) {
  if (!m || kind < 0 || kind > 1 || (prec != 0 && prec != 1) || W < 1 || W > HPSE_MAX_W) return -1;
  return m->threads[kind][prec][W];
}

extern "C" hpse_status hpse_work_counts(const hpse_mesh *m, double *vol_macs, double *face_macs) {
  if (!m) return HPSE_ERR_INVALID_ARG;
  double v = 0.0, f = 0.0;
  const bool var = m->coef_kind == HPSE_COEF_SCALAR, gen = m->coef_kind == HPSE_COEF_GENERAL;
  for (int e = 0; e < m->n_elem; ++e) {
    const double P = m->W[e] + 1, Q = 2 * m->W[e] + 1;
    // forward (n1, n2, n3) = (3,5,5), (2,3,2) or, for the general operator,
    // (3,6,10), and the same for the transpose
    const double n1 = (var || gen) ? 3 : 2, n2 = gen ? 6 : (var ? 5 : 3), n3 = gen ? 10 : (var ? 5 : 2);
    v += 2.0 * (n1 * Q * P * P * P + n2 * Q * Q * P * P + n3 * Q * Q * Q * P);
    for (int fi = 0; fi < 6; ++fi) {
      // traces (2 P^3 + 2 P^3 each side), norms (2 P^3 L2 + 3 x 4 P^3 H^{1/2}), transposes (~3 P^3)
      f += (m->nbr[6 * e + fi] >= 0) ? 23.0 * P * P * P : 15.0 * P * P * P;
    }
  }
  if (vol_macs) *vol_macs = v;
  if (face_macs) *face_macs = f;
  return HPSE_OK;
}

// ---------------------------------------------------------------------------
// PCG driver
// ---------------------------------------------------------------------------
static hpse_status ensure_work(hpse_mesh *m) {
  if (m->work) return HPSE_OK;
  std::unique_ptr<SolverWork> w(new SolverWork());
  const size_t n = (size_t)m->n_rhs * m->ndof;
  w->n = n;
  const size_t d = n * sizeof(double), f = n * sizeof(float);
  CK(w->x64.alloc(d));
  CK(w->r64.alloc(d));
  CK(w->z64.alloc(d));
  CK(w->pa64.alloc(d));
  CK(w->pb64.alloc(d));
  CK(w->q64.alloc(d));
  CK(w->ri64.alloc(d));
  CK(w->x32.alloc(f));
  CK(w->r32.alloc(f));
  CK(w->z32.alloc(f));
  CK(w->pa32.alloc(f));
  CK(w->pb32.alloc(f));
  CK(w->q32.alloc(f));
  const size_t ni = (size_t)std::max(1, n_items_vec(m));
  CK(w->part0.alloc(ni * sizeof(double)));
  CK(w->part1.alloc(ni * sizeof(double)));
  CK(w->part2.alloc(ni * sizeof(double)));
  const int npr = npr_of(m);
  CK(w->sc.alloc((size_t)12 * npr * sizeof(double)));
  CK(w->flags.alloc((size_t)(3 * npr + 1) * sizeof(int32_t)));
  CK(cudaMallocHost(&w->h_flags, (size_t)(3 * npr + 1) * sizeof(int32_t)));
  CK(cudaMallocHost(&w->h_sc, (size_t)12 * npr * sizeof(double)));
  CK(cudaStreamCreateWithFlags(&w->st, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&w->ev, cudaEventDisableTiming));
  m->work = std::move(w);
  return HPSE_OK;
}

// one PCG iteration (apply with fused direction update, alpha, update +
// preconditioner, beta); pin/pout are the ping-pong direction buffers
template <typename T>
static hpse_status pcg_iteration(hpse_mesh *m, T *x, T *r, T *z, T *pin, T *pout, T *q, cudaStream_t s) {
  SolverWork &w = *m->work;
  const int npr = npr_of(m);
  Scalars S = scalars_of(w, npr);
  ApplyArgsT<T> a = apply_args<T>(m, m->groups[0], pin, q);
  a.z = z;
  a.beta = S.beta;
  a.pnew = pout;
  a.partial = w.part0.as<double>();
  hpse_status st = launch_apply_all<T>(m, MODE_PCG, a, s);
  if (st != HPSE_OK) return st;
  k_fin_alpha<<<npr, 128, 0, s>>>(fin_args(m), S, w.part0.as<double>());
  CK(cudaGetLastError());
  ++g_launches;
  PrecArgsT<T> pa = prec_args<T>(m, m->groups[0]);
  pa.x = x;
  pa.r = r;
  pa.p = pout;
  pa.q = q;
  pa.zout = z;
  pa.alpha = S.alpha;
  pa.part_rr = w.part1.as<double>();
  pa.part_rz = w.part2.as<double>();
  st = launch_prec_all<T>(m, MODE_PCG, pa, s);
  if (st != HPSE_OK) return st;
  k_fin_beta<<<npr, 128, 0, s>>>(fin_args(m), S, w.part1.as<double>(), w.part2.as<double>());
  CK(cudaGetLastError());
  ++g_launches;
  return HPSE_OK;
}

// Run PCG on A x = r (x, r, z, pa, pb, q device buffers of type T) starting
// from x = 0, for the (problem, rhs) pairs with scale != 0 (or all when
// scale == nullptr), to relative tolerance rel_tol.  Uses a CUDA graph of
// `chunk` iterations (chunk even) and checks convergence on the host after
// each replay.  Returns the iterations done (max over pairs) in *iters.
template <typename T>
static hpse_status run_pcg(hpse_mesh *m, T *x, T *r, T *z, T *pa, T *pb, T *q, double rel_tol, int max_iter,
                           int chunk, const double *scale, double t_deadline, int *iters, int *status) {
  SolverWork &w = *m->work;
  cudaStream_t s = w.st;
  const int npr = npr_of(m);
  Scalars S = scalars_of(w, npr);
  const size_t nb = w.n * sizeof(T);
  *status = HPSE_OK;
  CK(cudaMemsetAsync(x, 0, nb, s));
  CK(cudaMemsetAsync(pa, 0, nb, s));
  CK(cudaMemsetAsync(S.status, 0, npr * sizeof(int32_t), s));
  // z = C^{-1} r ; rz, rr
  {
    PrecArgsT<T> p = prec_args<T>(m, m->groups[0]);
    p.rin = r;
    p.zout = z;
    hpse_status st = launch_prec_all<T>(m, MODE_PLAIN, p, s);
    if (st != HPSE_OK) return st;
    k_dot<T, T><<<n_items_vec(m), 128, 0, s>>>(elem_args(m), r, z, w.part0.as<double>());
    k_dot<T, T><<<n_items_vec(m), 128, 0, s>>>(elem_args(m), r, r, w.part1.as<double>());
    k_fin_init<<<npr, 128, 0, s>>>(fin_args(m), S, w.part0.as<double>(), w.part1.as<double>(), rel_tol, scale,
                                   0);
    CK(cudaGetLastError());
    g_launches += 3;
  }
  if (chunk < 2) chunk = 2;
  chunk += chunk & 1;
  const long long key = (long long)chunk * 4 + (sizeof(T) == 8 ? 0 : 1) * 2 + (x == (T *)w.x64.p ? 0 : 1);
  cudaGraphExec_t exec = nullptr;
  auto it = w.graphs.find(key);
  if (it == w.graphs.end()) {
    cudaGraph_t graph;
    const long long before = g_launches;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    hpse_status st = HPSE_OK;
    for (int i = 0; i < chunk && st == HPSE_OK; i += 2) {
      st = pcg_iteration<T>(m, x, r, z, pa, pb, q, s);
      if (st == HPSE_OK) st = pcg_iteration<T>(m, x, r, z, pb, pa, q, s);
    }
    if (st == HPSE_OK) {
      k_count_active<<<1, 256, 0, s>>>(S.active, npr, S.n_active);
      ++g_launches;
    }
    cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (st != HPSE_OK) return st;
    CK(ce);
    CK(cudaGraphInstantiate(&exec, graph, 0));
    cudaGraphDestroy(graph);
    w.graphs[key] = exec;
    w.graph_launches[key] = (int)(g_launches - before);
    g_launches = before;
  } else {
    exec = it->second;
  }
  const int per_replay = w.graph_launches[key];
  int done = 0;
  while (true) {
    CK(cudaGraphLaunch(exec, s));
    g_launches += per_replay;
    done += chunk;
    CK(cudaMemcpyAsync(w.h_flags, w.flags.p, (size_t)(3 * npr + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int n_active = w.h_flags[3 * npr];
    if (n_active == 0) break;
    if (done >= max_iter) {
      *status = HPSE_ERR_NO_CONVERGENCE;
      break;
    }
    if (t_deadline > 0) {
      const double now =
          std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
      if (now > t_deadline) {
        *status = HPSE_ERR_TIMEOUT;
        break;
      }
    }
  }
  int mx = 0;
  for (int i = 0; i < npr; ++i) {
    mx = std::max(mx, w.h_flags[npr + i]);
    if (w.h_flags[2 * npr + i] != HPSE_OK && *status == HPSE_OK) *status = w.h_flags[2 * npr + i];
  }
  *iters = mx;
  return HPSE_OK;
}

// r64 = b - A x64 (FP64) and per-pair relative residual / refinement scale
static hpse_status fp64_residual(hpse_mesh *m, const double *x64, double tol, double *rel, double *scale,
                                 double *rnorm, cudaStream_t s) {
  SolverWork &w = *m->work;
  ApplyArgsT<double> a = apply_args<double>(m, m->groups[0], x64, w.q64.as<double>());
  hpse_status st = launch_apply_all<double>(m, MODE_PLAIN, a, s);
  if (st != HPSE_OK) return st;
  k_residual<<<n_items_vec(m), 128, 0, s>>>(elem_args(m), m->d_b.as<double>(), w.q64.as<double>(),
                                           w.r64.as<double>(), w.part0.as<double>());
  k_fin_outer<<<npr_of(m), 128, 0, s>>>(fin_args(m), w.part0.as<double>(), m->d_bnorm2.as<double>(), tol, rel, scale,
                                        rnorm);
  CK(cudaGetLastError());
  g_launches += 2;
  return HPSE_OK;
}

// largest relative residual of the pairs; NaN if any is NaN (a plain
// std::max would drop it and report convergence)
static double max_rel(const double *rel, int npr) {
  double worst = 0.0;
  for (int i = 0; i < npr; ++i)
    if (std::isnan(rel[i]) || rel[i] > worst) worst = rel[i];
  return worst;
}

// PCG with residual refresh ("reliable updates"): one PCG iteration sequence
// with applies, preconditioner and vectors in T (vectors scaled by 1/||b||);
// whenever its recursive residual has dropped by the factor delta since the
// last refresh (delta = 0: only when it claims convergence), the correction is
// added to x in FP64, the true residual b - A x is recomputed with FP64
// applies, and the iteration's residual is replaced by it while the search
// direction is kept.  Stops when the FP64 residual meets ||b - A x|| <= tol ||b||
// for every (problem, rhs).  T = float: FP32 applies + FP64 refinement;
// T = double: FP64 PCG whose stopping test is made on the true residual.
template <typename T>
static hpse_status solve_reliable(hpse_mesh *m, const hpse_solve_opts *o, double *x, hpse_solve_report *rep,
                                  double deadline, double delta, int *status_out) {
  SolverWork &w = *m->work;
  cudaStream_t s = w.st;
  const int npr = npr_of(m);
  Scalars S = scalars_of(w, npr);
  double *sc_rel = w.sc.as<double>() + 8 * npr;
  double *sc_scale = w.sc.as<double>() + 9 * npr;
  double *sc_rnorm = w.sc.as<double>() + 10 * npr;
  double *sc_bn = w.sc.as<double>() + 11 * npr;  // ||b|| per pair, then 1/||b|| in sc_scale
  const int chunk0 = o->check_every > 0 ? o->check_every : 16;
  const int chunk = chunk0 + (chunk0 & 1);
  const size_t nb32 = w.n * sizeof(T);
  const bool dbl = sizeof(T) == 8;
  T *x32 = dbl ? (T *)w.x64.p : (T *)w.x32.p, *r32 = dbl ? (T *)w.ri64.p : (T *)w.r32.p;
  T *z32 = dbl ? (T *)w.z64.p : (T *)w.z32.p, *pa = dbl ? (T *)w.pa64.p : (T *)w.pa32.p;
  T *pb = dbl ? (T *)w.pb64.p : (T *)w.pb32.p, *q32 = dbl ? (T *)w.q64.p : (T *)w.q32.p;
  int status = HPSE_OK, updates = 0, applies = 0;
  // ||b|| and 1/||b|| per pair
  {
    std::vector<double> bn2(npr), bn(npr), ibn(npr);
    CK(cudaMemcpyAsync(bn2.data(), m->d_bnorm2.p, npr * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    bool finite = true;
    for (int i = 0; i < npr; ++i) {
      bn[i] = std::sqrt(bn2[i]);
      ibn[i] = bn[i] > 0 ? 1.0 / bn[i] : 0.0;
      finite = finite && std::isfinite(bn2[i]);
    }
    if (!finite) {
      // a non-finite right-hand side: nothing to iterate on
      rep->rel_residual = std::numeric_limits<double>::quiet_NaN();
      *status_out = HPSE_ERR_BREAKDOWN;
      return HPSE_OK;
    }
    CK(cudaMemcpyAsync(sc_bn, bn.data(), npr * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(sc_scale, ibn.data(), npr * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  // initial residual (x = 0 or the given x) and FP32 state
  if (o->zero_init) {
    CK(cudaMemcpyAsync(w.r64.p, m->d_b.p, w.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    hpse_status st = fp64_residual(m, x, o->tol, sc_rel, sc_rnorm, sc_rnorm, s);
    if (st != HPSE_OK) return st;
    ++applies;
  }
  k_scale_copy<T><<<n_items_vec(m), 128, 0, s>>>(elem_args(m), m->d_prob.as<int32_t>(), m->n_rhs,
                                                 w.r64.as<double>(), sc_scale, r32);
  CK(cudaMemsetAsync(x32, 0, nb32, s));
  CK(cudaMemsetAsync(pa, 0, nb32, s));
  CK(cudaMemsetAsync(S.status, 0, npr * sizeof(int32_t), s));
  {
    PrecArgsT<T> p = prec_args<T>(m, m->groups[0]);
    p.rin = r32;
    p.zout = z32;
    hpse_status st = launch_prec_all<T>(m, MODE_PLAIN, p, s);
    if (st != HPSE_OK) return st;
    k_dot<T, T><<<n_items_vec(m), 128, 0, s>>>(elem_args(m), r32, z32, w.part0.as<double>());
    k_dot<T, T><<<n_items_vec(m), 128, 0, s>>>(elem_args(m), r32, r32, w.part1.as<double>());
    k_fin_init<<<npr, 128, 0, s>>>(fin_args(m), S, w.part0.as<double>(), w.part1.as<double>(), o->tol, sc_scale, 1);
    CK(cudaGetLastError());
    g_launches += 4;
  }
  CK(cudaMemcpyAsync(w.h_sc, w.sc.p, (size_t)12 * npr * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<double> rr_ref(npr);
  for (int i = 0; i < npr; ++i) rr_ref[i] = w.h_sc[2 * npr + i];
  // graph of `chunk` iterations
  const long long key = (long long)chunk * 4 + (dbl ? 0 : 2) + 1;
  cudaGraphExec_t exec = nullptr;
  auto git = w.graphs.find(key);
  if (git == w.graphs.end()) {
    cudaGraph_t graph;
    const long long before = g_launches;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    hpse_status st = HPSE_OK;
    for (int i = 0; i < chunk && st == HPSE_OK; i += 2) {
      st = pcg_iteration<T>(m, x32, r32, z32, pa, pb, q32, s);
      if (st == HPSE_OK) st = pcg_iteration<T>(m, x32, r32, z32, pb, pa, q32, s);
    }
    if (st == HPSE_OK) {
      k_count_active<<<1, 256, 0, s>>>(S.active, npr, S.n_active);
      ++g_launches;
    }
    cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (st != HPSE_OK) return st;
    CK(ce);
    CK(cudaGraphInstantiate(&exec, graph, 0));
    cudaGraphDestroy(graph);
    w.graphs[key] = exec;
    w.graph_launches[key] = (int)(g_launches - before);
    g_launches = before;
  } else {
    exec = git->second;
  }
  const int per_replay = w.graph_launches[key];
  int done = 0;
  double worst = 1.0;
  // stagnation of the true residual at its attainable level (about eps
  // kappa(A) in FP64): the best level reached and the refresh that reached it
  double best = std::numeric_limits<double>::infinity();
  int best_at = 0;
  // stall of the recursive residual between refreshes (it sits at the working
  // precision's level, or a poor low-precision preconditioner stops its
  // descent): no pair's (r, r) has halved below its smallest value in 8
  // graph replays -> refresh early (the true residual then restarts it, and
  // the stagnation rule above ends a solve that cannot improve)
  std::vector<double> rr_min(rr_ref);
  int stalled = 0;
  while (true) {
    CK(cudaGraphLaunch(exec, s));
    g_launches += per_replay;
    done += chunk;
    CK(cudaMemcpyAsync(w.h_flags, w.flags.p, (size_t)(3 * npr + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(w.h_sc, w.sc.p, (size_t)12 * npr * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int n_active = w.h_flags[3 * npr];
    bool refresh = n_active == 0;
    for (int i = 0; i < npr && !refresh; ++i)
      if (w.h_flags[i] && w.h_sc[2 * npr + i] <= delta * delta * rr_ref[i]) refresh = true;
    for (int i = 0; i < npr; ++i)
      if (w.h_flags[2 * npr + i] == HPSE_ERR_BREAKDOWN) refresh = true;
    {
      bool improved = false;
      for (int i = 0; i < npr; ++i) {
        const double rr = w.h_sc[2 * npr + i];
        if (w.h_flags[i] && rr < 0.5 * rr_min[i]) {
          rr_min[i] = rr;
          improved = true;
        }
      }
      stalled = improved ? 0 : stalled + 1;
      if (stalled >= 8) refresh = true;
    }
    const bool capped = done >= o->max_iter || updates >= (o->max_sweeps > 0 ? o->max_sweeps : 200);
    double now = 0.0;
    if (deadline > 0)
      now = std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
    if (refresh || capped || (deadline > 0 && now > deadline)) {
      // x += ||b|| x32 ; x32 = 0 ; r64 = b - A x ; relative residuals
      k_add_scaled<T><<<n_items_vec(m), 128, 0, s>>>(elem_args(m), m->d_prob.as<int32_t>(), m->n_rhs, x32, sc_bn, x);
      CK(cudaGetLastError());
      ++g_launches;
      CK(cudaMemsetAsync(x32, 0, nb32, s));
      hpse_status st = fp64_residual(m, x, o->tol, sc_rel, sc_rnorm, sc_rnorm, s);
      if (st != HPSE_OK) return st;
      ++applies;
      ++updates;
      CK(cudaMemcpyAsync(w.h_sc, w.sc.p, (size_t)12 * npr * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      worst = max_rel(w.h_sc + 8 * npr, npr);
      if (verbose())
        fprintf(stderr, "[hpse] refresh %d after %d %s iterations: max rel residual %.3e\n", updates, done,
                dbl ? "FP64" : "FP32", worst);
      if (!std::isfinite(worst)) {
        status = HPSE_ERR_BREAKDOWN;
        break;
      }
      if (!(worst > o->tol)) break;
      if (capped) {
        status = HPSE_ERR_NO_CONVERGENCE;
        break;
      }
      if (deadline > 0 && now > deadline) {
        status = HPSE_ERR_TIMEOUT;
        break;
      }
      // the true residual has not halved in 16 refreshes: it sits at its
      // attainable level above the tolerance, more iterations cannot help
      if (worst < 0.5 * best) {
        best = worst;
        best_at = updates;
      } else if (updates - best_at >= 16) {
        status = HPSE_ERR_NO_CONVERGENCE;
        break;
      }
      // replace the FP32 residual by the true one, keep the direction
      k_scale_copy<T><<<n_items_vec(m), 128, 0, s>>>(elem_args(m), m->d_prob.as<int32_t>(), m->n_rhs,
                                                     w.r64.as<double>(), sc_scale, r32);
      PrecArgsT<T> p = prec_args<T>(m, m->groups[0]);
      p.rin = r32;
      p.zout = z32;
      st = launch_prec_all<T>(m, MODE_PLAIN, p, s);
      if (st != HPSE_OK) return st;
      k_dot<T, T><<<n_items_vec(m), 128, 0, s>>>(elem_args(m), r32, z32, w.part0.as<double>());
      k_dot<T, T><<<n_items_vec(m), 128, 0, s>>>(elem_args(m), r32, r32, w.part1.as<double>());
      k_fin_reliable<<<npr, 128, 0, s>>>(fin_args(m), S, w.part0.as<double>(), w.part1.as<double>(), sc_rel, o->tol);
      CK(cudaGetLastError());
      g_launches += 4;
      CK(cudaMemsetAsync(S.status, 0, npr * sizeof(int32_t), s));
      CK(cudaMemcpyAsync(w.h_sc, w.sc.p, (size_t)12 * npr * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int i = 0; i < npr; ++i) rr_ref[i] = rr_min[i] = w.h_sc[2 * npr + i];
      stalled = 0;
    }
  }
  int mx = 0;
  CK(cudaMemcpyAsync(w.h_flags, w.flags.p, (size_t)(3 * npr + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int i = 0; i < npr; ++i) mx = std::max(mx, w.h_flags[npr + i]);
  rep->iterations = mx;
  rep->sweeps = updates;
  rep->applies = mx + applies;
  rep->rel_residual = worst;
  *status_out = status;
  return HPSE_OK;
}

extern "C" hpse_status hpse_pcg_solve(hpse_mesh *m, const hpse_solve_opts *o, double *x, hpse_solve_report *rep,
                                      void *stream) {
  if (!m || !o || !rep) return HPSE_ERR_INVALID_ARG;
  memset(rep, 0, sizeof(*rep));
  if (!m->has_data) return HPSE_ERR_NO_DATA;
  if (!(o->tol > 0.0) || o->max_iter < 1 || (o->prec != HPSE_FP64 && o->prec != HPSE_FP32)) return HPSE_ERR_INVALID_ARG;
  if (m->ndof == 0) return HPSE_OK;
  if (!x) return HPSE_ERR_INVALID_ARG;
  CK(cudaSetDevice(m->device));
  hpse_status st = ensure_work(m);
  if (st != HPSE_OK) return st;
  SolverWork &w = *m->work;
  cudaStream_t us = (cudaStream_t)stream;
  cudaStream_t s = w.st;
  // order after the caller's stream
  CK(cudaEventRecord(w.ev, us));
  CK(cudaStreamWaitEvent(s, w.ev, 0));
  const int npr = npr_of(m);
  const size_t nb = w.n * sizeof(double);
  const double t0 = std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
  const double deadline = o->time_limit_s > 0 ? t0 + o->time_limit_s : 0.0;
  const int chunk = o->check_every > 0 ? o->check_every : 16;
  double *sc_rel = w.sc.as<double>() + 8 * npr;
  double *sc_scale = w.sc.as<double>() + 9 * npr;
  double *sc_rnorm = w.sc.as<double>() + 10 * npr;
  int total_it = 0, status = HPSE_OK, sweeps = 0, applies = 0;
  {
    // a non-finite right-hand side (||b||^2 is NaN or inf for some pair) is a
    // breakdown before any iteration, in every mode
    std::vector<double> bn2(npr);
    CK(cudaMemcpyAsync(bn2.data(), m->d_bnorm2.p, npr * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int i = 0; i < npr; ++i)
      if (!std::isfinite(bn2[i])) {
        rep->rel_residual = std::numeric_limits<double>::quiet_NaN();
        rep->status = HPSE_ERR_BREAKDOWN;
        CK(cudaEventRecord(w.ev, s));
        CK(cudaStreamWaitEvent(us, w.ev, 0));
        return HPSE_ERR_BREAKDOWN;
      }
  }
  if (o->zero_init) CK(cudaMemsetAsync(x, 0, nb, s));
  if (o->prec == HPSE_FP64) {
    // FP64 PCG; its convergence claim is checked on the true FP64 residual
    if (o->zero_init) CK(cudaMemsetAsync(x, 0, nb, s));
    st = solve_reliable<double>(m, o, x, rep, deadline, 0.0, &status);
    if (st != HPSE_OK) return st;
    CK(cudaEventRecord(w.ev, s));
    CK(cudaStreamWaitEvent(us, w.ev, 0));
    CK(cudaStreamSynchronize(s));
    rep->status = status;
    return (hpse_status)status;
  } else if (o->refine_mode == 0) {
    if (o->zero_init) CK(cudaMemsetAsync(x, 0, nb, s));
    const double delta = (o->inner_tol > 0 && o->inner_tol < 1) ? o->inner_tol : 1e-1;
    st = solve_reliable<float>(m, o, x, rep, deadline, delta, &status);
    if (st != HPSE_OK) return st;
    CK(cudaEventRecord(w.ev, s));
    CK(cudaStreamWaitEvent(us, w.ev, 0));
    CK(cudaStreamSynchronize(s));
    rep->status = status;
    return (hpse_status)status;
  } else {
    // FP32 operator applies inside FP64 iterative refinement
    const int max_sweeps = o->max_sweeps > 0 ? o->max_sweeps : 20;
    const double itol = o->inner_tol > 0 ? o->inner_tol : 1e-4;
    bool first = o->zero_init != 0;
    while (true) {
      if (first) {
        CK(cudaMemcpyAsync(w.r64.p, m->d_b.p, nb, cudaMemcpyDeviceToDevice, s));
        k_dot<double, double><<<n_items_vec(m), 128, 0, s>>>(elem_args(m), w.r64.as<double>(), w.r64.as<double>(),
                                                             w.part0.as<double>());
        k_fin_outer<<<npr, 128, 0, s>>>(fin_args(m), w.part0.as<double>(), m->d_bnorm2.as<double>(), o->tol, sc_rel,
                                        sc_scale, sc_rnorm);
        CK(cudaGetLastError());
        g_launches += 2;
        first = false;
      } else {
        st = fp64_residual(m, x, o->tol, sc_rel, sc_scale, sc_rnorm, s);
        if (st != HPSE_OK) return st;
        ++applies;
      }
      CK(cudaMemcpyAsync(w.h_sc, w.sc.p, (size_t)12 * npr * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      const double worst = max_rel(w.h_sc + 8 * npr, npr);
      bool any = false;
      for (int i = 0; i < npr; ++i)
        if (w.h_sc[9 * npr + i] != 0.0) any = true;
      rep->rel_residual = worst;
      if (verbose())
        fprintf(stderr, "[hpse] sweep %d: max rel residual %.3e, inner iterations so far %d\n", sweeps, worst,
                total_it);
      if (!std::isfinite(worst)) {
        status = HPSE_ERR_BREAKDOWN;
        break;
      }
      if (!any) break;
      if (sweeps >= max_sweeps || total_it >= o->max_iter) {
        status = HPSE_ERR_NO_CONVERGENCE;
        break;
      }
      // inner FP32 PCG on A d = r64 / ||r64||
      k_scale_to_f32<<<n_items_vec(m), 128, 0, s>>>(elem_args(m), m->d_prob.as<int32_t>(), m->n_rhs,
                                                    w.r64.as<double>(), sc_scale, w.r32.as<float>());
      CK(cudaGetLastError());
      ++g_launches;
      int it = 0, ist = HPSE_OK;
      st = run_pcg<float>(m, w.x32.as<float>(), w.r32.as<float>(), w.z32.as<float>(), w.pa32.as<float>(),
                          w.pb32.as<float>(), w.q32.as<float>(), itol, o->max_iter - total_it, chunk, sc_scale,
                          deadline, &it, &ist);
      if (st != HPSE_OK) return st;
      k_add_scaled_f32<<<n_items_vec(m), 128, 0, s>>>(elem_args(m), m->d_prob.as<int32_t>(), m->n_rhs,
                                                      w.x32.as<float>(), sc_rnorm, x);
      CK(cudaGetLastError());
      ++g_launches;
      total_it += it;
      applies += it;
      ++sweeps;
      if (ist == HPSE_ERR_BREAKDOWN) {
        status = ist;
        break;
      }
      if (ist == HPSE_ERR_TIMEOUT) {
        status = ist;
        break;
      }
    }
  }
  // final FP64 residual for the report (plain FP64 path)
  if (o->prec == HPSE_FP64) {
    st = fp64_residual(m, x, o->tol, sc_rel, sc_scale, sc_rnorm, s);
    if (st != HPSE_OK) return st;
    CK(cudaMemcpyAsync(w.h_sc, w.sc.p, (size_t)12 * npr * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    rep->rel_residual = max_rel(w.h_sc + 8 * npr, npr);
  }
  CK(cudaEventRecord(w.ev, s));
  CK(cudaStreamWaitEvent(us, w.ev, 0));
  CK(cudaStreamSynchronize(s));
  rep->iterations = total_it;
  rep->sweeps = sweeps;
  rep->applies = applies;
  rep->status = status;
  return (hpse_status)status;
}

extern "C" hpse_status hpse_h1_error(hpse_mesh *m, const double *u, const double *ref, const double *vq,
                                     const double *gq, double *out, void *stream) {
  // neighbourhood meshes: the difference of two discrete solutions only
  // (curved elements: both forms, through K and |J| per point)
  if (m && m->coord != HPSE_COORD_CARTESIAN && !m->curved && !ref) return HPSE_ERR_INVALID_ARG;
  if (m && m->curved && !m->has_geometry) return HPSE_ERR_NO_DATA;
  if (!m || !out) return HPSE_ERR_INVALID_ARG;
  if (m->ndof == 0) {
    for (int r = 0; r < m->n_rhs; ++r) out[2 * r] = out[2 * r + 1] = 0.0;
    return HPSE_OK;
  }
  if (!u || (!ref && (!vq || !gq))) return HPSE_ERR_INVALID_ARG;
  CK(cudaSetDevice(m->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int ni = n_items_all(m), nv = n_items_vec(m);
  DevBuf pe, pn, dtabs;
  CK(pe.alloc((size_t)std::max(1, nv) * sizeof(double)));
  CK(pn.alloc((size_t)std::max(1, nv) * sizeof(double)));
  std::vector<const double *> tp(HPSE_MAX_W + 1, nullptr);
  int Wmax = 1;
  for (auto &kv : m->d_qtab) {
    tp[kv.first] = kv.second.as<double>();
    Wmax = std::max(Wmax, kv.first);
  }
  CK(upload(dtabs, tp));
  H1Args A;
  memset(&A, 0, sizeof(A));
  A.n_rhs = m->n_rhs;
  A.ndof = m->ndof;
  A.nquad = m->nquad;
  A.dof_off = m->d_dof_off.as<int64_t>();
  A.coef_off = m->d_coef_off.as<int64_t>();
  A.elem_W = m->d_elem_W.as<int32_t>();
  A.geo = m->d_geo64.as<double>();
  A.qtab = dtabs.as<const double *>();
  A.u = u;
  A.ref = ref;
  A.vq = vq;
  A.gq = gq;
  A.part_err = pe.as<double>();
  A.part_nrm = pn.as<double>();
  A.hw = (m->coord != HPSE_COORD_CARTESIAN && !m->curved) ? m->d_h1w.as<double>() : nullptr;
  A.hc = m->coord == HPSE_COORD_VERTEX_EDGE ? 1.0 : 0.0;
  A.n_elem = m->n_elem;
  A.n_corner = m->n_corner;
  A.cW = m->d_cW.as<int32_t>();
  A.cw = m->d_ch1w.as<double>();
  A.cK = m->curved ? m->d_cKv.as<double>() : nullptr;
  A.cdet = m->curved ? m->d_cdet.as<double>() : nullptr;
  const int P = Wmax + 1, Q = 2 * Wmax + 1;
  const size_t smem = (size_t)(P * P * P + 2 * Q * P * P + 3 * Q * Q * P) * sizeof(double);
  CK(raise_smem((const void *)k_h1, m->device, (size_t)smem));
  k_h1<<<ni, 256, smem, s>>>(A);
  CK(cudaGetLastError());
  ++g_launches;
  if (m->n_corner > 0) {
    k_h1_corner<<<m->n_corner * m->n_rhs, 32, 0, s>>>(A);
    CK(cudaGetLastError());
    ++g_launches;
  }
  std::vector<double> he(nv), hn(nv);
  CK(cudaMemcpyAsync(he.data(), pe.p, (size_t)nv * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hn.data(), pn.p, (size_t)nv * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int r = 0; r < m->n_rhs; ++r) {
    double a = 0.0, b = 0.0;
    for (int e = 0; e < m->n_elem + m->n_corner; ++e) {
      a += he[(size_t)e * m->n_rhs + r];
      b += hn[(size_t)e * m->n_rhs + r];
    }
    out[2 * r] = a;
    out[2 * r + 1] = b;
  }
  return HPSE_OK;
}

// ---------------------------------------------------------------------------
// Residual map, its transpose and adjoint data gradients (FP64).
//
// The volume residual of eq. (4.2) sampled at the (2W+1)^3 GLL points,
//   z_q = sqrt(w_q J) (L u - f)_q,  L u = -a Lap u - grad a . grad u,
// its transpose S^T z, point values and derivatives of a DOF vector, the
// transpose of point evaluation, and the gradient of a solution functional
// J with respect to the data (f, a, grad a) at the points given the adjoint
// state lambda (A lambda = dJ/du):
//   dJ/df = w J L lambda
//   dJ/da = w J [Lap u L lambda + (L u - f) Lap lambda]
//   dJ/d(d_k a) = w J [d_k u L lambda + (L u - f) d_k lambda]
// (differentiate -lambda^T sum_q z_q dz_q/du with respect to each datum).
// ---------------------------------------------------------------------------
template <typename T>
struct FieldArgsT {
  int n_rhs;
  int64_t ndof, nquad;
  const int64_t *dof_off, *coef_off;
  const int32_t *elem_W;
  const double *geo;
  const double *const *qtab;  // per degree: B0, B1 (QxP), DQ, KQ (QxQ), wq (Q), B2 (QxP)
  const T *u;
  T *out;                     // [n_rhs][5][nquad]
};
typedef FieldArgsT<double> FieldArgs;

// (v, v_x, v_y, v_z, Lap v) of a DOF vector at the volume points; one block per (element, rhs)
// point fields in the precision T (FP64 tables rounded to T)
template <typename T>
__global__ void k_fields(FieldArgsT<T> A) {
  extern __shared__ __align__(16) unsigned char fields_raw[];
  T *sm = reinterpret_cast<T *>(fields_raw);
  const int item = blockIdx.x;
  const int e = item / A.n_rhs, r = item - e * A.n_rhs;
  const int W = A.elem_W[e], P = W + 1, Q = 2 * W + 1;
  const double *tb = A.qtab[W];
  const double *B0 = tb, *B1 = tb + Q * P, *B2 = tb + 2 * Q * P + 2 * Q * Q + Q;
  const double *geo = A.geo + (int64_t)e * 4;
  const T sx = (T)geo[0], sy = (T)geo[1], sz = (T)geo[2];
  T *blk = sm, *X0 = blk + P * P * P, *X1 = X0 + Q * P * P, *X2 = X1 + Q * P * P;
  T *Ta = X2 + Q * P * P, *Tb = Ta + Q * Q * P, *Tc = Tb + Q * Q * P;
  const int64_t base = (int64_t)r * A.ndof + A.dof_off[e];
  const int nt = blockDim.x;
  for (int t = threadIdx.x; t < P * P * P; t += nt) blk[t] = A.u[base + t];
  __syncthreads();
  for (int t = threadIdx.x; t < Q * P * P; t += nt) {
    const int qa = t % Q, l = t / Q;
    T a0 = 0, a1 = 0.0, a2 = 0.0;
    for (int i = 0; i < P; ++i) {
      const T v = blk[l * P + i];
      a0 += (T)B0[qa * P + i] * v;
      a1 += (T)B1[qa * P + i] * v;
      a2 += (T)B2[qa * P + i] * v;
    }
    X0[l * Q + qa] = a0;
    X1[l * Q + qa] = a1;
    X2[l * Q + qa] = a2;
  }
  __syncthreads();
  // pass A: T_a = B0y X0, T_b = B1y X0, T_c = B0y X1
  for (int t = threadIdx.x; t < Q * Q * P; t += nt) {
    const int qa = t % Q, qb = (t / Q) % Q, k = t / (Q * Q);
    T a = 0, b = 0.0, c = 0.0;
    for (int j = 0; j < P; ++j) {
      const T x0 = X0[(k * P + j) * Q + qa];
      a += (T)B0[qb * P + j] * x0;
      b += (T)B1[qb * P + j] * x0;
      c += (T)B0[qb * P + j] * X1[(k * P + j) * Q + qa];
    }
    Ta[t] = a;
    Tb[t] = b;
    Tc[t] = c;
  }
  __syncthreads();
  const int64_t ob = (int64_t)r * 5 * A.nquad + A.coef_off[e];
  for (int t = threadIdx.x; t < Q * Q * Q; t += nt) {
    const int qa = t % Q, qb = (t / Q) % Q, qc = t / (Q * Q);
    T v = 0, vz = 0.0, vzz = 0.0, vy = 0.0, vx = 0.0;
    for (int k = 0; k < P; ++k) {
      const int o = (k * Q + qb) * Q + qa;
      v += (T)B0[qc * P + k] * Ta[o];
      vz += (T)B1[qc * P + k] * Ta[o];
      vzz += (T)B2[qc * P + k] * Ta[o];
      vy += (T)B0[qc * P + k] * Tb[o];
      vx += (T)B0[qc * P + k] * Tc[o];
    }
    A.out[ob + t] = v;
    A.out[ob + A.nquad + t] = sx * vx;
    A.out[ob + 2 * A.nquad + t] = sy * vy;
    A.out[ob + 3 * A.nquad + t] = sz * vz;
    A.out[ob + 4 * A.nquad + t] = sz * sz * vzz;
  }
  __syncthreads();
  // pass B: T_a = B2y X0 (u_yy), T_b = B0y X2 (u_xx)
  for (int t = threadIdx.x; t < Q * Q * P; t += nt) {
    const int qa = t % Q, qb = (t / Q) % Q, k = t / (Q * Q);
    T a = 0, b = 0.0;
    for (int j = 0; j < P; ++j) {
      a += (T)B2[qb * P + j] * X0[(k * P + j) * Q + qa];
      b += (T)B0[qb * P + j] * X2[(k * P + j) * Q + qa];
    }
    Ta[t] = a;
    Tb[t] = b;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < Q * Q * Q; t += nt) {
    const int qa = t % Q, qb = (t / Q) % Q, qc = t / (Q * Q);
    T vyy = 0, vxx = 0.0;
    for (int k = 0; k < P; ++k) {
      const int o = (k * Q + qb) * Q + qa;
      vyy += (T)B0[qc * P + k] * Ta[o];
      vxx += (T)B0[qc * P + k] * Tb[o];
    }
    A.out[ob + 4 * A.nquad + t] += sy * sy * vyy + sx * sx * vxx;
  }
}

// y = sum_q rho_q d v(x_q) / dV (transpose of point evaluation); one block per (element, rhs)
__global__ void k_eval_T(FieldArgs A, const double *rho) {
  extern __shared__ double sm[];
  const int item = blockIdx.x;
  const int e = item / A.n_rhs, r = item - e * A.n_rhs;
  const int W = A.elem_W[e], P = W + 1, Q = 2 * W + 1;
  const double *B0 = A.qtab[W];
  double *R = sm, *T = R + Q * Q * Q, *X = T + Q * Q * P;
  const int nt = blockDim.x;
  const int64_t qb0 = (int64_t)r * A.nquad + A.coef_off[e];
  for (int t = threadIdx.x; t < Q * Q * Q; t += nt) R[t] = rho[qb0 + t];
  __syncthreads();
  for (int t = threadIdx.x; t < Q * Q * P; t += nt) {  // T[k][qb][qa]
    const int qa = t % Q, qb = (t / Q) % Q, k = t / (Q * Q);
    double s = 0.0;
    for (int qc = 0; qc < Q; ++qc) s += B0[qc * P + k] * R[(qc * Q + qb) * Q + qa];
    T[t] = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < Q * P * P; t += nt) {  // X[k][j][qa]
    const int qa = t % Q, j = (t / Q) % P, k = t / (Q * P);
    double s = 0.0;
    for (int qb = 0; qb < Q; ++qb) s += B0[qb * P + j] * T[(k * Q + qb) * Q + qa];
    X[t] = s;
  }
  __syncthreads();
  const int64_t base = (int64_t)r * A.ndof + A.dof_off[e];
  for (int t = threadIdx.x; t < P * P * P; t += nt) {
    const int i = t % P, l = t / P;
    double s = 0.0;
    for (int qa = 0; qa < Q; ++qa) s += B0[qa * P + i] * X[l * Q + qa];
    A.out[base + t] = s;
  }
}

// y = sum_q sum_k wf[r][k][q] (field_k v)(x_q) / dV: the transpose of
// hpse_eval_fields (fields v, v_x, v_y, v_z, Lap v); one block per (element,
// rhs).  The seven tensor terms (x, y, z matrices and scale) are transposed
// one after the other through the three stages of k_eval_T and summed.
__global__ void k_fields_T(FieldArgs A, const double *wf) {
  extern __shared__ double sm[];
  const int item = blockIdx.x;
  const int e = item / A.n_rhs, r = item - e * A.n_rhs;
  const int W = A.elem_W[e], P = W + 1, Q = 2 * W + 1;
  const double *B[3] = {A.qtab[W], A.qtab[W] + Q * P, A.qtab[W] + 2 * Q * P + 2 * Q * Q + Q};
  double *R = sm, *T = R + Q * Q * Q, *X = T + Q * Q * P, *Y = X + Q * P * P;
  const int nt = blockDim.x;
  const double *gs = A.geo + 4 * (int64_t)e;
  const int64_t nq = A.nquad;
  const int64_t qb0 = (int64_t)r * 5 * nq + A.coef_off[e];
  for (int t = threadIdx.x; t < P * P * P; t += nt) Y[t] = 0.0;
  // term: field, matrix orders along (x, y, z), scale
  const int fld[7] = {0, 1, 2, 3, 4, 4, 4};
  const int mx[7] = {0, 1, 0, 0, 2, 0, 0}, my[7] = {0, 0, 1, 0, 0, 2, 0}, mz[7] = {0, 0, 0, 1, 0, 0, 2};
  for (int term = 0; term < 7; ++term) {
    const double sc = term == 0 ? 1.0 : (term < 4 ? gs[term - 1] : gs[term - 4] * gs[term - 4]);
    const double *Mx = B[mx[term]], *My = B[my[term]], *Mz = B[mz[term]];
    __syncthreads();
    for (int t = threadIdx.x; t < Q * Q * Q; t += nt) R[t] = sc * wf[qb0 + fld[term] * nq + t];
    __syncthreads();
    for (int t = threadIdx.x; t < Q * Q * P; t += nt) {  // T[k][qb][qa]
      const int qa = t % Q, qb = (t / Q) % Q, k = t / (Q * Q);
      double s = 0.0;
      for (int qc = 0; qc < Q; ++qc) s += Mz[qc * P + k] * R[(qc * Q + qb) * Q + qa];
      T[t] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < Q * P * P; t += nt) {  // X[k][j][qa]
      const int qa = t % Q, j = (t / Q) % P, k = t / (Q * P);
      double s = 0.0;
      for (int qb = 0; qb < Q; ++qb) s += My[qb * P + j] * T[(k * Q + qb) * Q + qa];
      X[t] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < P * P * P; t += nt) {
      const int i = t % P, l = t / P;
      double s = 0.0;
      for (int qa = 0; qa < Q; ++qa) s += Mx[qa * P + i] * X[l * Q + qa];
      Y[t] += s;
    }
  }
  __syncthreads();
  const int64_t base = (int64_t)r * A.ndof + A.dof_off[e];
  for (int t = threadIdx.x; t < P * P * P; t += nt) A.out[base + t] = Y[t];
}

// residual map at the points: z = sqrt(wJ) (L u - f)
template <typename T>
__global__ void k_resid_points(int64_t nquad, int n_rhs, const double *aux, const double *f, const T *fields,
                               T *z) {
  const int64_t n = nquad * n_rhs;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / nquad, q = i - r * nquad;
    const T *fl = fields + r * 5 * nquad;
    const T wJ = (T)aux[q], a = (T)aux[nquad + q];
    const T Lu = -a * fl[4 * nquad + q] -
                 ((T)aux[2 * nquad + q] * fl[nquad + q] + (T)aux[3 * nquad + q] * fl[2 * nquad + q] +
                  (T)aux[4 * nquad + q] * fl[3 * nquad + q]);
    z[i] = sqrt(wJ) * (Lu - (T)f[i]);
  }
}

// rho = -sqrt(wJ) a z: the weights of S^T z in the sum-factorised transpose kernel
template <typename T>
__global__ void k_rho_from_z(int64_t nquad, int n_rhs, const double *aux, const T *z, double *rho) {
  const int64_t n = nquad * n_rhs;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = i % nquad;
    rho[i] = (double)(-sqrt((T)aux[q]) * (T)aux[nquad + q] * z[i]);
  }
}

// adjoint data gradient at the points
__global__ void k_data_grad(int64_t nquad, int n_rhs, const double *aux, const double *f, const double *uf,
                            const double *lf, double *out) {
  const int64_t n = nquad * n_rhs;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / nquad, q = i - r * nquad;
    const double *u = uf + r * 5 * nquad, *l = lf + r * 5 * nquad;
    const double wJ = aux[q], a = aux[nquad + q];
    const double ax = aux[2 * nquad + q], ay = aux[3 * nquad + q], az = aux[4 * nquad + q];
    const double ux = u[nquad + q], uy = u[2 * nquad + q], uz = u[3 * nquad + q], lu = u[4 * nquad + q];
    const double lx = l[nquad + q], ly = l[2 * nquad + q], lz = l[3 * nquad + q], ll = l[4 * nquad + q];
    const double Lu = -a * lu - (ax * ux + ay * uy + az * uz);
    const double Ll = -a * ll - (ax * lx + ay * ly + az * lz);
    const double res = f ? Lu - f[i] : Lu;
    double *o = out + r * 5 * nquad;
    o[q] = wJ * Ll;
    o[nquad + q] = wJ * (lu * Ll + res * ll);
    o[2 * nquad + q] = wJ * (ux * Ll + res * lx);
    o[3 * nquad + q] = wJ * (uy * Ll + res * ly);
    o[4 * nquad + q] = wJ * (uz * Ll + res * lz);
  }
}

// Vector-Jacobian product of k_data_grad at every point: given the cotangent
// ob[r][0..4][q] of its output, the cotangents of its inputs -- the fields of
// u (ub) and of lambda (lb), [r][0..4][q], and the data db[r][0..4][q] = (f,
// a, d_x a, d_y a, d_z a) per rhs (a and grad a are shared by the rhs: the
// caller sums db over r for them).  With f == nullptr the residual is L u (the
// bilinear form -d/dtheta lambda^T A u) and db[.][0] is zero.
//   c_L = wJ (ob0 + ob1 Lap u + ob2 u_x + ob3 u_y + ob4 u_z)   (d out / d L lambda)
//   c_R = wJ (ob1 Lap l + ob2 l_x + ob3 l_y + ob4 l_z)         (d out / d res)
__global__ void k_data_grad_vjp(int64_t nquad, int n_rhs, const double *aux, const double *f, const double *uf,
                                const double *lf, const double *ob, double *ub, double *lb, double *db) {
  const int64_t n = nquad * n_rhs;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / nquad, q = i - r * nquad;
    const int64_t o5 = r * 5 * nquad + q;
    const double *u = uf + o5, *l = lf + o5, *g = ob + o5;
    const double wJ = aux[q], a = aux[nquad + q];
    const double ad[3] = {aux[2 * nquad + q], aux[3 * nquad + q], aux[4 * nquad + q]};
    const double ud[3] = {u[nquad], u[2 * nquad], u[3 * nquad]}, lu = u[4 * nquad];
    const double ld[3] = {l[nquad], l[2 * nquad], l[3 * nquad]}, ll = l[4 * nquad];
    const double Lu = -a * lu - (ad[0] * ud[0] + ad[1] * ud[1] + ad[2] * ud[2]);
    const double Ll = -a * ll - (ad[0] * ld[0] + ad[1] * ld[1] + ad[2] * ld[2]);
    const double res = f ? Lu - f[i] : Lu;
    const double cL = wJ * (g[0] + g[nquad] * lu + g[2 * nquad] * ud[0] + g[3 * nquad] * ud[1] + g[4 * nquad] * ud[2]);
    const double cR = wJ * (g[nquad] * ll + g[2 * nquad] * ld[0] + g[3 * nquad] * ld[1] + g[4 * nquad] * ld[2]);
    double *uo = ub + o5, *lo = lb + o5, *dd = db + o5;
    uo[0] = 0.0;
    lo[0] = 0.0;
    uo[4 * nquad] = wJ * Ll * g[nquad] - a * cR;
    lo[4 * nquad] = wJ * res * g[nquad] - a * cL;
    for (int k = 0; k < 3; ++k) {
      uo[(1 + k) * nquad] = wJ * Ll * g[(2 + k) * nquad] - ad[k] * cR;
      lo[(1 + k) * nquad] = wJ * res * g[(2 + k) * nquad] - ad[k] * cL;
      dd[(2 + k) * nquad] = -ld[k] * cL - ud[k] * cR;
    }
    dd[0] = f ? -cR : 0.0;
    dd[nquad] = -ll * cL - lu * cR;
  }
}

template <typename T = double>
static FieldArgsT<T> field_args(const hpse_mesh *m, const T *u, T *out) {
  FieldArgsT<T> A;
  A.n_rhs = m->n_rhs;
  A.ndof = m->ndof;
  A.nquad = m->nquad;
  A.dof_off = m->d_dof_off.as<int64_t>();
  A.coef_off = m->d_coef_off.as<int64_t>();
  A.elem_W = m->d_elem_W.as<int32_t>();
  A.geo = m->d_geo64.as<double>();
  A.qtab = m->d_tabs_ptr.as<const double *>();
  A.u = u;
  A.out = out;
  return A;
}

static int max_degree(const hpse_mesh *m) {
  int w = 1;
  for (auto &kv : m->d_qtab) w = std::max(w, kv.first);
  return w;
}

template <typename T = double>
static hpse_status launch_fields(hpse_mesh *m, const T *u, T *out, cudaStream_t s) {
  const int W = max_degree(m), P = W + 1, Q = 2 * W + 1;
  const size_t smem = (size_t)(P * P * P + 3 * Q * P * P + 3 * Q * Q * P) * sizeof(T);
  CK(raise_smem((const void *)k_fields<T>, m->device, (size_t)smem));
  k_fields<T><<<n_items_all(m), 256, smem, s>>>(field_args<T>(m, u, out));
  CK(cudaGetLastError());
  ++g_launches;
  return HPSE_OK;
}

extern "C" hpse_status hpse_eval_fields(hpse_mesh *m, const double *u, double *out, void *stream) {
  // box meshes of the Laplacian or -div(a grad u) only
  if (m && (m->coord != HPSE_COORD_CARTESIAN || m->coef_kind == HPSE_COEF_GENERAL)) return HPSE_ERR_INVALID_ARG;
  if (!m) return HPSE_ERR_INVALID_ARG;
  if (m->ndof == 0) return HPSE_OK;
  if (!u || !out) return HPSE_ERR_INVALID_ARG;
  if (!m->has_data) return HPSE_ERR_NO_DATA;
  CK(cudaSetDevice(m->device));
  return launch_fields(m, u, out, (cudaStream_t)stream);
}

extern "C" hpse_status hpse_apply_eval_transpose(hpse_mesh *m, const double *rho, double *y, void *stream) {
  // box meshes of the Laplacian or -div(a grad u) only
  if (m && (m->coord != HPSE_COORD_CARTESIAN || m->coef_kind == HPSE_COEF_GENERAL)) return HPSE_ERR_INVALID_ARG;
  if (!m) return HPSE_ERR_INVALID_ARG;
  if (m->ndof == 0) return HPSE_OK;
  if (!rho || !y) return HPSE_ERR_INVALID_ARG;
  if (!m->has_data) return HPSE_ERR_NO_DATA;
  CK(cudaSetDevice(m->device));
  const int W = max_degree(m), P = W + 1, Q = 2 * W + 1;
  const size_t smem = (size_t)(Q * Q * Q + Q * Q * P + Q * P * P) * sizeof(double);
  CK(raise_smem((const void *)k_eval_T, m->device, (size_t)smem));
  k_eval_T<<<n_items_all(m), 256, smem, (cudaStream_t)stream>>>(field_args<double>(m, nullptr, y), rho);
  CK(cudaGetLastError());
  ++g_launches;
  return HPSE_OK;
}

extern "C" hpse_status hpse_apply_fields_transpose(hpse_mesh *m, const double *wf, double *y, void *stream) {
  // box meshes of the Laplacian or -div(a grad u) only
  if (m && (m->coord != HPSE_COORD_CARTESIAN || m->coef_kind == HPSE_COEF_GENERAL)) return HPSE_ERR_INVALID_ARG;
  if (!m) return HPSE_ERR_INVALID_ARG;
  if (m->ndof == 0) return HPSE_OK;
  if (!wf || !y) return HPSE_ERR_INVALID_ARG;
  if (!m->has_data) return HPSE_ERR_NO_DATA;
  CK(cudaSetDevice(m->device));
  const int W = max_degree(m), P = W + 1, Q = 2 * W + 1;
  const size_t smem = (size_t)(Q * Q * Q + Q * Q * P + Q * P * P + P * P * P) * sizeof(double);
  CK(raise_smem((const void *)k_fields_T, m->device, (size_t)smem));
  k_fields_T<<<n_items_all(m), 256, smem, (cudaStream_t)stream>>>(field_args<double>(m, nullptr, y), wf);
  CK(cudaGetLastError());
  ++g_launches;
  return HPSE_OK;
}

extern "C" hpse_status hpse_quad_weights(hpse_mesh *m, double *out, void *stream) {
  if (m && m->coord != HPSE_COORD_CARTESIAN) return HPSE_ERR_INVALID_ARG;  // box meshes only
  if (!m || (!out && m->nquad > 0)) return HPSE_ERR_INVALID_ARG;
  if (!m->has_data) return HPSE_ERR_NO_DATA;
  CK(cudaSetDevice(m->device));
  if (m->nquad)
    CK(cudaMemcpyAsync(out, m->d_aux.p, (size_t)m->nquad * sizeof(double), cudaMemcpyDeviceToDevice,
                       (cudaStream_t)stream));
  return HPSE_OK;
}

static hpse_status ensure_scratch(hpse_mesh *m, size_t fbytes) {
  const size_t nf = (size_t)5 * m->n_rhs * m->nquad * fbytes;
  const size_t nr = (size_t)m->n_rhs * m->nquad * sizeof(double);
  if (m->d_scr_fields.bytes < nf) CK(m->d_scr_fields.alloc(nf));
  if (m->d_scr_rho.bytes != nr) CK(m->d_scr_rho.alloc(nr));
  return HPSE_OK;
}

template <typename T>
static hpse_status residual_t(hpse_mesh *m, const T *u, T *z, cudaStream_t s) {
  hpse_status st = ensure_scratch(m, sizeof(T));
  if (st != HPSE_OK) return st;
  st = launch_fields<T>(m, u, (T *)m->d_scr_fields.p, s);
  if (st != HPSE_OK) return st;
  k_resid_points<T><<<1024, 256, 0, s>>>(m->nquad, m->n_rhs, m->d_aux.as<double>(), m->d_f.as<double>(),
                                         (const T *)m->d_scr_fields.p, z);
  CK(cudaGetLastError());
  ++g_launches;
  return HPSE_OK;
}

extern "C" hpse_status hpse_apply_residual(hpse_mesh *m, int32_t prec, const void *u, void *z, void *stream) {
  // box meshes of the Laplacian or -div(a grad u) only
  if (m && (m->coord != HPSE_COORD_CARTESIAN || m->coef_kind == HPSE_COEF_GENERAL)) return HPSE_ERR_INVALID_ARG;
  if (!m || (prec != HPSE_FP64 && prec != HPSE_FP32)) return HPSE_ERR_INVALID_ARG;
  if (m->ndof == 0) return HPSE_OK;
  if (!u || !z) return HPSE_ERR_INVALID_ARG;
  if (!m->has_data) return HPSE_ERR_NO_DATA;
  CK(cudaSetDevice(m->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == HPSE_FP64) return residual_t<double>(m, (const double *)u, (double *)z, s);
  return residual_t<float>(m, (const float *)u, (float *)z, s);
}

template <typename T>
static hpse_status transpose_t(hpse_mesh *m, const T *z, T *y, cudaStream_t s) {
  hpse_status st = ensure_scratch(m, sizeof(double));
  if (st != HPSE_OK) return st;
  k_rho_from_z<T><<<1024, 256, 0, s>>>(m->nquad, m->n_rhs, m->d_aux.as<double>(), z, m->d_scr_rho.as<double>());
  CK(cudaGetLastError());
  ++g_launches;
  ApplyArgsT<T> a = apply_args<T>(m, m->groups[0], nullptr, y);
  a.rho = m->d_scr_rho.as<double>();
  a.skip_faces = 1;
  return launch_apply_all<T>(m, MODE_TRANSPOSE, a, s);
}

extern "C" hpse_status hpse_apply_transpose(hpse_mesh *m, int32_t prec, const void *z, void *y, void *stream) {
  // box meshes of the Laplacian or -div(a grad u) only
  if (m && (m->coord != HPSE_COORD_CARTESIAN || m->coef_kind == HPSE_COEF_GENERAL)) return HPSE_ERR_INVALID_ARG;
  if (!m || (prec != HPSE_FP64 && prec != HPSE_FP32)) return HPSE_ERR_INVALID_ARG;
  if (m->ndof == 0) return HPSE_OK;
  if (!z || !y) return HPSE_ERR_INVALID_ARG;
  if (!m->has_data) return HPSE_ERR_NO_DATA;
  CK(cudaSetDevice(m->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == HPSE_FP64) return transpose_t<double>(m, (const double *)z, (double *)y, s);
  return transpose_t<float>(m, (const float *)z, (float *)y, s);
}

// the volume transpose in integration-by-parts form (eq. 5.45-5.48), per degree group
template <typename T>
static hpse_status transpose_ibp_t(hpse_mesh *m, const T *z, T *y, cudaStream_t s) {
  hpse_status st = ensure_scratch(m, sizeof(double));
  if (st != HPSE_OK) return st;
  k_rho_from_z<T><<<1024, 256, 0, s>>>(m->nquad, m->n_rhs, m->d_aux.as<double>(), z, m->d_scr_rho.as<double>());
  CK(cudaGetLastError());
  ++g_launches;
  const int pi = sizeof(T) == 8 ? 0 : 1;
  ApplyArgsT<T> base = apply_args<T>(m, m->groups[0], nullptr, y);
  base.rho = m->d_scr_rho.as<double>();
  base.skip_faces = 1;
  CK(group_fork(m, s));
  for (size_t gi = 0; gi < m->groups.size(); ++gi) {
    const Group &g = m->groups[gi];
    ApplyArgsT<T> a = base;
    a.elems = g.elems.as<int32_t>();
    a.n_group = g.n;
    CK(g_sets[pi][g.W].transpose_ibp(m->apply_coef, &a, g.n * m->n_rhs, group_stream(m, gi, s)));
    ++g_launches;
  }
  CK(group_join(m, s));
  return HPSE_OK;
}

extern "C" hpse_status hpse_apply_transpose_ibp(hpse_mesh *m, int32_t prec, const void *z, void *y, void *stream) {
  // box meshes of the Laplacian or -div(a grad u) only
  if (m && (m->coord != HPSE_COORD_CARTESIAN || m->coef_kind == HPSE_COEF_GENERAL)) return HPSE_ERR_INVALID_ARG;
  if (!m || (prec != HPSE_FP64 && prec != HPSE_FP32)) return HPSE_ERR_INVALID_ARG;
  if (m->ndof == 0) return HPSE_OK;
  if (!z || !y) return HPSE_ERR_INVALID_ARG;
  if (!m->has_data) return HPSE_ERR_NO_DATA;
  const int pi = prec == HPSE_FP64 ? 0 : 1;
  for (const Group &g : m->groups)
    if (g_sets[pi][g.W].ibp_smem(m->apply_coef) == 0) return HPSE_ERR_DEGREE;
  CK(cudaSetDevice(m->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == HPSE_FP64) return transpose_ibp_t<double>(m, (const double *)z, (double *)y, s);
  return transpose_ibp_t<float>(m, (const float *)z, (float *)y, s);
}

extern "C" hpse_status hpse_data_gradient(hpse_mesh *m, const double *ufields, const double *lfields, double *out,
                                          void *stream) {
  // box meshes of the Laplacian or -div(a grad u) only
  if (m && (m->coord != HPSE_COORD_CARTESIAN || m->coef_kind == HPSE_COEF_GENERAL)) return HPSE_ERR_INVALID_ARG;
  if (!m) return HPSE_ERR_INVALID_ARG;
  if (m->nquad == 0) return HPSE_OK;
  if (!ufields || !lfields || !out) return HPSE_ERR_INVALID_ARG;
  if (!m->has_data) return HPSE_ERR_NO_DATA;
  CK(cudaSetDevice(m->device));
  k_data_grad<<<1024, 256, 0, (cudaStream_t)stream>>>(m->nquad, m->n_rhs, m->d_aux.as<double>(), m->d_f.as<double>(),
                                                      ufields, lfields, out);
  CK(cudaGetLastError());
  ++g_launches;
  return HPSE_OK;
}

extern "C" hpse_status hpse_data_gradient_bilinear(hpse_mesh *m, const double *ufields, const double *lfields,
                                                   double *out, void *stream) {
  // box meshes of the Laplacian or -div(a grad u) only
  if (m && (m->coord != HPSE_COORD_CARTESIAN || m->coef_kind == HPSE_COEF_GENERAL)) return HPSE_ERR_INVALID_ARG;
  if (!m) return HPSE_ERR_INVALID_ARG;
  if (m->nquad == 0) return HPSE_OK;
  if (!ufields || !lfields || !out) return HPSE_ERR_INVALID_ARG;
  if (!m->has_data) return HPSE_ERR_NO_DATA;
  CK(cudaSetDevice(m->device));
  k_data_grad<<<1024, 256, 0, (cudaStream_t)stream>>>(m->nquad, m->n_rhs, m->d_aux.as<double>(), nullptr, ufields,
                                                      lfields, out);
  CK(cudaGetLastError());
  ++g_launches;
  return HPSE_OK;
}

extern "C" hpse_status hpse_data_gradient_vjp(hpse_mesh *m, int32_t with_f, const double *ufields,
                                              const double *lfields, const double *obar, double *ubar, double *lbar,
                                              double *dbar, void *stream) {
  // box meshes of the Laplacian or -div(a grad u) only
  if (m && (m->coord != HPSE_COORD_CARTESIAN || m->coef_kind == HPSE_COEF_GENERAL)) return HPSE_ERR_INVALID_ARG;
  if (!m || (with_f != 0 && with_f != 1)) return HPSE_ERR_INVALID_ARG;
  if (m->nquad == 0) return HPSE_OK;
  if (!ufields || !lfields || !obar || !ubar || !lbar || !dbar) return HPSE_ERR_INVALID_ARG;
  if (!m->has_data) return HPSE_ERR_NO_DATA;
  CK(cudaSetDevice(m->device));
  k_data_grad_vjp<<<1024, 256, 0, (cudaStream_t)stream>>>(m->nquad, m->n_rhs, m->d_aux.as<double>(),
                                                          with_f ? m->d_f.as<double>() : nullptr, ufields, lfields,
                                                          obar, ubar, lbar, dbar);
  CK(cudaGetLastError());
  ++g_launches;
  return HPSE_OK;
}

extern "C" hpse_status hpse_set_rhs(hpse_mesh *m, const double *b, void *stream) {
  if (!m) return HPSE_ERR_INVALID_ARG;
  if (!m->has_data) return HPSE_ERR_NO_DATA;
  if (m->ndof == 0) return HPSE_OK;
  if (!b) return HPSE_ERR_INVALID_ARG;
  CK(cudaSetDevice(m->device));
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nv = (size_t)m->n_rhs * m->ndof;
  CK(cudaMemcpyAsync(m->d_b.p, b, nv * sizeof(double), cudaMemcpyDeviceToDevice, s));
  DevBuf part;
  CK(part.alloc((size_t)std::max(1, n_items_vec(m)) * sizeof(double)));
  k_dot<double, double><<<n_items_vec(m), 128, 0, s>>>(elem_args(m), m->d_b.as<double>(), m->d_b.as<double>(),
                                                       part.as<double>());
  k_bnorm<<<npr_of(m), 128, 0, s>>>(fin_args(m), part.as<double>(), m->d_bnorm2.as<double>());
  CK(cudaGetLastError());
  g_launches += 2;
  CK(cudaStreamSynchronize(s));
  return HPSE_OK;
}


// ---------------------------------------------------------------------------
// H^1 norms without device allocation.
//
// Some callers cannot call cudaMalloc: applications whose device memory is
// owned entirely by another allocator (a framework's caching allocator or a
// fixed arena reserved at start-up), and latency-critical loops that must not
// trigger the device-wide synchronisation cudaFree implies.  This variant of
// hpse_h1_error keeps its scratch -- the per-(element, rhs) partial sums, the
// per-rhs results and the table-pointer array -- in the file-scope array
// below, which every GPU that loads this library holds until exit
// (HPSE_NOALLOC_BYTES of it).  Host code reaches that array only through the
// address cudaGetSymbolAddress returns for the current device (the array's
// name in host code is a host-side stand-in, not a device address).
// ---------------------------------------------------------------------------
#define HPSE_NOALLOC_MAX_ITEMS (1 << 17)  // n_elem * n_rhs
#define HPSE_NOALLOC_MAX_RHS 4096
#define HPSE_NOALLOC_MAX_DEVICES 64
#define HPSE_NOALLOC_DOUBLES (2 * HPSE_NOALLOC_MAX_ITEMS + 2 * HPSE_NOALLOC_MAX_RHS + 16)
// ---------------------------------------------------------------------------
// Conforming correction (Remark 4.3.0; the construction in the proof of Lemma
// 3.3.1, Appendix C.1) of box-element solutions, on the nodal values:
//   1. delta: trilinear, (u + delta) = the average of u at every element vertex
//      over the elements sharing it (0 on the Dirichlet boundary);
//   2. epsilon: per element edge the average of u + delta along it minus the
//      own trace, blended bilinearly in the other two variables;
//   3. nu: per face the average of the two traces of u + delta + epsilon
//      (0 on a Dirichlet face) minus the own trace, blended linearly in the
//      normal variable.
// Each correction is degree one in the blended variables, so p stays in the
// element's (W+1)^3 nodal space.  One CTA per (element, rhs) in each stage.
// ---------------------------------------------------------------------------
struct ConfArgs {
  int n_rhs;
  int64_t ndof;
  const int64_t *dof_off;
  const int32_t *elem_W, *nbr;
  const int32_t *vid, *vptr, *vmem, *vdir;  // vertex id per (element, corner), members (element * 8 + corner)
  const int32_t *eid, *eptr, *emem, *edir;  // edge id per (element, edge), members (element * 12 + edge)
  const double *const *lin;                 // per degree: (1 - x)/2 then (1 + x)/2 at the P GLL nodes
  const int32_t *fbc;                       // outer-face conditions (null: all Dirichlet)
};

// node (i, j, k) of corner c (bit a of c: the side along axis a)
__device__ __forceinline__ int conf_corner_node(int c, int P) {
  const int i = (c & 1) ? P - 1 : 0, j = ((c >> 1) & 1) ? P - 1 : 0, k = ((c >> 2) & 1) ? P - 1 : 0;
  return (k * P + j) * P + i;
}
// node t of element edge k = 4 a + s1 + 2 s2 (along axis a; s1, s2 the sides
// of the other two axes in increasing order)
__device__ __forceinline__ int conf_edge_node(int k, int t, int P) {
  const int a = k >> 2, s1 = k & 1, s2 = (k >> 1) & 1;
  int c[3];
  const int o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
  c[a] = t;
  c[o1] = s1 ? P - 1 : 0;
  c[o2] = s2 ? P - 1 : 0;
  return (c[2] * P + c[1]) * P + c[0];
}

__global__ void k_conf_vertex(ConfArgs A, const double *u, double *w) {
  __shared__ double d[8];
  const int e = blockIdx.x / A.n_rhs, r = blockIdx.x - e * A.n_rhs;
  const int P = A.elem_W[e] + 1;
  const int64_t rb = (int64_t)r * A.ndof;
  if (threadIdx.x < 8) {
    const int c = threadIdx.x, g = A.vid[e * 8 + c];
    double t = 0.0;
    if (!A.vdir[g]) {
      for (int m = A.vptr[g]; m < A.vptr[g + 1]; ++m) {
        const int em = A.vmem[m] >> 3, cm = A.vmem[m] & 7;
        t += u[rb + A.dof_off[em] + conf_corner_node(cm, A.elem_W[em] + 1)];
      }
      t /= (double)(A.vptr[g + 1] - A.vptr[g]);
    }
    d[c] = t - u[rb + A.dof_off[e] + conf_corner_node(c, P)];
  }
  __syncthreads();
  const double *L = A.lin[P - 1];
  const int64_t base = rb + A.dof_off[e];
  for (int t = threadIdx.x; t < P * P * P; t += blockDim.x) {
    const int i = t % P, j = (t / P) % P, k = t / (P * P);
    double s = u[base + t];
    for (int c = 0; c < 8; ++c)
      s += d[c] * L[(c & 1) * P + i] * L[((c >> 1) & 1) * P + j] * L[((c >> 2) & 1) * P + k];
    w[base + t] = s;
  }
}

// dynamic shared memory: 12 * P doubles
__global__ void k_conf_edge(ConfArgs A, const double *w, double *v) {
  extern __shared__ double gk[];
  const int e = blockIdx.x / A.n_rhs, r = blockIdx.x - e * A.n_rhs;
  const int P = A.elem_W[e] + 1;
  const int64_t rb = (int64_t)r * A.ndof, base = rb + A.dof_off[e];
  for (int q = threadIdx.x; q < 12 * P; q += blockDim.x) {
    const int k = q / P, t = q - k * P, g = A.eid[e * 12 + k];
    double tg = 0.0;
    if (!A.edir[g]) {
      for (int m = A.eptr[g]; m < A.eptr[g + 1]; ++m) {
        const int em = A.emem[m] / 12, km = A.emem[m] - 12 * em;
        tg += w[rb + A.dof_off[em] + conf_edge_node(km, t, A.elem_W[em] + 1)];
      }
      tg /= (double)(A.eptr[g + 1] - A.eptr[g]);
    }
    gk[q] = tg - w[base + conf_edge_node(k, t, P)];
  }
  __syncthreads();
  const double *L = A.lin[P - 1];
  for (int t = threadIdx.x; t < P * P * P; t += blockDim.x) {
    const int c[3] = {t % P, (t / P) % P, t / (P * P)};
    double s = w[base + t];
    for (int k = 0; k < 12; ++k) {
      const int a = k >> 2, o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
      s += gk[k * P + c[a]] * L[(k & 1) * P + c[o1]] * L[((k >> 1) & 1) * P + c[o2]];
    }
    v[base + t] = s;
  }
}

// dynamic shared memory: 6 * P * P doubles
__global__ void k_conf_face(ConfArgs A, const double *v, double *p) {
  extern __shared__ double cf[];
  const int e = blockIdx.x / A.n_rhs, r = blockIdx.x - e * A.n_rhs;
  const int P = A.elem_W[e] + 1, P2 = P * P;
  const int64_t rb = (int64_t)r * A.ndof, base = rb + A.dof_off[e];
  for (int q = threadIdx.x; q < 6 * P2; q += blockDim.x) {
    const int f = q / P2, sp = q - f * P2, p1 = sp % P, p2 = sp / P;
    const int a = f >> 1, side = f & 1, n = side ? P - 1 : 0;
    // face point (p1, p2) along (t1, t2), t1 < t2 the axes other than a
    auto node = [&](int nn) {
      if (a == 0) return (p2 * P + p1) * P + nn;
      if (a == 1) return (p2 * P + nn) * P + p1;
      return (nn * P + p2) * P + p1;
    };
    const double own = v[base + node(n)];
    const int nb = A.nbr[e * 6 + f];
    double tg = 0.0;
    if (nb >= 0) tg = 0.5 * (own + v[rb + A.dof_off[nb] + node(P - 1 - n)]);
    else if (A.fbc && A.fbc[e * 6 + f]) tg = own;  // a Neumann / Robin face is free
    cf[q] = tg - own;
  }
  __syncthreads();
  const double *L = A.lin[P - 1];
  for (int t = threadIdx.x; t < P * P * P; t += blockDim.x) {
    const int c[3] = {t % P, (t / P) % P, t / P2};
    double s = v[base + t];
    for (int f = 0; f < 6; ++f) {
      const int a = f >> 1, o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
      s += cf[f * P2 + c[o2] * P + c[o1]] * L[(f & 1) * P + c[a]];
    }
    p[base + t] = s;
  }
}

// topology of the conforming correction (box meshes), built once per handle
static hpse_status conf_setup(hpse_mesh *m) {
  const int E = m->n_elem;
  struct Key {
    int pr, kind;
    long long c[5];
    bool operator<(const Key &o) const {
      if (pr != o.pr) return pr < o.pr;
      if (kind != o.kind) return kind < o.kind;
      for (int i = 0; i < 5; ++i)
        if (c[i] != o.c[i]) return c[i] < o.c[i];
      return false;
    }
  };
  // coordinates to integer keys (1e-9 relative to the mesh's extent)
  double ext = 1.0;
  for (size_t i = 0; i < m->lo.size(); ++i) ext = std::max({ext, std::fabs(m->lo[i]), std::fabs(m->hi[i])});
  auto q = [&](double x) { return (long long)std::llround(x / (ext * 1e-9)); };
  auto X = [&](int e, int a, int side) { return side ? m->hi[3 * e + a] : m->lo[3 * e + a]; };
  auto dir_face = [&](int e, int f) { return m->nbr[6 * e + f] == -1 && m->fbc[6 * e + f] == 0; };
  std::map<Key, int> vmap, emap;
  std::vector<int> vid(8 * (size_t)E), eid(12 * (size_t)E), vdir, edir;
  std::vector<std::vector<int>> vmem, emem;
  for (int e = 0; e < E; ++e) {
    const int pr = m->prob[e];
    for (int c = 0; c < 8; ++c) {
      Key k{pr, 0, {q(X(e, 0, c & 1)), q(X(e, 1, (c >> 1) & 1)), q(X(e, 2, (c >> 2) & 1)), 0, 0}};
      auto it = vmap.find(k);
      int g;
      if (it == vmap.end()) {
        g = (int)vmem.size();
        vmap[k] = g;
        vmem.emplace_back();
        vdir.push_back(0);
      } else {
        g = it->second;
      }
      vid[8 * e + c] = g;
      vmem[g].push_back(8 * e + c);
      for (int a = 0; a < 3; ++a)
        if (dir_face(e, 2 * a + ((c >> a) & 1))) vdir[g] = 1;
    }
    for (int kk = 0; kk < 12; ++kk) {
      const int a = kk >> 2, s1 = kk & 1, s2 = (kk >> 1) & 1;
      const int o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
      Key k{pr, 1 + a, {q(X(e, o1, s1)), q(X(e, o2, s2)), q(X(e, a, 0)), q(X(e, a, 1)), 0}};
      auto it = emap.find(k);
      int g;
      if (it == emap.end()) {
        g = (int)emem.size();
        emap[k] = g;
        emem.emplace_back();
        edir.push_back(0);
      } else {
        g = it->second;
      }
      eid[12 * e + kk] = g;
      emem[g].push_back(12 * e + kk);
      if (dir_face(e, 2 * o1 + s1) || dir_face(e, 2 * o2 + s2)) edir[g] = 1;
    }
  }
  std::vector<int> vptr(1, 0), vm, eptr(1, 0), em;
  for (auto &l : vmem) {
    vm.insert(vm.end(), l.begin(), l.end());
    vptr.push_back((int)vm.size());
  }
  for (auto &l : emem) {
    em.insert(em.end(), l.begin(), l.end());
    eptr.push_back((int)em.size());
  }
  // linear blends per degree
  std::vector<double> lin;
  std::vector<size_t> loff(HPSE_MAX_W + 1, 0);
  for (auto &kv : m->tabs) {
    const hm::DegreeTables &t = kv.second;
    loff[kv.first] = lin.size();
    for (int side = 0; side < 2; ++side)
      for (int i = 0; i < t.P; ++i) lin.push_back(side ? 0.5 * (1.0 + t.xp[i]) : 0.5 * (1.0 - t.xp[i]));
  }
  CK(upload(m->d_cf_vid, vid));
  CK(upload(m->d_cf_vptr, vptr));
  CK(upload(m->d_cf_vmem, vm));
  CK(upload(m->d_cf_vdir, vdir));
  CK(upload(m->d_cf_eid, eid));
  CK(upload(m->d_cf_eptr, eptr));
  CK(upload(m->d_cf_emem, em));
  CK(upload(m->d_cf_edir, edir));
  CK(upload(m->d_cf_lin, lin));
  std::vector<const double *> lp(HPSE_MAX_W + 1, nullptr);
  for (auto &kv : m->tabs) lp[kv.first] = m->d_cf_lin.as<double>() + loff[kv.first];
  CK(upload(m->d_cf_linptr, lp));
  const size_t nv = (size_t)m->n_rhs * std::max<int64_t>(m->ndof, 1) * sizeof(double);
  CK(m->d_cf_w.alloc(nv));
  CK(m->d_cf_v.alloc(nv));
  m->conf_ready = true;
  return HPSE_OK;
}

extern "C" hpse_status hpse_conforming_correction(hpse_mesh *m, const double *u, double *p, void *stream) {
  // the vertex / edge / face averages assume one degree across every face
  if (m && m->has_mixed) return HPSE_ERR_DEGREE;
  if (!m || m->coord != HPSE_COORD_CARTESIAN) return HPSE_ERR_INVALID_ARG;  // box meshes only
  if (m->ndof == 0) return HPSE_OK;
  if (!u || !p) return HPSE_ERR_INVALID_ARG;
  CK(cudaSetDevice(m->device));
  if (!m->conf_ready) {
    const hpse_status st = conf_setup(m);
    if (st != HPSE_OK) return st;
  }
  ConfArgs A;
  A.n_rhs = m->n_rhs;
  A.ndof = m->ndof;
  A.dof_off = m->d_dof_off.as<int64_t>();
  A.elem_W = m->d_elem_W.as<int32_t>();
  A.nbr = m->d_nbr.as<int32_t>();
  A.vid = m->d_cf_vid.as<int32_t>();
  A.vptr = m->d_cf_vptr.as<int32_t>();
  A.vmem = m->d_cf_vmem.as<int32_t>();
  A.vdir = m->d_cf_vdir.as<int32_t>();
  A.eid = m->d_cf_eid.as<int32_t>();
  A.eptr = m->d_cf_eptr.as<int32_t>();
  A.emem = m->d_cf_emem.as<int32_t>();
  A.edir = m->d_cf_edir.as<int32_t>();
  A.lin = m->d_cf_linptr.as<const double *>();
  A.fbc = m->has_nr ? m->d_fbc.as<int32_t>() : nullptr;
  int Wmax = 1;
  for (auto &kv : m->tabs) Wmax = std::max(Wmax, kv.first);
  const int P = Wmax + 1, items = m->n_elem * m->n_rhs;
  cudaStream_t s = (cudaStream_t)stream;
  k_conf_vertex<<<items, 128, 0, s>>>(A, u, m->d_cf_w.as<double>());
  k_conf_edge<<<items, 128, 12 * P * sizeof(double), s>>>(A, m->d_cf_w.as<double>(), m->d_cf_v.as<double>());
  k_conf_face<<<items, 128, 6 * P * P * sizeof(double), s>>>(A, m->d_cf_v.as<double>(), p);
  CK(cudaGetLastError());
  g_launches += 3;
  return HPSE_OK;
}

static __device__ __align__(256) double g_noalloc_scratch[HPSE_NOALLOC_DOUBLES];

static double *g_noalloc_addr[HPSE_NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mutex;

// per-rhs deterministic sums of the k_h1 partials (one block per rhs)
__global__ void k_h1_reduce_noalloc(int n_elem, int n_rhs, const double *part_err, const double *part_nrm,
                                    double *out) {
  const int r = blockIdx.x;
  double a = 0.0, b = 0.0;
  for (int e = threadIdx.x; e < n_elem; e += blockDim.x) {
    a += part_err[(int64_t)e * n_rhs + r];
    b += part_nrm[(int64_t)e * n_rhs + r];
  }
  a = block_sum_d(a);
  b = block_sum_d(b);
  if (threadIdx.x == 0) {
    out[2 * r] = a;
    out[2 * r + 1] = b;
  }
}

extern "C" hpse_status hpse_h1_error_noalloc(hpse_mesh *m, const double *u, const double *ref, const double *vq,
                                             const double *gq, double *out, void *stream) {
  if (m && m->coord != HPSE_COORD_CARTESIAN) return HPSE_ERR_INVALID_ARG;  // box meshes only
  if (!m || !out) return HPSE_ERR_INVALID_ARG;
  if (m->ndof == 0) {
    for (int r = 0; r < m->n_rhs; ++r) out[2 * r] = out[2 * r + 1] = 0.0;
    return HPSE_OK;
  }
  if (!u || (!ref && (!vq || !gq))) return HPSE_ERR_INVALID_ARG;
  const int64_t ni = (int64_t)m->n_elem * m->n_rhs;
  if (ni > HPSE_NOALLOC_MAX_ITEMS || m->n_rhs > HPSE_NOALLOC_MAX_RHS) return HPSE_ERR_CAPACITY;
  if (m->device < 0 || m->device >= HPSE_NOALLOC_MAX_DEVICES) return HPSE_ERR_INVALID_ARG;
  CK(cudaSetDevice(m->device));
  // once per device, with that device current: the device address of the array
  double *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[m->device]) {
      void *p = nullptr;
      CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      g_noalloc_addr[m->device] = static_cast<double *>(p);
    }
    base = g_noalloc_addr[m->device];
  }
  double *part_err = base;
  double *part_nrm = base + HPSE_NOALLOC_MAX_ITEMS;
  double *res = base + 2 * HPSE_NOALLOC_MAX_ITEMS;
  const double **qtab = reinterpret_cast<const double **>(res + 2 * HPSE_NOALLOC_MAX_RHS);
  cudaStream_t s = (cudaStream_t)stream;
  const double *tp[HPSE_MAX_W + 1] = {nullptr};
  int Wmax = 1;
  for (auto &kv : m->d_qtab) {
    tp[kv.first] = kv.second.as<double>();
    Wmax = std::max(Wmax, kv.first);
  }
  CK(cudaMemcpyAsync(qtab, tp, sizeof(tp), cudaMemcpyHostToDevice, s));
  H1Args A;
  memset(&A, 0, sizeof(A));
  A.n_rhs = m->n_rhs;
  A.ndof = m->ndof;
  A.nquad = m->nquad;
  A.dof_off = m->d_dof_off.as<int64_t>();
  A.coef_off = m->d_coef_off.as<int64_t>();
  A.elem_W = m->d_elem_W.as<int32_t>();
  A.geo = m->d_geo64.as<double>();
  A.qtab = qtab;
  A.u = u;
  A.ref = ref;
  A.vq = vq;
  A.gq = gq;
  A.part_err = part_err;
  A.part_nrm = part_nrm;
  const int P = Wmax + 1, Q = 2 * Wmax + 1;
  const size_t smem = (size_t)(P * P * P + 2 * Q * P * P + 3 * Q * Q * P) * sizeof(double);
  CK(raise_smem((const void *)k_h1, m->device, (size_t)smem));
  // every partial and every result is overwritten: nothing needs clearing
  k_h1<<<(int)ni, 256, smem, s>>>(A);
  CK(cudaGetLastError());
  k_h1_reduce_noalloc<<<m->n_rhs, 256, 0, s>>>(m->n_elem, m->n_rhs, part_err, part_nrm, res);
  CK(cudaGetLastError());
  g_launches += 2;
  CK(cudaMemcpyAsync(out, res, (size_t)2 * m->n_rhs * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return HPSE_OK;
}

// ---------------------------------------------------------------------------
// One problem over several GPUs (Section 5.3): element partition along a
// space-filling curve and the block copies of the ghost exchange.
// ---------------------------------------------------------------------------
// Morton key of three 21-bit integer coordinates (bit-interleaved, x lowest)
static uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  uint64_t k = 0;
  for (int b = 0; b < 21; ++b) {
    k |= (uint64_t)((x >> b) & 1u) << (3 * b);
    k |= (uint64_t)((y >> b) & 1u) << (3 * b + 1);
    k |= (uint64_t)((z >> b) & 1u) << (3 * b + 2);
  }
  return k;
}

extern "C" hpse_status hpse_partition(const hpse_mesh_desc *d, int32_t n_parts, int32_t *owner) {
  if (!d || !owner || n_parts < 1 || d->n_elem < 0 || d->n_problem < 1) return HPSE_ERR_INVALID_ARG;
  if (d->coord != HPSE_COORD_CARTESIAN) return HPSE_ERR_INVALID_ARG;
  const int E = d->n_elem;
  if (E == 0) return HPSE_OK;
  if (!d->elem_W || !d->elem_problem || !d->elem_lo || !d->elem_hi) return HPSE_ERR_INVALID_ARG;
  // bounding box of each problem's element centres
  std::vector<double> blo(3 * (size_t)d->n_problem, 1e300), bhi(3 * (size_t)d->n_problem, -1e300);
  for (int e = 0; e < E; ++e) {
    const int p = d->elem_problem[e];
    if (p < 0 || p >= d->n_problem || d->elem_W[e] < 1 || d->elem_W[e] > HPSE_MAX_W) return HPSE_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a) {
      const double c = 0.5 * (d->elem_lo[3 * e + a] + d->elem_hi[3 * e + a]);
      if (!std::isfinite(c)) return HPSE_ERR_INVALID_ARG;
      blo[3 * p + a] = std::min(blo[3 * p + a], c);
      bhi[3 * p + a] = std::max(bhi[3 * p + a], c);
    }
  }
  std::vector<std::pair<std::pair<int, uint64_t>, int>> order((size_t)E);
  const double top = (double)((1u << 21) - 1);
  for (int e = 0; e < E; ++e) {
    const int p = d->elem_problem[e];
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
      const double c = 0.5 * (d->elem_lo[3 * e + a] + d->elem_hi[3 * e + a]);
      const double span = bhi[3 * p + a] - blo[3 * p + a];
      q[a] = span > 0.0 ? (uint32_t)std::lround((c - blo[3 * p + a]) / span * top) : 0u;
    }
    order[e] = {{p, morton3(q[0], q[1], q[2])}, e};
  }
  std::sort(order.begin(), order.end());
  double total = 0.0;
  for (int e = 0; e < E; ++e) total += std::pow((double)(d->elem_W[e] + 1), 3);
  // element at prefix weight s (its midpoint s + w/2) goes to part floor(n (s + w/2) / total)
  double s = 0.0;
  for (const auto &o : order) {
    const int e = o.second;
    const double w = std::pow((double)(d->elem_W[e] + 1), 3);
    int part = (int)std::floor((s + 0.5 * w) * n_parts / total);
    owner[e] = std::min(n_parts - 1, std::max(0, part));
    s += w;
  }
  return HPSE_OK;
}

template <typename T, bool PACK>
__global__ void k_move_blocks(int32_t n, int32_t n_rhs, int64_t ndof, int64_t buf_len, const int32_t *items,
                              const int64_t *buf_off, const int64_t *dof_off, const int32_t *item_n, const T *src,
                              T *dst) {
  const int i = blockIdx.x, r = blockIdx.y;
  if (i >= n) return;
  const int e = items[i];
  const int len = item_n[e];
  const int64_t v0 = (int64_t)r * ndof + dof_off[e], b0 = (int64_t)r * buf_len + buf_off[i];
  for (int t = threadIdx.x; t < len; t += blockDim.x) {
    if (PACK)
      dst[b0 + t] = src[v0 + t];
    else
      dst[v0 + t] = src[b0 + t];
  }
}

template <bool PACK>
static hpse_status move_blocks(const hpse_mesh *m, int32_t prec, const int32_t *items, const int64_t *buf_off,
                               int32_t n, int64_t buf_len, const void *src, void *dst, void *stream) {
  if (!m || (prec != HPSE_FP64 && prec != HPSE_FP32) || n < 0 || buf_len < 0) return HPSE_ERR_INVALID_ARG;
  if (n == 0 || m->ndof == 0) return HPSE_OK;
  if (!items || !buf_off || !src || !dst) return HPSE_ERR_INVALID_ARG;
  CK(cudaSetDevice(m->device));
  cudaStream_t s = (cudaStream_t)stream;
  const dim3 grid((unsigned)n, (unsigned)m->n_rhs);
  if (prec == HPSE_FP64)
    k_move_blocks<double, PACK><<<grid, 128, 0, s>>>(n, m->n_rhs, m->ndof, buf_len, items, buf_off,
                                                     m->d_dof_off.as<int64_t>(), m->d_item_n.as<int32_t>(),
                                                     (const double *)src, (double *)dst);
  else
    k_move_blocks<float, PACK><<<grid, 128, 0, s>>>(n, m->n_rhs, m->ndof, buf_len, items, buf_off,
                                                    m->d_dof_off.as<int64_t>(), m->d_item_n.as<int32_t>(),
                                                    (const float *)src, (float *)dst);
  CK(cudaGetLastError());
  ++g_launches;
  return HPSE_OK;
}

extern "C" hpse_status hpse_pack_blocks(const hpse_mesh *m, int32_t prec, const int32_t *items,
                                        const int64_t *buf_off, int32_t n, int64_t buf_len, const void *vec,
                                        void *buf, void *stream) {
  return move_blocks<true>(m, prec, items, buf_off, n, buf_len, vec, buf, stream);
}

extern "C" hpse_status hpse_unpack_blocks(const hpse_mesh *m, int32_t prec, const int32_t *items,
                                          const int64_t *buf_off, int32_t n, int64_t buf_len, const void *buf,
                                          void *vec, void *stream) {
  return move_blocks<false>(m, prec, items, buf_off, n, buf_len, buf, vec, stream);
}
