// inst_template.cuh -- launchers for one (REAL, WDEG) instantiation of
// kernels.cuh.  A generated translation unit defines REAL, WDEG,
// HPSE_REGISTER_NAME (and HPSE_DOUBLE for REAL = double), then includes this.
#include <vector>

#include "kernels.cuh"
#include "general.cuh"
#include "ibp.cuh"

namespace {

template <int COEF, int MODE>
cudaError_t launch_apply_t(const void *args, int n_items, int threads, cudaStream_t s) {
  (void)threads;  // the apply CTA size is fixed at compile time (NT)
  k_apply<COEF, MODE><<<n_items, NT, ApplyLayout<COEF>::BYTES, s>>>(*static_cast<const ApplyArgs *>(args));
  return cudaGetLastError();
}

cudaError_t apply_fn(int coef, int mode, const void *args, int n_items, int threads, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  if (coef == COEF_LAPLACE) {
    if (mode == MODE_PLAIN) return launch_apply_t<COEF_LAPLACE, MODE_PLAIN>(args, n_items, threads, s);
    if (mode == MODE_PCG) return launch_apply_t<COEF_LAPLACE, MODE_PCG>(args, n_items, threads, s);
    if (mode == MODE_TRANSPOSE) return launch_apply_t<COEF_LAPLACE, MODE_TRANSPOSE>(args, n_items, threads, s);
  } else if (coef == COEF_SCALAR) {
    if (mode == MODE_PLAIN) return launch_apply_t<COEF_SCALAR, MODE_PLAIN>(args, n_items, threads, s);
    if (mode == MODE_PCG) return launch_apply_t<COEF_SCALAR, MODE_PCG>(args, n_items, threads, s);
    if (mode == MODE_TRANSPOSE) return launch_apply_t<COEF_SCALAR, MODE_TRANSPOSE>(args, n_items, threads, s);
  } else if (coef == COEF_EDGE) {
    if (mode == MODE_PLAIN) return launch_apply_t<COEF_EDGE, MODE_PLAIN>(args, n_items, threads, s);
    if (mode == MODE_PCG) return launch_apply_t<COEF_EDGE, MODE_PCG>(args, n_items, threads, s);
    if (mode == MODE_TRANSPOSE) return launch_apply_t<COEF_EDGE, MODE_TRANSPOSE>(args, n_items, threads, s);
  } else if (coef == COEF_VERTEX) {
    if (mode == MODE_PLAIN) return launch_apply_t<COEF_VERTEX, MODE_PLAIN>(args, n_items, threads, s);
    if (mode == MODE_PCG) return launch_apply_t<COEF_VERTEX, MODE_PCG>(args, n_items, threads, s);
    if (mode == MODE_TRANSPOSE) return launch_apply_t<COEF_VERTEX, MODE_TRANSPOSE>(args, n_items, threads, s);
  } else if (coef == COEF_VERTEX_EDGE) {
    if (mode == MODE_PLAIN) return launch_apply_t<COEF_VERTEX_EDGE, MODE_PLAIN>(args, n_items, threads, s);
    if (mode == MODE_PCG) return launch_apply_t<COEF_VERTEX_EDGE, MODE_PCG>(args, n_items, threads, s);
    if (mode == MODE_TRANSPOSE)
      return launch_apply_t<COEF_VERTEX_EDGE, MODE_TRANSPOSE>(args, n_items, threads, s);
  } else if (coef == hpse::COEF_GENERAL) {
    if (mode == MODE_PLAIN) return launch_apply_gen<MODE_PLAIN>(args, n_items, s);
    if (mode == MODE_PCG) return launch_apply_gen<MODE_PCG>(args, n_items, s);
    if (mode == MODE_TRANSPOSE) return launch_apply_gen<MODE_TRANSPOSE>(args, n_items, s);
  }
  return cudaErrorInvalidValue;
}

size_t apply_smem_fn(int coef) {
  if (coef == COEF_SCALAR) return ApplyLayout<COEF_SCALAR>::BYTES;
  if (coef == COEF_EDGE) return ApplyLayout<COEF_EDGE>::BYTES;
  if (coef == COEF_VERTEX) return ApplyLayout<COEF_VERTEX>::BYTES;
  if (coef == COEF_VERTEX_EDGE) return ApplyLayout<COEF_VERTEX_EDGE>::BYTES;
  // 0: no instance of this degree and precision (its layout exceeds 227 KB)
  if (coef == hpse::COEF_GENERAL) return GenLayout::FITS ? GenLayout::BYTES : 0;
  return ApplyLayout<COEF_LAPLACE>::BYTES;
}

int apply_max_threads_fn(int) { return NT; }

cudaError_t precond_fn(int mode, const void *args, int n_items, int threads, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  (void)threads;  // CTA shape fixed at compile time: PC_ITEMS items of PC_TPI threads
  const int grid = (n_items + PC_ITEMS - 1) / PC_ITEMS;
  if (mode == MODE_PLAIN)
    k_precond<MODE_PLAIN><<<grid, PC_NT, PC_BYTES, s>>>(*static_cast<const PrecArgs *>(args));
  else if (mode == MODE_PCG)
    k_precond<MODE_PCG><<<grid, PC_NT, PC_BYTES, s>>>(*static_cast<const PrecArgs *>(args));
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <int COEF, int MODE>
cudaError_t set_smem_attr() {
  cudaError_t e = cudaFuncSetAttribute(k_apply<COEF, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)ApplyLayout<COEF>::BYTES);
  if (e != cudaSuccess) return e;
  // prefer the largest shared-memory carve-out so that several CTAs fit per SM
  return cudaFuncSetAttribute(k_apply<COEF, MODE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxShared);
}

// Upload this degree's tables (packed FP64, see registry.h) to constant
// memory of the current device, converting to REAL, and raise the dynamic
// shared-memory limit of the apply kernels.
cudaError_t upload_fn(const double *pk) {
  Tables t;
  int o = 0;
  for (int m = 0; m < 3; ++m)
    for (int i = 0; i < QP; ++i) t.B[m][i] = (real)pk[o++];
  // folded halves of B0, B1, B2 (even-odd decomposition), formed in FP64
  for (int m = 0; m < 3; ++m) {
    const double *b = pk + m * QP;
    for (int q = 0; q <= HQ; ++q)
      for (int j = 0; j < HPE; ++j) {
        const bool mid = (P & 1) && j == HP;
        t.FE[m][q * HPE + j] = (real)(mid ? b[q * P + j] : 0.5 * (b[q * P + j] + b[q * P + P - 1 - j]));
        t.FO[m][q * HPE + j] = (real)(mid ? 0.0 : 0.5 * (b[q * P + j] - b[q * P + P - 1 - j]));
      }
  }
  for (int i = 0; i < P * HPE; ++i) {
    t.XE[0][i] = make_float2((float)t.FE[0][i], (float)t.FE[0][i]);
    t.XE[1][i] = make_float2((float)t.FE[0][i], (float)t.FE[2][i]);
    t.XO[0][i] = make_float2((float)t.FO[0][i], (float)t.FO[0][i]);
    t.XO[1][i] = make_float2((float)t.FO[0][i], (float)t.FO[2][i]);
  }
  const double *pD = pk + o;
  for (int i = 0; i < P2; ++i) t.D[i] = (real)pk[o++];
  for (int i = 0; i < P2; ++i) t.S[i] = (real)pk[o++];
  const double *pM = pk + o;
  for (int i = 0; i < P2; ++i) t.MP[i] = (real)pk[o++];
  const double *pK = pk + o;
  for (int i = 0; i < P2; ++i) t.KP[i] = (real)pk[o++];
  // folded halves of D, D^T, MP, KP, MP + KP, M1 = D^T MP D, M12 = D^T (MP + KP) D
  // for the face phase, formed in FP64
  std::vector<double> M1(P2, 0.0), M12(P2, 0.0);
  for (int r = 0; r < P; ++r)
    for (int c = 0; c < P; ++c)
      for (int i = 0; i < P; ++i)
        for (int j = 0; j < P; ++j) {
          const double dd = pD[i * P + r] * pD[j * P + c];
          M1[r * P + c] += dd * pM[i * P + j];
          M12[r * P + c] += dd * (pM[i * P + j] + pK[i * P + j]);
        }
  for (int m = 0; m < 7; ++m)
    for (int i = 0; i < HPE; ++i)
      for (int j = 0; j < HPE; ++j) {
        auto x = [&](int r, int c) {
          switch (m) {
            case 0: return pD[r * P + c];
            case 1: return pD[c * P + r];
            case 2: return pM[r * P + c];
            case 3: return pK[r * P + c];
            case 4: return pM[r * P + c] + pK[r * P + c];
            case 5: return M1[r * P + c];
            default: return M12[r * P + c];
          }
        };
        const bool mid = (P & 1) && j == HP;
        t.PF[m][0][i * HPE + j] = (real)(mid ? x(i, j) : 0.5 * (x(i, j) + x(i, P - 1 - j)));
        t.PF[m][1][i * HPE + j] = (real)(mid ? 0.0 : 0.5 * (x(i, j) - x(i, P - 1 - j)));
      }
  for (int i = 0; i < Q; ++i) t.WQ[i] = (real)pk[o++];
  for (int i = 0; i < P; ++i) t.MU[i] = (real)pk[o++];
  cudaError_t err = cudaMemcpyToSymbol(c_tab, &t, sizeof(Tables));
  if (err != cudaSuccess) return err;
  // D_Q and D_Q^2 of the Q-point grid (integration-by-parts transpose), formed in FP64
  {
    IbpTables it;
    const double *dqp = pk + o;
    for (int i = 0; i < Q; ++i)
      for (int j = 0; j < Q; ++j) {
        double acc = 0.0;
        for (int m = 0; m < Q; ++m) acc += dqp[i * Q + m] * dqp[m * Q + j];
        it.DQ[i * Q + j] = (real)dqp[i * Q + j];
        it.DQ2[i * Q + j] = (real)acc;
      }
    o += Q2;
    err = cudaMemcpyToSymbol(c_ibp, &it, sizeof(IbpTables));
    if (err != cudaSuccess) return err;
  }
  cudaError_t e2;
  if ((e2 = set_smem_attr<COEF_LAPLACE, MODE_PLAIN>()) != cudaSuccess) return e2;
  if ((e2 = set_smem_attr<COEF_LAPLACE, MODE_PCG>()) != cudaSuccess) return e2;
  if ((e2 = set_smem_attr<COEF_LAPLACE, MODE_TRANSPOSE>()) != cudaSuccess) return e2;
  if ((e2 = set_smem_attr<COEF_SCALAR, MODE_PLAIN>()) != cudaSuccess) return e2;
  if ((e2 = set_smem_attr<COEF_SCALAR, MODE_PCG>()) != cudaSuccess) return e2;
  if ((e2 = set_smem_attr<COEF_SCALAR, MODE_TRANSPOSE>()) != cudaSuccess) return e2;
  if ((e2 = set_smem_attr<COEF_EDGE, MODE_PLAIN>()) != cudaSuccess) return e2;
  if ((e2 = set_smem_attr<COEF_EDGE, MODE_PCG>()) != cudaSuccess) return e2;
  if ((e2 = set_smem_attr<COEF_EDGE, MODE_TRANSPOSE>()) != cudaSuccess) return e2;
  if ((e2 = set_smem_attr<COEF_VERTEX, MODE_PLAIN>()) != cudaSuccess) return e2;
  if ((e2 = set_smem_attr<COEF_VERTEX, MODE_PCG>()) != cudaSuccess) return e2;
  if ((e2 = set_smem_attr<COEF_VERTEX, MODE_TRANSPOSE>()) != cudaSuccess) return e2;
  if ((e2 = set_smem_attr<COEF_VERTEX_EDGE, MODE_PLAIN>()) != cudaSuccess) return e2;
  if ((e2 = set_smem_attr<COEF_VERTEX_EDGE, MODE_PCG>()) != cudaSuccess) return e2;
  if ((e2 = set_smem_attr<COEF_VERTEX_EDGE, MODE_TRANSPOSE>()) != cudaSuccess) return e2;
  if ((e2 = set_smem_attr_gen<MODE_PLAIN>()) != cudaSuccess) return e2;
  if ((e2 = set_smem_attr_gen<MODE_PCG>()) != cudaSuccess) return e2;
  if ((e2 = set_smem_attr_gen<MODE_TRANSPOSE>()) != cudaSuccess) return e2;
  if ((e2 = set_smem_attr_ibp<COEF_LAPLACE>()) != cudaSuccess) return e2;
  if ((e2 = set_smem_attr_ibp<COEF_SCALAR>()) != cudaSuccess) return e2;
  if ((e2 = cudaFuncSetAttribute(k_precond<MODE_PLAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)PC_BYTES)) != cudaSuccess)
    return e2;
  if ((e2 = cudaFuncSetAttribute(k_precond<MODE_PCG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)PC_BYTES)) != cudaSuccess)
    return e2;
  return cudaSuccess;
}

cudaError_t transpose_ibp_fn(int coef, const void *args, int n_items, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  if (coef == COEF_LAPLACE) return launch_transpose_ibp_t<COEF_LAPLACE>(args, n_items, s);
  if (coef == COEF_SCALAR) return launch_transpose_ibp_t<COEF_SCALAR>(args, n_items, s);
  return cudaErrorInvalidValue;
}

size_t ibp_smem_fn(int coef) {
  if (coef == COEF_LAPLACE) return IbpLayout<COEF_LAPLACE>::FITS ? IbpLayout<COEF_LAPLACE>::BYTES : 0;
  if (coef == COEF_SCALAR) return IbpLayout<COEF_SCALAR>::FITS ? IbpLayout<COEF_SCALAR>::BYTES : 0;
  return 0;
}

static_assert(ApplyLayout<COEF_SCALAR>::BYTES <= 232448, "apply kernel exceeds 227 KB of shared memory");

}  // namespace

extern "C" void HPSE_REGISTER_NAME(hpse::KernelSet *ks) {
  ks->W = WDEG;
#if defined(HPSE_DOUBLE)
  ks->is_double = 1;
#else
  ks->is_double = 0;
#endif
  ks->upload = upload_fn;
  ks->apply = apply_fn;
  ks->apply_smem = apply_smem_fn;
  ks->apply_max_threads = apply_max_threads_fn;
  ks->precond = precond_fn;
  ks->transpose_ibp = transpose_ibp_fn;
  ks->ibp_smem = ibp_smem_fn;
}
