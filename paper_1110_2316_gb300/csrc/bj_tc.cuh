// bj_tc.cuh -- the element-block preconditioner products t = X r and
// z = X^T t (X = L^{-1}, A_ee = L L^T, FP32 inner solve) on the fifth-generation
// tensor cores: tcgen05.mma kind::tf32 with FP32 accumulators in tensor memory.
//
// A TF32 operand keeps 10 mantissa bits, so each FP32 operand is split into
// hi = rna_tf32(v) and lo = rna_tf32(v - hi), and every product takes three
// MMAs, hi*hi + hi*lo + lo*hi (the dropped lo*lo and the roundings of lo are
// about 2^-21 of |X| |r|): the products keep FP32 accuracy, so that the
// preconditioner stays the fixed SPD operator X~^T X~ of the FP32 factor X~
// that the CUDA-core products apply.
//
// Storage: per element the factor as 128 x 128 FP32 tiles, row-major, zero
// beyond n and outside the triangle: first the lower tiles of X (block row
// bi, block column bk <= bi, in row order), then the tiles of X^T with
// bk >= bi (row order), so that both products read K-major rows.
//
// One CTA (4 warps) per (element, 128-row tile, 64 right-hand sides): K in
// chunks of 32 (one 128-byte row per operand row), BJT_STAGES shared-memory stages of
// A hi/lo (128 x 32) and B hi/lo (64 x 32) in the canonical 128-byte-swizzled
// K-major layout (8-row atoms of 1 KB, 16-byte chunk j of row m at j ^ (m % 8)),
// filled from registers (the split needs them anyway; the next chunk's global
// loads are issued while the tensor core works on the current one); thread 0
// issues the 12 MMAs of a chunk (4 K-steps of 8 x 3 products, M = 128, N = 64)
// and commits them to the stage's mbarrier; the accumulator (128 lanes x 64
// columns of TMEM) is read back by all four warps (32 lanes each) and stored
// coalesced along the rows.  Every wait on an mbarrier is bounded: on expiry the
// CTA sets *err, stops issuing and still frees its TMEM.
#pragma once

constexpr int BJT = 128;                 // tile edge (rows per CTA, MMA M)
constexpr int BJT_N = 64;                // right-hand sides per CTA (MMA N)
constexpr int BJT_K = 32;                // K per stage: one 128-byte row of FP32
constexpr int BJT_THREADS = 128;
constexpr int BJT_A_BYTES = BJT * BJT_K * 4;    // 16 KB
constexpr int BJT_B_BYTES = BJT_N * BJT_K * 4;  // 8 KB
constexpr int BJT_STAGE_BYTES = 2 * BJT_A_BYTES + 2 * BJT_B_BYTES;
#if defined(HPSE_BJT_STAGES)
constexpr int BJT_STAGES = HPSE_BJT_STAGES;  // set at build time (pipeline-depth experiments)
#else
constexpr int BJT_STAGES = 1;  // 4 CTAs per SM hide more load latency than a second stage (measured)
#endif
constexpr int BJT_MINB = BJT_STAGES == 1 ? 4 : 2;  // CTAs per SM that the shared memory allows
constexpr size_t BJT_SMEM = BJT_STAGES * (size_t)BJT_STAGE_BYTES + 1024;  // stages + alignment slack
constexpr int BJT_TILE = BJT * BJT;      // floats per tile
constexpr int BJT_TMEM_COLS = 64;

// tiles per copy (X or X^T) of an n x n factor
__host__ __device__ inline int bjt_blocks(int n) {
  const int nbt = (n + BJT - 1) / BJT;
  return nbt * (nbt + 1) / 2;
}

struct BjTcArgs {
  const int32_t *elems;
  int32_t n_group;
  int32_t n;                // block size (W+1)^3
  int32_t n_rhs;
  int64_t ndof;
  const int64_t *dof_off;   // per element
  const int64_t *tile_off;  // per element: offset (floats) of its tile set
  int32_t *err;             // set when a bounded wait expired
};

__device__ __forceinline__ uint32_t bjt_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: canonical K-major layout with the 128-byte
// swizzle, 8-row atoms 1024 bytes apart (stride byte offset), start address in
// 16-byte units; bits 46-48 hold the fixed value 1 of the tcgen05 format
__device__ __forceinline__ uint64_t bjt_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor of kind::tf32: FP32 accumulator (bits 4-5 = 1), A and
// B TF32 (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28
constexpr uint32_t BJT_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BJT_N >> 3) << 17) |
                               ((uint32_t)(BJT >> 4) << 24);

__device__ __forceinline__ float bjt_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

__device__ __forceinline__ bool bjt_wait(uint32_t bar, uint32_t parity) {
  // bounded: about a second of polling at most
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// out = X in (TRANS = false: X lower) or X^T in (TRANS = true) for the
// group's elements.  grid: (n_group * ceil(n / 128), ceil(n_rhs / 64)), 128 threads,
// BJT_SMEM bytes of dynamic shared memory.
template <bool TRANS>
__global__ void __launch_bounds__(BJT_THREADS, BJT_MINB) k_bj_tc(BjTcArgs A, const float *Xt, const float *in, float *out) {
  extern __shared__ unsigned char bjt_raw[];
  __shared__ __align__(8) uint64_t bar[BJT_STAGES];
  __shared__ uint32_t s_tmem;
  __shared__ int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = A.n;
  const int nbt = (n + BJT - 1) / BJT;
  const int ge = blockIdx.x / nbt, bi = blockIdx.x - ge * nbt;
  const int e = A.elems[ge];
  const int r0 = blockIdx.y * BJT_N;
  const int64_t vb = A.dof_off[e];
  const int nblk = bjt_blocks(n);
  const float *tiles = Xt + A.tile_off[e] + (TRANS ? (int64_t)nblk * BJT_TILE : 0);
  // stage buffers on a 1024-byte boundary
  const uint32_t raw = bjt_smem(bjt_raw);
  unsigned char *sm = bjt_raw + (((raw + 1023u) & ~1023u) - raw);
  const uint32_t sbase = bjt_smem(sm);
  // K chunks of 32: X (lower) from 0 to the end of the diagonal tile, X^T from the diagonal tile on
  const int nk = (n + BJT_K - 1) / BJT_K;
  const int kc0 = TRANS ? 4 * bi : 0;
  const int kc1 = TRANS ? nk : min(4 * (bi + 1), nk);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(bjt_smem(&s_tmem)),
                 "r"(BJT_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < BJT_STAGES; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bjt_smem(&bar[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_bad = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  // registers of one chunk: A 8 float4 (rows q >> 3, 16-byte chunk q & 7 for
  // q = tid + 128 i), B 16 floats (right-hand side 16 warp + j, k = lane)
  float4 ra[8];
  float rb[16];
  auto load = [&](int kc) {
    const int bk = kc >> 2;
    const int b = TRANS ? (bi * nbt - bi * (bi - 1) / 2 + (bk - bi)) : (bi * (bi + 1) / 2 + bk);
    const float *blk = tiles + (int64_t)b * BJT_TILE + 32 * (kc & 3);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int q = tid + BJT_THREADS * i;
      ra[i] = *reinterpret_cast<const float4 *>(blk + (q >> 3) * BJT + 4 * (q & 7));
    }
    const int k = BJT_K * kc + lane;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int c = r0 + 16 * warp + j;
      rb[j] = (k < n && c < A.n_rhs) ? in[(int64_t)c * A.ndof + vb + k] : 0.0f;
    }
  };
  auto store = [&](int st) {
    unsigned char *sa_hi = sm + st * BJT_STAGE_BYTES, *sa_lo = sa_hi + BJT_A_BYTES;
    unsigned char *sb_hi = sa_lo + BJT_A_BYTES, *sb_lo = sb_hi + BJT_B_BYTES;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int q = tid + BJT_THREADS * i, m = q >> 3, c = q & 7;
      const int off = (m >> 3) * 1024 + (m & 7) * 128 + ((c ^ (m & 7)) << 4);
      const float4 v = ra[i];
      float4 h, l;
      h.x = bjt_tf32(v.x);
      h.y = bjt_tf32(v.y);
      h.z = bjt_tf32(v.z);
      h.w = bjt_tf32(v.w);
      l.x = bjt_tf32(v.x - h.x);
      l.y = bjt_tf32(v.y - h.y);
      l.z = bjt_tf32(v.z - h.z);
      l.w = bjt_tf32(v.w - h.w);
      *reinterpret_cast<float4 *>(sa_hi + off) = h;
      *reinterpret_cast<float4 *>(sa_lo + off) = l;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int nn = 16 * warp + j;
      const int off = (nn >> 3) * 1024 + (nn & 7) * 128 + ((((lane >> 2) ^ (nn & 7)) << 4) | ((lane & 3) << 2));
      const float h = bjt_tf32(rb[j]);
      *reinterpret_cast<float *>(sb_hi + off) = h;
      *reinterpret_cast<float *>(sb_lo + off) = bjt_tf32(rb[j] - h);
    }
  };

  load(kc0);
  int last = -1;
  for (int kc = kc0; kc < kc1; ++kc) {
    const int it = kc - kc0, st = it % BJT_STAGES;
    // the MMAs that last read this stage (iteration it - BJT_STAGES) are done
    if (it >= BJT_STAGES && tid == 0 && !bjt_wait(bjt_smem(&bar[st]), ((it - BJT_STAGES) / BJT_STAGES) & 1))
      s_bad = 1;
    __syncthreads();
    if (s_bad) break;
    store(st);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (kc + 1 < kc1) load(kc + 1);
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_hi = sbase + st * BJT_STAGE_BYTES, a_lo = a_hi + BJT_A_BYTES;
      const uint32_t b_hi = a_lo + BJT_A_BYTES, b_lo = b_hi + BJT_B_BYTES;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        // K-step s: 8 TF32 = 32 bytes further along the swizzled rows
        const uint64_t dah = bjt_desc(a_hi + 32 * s), dal = bjt_desc(a_lo + 32 * s);
        const uint64_t dbh = bjt_desc(b_hi + 32 * s), dbl = bjt_desc(b_lo + 32 * s);
        const uint64_t da[3] = {dah, dah, dal}, db[3] = {dbh, dbl, dbh};
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          const uint32_t acc = (it > 0 || s > 0 || p > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred q;\n\t"
              "setp.ne.b32 q, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n\t}" ::"r"(tmem),
              "l"(da[p]), "l"(db[p]), "r"(BJT_IDESC), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       bjt_smem(&bar[st]))
                   : "memory");
    }
    last = it;
  }
  // the last commit covers every MMA issued before it
  if (tid == 0 && !s_bad && last >= 0 &&
      !bjt_wait(bjt_smem(&bar[last % BJT_STAGES]), (last / BJT_STAGES) & 1))
    s_bad = 1;
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!s_bad) {
    const int row = BJT * bi + 32 * warp + lane;
#pragma unroll
    for (int c0 = 0; c0 < BJT_N; c0 += 16) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < n) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = r0 + c0 + j;
          if (c < A.n_rhs) out[(int64_t)c * A.ndof + vb + row] = __uint_as_float(v[j]);
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(A.err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BJT_TMEM_COLS) : "memory");
}

// tile set of every element of a group from the packed FP64 factor (row i at
// i (i + 1) / 2): lower tiles of X, then the tiles of X^T on and above the
// diagonal, FP32, zero outside the triangle and beyond n.
// grid: n_group * 2 * bjt_blocks(n), 256 threads.
__global__ void k_bj_tile(BjArgs A, const int64_t *tile_off, const double *X64, float *Xt) {
  const int n = A.n, nbt = (n + BJT - 1) / BJT, nblk = bjt_blocks(n);
  const int ge = blockIdx.x / (2 * nblk), rem = blockIdx.x - ge * 2 * nblk;
  const bool up = rem >= nblk;
  const int b = up ? rem - nblk : rem;
  int bi = 0, bk = 0;
  if (!up) {
    while ((bi + 1) * (bi + 2) / 2 <= b) ++bi;
    bk = b - bi * (bi + 1) / 2;
  } else {
    int cum = 0;
    while (cum + (nbt - bi) <= b) cum += nbt - bi++;
    bk = bi + (b - cum);
  }
  const int e = A.elems[ge];
  const double *Xe = X64 + A.blk_off[e];
  float *T = Xt + tile_off[e] + (int64_t)(up ? nblk + b : b) * BJT_TILE;
  for (int idx = threadIdx.x; idx < BJT_TILE; idx += blockDim.x) {
    const int i = BJT * bi + (idx >> 7), k = BJT * bk + (idx & 127);
    double v = 0.0;
    if (!up) {
      if (i < n && k <= i) v = Xe[pk(i, k)];
    } else {
      if (k < n && i <= k) v = Xe[pk(k, i)];
    }
    T[idx] = (float)v;
  }
}
