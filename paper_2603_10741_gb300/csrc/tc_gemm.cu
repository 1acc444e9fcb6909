// Principal-block x cell-multivector product on the 5th-generation tensor cores (tcgen05) for the
// BF16 mixed mode: the local part of K^-rom (Eq. ifetidp_precond, Section 3.3.1) for all cells,
//   Y[rows of cell s] = [G; Phi^T]_{key(s)} X_R^s,   G = (K_RR^r)^{-1} of the cell's principal,
// as a segmented GEMM over cells grouped by key: one CTA computes a 128-row x 64-cell tile of
// one key with A = the key's augmented matrix (BF16, K-major, rows padded to the K panel) and
// B = the 64 cells' remaining values, packed once per product into a BF16 buffer in key order
// (K-major), accumulating in FP32 in tensor memory.  Each operand is a BF16 pair (high part and
// the BF16 rounding of the remainder) and three products G_hi X_hi + G_hi X_lo + G_lo X_hi
// accumulate into the same tile: ~16-bit operands, which the preconditioner needs on the
// ill-conditioned local problems of the corner-only primal set (one BF16 rounding stalls FGMRES
// near 1e-4 there).  The epilogue reads the accumulator with tcgen05.ld and applies the
// per-cell scale 1/c_s on the G rows.
//
// Both operands are copied with 16-byte cp.async into shared memory in the canonical
// no-swizzle K-major layout (8-row x 16-byte core matrices; K-adjacent core matrices 128 B
// apart, 8-row groups 1024 B apart), two K panels in flight; one elected thread issues
// tcgen05.mma (M = 128, N = 64, K = 16 per instruction) and commits to the stage's mbarrier,
// which every thread waits on (bounded) before that stage is refilled.  48 KiB of shared memory
// and 64 tensor-memory columns per CTA let four CTAs share an SM.
#include "common.cuh"

namespace {

constexpr int TM = 128;   // rows of the tile (tensor-memory lanes)
constexpr int TN = 64;    // cells of the tile (accumulator columns)
constexpr int TK = 64;    // K panel staged per round
constexpr int KSTEP = 16; // K per tcgen05.mma, kind::f16
constexpr int TMEM_COLS = 64;     // one FP32 accumulator column per cell of the tile
constexpr int A_BYTES = TM * TK * 2;   // 16 KiB
constexpr int B_BYTES = TN * TK * 2;   // 8 KiB
constexpr size_t SMEM_BYTES = 2 * (A_BYTES + B_BYTES);   // two pipeline stages
constexpr uint32_t LBO = 128;              // K-adjacent core matrices
constexpr uint32_t SBO = (TK / 8) * 128;   // 8-row groups

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, N >> 3, M >> 4
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start, leading (K) and stride (8-row group) byte offsets,
// version 1, no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((LBO >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((SBO >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// element (row r, k) of a K-major panel with TK columns, in bf16 elements
__device__ __forceinline__ int core_off(int r, int k) {
  return (r >> 3) * (TK / 8) * 64 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  for (int i = 0; i < (1 << 20); ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(g), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Tensor-core tile: rows [i0, i0+128) of the key's augmented matrix (BF16, row stride ldg)
// times the 64 packed cell vectors at key-ordered positions [c0, c0+64) (BF16, row stride kp).
// K panels of 64 flow through a 2-stage shared-memory pipeline filled by cp.async: the loads of
// panel p+1 overlap the MMAs of panel p; a stage is refilled only after the mbarrier of the MMAs
// that read it has completed.
__global__ void __launch_bounds__(128)
    k_local_tc(int n_cells, int n_Kr, int n_Kc, int n_P, int ldg, int kp_pad, int64_t lo_off,
               const __nv_bfloat16* __restrict__ G16,
               const __nv_bfloat16* __restrict__ Xb, const int* __restrict__ tile_seg,
               const int* __restrict__ tile_c0, const int* __restrict__ seg_ptr, const int* __restrict__ perm,
               const double* __restrict__ cscale, const int* __restrict__ rr, const int* __restrict__ pdofs,
               double* __restrict__ Y, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int key = tile_seg[blockIdx.x];
  const int c0 = tile_c0[blockIdx.x];
  const int c_end = seg_ptr[key + 1];
  const int rows = n_Kr + n_P;
  const int i0 = blockIdx.y * TM;
  const __nv_bfloat16* g = G16 + (size_t)key * rows * ldg;
  auto stageA = [&](int st) { return smem_u32(smem) + st * (A_BYTES + B_BYTES); };
  auto stageB = [&](int st) { return smem_u32(smem) + st * (A_BYTES + B_BYTES) + A_BYTES; };
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(1) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  // Both operands are split into a high and a low BF16 part (G = G_hi + G_lo at lo_off elements
  // after G_hi; X = X_hi + X_lo, row layout [X_hi | X_lo]); three passes of P K panels each,
  // G_hi X_hi + G_hi X_lo + G_lo X_hi, accumulate into one FP32 tensor-memory tile
  const int P = (n_Kc + TK - 1) / TK;
  auto load_panel = [&](int p, int st) {
    const int pass = p / P;
    const int kp = (p - pass * P) * TK;                    // matrix column
    const int kx = (pass == 1 ? P * TK : 0) + kp;          // packed vector column
    const __nv_bfloat16* gp = pass == 2 ? g + lo_off : g;
    const uint32_t a0 = stageA(st), b0 = stageB(st);
    for (int t = tid; t < TM * (TK / 8); t += 128) {         // A: 128 rows x 8 chunks
      const int r = t >> 3, kc = t & 7;
      const int gi = i0 + r;
      const bool v = gi < rows;
      cp_async16(a0 + 2 * core_off(r, kc * 8), v ? (const void*)(gp + (size_t)gi * ldg + kp + kc * 8) : (const void*)G16,
                 v ? 16u : 0u);
    }
    for (int t = tid; t < TN * (TK / 8); t += 128) {         // B: 64 cells x 8 chunks
      const int c = t >> 3, kc = t & 7;
      const int pos = c0 + c;
      const bool v = pos < c_end;
      cp_async16(b0 + 2 * core_off(c, kc * 8),
                 v ? (const void*)(Xb + (size_t)pos * kp_pad + kx + kc * 8) : (const void*)Xb, v ? 16u : 0u);
    }
    cp_async_commit();
  };
  const int P2 = 3 * P;
  uint32_t ph[2] = {0u, 0u};
  bool ok = true;
  load_panel(0, 0);
  for (int p = 0; p < P2; ++p) {
    const int st = p & 1;
    if (p + 1 < P2) {
      const int nx = (p + 1) & 1;
      if (p >= 1) {                                           // MMAs of panel p-1 read stage nx
        const bool done = mbar_wait(smem_u32(&mbar[nx]), ph[nx]);
        ok = __syncthreads_and(done ? 1 : 0) != 0;
        if (!ok) break;
        ph[nx] ^= 1u;
      }
      load_panel(p + 1, nx);
      cp_async_wait<1>();                                     // panel p has landed
    } else {
      cp_async_wait<0>();
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int ks = 0; ks < TK / KSTEP; ++ks) {
        const uint64_t ad = make_desc(stageA(st) + ks * 2 * 128);
        const uint64_t bd = make_desc(stageB(st) + ks * 2 * 128);
        const uint32_t acc = (p > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred q;\n\t"
            "setp.ne.b32 q, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar[st]))
                   : "memory");
    }
  }
  if (ok) {
    const int last = (P2 - 1) & 1;
    const bool done = mbar_wait(smem_u32(&mbar[last]), ph[last]);
    ok = __syncthreads_and(done ? 1 : 0) != 0;
  }
  cp_async_wait<0>();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    // epilogue: warp w reads accumulator lanes 32w..32w+31 (tile rows), 16 columns at a time
    const int gi = i0 + warp * 32 + lane;
    const bool row_ok = gi < rows;
    const size_t orow = row_ok ? (size_t)(gi < n_Kr ? rr[gi] : pdofs[gi - n_Kr]) : 0;
#pragma unroll
    for (int cb = 0; cb < TN; cb += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row_ok) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int pos = c0 + cb + j;
          if (pos >= c_end) continue;
          const int s = perm[pos];
          const double v = (double)__uint_as_float(r[j]);
          Y[orow * n_cells + s] = gi < n_Kr ? v / cscale[s] : v;
        }
      }
    }
  } else {
    if (tid == 0) atomicOr(err, 4);
    // give MMAs still in flight a bounded chance to finish before the tensor memory is released
    mbar_wait(smem_u32(&mbar[0]), ph[0]);
    mbar_wait(smem_u32(&mbar[1]), ph[1]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// packed BF16 cell vectors in key order, split into a high and a low part so that the product
// sees the vector to ~16 mantissa bits (a single BF16 rounding of the vector, 8 bits, is
// renewed at every preconditioner application and stalls FGMRES near 1e-4):
//   Xb[pos][k] = hi, Xb[pos][kp + k] = lo,  hi + lo ~ X[rdofs[k]][perm[pos]],  zero beyond n_R
// (64-position x 64-k tiles through shared memory: gathered reads, 16-byte writes)
__global__ void k_pack_x(int n_cells, int n_R, int kp, const double* __restrict__ X, const int* __restrict__ perm,
                         const int* __restrict__ rdofs, __nv_bfloat16* __restrict__ Xb) {
  __shared__ __align__(16) __nv_bfloat16 tile[2][64][64 + 8];
  const int pos0 = blockIdx.x * 64, k0 = blockIdx.y * 64;
  for (int t = threadIdx.x; t < 64 * 64; t += blockDim.x) {
    const int kk = t / 64, pp = t % 64;                      // consecutive threads: consecutive positions
    const int pos = pos0 + pp, k = k0 + kk;
    float v = 0.f;
    if (pos < n_cells && k < n_R) v = (float)X[(size_t)rdofs[k] * n_cells + perm[pos]];
    const __nv_bfloat16 hi = __float2bfloat16(v);
    tile[0][pp][kk] = hi;
    tile[1][pp][kk] = __float2bfloat16(v - __bfloat162float(hi));
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 2 * 64 * 8; t += blockDim.x) {
    const int part = t / 512, pp = (t / 8) % 64, kc = t % 8;
    const int pos = pos0 + pp;
    if (pos < n_cells)
      *reinterpret_cast<uint4*>(Xb + (size_t)pos * 2 * kp + part * kp + k0 + kc * 8) =
          *reinterpret_cast<const uint4*>(&tile[part][pp][kc * 8]);
  }
}

// view of G (rows_v rows of n_K columns, row stride ldsrc, key stride kstride) -> BF16 high
// part [keys][rows_v][ld_dst] followed by the BF16 low part (G - hi) of the same shape, zero
// padded beyond n_K
__global__ void k_g_bf16_view(int64_t keys, int rows_v, int n_K, int ldsrc, int64_t kstride,
                              const double* __restrict__ G, int ld_dst, __nv_bfloat16* __restrict__ G16) {
  const int64_t n = keys * rows_v * ld_dst;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int64_t row = t / ld_dst;
  const int k = (int)(t % ld_dst);
  const int64_t key = row / rows_v;
  const int r = (int)(row % rows_v);
  const float v = k < n_K ? (float)G[key * kstride + (int64_t)r * ldsrc + k] : 0.f;
  const __nv_bfloat16 hi = __float2bfloat16(v);
  G16[t] = hi;
  G16[n + t] = __float2bfloat16(v - __bfloat162float(hi));
}

}  // namespace

// BF16 copies of the augmented local matrices (after the FP64 Gauss-Jordan sweep) for the three
// views of the local products (whole; dual columns; trailing dual block), rows padded to a
// multiple of the K panel
void run_g_to_bf16(lat_ctx* h, size_t n) {
  const int nR = h->n_R, nP = h->n_P, nI = h->n_I;
  const int64_t keys = (int64_t)(n / ((size_t)(nR + nP) * nR));
  const int64_t kstride = (int64_t)(nR + nP) * nR;
  for (int mode = 0; mode < 3; ++mode) {
    const int lo_r = mode == KINV_DUAL ? nI : 0, lo_c = mode == KINV_FULL ? 0 : nI;
    const int nKr = nR - lo_r, nKc = nR - lo_c;
    const int ld = std::max(TK, (nKc + TK - 1) / TK * TK);
    h->G16[mode].ensure((size_t)2 * keys * (nKr + nP) * ld);   // high and low parts
    h->g16_ld[mode] = ld;
    h->g16_lo[mode] = keys * (nKr + nP) * ld;
    const int64_t cnt = keys * (nKr + nP) * ld;
    LAT_LAUNCH(h, k_g_bf16_view<<<div_up(cnt, 256), 256, 0, h->stream>>>(keys, nKr + nP, nKc, nR, kstride,
                                                                          h->G.p + (size_t)lo_r * nR + lo_c, ld,
                                                                          h->G16[mode].p));
  }
  LAT_CHECK_LAUNCH();
}

// Y (rows of every cell, per the view: see KinvMode) = [G; Phi^T] X on the tensor cores.  The tile
// list groups cells of one key in runs of 64 (seg_bn = 64 in the mixed modes).
void run_local_tc(lat_ctx* h, const double* X, double* Y, KinvMode mode) {
  const int lo_r = mode == KINV_DUAL ? h->n_I : 0, lo_c = mode == KINV_FULL ? 0 : h->n_I;
  const int nKr = h->n_R - lo_r, nKc = h->n_R - lo_c;
  const int rows = nKr + h->n_P;
  const int kp = h->g16_ld[mode];
  const int* rr = h->rdofs.p + lo_r;
  const int* rc = h->rdofs.p + lo_c;
  h->Xb16.ensure((size_t)h->n_cells * 2 * h->g16_ld[KINV_FULL]);
  LAT_LAUNCH(h, k_pack_x<<<dim3(div_up(h->n_cells, 64), kp / 64), 256, 0, h->stream>>>(h->n_cells, nKc, kp, X,
                                                                                        h->perm.p, rc, h->Xb16.p));
  LAT_CUDA(cudaFuncSetAttribute(k_local_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
  dim3 grid(h->max_tiles, div_up(rows, TM));
  static const char* const tg[3] = {"local_tc", "local_tc_dual", "local_tc_dual_in"};
  KernelTimer kt(h, tg[mode]);
  LAT_LAUNCH(h, k_local_tc<<<grid, 128, SMEM_BYTES, h->stream>>>(h->n_cells, nKr, nKc, h->n_P, kp, 2 * kp,
                                                                  h->g16_lo[mode],
                                                                  h->G16[mode].p, h->Xb16.p, h->tile_seg.p,
                                                                  h->tile_c0.p, h->seg_ptr.p, h->perm.p,
                                                                  h->c_cell.p, rr, h->pdofs.p, Y, h->flag.p));
  LAT_CHECK_LAUNCH();
}
