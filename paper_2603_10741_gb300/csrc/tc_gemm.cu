// Principal-block x cell-multivector product on the 5th-generation tensor cores (tcgen05) for the
// BF16 mixed mode: the local part of K^-rom (Eq. ifetidp_precond, Section 3.3.1) for all cells,
//   Y[rows of cell s] = [G; Phi^T]_{key(s)} X_R^s,   G = (K_RR^r)^{-1} of the cell's principal,
// as a segmented GEMM over cells grouped by key: one CTA computes MW tiles of 128 rows x TN
// cells of one key (TN = 128, MW = 1 in use) with A = rows of the key's augmented matrix and
// B = the cells' remaining values, accumulating
// in FP32 in tensor memory.  Each operand is a BF16 pair (high part and the BF16 rounding of the
// remainder) and three products G_hi X_hi + G_hi X_lo + G_lo X_hi accumulate into the same
// tile: ~16-bit operands, which the preconditioner needs on the ill-conditioned local problems
// of the corner-only primal set (one BF16 rounding stalls FGMRES near 1e-4 there).  The
// epilogue reads the accumulators with tcgen05.ld and applies the per-cell scale 1/c_s on the G
// rows.
//
// Operand staging.  Both operands are stored in global memory already tiled in the layout the
// tensor core reads from shared memory: the canonical no-swizzle K-major layout (8-row x 16-byte
// core matrices; K-adjacent core matrices 128 B apart, 8-row groups 1024 B apart), one
// contiguous 16 KiB block per (key, 128-row tile, 64-wide K panel) for A and one block per
// (cell tile, K panel) for B.  A K panel is then MW + 1 bulk copies (cp.async.bulk, completing
// on an mbarrier with their byte count).  One elected thread issues
// the copies and the MMAs (M = 128, N = TN, K = 16 per instruction), commits each stage's MMAs
// to that stage's "empty" barrier before refilling it, and a final commit releases the
// epilogue.  A stage carries one K panel of both BF16 halves of A and of B (64 KiB for TN =
// 128), so the three products of the panel cost one load of each operand; three stages are in
// flight.  Every wait is bounded: on a timeout the kernel flags an error, gives outstanding
// work a bounded chance to finish, frees its tensor memory and returns.
#include "common.cuh"

namespace {

constexpr int TM = 128;   // rows of an M tile (tensor-memory lanes)
constexpr int TK = 64;    // K panel
constexpr int KSTEP = 16; // K per tcgen05.mma, kind::f16
constexpr int A_ELEMS = TM * TK;       // 8192 bf16 = 16 KiB per M tile and K panel
constexpr int A_BYTES = A_ELEMS * 2;
constexpr uint32_t LBO = 128;              // K-adjacent core matrices
constexpr uint32_t SBO = (TK / 8) * 128;   // 8-row groups

// per-configuration sizes: TN cells per tile, MW M tiles of 128 rows per CTA
template <int TN, int MW>
struct TcCfg {
  static constexpr int B_ELEMS = TN * TK;
  static constexpr int B_BYTES = B_ELEMS * 2;
  // a stage holds one K panel of both BF16 halves of A (MW tiles) and of B: the three products
  // of the panel are issued from one load
  static constexpr int STAGE_BYTES = 2 * (MW * A_BYTES + B_BYTES);
  static constexpr int STAGES = MW == 1 ? 3 : 2;   // TN = 128: 3 x 64 KiB, or 2 x 96 KiB for two M tiles
  static constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES;
  static constexpr int TMEM_COLS = MW * TN;   // MW accumulators of TN FP32 columns
  // instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, N >> 3, M >> 4
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                                    ((uint32_t)(TM >> 4) << 24);
};

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
__host__ __device__ __forceinline__ int core_off(int r, int k) {
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

__device__ __forceinline__ void mbar_init(uint32_t addr) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(1) : "memory");
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// Tensor-core tile: rows [128 mt, 128 (mt + MW)) of the key's view of [G; Phi^T] (MW M tiles,
// the last CTA of a key may have one) times the TN cells of tile `tile` (key-ordered positions
// [c0, c0 + TN)).  GT: tiled high parts [key][mt][kp][8192] (low parts lo_off elements later),
// XT: tiled cell vectors [tile][2 KP][TN x 64] (high panels 0..KP-1, low panels KP..2KP-1).
// Stage p holds K panel p of G_hi, G_lo, X_hi and X_lo; the products G_hi X_hi, G_hi X_lo and
// G_lo X_hi of the panel accumulate into the same tensor-memory tile.  With MW = 2 every B panel
// feeds two M tiles (two accumulators in tensor memory).
template <int TN, int MW>
__global__ void __launch_bounds__(128)
    k_local_tc(int n_cells, int n_Kr, int n_P, int MT, int KP, int64_t lo_off, const __nv_bfloat16* __restrict__ GT,
               const __nv_bfloat16* __restrict__ XT, const int* __restrict__ tile_seg,
               const int* __restrict__ tile_c0, const int* __restrict__ seg_ptr, const int* __restrict__ perm,
               const double* __restrict__ cscale, const int* __restrict__ rr, const int* __restrict__ pdofs,
               double* __restrict__ Y, int* __restrict__ err, int mul_scale) {
  using C = TcCfg<TN, MW>;
  constexpr int STAGES = C::STAGES;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x, mt0 = blockIdx.y * MW;
  const int nm = min(MW, MT - mt0);          // M tiles of this CTA
  const int key = tile_seg[tile];
  const int c0 = tile_c0[tile];
  const int c_end = seg_ptr[key + 1];
  const int rows = n_Kr + n_P;
  const int P2 = KP;
  const uint32_t stage_tx = (uint32_t)(2 * (nm * A_BYTES + C::B_BYTES));
  const uint32_t s0 = smem_u32(smem);
  // stage layout: [A_hi tiles | A_lo tiles | B_hi | B_lo]
  auto sA = [&](int st, int m, int half) {
    return s0 + (uint32_t)(st * C::STAGE_BYTES + (half * MW + m) * A_BYTES);
  };
  auto sB = [&](int st, int half) { return s0 + (uint32_t)(st * C::STAGE_BYTES + 2 * MW * A_BYTES + half * C::B_BYTES); };
  auto gA = [&](int kp, int m, int half) {
    return (const void*)(GT + (((size_t)key * MT + mt0 + m) * KP + kp) * A_ELEMS + (half ? lo_off : 0));
  };
  auto gB = [&](int kp, int half) {
    return (const void*)(XT + ((size_t)tile * 2 * KP + (half ? KP + kp : kp)) * C::B_ELEMS);
  };
  auto load = [&](int kp, int st) {
    const uint32_t bar = smem_u32(&full[st]);
    expect_tx(bar, stage_tx);
    for (int half = 0; half < 2; ++half) {
      for (int m = 0; m < nm; ++m) bulk_copy(sA(st, m, half), gA(kp, m, half), (uint32_t)A_BYTES, bar);
      bulk_copy(sB(st, half), gB(kp, half), (uint32_t)C::B_BYTES, bar);
    }
  };
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]));
      mbar_init(smem_u32(&empty[s]));
    }
    mbar_init(smem_u32(&done));
    fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (tid == 0) {
    // producer and MMA issuer in one thread: copies run up to STAGES panels ahead.  The stage of
    // panel p - 1 is refilled after panel p's MMAs are queued, so that the tensor pipe always has
    // a panel queued while the thread waits for the previous one to drain.
    int issued = 0;
    for (; issued < STAGES && issued < P2; ++issued) load(issued, issued);
    bool ok = true;
    for (int p = 0; p < P2; ++p) {
      const int st = p % STAGES;
      const uint32_t ph = (uint32_t)((p / STAGES) & 1);
      if (!mbar_wait(smem_u32(&full[st]), ph)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int m = 0; m < nm; ++m) {
#pragma unroll
        for (int ks = 0; ks < TK / KSTEP; ++ks) {
          // G_hi X_hi, G_hi X_lo, G_lo X_hi (the G_lo X_lo term is below the pairs' precision)
#pragma unroll
          for (int pass = 0; pass < 3; ++pass) {
            const uint64_t ad = make_desc(sA(st, m, pass == 2) + ks * 2 * 128);
            const uint64_t bd = make_desc(sB(st, pass == 1) + ks * 2 * 128);
            const uint32_t acc = (p > 0 || ks > 0 || pass > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred q;\n\t"
                "setp.ne.b32 q, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}" ::"r"(tmem + (uint32_t)(m * TN)),
                "l"(ad), "l"(bd), "r"(C::IDESC), "r"(acc)
                : "memory");
          }
        }
      }
      mma_commit(smem_u32(&empty[st]));
      if (p >= 1 && issued < P2) {
        // refill the previous panel's stage once its MMAs have read it
        const int sp = (p - 1) % STAGES;
        if (!mbar_wait(smem_u32(&empty[sp]), (uint32_t)(((p - 1) / STAGES) & 1))) {
          ok = false;
          break;
        }
        load(issued, sp);
        ++issued;
      }
    }
    if (!ok) {
      fail = 1;
      atomicOr(err, 4);
      // let copies in flight land (bounded) before the shared memory is released
      for (int q = 0; q < issued; ++q) mbar_wait(smem_u32(&full[q % STAGES]), (uint32_t)((q / STAGES) & 1));
    }
    mma_commit(smem_u32(&done));   // arrives when every MMA issued above has completed
  }
  // everyone: accumulators complete (bounded wait)
  const bool fin = mbar_wait(smem_u32(&done), 0);
  __syncthreads();
  const bool ok = fin && !fail;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (__syncthreads_and(ok ? 1 : 0)) {
    // epilogue: warp w reads accumulator lanes 32w..32w+31 (tile rows), 16 columns at a time,
    // and writes them through a per-warp transpose tile in the (now idle) pipeline shared memory,
    // so that the 16 lanes of a half-warp store 16 consecutive cells of one output row
    float* tb = reinterpret_cast<float*>(smem) + warp * 32 * 17;
    const int half = lane >> 4, j16 = lane & 15;
    for (int m = 0; m < nm; ++m) {
      const int row0 = (mt0 + m) * TM + warp * 32;
#pragma unroll 1
      for (int cb = 0; cb < TN; cb += 16) {
        uint32_t r[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(m * TN + cb);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) tb[lane * 17 + j] = __uint_as_float(r[j]);
        __syncwarp();
        const int pos = c0 + cb + j16;
        const bool col_ok = pos < c_end;
        const int s = col_ok ? perm[pos] : 0;
        // the cell's factor c_s (S_DD rows) or 1 / c_s (G rows), one division per column
        const double cs = col_ok ? cscale[s] : 1.0;
        const double fac = mul_scale ? cs : 1.0 / cs;
#pragma unroll 4
        for (int q = 0; q < 16; ++q) {
          const int rl = 2 * q + half;
          const int gi = row0 + rl;
          if (col_ok && gi < rows) {
            const size_t orow = (size_t)(gi < n_Kr ? rr[gi] : pdofs[gi - n_Kr]);
            const double v = (double)tb[rl * 17 + j16];
            Y[orow * n_cells + s] = gi < n_Kr ? v * fac : v;
          }
        }
        __syncwarp();
      }
    }
  } else if (tid == 0) {
    atomicOr(err, 4);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
  }
}

// cell vectors of every tile, BF16 pairs in the tiled layout: XT[tile][kx][core_off(c, k)] with
// kx = kp (high part) or KP + kp (low part), cell c = position c0 + c of the tile's key segment
// (zero past the segment's end), column kp * 64 + k of the view (zero beyond n_K).  One CTA per
// (tile, kp); gathered 8-byte reads, 16-byte writes.
template <int TN>
__global__ void k_pack_xt(int n_cells, int n_K, int KP, const double* __restrict__ X, const int* __restrict__ tile_seg,
                          const int* __restrict__ tile_c0, const int* __restrict__ seg_ptr, const int* __restrict__ perm,
                          const int* __restrict__ rc, __nv_bfloat16* __restrict__ XT) {
  constexpr int BE = TN * TK;
  __shared__ __align__(16) __nv_bfloat16 hi[BE], lo[BE];
  const int tile = blockIdx.x, kp = blockIdx.y;
  const int c0 = tile_c0[tile];
  const int c_end = seg_ptr[tile_seg[tile] + 1];
  for (int t = threadIdx.x; t < TN * TK; t += blockDim.x) {
    const int k = t / TN, c = t % TN;                          // consecutive threads: consecutive cells
    const int pos = c0 + c, gk = kp * TK + k;
    float v = 0.f;
    if (pos < c_end && gk < n_K) v = (float)X[(size_t)rc[gk] * n_cells + perm[pos]];
    const __nv_bfloat16 h = __float2bfloat16(v);
    hi[core_off(c, k)] = h;
    lo[core_off(c, k)] = __float2bfloat16(v - __bfloat162float(h));
  }
  __syncthreads();
  uint4* dh = reinterpret_cast<uint4*>(XT + ((size_t)tile * 2 * KP + kp) * BE);
  uint4* dl = reinterpret_cast<uint4*>(XT + ((size_t)tile * 2 * KP + KP + kp) * BE);
  for (int t = threadIdx.x; t < BE / 8; t += blockDim.x) {
    dh[t] = reinterpret_cast<const uint4*>(hi)[t];
    dl[t] = reinterpret_cast<const uint4*>(lo)[t];
  }
}

// the same tiles for an operand supported on the dual DOFs and given as B^T lambda (scaled by
// 1/multiplicity when lsc is given): each copy's value is formed from its multipliers through
// the per-(dual DOF, cell) table instead of being scattered into a zeroed local vector first
template <int TN>
__global__ void k_pack_lam(int n_cells, int n_D, int KP, const double* __restrict__ lam, const int2* __restrict__ lk,
                           const float* __restrict__ lsc, const int* __restrict__ tile_seg,
                           const int* __restrict__ tile_c0, const int* __restrict__ seg_ptr,
                           const int* __restrict__ perm, __nv_bfloat16* __restrict__ XT) {
  constexpr int BE = TN * TK;
  __shared__ __align__(16) __nv_bfloat16 hi[BE], lo[BE];
  const int tile = blockIdx.x, kp = blockIdx.y;
  const int c0 = tile_c0[tile];
  const int c_end = seg_ptr[tile_seg[tile] + 1];
  for (int t = threadIdx.x; t < TN * TK; t += blockDim.x) {
    const int k = t / TN, c = t % TN;                          // consecutive threads: consecutive cells
    const int pos = c0 + c, gk = kp * TK + k;
    float v = 0.f;
    if (pos < c_end && gk < n_D) {
      const size_t q = (size_t)gk * n_cells + perm[pos];
      // formed in FP32 (the value is rounded to FP32 and split into a BF16 pair anyway): only
      // the two multiplier reads convert from FP64, the FP64 pipe being the narrow one here
      const int2 l = lk[q];
      float a = 0.f;
      if (l.x) a = l.x > 0 ? __double2float_rn(lam[l.x - 1]) : -__double2float_rn(lam[-l.x - 1]);
      if (l.y) a += l.y > 0 ? __double2float_rn(lam[l.y - 1]) : -__double2float_rn(lam[-l.y - 1]);
      if (lsc) a *= lsc[q];
      v = a;
    }
    const __nv_bfloat16 h = __float2bfloat16(v);
    hi[core_off(c, k)] = h;
    lo[core_off(c, k)] = __float2bfloat16(v - __bfloat162float(h));
  }
  __syncthreads();
  uint4* dh = reinterpret_cast<uint4*>(XT + ((size_t)tile * 2 * KP + kp) * BE);
  uint4* dl = reinterpret_cast<uint4*>(XT + ((size_t)tile * 2 * KP + KP + kp) * BE);
  for (int t = threadIdx.x; t < BE / 8; t += blockDim.x) {
    dh[t] = reinterpret_cast<const uint4*>(hi)[t];
    dl[t] = reinterpret_cast<const uint4*>(lo)[t];
  }
}

// a view of G (rows_v rows of n_K columns from (G, row stride ldsrc, key stride kstride)) as BF16
// pairs in the tiled layout: GT[key][mt][kp][core_off(r, k)] high parts, the low parts
// (BF16 rounding of G - hi) lo_off elements later; zero outside the view
__global__ void k_g_tile(int64_t keys, int rows_v, int n_K, int MT, int KP, int ldsrc, int64_t kstride,
                         const double* __restrict__ G, int64_t lo_off, __nv_bfloat16* __restrict__ GT) {
  const int64_t n = keys * MT * KP * A_ELEMS;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int64_t blk = t / A_ELEMS;
  const int e = (int)(t % A_ELEMS);
  // invert core_off: e = (r >> 3) * 512 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7)
  const int r = (e >> 9) * 8 + ((e >> 3) & 7);
  const int k = ((e >> 6) & 7) * 8 + (e & 7);
  const int kp = (int)(blk % KP);
  const int64_t mk = blk / KP;
  const int mt = (int)(mk % MT);
  const int64_t key = mk / MT;
  const int gr = mt * TM + r, gk = kp * TK + k;
  const float v = (gr < rows_v && gk < n_K) ? (float)G[key * kstride + (int64_t)gr * ldsrc + gk] : 0.f;
  const __nv_bfloat16 h = __float2bfloat16(v);
  GT[t] = h;
  GT[lo_off + t] = __float2bfloat16(v - __bfloat162float(h));
}

}  // namespace

// BF16 pairs of the augmented local matrices (after the FP64 Gauss-Jordan sweep) for the three
// views of the local products (whole; dual columns; trailing dual block), tiled for the bulk
// copies of the tensor-core kernel
void run_g_to_bf16(lat_ctx* h, size_t n) {
  const int nR = h->n_R, nP = h->n_P, nI = h->n_I;
  const int64_t keys = (int64_t)(n / ((size_t)(nR + nP) * nR));
  const int64_t kstride = (int64_t)(nR + nP) * nR;
  for (int mode = 0; mode < 3; ++mode) {
    const int lo_r = mode == KINV_DUAL ? nI : 0, lo_c = mode == KINV_FULL ? 0 : nI;
    const int nKr = nR - lo_r, nKc = nR - lo_c;
    const int MT = div_up(nKr + nP, TM), KP = std::max(1, div_up(nKc, TK));
    const int64_t cnt = keys * MT * KP * A_ELEMS;
    h->G16[mode].ensure((size_t)2 * cnt);   // high and low parts
    h->g16_ld[mode] = KP;
    h->g16_lo[mode] = cnt;
    LAT_LAUNCH(h, k_g_tile<<<div_up(cnt, 256), 256, 0, h->stream>>>(keys, nKr + nP, nKc, MT, KP, nR, kstride,
                                                                      h->G.p + (size_t)lo_r * nR + lo_c, cnt,
                                                                      h->G16[mode].p));
  }
  // the dual Schur complements S_DD [keys][n_D][n_D] of the Dirichlet interface preconditioner
  const int nD = nR - nI;
  if (nD > 0 && h->SDD.p) {
    const int MT = div_up(nD, TM), KP = std::max(1, div_up(nD, TK));
    const int64_t cnt = keys * MT * KP * A_ELEMS;
    h->G16[3].ensure((size_t)2 * cnt);
    h->g16_ld[3] = KP;
    h->g16_lo[3] = cnt;
    LAT_LAUNCH(h, k_g_tile<<<div_up(cnt, 256), 256, 0, h->stream>>>(keys, nD, nD, MT, KP, nD, (int64_t)nD * nD,
                                                                      h->SDD.p, cnt, h->G16[3].p));
  }
  LAT_CHECK_LAUNCH();
}

namespace {

template <int TN, int MW>
void launch_tc(lat_ctx* h, const double* X, double* Y, KinvMode mode, const int* tseg, const int* tc0, int n_tiles,
               const double* lam = nullptr) {
  using C = TcCfg<TN, MW>;
  const int lo_r = mode == KINV_DUAL ? h->n_I : 0, lo_c = mode == KINV_FULL ? 0 : h->n_I;
  const int nKr = h->n_R - lo_r, nKc = h->n_R - lo_c;
  const int MT = div_up(nKr + h->n_P, TM);
  const int KP = h->g16_ld[mode];
  const int* rr = h->rdofs.p + lo_r;
  const int* rc = h->rdofs.p + lo_c;
  const int KPmax = std::max(1, div_up(h->n_R, TK));
  h->Xb16.ensure((size_t)n_tiles * 2 * KPmax * C::B_ELEMS);
  if (lam)   // the dual view's operand is B^T lambda (mode KINV_DUAL: columns = the dual DOFs)
    LAT_LAUNCH(h, k_pack_lam<TN><<<dim3(n_tiles, KP), 256, 0, h->stream>>>(h->n_cells, nKc, KP, lam, h->dual_lk.p,
                                                                            nullptr, tseg, tc0, h->seg_ptr.p,
                                                                            h->perm.p, h->Xb16.p));
  else
    LAT_LAUNCH(h, k_pack_xt<TN><<<dim3(n_tiles, KP), 256, 0, h->stream>>>(h->n_cells, nKc, KP, X, tseg, tc0,
                                                                           h->seg_ptr.p, h->perm.p, rc, h->Xb16.p));
  LAT_CUDA(cudaFuncSetAttribute(k_local_tc<TN, MW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)C::SMEM_BYTES));
  dim3 grid(n_tiles, div_up(MT, MW));
  static const char* const tg[3] = {"local_tc", "local_tc_dual", "local_tc_dual_in"};
  KernelTimer kt(h, tg[mode]);
  LAT_LAUNCH(h, (k_local_tc<TN, MW><<<grid, 128, C::SMEM_BYTES, h->stream>>>(
                    h->n_cells, nKr, h->n_P, MT, KP, h->g16_lo[mode], h->G16[mode].p, h->Xb16.p, tseg, tc0,
                    h->seg_ptr.p, h->perm.p, h->c_cell.p, rr, h->pdofs.p, Y, h->flag.p, 0)));
  LAT_CHECK_LAUNCH();
}

// the Dirichlet interface preconditioner's local products y_D = c_s S_DD x_D on the same tiles
// (dual rows and columns, no corner rows, scaled by c_s)
template <int TN>
void launch_sdd_tc(lat_ctx* h, const double* X, double* Y, const double* lam) {
  using C = TcCfg<TN, 1>;
  const int nD = h->n_R - h->n_I;
  const int MT = div_up(nD, TM);
  const int KP = h->g16_ld[3];
  const int* rd = h->rdofs.p + h->n_I;
  const int KPmax = std::max(1, div_up(h->n_R, TK));
  h->Xb16.ensure((size_t)h->max_tiles_tc * 2 * KPmax * C::B_ELEMS);
  if (lam)   // the operand is B_D^T lambda: B^T lambda scaled by 1/multiplicity
    LAT_LAUNCH(h, k_pack_lam<TN><<<dim3(h->max_tiles_tc, KP), 256, 0, h->stream>>>(
                      h->n_cells, nD, KP, lam, h->dual_lk.p, h->dual_lsc.p, h->tile_seg_tc.p, h->tile_c0_tc.p,
                      h->seg_ptr.p, h->perm.p, h->Xb16.p));
  else
    LAT_LAUNCH(h, k_pack_xt<TN><<<dim3(h->max_tiles_tc, KP), 256, 0, h->stream>>>(h->n_cells, nD, KP, X, h->tile_seg_tc.p,
                                                                                h->tile_c0_tc.p, h->seg_ptr.p, h->perm.p,
                                                                                rd, h->Xb16.p));
  LAT_CUDA(cudaFuncSetAttribute(k_local_tc<TN, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)C::SMEM_BYTES));
  dim3 grid(h->max_tiles_tc, MT);
  KernelTimer kt(h, "dual_schur_tc");
  LAT_LAUNCH(h, (k_local_tc<TN, 1><<<grid, 128, C::SMEM_BYTES, h->stream>>>(
                    h->n_cells, nD, 0, MT, KP, h->g16_lo[3], h->G16[3].p, h->Xb16.p, h->tile_seg_tc.p, h->tile_c0_tc.p,
                    h->seg_ptr.p, h->perm.p, h->c_cell.p, rd, h->pdofs.p, Y, h->flag.p, 1)));
  LAT_CHECK_LAUNCH();
}

}  // namespace

// Y (rows of every cell, per the view: see KinvMode) = [G; Phi^T] X on the tensor cores, on
// 128-cell tiles of each key's cells, one CTA per SM.
void run_local_tc(lat_ctx* h, const double* X, double* Y, KinvMode mode) {
  launch_tc<kTcCells, kTcRowTiles>(h, X, Y, mode, h->tile_seg_tc.p, h->tile_c0_tc.p, h->max_tiles_tc);
}

void run_sdd_tc(lat_ctx* h, const double* X, double* Y, const double* lam) { launch_sdd_tc<kTcCells>(h, X, Y, lam); }

// the dual view of [G; Phi^T] applied to B^T lambda (the interface operator's local products)
void run_local_tc_lam(lat_ctx* h, const double* lam, double* Y) {
  launch_tc<kTcCells, kTcRowTiles>(h, nullptr, Y, KINV_DUAL, h->tile_seg_tc.p, h->tile_c0_tc.p, h->max_tiles_tc, lam);
}
