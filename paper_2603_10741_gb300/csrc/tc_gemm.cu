// Principal-block x cell-multivector product on the 5th-generation tensor cores (tcgen05) for the
// BF16 mixed mode: the local part of K^-rom (Eq. ifetidp_precond, Section 3.3.1) for all cells,
//   Y[rows of cell s] = [G; Phi^T]_{key(s)} X_R^s,   G = (K_RR^r)^{-1} of the cell's principal,
// as a segmented GEMM over cells grouped by key: one CTA computes a 128-row x 64-cell tile of
// one key with A = the key's augmented matrix (BF16, K-major) and B = the 64 cells' remaining
// values (FP64 -> BF16 on load, K-major), accumulating in FP32 in tensor memory.  The epilogue
// reads the accumulator with tcgen05.ld and applies the per-cell scale 1/c_s on the G rows.
//
// Operands are staged by the CTA's threads into shared memory in the canonical no-swizzle
// K-major layout (8-row x 16-byte core matrices; K-adjacent core matrices 128 B apart, 8-row
// groups 1024 B apart); one elected thread issues tcgen05.mma (M = 128, N = 64, K = 16 per
// instruction) and commits to an mbarrier that every thread waits on (bounded) before the
// panel buffers are refilled.  Shared memory (64 KiB) and tensor memory (256 columns) are
// allocated above what the tile needs.
#include "common.cuh"

namespace {

constexpr int TM = 128;   // rows of the tile (tensor-memory lanes)
constexpr int TN = 64;    // cells of the tile (accumulator columns)
constexpr int TK = 64;    // K panel staged per round
constexpr int KSTEP = 16; // K per tcgen05.mma, kind::f16
constexpr int TMEM_COLS = 256;
constexpr size_t SMEM_BYTES = 64 * 1024;
constexpr int A_BYTES = TM * TK * 2;   // 16 KiB
constexpr int B_BYTES = TN * TK * 2;   // 8 KiB
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

__global__ void __launch_bounds__(128)
    k_local_tc(int n_cells, int n_R, int n_P, const __nv_bfloat16* __restrict__ G16,
               const int* __restrict__ tile_seg, const int* __restrict__ tile_c0, const int* __restrict__ seg_ptr,
               const int* __restrict__ perm, const double* __restrict__ cscale, const int* __restrict__ rdofs,
               const int* __restrict__ pdofs, const double* __restrict__ X, double* __restrict__ Y,
               int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(smem);
  __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(smem + A_BYTES);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int cells[TN];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x;
  const int key = tile_seg[tile];
  const int c0 = tile_c0[tile];
  const int c_end = seg_ptr[key + 1];
  const int rows = n_R + n_P;
  const int i0 = blockIdx.y * TM;
  const __nv_bfloat16* g = G16 + (size_t)key * rows * n_R;
  if (tid < TN) {
    const int c = c0 + tid;
    cells[tid] = c < c_end ? perm[c] : -1;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  const uint32_t mb = smem_u32(&mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  uint32_t parity = 0;
  bool ok = true;
  for (int kp = 0; kp < n_R && ok; kp += TK) {
    // A panel: rows i0.., K kp.. (16-byte chunks of 8 bf16)
    for (int t = tid; t < TM * (TK / 8); t += blockDim.x) {
      const int r = t / (TK / 8), kc = t % (TK / 8);
      const int gi = i0 + r, gk = kp + kc * 8;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (gi < rows && gk < n_R) {
        const __nv_bfloat16* src = g + (size_t)gi * n_R + gk;
        if (gk + 8 <= n_R && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
          v = *reinterpret_cast<const uint4*>(src);
        } else {
          union {
            uint4 u;
            __nv_bfloat16 h[8];
          } tmp;
#pragma unroll
          for (int e = 0; e < 8; ++e) tmp.h[e] = (gk + e < n_R) ? src[e] : __float2bfloat16(0.f);
          v = tmp.u;
        }
      }
      *reinterpret_cast<uint4*>(As + core_off(r, kc * 8)) = v;
    }
    // B panel: cells x K, converted from the FP64 saddle-point vector
    for (int t = tid; t < TN * TK; t += blockDim.x) {
      const int c = t % TN, kk = t / TN;
      const int gk = kp + kk, s = cells[c];
      const float v = (gk < n_R && s >= 0) ? (float)X[(size_t)rdofs[gk] * n_cells + s] : 0.f;
      Bs[core_off(c, kk)] = __float2bfloat16(v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int ks = 0; ks < TK / KSTEP; ++ks) {
        const uint64_t ad = make_desc(smem_u32(As) + ks * 2 * 128);
        const uint64_t bd = make_desc(smem_u32(Bs) + ks * 2 * 128);
        const uint32_t acc = (kp > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                   : "memory");
    }
    const bool done = mbar_wait(mb, parity);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ok = __syncthreads_and(done ? 1 : 0) != 0;   // CTA-uniform decision
    if (ok) parity ^= 1u;
  }
  if (ok) {
    // epilogue: warp w reads accumulator lanes 32w..32w+31 (tile rows), 16 columns at a time
    const int gi = i0 + warp * 32 + lane;
    const bool row_ok = gi < rows;
    const size_t orow = row_ok ? (size_t)(gi < n_R ? rdofs[gi] : pdofs[gi - n_R]) : 0;
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
          const int s = cells[cb + j];
          if (s < 0) continue;
          const double v = (double)__uint_as_float(r[j]);
          Y[orow * n_cells + s] = gi < n_R ? v / cscale[s] : v;
        }
      }
    }
  } else {
    if (tid == 0) atomicOr(err, 4);
    mbar_wait(mb, parity);  // give any MMA still in flight a bounded chance to finish
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

__global__ void k_d2bf(int64_t n, const double* __restrict__ x, __nv_bfloat16* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16((float)x[i]);
}

}  // namespace

// BF16 copy of the augmented local matrices (after the FP64 Gauss-Jordan sweep)
void run_g_to_bf16(lat_ctx* h, size_t n) {
  h->G16.ensure(n);
  LAT_LAUNCH(h, k_d2bf<<<std::min<int64_t>((int64_t)h->n_sm * 8, ((int64_t)n + 255) / 256), 256, 0, h->stream>>>(
                    (int64_t)n, h->G.p, h->G16.p));
  LAT_CHECK_LAUNCH();
}

// Y (local rows and corner rows of every cell) = [G; Phi^T] X on the tensor cores.  The tile
// list groups cells of one key in runs of 64 (seg_bn = 64 in the mixed modes).
void run_local_tc(lat_ctx* h, const double* X, double* Y) {
  const int rows = h->n_R + h->n_P;
  LAT_CUDA(cudaFuncSetAttribute(k_local_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
  dim3 grid(h->max_tiles, div_up(rows, TM));
  KernelTimer kt(h, "local_tc");
  LAT_LAUNCH(h, k_local_tc<<<grid, 128, SMEM_BYTES, h->stream>>>(h->n_cells, h->n_R, h->n_P, h->G16.p,
                                                                  h->tile_seg.p, h->tile_c0.p, h->seg_ptr.p,
                                                                  h->perm.p, h->c_cell.p, h->rdofs.p, h->pdofs.p,
                                                                  X, Y, h->flag.p));
  LAT_CHECK_LAUNCH();
}
