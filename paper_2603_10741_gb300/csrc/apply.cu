// Reduced tangent action (Eq. romstiffnessmatrix):  Y[:, s] = sum_r alpha_r^s K^r X[:, s]
// on cell-stacked multivectors [n_loc][n_cells], and the per-cell action of the plain path
// (every cell principal, alpha = I: Y[:, s] = K^s X[:, s]).
//
// Layout and mapping.  One thread per (cell s, local node a) computes the d outputs of node a.
// A warp holds 32 consecutive cells at the same node, so the reads of X and writes of Y are
// coalesced 32-cell rows, while the principal values K^r_ab are warp-uniform (one broadcast
// load per warp, L1 resident: all principals together are a few hundred KB).  The alpha
// combination is fused: per node block (a, b) the thread forms sum_r alpha_r^s K^r_ab in
// registers and multiplies by x_b once.
//
// FETI mode (Section 3.3.1): the input is the remaining part of a saddle-point vector, the primal
// values (corners, and edge nodes after enrichment) come from the global primal vector through
// the cell's primal map; outputs at fixed local DOFs are zeroed, outputs at primal rows are kept
// for the primal assembly.
#include "common.cuh"

namespace {

struct ApplyArgs {
  int n_cells, nn, n_P;
  int64_t nnz;
  const int* blk_ptr;
  const int* blk_col;
  const int* corner_of_node;  // FETI
  const int* pidx;            // FETI [n_cells][n_P]
  const uint8_t* loc_fixed;   // FETI [n_loc][n_cells]
  const double* xP;           // FETI primal vector
};

template <typename T, int D, bool FETI>
__device__ __forceinline__ void load_xb(const ApplyArgs& A, const T* __restrict__ X, int s, int b,
                                        T (&xb)[D]) {
  if (FETI) {
    const int c = A.corner_of_node[b];
    if (c >= 0) {
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const int p = A.pidx[(size_t)s * A.n_P + c * D + j];
        xb[j] = p >= 0 ? (T)A.xP[p] : T(0);
      }
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const size_t e = (size_t)(b * D + j) * A.n_cells + s;
    T v = X[e];
    if (FETI && A.loc_fixed[e]) v = T(0);
    xb[j] = v;
  }
}

template <typename T, int D, bool FETI>
__device__ __forceinline__ void store_ya(const ApplyArgs& A, T* __restrict__ Y, int s, int a,
                                         const T (&ya)[D]) {
  const bool corner = FETI && A.corner_of_node[a] >= 0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const size_t e = (size_t)(a * D + i) * A.n_cells + s;
    T v = ya[i];
    if (FETI && !corner && A.loc_fixed[e]) v = T(0);
    Y[e] = v;
  }
}

template <typename T, int D, bool FETI>
__global__ void __launch_bounds__(256)
    k_apply_reduced(ApplyArgs A, int n_r, const T* __restrict__ Kp, const T* __restrict__ alpha,
                    const T* __restrict__ X, T* __restrict__ Y) {
  const int s = blockIdx.x * 32 + threadIdx.x;
  const int a = blockIdx.y * blockDim.y + threadIdx.y;
  if (a >= A.nn) return;
  const bool live = s < A.n_cells;
  const int sc = live ? s : A.n_cells - 1;  // keep the warp converged for uniform loads
  T y[D];
#pragma unroll
  for (int i = 0; i < D; ++i) y[i] = T(0);
  for (int bi = A.blk_ptr[a]; bi < A.blk_ptr[a + 1]; ++bi) {
    const int b = A.blk_col[bi];
    T xb[D];
    load_xb<T, D, FETI>(A, X, sc, b, xb);
    T kt[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) kt[i][j] = T(0);
    for (int r = 0; r < n_r; ++r) {
      const T al = alpha[(size_t)r * A.n_cells + sc];
      const T* kb = Kp + (size_t)r * A.nnz + (size_t)bi * D * D;
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) kt[i][j] = fma(al, __ldg(kb + i * D + j), kt[i][j]);
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) y[i] = fma(kt[i][j], xb[j], y[i]);
  }
  if (live) store_ya<T, D, FETI>(A, Y, s, a, y);
}

// plain path: each cell its own K^s, [n_cells][nnz]
template <typename T, int D, bool FETI>
__global__ void __launch_bounds__(256)
    k_apply_percell(ApplyArgs A, const T* __restrict__ Kall, const T* __restrict__ X, T* __restrict__ Y) {
  const int s = blockIdx.x * 32 + threadIdx.x;
  const int a = blockIdx.y * blockDim.y + threadIdx.y;
  if (a >= A.nn || s >= A.n_cells) return;
  const T* K = Kall + (size_t)s * A.nnz;
  T y[D];
#pragma unroll
  for (int i = 0; i < D; ++i) y[i] = T(0);
  for (int bi = A.blk_ptr[a]; bi < A.blk_ptr[a + 1]; ++bi) {
    const int b = A.blk_col[bi];
    T xb[D];
    load_xb<T, D, FETI>(A, X, s, b, xb);
    const T* kb = K + (size_t)bi * D * D;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) y[i] = fma(kb[i * D + j], xb[j], y[i]);
  }
  store_ya<T, D, FETI>(A, Y, s, a, y);
}

// Shared-memory staged form.  A CTA is 8 warps; warp w owns local node a = 8 blockIdx.y + w and
// its lanes own CPT x 32 consecutive cells (the same cells for all 8 warps).  Per chunk of RCH
// principals the CTA stages the alpha values of its cells once, and each warp its node's
// principal blocks K^r_{a,:} into its own slice of shared memory; the warp keeps the neighbour
// values x_b of its cells in registers and for every principal forms z = K^r_{a,:} x
// (broadcast shared loads, CPT cells per load) before the alpha-weighted accumulation
// y += alpha_r^s z: the alpha combination is the epilogue of each principal's SpMV.
template <int D>
struct StageCfg {
  static constexpr int MAXNB = D == 2 ? 9 : 27;  // node blocks per row of a Q1 pattern
  static constexpr int CPT = D == 2 ? 2 : 1;     // cells per thread
};

template <typename T, int D>
__host__ __device__ constexpr int stage_rch() {
  return D == 2 ? (sizeof(T) == 4 ? 32 : 16) : (sizeof(T) == 4 ? 8 : 4);
}

template <typename T, int D, bool FETI>
__global__ void __launch_bounds__(256)
    k_apply_staged(ApplyArgs A, int n_r, const T* __restrict__ Kp, const T* __restrict__ alpha,
                   const T* __restrict__ X, T* __restrict__ Y) {
  constexpr int MAXNB = StageCfg<D>::MAXNB, CPT = StageCfg<D>::CPT, RCH = stage_rch<T, D>();
  constexpr int DD = D * D;
  constexpr int NC = 32 * CPT;                   // cells of the CTA (the same for its 8 warps)
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int a = blockIdx.y * 8 + warp;
  const bool active = a < A.nn;                  // idle warps still join the CTA barriers
  T* als = reinterpret_cast<T*>(sm_raw);                                  // alpha chunk [RCH][NC]
  T* ks = als + RCH * NC + (size_t)warp * MAXNB * RCH * DD;              // this warp's K blocks
  const int b0 = active ? A.blk_ptr[a] : 0;
  const int nb = active ? A.blk_ptr[a + 1] - b0 : 0;
  int cell[CPT];
  bool live[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int c = blockIdx.x * NC + k * 32 + lane;
    live[k] = active && c < A.n_cells;
    cell[k] = c < A.n_cells ? c : A.n_cells - 1;
  }
  T xb[MAXNB][D][CPT];
#pragma unroll
  for (int bi = 0; bi < MAXNB; ++bi) {
    if (bi < nb) {
      const int b = A.blk_col[b0 + bi];
#pragma unroll
      for (int k = 0; k < CPT; ++k) {
        T v[D];
        load_xb<T, D, FETI>(A, X, cell[k], b, v);
#pragma unroll
        for (int j = 0; j < D; ++j) xb[bi][j][k] = v[j];
      }
    } else {
#pragma unroll
      for (int j = 0; j < D; ++j)
#pragma unroll
        for (int k = 0; k < CPT; ++k) xb[bi][j][k] = T(0);
    }
  }
  T y[D][CPT];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int k = 0; k < CPT; ++k) y[i][k] = T(0);
  for (int r0 = 0; r0 < n_r; r0 += RCH) {
    const int nr = min(RCH, n_r - r0);
    __syncthreads();
    // the CTA's alpha values for this chunk of principals (one coalesced pass, no load latency
    // inside the principal loop), then this warp's principal blocks of node a
    for (int t = threadIdx.x; t < nr * NC; t += blockDim.x) {
      const int r = t / NC, c = t - r * NC;
      const int cc = blockIdx.x * NC + c;
      als[r * NC + c] = cc < A.n_cells ? alpha[(size_t)(r0 + r) * A.n_cells + cc] : T(0);
    }
    for (int t = lane; t < nb * nr * DD; t += 32) {   // one flat pass: loads in flight together
      const int bi = t / (nr * DD), rem = t - bi * nr * DD;
      const int r = rem / DD, e = rem - r * DD;
      ks[(bi * RCH + r) * DD + e] = Kp[(size_t)(r0 + r) * A.nnz + (size_t)(b0 + bi) * DD + e];
    }
    __syncthreads();
    if (!active) continue;
    for (int r = 0; r < nr; ++r) {
      T al[CPT];
#pragma unroll
      for (int k = 0; k < CPT; ++k) al[k] = als[r * NC + k * 32 + lane];
      T z[D][CPT];
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int k = 0; k < CPT; ++k) z[i][k] = T(0);
#pragma unroll
      for (int bi = 0; bi < MAXNB; ++bi) {
        if (bi < nb) {
          const T* kb = ks + (bi * RCH + r) * DD;
          T kv[DD];
#pragma unroll
          for (int e = 0; e < DD; ++e) kv[e] = kb[e];
#pragma unroll
          for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j)
#pragma unroll
              for (int k = 0; k < CPT; ++k) z[i][k] = fma(kv[i * D + j], xb[bi][j][k], z[i][k]);
        }
      }
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int k = 0; k < CPT; ++k) y[i][k] = fma(al[k], z[i][k], y[i][k]);
    }
  }
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    if (!live[k]) continue;
    T v[D];
#pragma unroll
    for (int i = 0; i < D; ++i) v[i] = y[i][k];
    store_ya<T, D, FETI>(A, Y, cell[k], a, v);
  }
}

// FP32 form with 16-byte accesses (used in 3D): a warp owns local node a, each lane 4 consecutive
// cells.
// Per principal r: z = sum_b K^r_ab x_b over the node's neighbour blocks (block values
// warp-uniform, loaded as float4 from blocks padded to a multiple of 4 values; x_b as float4 over
// the lane's 4 cells, L1 resident after the first principal), then y += alpha_r (x) z.  About 85 %
// of the issued instructions are multiply-adds.  Needs n_cells % 4 == 0 (16-byte aligned rows).
template <int D>
__global__ void __launch_bounds__(256)
    k_apply_v4(int n_cells, int nn, const int* __restrict__ blk_ptr, const int* __restrict__ blk_col, int64_t nblk,
               int n_r, const float* __restrict__ Kb, const float* __restrict__ alpha, const float* __restrict__ X,
               float* __restrict__ Y) {
  constexpr int DDP = D == 2 ? 4 : 12;   // padded block length
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int a = blockIdx.y * 8 + warp;
  const int c0 = (blockIdx.x * 32 + lane) * 4;
  if (a >= nn || c0 >= n_cells) return;
  const int b0 = blk_ptr[a], b1 = blk_ptr[a + 1];
  float4 y[D];
#pragma unroll
  for (int i = 0; i < D; ++i) y[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int r = 0; r < n_r; ++r) {
    float4 z[D];
#pragma unroll
    for (int i = 0; i < D; ++i) z[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    const float* kr = Kb + (size_t)r * nblk * DDP;
    for (int bi = b0; bi < b1; ++bi) {
      const int b = blk_col[bi];
      float4 x[D];
#pragma unroll
      for (int j = 0; j < D; ++j) x[j] = __ldg(reinterpret_cast<const float4*>(X + (size_t)(b * D + j) * n_cells + c0));
      float k[DDP];
#pragma unroll
      for (int q = 0; q < DDP / 4; ++q) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(kr + (size_t)bi * DDP) + q);
        k[4 * q] = v.x;
        k[4 * q + 1] = v.y;
        k[4 * q + 2] = v.z;
        k[4 * q + 3] = v.w;
      }
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
          const float kv = k[i * D + j];
          z[i].x = fmaf(kv, x[j].x, z[i].x);
          z[i].y = fmaf(kv, x[j].y, z[i].y);
          z[i].z = fmaf(kv, x[j].z, z[i].z);
          z[i].w = fmaf(kv, x[j].w, z[i].w);
        }
    }
    const float4 al = __ldg(reinterpret_cast<const float4*>(alpha + (size_t)r * n_cells + c0));
#pragma unroll
    for (int i = 0; i < D; ++i) {
      y[i].x = fmaf(al.x, z[i].x, y[i].x);
      y[i].y = fmaf(al.y, z[i].y, y[i].y);
      y[i].z = fmaf(al.z, z[i].z, y[i].z);
      y[i].w = fmaf(al.w, z[i].w, y[i].w);
    }
  }
#pragma unroll
  for (int i = 0; i < D; ++i) *reinterpret_cast<float4*>(Y + (size_t)(a * D + i) * n_cells + c0) = y[i];
}

// principal blocks [n_r][nblk][9] -> [n_r][nblk][12] (zero padded) for 16-byte loads in 3D
__global__ void k_pad12(int64_t n_blocks, const float* __restrict__ K, float* __restrict__ Kb) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n_blocks * 12) return;
  const int64_t blk = t / 12;
  const int e = (int)(t % 12);
  Kb[t] = e < 9 ? K[blk * 9 + e] : 0.f;
}

template <typename T, int D, bool FETI>
void launch(lat_ctx* h, const ApplyArgs& A, const T* Kp, const T* alpha, const T* X, T* Y) {
  if (h->force_all) {
    dim3 blk(32, 8);
    dim3 grid(div_up(h->n_cells, 32), div_up(h->n_nodes_cell, 8));
    KernelTimer kt(h, "apply_percell");
    LAT_LAUNCH(h, k_apply_percell<T, D, FETI><<<grid, blk, 0, h->stream>>>(A, Kp, X, Y));
  } else if (D == 3 && sizeof(T) == 4 && !FETI && h->n_cells % 4 == 0) {
    // 3D FP32 (measured 2.5x faster than the per-(cell, node) form on the strut lattice; in 2D
    // the staged form is faster: its 9 neighbour blocks stay in registers across principals)
    const int64_t nblk = h->nnz / (D * D);
    const float* Kb = reinterpret_cast<const float*>(Kp);
    if (D == 3) {
      if (h->kp12_version != h->sel_version) {
        const int64_t nb = (int64_t)h->n_r * nblk;
        h->Kp12.ensure((size_t)nb * 12);
        LAT_LAUNCH(h, k_pad12<<<div_up(nb * 12, 256), 256, 0, h->stream>>>(nb, h->Kp32.p, h->Kp12.p));
        h->kp12_version = h->sel_version;
      }
      Kb = h->Kp12.p;
    }
    dim3 grid(div_up(h->n_cells, 128), div_up(h->n_nodes_cell, 8));
    KernelTimer kt(h, "apply_reduced");
    LAT_LAUNCH(h, k_apply_v4<D><<<grid, 256, 0, h->stream>>>(h->n_cells, h->n_nodes_cell, h->blk_ptr.p, h->blk_col.p,
                                                              nblk, h->n_r, Kb, reinterpret_cast<const float*>(alpha),
                                                              reinterpret_cast<const float*>(X),
                                                              reinterpret_cast<float*>(Y)));
  } else {
    KernelTimer kt(h, "apply_reduced");
    if (D == 3 && sizeof(T) == 4) {
      // FP32 in 3D: a thread per (cell, node) with the alpha-combined block formed in registers
      // needs no staging and keeps more warps in flight; the staged form's 81 neighbour values
      // per thread cost it occupancy (measured 2x slower for N_r = 4 to 64 on the strut
      // lattice; in FP64 the staged form is the faster one)
      dim3 blk(32, 8);
      dim3 grid(div_up(h->n_cells, 32), div_up(h->n_nodes_cell, 8));
      LAT_LAUNCH(h, k_apply_reduced<T, D, FETI><<<grid, blk, 0, h->stream>>>(A, h->n_r, Kp, alpha, X, Y));
    } else {
      constexpr int MAXNB = StageCfg<D>::MAXNB, CPT = StageCfg<D>::CPT, RCH = stage_rch<T, D>();
      const size_t shm = ((size_t)RCH * 32 * CPT + (size_t)8 * MAXNB * RCH * D * D) * sizeof(T);
      LAT_CUDA(cudaFuncSetAttribute(k_apply_staged<T, D, FETI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
      dim3 grid(div_up(h->n_cells, 32 * CPT), div_up(h->n_nodes_cell, 8));
      LAT_LAUNCH(h, k_apply_staged<T, D, FETI><<<grid, 256, shm, h->stream>>>(A, h->n_r, Kp, alpha, X, Y));
    }
  }
  LAT_CHECK_LAUNCH();
}

template <typename T>
void dispatch(lat_ctx* h, const ApplyArgs& A, const T* Kp, const T* alpha, const T* X, T* Y, bool feti) {
  if (h->dim == 2) {
    if (feti) launch<T, 2, true>(h, A, Kp, alpha, X, Y);
    else launch<T, 2, false>(h, A, Kp, alpha, X, Y);
  } else {
    if (feti) launch<T, 3, true>(h, A, Kp, alpha, X, Y);
    else launch<T, 3, false>(h, A, Kp, alpha, X, Y);
  }
}

}  // namespace

void run_apply(lat_ctx* h, const void* x, void* y, int dtype, const double* xP, bool feti) {
  LAT_REQUIRE(h->n_r > 0 && h->Kp.p, LAT_EINVAL, "no principal cells selected");
  ApplyArgs A{h->n_cells, h->n_nodes_cell, h->n_P, h->nnz, h->blk_ptr.p, h->blk_col.p,
              h->corner_of_node.p, h->pidx.p, h->loc_fixed.p, xP};
  if (dtype == 0) {
    dispatch<double>(h, A, h->Kp.p, h->alpha.p, (const double*)x, (double*)y, feti);
  } else {
    LAT_REQUIRE(h->Kp32.p && (h->force_all || h->alpha32.p), LAT_EINVAL,
                "FP32 action needs a handle created in a mixed precision mode");
    dispatch<float>(h, A, h->Kp32.p, h->alpha32.p, (const float*)x, (float*)y, feti);
  }
}

extern "C" lat_status apply_reduced_tangent(lat_handle h, const void* x, void* y, int32_t dtype) {
  if (!h || !x || !y || (dtype != 0 && dtype != 1)) return LAT_EINVAL;
  return guard(h, [&] { run_apply(h, x, y, dtype, nullptr, false); });
}
