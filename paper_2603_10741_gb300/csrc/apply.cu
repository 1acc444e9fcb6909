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
#include <algorithm>
#include <iterator>
#include <vector>

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

// The FP32 action in 2D: four CTAs per SM (64 registers) measured 1.4x faster than the three
// that an unconstrained choice of 72 registers allows
template <typename T, int D, bool FETI>
__host__ __device__ constexpr int stage_min_blocks() {
  return D == 2 && sizeof(T) == 4 && !FETI ? 4 : 1;
}

template <typename T, int D, bool FETI>
__global__ void __launch_bounds__(256, stage_min_blocks<T, D, FETI>())
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

// FP32 form in 3D: node groups staged in shared memory.  A CTA owns one group of GR nodes of the
// cell (chosen at setup so that their neighbourhoods overlap) and 128 consecutive cells.  It
// copies, with cp.async and all copies in flight at once, the x rows of the union of the group's
// neighbour nodes for its 128 cells (3 rows of 512 B per union node) and the group's principal
// blocks (a chunk of principals at a time) into shared memory; then warp w forms node w's three
// outputs for its lane's 4 cells: per principal z = sum_b K^r_ab x_b (block values broadcast,
// x_b as one 16-byte shared load per DOF, the union position of b broadcast by shuffle), and
// y += alpha_r (x) z.  No load of the inner loop waits on L2.  PAIR uses packed FP32x2
// multiply-adds over cell pairs.  Needs n_cells % 4 == 0 (16-byte aligned rows).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Grid: x = node group, y = cell tile, so that the groups of one tile run close together and
// find its x rows in L2.  (64-cell tiles, two cells per lane, half the shared memory per CTA,
// were measured slower for every N_r on 8000 strut cells.)
template <int GR, bool PAIR, int TW>
__global__ void __launch_bounds__(GR * 32)
    k_apply_groups(int n_cells, const int* __restrict__ grp_rows, const int* __restrict__ grp_ucptr,
                   const int* __restrict__ grp_ucol, const int* __restrict__ grp_pp, const int* __restrict__ pair_u,
                   int64_t n_pairs, int n_r, int rch, const float* __restrict__ Kg, const float* __restrict__ alpha,
                   const float* __restrict__ X, float* __restrict__ Y) {
  constexpr int CPL = TW / 32;
  static_assert(CPL == 4, "four cells per lane: 16-byte rows");
  extern __shared__ __align__(16) float smf[];
  const int g = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile0 = blockIdx.y * TW;
  const int nct = min(TW, n_cells - tile0);                  // a multiple of 4
  const int u0 = grp_ucptr[g], nu = grp_ucptr[g + 1] - u0;
  const int gp0 = grp_pp[g * (GR + 1)], np = grp_pp[g * (GR + 1) + GR] - gp0;
  float* xs = smf;                                           // [nu * 3][TW]
  float* ks = smf + (size_t)nu * 3 * TW;                     // [rch][np][12]
  const bool live = lane * CPL < nct;
  for (int t = warp; t < nu * 3; t += GR) {
    const int b = grp_ucol[u0 + t / 3], j = t % 3;
    float* dst = xs + (size_t)t * TW + lane * CPL;
    const float* src = X + (size_t)(b * 3 + j) * n_cells + tile0 + lane * CPL;
    if (live) cp_async16(dst, src);
    else *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  const int a = grp_rows[g * GR + warp];
  const int q0 = grp_pp[g * (GR + 1) + warp] - gp0, nq = grp_pp[g * (GR + 1) + warp + 1] - gp0 - q0;
  const int myu = lane < nq ? pair_u[gp0 + q0 + lane] : 0;  // nq <= 27
  const int c = live ? tile0 + lane * CPL : 0;
  float2 y[3][CPL / 2];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int h = 0; h < CPL / 2; ++h) y[i][h] = make_float2(0.f, 0.f);
  for (int r0 = 0; r0 < n_r; r0 += rch) {
    const int nr = min(rch, n_r - r0);
    if (r0 > 0) __syncthreads();                             // the previous chunk is consumed
    for (int t = threadIdx.x; t < nr * np * 3; t += GR * 32) {
      const int rr = t / (np * 3), rem = t - rr * np * 3;
      cp_async16(ks + (size_t)rr * np * 12 + rem * 4, Kg + ((size_t)(r0 + rr) * n_pairs + gp0) * 12 + rem * 4);
    }
    cp_async_wait_all();
    __syncthreads();
    if (a < 0) continue;                                     // warp-uniform
    for (int rr = 0; rr < nr; ++rr) {
      float2 z[3][CPL / 2];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int h = 0; h < CPL / 2; ++h) z[i][h] = make_float2(0.f, 0.f);
      const float* kq = ks + ((size_t)rr * np + q0) * 12;
#pragma unroll 4
      for (int i = 0; i < nq; ++i) {
        const int u = __shfl_sync(0xffffffffu, myu, i);
        float2 x[3][CPL / 2];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float* xr = xs + (size_t)(u * 3 + j) * TW + lane * CPL;
          const float4 v = *reinterpret_cast<const float4*>(xr);
          x[j][0] = make_float2(v.x, v.y);
          x[j][1] = make_float2(v.z, v.w);
        }
        float k[12];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          const float4 w = *reinterpret_cast<const float4*>(kq + (size_t)i * 12 + 4 * t);
          k[4 * t] = w.x; k[4 * t + 1] = w.y; k[4 * t + 2] = w.z; k[4 * t + 3] = w.w;
        }
#pragma unroll
        for (int ii = 0; ii < 3; ++ii)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const float kv = k[ii * 3 + j];
#pragma unroll
            for (int h = 0; h < CPL / 2; ++h) {
              if (PAIR) {
                z[ii][h] = __ffma2_rn(make_float2(kv, kv), x[j][h], z[ii][h]);
              } else {
                z[ii][h].x = fmaf(kv, x[j][h].x, z[ii][h].x);
                z[ii][h].y = fmaf(kv, x[j][h].y, z[ii][h].y);
              }
            }
          }
      }
      float2 al[CPL / 2];
      {
        const float4 v = __ldg(reinterpret_cast<const float4*>(alpha + (size_t)(r0 + rr) * n_cells + c));
        al[0] = make_float2(v.x, v.y);
        al[1] = make_float2(v.z, v.w);
      }
#pragma unroll
      for (int ii = 0; ii < 3; ++ii)
#pragma unroll
        for (int h = 0; h < CPL / 2; ++h) y[ii][h] = __ffma2_rn(al[h], z[ii][h], y[ii][h]);
    }
  }
  if (a < 0 || !live) return;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float* yr = Y + (size_t)(a * 3 + i) * n_cells + c;
    *reinterpret_cast<float4*>(yr) = make_float4(y[i][0].x, y[i][0].y, y[i][1].x, y[i][1].y);
  }
}

// principal blocks [n_r][n_blk][9] -> group order [n_r][n_blk][12] (zero padded, 16-byte rows)
__global__ void k_group_blocks(int64_t n_blk, int n_r, const int* __restrict__ perm, const float* __restrict__ K,
                               float* __restrict__ Kg) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n_r * n_blk * 12) return;
  const int64_t pr = t / 12;
  const int e = (int)(t % 12);
  const int64_t r = pr / n_blk, p = pr - r * n_blk;
  Kg[t] = e < 9 ? K[(r * n_blk + perm[p]) * 9 + e] : 0.f;
}

constexpr size_t kGroupSmemBudget = 110 * 1024;   // two CTAs per SM
constexpr size_t kSmemOptin = 227 * 1024;

// shared memory of one CTA for n_r principals (rch of them staged at a time); 0 if it cannot fit
size_t group_smem(const lat_ctx::NodeGroups& G, int n_r, int* rch) {
  const size_t xb = (size_t)G.nu_max * 3 * 128 * sizeof(float), kb = (size_t)G.np_max * 12 * sizeof(float);
  if (xb + kb > kSmemOptin) return 0;
  const int64_t fit = xb + kb <= kGroupSmemBudget ? (int64_t)((kGroupSmemBudget - xb) / kb) : 1;
  *rch = (int)std::max<int64_t>(1, std::min<int64_t>(fit, n_r));
  return xb + (size_t)*rch * kb;
}

struct GroupPlan {
  const lat_ctx::NodeGroups* G = nullptr;
  int rch = 1;
  size_t shm = 0;
};

// Groups of 16 nodes read fewer union rows per output row and win when the action is one
// principal over many waves of CTAs (measured 1.3x faster on 8000 strut cells); groups of 8 keep
// more CTAs in flight and win otherwise.  False when no group size fits in shared memory (the
// per-(cell, node) kernel runs then).
bool group_plan(lat_ctx* h, GroupPlan* p) {
  if (h->ng[0].n_grp == 0) return false;
  const int64_t tiles = div_up(h->n_cells, 128);
  const bool wide = h->n_r == 1 && tiles * h->ng[1].n_grp >= 8LL * h->n_sm;
  for (int k : {wide ? 1 : 0, 0}) {
    p->G = &h->ng[k];
    p->shm = group_smem(*p->G, h->n_r, &p->rch);
    if (p->shm > 0) return true;
  }
  return false;
}

template <typename T, int D, bool FETI>
void launch(lat_ctx* h, const ApplyArgs& A, const T* Kp, const T* alpha, const T* X, T* Y) {
  GroupPlan gp;
  if (h->force_all) {
    dim3 blk(32, 8);
    dim3 grid(div_up(h->n_cells, 32), div_up(h->n_nodes_cell, 8));
    KernelTimer kt(h, sizeof(T) == 4 ? "apply_percell_fp32" : "apply_percell");
    LAT_LAUNCH(h, k_apply_percell<T, D, FETI><<<grid, blk, 0, h->stream>>>(A, Kp, X, Y));
  } else if (D == 3 && sizeof(T) == 4 && !FETI && h->n_cells % 4 == 0 &&
             ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15) == 0 && group_plan(h, &gp)) {
    // 3D FP32: node groups staged in shared memory (16-byte copies of X rows and 16-byte stores
    // of Y rows: taken only for 16-byte aligned vectors, the per-(cell, node) kernel otherwise)
    const lat_ctx::NodeGroups& G = *gp.G;
    const int rch = gp.rch;
    const size_t shm = gp.shm;
    const int64_t tiles = div_up(h->n_cells, 128);
    const int64_t nblk = h->n_blk;
    if (h->kg_version != h->sel_version || h->kg_gr != G.GR) {
      h->Kg.ensure((size_t)h->n_r * nblk * 12);
      LAT_LAUNCH(h, k_group_blocks<<<div_up((int64_t)h->n_r * nblk * 12, 256), 256, 0, h->stream>>>(
                        nblk, h->n_r, G.perm.p, h->Kp32.p, h->Kg.p));
      h->kg_version = h->sel_version;
      h->kg_gr = G.GR;
    }
    const dim3 grid(G.n_grp, (unsigned)tiles);
    const float* al = reinterpret_cast<const float*>(alpha);
    const float* xx = reinterpret_cast<const float*>(X);
    float* yy = reinterpret_cast<float*>(Y);
    KernelTimer kt(h, "apply_reduced_fp32");
    auto go = [&](auto kern, int threads) {
      LAT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
      LAT_LAUNCH(h, kern<<<grid, threads, shm, h->stream>>>(h->n_cells, G.rows.p, G.ucptr.p, G.ucol.p, G.pp.p,
                                                           G.pair_u.p, nblk, h->n_r, rch, h->Kg.p, al, xx, yy));
    };
    if (G.GR == 16) go(k_apply_groups<16, false, 128>, 16 * 32);
    else go(k_apply_groups<8, true, 128>, 8 * 32);
  } else {
    KernelTimer kt(h, sizeof(T) == 4 ? "apply_reduced_fp32" : "apply_reduced");
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

// Node groups for the 3D FP32 action: greedy in node order, each group takes a seed node and then,
// up to GR nodes, the unassigned neighbour that grows the union of the group's neighbour nodes
// least (ties: the lowest node).  Every node lies in one group, so the groups' block pairs are a
// permutation of the block pattern.
namespace {
void build_groups(lat_ctx* h, int GR, lat_ctx::NodeGroups& G) {
  const int nn = h->n_nodes_cell;
  const auto& bp = h->h_blk_ptr;
  const auto& bc = h->h_blk_col;
  auto cols_of = [&](int a) {
    std::vector<int> W(bc.begin() + bp[a], bc.begin() + bp[a + 1]);
    std::sort(W.begin(), W.end());
    return W;
  };
  std::vector<char> left(nn, 1);
  std::vector<int> rows, ucptr{0}, ucol, pp, pair_u, perm;
  G.GR = GR;
  G.nu_max = G.np_max = 0;
  for (int seed = 0; seed < nn; ++seed) {
    if (!left[seed]) continue;
    std::vector<int> grp{seed};
    left[seed] = 0;
    std::vector<int> U = cols_of(seed);
    while ((int)grp.size() < GR) {
      int best = -1;
      std::vector<int> bestU;
      for (int b : U) {
        if (!left[b]) continue;
        const std::vector<int> W = cols_of(b);
        std::vector<int> un;
        std::set_union(U.begin(), U.end(), W.begin(), W.end(), std::back_inserter(un));
        if (best < 0 || un.size() < bestU.size()) {
          best = b;
          bestU.swap(un);
        }
      }
      if (best < 0) break;
      grp.push_back(best);
      left[best] = 0;
      U.swap(bestU);
    }
    const int base = (int)perm.size();
    for (int q = 0; q < GR; ++q) {
      rows.push_back(q < (int)grp.size() ? grp[q] : -1);
      pp.push_back((int)perm.size());
      if (q >= (int)grp.size()) continue;
      for (int bi = bp[grp[q]]; bi < bp[grp[q] + 1]; ++bi) {
        pair_u.push_back((int)(std::lower_bound(U.begin(), U.end(), bc[bi]) - U.begin()));
        perm.push_back(bi);
      }
    }
    pp.push_back((int)perm.size());
    G.np_max = std::max(G.np_max, (int)perm.size() - base);
    G.nu_max = std::max(G.nu_max, (int)U.size());
    ucol.insert(ucol.end(), U.begin(), U.end());
    ucptr.push_back((int)ucol.size());
  }
  G.n_grp = (int)ucptr.size() - 1;
  G.rows.upload(rows, h->stream);
  G.ucptr.upload(ucptr, h->stream);
  G.ucol.upload(ucol, h->stream);
  G.pp.upload(pp, h->stream);
  G.pair_u.upload(pair_u, h->stream);
  G.perm.upload(perm, h->stream);
  LAT_CUDA(cudaStreamSynchronize(h->stream));   // the host vectors go out of scope
}
}  // namespace

void build_node_groups(lat_ctx* h) {
  build_groups(h, 8, h->ng[0]);
  build_groups(h, 16, h->ng[1]);
}

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
