// Explicit inverse of the FETI-DP coarse matrix through its block-tridiagonal structure (FP64).
//
// The coarse matrix S_PP = sum_s A_P^{sT} S^s A_P^s (Section 3.3.1) couples the primal DOFs of
// one cell only.  Grouping the primal DOFs by the layer of cells along the load axis (a node
// belongs to the highest, or the lowest, layer among its cells) makes it block tridiagonal:
// blocks A_i on the diagonal, B_i coupling block i to block i+1.  Its inverse X follows from the
// recurrences
//   D_0 = A_0,            D_i = A_i - B_{i-1}^T D_{i-1}^{-1} B_{i-1}       (forward)
//   E_{N-1} = A_{N-1},    E_i = A_i - B_i E_{i+1}^{-1} B_i^T                (backward)
//   X_ii = (D_i - B_i E_{i+1}^{-1} B_i^T)^{-1}
//   X_ij = U_i X_{i+1,j},  U_i = -D_i^{-1} B_i          (i < j, computed wave by wave in j - i)
//   X_ji = X_ij^T
// at a cost of about N^2 m^3 instead of the (N m)^3 of a dense inversion.  The forward and the
// backward recurrence are independent; they advance together, one step of each per batched
// launch.  Blocks are stored padded to a common size m (identity on the padding); the result is
// scattered into the dense inverse used by the mixed-precision coarse solves.
//
// The FP64 solves use the forward factors alone (block LU, no inverse formed):
//   y_0 = g_0,   y_i = g_i - U_{i-1}^T y_{i-1}        (U_i^T = B_i^T D_i^{-1}, D_i symmetric)
//   w_i = D_i^{-1} y_i                                 (all blocks at once)
//   x_{N-1} = w_{N-1},   x_i = w_i - U_i x_{i+1}
// which is 3 N m^2 multiply-adds per solve instead of N^2 m^2.  The two sweeps are sequential
// in i.  For blocks of up to 512 rows each sweep runs in one thread-block cluster (16 CTAs where
// the device allows it, else 8) that splits the m rows of every step, prefetches the next step's
// rows with cp.async and exchanges the new block vector through distributed shared memory, one
// cluster barrier per step.  Larger blocks do not stream fast enough through one cluster: there
// the whole solve is one cooperative launch over every SM (k_cb_solve_coop, a grid barrier per
// step, each CTA's rows of the next blocks brought in by bulk copies ahead of time), or on
// request one launch per step (k_cb_step, k_cb_step32).
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kMaxBatch = 64;

struct BatchPtrs {
  const double* a[kMaxBatch];
  const double* b[kMaxBatch];
  double* c[kMaxBatch];
};

// C_z = alpha op(A_z) op(B_z) + beta C_z for m x m row-major blocks (T x T tiles, FP64; T = 16,
// 32 or 64 so that small batches still spread over the SMs)
template <bool TA, bool TB, int T>
__global__ void __launch_bounds__(256) k_bgemm(int m, BatchPtrs P, double alpha, double beta) {
  constexpr int U = T / 16;
  const int z = blockIdx.z;
  const double* A = P.a[z];
  const double* B = P.b[z];
  double* C = P.c[z];
  __shared__ double As[T][33];
  __shared__ double Bs[32][T + 1];
  const int i0 = blockIdx.y * T, j0 = blockIdx.x * T;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[U][U];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < U; ++v) acc[u][v] = 0.0;
  for (int k0 = 0; k0 < m; k0 += 32) {
    __syncthreads();
    for (int t = threadIdx.x; t < T * 32; t += blockDim.x) {
      const int r = t / 32, c = t % 32;
      const int gi = i0 + r, gk = k0 + c;
      double v = 0.0;
      if (gi < m && gk < m) v = TA ? A[(size_t)gk * m + gi] : A[(size_t)gi * m + gk];
      As[r][c] = v;
    }
    for (int t = threadIdx.x; t < 32 * T; t += blockDim.x) {
      const int r = t / T, c = t % T;
      const int gk = k0 + r, gj = j0 + c;
      double v = 0.0;
      if (gk < m && gj < m) v = TB ? B[(size_t)gj * m + gk] : B[(size_t)gk * m + gj];
      Bs[r][c] = v;
    }
    __syncthreads();
    const int lim = min(32, m - k0);   // no multiply-adds on the zero padding of the last chunk
#pragma unroll 8
    for (int l = 0; l < lim; ++l) {
      double av[U], bv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) av[u] = As[ty + 16 * u][l];
#pragma unroll
      for (int v = 0; v < U; ++v) bv[v] = Bs[l][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int gi = i0 + ty + 16 * u;
    if (gi >= m) continue;
#pragma unroll
    for (int v = 0; v < U; ++v) {
      const int gj = j0 + tx + 16 * v;
      if (gj >= m) continue;
      double* dst = C + (size_t)gi * m + gj;
      *dst = alpha * acc[u][v] + (beta == 0.0 ? 0.0 : beta * *dst);
    }
  }
}

// coarse entries into the block storage [A_0..A_{N-1} | B_0..B_{N-2}]
__global__ void k_coarse_blocks(int64_t n_ent, int n_P, const int* __restrict__ ptr, const int* __restrict__ src,
                                const int* __restrict__ slot_of_cell, const double* __restrict__ cscale,
                                const double* __restrict__ S, const int64_t* __restrict__ dest,
                                double* __restrict__ AB) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n_ent) return;
  const int64_t d = dest[e];
  if (d < 0) return;
  double v = 0;
  for (int c = ptr[e]; c < ptr[e + 1]; ++c) {
    const int code = src[c];
    const int s = code / (n_P * n_P), ij = code % (n_P * n_P);
    v += cscale[s] * S[(size_t)slot_of_cell[s] * n_P * n_P + ij];
  }
  AB[d] = v;
}

// identity on the padding rows of the diagonal blocks
__global__ void k_pad_identity(int nb, int m, const int* __restrict__ perm, double* __restrict__ A) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nb * m) return;
  if (perm[t] < 0) {
    const int b = t / m, l = t % m;
    A[(size_t)b * m * m + (size_t)l * m + l] = 1.0;
  }
}

// dst_b = src_b^T for nb m x m blocks
__global__ void k_transpose_blocks(int nb, int m, const double* __restrict__ src, double* __restrict__ dst) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t mm = (int64_t)m * m;
  if (t >= nb * mm) return;
  const int64_t b = t / mm, r = (t % mm) / m, c = t % m;
  dst[b * mm + c * m + r] = src[t];
}

// dense inverse from the blocks: Inv[p][q] = X_{bp,bq}[lp][lq] (upper blocks, lower by symmetry)
__global__ void k_scatter_inverse(int nb, int m, const int* __restrict__ perm, const double* __restrict__ X,
                                  int64_t np, double* __restrict__ Inv) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t tot = (int64_t)nb * m * nb * m;
  if (t >= tot) return;
  const int64_t row = t / ((int64_t)nb * m), col = t % ((int64_t)nb * m);
  const int p = perm[row], q = perm[col];
  if (p < 0 || q < 0) return;
  const int bi = (int)(row / m), li = (int)(row % m), bj = (int)(col / m), lj = (int)(col % m);
  double v;
  if (bi <= bj) v = X[(((size_t)bi * nb + bj) * m + li) * m + lj];
  else v = X[(((size_t)bj * nb + bi) * m + lj) * m + li];
  Inv[(size_t)p * np + q] = v;
}

template <bool TA, bool TB>
void bgemm(lat_ctx* h, int m, std::vector<const double*> a, std::vector<const double*> b, std::vector<double*> c,
           double alpha, double beta) {
  for (size_t z0 = 0; z0 < a.size(); z0 += kMaxBatch) {
    BatchPtrs P{};
    const int nz = (int)std::min<size_t>(kMaxBatch, a.size() - z0);
    for (int z = 0; z < nz; ++z) {
      P.a[z] = a[z0 + z];
      P.b[z] = b[z0 + z];
      P.c[z] = c[z0 + z];
    }
    const int T = fp64_tile(m, nz, h->n_sm);
    if (T == 64)
      LAT_LAUNCH(h, (k_bgemm<TA, TB, 64><<<dim3(div_up(m, 64), div_up(m, 64), nz), 256, 0, h->stream>>>(m, P, alpha, beta)));
    else if (T == 32)
      LAT_LAUNCH(h, (k_bgemm<TA, TB, 32><<<dim3(div_up(m, 32), div_up(m, 32), nz), 256, 0, h->stream>>>(m, P, alpha, beta)));
    else
      LAT_LAUNCH(h, (k_bgemm<TA, TB, 16><<<dim3(div_up(m, 16), div_up(m, 16), nz), 256, 0, h->stream>>>(m, P, alpha, beta)));
    LAT_CHECK_LAUNCH();
  }
}

__device__ __forceinline__ void cp_async8(double* smem, const double* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One sweep of the block-LU solve in one cluster.  Step s handles block b = s (forward) or
// N-1-s (backward): v_b = rhs_b - M_s v_prev with M_s = U_{b-1}^T (forward, stored transposed as
// Ut) or U_b (backward), and v_b = rhs_b at step 0.  CTA c of the cluster owns rows
// [c R, c R + R) of every block.  Its rows' right-hand sides for all blocks are loaded once at
// the start, the next step's matrix rows are prefetched with cp.async, and each new value is
// stored straight into every peer's copy of the block vector (distributed shared memory, two
// copies alternating by step), so that a step is one cluster barrier and no remote load; the
// results stay in shared memory until the last step (a global store before the barrier would
// put its L2 round trip on every step).  The
// forward sweep reads rhs from the primal vector g through perm (0 on padding) and writes y in
// block layout; the backward sweep reads w in block layout and scatters x to the primal vector.
template <bool FWD>
__global__ void __launch_bounds__(256)
    k_coarse_sweep(int N, int m, int R, const double* __restrict__ Mblk, const double* __restrict__ rhs,
                   const int* __restrict__ perm, double* __restrict__ out, int pre) {
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank(), C = (int)cl.num_blocks();
  extern __shared__ __align__(16) double csm[];
  const int mp = (m + 1) & ~1, Rp = (R + 1) & ~1;
  double* vbuf = csm;                   // [2][mp] block vector of the previous step, by parity
  double* rs = csm + 2 * mp;            // [N][Rp] this CTA's right-hand sides
  double* os = rs + (size_t)N * Rp;     // [N][Rp] this CTA's results (written out at the end)
  double* Ms = os + (size_t)N * Rp;     // [2][R][m] prefetched rows (pre)
  const int r0 = c * R, nr = max(0, min(R, m - r0));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const size_t mm = (size_t)m * m;
  auto mat = [&](int st) { return Mblk + (size_t)(FWD ? st - 1 : N - 1 - st) * mm + (size_t)r0 * m; };
  auto put = [&](int b, int r, double v) {
    if (FWD) out[(size_t)b * m + r] = v;
    else {
      const int p = perm[(size_t)b * m + r];
      if (p >= 0) out[p] = v;
    }
  };
  auto prefetch = [&](int st) {
    const double* src = mat(st);
    double* dst = Ms + (size_t)(st & 1) * R * m;
    for (int t = threadIdx.x; t < nr * m; t += blockDim.x) cp_async8(dst + t, src + t);
    cp_async_commit();
  };
  if (pre) {
    if (N > 1) prefetch(1);
    else cp_async_commit();
  }
  for (int t = threadIdx.x; t < N * nr; t += blockDim.x) {
    const int b = t / nr, lr = t - b * nr;
    double v;
    if (FWD) {
      const int p = perm[(size_t)b * m + r0 + lr];
      v = p >= 0 ? rhs[p] : 0.0;
    } else {
      v = rhs[(size_t)b * m + r0 + lr];
    }
    rs[(size_t)b * Rp + lr] = v;
  }
  // every CTA of the cluster must be running before a peer's shared memory is written
  cl.sync();
  {
    const int b = FWD ? 0 : N - 1;
    for (int t = threadIdx.x; t < nr * C; t += blockDim.x) {
      const int lr = t / C, q = t - lr * C;
      const double v = rs[(size_t)b * Rp + lr];
      cl.map_shared_rank(vbuf, q)[r0 + lr] = v;
      if (q == 0) os[(size_t)b * Rp + lr] = v;
    }
  }
  cl.sync();
  for (int st = 1; st < N; ++st) {
    if (pre) {
      if (st + 1 < N) prefetch(st + 1);
      else cp_async_commit();
      cp_async_wait_1();
      __syncthreads();
    }
    const int b = FWD ? st : N - 1 - st;
    const double* vin = vbuf + (size_t)((st - 1) & 1) * mp;
    const size_t vout = (size_t)(st & 1) * mp;
    for (int lr = warp; lr < nr; lr += nw) {
      const double* Mrow = pre ? Ms + (size_t)(st & 1) * R * m + (size_t)lr * m : mat(st) + (size_t)lr * m;
      double a0 = 0.0, a1 = 0.0;
      int k = lane;
      for (; k + 32 < m; k += 64) {
        a0 = fma(Mrow[k], vin[k], a0);
        a1 = fma(Mrow[k + 32], vin[k + 32], a1);
      }
      if (k < m) a0 = fma(Mrow[k], vin[k], a0);
      const double v = rs[(size_t)b * Rp + lr] - warp_sum(a0 + a1);   // every lane holds the sum
      if (lane < C) cl.map_shared_rank(vbuf, lane)[vout + r0 + lr] = v;
      if (lane == 0) os[(size_t)b * Rp + lr] = v;
    }
    cl.sync();   // only shared-memory stores precede it: no global store on the step's path
  }
  if (pre) cp_async_wait_0();
  for (int t = threadIdx.x; t < N * nr; t += blockDim.x) {
    const int b = t / nr, lr = t - b * nr;
    put(b, r0 + lr, os[(size_t)b * Rp + lr]);
  }
}

// w_t = (D_b^{-1} y_b)_l for every row t = b m + l of the block layout (one warp per row)
__global__ void __launch_bounds__(256) k_coarse_dinv(int N, int m, const double* __restrict__ Dinv,
                                                     const double* __restrict__ y, double* __restrict__ w) {
  const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= (int64_t)N * m) return;
  const int64_t b = t / m, l = t - b * m;
  const double* row = Dinv + (size_t)b * m * m + (size_t)l * m;
  const double* yb = y + (size_t)b * m;
  double acc = 0.0;
  for (int k = lane; k < m; k += 32) acc = fma(row[k], yb[k], acc);
  acc = warp_sum(acc);
  if (lane == 0) w[t] = acc;
}

// Wide block steps for large blocks: one launch per step of the recurrence, a warp per row of
// the m x m block over the whole GPU (a 16-CTA cluster cannot stream an m = 1323 block of 14 MB
// fast enough: ~70 us per step measured on the 20^3 strut lattice, against a few us here).
//   k_cb_rhs:     rhs in block layout from the primal vector (0 on padding)
//   k_cb_step:    out = rs - M vin for one block (M row-major m x m)
//   k_cb_scatter: block layout -> primal vector
__global__ void k_cb_rhs(int64_t rows, const int* __restrict__ perm, const double* __restrict__ g,
                         double* __restrict__ rhs) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= rows) return;
  const int p = perm[t];
  rhs[t] = p >= 0 ? g[p] : 0.0;
}

// streaming 16-byte loads as volatile asm: issued in program order ahead of their uses, so that
// a chunk's loads are all in flight before the first multiply-add
__device__ __forceinline__ float4 ld_stream4(const float4* p) {
  float4 r;
  asm volatile("ld.global.cs.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "l"(p));
  return r;
}
__device__ __forceinline__ double2 ld_stream2(const double2* p) {
  double2 r;
  asm volatile("ld.global.cs.v2.f64 {%0, %1}, [%2];" : "=d"(r.x), "=d"(r.y) : "l"(p));
  return r;
}

__global__ void __launch_bounds__(256) k_cb_step(int m, const double* __restrict__ M, const double* __restrict__ vin,
                                                 const double* __restrict__ rs, double* __restrict__ out) {
  // m is even (padded blocks): a row is m / 2 16-byte pairs.  The block vector is staged in
  // shared memory once per CTA; every lane then issues all its row loads of a chunk (up to 12
  // in flight) before the first multiply-add, loads past the row end reading its last element
  // (in bounds) weighted by 0
  constexpr int U = 12;
  extern __shared__ __align__(16) double vsh[];
  for (int i = threadIdx.x; i < m; i += blockDim.x) vsh[i] = vin[i];
  __syncthreads();
  const int row = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  const double2* a = reinterpret_cast<const double2*>(M + (size_t)row * m);
  const double2* v = reinterpret_cast<const double2*>(vsh);
  const int h2 = m >> 1;
  double acc0 = 0.0, acc1 = 0.0;
  for (int k0 = 0; k0 < h2; k0 += 32 * U) {
    double2 p[U];
#pragma unroll
    for (int u = 0; u < U; ++u) p[u] = ld_stream2(a + min(k0 + lane + 32 * u, h2 - 1));
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + lane + 32 * u;
      const double w = k < h2 ? 1.0 : 0.0;
      const double2 x = v[min(k, h2 - 1)];
      acc0 = fma(w * p[u].x, x.x, acc0);
      acc1 = fma(w * p[u].y, x.y, acc1);
    }
  }
  const double s = warp_sum(acc0 + acc1);
  if (lane == 0) out[row] = rs[row] - s;
}

// the same with FP32 factors (mixed modes): products in FP32, vectors FP64 (staged as FP32 in
// shared memory); m a multiple of 4
__global__ void __launch_bounds__(256) k_cb_step32(int m, const float* __restrict__ M, const double* __restrict__ vin,
                                                   const double* __restrict__ rs, double* __restrict__ out) {
  constexpr int U = 12;
  extern __shared__ __align__(16) float vshf[];
  for (int i = threadIdx.x; i < m; i += blockDim.x) vshf[i] = (float)vin[i];
  __syncthreads();
  const int row = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  const float4* a = reinterpret_cast<const float4*>(M + (size_t)row * m);
  const float4* v = reinterpret_cast<const float4*>(vshf);
  const int h4 = m >> 2;
  float acc = 0.f;
  for (int k0 = 0; k0 < h4; k0 += 32 * U) {
    float4 p[U];
#pragma unroll
    for (int u = 0; u < U; ++u) p[u] = ld_stream4(a + min(k0 + lane + 32 * u, h4 - 1));
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + lane + 32 * u;
      const float w = k < h4 ? 1.f : 0.f;
      const float4 x = v[min(k, h4 - 1)];
      acc = fmaf(w, fmaf(p[u].x, x.x, fmaf(p[u].y, x.y, fmaf(p[u].z, x.z, p[u].w * x.w))), acc);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[row] = rs[row] - (double)acc;
}

// w_t = (D_b^{-1} y_b)_l with FP32 D^{-1} (one warp per row)
__global__ void __launch_bounds__(256) k_coarse_dinv32(int N, int m, const float* __restrict__ Dinv,
                                                       const double* __restrict__ y, double* __restrict__ w) {
  const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= (int64_t)N * m) return;
  const int64_t b = t / m, l = t - b * m;
  const float* row = Dinv + (size_t)b * m * m + (size_t)l * m;
  const double* yb = y + (size_t)b * m;
  float acc = 0.f;
  for (int k = lane; k < m; k += 32) acc = fmaf(row[k], (float)yb[k], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) w[t] = (double)acc;
}

__global__ void k_d2f_blocks(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

// The whole block-LU solve in one cooperative launch (one CTA per SM, every CTA resident): the
// right-hand side gather, the forward recurrence y_b = g_b - U_{b-1}^T y_{b-1}, w = D^{-1} y,
// the backward recurrence x_b = w_b - U_b x_{b+1} and the scatter, with a grid-wide barrier
// between dependent steps instead of a kernel launch.  CTA c owns rows [c m / G, (c + 1) m / G)
// of every step's m x m block; those rows are contiguous, and one bulk copy (cp.async.bulk,
// completing on an mbarrier) brings the rows of step k + 2 into a shared-memory buffer while
// steps k and k + 1 run, so a step waits only for its input vector (staged in shared memory by
// every CTA), a product from shared memory and the barrier.  w = D^{-1} y streams its N blocks
// from global memory with a warp per row over the whole GPU.  T = float for the FP32 factor
// copies of the mixed modes (FP32 products, as the per-step kernels), double otherwise; m is a
// multiple of 4 (16-byte rows).  A bulk copy that has not landed after a bounded wait sets bit 8
// of *err; the kernel still passes every grid barrier and waits once more for such a copy
// before it returns.
constexpr int kCoopThreads = 512;

template <typename T> struct CoopVec;
template <> struct CoopVec<float> {
  using V = float4;
  static constexpr int W = 4;
  __device__ static float dot(const float4& a, const float4& b, float acc) {
    acc = fmaf(a.x, b.x, acc);
    acc = fmaf(a.y, b.y, acc);
    acc = fmaf(a.z, b.z, acc);
    return fmaf(a.w, b.w, acc);
  }
  __device__ static float4 from(const double* v) {
    const double2 p = __ldcg(reinterpret_cast<const double2*>(v));
    const double2 q = __ldcg(reinterpret_cast<const double2*>(v) + 1);
    return make_float4((float)p.x, (float)p.y, (float)q.x, (float)q.y);
  }
};
template <> struct CoopVec<double> {
  using V = double2;
  static constexpr int W = 2;
  __device__ static double dot(const double2& a, const double2& b, double acc) {
    acc = fma(a.x, b.x, acc);
    return fma(a.y, b.y, acc);
  }
  __device__ static double2 from(const double* v) { return __ldcg(reinterpret_cast<const double2*>(v)); }
};

// one row of a block (shared or global memory) against a vector staged in shared memory
template <typename T>
__device__ __forceinline__ T coop_row_dot(const T* a, const T* v, int m, int lane) {
  using CV = CoopVec<T>;
  using V = typename CV::V;
  const V* a4 = reinterpret_cast<const V*>(a);
  const V* v4 = reinterpret_cast<const V*>(v);
  const int n4 = m / CV::W;
  T acc0 = 0, acc1 = 0;
  int k = lane;
  for (; k + 32 < n4; k += 64) {
    acc0 = CV::dot(a4[k], v4[k], acc0);
    acc1 = CV::dot(a4[k + 32], v4[k + 32], acc1);
  }
  if (k < n4) acc0 = CV::dot(a4[k], v4[k], acc0);
  return warp_sum(acc0 + acc1);
}

// one row of a block in global memory against a vector in global memory (FP64), with up to
// 8 vector loads of the row in flight per lane
template <typename T>
__device__ __forceinline__ T coop_row_dot_global(const T* __restrict__ a, const double* v, int m, int lane) {
  using CV = CoopVec<T>;
  using V = typename CV::V;
  constexpr int U = 8;
  const V* a4 = reinterpret_cast<const V*>(a);
  const int n4 = m / CV::W;
  T acc = 0;
  for (int k0 = 0; k0 < n4; k0 += 32 * U) {
    V r[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u * 32 + lane;
      r[u] = __ldcs(a4 + (k < n4 ? k : 0));
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u * 32 + lane;
      if (k < n4) acc = CV::dot(r[u], CV::from(v + (size_t)k * CV::W), acc);
    }
  }
  return warp_sum(acc);
}

__device__ __forceinline__ bool coop_wait(uint32_t addr, uint32_t parity) {
  for (int i = 0; i < (1 << 22); ++i) {
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

size_t coop_smem_bytes(int m, int rows_max, size_t elem) {
  return 16 + (((size_t)m * elem + 15) & ~(size_t)15) + 2 * (size_t)rows_max * m * elem;
}

template <typename T>
__global__ void __launch_bounds__(kCoopThreads, 1)
    k_cb_solve_coop(int N, int m, int rows_max, const T* __restrict__ Ut, const T* __restrict__ U,
                    const T* __restrict__ Dinv, const int* __restrict__ perm, const double* __restrict__ g,
                    double* rb, double* y, double* w, double* __restrict__ x, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char coop_smem[];
  cg::grid_group grid = cg::this_grid();
  const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(coop_smem);
  T* vs = reinterpret_cast<T*>(coop_smem + 16);
  T* buf = reinterpret_cast<T*>(coop_smem + 16 + (((size_t)m * sizeof(T) + 15) & ~(size_t)15));
  const size_t mm = (size_t)m * m, bstride = (size_t)rows_max * m;
  const int G = gridDim.x, c = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarp_cta = blockDim.x >> 5;
  const int r0 = (int)((int64_t)c * m / G), nr = (int)((int64_t)(c + 1) * m / G) - r0;
  const int n_tasks = 2 * (N - 1);
  // task k < N - 1: forward step b = k + 1 with U_k^T; task k >= N - 1: backward step
  // b = 2N - 3 - k with U_b
  auto task_rows = [&](int k) -> const T* {
    const T* M = k < N - 1 ? Ut + (size_t)k * mm : U + (size_t)(2 * N - 3 - k) * mm;
    return M + (size_t)r0 * m;
  };
  auto prefetch = [&](int k) {
    if (k >= n_tasks || nr == 0 || threadIdx.x != 0) return;
    const uint32_t bar = bar0 + 8 * (k & 1), bytes = (uint32_t)((size_t)nr * m * sizeof(T));
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(buf + (k & 1) * bstride);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(task_rows(k)), "r"(bytes), "r"(bar)
                 : "memory");
  };
  bool late[2] = {false, false};
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  prefetch(0);
  prefetch(1);
  const int64_t rows = (int64_t)N * m;
  const int64_t tid = (int64_t)c * blockDim.x + threadIdx.x, nthr = (int64_t)G * blockDim.x;
  for (int64_t t = tid; t < rows; t += nthr) {
    const int p = perm[t];
    const double val = p >= 0 ? g[p] : 0.0;
    rb[t] = val;
    if (t < m) y[t] = val;
  }
  grid.sync();
  // one recurrence step: out_r = rs_r - (M v)_r for this CTA's rows, M's rows in buffer k & 1
  auto step = [&](int k, const double* v, const double* rs, double* out) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) vs[i] = (T)__ldcg(v + i);
    __syncthreads();
    if (nr > 0 && !coop_wait(bar0 + 8 * (k & 1), (uint32_t)((k >> 1) & 1))) {
      late[k & 1] = true;
      if (threadIdx.x == 0) atomicOr(err, 8);
    }
    const T* Mb = buf + (k & 1) * bstride;
    for (int lr = warp; lr < nr; lr += nwarp_cta) {
      const T d = coop_row_dot(Mb + (size_t)lr * m, vs, m, lane);
      if (lane == 0) out[r0 + lr] = __ldcg(rs + r0 + lr) - (double)d;
    }
    __syncthreads();
    prefetch(k + 2);
    grid.sync();
  };
  for (int k = 0; k < N - 1; ++k) step(k, y + (size_t)k * m, rb + (size_t)(k + 1) * m, y + (size_t)(k + 1) * m);
  {
    const int64_t gwarp = tid >> 5, nwarp = nthr >> 5;
    for (int64_t t = gwarp; t < rows; t += nwarp) {
      const int64_t b = t / m, l = t - b * m;
      const T d = coop_row_dot_global(Dinv + (size_t)b * mm + (size_t)l * m, y + (size_t)b * m, m, lane);
      if (lane == 0) {
        w[t] = (double)d;
        if (b == N - 1) rb[t] = (double)d;   // x_{N-1} = w_{N-1}; rb holds x in block layout from here on
      }
    }
  }
  grid.sync();
  for (int k = N - 1; k < n_tasks; ++k) {
    const int b = 2 * N - 3 - k;
    step(k, rb + (size_t)(b + 1) * m, w + (size_t)b * m, rb + (size_t)b * m);
  }
  for (int64_t t = tid; t < rows; t += nthr) {
    const int p = perm[t];
    if (p >= 0) x[p] = __ldcg(rb + t);
  }
  // a copy that was late is still owed to this CTA's shared memory: give it a bounded chance
  for (int j = 0; j < 2; ++j)
    if (late[j]) coop_wait(bar0 + 8 * j, (uint32_t)(((n_tasks - 1 - ((n_tasks - 1 - j) & 1)) >> 1) & 1));
}

__global__ void k_cb_scatter(int64_t rows, const int* __restrict__ perm, const double* __restrict__ xb,
                             double* __restrict__ x) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= rows) return;
  const int p = perm[t];
  if (p >= 0) x[p] = xb[t];
}

template <bool FWD>
void launch_sweep(lat_ctx* h, const double* M, const double* rhs, double* out) {
  const int C = h->cb_cluster, R = div_up(h->cb_m, C);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = h->cb_shm;
  cfg.stream = h->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  LAT_LAUNCH(h, LAT_CUDA(cudaLaunchKernelEx(&cfg, k_coarse_sweep<FWD>, h->cb_n, h->cb_m, R, M, rhs,
                                            (const int*)h->cb_perm.p, out, h->cb_pre)));
}

}  // namespace

void run_coarse_blocked(lat_ctx* h, const double* S, int64_t np, bool dense) {
  const int N = h->cb_n, m = h->cb_m;
  const size_t mm = (size_t)m * m;
  const int N1 = std::max(1, N - 1);
  h->cb_A.ensure(std::max<size_t>(1, (size_t)(2 * N - 1) * mm));   // A blocks then B blocks
  double* A = h->cb_A.p;
  double* Bk = A + (size_t)N * mm;
  h->cb_Dinv.ensure(2 * (size_t)N * mm);   // [D_0^-1 .. D_{N-1}^-1 | E_{N-1}^-1 .. E_0^-1]
  h->cb_Einv.ensure((size_t)N1 * mm);      // B_i^T
  h->cb_U.ensure((size_t)N1 * mm);         // D_i^-1 B_i  (= -U_i)
  h->cb_T.ensure((size_t)N1 * mm);         // E_{i+1}^-1 B_i^T
  if (dense) h->cb_X.ensure((size_t)N * N * mm);
  else h->cb_X.release();
  double *DE = h->cb_Dinv.p, *Bt = h->cb_Einv.p, *U = h->cb_U.p, *T = h->cb_T.p, *X = h->cb_X.p;   // X: dense only
  const int64_t half = (int64_t)N * mm;    // stride from D_k^-1 to the k-th backward inverse
  auto blk = [&](double* base, int i) { return base + (size_t)i * mm; };
  auto erev = [&](int k) { return DE + half + (size_t)k * mm; };   // E_{N-1-k}^-1
  auto xb = [&](int i, int j) { return X + ((size_t)i * N + j) * mm; };
  auto cpy = [&](double* dst, const double* src) {
    LAT_CUDA(cudaMemcpyAsync(dst, src, mm * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  };
  LAT_CUDA(cudaMemsetAsync(A, 0, (size_t)(2 * N - 1) * mm * sizeof(double), h->stream));
  const int64_t n_ent = (int64_t)h->coarse_row.n;
  LAT_LAUNCH(h, k_coarse_blocks<<<div_up(n_ent, 256), 256, 0, h->stream>>>(n_ent, h->n_P, h->coarse_ptr.p,
      h->coarse_src.p, h->key_slot.p, h->c_cell.p, h->Sloc.p, h->cb_dest.p, A));
  LAT_LAUNCH(h, k_pad_identity<<<div_up((int64_t)N * m, 256), 256, 0, h->stream>>>(N, m, h->cb_perm.p, A));
  if (N > 1)
    LAT_LAUNCH(h, k_transpose_blocks<<<div_up((int64_t)(N - 1) * mm, 256), 256, 0, h->stream>>>(N - 1, m, Bk, Bt));
  LAT_CHECK_LAUNCH();
  (void)S;
  if (!dense) {
    // forward recurrence only: D_i^{-1} in place, U_{i-1} = D_{i-1}^{-1} B_{i-1}
    cpy(blk(DE, 0), blk(A, 0));
    gj_invert(h, DE, m, 1, (int64_t)mm, 8);
    for (int i = 1; i < N; ++i) {
      bgemm<false, false>(h, m, {blk(DE, i - 1)}, {blk(Bk, i - 1)}, {blk(U, i - 1)}, 1.0, 0.0);
      cpy(blk(DE, i), blk(A, i));
      bgemm<false, false>(h, m, {blk(Bt, i - 1)}, {blk(U, i - 1)}, {blk(DE, i)}, -1.0, 1.0);
      gj_invert(h, blk(DE, i), m, 1, (int64_t)mm, 8);
    }
    // U_i^T for the forward sweep, and the sweep buffers
    h->cb_Ut.ensure((size_t)N1 * mm);
    if (N > 1)
      LAT_LAUNCH(h, k_transpose_blocks<<<div_up((int64_t)(N - 1) * mm, 256), 256, 0, h->stream>>>(N - 1, m, U,
                                                                                                   h->cb_Ut.p));
    h->cb_y.ensure((size_t)N * m);
    h->cb_w.ensure((size_t)N * m);
    if (h->prec != LAT_FP64 && h->cb_wide) {
      // the mixed modes apply the FP64 factors as FP32 copies, like the rest of their
      // preconditioner (the factorisation stays FP64)
      h->cb_U32.ensure((size_t)N1 * mm);
      h->cb_Ut32.ensure((size_t)N1 * mm);
      h->cb_Dinv32.ensure((size_t)N * mm);
      const int g = 4 * h->n_sm;
      LAT_LAUNCH(h, k_d2f_blocks<<<g, 256, 0, h->stream>>>((int64_t)N1 * mm, U, h->cb_U32.p));
      LAT_LAUNCH(h, k_d2f_blocks<<<g, 256, 0, h->stream>>>((int64_t)N1 * mm, h->cb_Ut.p, h->cb_Ut32.p));
      LAT_LAUNCH(h, k_d2f_blocks<<<g, 256, 0, h->stream>>>((int64_t)N * mm, DE, h->cb_Dinv32.p));
    } else {
      h->cb_U32.release();
      h->cb_Ut32.release();
      h->cb_Dinv32.release();
    }
    LAT_CHECK_LAUNCH();
    return;
  }
  // step 0: D_0 = A_0 (kept in X_00 until the diagonal update), E_{N-1} = A_{N-1}
  cpy(xb(0, 0), blk(A, 0));
  cpy(blk(DE, 0), blk(A, 0));
  cpy(erev(0), blk(A, N - 1));
  gj_invert(h, DE, m, 2, half, 8);
  // step k: forward i = k and backward e = N-1-k, each pair in one batched launch
  for (int k = 1; k < N; ++k) {
    const int i = k, e = N - 1 - k;
    bgemm<false, false>(h, m, {blk(DE, i - 1), erev(k - 1)}, {blk(Bk, i - 1), blk(Bt, e)}, {blk(U, i - 1), blk(T, e)},
                        1.0, 0.0);
    cpy(xb(i, i), blk(A, i));
    cpy(erev(k), blk(A, e));
    bgemm<false, false>(h, m, {blk(Bt, i - 1), blk(Bk, e)}, {blk(U, i - 1), blk(T, e)}, {xb(i, i), erev(k)}, -1.0, 1.0);
    cpy(blk(DE, i), xb(i, i));
    gj_invert(h, blk(DE, k), m, 2, half, 8);
  }
  // X_ii <- D_i - B_i E_{i+1}^{-1} B_i^T, then the diagonal blocks of the inverse
  if (N > 1) {
    std::vector<const double*> a, b;
    std::vector<double*> c;
    for (int i = 0; i + 1 < N; ++i) {
      a.push_back(blk(Bk, i));
      b.push_back(blk(T, i));
      c.push_back(xb(i, i));
    }
    bgemm<false, false>(h, m, a, b, c, -1.0, 1.0);
  }
  gj_invert(h, X, m, N, (int64_t)(N + 1) * mm, 8);
  // upper blocks, wave by wave in d = j - i:  X_ij = U_i X_{i+1,j} = -(D_i^-1 B_i) X_{i+1,j}
  for (int d = 1; d < N; ++d) {
    std::vector<const double*> a, b;
    std::vector<double*> c;
    for (int j = d; j < N; ++j) {
      a.push_back(blk(U, j - d));
      b.push_back(xb(j - d + 1, j));
      c.push_back(xb(j - d, j));
    }
    bgemm<false, false>(h, m, a, b, c, -1.0, 0.0);
  }
  const int64_t tot = (int64_t)N * m * N * m;
  LAT_LAUNCH(h, k_scatter_inverse<<<div_up(tot, 256), 256, 0, h->stream>>>(N, m, h->cb_perm.p, X, np,
                                                                            h->CoarseInv.p));
  LAT_CHECK_LAUNCH();
}

// CTAs of the cooperative whole-solve launch: one per SM when every CTA fits with its shared
// memory (the FP64 factors' size, the larger of the two) and the device runs cooperative
// launches, else 0 (the per-step launches are used)
int coarse_coop_grid(lat_ctx* h) {
  int dev = 0, coop = 0, max_shm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
  if (cudaDeviceGetAttribute(&max_shm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  const int G = h->n_sm, m = h->cb_m;
  if (G <= 0 || m % 4 != 0) return 0;
  const int rmax = (int)div_up((int64_t)m, G);
  const size_t s64 = coop_smem_bytes(m, rmax, sizeof(double)), s32 = coop_smem_bytes(m, rmax, sizeof(float));
  if (s64 > (size_t)max_shm) return 0;
  int per_sm32 = 0, per_sm64 = 0;
  bool ok = cudaFuncSetAttribute(k_cb_solve_coop<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s32) ==
                cudaSuccess &&
            cudaFuncSetAttribute(k_cb_solve_coop<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s64) ==
                cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm32, k_cb_solve_coop<float>, kCoopThreads, s32) ==
                cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm64, k_cb_solve_coop<double>, kCoopThreads, s64) ==
                cudaSuccess;
  cudaGetLastError();   // a refused size is not an error of the library
  return ok && per_sm32 >= 1 && per_sm64 >= 1 ? G : 0;
}

// Cluster size and shared memory of the FP64 block-LU sweeps; false when the device runs no
// cluster of at least 8 CTAs with them (the dense inverse is used then).
bool coarse_block_plan(lat_ctx* h, bool fallback) {
  const int m = h->cb_m;
  for (int C : {16, 8}) {
    if (fallback && C == 16) continue;   // the forms taken when 16-CTA clusters or prefetch do not fit
    const int R = div_up(m, C);
    const int mp = (m + 1) & ~1, Rp = (R + 1) & ~1;
    const size_t base = (size_t)(2 * mp + 2 * (size_t)h->cb_n * Rp) * sizeof(double);
    size_t shm = base + 2 * (size_t)R * m * sizeof(double);
    int pre = 1;
    if (shm > 200 * 1024 || fallback) {
      shm = base;
      pre = 0;
    }
    if (shm > 200 * 1024) continue;
    bool ok = true;
    for (auto fn : {(const void*)k_coarse_sweep<true>, (const void*)k_coarse_sweep<false>}) {
      if (C > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) ok = false;
      if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) != cudaSuccess) ok = false;
    }
    if (ok) {
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(C);
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = shm;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int n = 0;
      ok = cudaOccupancyMaxActiveClusters(&n, k_coarse_sweep<true>, &cfg) == cudaSuccess && n >= 1;
    }
    cudaGetLastError();   // a refused size is not an error of the library
    if (ok) {
      h->cb_cluster = C;
      h->cb_shm = shm;
      h->cb_pre = pre;
      return true;
    }
  }
  h->cb_cluster = 0;
  return false;
}

// x_P = S_PP^{-1} g_P by the block-LU sweeps (FP64)
void run_coarse_block_solve(lat_ctx* h, const double* g, double* x) {
  const int N = h->cb_n, m = h->cb_m;
  const int64_t rows = (int64_t)N * m;
  const size_t mm = (size_t)m * m;
  if (h->cb_wide && h->cb_coop_grid > 0) {
    // one cooperative launch for the whole solve
    h->cb_r.ensure((size_t)rows);
    const bool f32 = h->cb_U32.p != nullptr;
    const int G = h->cb_coop_grid, rmax = (int)div_up((int64_t)m, G);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(kCoopThreads);
    cfg.dynamicSmemBytes = coop_smem_bytes(m, rmax, f32 ? sizeof(float) : sizeof(double));
    cfg.stream = h->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (f32)
      LAT_LAUNCH(h, LAT_CUDA(cudaLaunchKernelEx(&cfg, k_cb_solve_coop<float>, N, m, rmax, (const float*)h->cb_Ut32.p,
                                                (const float*)h->cb_U32.p, (const float*)h->cb_Dinv32.p,
                                                (const int*)h->cb_perm.p, g, h->cb_r.p, h->cb_y.p, h->cb_w.p, x,
                                                h->flag.p)));
    else
      LAT_LAUNCH(h, LAT_CUDA(cudaLaunchKernelEx(&cfg, k_cb_solve_coop<double>, N, m, rmax,
                                                (const double*)h->cb_Ut.p, (const double*)h->cb_U.p,
                                                (const double*)h->cb_Dinv.p, (const int*)h->cb_perm.p, g,
                                                h->cb_r.p, h->cb_y.p, h->cb_w.p, x, h->flag.p)));
    return;
  }
  if (h->cb_wide) {
    // y_b = g_b - U_{b-1}^T y_{b-1};  w = D^{-1} y;  x_b = w_b - U_b x_{b+1}
    h->cb_r.ensure((size_t)rows);
    double *rb = h->cb_r.p, *y = h->cb_y.p, *w = h->cb_w.p;
    const int rb_grid = (int)div_up(rows, 256), st_grid = (int)div_up((int64_t)m * 32, 256);
    const bool f32 = h->cb_U32.p != nullptr;
    auto step = [&](const double* M64, const float* M32, const double* vin, const double* rs, double* out) {
      if (f32) LAT_LAUNCH(h, k_cb_step32<<<st_grid, 256, m * sizeof(float), h->stream>>>(m, M32, vin, rs, out));
      else LAT_LAUNCH(h, k_cb_step<<<st_grid, 256, m * sizeof(double), h->stream>>>(m, M64, vin, rs, out));
    };
    LAT_LAUNCH(h, k_cb_rhs<<<rb_grid, 256, 0, h->stream>>>(rows, h->cb_perm.p, g, rb));
    LAT_CUDA(cudaMemcpyAsync(y, rb, m * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    for (int b = 1; b < N; ++b)
      step(h->cb_Ut.p + (size_t)(b - 1) * mm, h->cb_Ut32.p + (size_t)(b - 1) * mm, y + (size_t)(b - 1) * m,
           rb + (size_t)b * m, y + (size_t)b * m);
    if (f32)
      LAT_LAUNCH(h, k_coarse_dinv32<<<div_up(rows * 32, 256), 256, 0, h->stream>>>(N, m, h->cb_Dinv32.p, y, w));
    else
      LAT_LAUNCH(h, k_coarse_dinv<<<div_up(rows * 32, 256), 256, 0, h->stream>>>(N, m, h->cb_Dinv.p, y, w));
    double* xb = rb;   // the right-hand sides are consumed
    LAT_CUDA(cudaMemcpyAsync(xb + (size_t)(N - 1) * m, w + (size_t)(N - 1) * m, m * sizeof(double),
                             cudaMemcpyDeviceToDevice, h->stream));
    for (int b = N - 2; b >= 0; --b)
      step(h->cb_U.p + (size_t)b * mm, h->cb_U32.p + (size_t)b * mm, xb + (size_t)(b + 1) * m, w + (size_t)b * m,
           xb + (size_t)b * m);
    LAT_LAUNCH(h, k_cb_scatter<<<rb_grid, 256, 0, h->stream>>>(rows, h->cb_perm.p, xb, x));
    LAT_CHECK_LAUNCH();
    return;
  }
  launch_sweep<true>(h, h->cb_Ut.p, g, h->cb_y.p);
  LAT_LAUNCH(h, k_coarse_dinv<<<div_up(rows * 32, 256), 256, 0, h->stream>>>(N, m, h->cb_Dinv.p, h->cb_y.p,
                                                                             h->cb_w.p));
  LAT_CHECK_LAUNCH();
  launch_sweep<false>(h, h->cb_U.p, h->cb_w.p, x);
}
