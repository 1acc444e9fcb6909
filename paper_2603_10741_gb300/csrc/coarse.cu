// Explicit inverse of the FETI-DP coarse matrix through its block-tridiagonal structure (FP64).
//
// The coarse matrix S_PP = sum_s A_P^{sT} S^s A_P^s (Section 3.3.1) couples the primal DOFs of
// one cell only.  Grouping the primal DOFs by the layer of cells along the load axis (a node
// belongs to the highest layer among its cells) makes it block tridiagonal: blocks A_i on the
// diagonal, B_i coupling block i to block i+1.  Its inverse X follows from the recurrences
//   D_0 = A_0,            D_i = A_i - B_{i-1}^T D_{i-1}^{-1} B_{i-1}       (forward)
//   E_{N-1} = A_{N-1},    E_i = A_i - B_i E_{i+1}^{-1} B_i^T                (backward)
//   X_ii = (D_i - B_i E_{i+1}^{-1} B_i^T)^{-1}
//   X_ij = U_i X_{i+1,j},  U_i = -D_i^{-1} B_i          (i < j, computed wave by wave in j - i)
//   X_ji = X_ij^T
// at a cost of about N^2 m^3 instead of the (N m)^3 of a dense inversion.  Blocks are stored
// padded to a common size m (identity on the padding); the result is scattered into the dense
// inverse used by the coarse solves.
#include <algorithm>

#include "common.cuh"

namespace {

constexpr int kMaxBatch = 64;

struct BatchPtrs {
  const double* a[kMaxBatch];
  const double* b[kMaxBatch];
  double* c[kMaxBatch];
};

// C_z = alpha op(A_z) op(B_z) + beta C_z for m x m row-major blocks (64 x 64 tiles, FP64)
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_bgemm(int m, BatchPtrs P, double alpha, double beta) {
  const int z = blockIdx.z;
  const double* A = P.a[z];
  const double* B = P.b[z];
  double* C = P.c[z];
  __shared__ double As[64][33];
  __shared__ double Bs[32][65];
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
  for (int k0 = 0; k0 < m; k0 += 32) {
    __syncthreads();
    for (int t = threadIdx.x; t < 64 * 32; t += blockDim.x) {
      const int r = t / 32, c = t % 32;
      const int gi = i0 + r, gk = k0 + c;
      double v = 0.0;
      if (gi < m && gk < m) v = TA ? A[(size_t)gk * m + gi] : A[(size_t)gi * m + gk];
      As[r][c] = v;
    }
    for (int t = threadIdx.x; t < 32 * 64; t += blockDim.x) {
      const int r = t / 64, c = t % 64;
      const int gk = k0 + r, gj = j0 + c;
      double v = 0.0;
      if (gk < m && gj < m) v = TB ? B[(size_t)gj * m + gk] : B[(size_t)gk * m + gj];
      Bs[r][c] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int l = 0; l < 32; ++l) {
      double av[4], bv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) av[u] = As[ty + 16 * u][l];
#pragma unroll
      for (int v = 0; v < 4; ++v) bv[v] = Bs[l][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int gi = i0 + ty + 16 * u;
    if (gi >= m) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
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

__global__ void k_axpby_blocks(int64_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
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
    dim3 grid(div_up(m, 64), div_up(m, 64), nz);
    LAT_LAUNCH(h, (k_bgemm<TA, TB><<<grid, 256, 0, h->stream>>>(m, P, alpha, beta)));
    LAT_CHECK_LAUNCH();
  }
}

}  // namespace

void run_coarse_blocked(lat_ctx* h, const double* S, int64_t np) {
  const int N = h->cb_n, m = h->cb_m;
  const size_t mm = (size_t)m * m;
  h->cb_A.ensure(std::max<size_t>(1, (size_t)(2 * N - 1) * mm));   // A blocks then B blocks
  double* A = h->cb_A.p;
  double* Bk = A + (size_t)N * mm;
  h->cb_Dinv.ensure(N * mm);
  h->cb_Einv.ensure(N * mm);
  h->cb_U.ensure(std::max(1, N - 1) * mm);
  h->cb_T.ensure(mm);
  h->cb_X.ensure((size_t)N * N * mm);
  double *Dinv = h->cb_Dinv.p, *Einv = h->cb_Einv.p, *U = h->cb_U.p, *T = h->cb_T.p, *X = h->cb_X.p;
  auto blk = [&](double* base, int i) { return base + (size_t)i * mm; };
  auto xb = [&](int i, int j) { return X + ((size_t)i * N + j) * mm; };
  LAT_CUDA(cudaMemsetAsync(A, 0, (size_t)(2 * N - 1) * mm * sizeof(double), h->stream));
  const int64_t n_ent = (int64_t)h->coarse_row.n;
  LAT_LAUNCH(h, k_coarse_blocks<<<div_up(n_ent, 256), 256, 0, h->stream>>>(n_ent, h->n_P, h->coarse_ptr.p,
      h->coarse_src.p, h->key_slot.p, h->c_cell.p, h->Sloc.p, h->cb_dest.p, A));
  LAT_LAUNCH(h, k_pad_identity<<<div_up((int64_t)N * m, 256), 256, 0, h->stream>>>(N, m, h->cb_perm.p, A));
  LAT_CHECK_LAUNCH();
  (void)S;
  // forward: D_i (kept in X_ii until the backward sweep), D_i^{-1}, U_{i-1} = -D_{i-1}^{-1} B_{i-1}
  LAT_CUDA(cudaMemcpyAsync(xb(0, 0), blk(A, 0), mm * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  LAT_CUDA(cudaMemcpyAsync(blk(Dinv, 0), blk(A, 0), mm * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  gj_invert(h, blk(Dinv, 0), m, 1, (int64_t)mm, 8);
  for (int i = 1; i < N; ++i) {
    bgemm<false, false>(h, m, {blk(Dinv, i - 1)}, {blk(Bk, i - 1)}, {blk(U, i - 1)}, -1.0, 0.0);
    LAT_CUDA(cudaMemcpyAsync(xb(i, i), blk(A, i), mm * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    bgemm<true, false>(h, m, {blk(Bk, i - 1)}, {blk(U, i - 1)}, {xb(i, i)}, 1.0, 1.0);   // A_i + B^T U
    LAT_CUDA(cudaMemcpyAsync(blk(Dinv, i), xb(i, i), mm * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    gj_invert(h, blk(Dinv, i), m, 1, (int64_t)mm, 8);
  }
  // backward: E_i^{-1}; X_ii <- D_i - B_i E_{i+1}^{-1} B_i^T
  LAT_CUDA(cudaMemcpyAsync(blk(Einv, N - 1), blk(A, N - 1), mm * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  gj_invert(h, blk(Einv, N - 1), m, 1, (int64_t)mm, 8);
  for (int i = N - 2; i >= 0; --i) {
    bgemm<false, true>(h, m, {blk(Einv, i + 1)}, {blk(Bk, i)}, {T}, 1.0, 0.0);           // E^{-1} B^T
    bgemm<false, false>(h, m, {blk(Bk, i)}, {T}, {xb(i, i)}, -1.0, 1.0);                // X_ii -= B T
    if (i > 0) {
      LAT_CUDA(cudaMemcpyAsync(blk(Einv, i), blk(A, i), mm * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
      bgemm<false, false>(h, m, {blk(Bk, i)}, {T}, {blk(Einv, i)}, -1.0, 1.0);          // E_i
      gj_invert(h, blk(Einv, i), m, 1, (int64_t)mm, 8);
    }
  }
  // diagonal blocks of the inverse (batched, stride N+1 blocks)
  gj_invert(h, X, m, N, (int64_t)(N + 1) * mm, 8);
  // upper blocks, wave by wave in d = j - i
  for (int d = 1; d < N; ++d) {
    std::vector<const double*> a, b;
    std::vector<double*> c;
    for (int j = d; j < N; ++j) {
      a.push_back(blk(U, j - d));
      b.push_back(xb(j - d + 1, j));
      c.push_back(xb(j - d, j));
    }
    bgemm<false, false>(h, m, a, b, c, 1.0, 0.0);
  }
  const int64_t tot = (int64_t)N * m * N * m;
  LAT_LAUNCH(h, k_scatter_inverse<<<div_up(tot, 256), 256, 0, h->stream>>>(N, m, h->cb_perm.p, X, np,
                                                                            h->CoarseInv.p));
  LAT_CHECK_LAUNCH();
}
