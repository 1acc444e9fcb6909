// FETI-DP saddle-point operator, the block preconditioner of Eq. (ifetidp_precond) built on the
// principal cells, FGMRES, Newton-Raphson with Armijo backtracking and the adjoint gradient.
//
// Saddle-point vectors (Section 3.3.1) are [local part | primal part | multipliers]:
//   local part  [n_loc][n_cells]  remaining (interior + dual) DOFs of every cell; corner rows and
//                                 Dirichlet rows are kept at zero,
//   primal part [n_primal]        free corner DOFs, assembled globally,
//   multipliers [n_lambda]        one per pair of consecutive copies of a free dual DOF.
// The operator is A = [K~ B^T; B 0] with K~ the partially assembled reduced tangent (the cell-wise
// action of Eq. romstiffnessmatrix with the primal values gathered at the corners).
//
// Preconditioner (Eq. ifetidp_precond):
//   t = K^-rom v_u;  y = v_l - B t;  z_l = -PCG_k(B K^-rom B^T, y);  w_u = K^-rom (v_u - B^T z_l)
// K^-rom is the FETI-DP partially assembled inverse built from the principal cells: every cell s
// is tied to one principal r(s) (largest coefficient alpha_r^s) and its boundary-condition class,
// and uses that principal's exact local pieces
//   G^r = (K_RR^r)^{-1},  Phi^r = -G^r K_RP^r,  S^r = K_PP^r + K_RP^{rT} Phi^r,
// scaled by c_s = sum_r alpha_r^s (K^s ~ c_s K^{r(s)}): K_RR^{s,-1} ~ G^{r(s)} / c_s,
// Phi^s ~ Phi^{r(s)}, S^s ~ c_s S^{r(s)}.  The coarse matrix sum_s A_P^{sT} S^s A_P^s is FP64 and
// inverted explicitly.  With every cell principal this is the exact partially assembled inverse.
// The interface sub-preconditioner is k PCG iterations on B K^-rom B^T with the lumped
// preconditioner B_D K~_dd B_D^T (multiplicity scaling).
#include <algorithm>
#include <cfloat>
#include <chrono>
#include <cmath>

#include "common.cuh"

namespace {

// ---------------------------------------------------------------------------------------------
// elementwise and reduction kernels on saddle-point vectors
// ---------------------------------------------------------------------------------------------
constexpr int kRed = 512;

__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

// PCG scalars (see k_sum_part_pcg): sc[0] rz, sc[1] pq, sc[2] rz_new, sc[3] alpha, sc[4] beta,
// sc[5] frozen (once p.q <= 0 or r.z <= 0 the iteration stops updating)
// p = z + b[0] p  (p left unchanged when the iteration is frozen)
__global__ void k_xpby_s(int64_t n, const double* __restrict__ z, const double* __restrict__ b,
                         const double* __restrict__ frozen, double* __restrict__ p) {
  if (frozen[0] != 0.0) return;
  const double c = b[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + c * p[i];
}

__global__ void k_dot_part(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                           double* __restrict__ part) {
  __shared__ double red[32];
  double v = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v += a[i] * b[i];
  v = block_sum(v, red);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

__global__ void k_sum_part(int n, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double red[32];
  double v = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
  v = block_sum(v, red);
  if (threadIdx.x == 0) out[0] = v;
}

// the same sum into the PCG scalars, followed by the step length (step = 0: sc[1] = p.q,
// alpha = rz / pq) or the direction coefficient (step = 1: sc[2] = r.z, beta = rz_new / rz),
// with the breakdown guard that freezes the iteration: one launch per PCG dot and scalar
__global__ void k_sum_part_pcg(int n, const double* __restrict__ part, double* __restrict__ sc, int step) {
  __shared__ double red[32];
  double v = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
  v = block_sum(v, red);
  if (threadIdx.x == 0) {
    if (step == 0) {
      sc[1] = v;
      const bool ok = sc[5] == 0.0 && sc[1] > 0.0 && sc[0] > 0.0;
      if (!ok) sc[5] = 1.0;
      sc[3] = ok ? sc[0] / sc[1] : 0.0;
    } else {
      sc[2] = v;
      const bool ok = sc[5] == 0.0 && sc[2] > 0.0 && sc[0] > 0.0;
      if (!ok) sc[5] = 1.0;
      sc[4] = ok ? sc[2] / sc[0] : 0.0;
      sc[0] = sc[2];
    }
  }
}

// x += a[0] p and r -= a[0] q in one pass (the PCG updates of solution and residual)
__global__ void k_axpy2_s(int64_t n, const double* __restrict__ a, const double* __restrict__ p,
                          const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r) {
  const double c = a[0];
  if (c == 0.0) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += c * p[i];
    r[i] -= c * q[i];
  }
}

// partial dots of w against the first m vectors of V (stride n): part[i][block]
__global__ void k_multidot_part(int64_t n, int m, const double* __restrict__ V, const double* __restrict__ w,
                                double* __restrict__ part) {
  __shared__ double red[32];
  for (int i = 0; i < m; ++i) {
    const double* vi = V + (size_t)i * n;
    double v = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
      v += vi[k] * w[k];
    v = block_sum(v, red);
    if (threadIdx.x == 0) part[(size_t)i * gridDim.x + blockIdx.x] = v;
  }
}

__global__ void k_multidot_final(int nb, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double red[32];
  const int i = blockIdx.x;
  double v = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[(size_t)i * nb + b];
  v = block_sum(v, red);
  if (threadIdx.x == 0) out[i] = v;
}

// w -= sum_i h[i] V_i  (and accumulate into hacc when given)
__global__ void k_multi_axpy(int64_t n, int m, const double* __restrict__ V, const double* __restrict__ hcoef,
                             double sgn, double* __restrict__ w) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double v = w[k];
    for (int i = 0; i < m; ++i) v += sgn * hcoef[i] * V[(size_t)i * n + k];
    w[k] = v;
  }
}

__global__ void k_scale_dev(int64_t n, const double* __restrict__ x, const double* __restrict__ nrm2,
                            double* __restrict__ y) {
  const double s = 1.0 / sqrt(nrm2[0]);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i] * s;
}

// ---------------------------------------------------------------------------------------------
// FETI-DP index kernels
// ---------------------------------------------------------------------------------------------
// yP[p] = (accumulate ? yP[p] : 0) + sum over the copies of p of loc[entry]
__global__ void k_primal_assemble(int64_t n_primal, const int* __restrict__ pptr, const int* __restrict__ pc,
                                  const double* __restrict__ loc, double* __restrict__ yP, int accumulate,
                                  const double* __restrict__ base = nullptr) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n_primal) return;
  double v = base ? base[p] : (accumulate ? yP[p] : 0.0);   // yP = base + sum when base is given
  for (int c = pptr[p]; c < pptr[p + 1]; ++c) v += loc[pc[c]];
  yP[p] = v;
}

// zero the corner rows of a local vector (entries listed per primal dof) -- all corner rows
__global__ void k_zero_rows(int n_cells, int n_P, const int* __restrict__ pdofs, double* __restrict__ loc) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_cells) return;
  for (int j = 0; j < n_P; ++j) loc[(size_t)pdofs[j] * n_cells + s] = 0.0;
}

// lambda_l = x[p_l] - x[m_l]  (B x), or lambda += ...
__global__ void k_jump(int64_t L, const int* __restrict__ lp, const int* __restrict__ lm,
                       const double* __restrict__ x, double a, double* __restrict__ lam, int accumulate) {
  int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= L) return;
  double v = a * (x[lp[l]] - x[lm[l]]);
  lam[l] = accumulate ? lam[l] + v : v;
}

// y[dual entry] += a * (B^T lambda) (optionally scaled by 1/multiplicity)
__global__ void k_jump_t(int64_t nd, const int* __restrict__ de, const int* __restrict__ l1,
                         const int* __restrict__ l2, const double* __restrict__ scale,
                         const double* __restrict__ lam, double a, double* __restrict__ y) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nd) return;
  double v = 0;
  int c1 = l1[e], c2 = l2[e];
  if (c1) v += (c1 > 0 ? 1.0 : -1.0) * lam[abs(c1) - 1];
  if (c2) v += (c2 > 0 ? 1.0 : -1.0) * lam[abs(c2) - 1];
  if (scale) v *= scale[e];
  y[de[e]] += a * v;
}

// scaled jump  lambda_l = (x[p] * s_p - x[m] * s_m)  with per-entry scaling gathered from a
// dense scale array indexed like the local vector
__global__ void k_jump_scaled(int64_t L, const int* __restrict__ lp, const int* __restrict__ lm,
                              const double* __restrict__ x, const double* __restrict__ wloc,
                              double* __restrict__ lam) {
  int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= L) return;
  lam[l] = x[lp[l]] * wloc[lp[l]] - x[lm[l]] * wloc[lm[l]];
}

__global__ void k_fill_dual_weights(int64_t nd, const int* __restrict__ de, const double* __restrict__ sc,
                                    double* __restrict__ wloc) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < nd) wloc[de[e]] = sc[e];
}

// saddle-point vector -> global vector: corners from the primal part, other DOFs the mean of
// their copies, Dirichlet DOFs zero
__global__ void k_to_global(int64_t n_nodes, int D, int nn, int n_cells, int n_P, const int* __restrict__ cptr,
                            const int* __restrict__ cidx, const int* __restrict__ corner_of_node,
                            const int* __restrict__ pidx, const uint8_t* __restrict__ fixed,
                            const double* __restrict__ loc, const double* __restrict__ xP,
                            double* __restrict__ u) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n_nodes) return;
  const int c0 = cptr[g], c1 = cptr[g + 1];
  const int s0 = cidx[c0] / nn, a0 = cidx[c0] % nn;
  const int corner = corner_of_node[a0];
  for (int i = 0; i < D; ++i) {
    double v = 0;
    if (!fixed[g * D + i]) {
      if (corner >= 0) {
        const int p = pidx[(size_t)s0 * n_P + corner * D + i];
        v = p >= 0 ? xP[p] : 0.0;
      } else {
        for (int c = c0; c < c1; ++c) {
          const int s = cidx[c] / nn, a = cidx[c] % nn;
          v += loc[(size_t)(a * D + i) * n_cells + s];
        }
        v /= (double)(c1 - c0);
      }
    }
    u[g * D + i] = v;
  }
}

// global vector -> saddle-point vector (split: local values divided by the multiplicity so that
// the copies sum to the global value)
__global__ void k_from_global(int64_t n_nodes, int D, int nn, int n_cells, int n_P, const int* __restrict__ cptr,
                              const int* __restrict__ cidx, const int* __restrict__ corner_of_node,
                              const int* __restrict__ pidx, const uint8_t* __restrict__ fixed,
                              const double* __restrict__ u, int split, double* __restrict__ loc,
                              double* __restrict__ xP) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n_nodes) return;
  const int c0 = cptr[g], c1 = cptr[g + 1];
  const int s0 = cidx[c0] / nn, a0 = cidx[c0] % nn;
  const int corner = corner_of_node[a0];
  for (int i = 0; i < D; ++i) {
    const bool fx = fixed[g * D + i];
    const double v = fx ? 0.0 : u[g * D + i];
    if (corner >= 0) {
      const int p = pidx[(size_t)s0 * n_P + corner * D + i];
      if (p >= 0) xP[p] = v;
      for (int c = c0; c < c1; ++c) {
        const int s = cidx[c] / nn, a = cidx[c] % nn;
        loc[(size_t)(a * D + i) * n_cells + s] = 0.0;
      }
    } else {
      const double w = split ? v / (double)(c1 - c0) : v;
      for (int c = c0; c < c1; ++c) {
        const int s = cidx[c] / nn, a = cidx[c] % nn;
        loc[(size_t)(a * D + i) * n_cells + s] = w;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// preconditioner setup kernels
// ---------------------------------------------------------------------------------------------
// per cell: the principal whose normalised snapshot is nearest (largest cosine), and the
// least-squares scale c_s of K^s ~ c_s K^{r(s)} in the snapshot inner product.  The cosines come
// from the greedy's coordinates: <t^s, t^{s_r}> / (|t^s| |t^{s_r}|) = sum_i beta_i^s beta_i^{s_r}
// (the residuals of principal snapshots vanish), so c_s = |t^s| cos / |t^{s_r}|.  Principal cells
// get themselves with c = 1.
__global__ void k_cell_keys(int n_cells, int n_r, int force_all, const double* __restrict__ beta,
                            const double* __restrict__ norms, const int* __restrict__ S,
                            const int* __restrict__ cls, int n_classes, int* __restrict__ key,
                            double* __restrict__ cscale) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_cells) return;
  int best = 0;
  double c = 1.0;
  if (force_all) {
    best = s;
  } else {
    double bv = -DBL_MAX;
    for (int r = 0; r < n_r; ++r) {
      const int sr = S[r];
      double dot = 0;
      for (int i = 0; i <= r; ++i) dot += beta[(size_t)i * n_cells + s] * beta[(size_t)i * n_cells + sr];
      if (dot > bv) {
        bv = dot;
        best = r;
      }
    }
    const double cs = norms[s] * bv / norms[S[best]];
    c = cs > 0 ? cs : 1.0;
  }
  key[s] = best * n_classes + cls[s];
  cscale[s] = c;
}

// dense local blocks of principal r for key slot k: K_RR (into G, identity on fixed remaining
// rows), K_RP and K_PP, from the pattern values, masked with the class representative
template <int D>
__global__ void k_densify(int n_keys, const int* __restrict__ key_list, int n_classes,
                          const int* __restrict__ class_rep, int n_cells, int nn, const int* __restrict__ blk_ptr,
                          const int* __restrict__ blk_col, int64_t nnz, const double* __restrict__ Kp,
                          const int* __restrict__ rpos, const int* __restrict__ corner_of_node,
                          const uint8_t* __restrict__ loc_fixed, int n_R, int n_P,
                          double* __restrict__ G, double* __restrict__ KRP, double* __restrict__ KPP) {
  const int k = blockIdx.y;
  const int key = key_list[k];
  const int r = key / n_classes, cl = key % n_classes;
  const int rep = class_rep[cl];
  const double* K = Kp + (size_t)r * nnz;
  double* g = G + (size_t)k * (n_R + n_P) * n_R;
  double* krp = KRP + (size_t)k * n_R * n_P;
  double* kpp = KPP + (size_t)k * n_P * n_P;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nn; a += gridDim.x * blockDim.x) {
    const int ca = corner_of_node[a];
    for (int bi = blk_ptr[a]; bi < blk_ptr[a + 1]; ++bi) {
      const int b = blk_col[bi];
      const int cb = corner_of_node[b];
      for (int i = 0; i < D; ++i) {
        const int ka = a * D + i;
        const bool fa = ca < 0 && loc_fixed[(size_t)ka * n_cells + rep];
        for (int j = 0; j < D; ++j) {
          const int kb = b * D + j;
          const bool fb = cb < 0 && loc_fixed[(size_t)kb * n_cells + rep];
          double v = K[(size_t)bi * D * D + i * D + j];
          if (fa || fb) v = 0.0;
          if (ca < 0 && cb < 0) {
            if (fa && ka == kb) v = 1.0;
            g[(size_t)rpos[ka] * n_R + rpos[kb]] = v;
          } else if (ca < 0 && cb >= 0) {
            krp[(size_t)rpos[ka] * n_P + cb * D + j] = v;
          } else if (ca >= 0 && cb >= 0) {
            kpp[(size_t)(ca * D + i) * n_P + cb * D + j] = v;
          }
        }
      }
    }
  }
}

// --- blocked in-place Gauss-Jordan inversion of SPD matrices (batched) -----------------------
// step with pivot block p = [k0, k0+kw):  Pi = A_pp^{-1};  A_ij -= A_ip Pi A_pj (i,j not in p);
// A_pj = Pi A_pj;  A_ip = -A_ip Pi;  A_pp = Pi.
constexpr int GJB = 32;

__global__ void k_gj_pivot(int n, int64_t bs, int k0, int kw, double* __restrict__ A, double* __restrict__ Pinv,
                           double* __restrict__ Cbuf, int* __restrict__ flag, int neg_bit) {
  __shared__ double M[GJB][GJB + 1];
  const int b = blockIdx.x;
  double* a = A + (size_t)b * bs;
  const int t = threadIdx.x;  // 1024 threads: (i, j)
  const int i = t / GJB, j = t % GJB;
  if (i < kw && j < kw) M[i][j] = a[(size_t)(k0 + i) * n + k0 + j];
  // column panel copy (old values) for the trailing update
  for (int r = t; r < n * kw; r += blockDim.x) {
    const int row = r / kw, c = r % kw;
    Cbuf[((size_t)b * n + row) * GJB + c] = a[(size_t)row * n + k0 + c];
  }
  __syncthreads();
  // one reciprocal per pivot (thread 0) and the scaled pivot row, then one multiply-add per entry:
  // FP64 runs at two multiply-adds per clock per SM, so the 32 x 32 sweep is kept to the minimum
  __shared__ double rowp[GJB];
  __shared__ double dsh;
  for (int p = 0; p < kw; ++p) {
    if (t == 0) {
      const double piv = M[p][p];
      if (!(fabs(piv) > 0.0) || !isfinite(piv)) atomicOr(flag, 1);
      else if (piv < 0.0) atomicOr(flag, neg_bit);
      dsh = piv != 0.0 ? 1.0 / piv : 0.0;
    }
    __syncthreads();
    const double d = dsh;
    if (t < kw) rowp[t] = t == p ? d : M[p][t] * d;   // new pivot row
    double mip = 0.0, mij = 0.0;
    if (i < kw && j < kw) {
      mip = M[i][p];
      mij = M[i][j];
    }
    __syncthreads();
    if (i < kw && j < kw) {
      if (i == p) M[i][j] = rowp[j];
      else if (j == p) M[i][j] = -mip * d;
      else M[i][j] = fma(-mip, rowp[j], mij);
    }
    __syncthreads();
  }
  if (i < kw && j < kw) Pinv[(size_t)b * GJB * GJB + i * GJB + j] = M[i][j];
}

// Rbuf[b][m][j] = sum_l Pinv[m][l] A[k0+l][j]  (new pivot rows); a CTA covers 8 columns and
// every thread one (m, j) entry, so that even a single matrix spreads over many SMs
__global__ void __launch_bounds__(256) k_gj_rows(int n, int64_t bs, int k0, int kw, const double* __restrict__ A,
                                                 const double* __restrict__ Pinv, double* __restrict__ Rbuf) {
  const int b = blockIdx.y;
  const double* a = A + (size_t)b * bs;
  const double* P = Pinv + (size_t)b * GJB * GJB;
  __shared__ double Ps[GJB][GJB + 1];
  __shared__ double Cs[GJB][8];
  const int j0 = blockIdx.x * 8;
  for (int t = threadIdx.x; t < GJB * GJB; t += blockDim.x) {
    const int r = t / GJB, c = t % GJB;
    Ps[r][c] = (r < kw && c < kw) ? P[t] : 0.0;
  }
  {
    const int l = threadIdx.x / 8, c = threadIdx.x % 8;
    const int gj = j0 + c;
    Cs[l][c] = (l < kw && gj < n) ? a[(size_t)(k0 + l) * n + gj] : 0.0;
  }
  __syncthreads();
  const int m = threadIdx.x / 8, c = threadIdx.x % 8;
  const int j = j0 + c;
  if (m >= kw || j >= n) return;
  double v;
  if (j >= k0 && j < k0 + kw) {
    v = Ps[m][j - k0];
  } else {
    v = 0.0;
#pragma unroll 8
    for (int l = 0; l < GJB; ++l) v = fma(Ps[m][l], Cs[l][c], v);
  }
  Rbuf[((size_t)b * GJB + m) * n + j] = v;
}

// trailing update over T x T tiles (T = 16, 32 or 64: small batches take small tiles so that
// every SM gets work); every tile reads only Cbuf / Rbuf / Pinv, so tiles are independent
template <int T>
__global__ void __launch_bounds__(256) k_gj_update(int n, int64_t bs, int k0, int kw, double* __restrict__ A,
                                                   const double* __restrict__ Pinv, const double* __restrict__ Cbuf,
                                                   const double* __restrict__ Rbuf) {
  constexpr int U = T / 16;
  const int b = blockIdx.z;
  double* a = A + (size_t)b * bs;
  const double* C = Cbuf + (size_t)b * n * GJB;
  const double* R = Rbuf + (size_t)b * GJB * n;
  const double* P = Pinv + (size_t)b * GJB * GJB;
  __shared__ double Cs[T][GJB + 1];
  __shared__ double Rs[GJB][T + 1];
  const int i0 = blockIdx.y * T, j0 = blockIdx.x * T;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  for (int t = threadIdx.x; t < T * GJB; t += blockDim.x) {
    const int r = t / GJB, c = t % GJB;
    const int gi = i0 + r;
    Cs[r][c] = (gi < n && c < kw) ? C[(size_t)gi * GJB + c] : 0.0;
  }
  for (int t = threadIdx.x; t < GJB * T; t += blockDim.x) {
    const int r = t / T, c = t % T;
    const int gj = j0 + c;
    double v = 0.0;
    if (gj < n && r < kw) v = (gj >= k0 && gj < k0 + kw) ? P[r * GJB + (gj - k0)] : R[(size_t)r * n + gj];
    Rs[r][c] = v;
  }
  __syncthreads();
  double acc[U][U];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < U; ++v) acc[u][v] = 0.0;
  for (int l = 0; l < kw; ++l) {
    double cv[U], rv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) cv[u] = Cs[ty + 16 * u][l];
#pragma unroll
    for (int v = 0; v < U; ++v) rv[v] = Rs[l][tx + 16 * v];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int v = 0; v < U; ++v) acc[u][v] = fma(cv[u], rv[v], acc[u][v]);
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int gi = i0 + ty + 16 * u;
    if (gi >= n) continue;
    const bool ip = gi >= k0 && gi < k0 + kw;
#pragma unroll
    for (int v = 0; v < U; ++v) {
      const int gj = j0 + tx + 16 * v;
      if (gj >= n) continue;
      const bool jp = gj >= k0 && gj < k0 + kw;
      double* dst = a + (size_t)gi * n + gj;
      if (ip) *dst = jp ? P[(gi - k0) * GJB + (gj - k0)] : R[(size_t)(gi - k0) * n + gj];
      else if (jp) *dst = -acc[u][v];        // -A_ip Pi   (Rs holds Pi on pivot columns)
      else *dst -= acc[u][v];                // A_ij - A_ip (Pi A_pj)
    }
  }
}

// trailing block of a partly swept matrix: snap[b][i][j] = A[split + i][split + j]
__global__ void k_gj_snapshot(int n, int64_t bs, int split, const double* __restrict__ A, double* __restrict__ snap) {
  const int b = blockIdx.y;
  const int m = n - split;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * m) return;
  const int i = (int)(t / m), j = (int)(t % m);
  snap[(size_t)b * m * m + t] = A[(size_t)b * bs + (size_t)(split + i) * n + split + j];
}

// Phi = -G K_RP [k][n_R][n_P]; Phi^T is also stored as rows n_R.. of the augmented local
// matrix [G; Phi^T] ((n_R + n_P) x n_R per key), so that one GEMM gives G x and Phi^T x
__global__ void k_phi(int n_R, int n_P, double* __restrict__ G, const double* __restrict__ KRP,
                      double* __restrict__ Phi) {
  const int k = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_R * n_P) return;
  const int i = t / n_P, j = t % n_P;
  double* gk = G + (size_t)k * (n_R + n_P) * n_R;
  const double* g = gk + (size_t)i * n_R;
  const double* b = KRP + (size_t)k * n_R * n_P;
  double v = 0;
  for (int l = 0; l < n_R; ++l) v += g[l] * b[(size_t)l * n_P + j];
  Phi[(size_t)k * n_R * n_P + t] = -v;
  gk[(size_t)(n_R + j) * n_R + i] = -v;
}

// S = K_PP + K_RP^T Phi  (in place on KPP)   [k][n_P][n_P]
__global__ void k_schur(int n_R, int n_P, const double* __restrict__ KRP, const double* __restrict__ Phi,
                        double* __restrict__ S) {
  const int k = blockIdx.x;
  for (int t = threadIdx.x; t < n_P * n_P; t += blockDim.x) {
    const int i = t / n_P, j = t % n_P;
    const double* a = KRP + (size_t)k * n_R * n_P;
    const double* b = Phi + (size_t)k * n_R * n_P;
    double v = 0;
    for (int l = 0; l < n_R; ++l) v += a[(size_t)l * n_P + i] * b[(size_t)l * n_P + j];
    S[(size_t)k * n_P * n_P + t] += v;
  }
}

// coarse matrix entries: sum over contributions c_s S^{slot(s)}[i][j]
__global__ void k_coarse(int64_t n_ent, int64_t n_primal, int n_P, const int* __restrict__ row,
                         const int* __restrict__ col, const int* __restrict__ ptr, const int* __restrict__ src,
                         const int* __restrict__ slot_of_cell, const double* __restrict__ cscale,
                         const double* __restrict__ S, double* __restrict__ C) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n_ent) return;
  double v = 0;
  for (int c = ptr[e]; c < ptr[e + 1]; ++c) {
    const int code = src[c];
    const int s = code / (n_P * n_P), ij = code % (n_P * n_P);
    v += cscale[s] * S[(size_t)slot_of_cell[s] * n_P * n_P + ij];
  }
  C[(size_t)row[e] * n_primal + col[e]] = v;
}


// saddle-point local part -> plain FP32 cell-stacked vector for the FP32 action: corner rows from
// the primal part through pidx (0 for a Dirichlet primal DOF), other rows copied, Dirichlet rows 0
// (the operand the FETI-mode action kernels form on the fly)
__global__ void k_feti_pack32(int n_cells, int D, int n_P, const int* __restrict__ corner_of_node,
                              const int* __restrict__ pidx, const uint8_t* __restrict__ fixed,
                              const double* __restrict__ v, const double* __restrict__ xP, float* __restrict__ x) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y;
  if (s >= n_cells) return;
  const int c = corner_of_node[a];
  for (int i = 0; i < D; ++i) {
    const size_t e = (size_t)(a * D + i) * n_cells + s;
    double val;
    if (c >= 0) {
      const int p = pidx[(size_t)s * n_P + c * D + i];
      val = p >= 0 ? xP[p] : 0.0;
    } else {
      val = fixed[e] ? 0.0 : v[e];
    }
    x[e] = (float)val;
  }
}

// FP32 action result -> saddle-point local part (FP64): Dirichlet rows of non-corner DOFs 0,
// corner rows kept for the primal assembly that follows
__global__ void k_feti_unpack64(int n_cells, int D, const int* __restrict__ corner_of_node,
                                const uint8_t* __restrict__ fixed, const float* __restrict__ y,
                                double* __restrict__ w) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y;
  if (s >= n_cells) return;
  const bool corner = corner_of_node[a] >= 0;
  for (int i = 0; i < D; ++i) {
    const size_t e = (size_t)(a * D + i) * n_cells + s;
    w[e] = (!corner && fixed[e]) ? 0.0 : (double)y[e];
  }
}

__global__ void k_d2f(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

// FP32 copy of a rows x cols FP64 matrix with the rows padded to ld (zeros)
__global__ void k_d2f_pad(int64_t rows, int64_t cols, int64_t ld, const double* __restrict__ x, float* __restrict__ y) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < rows * ld; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / ld, c = t % ld;
    y[t] = c < cols ? (float)x[r * cols + c] : 0.f;
  }
}

// ---------------------------------------------------------------------------------------------
// K^-rom application kernels
// ---------------------------------------------------------------------------------------------
// Local part of K^-rom and the coarse restriction in one product with the augmented matrix
// [G; Phi^T] of the cell's key:  rows i < n_R give y_R = (1/c_s) G x_R (written to the cell's
// remaining rows), rows n_R + j give (Phi^T x_R)_j (written to the cell's corner rows, unscaled).
__device__ __forceinline__ size_t out_row(int i, int n_R, const int* __restrict__ rdofs,
                                          const int* __restrict__ pdofs) {
  return (size_t)(i < n_R ? rdofs[i] : pdofs[i - n_R]);
}

// The local products below read a view of the augmented per-key matrix [G; Phi^T]: n_Kr rows of
// G followed by the n_P rows of Phi^T, n_Kc columns, row stride ldg, key stride kstride; view
// row r < n_Kr belongs to the local DOF rr[r], view column c to rc[c].  The whole matrix is the
// view from row and column 0 with n_Kr = n_Kc = n_R.  Inputs that vanish off the dual DOFs (the
// last n_R - n_I remaining DOFs) need only the columns from n_I on; inside the interface solve
// only the dual rows of the output are read as well (the trailing dual block).

// plain path / many keys: one CTA per cell, warp per row
template <typename TG>
__global__ void __launch_bounds__(256)
    k_local_gemv(int n_cells, int n_Kr, int n_Kc, int n_P, int ldg, int64_t kstride, const TG* __restrict__ G,
                 const int* __restrict__ slot, const double* __restrict__ cscale, const int* __restrict__ rr,
                 const int* __restrict__ rc, const int* __restrict__ pdofs, const double* __restrict__ X,
                 double* __restrict__ Y) {
  extern __shared__ double xs[];
  const int s = blockIdx.x;
  for (int k = threadIdx.x; k < n_Kc; k += blockDim.x) xs[k] = X[(size_t)rc[k] * n_cells + s];
  __syncthreads();
  const int rows = n_Kr + n_P;
  const TG* g = G + (size_t)slot[s] * kstride;
  const double inv = 1.0 / cscale[s];
  // the cell's rows are shared by the gridDim.y CTAs of the cell (several when cells are few)
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int wid = blockIdx.y * nw + (threadIdx.x >> 5), nwt = gridDim.y * nw;
  for (int i = wid; i < rows; i += nwt) {
    const TG* gi = g + (size_t)i * ldg;
    double v = 0;
    for (int k = lane; k < n_Kc; k += 32) v += (double)gi[k] * xs[k];
    v = warp_sum(v);
    if (lane == 0) Y[out_row(i, n_Kr, rr, pdofs) * n_cells + s] = i < n_Kr ? v * inv : v;
  }
}

// few keys: segmented GEMM over 64 rows x BN cells of one key, cells in key order (perm);
// FP32 operands accumulate in FP32 (TG = float), FP64 in FP64 (BN a multiple of 16).
template <typename TG, int BN>
__global__ void __launch_bounds__(256)
    k_local_segmm(int n_cells, int n_Kr, int n_Kc, int n_P, int ldg, int64_t kstride, int scale_mul,
                  const TG* __restrict__ G,
                  const int* __restrict__ tile_seg,
                  const int* __restrict__ tile_c0, const int* __restrict__ seg_ptr, const int* __restrict__ perm,
                  const double* __restrict__ cscale, const int* __restrict__ rr, const int* __restrict__ rc,
                  const int* __restrict__ pdofs,
                  const double* __restrict__ X, double* __restrict__ Y) {
  constexpr int NV = BN / 16;
  const int tile = blockIdx.x;
  const int k = tile_seg[tile];
  const int c0 = tile_c0[tile];
  const int c_end = seg_ptr[k + 1];
  const int rows = n_Kr + n_P;
  const int i0 = blockIdx.y * 64;
  const TG* g = G + (size_t)k * kstride;
  __shared__ TG Gs[64][33];
  __shared__ TG Xs[32][BN + 1];
  __shared__ int cells[BN];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  if (threadIdx.x < BN) {
    const int c = c0 + threadIdx.x;
    cells[threadIdx.x] = c < c_end ? perm[c] : -1;
  }
  TG acc[4][NV];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[u][v] = TG(0);
  for (int l0 = 0; l0 < n_Kc; l0 += 32) {
    __syncthreads();
    for (int t = threadIdx.x; t < 64 * 32; t += blockDim.x) {
      const int r = t / 32, c = t % 32;
      const int gi = i0 + r, gl = l0 + c;
      Gs[r][c] = (gi < rows && gl < n_Kc) ? g[(size_t)gi * ldg + gl] : TG(0);
    }
    for (int t = threadIdx.x; t < 32 * BN; t += blockDim.x) {
      const int r = t / BN, c = t % BN;
      const int gl = l0 + r, s = cells[c];
      Xs[r][c] = (gl < n_Kc && s >= 0) ? (TG)X[(size_t)rc[gl] * n_cells + s] : TG(0);
    }
    __syncthreads();
    const int lim = min(32, n_Kc - l0);   // no multiply-adds on the padding of the last chunk
#pragma unroll 8
    for (int l = 0; l < lim; ++l) {
      TG gv[4], xv[NV];
#pragma unroll
      for (int u = 0; u < 4; ++u) gv[u] = Gs[ty + 16 * u][l];
#pragma unroll
      for (int v = 0; v < NV; ++v) xv[v] = Xs[l][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[u][v] = fma(gv[u], xv[v], acc[u][v]);
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int s = cells[tx + 16 * v];
    if (s < 0) continue;
    const double inv = scale_mul ? cscale[s] : 1.0 / cscale[s];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int gi = i0 + ty + 16 * u;
      if (gi < rows) Y[out_row(gi, n_Kr, rr, pdofs) * n_cells + s] = gi < n_Kr ? (double)acc[u][v] * inv
                                                                            : (double)acc[u][v];
    }
  }
}

// FP64 variant with 4 cells per tile: one output per thread (64 rows x 4 cells).  The FP64 pipe
// is the bound (two FP64 multiply-adds per clock per SM), so shared-memory traffic is free and a
// narrow tile only trims the multiply-adds spent on the padding of short key segments.
__global__ void __launch_bounds__(256)
    k_local_segmm_n4(int n_cells, int n_Kr, int n_Kc, int n_P, int ldg, int64_t kstride, int scale_mul,
                     const double* __restrict__ G,
                     const int* __restrict__ tile_seg,
                     const int* __restrict__ tile_c0, const int* __restrict__ seg_ptr, const int* __restrict__ perm,
                     const double* __restrict__ cscale, const int* __restrict__ rr, const int* __restrict__ rc,
                     const int* __restrict__ pdofs,
                     const double* __restrict__ X, double* __restrict__ Y) {
  constexpr int BN = 4;
  const int tile = blockIdx.x;
  const int k = tile_seg[tile];
  const int c0 = tile_c0[tile];
  const int c_end = seg_ptr[k + 1];
  const int rows = n_Kr + n_P;
  const int i0 = blockIdx.y * 64;
  const double* g = G + (size_t)k * kstride;
  __shared__ double Gs[64][33];
  __shared__ double Xs[32][BN];
  __shared__ int cells[BN];
  const int tx = threadIdx.x % BN, ty = threadIdx.x / BN;
  if (threadIdx.x < BN) {
    const int c = c0 + threadIdx.x;
    cells[threadIdx.x] = c < c_end ? perm[c] : -1;
  }
  double acc = 0.0;
  for (int l0 = 0; l0 < n_Kc; l0 += 32) {
    __syncthreads();
    for (int t = threadIdx.x; t < 64 * 32; t += blockDim.x) {
      const int r = t / 32, c = t % 32;
      const int gi = i0 + r, gl = l0 + c;
      Gs[r][c] = (gi < rows && gl < n_Kc) ? g[(size_t)gi * ldg + gl] : 0.0;
    }
    if (threadIdx.x < 32 * BN) {
      const int r = threadIdx.x / BN, c = threadIdx.x % BN;
      const int gl = l0 + r, s = cells[c];
      Xs[r][c] = (gl < n_Kc && s >= 0) ? X[(size_t)rc[gl] * n_cells + s] : 0.0;
    }
    __syncthreads();
    const int lim = min(32, n_Kc - l0);   // no multiply-adds on the padding of the last chunk
#pragma unroll 8
    for (int l = 0; l < lim; ++l) acc = fma(Gs[ty][l], Xs[l][tx], acc);
  }
  const int s = cells[tx];
  const int gi = i0 + ty;
  if (s >= 0 && gi < rows)
    Y[out_row(gi, n_Kr, rr, pdofs) * n_cells + s] =
        gi < n_Kr ? acc * (scale_mul ? cscale[s] : 1.0 / cscale[s]) : acc;
}

// Dirichlet interface preconditioner, local part: y_D = c_s S_DD^{slot(s)} x_D on the dual rows
// (S_DD = K_DD - K_DI K_II^{-1} K_ID of the cell's principal, one CTA per cell, warp per row)
template <typename TS>
__global__ void __launch_bounds__(256)
    k_dual_schur(int n_cells, int n_I, int n_D, const TS* __restrict__ SDD, const int* __restrict__ slot,
                 const double* __restrict__ cscale, const int* __restrict__ rdofs, const double* __restrict__ X,
                 double* __restrict__ Y) {
  extern __shared__ __align__(16) unsigned char xs_raw[];
  TS* xs = reinterpret_cast<TS*>(xs_raw);   // products and sums in TS: FP32 in the mixed modes
  const int s = blockIdx.x;
  for (int k = threadIdx.x; k < n_D; k += blockDim.x) xs[k] = (TS)X[(size_t)rdofs[n_I + k] * n_cells + s];
  __syncthreads();
  const TS* S = SDD + (size_t)slot[s] * n_D * n_D;
  const double c = cscale[s];
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int wid = blockIdx.y * nw + (threadIdx.x >> 5), nwt = gridDim.y * nw;
  for (int i = wid; i < n_D; i += nwt) {
    const TS* si = S + (size_t)i * n_D;
    TS v = 0;
    for (int k = lane; k < n_D; k += 32) v = fma(si[k], xs[k], v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) Y[(size_t)rdofs[n_I + i] * n_cells + s] = c * (double)v;
  }
}

// corner values of every cell from the primal vector: tP[j][s] = xP[pidx[s][j]] (0 for a
// Dirichlet primal DOF), in the precision of the product that follows
template <typename T>
__global__ void k_gather_tp(int n_cells, int n_P, const int* __restrict__ pidx, const double* __restrict__ xP,
                            T* __restrict__ tP) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n_cells * n_P) return;
  const int s = (int)(t / n_P), j = (int)(t - (int64_t)s * n_P);
  const int p = pidx[t];
  tP[(size_t)j * n_cells + s] = p >= 0 ? (T)xP[p] : T(0);
}

// Y_R^s += Phi^{slot(s)} tP[:, s] on rows [RB y, RB (y + 1)) of the view (a thread per cell: the
// cell's corner values are coalesced reads that stay in L1 across the RB rows, Phi rows are
// broadcast within a warp of cells of one key); rows n_K.. of the grid clear the corner rows
// (their values went to g_P).  T = FP32 in the mixed modes (an FP32 copy of Phi, part of their
// FP32 preconditioner).
template <typename T>
__global__ void __launch_bounds__(128)
    k_phi_rows(int n_cells, int n_K, int n_P, int RB, int64_t kstride, const T* __restrict__ Phi,
               const int* __restrict__ slot, const int* __restrict__ rdofs, const T* __restrict__ tP,
               const uint8_t* __restrict__ fixed, const int* __restrict__ pdofs, double* __restrict__ Y) {
  const int s = blockIdx.x * 128 + threadIdx.x;
  if (s >= n_cells) return;
  const T* tp = tP + s;
  const int i0 = blockIdx.y * RB, i1 = min(i0 + RB, n_K + n_P);
  const T* phs = Phi + (size_t)slot[s] * kstride;
  for (int i = i0; i < i1; ++i) {
    if (i >= n_K) {
      Y[(size_t)pdofs[i - n_K] * n_cells + s] = 0.0;
      continue;
    }
    const T* ph = phs + (size_t)i * n_P;
    T v = 0;
    for (int j = 0; j < n_P; ++j) v = fma(ph[j], tp[(size_t)j * n_cells], v);
    const size_t e = (size_t)rdofs[i] * n_cells + s;
    Y[e] = fixed[e] ? 0.0 : Y[e] + (double)v;
  }
}


// y = A x for a dense row-major matrix (warp per row)
__global__ void k_gemv(int64_t n, const double* __restrict__ A, const double* __restrict__ x, double* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  const double* a = A + (size_t)row * n;
  double v = 0;
  for (int64_t k = lane; k < n; k += 32) v += a[k] * x[k];
  v = warp_sum(v);
  if (lane == 0) y[row] = v;
}

// the same for an even n whose x fits in shared memory: x staged once per CTA (instead of once
// per row from L2), each row streamed with 16-byte loads by one warp, four loads in flight per
// lane, one row per warp so that every row starts in the first wave.  HBM bound: 8 n^2 bytes.
__global__ void __launch_bounds__(512) k_gemv_xs(int n, const double* __restrict__ A, const double* __restrict__ x,
                                                double* __restrict__ y) {
  extern __shared__ double xs[];
  for (int k = threadIdx.x; k < n; k += blockDim.x) xs[k] = x[k];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int h2 = n / 2;
  const double2* xs2 = reinterpret_cast<const double2*>(xs);
  for (int row = blockIdx.x * nw + wid; row < n; row += gridDim.x * nw) {
    const double2* a = reinterpret_cast<const double2*>(A + (size_t)row * n);
    // eight independent accumulators: the FP64 multiply-add latency is not on a chain
    double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int k = lane;
    for (; k + 96 < h2; k += 128) {   // four 16-byte loads in flight per lane
      const double2 p0 = __ldcs(a + k), p1 = __ldcs(a + k + 32), p2 = __ldcs(a + k + 64), p3 = __ldcs(a + k + 96);
      const double2 x0 = xs2[k], x1 = xs2[k + 32], x2 = xs2[k + 64], x3 = xs2[k + 96];
      v[0] = fma(p0.x, x0.x, v[0]);
      v[1] = fma(p0.y, x0.y, v[1]);
      v[2] = fma(p1.x, x1.x, v[2]);
      v[3] = fma(p1.y, x1.y, v[3]);
      v[4] = fma(p2.x, x2.x, v[4]);
      v[5] = fma(p2.y, x2.y, v[5]);
      v[6] = fma(p3.x, x3.x, v[6]);
      v[7] = fma(p3.y, x3.y, v[7]);
    }
    for (; k < h2; k += 32) {
      const double2 p = __ldcs(a + k);
      v[0] = fma(p.x, xs2[k].x, v[0]);
      v[1] = fma(p.y, xs2[k].y, v[1]);
    }
    const double s = warp_sum(((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])));
    if (lane == 0) y[row] = s;
  }
}

// FP32 copy of the coarse inverse for the mixed modes (rows padded with zeros to ld, a multiple
// of 4): FP32 products and sums, 4 n ld bytes per product
__global__ void __launch_bounds__(512) k_gemv_xs_f32(int n, int ld, const float* __restrict__ A,
                                                    const double* __restrict__ x, double* __restrict__ y) {
  extern __shared__ float xf[];
  for (int k = threadIdx.x; k < ld; k += blockDim.x) xf[k] = k < n ? (float)x[k] : 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int h4 = ld / 4;
  const float4* xs4 = reinterpret_cast<const float4*>(xf);
  for (int row = blockIdx.x * nw + wid; row < n; row += gridDim.x * nw) {
    const float4* a = reinterpret_cast<const float4*>(A + (size_t)row * ld);
    float v0 = 0.f, v1 = 0.f;
    int k = lane;
    for (; k + 32 < h4; k += 64) {
      const float4 p = __ldcs(a + k), q = __ldcs(a + k + 32);
      const float4 xp = xs4[k], xq = xs4[k + 32];
      v0 = fmaf(p.x, xp.x, fmaf(p.y, xp.y, fmaf(p.z, xp.z, fmaf(p.w, xp.w, v0))));
      v1 = fmaf(q.x, xq.x, fmaf(q.y, xq.y, fmaf(q.z, xq.z, fmaf(q.w, xq.w, v1))));
    }
    for (; k < h4; k += 32) {
      const float4 p = __ldcs(a + k);
      const float4 xp = xs4[k];
      v0 = fmaf(p.x, xp.x, fmaf(p.y, xp.y, fmaf(p.z, xp.z, fmaf(p.w, xp.w, v0))));
    }
    float v = v0 + v1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) y[row] = (double)v;
  }
}

// FGMRES small dense work on one thread: Hessenberg column j (in Hh[(m+1) x m], column major)
// after the Arnoldi step; Givens rotations in small[0..m) cs, [m..2m) sn, g in [2m..3m+1)
__global__ void k_givens(int j, int m, double* __restrict__ H, double* __restrict__ small,
                         const double* __restrict__ hcol, const double* __restrict__ nrm2, double* __restrict__ est) {
  double* cs = small;
  double* sn = small + m;
  double* g = small + 2 * m;
  double* col = H + (size_t)j * (m + 1);
  for (int i = 0; i <= j; ++i) col[i] = hcol[i];
  col[j + 1] = sqrt(nrm2[0]);
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double a = col[j], b = col[j + 1];
  const double r = hypot(a, b);
  cs[j] = r > 0 ? a / r : 1.0;
  sn[j] = r > 0 ? b / r : 0.0;
  col[j] = r;
  col[j + 1] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  est[0] = fabs(g[j + 1]);
}

__global__ void k_gmres_init(int m, double* __restrict__ small, const double* __restrict__ nrm2) {
  for (int i = 0; i < 3 * m + 1; ++i) small[i] = 0.0;
  small[2 * m] = sqrt(nrm2[0]);
}

// back substitution H y = g for the first k columns; y written to out[0..k)
__global__ void k_gmres_solve(int k, int m, const double* __restrict__ H, const double* __restrict__ small,
                              double* __restrict__ y) {
  const double* g = small + 2 * m;
  for (int i = k - 1; i >= 0; --i) {
    double v = g[i];
    for (int l = i + 1; l < k; ++l) v -= H[(size_t)l * (m + 1) + i] * y[l];
    y[i] = v / H[(size_t)i * (m + 1) + i];
  }
}

// CTAs per cell of the warp-per-row local products: one while the cells fill the GPU, more for
// small lattices (at least 64 rows per CTA) so that a handful of cells still reaches every SM
int split_rows(const lat_ctx* h, int n_cells, int rows) {
  const int want = (int)div_up(2 * h->n_sm, std::max(1, n_cells));
  return std::max(1, std::min(want, (int)div_up(rows, 64)));
}

// cells per segmented-GEMM tile: 4 in FP64, 64 in the mixed modes
int seg_bn(lat_ctx* h) { return h->prec == LAT_FP64 ? 4 : 64; }

int red_blocks(int64_t n) { return (int)std::min<int64_t>(kRed, std::max<int64_t>(1, (n + 255) / 256)); }
int ew_blocks(lat_ctx* h, int64_t n) {
  return (int)std::min<int64_t>((int64_t)h->n_sm * 8, std::max<int64_t>(1, (n + 255) / 256));
}

// device dot -> out[0] (no host sync)
void dev_dot(lat_ctx* h, int64_t n, const double* a, const double* b, double* out) {
  const int nb = red_blocks(n);
  LAT_LAUNCH(h, k_dot_part<<<nb, 256, 0, h->stream>>>(n, a, b, h->red_part.p + 1024));
  LAT_LAUNCH(h, k_sum_part<<<1, 512, 0, h->stream>>>(nb, h->red_part.p + 1024, out));
}

struct SolverTmp {
  double *a, *b, *c;
};

// ---------------------------------------------------------------------------------------------
// preconditioner setup
// ---------------------------------------------------------------------------------------------
}  // namespace

// invert `batch` n x n matrices stored with a stride of bs elements (in place).  With split in
// (0, n) the pivot blocks stop at `split` once: the trailing block [split, n)^2 then holds the
// Schur complement A_22 - A_21 A_11^{-1} A_12, copied to snap ([batch][n-split]^2) before the
// sweep continues.
void gj_invert(lat_ctx* h, double* A, int n, int batch, int64_t bs, int neg_bit, int split,
               double* snap) {
  // workspace kept in the handle: no allocation and no host synchronisation per inversion
  DBuf<double>& Pinv = h->gj_P;
  DBuf<double>& Cbuf = h->gj_C;
  DBuf<double>& Rbuf = h->gj_R;
  Pinv.ensure((size_t)batch * GJB * GJB);
  Cbuf.ensure((size_t)batch * n * GJB);
  Rbuf.ensure((size_t)batch * GJB * n);
  if (snap && split == 0) {
    LAT_LAUNCH(h, k_gj_snapshot<<<dim3(div_up((int64_t)n * n, 256), batch), 256, 0, h->stream>>>(n, bs, 0, A, snap));
    LAT_CHECK_LAUNCH();
  }
  for (int k0 = 0; k0 < n;) {
    int kw = std::min(GJB, n - k0);
    if (split > 0 && k0 < split) kw = std::min(kw, split - k0);
    {
      KernelTimer kt(h, "gj_pivot");
      LAT_LAUNCH(h, k_gj_pivot<<<batch, 1024, 0, h->stream>>>(n, bs, k0, kw, A, Pinv.p, Cbuf.p, h->flag.p, neg_bit));
      LAT_LAUNCH(h, k_gj_rows<<<dim3(div_up(n, 8), batch), 256, 0, h->stream>>>(n, bs, k0, kw, A, Pinv.p, Rbuf.p));
    }
    {
      KernelTimer kt(h, "gj_update");
      const int T = fp64_tile(n, batch, h->n_sm);
      if (T == 64)
        LAT_LAUNCH(h, k_gj_update<64><<<dim3(div_up(n, 64), div_up(n, 64), batch), 256, 0, h->stream>>>(
                          n, bs, k0, kw, A, Pinv.p, Cbuf.p, Rbuf.p));
      else if (T == 32)
        LAT_LAUNCH(h, k_gj_update<32><<<dim3(div_up(n, 32), div_up(n, 32), batch), 256, 0, h->stream>>>(
                          n, bs, k0, kw, A, Pinv.p, Cbuf.p, Rbuf.p));
      else
        LAT_LAUNCH(h, k_gj_update<16><<<dim3(div_up(n, 16), div_up(n, 16), batch), 256, 0, h->stream>>>(
                          n, bs, k0, kw, A, Pinv.p, Cbuf.p, Rbuf.p));
    }
    LAT_CHECK_LAUNCH();
    k0 += kw;
    if (snap && k0 == split && split < n) {
      const int m = n - split;
      LAT_LAUNCH(h, k_gj_snapshot<<<dim3(div_up((int64_t)m * m, 256), batch), 256, 0, h->stream>>>(n, bs, split, A, snap));
      LAT_CHECK_LAUNCH();
    }
  }
}


namespace {
}  // namespace

// principal tangents the local blocks are built from: the full K^r, or its material part
// evaluated at u_glob for the same principal cells (precond_tangent, Section 3.1.4)
bool precond_material(const lat_ctx* h, const lat_newton_opts* o) {
  const int pt = o ? o->precond_tangent : -1;
  return pt == 1 || (pt < 0 && h->dim == 3);
}

void run_prepare_solver(lat_ctx* h, const lat_newton_opts* o, const double* u_glob) {
  LAT_REQUIRE(h->n_r > 0, LAT_EINVAL, "select principal cells first");
  const double* Kpre = h->Kp.p;
  if (precond_material(h, o)) {
    LAT_REQUIRE(u_glob, LAT_EINVAL, "the material-part preconditioner needs the state");
    h->Kp_mat.ensure((size_t)h->n_r * h->nnz);
    bool neg = false;
    run_tangent(h, u_glob, 0, h->force_all ? nullptr : h->S.p, h->n_r, h->Kp_mat.p, &neg, false);
    LAT_REQUIRE(!neg, LAT_ENEG_JACOBIAN, "det F <= 0 in a principal tangent");
    Kpre = h->Kp_mat.p;
  }
  drop_pcg_graph(h);   // buffers and sizes below may change
  const int ns = h->n_cells, nR = h->n_R, nP = h->n_P;
  h->flag.ensure(4);
  h->red_part.ensure(4096);
  LAT_CUDA(cudaMemsetAsync(h->flag.p, 0, 4 * sizeof(int), h->stream));
  // keys and scales
  h->key_of_cell.ensure(ns);
  h->c_cell.ensure(ns);
  LAT_LAUNCH(h, k_cell_keys<<<div_up(ns, 256), 256, 0, h->stream>>>(ns, h->n_r, h->force_all ? 1 : 0, h->g_beta.p,
      h->g_norms.p, h->S.p, h->cell_class.p, h->n_classes, h->key_of_cell.p, h->c_cell.p));
  LAT_CHECK_LAUNCH();
  std::vector<int> keys(ns);
  LAT_CUDA(cudaMemcpyAsync(keys.data(), h->key_of_cell.p, ns * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  LAT_CUDA(cudaStreamSynchronize(h->stream));
  // segments: cells grouped by key (stable, cell order inside a key)
  std::vector<int> uniq(keys);
  std::sort(uniq.begin(), uniq.end());
  uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
  const int nk = (int)uniq.size();
  const int n_key_space = h->n_r * h->n_classes;
  std::vector<int> slot(n_key_space, -1);
  for (int k = 0; k < nk; ++k) slot[uniq[k]] = k;
  std::vector<int> cnt(nk + 1, 0), perm(ns), slot_cell(ns);
  for (int s = 0; s < ns; ++s) {
    slot_cell[s] = slot[keys[s]];
    cnt[slot_cell[s] + 1]++;
  }
  for (int k = 0; k < nk; ++k) cnt[k + 1] += cnt[k];
  std::vector<int> fill(cnt.begin(), cnt.end() - 1);
  for (int s = 0; s < ns; ++s) perm[fill[slot_cell[s]]++] = s;
  std::vector<int> tseg, tc0;
  for (int k = 0; k < nk; ++k)
    for (int c = cnt[k]; c < cnt[k + 1]; c += seg_bn(h)) {
      tseg.push_back(k);
      tc0.push_back(c);
    }
  h->n_keys = nk;
  h->key_list.upload(uniq, h->stream);
  h->perm.upload(perm, h->stream);
  h->seg_ptr.upload(cnt, h->stream);
  h->tile_seg.upload(tseg, h->stream);
  h->tile_c0.upload(tc0, h->stream);
  h->max_tiles = (int)tseg.size();
  if (h->prec == LAT_MIXED_BF16) {
    std::vector<int> tseg_tc, tc0_tc;
    for (int k = 0; k < nk; ++k)
      for (int c = cnt[k]; c < cnt[k + 1]; c += kTcCells) {
        tseg_tc.push_back(k);
        tc0_tc.push_back(c);
      }
    h->tile_seg_tc.upload(tseg_tc, h->stream);
    h->tile_c0_tc.upload(tc0_tc, h->stream);
    h->max_tiles_tc = (int)tseg_tc.size();
  }
  h->key_slot.upload(slot_cell, h->stream);  // slot of each cell
  // dense local blocks
  const int64_t gstride = (int64_t)(nR + nP) * nR;   // augmented [G; Phi^T] per key
  const size_t gsz = (size_t)nk * gstride;
  h->G.ensure(gsz);
  h->KRP.ensure((size_t)nk * nR * nP);
  h->Sloc.ensure((size_t)nk * nP * nP);
  h->Phi.ensure((size_t)nk * nR * nP);
  LAT_CUDA(cudaMemsetAsync(h->G.p, 0, gsz * sizeof(double), h->stream));
  LAT_CUDA(cudaMemsetAsync(h->KRP.p, 0, (size_t)nk * nR * nP * sizeof(double), h->stream));
  LAT_CUDA(cudaMemsetAsync(h->Sloc.p, 0, (size_t)nk * nP * nP * sizeof(double), h->stream));
  DBuf<int>& crep = h->class_rep_d;
  crep.upload(h->class_rep, h->stream);
  {
    KernelTimer kt(h, "densify");
    dim3 grid(div_up(h->n_nodes_cell, 128), nk);
    if (h->dim == 2)
      LAT_LAUNCH(h, k_densify<2><<<grid, 128, 0, h->stream>>>(nk, h->key_list.p, h->n_classes, crep.p, ns, h->n_nodes_cell,
          h->blk_ptr.p, h->blk_col.p, h->nnz, Kpre, h->rpos.p, h->corner_of_node.p, h->loc_fixed.p,
          nR, nP, h->G.p, h->KRP.p, h->Sloc.p));
    else
      LAT_LAUNCH(h, k_densify<3><<<grid, 128, 0, h->stream>>>(nk, h->key_list.p, h->n_classes, crep.p, ns, h->n_nodes_cell,
          h->blk_ptr.p, h->blk_col.p, h->nnz, Kpre, h->rpos.p, h->corner_of_node.p, h->loc_fixed.p,
          nR, nP, h->G.p, h->KRP.p, h->Sloc.p));
    LAT_CHECK_LAUNCH();
  }
  const int nD = nR - h->n_I;
  h->SDD.ensure((size_t)nk * nD * nD);
  gj_invert(h, h->G.p, nR, nk, gstride, 2, h->n_I, h->SDD.p);
  h->iface = o ? o->interface_precond : 0;
  {
    KernelTimer kt(h, "phi_schur");
    LAT_LAUNCH(h, k_phi<<<dim3(div_up(nR * nP, 128), nk), 128, 0, h->stream>>>(nR, nP, h->G.p, h->KRP.p, h->Phi.p));
    LAT_LAUNCH(h, k_schur<<<nk, 64, 0, h->stream>>>(nR, nP, h->KRP.p, h->Phi.p, h->Sloc.p));
    LAT_CHECK_LAUNCH();
  }
  // coarse matrix, FP64: block LU factors or the explicit inverse.  On the 32x32 ring lattice
  // at enrichment level 1 (32 blocks of 196) a block-LU solve takes 196 us (62 dependent block
  // steps of ~3 us, one cluster barrier each) against 110 us for the dense product, so the dense
  // inverse is kept while it is small; its N^2 m^3 build and N^2 m^2 storage decide beyond that.
  const int64_t np = h->n_primal;
  const int want = o ? o->coarse_block_lu : -1;
  h->cb_wide = want == 2 || want == 4 || (want != 3 && h->cb_m > kWideSweepRows);
  h->cb_coop_grid = h->cb_wide && want != 2 ? coarse_coop_grid(h) : 0;
  h->cb_solve = np > 0 && h->coarse_blocked &&
                (want >= 1 || (want < 0 && (int64_t)h->cb_n * h->cb_m > kDenseCoarseLimit)) &&
                (h->cb_wide || coarse_block_plan(h, want == 3));
  if (h->cb_solve) {
    h->CoarseInv.release();
    h->CoarseInv32.release();
    KernelTimer kt(h, "coarse_blocked");
    run_coarse_blocked(h, h->Sloc.p, np, false);
  } else if (np > 0) {
    h->CoarseInv.ensure((size_t)np * np);
    LAT_CUDA(cudaMemsetAsync(h->CoarseInv.p, 0, (size_t)np * np * sizeof(double), h->stream));
    if (h->coarse_blocked) {
      KernelTimer kt(h, "coarse_blocked");
      run_coarse_blocked(h, h->Sloc.p, np, true);
    } else {
      const int64_t n_ent = (int64_t)h->coarse_row.n;
      LAT_LAUNCH(h, k_coarse<<<div_up(n_ent, 256), 256, 0, h->stream>>>(n_ent, np, nP, h->coarse_row.p,
          h->coarse_col.p, h->coarse_ptr.p, h->coarse_src.p, h->key_slot.p, h->c_cell.p, h->Sloc.p, h->CoarseInv.p));
      LAT_CHECK_LAUNCH();
      gj_invert(h, h->CoarseInv.p, (int)np, 1, np * np, 8);
    }
  }
  int fl = 0;
  LAT_CUDA(cudaMemcpyAsync(&fl, h->flag.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  LAT_CUDA(cudaStreamSynchronize(h->stream));
  LAT_REQUIRE(!(fl & 1), LAT_EINDEFINITE, "a local remaining-DOF matrix or the coarse matrix is singular");
  h->indefinite = (fl & 2) != 0;          // a principal's remaining block has a negative pivot
  h->coarse_indefinite = (fl & 8) != 0;   // the coarse matrix has a negative pivot
  if (h->prec == LAT_MIXED_BF16) run_g_to_bf16(h, gsz);
  if (h->prec != LAT_FP64) {
    h->G32.ensure(gsz);
    LAT_LAUNCH(h, k_d2f<<<ew_blocks(h, gsz), 256, 0, h->stream>>>(gsz, h->G.p, h->G32.p));
    const size_t psz = (size_t)nk * nR * nP;
    h->Phi32.ensure(std::max<size_t>(1, psz));
    LAT_LAUNCH(h, k_d2f<<<ew_blocks(h, std::max<size_t>(1, psz)), 256, 0, h->stream>>>(psz, h->Phi.p, h->Phi32.p));
    const size_t dsz = (size_t)nk * nD * nD;
    h->SDD32.ensure(dsz);
    LAT_LAUNCH(h, k_d2f<<<ew_blocks(h, dsz), 256, 0, h->stream>>>(dsz, h->SDD.p, h->SDD32.p));
    if (np > 0 && !h->cb_solve) {
      const int64_t ldc = (np + 3) / 4 * 4;   // rows padded to 16 bytes for vector loads
      h->CoarseInv32.ensure((size_t)np * ldc);
      h->coarse32_ld = ldc;
      LAT_LAUNCH(h, k_d2f_pad<<<ew_blocks(h, np * ldc), 256, 0, h->stream>>>(np, np, ldc, h->CoarseInv.p,
                                                                             h->CoarseInv32.p));
    }
    LAT_CHECK_LAUNCH();
  }
  // temporaries
  for (int i = 0; i < 6; ++i) h->kv_tmp[i].ensure(h->n_krylov);
  h->pcg_ws.ensure(std::max<size_t>(1, (size_t)5 * h->n_lambda));
  h->gP.ensure(std::max<int64_t>(np, 1));
  h->xP.ensure(std::max<int64_t>(np, 1));
}

namespace {

double* loc_of(lat_ctx* h, double* v) { return v; }
double* pr_of(lat_ctx* h, double* v) { return v + (size_t)h->n_loc * h->n_cells; }
double* la_of(lat_ctx* h, double* v) { return v + (size_t)h->n_loc * h->n_cells + h->n_primal; }
const double* pr_of(lat_ctx* h, const double* v) { return v + (size_t)h->n_loc * h->n_cells; }
const double* la_of(lat_ctx* h, const double* v) { return v + (size_t)h->n_loc * h->n_cells + h->n_primal; }

// w_u = K~ v_u (+ B^T v_l when with_bt), w_l = B v_u  (saddle-point operator)
// op32: the reduced tangent action in FP32 (the operator of the mixed modes' inner GMRES).  The
// partially assembled vector goes to a plain FP32 cell-stacked vector (corner rows gathered from
// the primal part, Dirichlet rows zero), the FP32 copies of K^r and alpha act on it with the
// plain (non-FETI) action kernels, and the result comes back to FP64 with the Dirichlet rows of
// non-corner DOFs cleared; index work (primal assembly, jumps) is the same.  The outer FGMRES
// always takes the FP64 action, so the system it solves to its tolerance is the FP64 one.
void feti_operator(lat_ctx* h, const double* v, double* w, bool with_lambda, bool op32 = false) {
  const double* vP = pr_of(h, v);
  if (op32) {
    const int64_t nloc = (int64_t)h->n_loc * h->n_cells;
    h->x32.ensure(nloc);
    h->y32.ensure(nloc);
    const dim3 grid(div_up(h->n_cells, 256), h->n_nodes_cell);
    LAT_LAUNCH(h, k_feti_pack32<<<grid, 256, 0, h->stream>>>(h->n_cells, h->dim, h->n_P, h->corner_of_node.p,
        h->pidx.p, h->loc_fixed.p, v, vP, h->x32.p));
    run_apply(h, h->x32.p, h->y32.p, 1, nullptr, false);
    LAT_LAUNCH(h, k_feti_unpack64<<<grid, 256, 0, h->stream>>>(h->n_cells, h->dim, h->corner_of_node.p,
        h->loc_fixed.p, h->y32.p, w));
    LAT_CHECK_LAUNCH();
  } else {
    run_apply(h, v, w, 0, vP, true);
  }
  // primal rows -> assembled primal part, then clear corner rows
  if (h->n_primal)
    LAT_LAUNCH(h, k_primal_assemble<<<div_up(h->n_primal, 256), 256, 0, h->stream>>>(h->n_primal, h->p_copy_ptr.p,
        h->p_copy.p, w, pr_of(h, w), 0));
  LAT_LAUNCH(h, k_zero_rows<<<div_up(h->n_cells, 256), 256, 0, h->stream>>>(h->n_cells, h->n_P, h->pdofs.p, w));
  if (h->n_lambda) {
    if (with_lambda)
      LAT_LAUNCH(h, k_jump_t<<<div_up(h->n_dual, 256), 256, 0, h->stream>>>(h->n_dual, h->dual_entry.p, h->dual_l1.p,
          h->dual_l2.p, nullptr, la_of(h, v), 1.0, w));
    LAT_LAUNCH(h, k_jump<<<div_up(h->n_lambda, 256), 256, 0, h->stream>>>(h->n_lambda, h->lam_p.p, h->lam_m.p, v, 1.0,
                                                              la_of(h, w), 0));
  }
  LAT_CHECK_LAUNCH();
}

// x_P = S_PP^{-1} g_P: by block LU on layered lattices in FP64 mode, else with the explicit
// inverse of the coarse matrix (computed in FP64; the mixed modes apply an FP32 copy, like the
// rest of their preconditioner)
void run_coarse_solve(lat_ctx* h, const double* g, double* x) {
  const int64_t np = h->n_primal;
  if (h->cb_solve) {
    KernelTimer kt(h, "coarse_solve");
    run_coarse_block_solve(h, g, x);
    return;
  }
  KernelTimer kt(h, "coarse_gemv");
  const size_t shm = (size_t)np * sizeof(double);
  if (h->prec != LAT_FP64 && h->CoarseInv32.p && shm <= 200 * 1024) {
    const int ldc = (int)h->coarse32_ld;
    const size_t shf = (size_t)ldc * sizeof(float);
    LAT_CUDA(cudaFuncSetAttribute(k_gemv_xs_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shf));
    LAT_LAUNCH(h, k_gemv_xs_f32<<<(int)div_up(np, 16), 512, shf, h->stream>>>((int)np, ldc, h->CoarseInv32.p, g, x));
  } else if (np % 2 == 0 && shm <= 200 * 1024) {
    LAT_CUDA(cudaFuncSetAttribute(k_gemv_xs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    const int grid = (int)div_up(np, 16);   // 16 warps per CTA, one row each
    LAT_LAUNCH(h, k_gemv_xs<<<grid, 512, shm, h->stream>>>((int)np, h->CoarseInv.p, g, x));
  } else {
    LAT_LAUNCH(h, k_gemv<<<div_up(np * 32, 256), 256, 0, h->stream>>>(np, h->CoarseInv.p, g, x));
  }
}

// w_u = K^-rom v_u  (local part and primal part; multiplier part untouched).
//   KINV_FULL     any v_R; every remaining and corner row of w is formed;
//   KINV_DUAL_IN  v_R vanishes off the dual DOFs: the product reads the dual columns only;
//   KINV_DUAL     the same, and only the dual and corner rows of w are formed (the interface
//                 operator B K^-rom B^T reads no others): the trailing dual block,
//                 (n_R - n_I + n_P) x (n_R - n_I) instead of (n_R + n_P) x n_R.
//   lam (KINV_DUAL on the tensor-core path only): v is B^T lam on the dual DOFs and zero
//                 elsewhere, formed by the product's operand packing (v is not read).
void kinv(lat_ctx* h, const double* v, double* w, KinvMode mode = KINV_FULL, const double* lam = nullptr) {
  const int ns = h->n_cells, nR = h->n_R, nP = h->n_P;
  const int lo_r = mode == KINV_DUAL ? h->n_I : 0;   // first row and column of the view
  const int lo_c = mode == KINV_FULL ? 0 : h->n_I;
  const int nKr = nR - lo_r, nKc = nR - lo_c;
  const int64_t kstride = (int64_t)(nR + nP) * nR;
  const size_t off = (size_t)lo_r * nR + lo_c;
  const int* rr = h->rdofs.p + lo_r;
  const int* rc = h->rdofs.p + lo_c;
  static const char* const tg_gemv[3] = {"local_gemv", "local_gemv_dual", "local_gemv_dual_in"};
  static const char* const tg_segmm[3] = {"local_segmm", "local_segmm_dual", "local_segmm_dual_in"};
  double* wl = loc_of(h, w);
  // y_R = G~ v_R and Phi^T v_R (corner rows of wl) in one product
  const bool gemv = (int64_t)h->n_keys * 8 > ns;
  const bool lo = h->prec != LAT_FP64;
  if (gemv) {
    KernelTimer kt(h, tg_gemv[mode]);
    const size_t shm = (size_t)nKc * sizeof(double);
    if (lo) {
      LAT_CUDA(cudaFuncSetAttribute(k_local_gemv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
      LAT_LAUNCH(h, k_local_gemv<float><<<dim3(ns, split_rows(h, ns, nKr + nP)), 256, shm, h->stream>>>(ns, nKr, nKc, nP, nR, kstride, h->G32.p + off,
          h->key_slot.p, h->c_cell.p, rr, rc, h->pdofs.p, v, wl));
    } else {
      LAT_CUDA(cudaFuncSetAttribute(k_local_gemv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
      LAT_LAUNCH(h, k_local_gemv<double><<<dim3(ns, split_rows(h, ns, nKr + nP)), 256, shm, h->stream>>>(ns, nKr, nKc, nP, nR, kstride, h->G.p + off,
          h->key_slot.p, h->c_cell.p, rr, rc, h->pdofs.p, v, wl));
    }
  } else if (h->prec == LAT_MIXED_BF16) {
    // tcgen05, BF16 operands, FP32 accumulation
    if (lam) run_local_tc_lam(h, lam, wl);
    else run_local_tc(h, v, wl, mode);
  } else {
    KernelTimer kt(h, tg_segmm[mode]);
    dim3 grid(h->max_tiles, div_up(nKr + nP, 64));
    if (lo)
      LAT_LAUNCH(h, k_local_segmm<float, 64><<<grid, 256, 0, h->stream>>>(ns, nKr, nKc, nP, nR, kstride, 0,
          h->G32.p + off, h->tile_seg.p, h->tile_c0.p, h->seg_ptr.p, h->perm.p, h->c_cell.p, rr, rc, h->pdofs.p, v, wl));
    else
      LAT_LAUNCH(h, k_local_segmm_n4<<<grid, 256, 0, h->stream>>>(ns, nKr, nKc, nP, nR, kstride, 0, h->G.p + off,
          h->tile_seg.p, h->tile_c0.p, h->seg_ptr.p, h->perm.p, h->c_cell.p, rr, rc, h->pdofs.p, v, wl));
  }
  LAT_CHECK_LAUNCH();
  if (h->n_primal) {
    // g_P = v_P + sum_s A_P^T Phi^T v_R   (from the corner rows of wl)
    LAT_LAUNCH(h, k_primal_assemble<<<div_up(h->n_primal, 256), 256, 0, h->stream>>>(h->n_primal, h->p_copy_ptr.p,
        h->p_copy.p, wl, h->gP.p, lam ? 0 : 1, lam ? nullptr : pr_of(h, v)));
    run_coarse_solve(h, h->gP.p, pr_of(h, w));
  }
  if (h->n_primal) {
    // w_R += Phi x_P on the view's rows (corner values gathered per cell first); the extra nP
    // rows clear the corner rows
    constexpr int RB = 32;
    const dim3 grid(div_up(ns, 128), div_up(nKr + nP, RB));
    const int64_t gt = (int64_t)ns * nP;
    if (lo && h->Phi32.p) {
      h->tP32.ensure((size_t)gt);
      LAT_LAUNCH(h, k_gather_tp<float><<<div_up(gt, 256), 256, 0, h->stream>>>(ns, nP, h->pidx.p, pr_of(h, w),
                                                                               h->tP32.p));
      LAT_LAUNCH(h, k_phi_rows<float><<<grid, 128, 0, h->stream>>>(
          ns, nKr, nP, RB, (int64_t)nR * nP, h->Phi32.p + (size_t)lo_r * nP, h->key_slot.p, rr, h->tP32.p,
          h->loc_fixed.p, h->pdofs.p, wl));
    } else {
      h->tP.ensure((size_t)gt);
      LAT_LAUNCH(h, k_gather_tp<double><<<div_up(gt, 256), 256, 0, h->stream>>>(ns, nP, h->pidx.p, pr_of(h, w),
                                                                                h->tP.p));
      LAT_LAUNCH(h, k_phi_rows<double><<<grid, 128, 0, h->stream>>>(
          ns, nKr, nP, RB, (int64_t)nR * nP, h->Phi.p + (size_t)lo_r * nP, h->key_slot.p, rr, h->tP.p,
          h->loc_fixed.p, h->pdofs.p, wl));
    }
    LAT_CHECK_LAUNCH();
  } else {
    LAT_LAUNCH(h, k_zero_rows<<<div_up(ns, 256), 256, 0, h->stream>>>(ns, nP, h->pdofs.p, wl));
  }
}

// S_op p = B K^-rom B^T p (multiplier vectors); uses tmp (saddle sized) as scratch
// the tensor-core path forms B^T lambda inside its operand packing (no zeroed local vector, no
// scatter): BF16 mode with the segmented products (few keys)
bool fused_dual(const lat_ctx* h) { return h->prec == LAT_MIXED_BF16 && (int64_t)h->n_keys * 8 <= h->n_cells; }

void dual_op(lat_ctx* h, const double* p, double* q, double* t1, double* t2) {
  const int64_t nloc = (int64_t)h->n_loc * h->n_cells;
  if (fused_dual(h)) {
    kinv(h, nullptr, t2, KINV_DUAL, p);
  } else {
    LAT_CUDA(cudaMemsetAsync(t1, 0, (nloc + h->n_primal) * sizeof(double), h->stream));
    LAT_LAUNCH(h, k_jump_t<<<div_up(h->n_dual, 256), 256, 0, h->stream>>>(h->n_dual, h->dual_entry.p, h->dual_l1.p,
                                                            h->dual_l2.p, nullptr, p, 1.0, t1));
    LAT_CHECK_LAUNCH();
    kinv(h, t1, t2, KINV_DUAL);   // t1 vanishes off the dual DOFs; only dual rows of t2 are read
  }
  LAT_LAUNCH(h, k_jump<<<div_up(h->n_lambda, 256), 256, 0, h->stream>>>(h->n_lambda, h->lam_p.p, h->lam_m.p, t2, 1.0, q, 0));
  LAT_CHECK_LAUNCH();
}

// lumped preconditioner z = B_D K~_dd B_D^T r
void dual_precond(lat_ctx* h, const double* r, double* z, double* t1, double* t2, double* wloc) {
  const int64_t nloc = (int64_t)h->n_loc * h->n_cells;
  const bool fused = h->iface == 0 && fused_dual(h);
  if (!fused) {
    LAT_CUDA(cudaMemsetAsync(t1, 0, (nloc + h->n_primal) * sizeof(double), h->stream));
    LAT_LAUNCH(h, k_jump_t<<<div_up(h->n_dual, 256), 256, 0, h->stream>>>(h->n_dual, h->dual_entry.p, h->dual_l1.p,
                                                            h->dual_l2.p, h->dual_scale.p, r, 1.0, t1));
    LAT_CHECK_LAUNCH();
  }
  if (h->iface == 0) {
    // Dirichlet: local dual Schur complements of the cells' principals, c_s S_DD^{slot(s)} x_D;
    // with few keys as a segmented product over the key-ordered cells (as the local inverses)
    const int nD = h->n_R - h->n_I;
    const size_t shm = (size_t)nD * sizeof(double);
    const bool seg = (int64_t)h->n_keys * 8 <= h->n_cells;
    if (fused) {
      run_sdd_tc(h, nullptr, t2, r);   // tcgen05, BF16 operand pairs, FP32 accumulation; operand B_D^T r
    } else if (seg) {
      KernelTimer kt(h, "dual_schur");
      const int* rd = h->rdofs.p + h->n_I;
      dim3 grid(h->max_tiles, div_up(nD, 64));
      if (h->prec == LAT_FP64)
        LAT_LAUNCH(h, k_local_segmm_n4<<<grid, 256, 0, h->stream>>>(h->n_cells, nD, nD, 0, nD, (int64_t)nD * nD, 1,
            h->SDD.p, h->tile_seg.p, h->tile_c0.p, h->seg_ptr.p, h->perm.p, h->c_cell.p, rd, rd, h->pdofs.p, t1, t2));
      else
        LAT_LAUNCH(h, k_local_segmm<float, 64><<<grid, 256, 0, h->stream>>>(h->n_cells, nD, nD, 0, nD,
            (int64_t)nD * nD, 1, h->SDD32.p, h->tile_seg.p, h->tile_c0.p, h->seg_ptr.p, h->perm.p, h->c_cell.p, rd,
            rd, h->pdofs.p, t1, t2));
    } else if (h->prec == LAT_FP64) {
      LAT_CUDA(cudaFuncSetAttribute(k_dual_schur<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
      LAT_LAUNCH(h, k_dual_schur<double><<<dim3(h->n_cells, split_rows(h, h->n_cells, nD)), 256, shm, h->stream>>>(h->n_cells, h->n_I, nD, h->SDD.p,
          h->key_slot.p, h->c_cell.p, h->rdofs.p, t1, t2));
    } else {
      LAT_CUDA(cudaFuncSetAttribute(k_dual_schur<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
      LAT_LAUNCH(h, k_dual_schur<float><<<dim3(h->n_cells, split_rows(h, h->n_cells, nD)), 256, shm, h->stream>>>(h->n_cells, h->n_I, nD, h->SDD32.p,
          h->key_slot.p, h->c_cell.p, h->rdofs.p, t1, t2));
    }
  } else if (h->prec == LAT_FP64) {
    // lumped: K~ on the dual-only local vector (corners zero: primal part of t1 is zero)
    run_apply(h, t1, t2, 0, pr_of(h, t1), true);
  } else {
    h->x32.ensure(nloc);
    h->y32.ensure(nloc);
    LAT_LAUNCH(h, k_d2f<<<ew_blocks(h, nloc), 256, 0, h->stream>>>(nloc, t1, h->x32.p));
    run_apply(h, h->x32.p, h->y32.p, 1, pr_of(h, t1), true);
    run_f2d(h, nloc, h->y32.p, t2);
  }
  LAT_LAUNCH(h, k_jump_scaled<<<div_up(h->n_lambda, 256), 256, 0, h->stream>>>(h->n_lambda, h->lam_p.p, h->lam_m.p, t2, wloc, z));
  LAT_CHECK_LAUNCH();
}

}  // namespace

void run_feti_operator(lat_ctx* h, const double* v, double* w) { feti_operator(h, v, w, true); }

void run_kinv(lat_ctx* h, const double* v, double* w) {
  kinv(h, v, w);
  if (h->n_lambda)
    LAT_CUDA(cudaMemcpyAsync(la_of(h, w), la_of(h, v), h->n_lambda * sizeof(double), cudaMemcpyDeviceToDevice,
                             h->stream));
}

void run_block_precond(lat_ctx* h, const double* v, double* w, int pcg_iters, double pcg_rtol) {
  const int64_t L = h->n_lambda;
  double* t = h->kv_tmp[2].p;   // K^-rom v_u, later v_u - B^T z
  double* t1 = h->kv_tmp[3].p;
  double* t2 = h->kv_tmp[4].p;
  double* pv = h->pcg_ws.p;     // five multiplier-sized work vectors
  if (L == 0) {
    kinv(h, v, w);
    return;
  }
  kinv(h, v, t);
  double* y = pv;            // rhs of the interface solve, then residual r
  double* x = pv + L;        // solution
  double* z = pv + 2 * L;
  double* p = pv + 3 * L;
  double* q = pv + 4 * L;
  double* wloc = h->kv_tmp[1].p;  // dual weights (1/multiplicity) as a dense local array
  LAT_REQUIRE((size_t)5 * L <= h->pcg_ws.n, LAT_EINVAL, "multiplier work space too small");
  const int64_t nloc = (int64_t)h->n_loc * h->n_cells;
  LAT_CUDA(cudaMemsetAsync(wloc, 0, nloc * sizeof(double), h->stream));
  LAT_LAUNCH(h, k_fill_dual_weights<<<div_up(h->n_dual, 256), 256, 0, h->stream>>>(h->n_dual, h->dual_entry.p, h->dual_scale.p, wloc));
  // y = v_l - B t
  LAT_CUDA(cudaMemcpyAsync(y, la_of(h, v), L * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  LAT_LAUNCH(h, k_jump<<<div_up(L, 256), 256, 0, h->stream>>>(L, h->lam_p.p, h->lam_m.p, t, -1.0, y, 1));
  LAT_CHECK_LAUNCH();
  // PCG on S x = y from x = 0
  LAT_CUDA(cudaMemsetAsync(x, 0, L * sizeof(double), h->stream));
  double* sc = h->red_part.p + 3000;  // PCG scalars, see k_sum_part_pcg
  if (pcg_iters > 0) {
    // PCG until the preconditioned residual r^T M r has dropped by pcg_rtol^2 (checked on the
    // host after every iteration), at most pcg_iters iterations, or until breakdown.  One
    // iteration updates the search direction first (p = z + beta p; p = z on the first pass, from
    // p = 0 and beta = 0), so that every iteration is the same sequence of launches: outside the
    // kernel-timing mode it is captured once per preconditioner setup as a CUDA graph and replayed.
    LAT_CUDA(cudaMemsetAsync(sc, 0, 8 * sizeof(double), h->stream));
    dual_precond(h, y, z, t1, t2, wloc);
    LAT_CUDA(cudaMemsetAsync(p, 0, L * sizeof(double), h->stream));
    dev_dot(h, L, y, z, sc);
    double rz0 = -1.0;
    if (pcg_rtol > 0) {
      LAT_CUDA(cudaMemcpyAsync(h->h_pinned + 8, sc, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      LAT_CUDA(cudaStreamSynchronize(h->stream));
      rz0 = h->h_pinned[8];
    }
    const int nb = ew_blocks(h, L);
    const bool check = pcg_rtol > 0;
    auto body = [&]() {
      LAT_LAUNCH(h, k_xpby_s<<<nb, 256, 0, h->stream>>>(L, z, sc + 4, sc + 5, p));
      dual_op(h, p, q, t1, t2);
      const int rb = red_blocks(L);
      LAT_LAUNCH(h, k_dot_part<<<rb, 256, 0, h->stream>>>(L, p, q, h->red_part.p + 1024));
      LAT_LAUNCH(h, k_sum_part_pcg<<<1, 512, 0, h->stream>>>(rb, h->red_part.p + 1024, sc, 0));   // alpha
      LAT_LAUNCH(h, k_axpy2_s<<<nb, 256, 0, h->stream>>>(L, sc + 3, p, q, x, y));
      dual_precond(h, y, z, t1, t2, wloc);
      LAT_LAUNCH(h, k_dot_part<<<rb, 256, 0, h->stream>>>(L, y, z, h->red_part.p + 1024));
      LAT_LAUNCH(h, k_sum_part_pcg<<<1, 512, 0, h->stream>>>(rb, h->red_part.p + 1024, sc, 1));   // beta
      if (check)
        LAT_CUDA(cudaMemcpyAsync(h->h_pinned + 8, sc, 6 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      LAT_CHECK_LAUNCH();
    };
    bool graph = (!h->timing || h->timing_apply_only) && h->graphs_ok;
    if (graph && (!h->pcg_exec || h->pcg_exec_check != (int)check)) {
      if (h->pcg_exec) {
        cudaGraphExecDestroy(h->pcg_exec);
        h->pcg_exec = nullptr;
      }
      // captured on a private stream (the caller's may be the legacy default stream, which
      // cannot be captured); replays are ordered on the handle's stream
      const int64_t n0 = h->n_launch;
      if (!h->cap_stream) LAT_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
      cudaStream_t user = h->stream;
      cudaGraph_t g = nullptr;
      cudaError_t e1 = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed);
      if (e1 == cudaSuccess) {
        h->stream = h->cap_stream;
        try {
          body();
        } catch (const LatError&) {
          graph = false;
        }
        h->stream = user;
        e1 = cudaStreamEndCapture(h->cap_stream, &g);
      }
      if (graph && e1 == cudaSuccess && g && cudaGraphInstantiate(&h->pcg_exec, g, 0) == cudaSuccess) {
        h->pcg_graph_kernels = h->n_launch - n0;
        h->pcg_exec_check = (int)check;
      } else {
        graph = false;
        h->graphs_ok = false;   // this handle keeps the launch-by-launch path from now on
        h->pcg_exec = nullptr;
      }
      if (g) cudaGraphDestroy(g);
      h->n_launch = n0;
      cudaGetLastError();
    }
    int it = 0;
    for (; it < pcg_iters; ++it) {
      if (graph) {
        LAT_CUDA(cudaGraphLaunch(h->pcg_exec, h->stream));
        h->n_launch += h->pcg_graph_kernels;
      } else {
        body();
      }
      if (check) {
        LAT_CUDA(cudaStreamSynchronize(h->stream));
        const double rz = h->h_pinned[8], frozen = h->h_pinned[13];
        if (frozen != 0.0 || !(rz0 > 0) || rz <= pcg_rtol * pcg_rtol * rz0) break;
      }
    }
    h->pcg_its_total += std::min(it + 1, pcg_iters);
  }
  // z_l = -x ;  w_u = K^-rom (v_u - B^T z_l) = K^-rom v_u + K^-rom B^T x, the first term kept in t
  // from above and the second with the dual columns only (B^T x vanishes off the dual DOFs)
  LAT_CUDA(cudaMemsetAsync(t1, 0, (nloc + h->n_primal) * sizeof(double), h->stream));
  LAT_LAUNCH(h, k_jump_t<<<div_up(h->n_dual, 256), 256, 0, h->stream>>>(h->n_dual, h->dual_entry.p, h->dual_l1.p,
                                                          h->dual_l2.p, nullptr, x, 1.0, t1));
  LAT_CHECK_LAUNCH();
  kinv(h, t1, w, KINV_DUAL_IN);
  LAT_LAUNCH(h, k_axpby<<<ew_blocks(h, nloc + h->n_primal), 256, 0, h->stream>>>(nloc + h->n_primal, 1.0, t, 1.0, w));
  LAT_LAUNCH(h, k_axpby<<<ew_blocks(h, L), 256, 0, h->stream>>>(L, -1.0, x, 0.0, la_of(h, w)));
  LAT_CHECK_LAUNCH();
}

namespace {

// one FGMRES level: its Krylov basis V, preconditioned vectors Z, Hessenberg matrix, Givens
// data, device scalars and the operator output vector
struct GmresLevel {
  DBuf<double>* V;
  DBuf<double>* Z;
  DBuf<double>* H;
  DBuf<double>* small;
  DBuf<double>* scal;
  double* w;
};

// right-preconditioned restarted FGMRES from x (in/out, or zero when x_zero); returns iterations,
// *rel = final estimate.  op32 selects the FP32 reduced tangent action as the operator.
template <typename Prec>
int fgmres_core(lat_ctx* h, const GmresLevel& L, const double* b, double* x, bool x_zero, double rtol,
                int max_it, int restart, bool op32, Prec&& precond, double* rel_out) {
  const int64_t n = h->n_krylov;
  const int m = std::max(2, restart);
  LAT_REQUIRE(m <= 190, LAT_EINVAL, "krylov_restart too large (max 190)");
  L.V->ensure((size_t)(m + 1) * n);
  L.Z->ensure((size_t)m * n);
  L.H->ensure((size_t)(m + 1) * m + 4 * (m + 1));
  L.small->ensure(3 * m + 8);
  L.scal->ensure(8 + 4 * (m + 2));
  const int nb = red_blocks(n);
  h->dots_part.ensure((size_t)(m + 1) * nb);
  double* sc = L.scal->p;              // [0] nrm2, [1] estimate
  double* hcol = sc + 8;
  double* h2 = hcol + (m + 2);
  double* yv = h2 + (m + 2);
  double* w = L.w;
  const int eb = ew_blocks(h, n);
  double* hp = h->h_pinned;
  dev_dot(h, n, b, b, sc);
  LAT_CUDA(cudaMemcpyAsync(hp, sc, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LAT_CUDA(cudaStreamSynchronize(h->stream));
  const double bnorm = std::sqrt(hp[0]);
  if (x_zero) LAT_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), h->stream));
  if (bnorm == 0.0) {
    LAT_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), h->stream));
    if (rel_out) *rel_out = 0;
    return 0;
  }
  int total = 0;
  double rel = 1.0;
  bool first = true;
  while (total < max_it) {
    // r = b - A x  (r = b for a zero start)
    if (first && x_zero) {
      LAT_CUDA(cudaMemcpyAsync(w, b, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
      rel = 1.0;
    } else {
      feti_operator(h, x, w, true, op32);
      LAT_LAUNCH(h, k_axpby<<<eb, 256, 0, h->stream>>>(n, 1.0, b, -1.0, w));
      dev_dot(h, n, w, w, sc);
      LAT_CUDA(cudaMemcpyAsync(hp, sc, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      LAT_CUDA(cudaStreamSynchronize(h->stream));
      rel = std::sqrt(hp[0]) / bnorm;
      if (rel <= rtol) break;
    }
    first = false;
    LAT_LAUNCH(h, k_scale_dev<<<eb, 256, 0, h->stream>>>(n, w, sc, L.V->p));
    LAT_LAUNCH(h, k_gmres_init<<<1, 1, 0, h->stream>>>(m, L.small->p, sc));
    int j = 0;
    for (; j < m && total < max_it; ++j, ++total) {
      double* vj = L.V->p + (size_t)j * n;
      double* zj = L.Z->p + (size_t)j * n;
      precond(vj, zj);
      feti_operator(h, zj, w, true, op32);
      // CGS with one re-orthogonalisation
      KernelTimer kt(h, "krylov_orth");
      for (int pass = 0; pass < 2; ++pass) {
        LAT_LAUNCH(h, k_multidot_part<<<nb, 256, 0, h->stream>>>(n, j + 1, L.V->p, w, h->dots_part.p));
        LAT_LAUNCH(h, k_multidot_final<<<j + 1, 256, 0, h->stream>>>(nb, h->dots_part.p, pass == 0 ? hcol : h2));
        LAT_LAUNCH(h, k_multi_axpy<<<eb, 256, 0, h->stream>>>(n, j + 1, L.V->p, pass == 0 ? hcol : h2, -1.0, w));
      }
      LAT_LAUNCH(h, k_axpby<<<1, 256, 0, h->stream>>>(j + 1, 1.0, h2, 1.0, hcol));
      dev_dot(h, n, w, w, sc);
      LAT_LAUNCH(h, k_givens<<<1, 1, 0, h->stream>>>(j, m, L.H->p, L.small->p, hcol, sc, sc + 1));
      LAT_LAUNCH(h, k_scale_dev<<<eb, 256, 0, h->stream>>>(n, w, sc, L.V->p + (size_t)(j + 1) * n));
      LAT_CHECK_LAUNCH();
      LAT_CUDA(cudaMemcpyAsync(hp, sc, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      LAT_CUDA(cudaStreamSynchronize(h->stream));
      rel = hp[1] / bnorm;
      if (rel <= rtol || !(hp[0] > 0.0)) {
        ++j;
        ++total;
        break;
      }
    }
    // x += Z y
    LAT_LAUNCH(h, k_gmres_solve<<<1, 1, 0, h->stream>>>(j, m, L.H->p, L.small->p, yv));
    LAT_LAUNCH(h, k_multi_axpy<<<eb, 256, 0, h->stream>>>(n, j, L.Z->p, yv, 1.0, x));
    LAT_CHECK_LAUNCH();
    if (rel <= rtol) break;
  }
  if (rel_out) *rel_out = rel;
  return total;
}

}  // namespace

// FGMRES on the saddle-point system (Section 3.3.1) with the FP64 reduced tangent action.  Its
// preconditioner is the block preconditioner of Eq. (ifetidp_precond), or, in the mixed modes
// with inner_its > 0, an inner flexible GMRES whose operator is the FP32 reduced tangent action
// and whose preconditioner is the block preconditioner (mixed precision inside a flexible
// Krylov method: the FP32 action and preconditioner only shape the search directions).
int run_fgmres(lat_ctx* h, const double* b, double* x, const lat_newton_opts* o, double* rel_out) {
  GmresLevel outer{&h->V, &h->Zk, &h->Hh, &h->gmres_small, &h->kscal[0], h->kv_tmp[0].p};
  auto block = [&](const double* v, double* z) { run_block_precond(h, v, z, o->pcg_iters, o->pcg_rtol); };
  int total;
  if (h->prec != LAT_FP64 && o->inner_its > 0) {
    GmresLevel inner{&h->V2, &h->Z2, &h->Hh2, &h->gmres_small2, &h->kscal[1], h->kv_tmp[1].p};
    // an inner solve that misses inner_rtol within inner_its iterations (strongly indefinite
    // states, e.g. the affine predictor of the first load step) spent its iterations for little
    // gain: the rest of this solve then takes the block preconditioner directly (FGMRES allows
    // the preconditioner to change from one iteration to the next)
    bool stalled = false;
    auto nested = [&](const double* v, double* z) {
      if (stalled) {
        block(v, z);
        return;
      }
      double r = 0;
      h->inner_its_total += fgmres_core(h, inner, v, z, true, o->inner_rtol, o->inner_its, o->inner_its, true,
                                        block, &r);
      stalled = r > o->inner_rtol;
    };
    total = fgmres_core(h, outer, b, x, false, o->krylov_rtol, o->krylov_max_it, o->krylov_restart, false, nested,
                        rel_out);
  } else {
    total = fgmres_core(h, outer, b, x, false, o->krylov_rtol, o->krylov_max_it, o->krylov_restart, false, block,
                        rel_out);
  }
  if (h->prec == LAT_MIXED_BF16 || (h->cb_solve && h->cb_wide && h->cb_coop_grid > 0)) {
    int fl = 0;
    LAT_CUDA(cudaMemcpyAsync(&fl, h->flag.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    LAT_REQUIRE(!(fl & 4), LAT_ETIMEOUT, "a tensor-core wait in the local product gave up");
    LAT_REQUIRE(!(fl & 8), LAT_ETIMEOUT, "a block-row copy of the cooperative coarse solve did not land");
  }
  return total;
}

void run_feti_to_global(lat_ctx* h, const double* v, double* u) {
  LAT_LAUNCH(h, k_to_global<<<div_up(h->n_glob_nodes, 256), 256, 0, h->stream>>>(h->n_glob_nodes, h->dim, h->n_nodes_cell,
      h->n_cells, h->n_P, h->copy_ptr.p, h->copy_idx.p, h->corner_of_node.p, h->pidx.p, h->dof_fixed.p,
      v, pr_of(h, v), u));
  LAT_CHECK_LAUNCH();
}

void run_feti_from_global(lat_ctx* h, const double* u, double* v, bool split) {
  LAT_CUDA(cudaMemsetAsync(v, 0, h->n_krylov * sizeof(double), h->stream));
  LAT_LAUNCH(h, k_from_global<<<div_up(h->n_glob_nodes, 256), 256, 0, h->stream>>>(h->n_glob_nodes, h->dim, h->n_nodes_cell,
      h->n_cells, h->n_P, h->copy_ptr.p, h->copy_idx.p, h->corner_of_node.p, h->pidx.p, h->dof_fixed.p,
      u, split ? 1 : 0, v, pr_of(h, v)));
  LAT_CHECK_LAUNCH();
}

void run_axpy(lat_ctx* h, int64_t n, double a, const double* x, double* y) {
  LAT_LAUNCH(h, k_axpby<<<ew_blocks(h, n), 256, 0, h->stream>>>(n, a, x, 1.0, y));
  LAT_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------------------------
// Newton, adjoint and the remaining entry points
// ---------------------------------------------------------------------------------------------
// FETI-DP setup with adaptive primal enrichment (Section 3.3.2): while the remaining block of
// some principal, or the coarse matrix, is not positive definite, add primal nodes on every cell
// edge, for all cells alike, rebuild the index sets and set up again; the enrichment is kept for
// later iterations.  (With definite remaining blocks the coarse matrix loses definiteness when a
// cell's local Schur complement does: inertia(K^s) = inertia(K_RR^s) + inertia(S^s); the edge
// nodes tie the cells' free sides to their neighbours, which removes those modes.)
void prepare_enriched(lat_ctx* h, const lat_newton_opts* o, const double* u_glob) {
  if (h->enrich_level < o->min_enrich) {
    build_feti(h, std::min(o->min_enrich, o->max_enrich));
    if (h->verbose)
      std::fprintf(stderr, "[lattice] primal enrichment level %d (start): %d primal DOFs per cell, %lld coarse DOFs\n",
                   h->enrich_level, h->n_P, (long long)h->n_primal);
  }
  run_prepare_solver(h, o, u_glob);
  while ((h->indefinite || h->coarse_indefinite) && h->enrich_level < o->max_enrich) {
    build_feti(h, h->enrich_level + 1);
    if (h->verbose)
      std::fprintf(stderr, "[lattice] primal enrichment level %d: %d primal DOFs per cell, %lld coarse DOFs\n",
                   h->enrich_level, h->n_P, (long long)h->n_primal);
    run_prepare_solver(h, o, u_glob);
  }
}

namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

void check_opts(const lat_newton_opts* o) {
  LAT_REQUIRE(o, LAT_EINVAL, "options required");
  LAT_REQUIRE(o->krylov_restart >= 2 && o->krylov_restart <= 190, LAT_EINVAL, "krylov_restart in [2, 190]");
  LAT_REQUIRE(o->krylov_max_it >= 1 && o->newton_max_it >= 1 && o->armijo_max_m >= 0 && o->pcg_iters >= 0,
              LAT_EINVAL, "iteration caps must be positive");
  LAT_REQUIRE(o->force_all || o->max_nr >= 1, LAT_EINVAL, "max_nr must be >= 1");
  LAT_REQUIRE(o->pcg_rtol >= 0 && o->pcg_rtol < 1, LAT_EINVAL, "pcg_rtol in [0, 1)");
  LAT_REQUIRE(o->interface_precond == 0 || o->interface_precond == 1, LAT_EINVAL, "interface_precond is 0 or 1");
  LAT_REQUIRE(o->max_enrich >= 0 && o->max_enrich <= 6, LAT_EINVAL, "max_enrich in [0, 6]");
  LAT_REQUIRE(o->coarse_block_lu >= -1 && o->coarse_block_lu <= 4, LAT_EINVAL, "coarse_block_lu in [-1, 4]");
  LAT_REQUIRE(o->precond_tangent >= -1 && o->precond_tangent <= 1, LAT_EINVAL, "precond_tangent in {-1, 0, 1}");
  LAT_REQUIRE(o->min_enrich >= 0 && o->min_enrich <= o->max_enrich, LAT_EINVAL, "min_enrich in [0, max_enrich]");
  LAT_REQUIRE(o->inner_its >= 0 && o->inner_its <= 190, LAT_EINVAL, "inner_its in [0, 190]");
  LAT_REQUIRE(o->inner_rtol >= 0 && o->inner_rtol < 1, LAT_EINVAL, "inner_rtol in [0, 1)");
  LAT_REQUIRE(o->snapshot == 0 || o->snapshot == 1, LAT_EINVAL, "snapshot is 0 or 1");
  LAT_REQUIRE(o->eps_refine >= 0 && o->eps_refine <= 12, LAT_EINVAL, "eps_refine in [0, 12]");
  LAT_REQUIRE(o->eps_refine_rate > 0 && o->eps_refine_rate <= 1, LAT_EINVAL, "eps_refine_rate in (0, 1]");
}

// FETI rhs of K du = -r: the assembled residual -r split evenly over the copies of each
// remaining DOF, assembled on the free primal DOFs, zero multipliers.  Any split that sums to -r
// gives the same du; the even split keeps ||rhs|| ~ ||r_F|| (the raw per-cell forces do not
// cancel at interfaces and would make the relative Krylov tolerance an absolute floor).
void newton_rhs(lat_ctx* h, const double* r_glob, double* b) {
  run_feti_from_global(h, r_glob, b, true);
  LAT_LAUNCH(h, k_axpby<<<ew_blocks(h, h->n_krylov), 256, 0, h->stream>>>(h->n_krylov, 0.0, b, -1.0, b));
  LAT_CHECK_LAUNCH();
}

}  // namespace

extern "C" lat_status lattice_default_opts(lat_handle h, lat_newton_opts* o) {
  if (!h || !o) return LAT_EINVAL;
  o->eps = h->dim == 2 ? 3e-4 : 5e-3;
  o->max_nr = 256;
  o->force_all = 0;
  o->newton_rtol = 1e-8;
  o->newton_max_it = 30;
  o->krylov_rtol = h->prec == LAT_FP64 ? 1e-10 : 1e-6;
  o->krylov_max_it = 600;
  o->krylov_restart = 60;
  o->pcg_iters = 100;
  o->armijo_max_m = 30;
  o->pcg_rtol = 3e-2;
  o->interface_precond = 0;
  o->max_enrich = 3;
  o->coarse_block_lu = -1;
  o->precond_tangent = -1;
  o->min_enrich = 0;
  o->inner_its = h->prec == LAT_FP64 ? 0 : 20;
  o->inner_rtol = 1e-2;
  o->snapshot = 0;
  o->eps_refine = 2;
  o->eps_refine_rate = 0.5;
  return LAT_OK;
}

extern "C" lat_status newton_step(lat_handle h, double* u, int32_t max_iterations, const lat_newton_opts* o,
                                  lat_newton_report* rep) {
  if (!h || !u) return LAT_EINVAL;
  lat_newton_report R{};
  lat_status st = guard(h, [&] {
    check_opts(o);
    const int64_t nd = h->n_dof;
    h->f_cells.ensure((size_t)h->n_loc * h->n_cells);
    h->r_glob.ensure(nd);
    DBuf<double> du, ut;
    du.ensure(nd);
    ut.ensure(nd);
    double t0 = now_ms();
    bool neg = false;
    h->pcg_its_total = 0;
    h->inner_its_total = 0;
    run_residual(h, u, h->f_cells.p, h->r_glob.p, nullptr, &neg);
    LAT_REQUIRE(!neg, LAT_ENEG_JACOBIAN, "det F <= 0 at the initial guess");
    double rn = run_norm_free(h, h->r_glob.p);
    double floor = 1e-12 * run_norm_all(h, h->r_glob.p);
    R.t_residual_ms += now_ms() - t0;
    R.r0_norm = rn;
    const double r0 = rn;
    const int cap = max_iterations > 0 ? max_iterations : o->newton_max_it;
    int it = 0;
    double eps = o->eps;
    bool slow_prev = false;
    while (!(rn <= o->newton_rtol * r0 || rn <= floor) && it < cap) {
      double ta = now_ms();
      h->snap_kind = o->snapshot;
      select_cells(h, u, eps, o->max_nr, o->force_all != 0);
      double tb = now_ms();
      R.t_select_ms += tb - ta;
      prepare_enriched(h, o, u);
      double tc = now_ms();
      R.t_setup_ms += tc - tb;
      R.n_r_last = h->n_r;
      DBuf<double> rhs, sol;
      rhs.ensure(h->n_krylov);
      sol.ensure(h->n_krylov);
      newton_rhs(h, h->r_glob.p, rhs.p);
      LAT_CUDA(cudaMemsetAsync(sol.p, 0, h->n_krylov * sizeof(double), h->stream));
      double rel = 0;
      R.krylov_its_total += run_fgmres(h, rhs.p, sol.p, o, &rel);
      run_feti_to_global(h, sol.p, du.p);
      double td = now_ms();
      R.t_krylov_ms += td - tc;
      // Armijo backtracking (Section 2.2.5)
      bool accepted = false;
      double step = 1.0, rt = 0;
      int mm = 0;
      for (; mm <= o->armijo_max_m; ++mm, step *= 0.5) {
        LAT_CUDA(cudaMemcpyAsync(ut.p, u, nd * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        run_axpy(h, nd, step, du.p, ut.p);
        bool ng = false;
        run_residual(h, ut.p, h->f_cells.p, h->r_glob.p, nullptr, &ng);
        if (ng) continue;
        rt = run_norm_free(h, h->r_glob.p);
        if (rt <= (1.0 - 1e-4 * step) * rn) {
          accepted = true;
          break;
        }
      }
      R.t_linesearch_ms += now_ms() - td;
      R.armijo_m_max = std::max(R.armijo_m_max, mm);
      if (h->verbose)
        std::fprintf(stderr, "[lattice] newton it %d |r|=%.3e rel=%.3e eps=%.1e N_r=%d keys=%d enrich=%d indef=%d/%d krylov=%d inner=%lld pcg=%lld (rel %.1e) m=%d%s\n",
                     it, rn, rn / r0, eps, h->n_r, h->n_keys, h->enrich_level, (int)h->indefinite, (int)h->coarse_indefinite,
                     R.krylov_its_total, (long long)h->inner_its_total, (long long)h->pcg_its_total, rel, mm,
                     accepted ? "" : " REJECTED");
      if (!accepted) {
        // leave u and the residual buffers consistent with u
        run_residual(h, u, h->f_cells.p, h->r_glob.p, nullptr, &neg);
        if (!o->force_all && R.eps_refinements < o->eps_refine) {
          // the reduced tangent is too coarse for a descent direction here: the same iterate
          // again with a tenfold tighter reduced-basis tolerance (more principal cells)
          ++R.eps_refinements;
          eps *= 0.1;
          slow_prev = false;
          continue;
        }
        R.r_norm = rn;
        R.eps_last = eps;
        R.iterations = it;
        throw LatError{LAT_ENOT_CONVERGED, "Armijo line search found no acceptable step"};
      }
      LAT_CUDA(cudaMemcpyAsync(u, ut.p, nd * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
      // two accepted steps in a row that reduce the residual by less than eps_refine_rate: the
      // reduced tangent limits the (linear) convergence, so the next iteration selects with a
      // tenfold tighter tolerance (one slow step alone may be the nonlinearity far from the
      // solution, which a finer tangent would not help)
      const bool slow = rt > o->eps_refine_rate * rn;
      if (!o->force_all && slow && slow_prev && R.eps_refinements < o->eps_refine) {
        ++R.eps_refinements;
        eps *= 0.1;
        slow_prev = false;
      } else {
        slow_prev = slow;
      }
      rn = rt;
      floor = 1e-12 * run_norm_all(h, h->r_glob.p);
      ++it;
      rhs.release();
      sol.release();
    }
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    R.iterations = it;
    R.r_norm = rn;
    R.pcg_its_total = (int32_t)h->pcg_its_total;
    R.inner_its_total = (int32_t)h->inner_its_total;
    R.enrich_level = h->enrich_level;
    R.eps_last = eps;
    R.converged = (rn <= o->newton_rtol * r0 || rn <= floor) ? 1 : 0;
    du.release();
    ut.release();
  });
  if (rep) *rep = R;
  return st;
}

extern "C" lat_status lattice_prepare_solver(lat_handle h, const double* u, const lat_newton_opts* o) {
  if (!h || !u) return LAT_EINVAL;
  return guard(h, [&] {
    check_opts(o);
    prepare_enriched(h, o, u);
  });
}

extern "C" lat_status tangent_solve(lat_handle h, const double* rhs, double* x, const lat_newton_opts* o,
                                    int32_t* iters, double* rel) {
  if (!h || !rhs || !x) return LAT_EINVAL;
  return guard(h, [&] {
    check_opts(o);
    LAT_REQUIRE(h->n_keys > 0, LAT_EINVAL, "call lattice_prepare_solver first");
    DBuf<double> b, sol;
    b.ensure(h->n_krylov);
    sol.ensure(h->n_krylov);
    run_feti_from_global(h, rhs, b.p, true);
    LAT_CUDA(cudaMemsetAsync(sol.p, 0, h->n_krylov * sizeof(double), h->stream));
    double r = 0;
    const int it = run_fgmres(h, b.p, sol.p, o, &r);
    run_feti_to_global(h, sol.p, x);
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    if (iters) *iters = it;
    if (rel) *rel = r;
  });
}

extern "C" lat_status feti_apply(lat_handle h, int32_t mode, const double* v, double* w) {
  if (!h || !v || !w) return LAT_EINVAL;
  return guard(h, [&] {
    LAT_REQUIRE(h->n_keys > 0, LAT_EINVAL, "call lattice_prepare_solver first");
    if (mode == 0) run_feti_operator(h, v, w);
    else if (mode == 1) run_kinv(h, v, w);
    else if (mode == 2) run_block_precond(h, v, w, 5, 0.0);
    else throw LatError{LAT_EINVAL, "mode must be 0, 1 or 2"};
    LAT_CUDA(cudaStreamSynchronize(h->stream));
  });
}

extern "C" lat_status feti_to_global(lat_handle h, const double* v, double* u) {
  if (!h || !v || !u) return LAT_EINVAL;
  return guard(h, [&] { run_feti_to_global(h, v, u); });
}

extern "C" lat_status feti_from_global(lat_handle h, const double* u, double* v) {
  if (!h || !v || !u) return LAT_EINVAL;
  return guard(h, [&] { run_feti_from_global(h, u, v, false); });
}

extern "C" lat_status adjoint_gradient(lat_handle h, const double* u, const lat_newton_opts* o, double* grad,
                                       double* J, lat_newton_report* rep) {
  if (!h || !u || !grad) return LAT_EINVAL;
  lat_newton_report R{};
  lat_status st = guard(h, [&] {
    check_opts(o);
    const int64_t nd = h->n_dof;
    h->f_cells.ensure((size_t)h->n_loc * h->n_cells);
    h->r_glob.ensure(nd);
    bool neg = false;
    run_residual(h, u, h->f_cells.p, h->r_glob.p, nullptr, &neg);
    LAT_REQUIRE(!neg, LAT_ENEG_JACOBIAN, "det F <= 0 at the adjoint state");
    if (J) *J = run_dot_fixed(h, u, h->r_glob.p);
    DBuf<double> vD, bF, lam, d, y, rhs, sol, del;
    for (auto* p : {&vD, &bF, &lam, &d, &y, &del}) p->ensure(nd);
    rhs.ensure(h->n_krylov);
    sol.ensure(h->n_krylov);
    // v_D = u on the Dirichlet DOFs, 0 elsewhere;  b_F = (K v_D)_F = K_FD u_D
    run_mask(h, u, vD.p, 1);
    run_tangent_apply_exact(h, u, vD.p, y.p);
    run_mask(h, y.p, bF.p, 0);
    const double bnorm = run_norm_free(h, bF.p);
    LAT_CUDA(cudaMemsetAsync(lam.p, 0, nd * sizeof(double), h->stream));
    LAT_CUDA(cudaMemcpyAsync(d.p, bF.p, nd * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    h->snap_kind = o->snapshot;
    double eps = o->eps;
    select_cells(h, u, eps, o->max_nr, o->force_all != 0);
    prepare_enriched(h, o, u);
    double dn = bnorm;
    R.r0_norm = bnorm;
    int it = 0;
    const double tol = std::max(o->newton_rtol * 1e-2, 1e-12);
    while (bnorm > 0 && dn > tol * bnorm && it < o->newton_max_it) {
      run_feti_from_global(h, d.p, rhs.p, true);
      LAT_CUDA(cudaMemsetAsync(sol.p, 0, h->n_krylov * sizeof(double), h->stream));
      double rel = 0;
      R.krylov_its_total += run_fgmres(h, rhs.p, sol.p, o, &rel);
      run_feti_to_global(h, sol.p, del.p);
      run_axpy(h, nd, 1.0, del.p, lam.p);
      // defect d = b_F - (K lambda)_F with the exact tangent action
      run_tangent_apply_exact(h, u, lam.p, y.p);
      LAT_CUDA(cudaMemcpyAsync(d.p, bF.p, nd * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
      run_axpy(h, nd, -1.0, y.p, d.p);
      run_mask(h, d.p, d.p, 0);
      const double prev = dn;
      dn = run_norm_free(h, d.p);
      ++it;
      // the correction contracts the defect by || I - K~^{-1} K || (a linear iteration): above
      // eps_refine_rate the reduced tangent is too coarse, and the selection is redone with a
      // tenfold tighter tolerance
      if (!o->force_all && dn > o->eps_refine_rate * prev && R.eps_refinements < o->eps_refine &&
          dn > tol * bnorm) {
        ++R.eps_refinements;
        eps *= 0.1;
        select_cells(h, u, eps, o->max_nr, false);
        prepare_enriched(h, o, u);
      }
    }
    R.n_r_last = h->n_r;
    R.eps_last = eps;
    R.iterations = it;
    R.r_norm = dn;
    R.converged = (bnorm == 0 || dn <= tol * bnorm) ? 1 : 0;
    // w = -lambda on free DOFs, u_D on Dirichlet DOFs
    run_adjoint_w(h, lam.p, u, y.p);
    run_grad_mu(h, u, y.p, grad);
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    for (auto* p : {&vD, &bF, &lam, &d, &y, &rhs, &sol, &del}) p->release();
    LAT_REQUIRE(R.converged, LAT_ENOT_CONVERGED, "adjoint defect correction did not converge");
  });
  if (rep) *rep = R;
  return st;
}

// --- small helpers used above ----------------------------------------------------------------
namespace {
__global__ void k_f2d(int64_t n, const float* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}
__global__ void k_mask(int64_t n, const double* __restrict__ x, const uint8_t* __restrict__ fixed, int keep_fixed,
                       double* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = ((fixed[i] != 0) == (keep_fixed != 0)) ? x[i] : 0.0;
}
__global__ void k_adj_w(int64_t n, const double* __restrict__ lam, const double* __restrict__ u,
                        const uint8_t* __restrict__ fixed, double* __restrict__ w) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) w[i] = fixed[i] ? u[i] : -lam[i];
}
}  // namespace

void run_f2d(lat_ctx* h, int64_t n, const float* x, double* y) {
  LAT_LAUNCH(h, k_f2d<<<ew_blocks(h, n), 256, 0, h->stream>>>(n, x, y));
  LAT_CHECK_LAUNCH();
}
void run_mask(lat_ctx* h, const double* x, double* y, int keep_fixed) {
  LAT_LAUNCH(h, k_mask<<<div_up(h->n_dof, 256), 256, 0, h->stream>>>(h->n_dof, x, h->dof_fixed.p, keep_fixed, y));
  LAT_CHECK_LAUNCH();
}
void run_adjoint_w(lat_ctx* h, const double* lam, const double* u, double* w) {
  LAT_LAUNCH(h, k_adj_w<<<div_up(h->n_dof, 256), 256, 0, h->stream>>>(h->n_dof, lam, u, h->dof_fixed.p, w));
  LAT_CHECK_LAUNCH();
}
