// Per-cell residual and tangent evaluation at quadrature points, the matrix-free exact tangent
// action, the mu-derivative of the internal force, the local-to-global scatter and FP64 norms.
//
// One CTA per cell.  The cell's displacements are gathered into shared memory through the
// Boolean map A^s (Eq. residualvector); elements are processed colour by colour so that the
// element contributions of one colour never touch the same local node, which makes the
// accumulation race free without atomics and deterministic.
//
// Kinematics and stress use the first Piola-Kirchhoff form of the neo-Hookean law of
// Eq. (sig_eq): with F = I + sum_a u_a (x) grad_X phi_a (Section 3.1.3), J = det F,
//   P = J sigma F^{-T} = mu (F - F^{-T}) + lam ln J F^{-T},
//   f_a = sum_q W_q P grad_X phi_a                 (Eq. internalloadvec pulled back, dx = J dX)
// and the tangent of Section 3.1.4 pulled back to the reference cell (Eq. stiffmatPulledback):
//   K_ab = sum_q W_q [ mu (g_a . g_b) I + lam h_a h_b^T + (mu - lam ln J) h_b h_a^T ],
//   g = grad_X phi, h = F^{-T} g = grad_x phi,
// which equals the contraction of D_ijkl = C_ikjl + delta_ij sigma_kl (Eq. const_eq) with
// grad_x phi_a (x) grad_x phi_b times J.
#include <cfloat>

#include "common.cuh"

namespace {

constexpr int kCellThreads = 256;

struct GeomArgs {
  const double* gradX;   // [n_el][nq][nen][D]
  const double* W;       // [n_el][nq]
  const int* elems;      // [n_el][nen]
  const int* color_elems;
  int nq;
};

__device__ __forceinline__ void load_cell_u(const double* __restrict__ u_glob,
                                            const int* __restrict__ cnodes, int nn, int D,
                                            double* __restrict__ u_loc) {
  for (int k = threadIdx.x; k < nn * D; k += blockDim.x) {
    int a = k / D, i = k - a * D;
    u_loc[k] = u_glob[(int64_t)cnodes[a] * D + i];
  }
}

// ---------------------------------------------------------------------------------------------
// residual: f^{int,s} for every cell, cell-stacked output [n_loc][n_cells]
// ---------------------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(kCellThreads)
    k_residual(int n_cells, int nn, GeomArgs g, ColorTable ct, const int* __restrict__ cell_nodes,
               const double* __restrict__ mu_cell, double mu_override, double lam,
               const double* __restrict__ u_glob, double* __restrict__ f_cells,
               double* __restrict__ minJ_cell) {
  constexpr int NEN = 1 << D;
  extern __shared__ double sm[];
  double* u_loc = sm;
  double* f_loc = sm + nn * D;
  __shared__ double red[32];
  const int s = blockIdx.x;
  load_cell_u(u_glob, cell_nodes + (size_t)s * nn, nn, D, u_loc);
  for (int k = threadIdx.x; k < nn * D; k += blockDim.x) f_loc[k] = 0.0;
  __syncthreads();
  const double mu = mu_override >= 0 ? mu_override : mu_cell[s];
  double minJ = DBL_MAX;
  for (int c = 0; c < ct.n; ++c) {
    for (int t = ct.start[c] + threadIdx.x; t < ct.start[c + 1]; t += blockDim.x) {
      const int e = g.color_elems[t];
      int nd[NEN];
      double ue[NEN][D], fe[NEN][D];
#pragma unroll
      for (int a = 0; a < NEN; ++a) {
        nd[a] = g.elems[e * NEN + a];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          ue[a][i] = u_loc[nd[a] * D + i];
          fe[a][i] = 0.0;
        }
      }
      for (int q = 0; q < g.nq; ++q) {
        const double* gq = g.gradX + ((size_t)(e * g.nq + q) * NEN) * D;
        double gr[NEN][D];
#pragma unroll
        for (int a = 0; a < NEN; ++a)
#pragma unroll
          for (int k = 0; k < D; ++k) gr[a][k] = gq[a * D + k];
        double F[D][D], Fi[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
          for (int k = 0; k < D; ++k) {
            double v = (i == k) ? 1.0 : 0.0;
#pragma unroll
            for (int a = 0; a < NEN; ++a) v += ue[a][i] * gr[a][k];
            F[i][k] = v;
          }
        const double J = det_inv<D>(F, Fi);
        minJ = fmin(minJ, J);
        const double lnJ = J > 0 ? log(J) : 0.0;
        const double w = g.W[e * g.nq + q];
        double P[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
          for (int k = 0; k < D; ++k) P[i][k] = w * (mu * (F[i][k] - Fi[k][i]) + lam * lnJ * Fi[k][i]);
#pragma unroll
        for (int a = 0; a < NEN; ++a)
#pragma unroll
          for (int i = 0; i < D; ++i) {
            double v = 0;
#pragma unroll
            for (int k = 0; k < D; ++k) v += P[i][k] * gr[a][k];
            fe[a][i] += v;
          }
      }
#pragma unroll
      for (int a = 0; a < NEN; ++a)
#pragma unroll
        for (int i = 0; i < D; ++i) f_loc[nd[a] * D + i] += fe[a][i];
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < nn * D; k += blockDim.x) f_cells[(size_t)k * n_cells + s] = f_loc[k];
  minJ = -block_max(-minJ, red);
  if (threadIdx.x == 0 && minJ_cell) minJ_cell[s] = minJ;
}

// ---------------------------------------------------------------------------------------------
// tangent: K^s on the shared pattern for a list of cells, [n_sel][nnz], K_out zeroed first
// one thread per (element of the colour, local node a): the d x (2^d d) row block of K_e
// ---------------------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(kCellThreads)
    k_tangent(int nn, GeomArgs g, ColorTable ct, const int* __restrict__ cell_nodes,
              const int* __restrict__ cells, const int* __restrict__ elem_blk,
              const double* __restrict__ mu_cell, double lam, const double* __restrict__ u_glob,
              int64_t nnz, double* __restrict__ K_out, double* __restrict__ minJ_out, int geo) {
  constexpr int NEN = 1 << D;
  extern __shared__ double sm[];
  double* u_loc = sm;
  __shared__ double red[32];
  const int si = blockIdx.x;
  const int s = cells ? cells[si] : si;
  load_cell_u(u_glob, cell_nodes + (size_t)s * nn, nn, D, u_loc);
  __syncthreads();
  const double mu = mu_cell[s];
  double* K = K_out + (size_t)si * nnz;
  double minJ = DBL_MAX;
  for (int c = 0; c < ct.n; ++c) {
    const int n_t = (ct.start[c + 1] - ct.start[c]) * NEN;
    for (int t = threadIdx.x; t < n_t; t += blockDim.x) {
      const int e = g.color_elems[ct.start[c] + t / NEN];
      const int a = t % NEN;
      int nd[NEN];
#pragma unroll
      for (int b = 0; b < NEN; ++b) nd[b] = g.elems[e * NEN + b];
      double acc[NEN][D][D];
#pragma unroll
      for (int b = 0; b < NEN; ++b)
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
          for (int j = 0; j < D; ++j) acc[b][i][j] = 0.0;
      for (int q = 0; q < g.nq; ++q) {
        const double* gq = g.gradX + ((size_t)(e * g.nq + q) * NEN) * D;
        double F[D][D], Fi[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
          for (int k = 0; k < D; ++k) F[i][k] = (i == k) ? 1.0 : 0.0;
#pragma unroll
        for (int b = 0; b < NEN; ++b)
#pragma unroll
          for (int i = 0; i < D; ++i) {
            const double ub = u_loc[nd[b] * D + i];
#pragma unroll
            for (int k = 0; k < D; ++k) F[i][k] += ub * gq[b * D + k];
          }
        const double J = det_inv<D>(F, Fi);
        minJ = fmin(minJ, J);
        const double lnJ = J > 0 ? log(J) : 0.0;
        const double w = g.W[e * g.nq + q];
        const double cm = w * mu, cl = w * lam, cg = w * (mu - lam * lnJ);
        double ga[D], ha[D];
#pragma unroll
        for (int k = 0; k < D; ++k) ga[k] = gq[a * D + k];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          double v = 0;
#pragma unroll
          for (int k = 0; k < D; ++k) v += Fi[k][i] * ga[k];
          ha[i] = v;
        }
#pragma unroll
        for (int b = 0; b < NEN; ++b) {
          double gb[D], hb[D], gab = 0, hab = 0;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            gb[k] = gq[b * D + k];
            gab += ga[k] * gb[k];
          }
#pragma unroll
          for (int i = 0; i < D; ++i) {
            double v = 0;
#pragma unroll
            for (int k = 0; k < D; ++k) v += Fi[k][i] * gb[k];
            hb[i] = v;
            hab += ha[i] * v;
          }
          // diagonal term: mu g_a.g_b holds the geometric part delta_ij J h_a^T sigma h_b =
          // mu (g_a.g_b - h_a.h_b) + lam ln J h_a.h_b; without it (geo = 0) what remains is the
          // material part, the contraction of C_ikjl alone: (mu - lam ln J) h_a.h_b
          const double dg = geo ? cm * gab : cg * hab;
#pragma unroll
          for (int i = 0; i < D; ++i)
#pragma unroll
            for (int j = 0; j < D; ++j)
              acc[b][i][j] += (i == j ? dg : 0.0) + cl * ha[i] * hb[j] + cg * hb[i] * ha[j];
        }
      }
      const int* eb = elem_blk + (e * NEN + a) * NEN;
#pragma unroll
      for (int b = 0; b < NEN; ++b) {
        double* Kb = K + (size_t)eb[b] * D * D;
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
          for (int j = 0; j < D; ++j) Kb[i * D + j] += acc[b][i][j];
      }
    }
    __syncthreads();
  }
  if (minJ_out) {
    minJ = -block_max(-minJ, red);
    if (threadIdx.x == 0) minJ_out[si] = minJ;
  }
}

// ---------------------------------------------------------------------------------------------
// D^ref snapshots (the Remark after Eq. snapshots): the pulled-back tangent tensor of Eq.
// (tensorfunctionPulledback) at the one-point rule of every element,
//   D^ref_ijmn = |det J| sum_kl D_ijkl G_mk G_nl,   G = J^{-1}, J = dx/dxi = F J0,
//   D_ijkl = C_ikjl + delta_ij sigma_kl  (Eq. const_eq, Section 3.1.4), which expands to
//   D^ref_ijmn = |det J| [lam/J G_mi G_nj + c (delta_ij (G G^T)_mn + G_mj G_ni)
//                         + delta_ij (G sigma G^T)_mn],   c = (mu - lam ln J) / J.
// J0^{-1} follows from the reference gradients at the centre: the Q1 corner signs xi_a satisfy
// sum_a xi_a,m xi_a,m' = 2^d delta, so (J0^{-1})_mk = sum_a xi_a,m dphi_a/dX_k.  A thread per
// (cell, element); output [n_cells][n_el * d^4], entries (element, i, j, m, n) last fastest.
// ---------------------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(128)
    k_dref(int n_cells, int n_el, int nn, GeomArgs g, const int* __restrict__ cell_nodes,
           const double* __restrict__ mu_cell, double lam, const double* __restrict__ u_glob,
           double* __restrict__ T, double* __restrict__ minJ_cell) {
  constexpr int NEN = 1 << D;
  constexpr int D4 = D * D * D * D;
  const int s = blockIdx.y;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  __shared__ double red[32];
  double myJ = DBL_MAX;
  if (e < n_el) {
    const int* cn = cell_nodes + (size_t)s * nn;
    const double* gq = g.gradX + (size_t)e * NEN * D;   // one point per element
    double F[D][D], Fi[D][D], Ji0[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int k = 0; k < D; ++k) {
        F[i][k] = (i == k) ? 1.0 : 0.0;
        Ji0[i][k] = 0.0;
      }
#pragma unroll
    for (int a = 0; a < NEN; ++a) {
      const int node = g.elems[e * NEN + a];
      const int64_t gn = cn[node];
      // Q1 corner a in the counter-clockwise / bottom-then-top order: signs of xi_a
      const double sx = ((a & 3) == 1 || (a & 3) == 2) ? 1.0 : -1.0;
      const double sy = ((a & 3) >= 2) ? 1.0 : -1.0;
      const double sz = a >= 4 ? 1.0 : -1.0;
      const double sg[3] = {sx, sy, sz};
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const double ui = u_glob[gn * D + i];
#pragma unroll
        for (int k = 0; k < D; ++k) F[i][k] += ui * gq[a * D + k];
      }
#pragma unroll
      for (int m = 0; m < D; ++m)
#pragma unroll
        for (int k = 0; k < D; ++k) Ji0[m][k] += sg[m] * gq[a * D + k];
    }
    const double J = det_inv<D>(F, Fi);
    myJ = J;
    const double lnJ = J > 0 ? log(J) : 0.0;
    const double mu = mu_cell[s];
    const double detJ0 = g.W[e] / (double)(1 << D);         // one-point weight 2^d |det J0|
    const double dJ = fabs(J) * detJ0;
    double G[D][D];                                         // J^{-1} = J0^{-1} F^{-1}
#pragma unroll
    for (int m = 0; m < D; ++m)
#pragma unroll
      for (int k = 0; k < D; ++k) {
        double v = 0;
#pragma unroll
        for (int p = 0; p < D; ++p) v += Ji0[m][p] * Fi[p][k];
        G[m][k] = v;
      }
    double sig[D][D];                                       // Eq. (sig_eq)
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
      for (int l = 0; l < D; ++l) {
        double b = 0;
#pragma unroll
        for (int p = 0; p < D; ++p) b += F[k][p] * F[l][p];
        sig[k][l] = mu / J * (b - (k == l ? 1.0 : 0.0)) + (k == l ? lam * lnJ / J : 0.0);
      }
    double A[D][D], Sg[D][D];
#pragma unroll
    for (int m = 0; m < D; ++m)
#pragma unroll
      for (int n = 0; n < D; ++n) {
        double a1 = 0, a2 = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          a1 += G[m][k] * G[n][k];
          double t = 0;
#pragma unroll
          for (int l = 0; l < D; ++l) t += sig[k][l] * G[n][l];
          a2 += G[m][k] * t;
        }
        A[m][n] = a1;
        Sg[m][n] = a2;
      }
    const double cl = lam / J, cc = (mu - lam * lnJ) / J;
    double* out = T + (size_t)s * n_el * D4 + (size_t)e * D4;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j)
#pragma unroll
        for (int m = 0; m < D; ++m)
#pragma unroll
          for (int n = 0; n < D; ++n) {
            double v = cl * G[m][i] * G[n][j] + cc * G[m][j] * G[n][i];
            if (i == j) v += cc * A[m][n] + Sg[m][n];
            out[((i * D + j) * D + m) * D + n] = dJ * v;
          }
  }
  const double mj = -block_max(-myJ, red);
  if (threadIdx.x == 0 && minJ_cell) {
    // the CTAs of a cell combine through an atomic-free per-(cell, CTA) slot
    minJ_cell[(size_t)s * gridDim.x + blockIdx.x] = mj;
  }
}

// ---------------------------------------------------------------------------------------------
// exact tangent action y = K(u) v without storing K (matrix free, full rule):
//   dP_iK = mu dF_iK + lam tr(F^{-1} dF) F^{-1}_Ki + (mu - lam ln J) (F^{-1} dF F^{-1})_Ki
// output cell-stacked local forces [n_loc][n_cells]
// ---------------------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(kCellThreads)
    k_tangent_apply(int n_cells, int nn, GeomArgs g, ColorTable ct, const int* __restrict__ cell_nodes,
                    const double* __restrict__ mu_cell, double lam, const double* __restrict__ u_glob,
                    const double* __restrict__ v_glob, double* __restrict__ y_cells) {
  constexpr int NEN = 1 << D;
  extern __shared__ double sm[];
  double* u_loc = sm;
  double* v_loc = sm + nn * D;
  double* y_loc = sm + 2 * nn * D;
  const int s = blockIdx.x;
  load_cell_u(u_glob, cell_nodes + (size_t)s * nn, nn, D, u_loc);
  load_cell_u(v_glob, cell_nodes + (size_t)s * nn, nn, D, v_loc);
  for (int k = threadIdx.x; k < nn * D; k += blockDim.x) y_loc[k] = 0.0;
  __syncthreads();
  const double mu = mu_cell[s];
  for (int c = 0; c < ct.n; ++c) {
    for (int t = ct.start[c] + threadIdx.x; t < ct.start[c + 1]; t += blockDim.x) {
      const int e = g.color_elems[t];
      int nd[NEN];
      double ye[NEN][D];
#pragma unroll
      for (int a = 0; a < NEN; ++a) {
        nd[a] = g.elems[e * NEN + a];
#pragma unroll
        for (int i = 0; i < D; ++i) ye[a][i] = 0.0;
      }
      for (int q = 0; q < g.nq; ++q) {
        const double* gq = g.gradX + ((size_t)(e * g.nq + q) * NEN) * D;
        double F[D][D], dF[D][D], Fi[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
          for (int k = 0; k < D; ++k) {
            double f = (i == k) ? 1.0 : 0.0, df = 0.0;
#pragma unroll
            for (int a = 0; a < NEN; ++a) {
              f += u_loc[nd[a] * D + i] * gq[a * D + k];
              df += v_loc[nd[a] * D + i] * gq[a * D + k];
            }
            F[i][k] = f;
            dF[i][k] = df;
          }
        const double J = det_inv<D>(F, Fi);
        const double lnJ = J > 0 ? log(J) : 0.0;
        const double w = g.W[e * g.nq + q];
        double tr = 0, FdF[D][D];
#pragma unroll
        for (int K = 0; K < D; ++K)
#pragma unroll
          for (int L = 0; L < D; ++L) {
            double v = 0;
#pragma unroll
            for (int j = 0; j < D; ++j) v += Fi[K][j] * dF[j][L];
            FdF[K][L] = v;   // (F^{-1} dF)_KL
          }
#pragma unroll
        for (int K = 0; K < D; ++K) tr += FdF[K][K];
        double dP[D][D];
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
          for (int K = 0; K < D; ++K) {
            double m = 0;
#pragma unroll
            for (int L = 0; L < D; ++L) m += FdF[K][L] * Fi[L][i];
            dP[i][K] = w * (mu * dF[i][K] + lam * tr * Fi[K][i] + (mu - lam * lnJ) * m);
          }
#pragma unroll
        for (int a = 0; a < NEN; ++a)
#pragma unroll
          for (int i = 0; i < D; ++i) {
            double v = 0;
#pragma unroll
            for (int K = 0; K < D; ++K) v += dP[i][K] * gq[a * D + K];
            ye[a][i] += v;
          }
      }
#pragma unroll
      for (int a = 0; a < NEN; ++a)
#pragma unroll
        for (int i = 0; i < D; ++i) y_loc[nd[a] * D + i] += ye[a][i];
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < nn * D; k += blockDim.x) y_cells[(size_t)k * n_cells + s] = y_loc[k];
}

// r[g] = sum over the copies of global node g of the cell-stacked local values
__global__ void k_scatter(int64_t n_nodes, int dim, int nn, int n_cells, const int* __restrict__ cptr,
                          const int* __restrict__ cidx, const double* __restrict__ f_cells,
                          double* __restrict__ r) {
  int64_t gnode = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gnode >= n_nodes) return;
  for (int i = 0; i < dim; ++i) {
    double v = 0;
    for (int c = cptr[gnode]; c < cptr[gnode + 1]; ++c) {
      int sa = cidx[c];
      int s = sa / nn, a = sa - s * nn;
      v += f_cells[(size_t)(a * dim + i) * n_cells + s];
    }
    r[gnode * dim + i] = v;
  }
}

// grad[s] = sum_k w_loc[k,s] * f_mu[k,s] (cell-stacked inputs)
__global__ void k_cell_dot(int n_cells, int n_loc, const double* __restrict__ w_glob,
                           const int* __restrict__ cell_nodes, int nn, int dim,
                           const double* __restrict__ f_cells, double* __restrict__ out) {
  __shared__ double red[32];
  const int s = blockIdx.x;
  double v = 0;
  for (int k = threadIdx.x; k < n_loc; k += blockDim.x) {
    int a = k / dim, i = k - a * dim;
    v += w_glob[(int64_t)cell_nodes[(size_t)s * nn + a] * dim + i] * f_cells[(size_t)k * n_cells + s];
  }
  v = block_sum(v, red);
  if (threadIdx.x == 0) out[s] = v;
}

// deterministic two-stage reductions over global vectors
constexpr int kRedBlocks = 512;

__global__ void k_sumsq_masked(int64_t n, const double* __restrict__ x, const uint8_t* __restrict__ fixed,
                               int want_fixed, double* __restrict__ part) {
  __shared__ double red[32];
  double v = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if ((fixed[i] != 0) == (want_fixed != 0)) v += x[i] * x[i];
  v = block_sum(v, red);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

__global__ void k_dot_masked(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                             const uint8_t* __restrict__ fixed, double* __restrict__ part) {
  __shared__ double red[32];
  double v = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (fixed[i]) v += a[i] * b[i];
  v = block_sum(v, red);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
}

__global__ void k_final_sum(int n, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double red[32];
  double v = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
  v = block_sum(v, red);
  if (threadIdx.x == 0) out[0] = v;
}

__global__ void k_min_reduce(int n, const double* __restrict__ x, double* __restrict__ out) {
  __shared__ double red[32];
  double v = DBL_MAX;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v = fmin(v, x[i]);
  v = -block_max(-v, red);
  if (threadIdx.x == 0) out[0] = v;
}

ColorTable colors(lat_ctx* h) {
  ColorTable ct;
  ct.n = (int)h->color_start.size() - 1;
  LAT_REQUIRE(ct.n <= 32, LAT_EINVAL, "too many element colours");
  for (int c = 0; c <= ct.n; ++c) ct.start[c] = h->color_start[c];
  return ct;
}

GeomArgs geom(lat_ctx* h, int quad) {
  return GeomArgs{h->gradX[quad].p, h->W[quad].p, h->elems.p, h->color_elems.p, h->nq[quad]};
}

double* scratch_scalars(lat_ctx* h) {
  h->red_part.ensure(4096);
  return h->red_part.p;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------
void run_residual(lat_ctx* h, const double* u_glob, double* f_cells, double* r_glob,
                  double* min_detF_host, bool* negJ) {
  const size_t shm = 2 * (size_t)h->n_loc * sizeof(double);
  h->minJ_cell.ensure(h->n_cells);
  auto g = geom(h, 0);
  auto ct = colors(h);
  KernelTimer kt(h, "residual");
  if (h->dim == 2) {
    LAT_LAUNCH(h, k_residual<2><<<h->n_cells, kCellThreads, shm, h->stream>>>(h->n_cells, h->n_nodes_cell, g, ct,
        h->cell_nodes.p, h->mu_cell.p, -1.0, h->lam, u_glob, f_cells, h->minJ_cell.p));
  } else {
    LAT_CUDA(cudaFuncSetAttribute(k_residual<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    LAT_LAUNCH(h, k_residual<3><<<h->n_cells, kCellThreads, shm, h->stream>>>(h->n_cells, h->n_nodes_cell, g, ct,
        h->cell_nodes.p, h->mu_cell.p, -1.0, h->lam, u_glob, f_cells, h->minJ_cell.p));
  }
  LAT_CHECK_LAUNCH();
  if (r_glob) {
    LAT_LAUNCH(h, k_scatter<<<div_up(h->n_glob_nodes, 256), 256, 0, h->stream>>>(h->n_glob_nodes, h->dim,
        h->n_nodes_cell, h->n_cells, h->copy_ptr.p, h->copy_idx.p, f_cells, r_glob));
    LAT_CHECK_LAUNCH();
  }
  double* sc = scratch_scalars(h);
  LAT_LAUNCH(h, k_min_reduce<<<1, 1024, 0, h->stream>>>(h->n_cells, h->minJ_cell.p, sc));
  LAT_CHECK_LAUNCH();
  LAT_CUDA(cudaMemcpyAsync(h->h_pinned, sc, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LAT_CUDA(cudaStreamSynchronize(h->stream));
  if (min_detF_host) *min_detF_host = h->h_pinned[0];
  if (negJ) *negJ = !(h->h_pinned[0] > 0.0);
}

void run_tangent(lat_ctx* h, const double* u_glob, int quad, const int* cells, int n_sel,
                 double* K_out, bool* negJ, bool geometric) {
  if (n_sel <= 0) return;
  LAT_CUDA(cudaMemsetAsync(K_out, 0, (size_t)n_sel * h->nnz * sizeof(double), h->stream));
  const size_t shm = (size_t)h->n_loc * sizeof(double);
  h->minJ_cell.ensure(std::max(h->n_cells, n_sel));
  auto g = geom(h, quad);
  auto ct = colors(h);
  KernelTimer kt(h, quad ? "tangent_reduced" : (geometric ? "tangent_full" : "tangent_material"));
  if (h->dim == 2) {
    LAT_LAUNCH(h, k_tangent<2><<<n_sel, kCellThreads, shm, h->stream>>>(h->n_nodes_cell, g, ct, h->cell_nodes.p,
        cells, h->elem_blk.p, h->mu_cell.p, h->lam, u_glob, h->nnz, K_out, h->minJ_cell.p, geometric ? 1 : 0));
  } else {
    LAT_CUDA(cudaFuncSetAttribute(k_tangent<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    LAT_LAUNCH(h, k_tangent<3><<<n_sel, kCellThreads, shm, h->stream>>>(h->n_nodes_cell, g, ct, h->cell_nodes.p,
        cells, h->elem_blk.p, h->mu_cell.p, h->lam, u_glob, h->nnz, K_out, h->minJ_cell.p, geometric ? 1 : 0));
  }
  LAT_CHECK_LAUNCH();
  if (negJ) {
    double* sc = scratch_scalars(h);
    LAT_LAUNCH(h, k_min_reduce<<<1, 1024, 0, h->stream>>>(n_sel, h->minJ_cell.p, sc));
    LAT_CHECK_LAUNCH();
    LAT_CUDA(cudaMemcpyAsync(h->h_pinned, sc, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    *negJ = !(h->h_pinned[0] > 0.0);
  }
}

// D^ref snapshots of every cell: T [n_cells][n_el * d^4]
void run_dref_snapshots(lat_ctx* h, const double* u_glob, double* T, bool* negJ) {
  const int nb = div_up(h->n_el, 128);
  h->minJ_cell.ensure((size_t)h->n_cells * nb);
  auto g = geom(h, 1);
  const dim3 grid(nb, h->n_cells);
  KernelTimer kt(h, "dref_snapshots");
  if (h->dim == 2)
    LAT_LAUNCH(h, k_dref<2><<<grid, 128, 0, h->stream>>>(h->n_cells, h->n_el, h->n_nodes_cell, g, h->cell_nodes.p,
                                                          h->mu_cell.p, h->lam, u_glob, T, h->minJ_cell.p));
  else
    LAT_LAUNCH(h, k_dref<3><<<grid, 128, 0, h->stream>>>(h->n_cells, h->n_el, h->n_nodes_cell, g, h->cell_nodes.p,
                                                          h->mu_cell.p, h->lam, u_glob, T, h->minJ_cell.p));
  LAT_CHECK_LAUNCH();
  if (negJ) {
    double* sc = scratch_scalars(h);
    LAT_LAUNCH(h, k_min_reduce<<<1, 1024, 0, h->stream>>>((int)((int64_t)h->n_cells * nb), h->minJ_cell.p, sc));
    LAT_CHECK_LAUNCH();
    LAT_CUDA(cudaMemcpyAsync(h->h_pinned, sc, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    *negJ = !(h->h_pinned[0] > 0.0);
  }
}

void run_tangent_apply_exact(lat_ctx* h, const double* u_glob, const double* v_glob, double* y_glob) {
  h->f_cells.ensure((size_t)h->n_loc * h->n_cells);
  const size_t shm = 3 * (size_t)h->n_loc * sizeof(double);
  auto g = geom(h, 0);
  auto ct = colors(h);
  if (h->dim == 2) {
    LAT_LAUNCH(h, k_tangent_apply<2><<<h->n_cells, kCellThreads, shm, h->stream>>>(h->n_cells, h->n_nodes_cell, g,
        ct, h->cell_nodes.p, h->mu_cell.p, h->lam, u_glob, v_glob, h->f_cells.p));
  } else {
    LAT_CUDA(cudaFuncSetAttribute(k_tangent_apply<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    LAT_LAUNCH(h, k_tangent_apply<3><<<h->n_cells, kCellThreads, shm, h->stream>>>(h->n_cells, h->n_nodes_cell, g,
        ct, h->cell_nodes.p, h->mu_cell.p, h->lam, u_glob, v_glob, h->f_cells.p));
  }
  LAT_CHECK_LAUNCH();
  LAT_LAUNCH(h, k_scatter<<<div_up(h->n_glob_nodes, 256), 256, 0, h->stream>>>(h->n_glob_nodes, h->dim,
      h->n_nodes_cell, h->n_cells, h->copy_ptr.p, h->copy_idx.p, h->f_cells.p, y_glob));
  LAT_CHECK_LAUNCH();
}

// grad[s] = w^{sT} f_mu^s(u^s): internal force with mu -> base mu, lam -> 0 (d f / d theta_s)
void run_grad_mu(lat_ctx* h, const double* u_glob, const double* w_glob, double* grad) {
  h->f_cells.ensure((size_t)h->n_loc * h->n_cells);
  h->minJ_cell.ensure(h->n_cells);
  const size_t shm = 2 * (size_t)h->n_loc * sizeof(double);
  auto g = geom(h, 0);
  auto ct = colors(h);
  if (h->dim == 2) {
    LAT_LAUNCH(h, k_residual<2><<<h->n_cells, kCellThreads, shm, h->stream>>>(h->n_cells, h->n_nodes_cell, g, ct,
        h->cell_nodes.p, h->mu_cell.p, h->mu, 0.0, u_glob, h->f_cells.p, h->minJ_cell.p));
  } else {
    LAT_CUDA(cudaFuncSetAttribute(k_residual<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    LAT_LAUNCH(h, k_residual<3><<<h->n_cells, kCellThreads, shm, h->stream>>>(h->n_cells, h->n_nodes_cell, g, ct,
        h->cell_nodes.p, h->mu_cell.p, h->mu, 0.0, u_glob, h->f_cells.p, h->minJ_cell.p));
  }
  LAT_CHECK_LAUNCH();
  LAT_LAUNCH(h, k_cell_dot<<<h->n_cells, 256, 0, h->stream>>>(h->n_cells, h->n_loc, w_glob, h->cell_nodes.p,
      h->n_nodes_cell, h->dim, h->f_cells.p, grad));
  LAT_CHECK_LAUNCH();
}

double run_norm_free(lat_ctx* h, const double* r) {
  double* sc = scratch_scalars(h);
  LAT_LAUNCH(h, k_sumsq_masked<<<kRedBlocks, 256, 0, h->stream>>>(h->n_dof, r, h->dof_fixed.p, 0, sc + 16));
  LAT_LAUNCH(h, k_final_sum<<<1, 512, 0, h->stream>>>(kRedBlocks, sc + 16, sc));
  LAT_CHECK_LAUNCH();
  LAT_CUDA(cudaMemcpyAsync(h->h_pinned, sc, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LAT_CUDA(cudaStreamSynchronize(h->stream));
  return std::sqrt(h->h_pinned[0]);
}

double run_norm_all(lat_ctx* h, const double* r) {
  double* sc = scratch_scalars(h);
  LAT_LAUNCH(h, k_sumsq_masked<<<kRedBlocks, 256, 0, h->stream>>>(h->n_dof, r, h->dof_fixed.p, 0, sc + 16));
  LAT_LAUNCH(h, k_sumsq_masked<<<kRedBlocks, 256, 0, h->stream>>>(h->n_dof, r, h->dof_fixed.p, 1, sc + 16 + kRedBlocks));
  LAT_LAUNCH(h, k_final_sum<<<1, 512, 0, h->stream>>>(2 * kRedBlocks, sc + 16, sc));
  LAT_CHECK_LAUNCH();
  LAT_CUDA(cudaMemcpyAsync(h->h_pinned, sc, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LAT_CUDA(cudaStreamSynchronize(h->stream));
  return std::sqrt(h->h_pinned[0]);
}

double run_dot_fixed(lat_ctx* h, const double* a, const double* b) {
  double* sc = scratch_scalars(h);
  LAT_LAUNCH(h, k_dot_masked<<<kRedBlocks, 256, 0, h->stream>>>(h->n_dof, a, b, h->dof_fixed.p, sc + 16));
  LAT_LAUNCH(h, k_final_sum<<<1, 512, 0, h->stream>>>(kRedBlocks, sc + 16, sc));
  LAT_CHECK_LAUNCH();
  LAT_CUDA(cudaMemcpyAsync(h->h_pinned, sc, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LAT_CUDA(cudaStreamSynchronize(h->stream));
  return h->h_pinned[0];
}

// ---------------------------------------------------------------------------------------------
// entry point
// ---------------------------------------------------------------------------------------------
extern "C" lat_status assemble_residual_tangent(lat_handle h, const double* u_glob, int32_t quad,
                                                const int32_t* cells, int32_t n_sel, double* r_glob,
                                                double* f_cells, double* K_vals, double* min_detF) {
  if (!h || !u_glob) return LAT_EINVAL;
  return guard(h, [&] {
    LAT_REQUIRE(quad == 0 || quad == 1, LAT_EINVAL, "quad must be 0 (full) or 1 (reduced)");
    LAT_REQUIRE(n_sel >= 0, LAT_EINVAL, "negative cell count");
    LAT_REQUIRE(cells != nullptr || n_sel == h->n_cells, LAT_EINVAL, "n_sel must equal n_cells when cells is NULL");
    LAT_REQUIRE(!(cells && (r_glob || f_cells)), LAT_EINVAL, "residual outputs need all cells");
    if (cells && n_sel > 0) {
      std::vector<int> hc(n_sel);
      LAT_CUDA(cudaMemcpy(hc.data(), cells, n_sel * sizeof(int), cudaMemcpyDeviceToHost));
      for (int c : hc) LAT_REQUIRE(c >= 0 && c < h->n_cells, LAT_EINVAL, "cell index out of range");
    }
    bool neg = false;
    double mdf = DBL_MAX;
    if (r_glob || f_cells) {
      double* fc = f_cells;
      if (!fc) {
        h->f_cells.ensure((size_t)h->n_loc * h->n_cells);
        fc = h->f_cells.p;
      }
      run_residual(h, u_glob, fc, r_glob, &mdf, &neg);
    }
    if (K_vals && n_sel > 0) {
      bool n2 = false;
      run_tangent(h, u_glob, quad, cells, n_sel, K_vals, &n2);
      neg = neg || n2;
      mdf = std::min(mdf, h->h_pinned[0]);
    }
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    if (min_detF) *min_detF = mdf;
    if (neg) throw LatError{LAT_ENEG_JACOBIAN, "det F <= 0 at some quadrature point"};
  });
}
