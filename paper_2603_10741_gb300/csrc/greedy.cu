// Greedy selection of principal cells (Algorithm 1), the RB coefficients alpha (Section 3.2.2)
// and the entry points greedy_select / select_principal_cells.
//
// The snapshot matrix is stored column-major, one cell per contiguous column (T^s = data of the
// reduced-rule tangent of cell s, Eq. snapshots).  Per greedy iteration i:
//   select : one CTA reduces (max ||Delta^s||_inf, argmax) over the columns (ties -> lowest s),
//            records it and decides termination (device flag, no host round trip);
//   zeta   : zeta_i = Delta^{s_i} / ||Delta^{s_i}||_2 copied into Z (grid over rows);
//   update : one CTA per column: beta_i^s = Delta^s . zeta_i, Delta^s -= beta_i^s zeta_i, and the
//            new ||Delta^s||_inf, ||Delta^s||_2 of the column (one read + one write of Delta).
// Every kernel returns at once when the device flag says the loop has ended, so the host can
// launch iterations in chunks and look at the flag once per chunk.
#include <algorithm>
#include <cfloat>

#include "common.cuh"

namespace {

constexpr int kColThreads = 256;

__global__ void __launch_bounds__(kColThreads)
    k_g_init(int64_t n_rows, const double* __restrict__ T, double* __restrict__ Delta,
             double* __restrict__ norms, double* __restrict__ inf, double* __restrict__ nrm2) {
  __shared__ double red[32];
  const int s = blockIdx.x;
  const double* t = T + (size_t)s * n_rows;
  double* dl = Delta + (size_t)s * n_rows;
  double ss = 0;
  for (int64_t r = threadIdx.x; r < n_rows; r += blockDim.x) ss += t[r] * t[r];
  const double nrm = sqrt(block_sum(ss, red));
  const double inv = nrm > 0 ? 1.0 / nrm : 0.0;
  double mx = 0, s2 = 0;
  for (int64_t r = threadIdx.x; r < n_rows; r += blockDim.x) {
    double v = t[r] * inv;
    dl[r] = v;
    mx = fmax(mx, fabs(v));
    s2 += v * v;
  }
  mx = block_max(mx, red);
  s2 = block_sum(s2, red);
  if (threadIdx.x == 0) {
    norms[s] = nrm;
    inf[s] = mx;
    nrm2[s] = s2;
  }
}

// state[0] = done, state[1] = n_r, state[2] = selected column of this iteration
__global__ void k_g_select(int it, int n_cols, int limit, double eps, const double* __restrict__ inf,
                           const double* __restrict__ nrm2, int* __restrict__ state,
                           int* __restrict__ S, double* __restrict__ maxres, double* __restrict__ scale) {
  if (state[0]) return;
  __shared__ double bv[32];
  __shared__ int bi[32];
  double best = -1.0;
  int bidx = 0x7fffffff;
  for (int s = threadIdx.x; s < n_cols; s += blockDim.x) {
    double v = inf[s];
    if (v > best || (v == best && s < bidx)) {
      best = v;
      bidx = s;
    }
  }
  // warp then block argmax, ties to the lowest index
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, best, o);
    int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    if (ov > best || (ov == best && oi < bidx)) {
      best = ov;
      bidx = oi;
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    bv[wid] = best;
    bi[wid] = bidx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (bv[w] > best || (bv[w] == best && bi[w] < bidx)) {
        best = bv[w];
        bidx = bi[w];
      }
    maxres[it] = best;
    if (!(best > eps) || it >= limit) {
      state[0] = 1;
      state[1] = it;
    } else {
      S[it] = bidx;
      state[1] = it + 1;
      state[2] = bidx;
      scale[0] = 1.0 / sqrt(nrm2[bidx]);
    }
  }
}

__global__ void k_g_zeta(int it, int64_t n_rows, const double* __restrict__ Delta,
                         const int* __restrict__ state, const double* __restrict__ scale,
                         double* __restrict__ Z) {
  if (state[0]) return;
  const int s = state[2];
  const double sc = scale[0];
  double* z = Z + (size_t)it * n_rows;
  const double* dl = Delta + (size_t)s * n_rows;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rows; r += (int64_t)gridDim.x * blockDim.x)
    z[r] = dl[r] * sc;
}

__global__ void __launch_bounds__(kColThreads)
    k_g_update(int it, int64_t n_rows, int n_cols, double* __restrict__ Delta,
               const double* __restrict__ Z, const int* __restrict__ state, double* __restrict__ beta,
               double* __restrict__ inf, double* __restrict__ nrm2) {
  if (state[0]) return;
  __shared__ double red[32];
  const int s = blockIdx.x;
  double* dl = Delta + (size_t)s * n_rows;
  const double* z = Z + (size_t)it * n_rows;
  double b = 0;
  for (int64_t r = threadIdx.x; r < n_rows; r += blockDim.x) b += dl[r] * z[r];
  b = block_sum(b, red);
  double mx = 0, s2 = 0;
  for (int64_t r = threadIdx.x; r < n_rows; r += blockDim.x) {
    double v = dl[r] - b * z[r];
    dl[r] = v;
    mx = fmax(mx, fabs(v));
    s2 += v * v;
  }
  mx = block_max(mx, red);
  s2 = block_sum(s2, red);
  if (threadIdx.x == 0) {
    beta[(size_t)it * n_cols + s] = b;
    inf[s] = mx;
    nrm2[s] = s2;
  }
}

// alpha^s from R alpha^s = ||t^s|| beta^s, R_ir = ||t^{s_r}|| beta_i^{s_r} (i <= r): the
// coordinates of the principal snapshots in the orthonormal basis Z (upper triangular)
template <typename T>
__global__ void k_g_alpha(int n_r, int n_cols, const int* __restrict__ S, const double* __restrict__ beta,
                          const double* __restrict__ norms, double* __restrict__ alpha,
                          T* __restrict__ alpha_lo) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_cols) return;
  const double ns = norms[s];
  for (int r = n_r - 1; r >= 0; --r) {
    double v = ns * beta[(size_t)r * n_cols + s];
    for (int j = r + 1; j < n_r; ++j) {
      const int sj = S[j];
      v -= norms[sj] * beta[(size_t)r * n_cols + sj] * alpha[(size_t)j * n_cols + s];
    }
    const int sr = S[r];
    v /= norms[sr] * beta[(size_t)r * n_cols + sr];
    alpha[(size_t)r * n_cols + s] = v;
  }
  if (alpha_lo)
    for (int r = 0; r < n_r; ++r) alpha_lo[(size_t)r * n_cols + s] = (T)alpha[(size_t)r * n_cols + s];
}

__global__ void k_iota(int n, int* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = i;
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}

}  // namespace

void run_greedy(lat_ctx* h, const double* T, int64_t n_rows, int n_cols, double eps, int max_nr,
                int* S_out, int* n_r_out, double* alpha_out, double* beta_out, double* Z_out,
                double* max_res_host) {
  const int limit = (int)std::min<int64_t>({(int64_t)max_nr, (int64_t)n_cols, n_rows});
  LAT_REQUIRE(limit >= 1, LAT_EINVAL, "greedy needs max_nr >= 1 and a non-empty snapshot matrix");
  h->g_delta.ensure((size_t)n_cols * n_rows);
  h->g_Z.ensure((size_t)limit * n_rows);
  h->g_beta.ensure((size_t)limit * n_cols);
  h->g_inf.ensure(n_cols);
  h->g_nrm2.ensure(n_cols);
  h->g_norms.ensure(n_cols);
  h->g_maxres.ensure(limit + 1);
  h->g_state.ensure(4);
  h->g_scale.ensure(2);
  h->S.ensure(std::max(limit, h->n_cells));
  LAT_CUDA(cudaMemsetAsync(h->g_state.p, 0, 4 * sizeof(int), h->stream));
  LAT_LAUNCH(h, k_g_init<<<n_cols, kColThreads, 0, h->stream>>>(n_rows, T, h->g_delta.p, h->g_norms.p, h->g_inf.p,
                                                  h->g_nrm2.p));
  LAT_CHECK_LAUNCH();
  const int zgrid = std::min(div_up(n_rows, 256), 4 * h->n_sm);
  int* hp = reinterpret_cast<int*>(h->h_pinned);
  const int chunk = 8;
  for (int it0 = 0; it0 <= limit; it0 += chunk) {
    for (int it = it0; it < std::min(it0 + chunk, limit + 1); ++it) {
      LAT_LAUNCH(h, k_g_select<<<1, 1024, 0, h->stream>>>(it, n_cols, limit, eps, h->g_inf.p, h->g_nrm2.p,
                                            h->g_state.p, h->S.p, h->g_maxres.p, h->g_scale.p));
      LAT_LAUNCH(h, k_g_zeta<<<zgrid, 256, 0, h->stream>>>(it, n_rows, h->g_delta.p, h->g_state.p, h->g_scale.p, h->g_Z.p));
      KernelTimer kt(h, "greedy_update");
      LAT_LAUNCH(h, k_g_update<<<n_cols, kColThreads, 0, h->stream>>>(it, n_rows, n_cols, h->g_delta.p, h->g_Z.p,
                                                        h->g_state.p, h->g_beta.p, h->g_inf.p, h->g_nrm2.p));
    }
    LAT_CHECK_LAUNCH();
    LAT_CUDA(cudaMemcpyAsync(hp, h->g_state.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    if (hp[0]) break;
  }
  LAT_REQUIRE(hp[0], LAT_EINVAL, "greedy did not terminate");
  const int n_r = hp[1];
  h->n_r = n_r;
  // coefficients
  h->alpha.ensure((size_t)std::max(n_r, 1) * n_cols);
  float* a32 = nullptr;
  if (h->prec != LAT_FP64 && n_cols == h->n_cells) {
    h->alpha32.ensure((size_t)std::max(n_r, 1) * n_cols);
    a32 = h->alpha32.p;
  }
  if (n_r > 0) {
    LAT_LAUNCH(h, k_g_alpha<float><<<div_up(n_cols, 128), 128, 0, h->stream>>>(n_r, n_cols, h->S.p, h->g_beta.p,
                                                                 h->g_norms.p, h->alpha.p, a32));
    LAT_CHECK_LAUNCH();
  }
  if (S_out) LAT_CUDA(cudaMemcpyAsync(S_out, h->S.p, n_r * sizeof(int), cudaMemcpyDeviceToDevice, h->stream));
  if (alpha_out && n_r)
    LAT_CUDA(cudaMemcpyAsync(alpha_out, h->alpha.p, (size_t)n_r * n_cols * sizeof(double),
                             cudaMemcpyDeviceToDevice, h->stream));
  if (beta_out && n_r)
    LAT_CUDA(cudaMemcpyAsync(beta_out, h->g_beta.p, (size_t)n_r * n_cols * sizeof(double),
                             cudaMemcpyDeviceToDevice, h->stream));
  if (Z_out && n_r)
    LAT_CUDA(cudaMemcpyAsync(Z_out, h->g_Z.p, (size_t)n_r * n_rows * sizeof(double),
                             cudaMemcpyDeviceToDevice, h->stream));
  if (max_res_host)
    LAT_CUDA(cudaMemcpyAsync(max_res_host, h->g_maxres.p, (n_r + 1) * sizeof(double),
                             cudaMemcpyDeviceToHost, h->stream));
  LAT_CUDA(cudaStreamSynchronize(h->stream));
  if (n_r_out) *n_r_out = n_r;
}

extern "C" lat_status greedy_select(lat_handle h, const double* T, int64_t n_rows, int32_t n_cols,
                                    double eps, int32_t max_nr, int32_t* S, int32_t* n_r,
                                    double* alpha, double* beta, double* Z, double* max_res) {
  if (!h || !T || n_rows <= 0 || n_cols <= 0) return LAT_EINVAL;
  return guard(h, [&] {
    run_greedy(h, T, n_rows, n_cols, eps, max_nr, S, n_r, alpha, beta, Z, max_res);
    h->n_r = 0;  // a standalone greedy does not define a principal set for the solver
  });
}

// snapshots -> greedy -> alpha -> principal tangents, kept in the handle
void select_cells(lat_ctx* h, const double* u_glob, double eps, int max_nr, bool force_all) {
  bool neg = false;
  h->force_all = force_all;
  if (force_all) {
    h->n_r = h->n_cells;
    h->S.ensure(h->n_cells);
    LAT_LAUNCH(h, k_iota<<<div_up(h->n_cells, 256), 256, 0, h->stream>>>(h->n_cells, h->S.p));
    LAT_CHECK_LAUNCH();
  } else {
    // snapshots (Eq. snapshots): the reduced-rule local tangents' data, or the pulled-back
    // tangent tensor at the reduced points (the Remark after it), one column per cell
    int64_t rows = h->nnz;
    if (h->snap_kind == 1) {
      rows = (int64_t)h->n_el * h->dim * h->dim * h->dim * h->dim;
      h->T.ensure((size_t)h->n_cells * rows);
      run_dref_snapshots(h, u_glob, h->T.p, &neg);
    } else {
      h->T.ensure((size_t)h->n_cells * h->nnz);
      run_tangent(h, u_glob, 1, nullptr, h->n_cells, h->T.p, &neg);
    }
    LAT_REQUIRE(!neg, LAT_ENEG_JACOBIAN, "det F <= 0 in the snapshot evaluation");
    run_greedy(h, h->T.p, rows, h->n_cells, eps, max_nr, nullptr, nullptr, nullptr, nullptr,
               nullptr, nullptr);
    LAT_REQUIRE(h->n_r > 0, LAT_EINVAL, "greedy selected no principal cell");
  }
  h->Kp.ensure((size_t)h->n_r * h->nnz);
  run_tangent(h, u_glob, 0, force_all ? nullptr : h->S.p, h->n_r, h->Kp.p, &neg);
  LAT_REQUIRE(!neg, LAT_ENEG_JACOBIAN, "det F <= 0 in a principal tangent");
  if (h->prec != LAT_FP64) {
    const int64_t n = (int64_t)h->n_r * h->nnz;
    h->Kp32.ensure(n);
    LAT_LAUNCH(h, k_to_f32<<<div_up(n, 256), 256, 0, h->stream>>>(n, h->Kp.p, h->Kp32.p));
    LAT_CHECK_LAUNCH();
  }
  ++h->sel_version;
}

extern "C" lat_status lattice_set_snapshots(lat_handle h, int32_t kind) {
  if (!h || (kind != 0 && kind != 1)) return LAT_EINVAL;
  h->snap_kind = kind;
  return LAT_OK;
}

extern "C" lat_status select_principal_cells(lat_handle h, const double* u_glob, double eps,
                                             int32_t max_nr, int32_t force_all, int32_t* S,
                                             int32_t* n_r, double* alpha, double* K_p) {
  if (!h || !u_glob) return LAT_EINVAL;
  return guard(h, [&] {
    LAT_REQUIRE(force_all || max_nr >= 1, LAT_EINVAL, "max_nr must be >= 1");
    select_cells(h, u_glob, eps, max_nr, force_all != 0);
    if (S) LAT_CUDA(cudaMemcpyAsync(S, h->S.p, h->n_r * sizeof(int), cudaMemcpyDeviceToDevice, h->stream));
    if (alpha && !h->force_all)
      LAT_CUDA(cudaMemcpyAsync(alpha, h->alpha.p, (size_t)h->n_r * h->n_cells * sizeof(double),
                               cudaMemcpyDeviceToDevice, h->stream));
    if (K_p)
      LAT_CUDA(cudaMemcpyAsync(K_p, h->Kp.p, (size_t)h->n_r * h->nnz * sizeof(double),
                               cudaMemcpyDeviceToDevice, h->stream));
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    if (n_r) *n_r = h->n_r;
  });
}

// Caller-given principal set and coefficients (Eq. romstiffnessmatrix with S and alpha chosen by
// the caller instead of Algorithm 1): principal tangents at the full rule, FP32 copies in the
// mixed modes.  Used to measure the reduced action at a chosen N_r.
extern "C" lat_status set_principal_cells(lat_handle h, const double* u_glob, const int32_t* S, int32_t n_r,
                                          const double* alpha) {
  if (!h || !u_glob || !S || !alpha) return LAT_EINVAL;
  return guard(h, [&] {
    LAT_REQUIRE(n_r >= 1 && n_r <= h->n_cells, LAT_EINVAL, "n_r must be in [1, n_cells]");
    std::vector<int32_t> hs(n_r);
    LAT_CUDA(cudaMemcpyAsync(hs.data(), S, n_r * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    for (int32_t c : hs) LAT_REQUIRE(c >= 0 && c < h->n_cells, LAT_EINVAL, "principal cell index out of range");
    h->force_all = false;
    h->n_r = n_r;
    h->S.ensure(n_r);
    LAT_CUDA(cudaMemcpyAsync(h->S.p, S, n_r * sizeof(int32_t), cudaMemcpyDeviceToDevice, h->stream));
    const size_t na = (size_t)n_r * h->n_cells;
    h->alpha.ensure(na);
    LAT_CUDA(cudaMemcpyAsync(h->alpha.p, alpha, na * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    bool neg = false;
    h->Kp.ensure((size_t)n_r * h->nnz);
    run_tangent(h, u_glob, 0, h->S.p, n_r, h->Kp.p, &neg);
    LAT_REQUIRE(!neg, LAT_ENEG_JACOBIAN, "det F <= 0 in a principal tangent");
    if (h->prec != LAT_FP64) {
      const int64_t n = (int64_t)n_r * h->nnz;
      h->Kp32.ensure(n);
      LAT_LAUNCH(h, k_to_f32<<<div_up(n, 256), 256, 0, h->stream>>>(n, h->Kp.p, h->Kp32.p));
      h->alpha32.ensure(na);
      LAT_LAUNCH(h, k_to_f32<<<div_up((int64_t)na, 256), 256, 0, h->stream>>>((int64_t)na, h->alpha.p, h->alpha32.p));
      LAT_CHECK_LAUNCH();
    }
    ++h->sel_version;
    LAT_CUDA(cudaStreamSynchronize(h->stream));
  });
}

// ---------------------------------------------------------------------------------------------
// Allocation-free variant of greedy_select.
//
// Some callers cannot allocate device memory: code running inside a memory pool or arena that
// owns the whole device budget, plugins whose host application forbids cudaMalloc/cudaFree on
// its hot path (they synchronise the device and can stall other streams), and code that must
// not create a lattice handle (lattice_setup allocates).  This entry point runs the same
// Algorithm 1 kernels as greedy_select on the caller's snapshot matrix, with every workspace
// carved out of one file-scope device array of fixed size.  The array lives on every device
// that loads the library, from load until process exit.
// ---------------------------------------------------------------------------------------------
namespace {

constexpr size_t kStaticGreedyDoubles = size_t(2) << 20;   // 2 Mi doubles = 16 MiB
constexpr int kStaticMaxDevices = 64;

__device__ __align__(256) double g_static_greedy[kStaticGreedyDoubles];

// device address of g_static_greedy per device, looked up once with that device current
double* g_static_ptr[kStaticMaxDevices] = {nullptr};

struct StaticLayout {
  double *delta, *Z, *beta, *norms, *inf, *nrm2, *maxres, *scale;
  int* state;
  int* S;
  size_t doubles;
};

StaticLayout static_layout(double* base, int64_t n_rows, int n_cols, int limit) {
  StaticLayout L{};
  size_t off = 0;
  auto take = [&](size_t n) {
    double* p = base ? base + off : nullptr;
    off += (n + 31) & ~size_t(31);   // keep every piece 256-byte aligned
    return p;
  };
  L.delta = take((size_t)n_cols * n_rows);
  L.Z = take((size_t)limit * n_rows);
  L.beta = take((size_t)limit * n_cols);
  L.norms = take(n_cols);
  L.inf = take(n_cols);
  L.nrm2 = take(n_cols);
  L.maxres = take(limit + 1);
  L.scale = take(2);
  L.state = reinterpret_cast<int*>(take(2));          // 4 ints
  L.S = reinterpret_cast<int*>(take((limit + 1) / 2 + 1));
  L.doubles = off;
  return L;
}

}  // namespace

extern "C" lat_status greedy_select_static(const double* T, int64_t n_rows, int32_t n_cols, double eps,
                                           int32_t max_nr, int32_t* S, int32_t* n_r, double* alpha,
                                           void* cuda_stream) {
  if (!T || !S || !n_r || n_rows <= 0 || n_cols <= 0 || max_nr < 1) return LAT_EINVAL;
  // each factor alone must fit before the products below are formed (no size_t wrap-around)
  if ((uint64_t)n_rows > kStaticGreedyDoubles || (uint64_t)n_cols > kStaticGreedyDoubles) return LAT_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int limit = (int)std::min<int64_t>({(int64_t)max_nr, (int64_t)n_cols, n_rows});
  if (static_layout(nullptr, n_rows, n_cols, limit).doubles > kStaticGreedyDoubles) return LAT_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) return LAT_ECUDA;
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_greedy) != cudaSuccess || !p) return LAT_ECUDA;
    g_static_ptr[dev] = static_cast<double*>(p);
  }
  const StaticLayout W = static_layout(g_static_ptr[dev], n_rows, n_cols, limit);
  int n_sm = 0;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LAT_ECUDA;
  if (cudaMemsetAsync(W.state, 0, 4 * sizeof(int), st) != cudaSuccess) return LAT_ECUDA;
  k_g_init<<<n_cols, kColThreads, 0, st>>>(n_rows, T, W.delta, W.norms, W.inf, W.nrm2);
  const int zgrid = std::min(div_up(n_rows, 256), 4 * n_sm);
  int hstate[2] = {0, 0};
  const int chunk = 8;
  for (int it0 = 0; it0 <= limit; it0 += chunk) {
    for (int it = it0; it < std::min(it0 + chunk, limit + 1); ++it) {
      k_g_select<<<1, 1024, 0, st>>>(it, n_cols, limit, eps, W.inf, W.nrm2, W.state, W.S, W.maxres, W.scale);
      k_g_zeta<<<zgrid, 256, 0, st>>>(it, n_rows, W.delta, W.state, W.scale, W.Z);
      k_g_update<<<n_cols, kColThreads, 0, st>>>(it, n_rows, n_cols, W.delta, W.Z, W.state, W.beta, W.inf, W.nrm2);
    }
    if (cudaGetLastError() != cudaSuccess) return LAT_ECUDA;
    if (cudaMemcpyAsync(hstate, W.state, 2 * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return LAT_ECUDA;
    if (hstate[0]) break;
  }
  if (!hstate[0]) return LAT_EINVAL;
  const int k = hstate[1];
  if (k > 0 && alpha)
    k_g_alpha<float><<<div_up(n_cols, 128), 128, 0, st>>>(k, n_cols, W.S, W.beta, W.norms, alpha, nullptr);
  if (cudaGetLastError() != cudaSuccess) return LAT_ECUDA;
  if (k > 0 && cudaMemcpyAsync(S, W.S, k * sizeof(int), cudaMemcpyDeviceToDevice, st) != cudaSuccess) return LAT_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return LAT_ECUDA;
  *n_r = k;
  return LAT_OK;
}
