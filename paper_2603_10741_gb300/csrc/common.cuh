// Internal definitions shared by the translation units of liblattice.so.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "lattice.h"

// ------------------------------------------------------------------------------------------
// error handling: every entry point returns lat_status, the message goes to h->err
// ------------------------------------------------------------------------------------------
struct LatError {
  lat_status code;
  std::string msg;
};

#define LAT_CUDA(call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      throw LatError{e_ == cudaErrorMemoryAllocation ? LAT_ENOMEM : LAT_ECUDA,             \
                     std::string(#call) + ": " + cudaGetErrorString(e_)};                  \
  } while (0)

#define LAT_CHECK_LAUNCH() LAT_CUDA(cudaGetLastError())

// every kernel launch of the library goes through this wrapper, which counts it on the handle
#define LAT_LAUNCH(h, ...)   \
  do {                       \
    ++(h)->n_launch;         \
    __VA_ARGS__;             \
  } while (0)

#define LAT_REQUIRE(cond, code, text)                                                      \
  do {                                                                                     \
    if (!(cond)) throw LatError{code, text};                                               \
  } while (0)

// ------------------------------------------------------------------------------------------
// device buffers owned by the handle
// ------------------------------------------------------------------------------------------
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void ensure(size_t count) {
    if (count <= n && p) return;
    release();
    if (count == 0) return;
    LAT_CUDA(cudaMalloc(&p, count * sizeof(T)));
    n = count;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  void upload(const std::vector<T>& v, cudaStream_t st) {
    ensure(v.size());
    if (!v.empty())
      LAT_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  }
};

// ------------------------------------------------------------------------------------------
// the handle
// ------------------------------------------------------------------------------------------
struct lat_ctx {
  // sizes
  int dim = 0, nen = 0, n_cells = 0, n_nodes_cell = 0, n_el = 0, n_loc = 0, n_blk = 0;
  int64_t nnz = 0, n_glob_nodes = 0, n_dof = 0;
  int nq[2] = {0, 0};  // [0] full rule, [1] reduced rule (per element)
  double mu = 0, lam = 0;
  lat_precision prec = LAT_FP64;
  cudaStream_t stream = nullptr;
  std::string err;
  int n_sm = 0;

  // reference cell
  DBuf<double> gradX[2], W[2];  // [n_el][nq][nen][dim], [n_el][nq]
  DBuf<int> elems;              // [n_el][nen]
  DBuf<int> elem_blk;           // [n_el][nen][nen] block index of (a, b)
  std::vector<int> color_start; // host offsets into color_elems
  DBuf<int> color_elems;
  DBuf<int> blk_ptr, blk_col;   // node-block CSR of the local pattern
  std::vector<int> h_blk_ptr, h_blk_col;

  // lattice
  DBuf<int> cell_nodes;               // [n_cells][n_nodes_cell]
  DBuf<double> mu_cell;               // [n_cells] mu * theta_s
  std::vector<double> h_mu_scale;
  DBuf<int> copy_ptr, copy_idx;       // global node -> copies s*n_nodes_cell + a
  DBuf<uint8_t> dof_fixed;            // [n_dof]
  DBuf<double> dir_unit, aff_unit;    // [n_dof]
  std::vector<uint8_t> h_dof_fixed;
  std::vector<double> h_X_ref;          // host copies kept to rebuild the FETI-DP index sets
  std::vector<int> h_cell_nodes, h_cptr, h_cidx;
  int enrich_level = 0;                 // primal enrichment level (Section 3.3.2)

  // FETI-DP structure
  int n_P = 0, n_R = 0;               // local primal (corner) / remaining dofs
  int n_I = 0;                        // interior dofs: rdofs[0, n_I); dual dofs follow
  DBuf<int> corner_of_node;           // [n_nodes_cell] corner id or -1
  DBuf<int> rdofs, pdofs;             // [n_R], [n_P] local dof ids
  DBuf<int> rpos;                     // [n_loc] position in rdofs or -1
  DBuf<int> pidx;                     // [n_cells][n_P] free global primal index or -1
  int64_t n_primal = 0, n_lambda = 0, n_krylov = 0;
  DBuf<int> p_copy_ptr, p_copy;       // primal dof -> local entries k*n_cells+s (P rows)
  DBuf<uint8_t> loc_fixed;            // [n_loc][n_cells] 1 = fixed local entry (or P row)
  DBuf<int> lam_p, lam_m;             // [n_lambda] local entries of the +/- copies
  DBuf<int> dual_entry, dual_l1, dual_l2;  // dual copies and their multipliers (+-(l+1), 0 = none)
  DBuf<double> dual_scale;            // [n_dual] 1/multiplicity of the node
  DBuf<int2> dual_lk;                 // [n_D][n_cells] signed multipliers (l1, l2) of each dual copy
  DBuf<float> dual_lsc;               // [n_D][n_cells] its 1/multiplicity
  int64_t n_dual = 0;
  int n_classes = 0;
  DBuf<int> cell_class;               // [n_cells] boundary-condition class
  std::vector<int> class_rep;         // representative cell per class
  DBuf<int> coarse_ptr, coarse_src;   // coarse matrix entries -> (cell, i, j) contributions
  DBuf<int> coarse_row, coarse_col;
  // block-tridiagonal coarse structure (coarse DOFs grouped by the cell layer along the load
  // axis); empty when the lattice does not give one
  bool coarse_blocked = false;
  int cb_n = 0, cb_m = 0;                 // number of blocks, padded block size
  bool cb_solve = false;                  // FP64 coarse solves by block LU (no dense inverse)
  bool cb_wide = false;                   // block-LU solves over the whole GPU (else cluster sweeps)
  int cb_coop_grid = -1;                  // CTAs of the cooperative whole-solve launch (0: per-step launches)
  int cb_cluster = 0, cb_pre = 0;         // CTAs per cluster of the sweeps, rows prefetched
  size_t cb_shm = 0;
  DBuf<int64_t> cb_dest;                  // coarse entry -> index in [A blocks | B blocks], -1 skip
  DBuf<int> cb_perm;                      // block position (b*m + l) -> primal DOF or -1
  std::vector<int32_t> h_cell_layer;
  DBuf<double> cb_A, cb_B, cb_Dinv, cb_Einv, cb_U, cb_V, cb_T, cb_X;
  DBuf<double> cb_Ut, cb_y, cb_w, cb_r; // block-LU solves: U_i^T, forward result, D^-1 y, rhs / x
  DBuf<float> cb_U32, cb_Ut32, cb_Dinv32; // FP32 copies of the factors (mixed modes, whole-GPU steps)

  // selection state
  int n_r = 0;
  bool force_all = false;
  int snap_kind = 0;                  // snapshots: 0 reduced-rule tangent data, 1 D^ref at the reduced points
  DBuf<int> S;                        // [n_r]
  DBuf<double> alpha;                 // [n_r][n_cells]
  DBuf<float> alpha32;
  DBuf<double> Kp;                    // [n_r][nnz]
  DBuf<float> Kp32;
  DBuf<double> Kp_mat;                // [n_r][nnz] material part of K^r (preconditioner option)
  // 3D FP32 reduced action: the cell's nodes in groups of GR = 8 and 16 (one CTA each), with the
  // union of each group's neighbour nodes and its node blocks in group order (built at setup)
  struct NodeGroups {
    int GR = 0, n_grp = 0, nu_max = 0, np_max = 0;
    DBuf<int> rows;    // [n_grp][GR] node of each warp, -1 for none
    DBuf<int> ucptr;   // [n_grp + 1] into ucol
    DBuf<int> ucol;    // union of the group's neighbour nodes, ascending
    DBuf<int> pp;      // [n_grp][GR + 1] block ranges of the group's rows (global block-pair index)
    DBuf<int> pair_u;  // [n_blk] position of the pair's column node in its group's union
    DBuf<int> perm;    // [n_blk] CSR block index of each pair
  } ng[2];
  DBuf<float> Kg;                     // [n_r][n_blk][12] FP32 principal blocks in group order
  int64_t sel_version = 0, kg_version = -1;   // principal-set changes / the group-order copy's
  int kg_gr = 0;
  // greedy workspaces
  DBuf<double> g_delta, g_Z, g_beta, g_inf, g_nrm2, g_norms, g_part, g_maxres;
  DBuf<int> g_state;                  // [0] done, [1] n_r, [2] s_next
  DBuf<double> g_scale;
  // assembly workspaces
  DBuf<double> f_cells, r_glob, minJ_cell, T;
  DBuf<int> negJ;

  // solver state
  int n_keys = 0;
  DBuf<int> key_of_cell, key_slot, perm, seg_ptr, tile_seg, tile_c0, key_list, solver_int;
  DBuf<double> delta_cell, c_cell;    // per-cell inverse weight and scale
  DBuf<double> G, Phi, Sloc;          // [n_keys][n_R][n_R], [n_keys][n_R][n_P], [n_keys][n_P][n_P]
  DBuf<float> G32;
  DBuf<double> SDD;                   // [n_keys][n_D][n_D] dual Schur complements
  DBuf<float> SDD32;
  DBuf<double> gj_P, gj_C, gj_R;      // Gauss-Jordan workspace (pivot inverse, column and row panels)
  DBuf<int> class_rep_d;
  DBuf<__nv_bfloat16> G16[4], Xb16;    // BF16 local matrices (one view per KinvMode, then the dual
                                       // Schur complements S_DD), packed cell vectors
  int g16_ld[4] = {0, 0, 0, 0};        // their row strides
  int64_t g16_lo[4] = {0, 0, 0, 0};    // offset of the low BF16 part after the high part
  DBuf<double> KRP, Coarse, CoarseInv;
  DBuf<float> CoarseInv32;             // FP32 copy of the coarse inverse (mixed modes)
  int64_t coarse32_ld = 0;             // its row stride (a multiple of 4)
  DBuf<double> tP, gP, xP;            // per-cell primal buffer [n_P][n_cells], primal vectors
  DBuf<float> tP32, Phi32;            // FP32 per-cell primal buffer and Phi copy (mixed modes)
  DBuf<float> x32, y32;               // mixed-precision local vectors
  DBuf<double> kv_tmp[6];             // saddle-point sized temporaries
  DBuf<double> pcg_ws;                // interface PCG vectors (5 x n_lambda)
  DBuf<double> V, Zk, Hh, gmres_small, dots_part;
  DBuf<double> kscal[2];              // FGMRES device scalars of the outer and the inner level
  DBuf<double> V2, Z2, Hh2, gmres_small2;   // inner FGMRES (FP32 operator) of the mixed modes
  int64_t inner_its_total = 0;        // inner FGMRES iterations since the last reset
  DBuf<int> flag;
  DBuf<double> red_part;            // reduction scratch
  int max_tiles = 0;
  DBuf<int> tile_seg_tc, tile_c0_tc;  // key segments in tiles of kTcCells cells (tensor-core products)
  int max_tiles_tc = 0;
  bool indefinite = false;              // a principal's remaining block had a negative pivot
  bool coarse_indefinite = false;       // the coarse matrix had a negative pivot
  int64_t pcg_its_total = 0;            // interface PCG iterations since the last reset
  int64_t n_launch = 0;                 // kernels launched through this handle
  int iface = 0;                        // interface preconditioner: 0 Dirichlet, 1 lumped
  bool verbose = false;                 // LATTICE_VERBOSE=1: per-iteration log on stderr
  double *h_pinned = nullptr;          // small pinned host scratch

  // optional per-kernel timing: CUDA events recorded on the launching stream around the
  // launches of named kernels (lattice_set_timing / lattice_kernel_time)
  bool timing = false;
  bool timing_apply_only = false;       // time only the reduced / plain tangent action kernels
  // interface PCG iteration captured as a CUDA graph (dropped whenever the solver is set up)
  cudaGraphExec_t pcg_exec = nullptr;
  cudaStream_t cap_stream = nullptr;    // private stream the graph is captured on
  int pcg_exec_check = -1;              // whether the captured iteration copies its scalars out
  int64_t pcg_graph_kernels = 0;        // kernels in one replay (added to n_launch per replay)
  bool graphs_ok = true;
  std::map<std::string, std::vector<std::pair<cudaEvent_t, cudaEvent_t>>> ev;
  std::vector<cudaEvent_t> ev_pool;
};

// RAII bracket: records a start event now and a stop event at scope exit when timing is on
struct KernelTimer {
  lat_ctx* h;
  const char* name;
  cudaEvent_t a = nullptr, b = nullptr;
  static cudaEvent_t take(lat_ctx* h) {
    if (!h->ev_pool.empty()) {
      cudaEvent_t e = h->ev_pool.back();
      h->ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  KernelTimer(lat_ctx* h_, const char* n) : h(h_), name(n) {
    if (!h->timing) return;
    if (h->timing_apply_only && std::strncmp(n, "apply_", 6) != 0) return;
    a = take(h);
    b = take(h);
    cudaEventRecord(a, h->stream);
  }
  ~KernelTimer() {
    if (!a) return;
    cudaEventRecord(b, h->stream);
    h->ev[name].push_back({a, b});
  }
};

// run f, converting LatError and std exceptions into a status and h->err
template <typename F>
static lat_status guard(lat_ctx* h, F&& f) {
  try {
    f();
    return LAT_OK;
  } catch (const LatError& e) {
    if (h) h->err = e.msg;
    return e.code;
  } catch (const std::exception& e) {
    if (h) h->err = e.what();
    return LAT_EINVAL;
  }
}

// element colours passed by value to the per-cell kernels
struct ColorTable {
  int n;
  int start[33];
};

// ------------------------------------------------------------------------------------------
// small helpers
// ------------------------------------------------------------------------------------------
static inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

template <int D>
__device__ __forceinline__ double det_inv(const double (&F)[D][D], double (&Fi)[D][D]);

template <>
__device__ __forceinline__ double det_inv<2>(const double (&F)[2][2], double (&Fi)[2][2]) {
  double J = F[0][0] * F[1][1] - F[0][1] * F[1][0];
  double r = 1.0 / J;
  Fi[0][0] = F[1][1] * r;
  Fi[0][1] = -F[0][1] * r;
  Fi[1][0] = -F[1][0] * r;
  Fi[1][1] = F[0][0] * r;
  return J;
}

template <>
__device__ __forceinline__ double det_inv<3>(const double (&F)[3][3], double (&Fi)[3][3]) {
  double c00 = F[1][1] * F[2][2] - F[1][2] * F[2][1];
  double c01 = F[1][2] * F[2][0] - F[1][0] * F[2][2];
  double c02 = F[1][0] * F[2][1] - F[1][1] * F[2][0];
  double J = F[0][0] * c00 + F[0][1] * c01 + F[0][2] * c02;
  double r = 1.0 / J;
  Fi[0][0] = c00 * r;
  Fi[1][0] = c01 * r;
  Fi[2][0] = c02 * r;
  Fi[0][1] = (F[0][2] * F[2][1] - F[0][1] * F[2][2]) * r;
  Fi[1][1] = (F[0][0] * F[2][2] - F[0][2] * F[2][0]) * r;
  Fi[2][1] = (F[0][1] * F[2][0] - F[0][0] * F[2][1]) * r;
  Fi[0][2] = (F[0][1] * F[1][2] - F[0][2] * F[1][1]) * r;
  Fi[1][2] = (F[0][2] * F[1][0] - F[0][0] * F[1][2]) * r;
  Fi[2][2] = (F[0][0] * F[1][1] - F[0][1] * F[1][0]) * r;
  return J;
}

// deterministic block reductions (fixed shape, fixed order)
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// block-wide sum for blockDim.x a multiple of 32 (<= 1024); all threads get the result
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh /* >= 32 */) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T t = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  T out = sh[0];
  __syncthreads();
  return out;
}
template <typename T>
__device__ __forceinline__ T block_max(T v, T* sh) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T t = (threadIdx.x < nw) ? sh[threadIdx.x] : T(-1e300);
  if (wid == 0) t = warp_max(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  T out = sh[0];
  __syncthreads();
  return out;
}

// ------------------------------------------------------------------------------------------
// cross-unit launchers (defined in the .cu files)
// ------------------------------------------------------------------------------------------
void run_residual(lat_ctx* h, const double* u_glob, double* f_cells, double* r_glob,
                  double* min_detF_host, bool* negJ);
void run_tangent(lat_ctx* h, const double* u_glob, int quad, const int* cells, int n_sel,
                 double* K_out, bool* negJ, bool geometric = true);
void run_dref_snapshots(lat_ctx* h, const double* u_glob, double* T, bool* negJ);
void run_tangent_apply_exact(lat_ctx* h, const double* u_glob, const double* v_glob,
                             double* y_glob);
void run_grad_mu(lat_ctx* h, const double* u_glob, const double* w_glob, double* grad);
double run_norm_free(lat_ctx* h, const double* r_glob);
double run_norm_all(lat_ctx* h, const double* r_glob);
double run_dot_fixed(lat_ctx* h, const double* a, const double* b);
void run_greedy(lat_ctx* h, const double* T, int64_t n_rows, int n_cols, double eps, int max_nr,
                int* S_out, int* n_r_out, double* alpha_out, double* beta_out, double* Z_out,
                double* max_res_host);
void run_apply(lat_ctx* h, const void* x, void* y, int dtype, const double* xP, bool feti);
void build_node_groups(lat_ctx* h);
void run_prepare_solver(lat_ctx* h, const lat_newton_opts* o, const double* u_glob);
// square tile (64, 32 or 16) for batched FP64 products over n x n matrices: the least padded
// work per busy SM (padding of n to the tile, and the share of the SMs the tiles occupy)
inline int fp64_tile(int n, int64_t batch, int n_sm) {
  int best = 64;
  double best_cost = 1e300;
  for (int T : {64, 32, 16}) {
    const int64_t per = (n + T - 1) / T;
    const double waste = (double)(per * T) * (per * T) / ((double)n * n);
    const double busy = std::min(1.0, (double)(batch * per * per) / n_sm);
    const double cost = waste / busy;
    if (cost < best_cost * 0.9) {   // prefer the larger tile unless clearly better
      best_cost = cost;
      best = T;
    }
  }
  return best;
}

inline void drop_pcg_graph(lat_ctx* h) {
  if (h->pcg_exec) cudaGraphExecDestroy(h->pcg_exec);
  h->pcg_exec = nullptr;
}
void run_feti_operator(lat_ctx* h, const double* v, double* w);
void run_kinv(lat_ctx* h, const double* v, double* w);
void run_block_precond(lat_ctx* h, const double* v, double* w, int pcg_iters, double pcg_rtol);
int run_fgmres(lat_ctx* h, const double* b, double* x, const lat_newton_opts* o, double* rel_out);
void run_feti_to_global(lat_ctx* h, const double* v, double* u);
void run_feti_from_global(lat_ctx* h, const double* u, double* v, bool split);
void run_axpy(lat_ctx* h, int64_t n, double a, const double* x, double* y);
void run_f2d(lat_ctx* h, int64_t n, const float* x, double* y);
void run_mask(lat_ctx* h, const double* x, double* y, int keep_fixed);
void run_adjoint_w(lat_ctx* h, const double* lam, const double* u, double* w);
void select_cells(lat_ctx* h, const double* u_glob, double eps, int max_nr, bool force_all);
void build_feti(lat_ctx* h, int level);
void prepare_enriched(lat_ctx* h, const lat_newton_opts* o, const double* u_glob);
void gj_invert(lat_ctx* h, double* A, int n, int batch, int64_t bs, int neg_bit, int split = -1,
               double* snap = nullptr);
void run_coarse_blocked(lat_ctx* h, const double* S, int64_t np, bool dense);
bool coarse_block_plan(lat_ctx* h, bool fallback = false);
int coarse_coop_grid(lat_ctx* h);
constexpr int64_t kDenseCoarseLimit = 8192;   // largest padded coarse size N m kept as a dense inverse
constexpr int kWideSweepRows = 512;           // block-LU steps of larger blocks run over the whole GPU
constexpr int kTcCells = 128;                 // cells per tensor-core tile (the MMA's N)
constexpr int kTcRowTiles = 1;                // 128-row tiles per tensor-core CTA (sharing each B panel)
void run_coarse_block_solve(lat_ctx* h, const double* g, double* x);
void run_g_to_bf16(lat_ctx* h, size_t n);
// which part of the local inverse a product uses (see kinv in feti.cu)
enum KinvMode { KINV_FULL = 0, KINV_DUAL = 1, KINV_DUAL_IN = 2 };
void run_local_tc(lat_ctx* h, const double* X, double* Y, KinvMode mode);
void run_sdd_tc(lat_ctx* h, const double* X, double* Y, const double* lam = nullptr);
void run_local_tc_lam(lat_ctx* h, const double* lam, double* Y);
