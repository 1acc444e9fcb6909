// lattice_setup and the small entry points: reference-cell geometry, local sparsity pattern,
// element colouring, local-to-global maps, FETI-DP index sets, predictor, gather, checkpoints.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <numeric>
#include <set>

#include "common.cuh"

namespace {

// Q1 local node positions in [-1,1]^d: counter-clockwise (2D), bottom face then top face (3D)
void q1_node(int d, int a, double* xi) {
  static const int sq[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
  xi[0] = sq[a & 3][0];
  xi[1] = sq[a & 3][1];
  if (d == 3) xi[2] = (a < 4) ? -1.0 : 1.0;
}

// Gauss-Legendre points: full rule = 2 points per direction (+-1/sqrt 3, weight 1),
// reduced rule = the element centre with weight 2^d (Section 3.1.5 and Eq. snapshots)
void gauss(int d, int reduced, std::vector<std::vector<double>>& pts, std::vector<double>& w) {
  pts.clear();
  w.clear();
  if (reduced) {
    pts.push_back(std::vector<double>(d, 0.0));
    w.push_back(std::pow(2.0, d));
    return;
  }
  const double g = 1.0 / std::sqrt(3.0);
  int nq = 1 << d;
  for (int q = 0; q < nq; ++q) {
    std::vector<double> p(d);
    for (int k = 0; k < d; ++k) p[k] = ((q >> k) & 1) ? g : -g;
    pts.push_back(p);
    w.push_back(1.0);
  }
}

void build_geometry(lat_ctx* h, const double* X, const int* E) {
  const int d = h->dim, nen = h->nen;
  for (int red = 0; red < 2; ++red) {
    std::vector<std::vector<double>> pts;
    std::vector<double> wq;
    gauss(d, red, pts, wq);
    const int nq = (int)pts.size();
    h->nq[red] = nq;
    std::vector<double> gX((size_t)h->n_el * nq * nen * d), Wv((size_t)h->n_el * nq);
    for (int e = 0; e < h->n_el; ++e) {
      for (int q = 0; q < nq; ++q) {
        // reference shape-function gradients d phi_a / d xi
        double dphi[8][3];
        for (int a = 0; a < nen; ++a) {
          double na[3];
          q1_node(d, a, na);
          for (int k = 0; k < d; ++k) {
            double v = na[k] / (double)(1 << d);
            for (int m = 0; m < d; ++m)
              if (m != k) v *= (1.0 + na[m] * pts[q][m]);
            dphi[a][k] = v;
          }
        }
        double J0[3][3] = {{0}};
        for (int a = 0; a < nen; ++a) {
          const double* xa = X + (size_t)E[e * nen + a] * d;
          for (int k = 0; k < d; ++k)
            for (int l = 0; l < d; ++l) J0[k][l] += xa[k] * dphi[a][l];
        }
        double det, inv[3][3];
        if (d == 2) {
          det = J0[0][0] * J0[1][1] - J0[0][1] * J0[1][0];
          inv[0][0] = J0[1][1] / det;
          inv[0][1] = -J0[0][1] / det;
          inv[1][0] = -J0[1][0] / det;
          inv[1][1] = J0[0][0] / det;
        } else {
          double c00 = J0[1][1] * J0[2][2] - J0[1][2] * J0[2][1];
          double c01 = J0[1][2] * J0[2][0] - J0[1][0] * J0[2][2];
          double c02 = J0[1][0] * J0[2][1] - J0[1][1] * J0[2][0];
          det = J0[0][0] * c00 + J0[0][1] * c01 + J0[0][2] * c02;
          inv[0][0] = c00 / det;
          inv[1][0] = c01 / det;
          inv[2][0] = c02 / det;
          inv[0][1] = (J0[0][2] * J0[2][1] - J0[0][1] * J0[2][2]) / det;
          inv[1][1] = (J0[0][0] * J0[2][2] - J0[0][2] * J0[2][0]) / det;
          inv[2][1] = (J0[0][1] * J0[2][0] - J0[0][0] * J0[2][1]) / det;
          inv[0][2] = (J0[0][1] * J0[1][2] - J0[0][2] * J0[1][1]) / det;
          inv[1][2] = (J0[0][2] * J0[1][0] - J0[0][0] * J0[1][2]) / det;
          inv[2][2] = (J0[0][0] * J0[1][1] - J0[0][1] * J0[1][0]) / det;
        }
        LAT_REQUIRE(det > 0, LAT_EINVAL, "reference element with non-positive Jacobian");
        // d phi / dX_k = sum_l d phi / d xi_l * (J0^{-1})_{lk}
        for (int a = 0; a < nen; ++a)
          for (int k = 0; k < d; ++k) {
            double v = 0;
            for (int l = 0; l < d; ++l) v += dphi[a][l] * inv[l][k];
            gX[(((size_t)e * nq + q) * nen + a) * d + k] = v;
          }
        Wv[(size_t)e * nq + q] = wq[q] * det;
      }
    }
    h->gradX[red].upload(gX, h->stream);
    h->W[red].upload(Wv, h->stream);
  }
}

void build_pattern_and_colors(lat_ctx* h, const int* E) {
  const int nen = h->nen, nn = h->n_nodes_cell;
  std::vector<std::set<int>> nbr(nn);
  for (int e = 0; e < h->n_el; ++e)
    for (int a = 0; a < nen; ++a)
      for (int b = 0; b < nen; ++b) nbr[E[e * nen + a]].insert(E[e * nen + b]);
  h->h_blk_ptr.assign(nn + 1, 0);
  h->h_blk_col.clear();
  for (int a = 0; a < nn; ++a) {
    h->h_blk_ptr[a + 1] = h->h_blk_ptr[a] + (int)nbr[a].size();
    for (int b : nbr[a]) h->h_blk_col.push_back(b);
  }
  h->n_blk = h->h_blk_ptr[nn];
  // the staged apply keeps one row of node blocks per warp: at most 3^d blocks (Q1 stencil)
  for (int a = 0; a < nn; ++a)
    LAT_REQUIRE(h->h_blk_ptr[a + 1] - h->h_blk_ptr[a] <= (h->dim == 2 ? 9 : 27), LAT_EINVAL,
                "a node couples to more than 3^d nodes: not a Q1 mesh");
  h->nnz = (int64_t)h->n_blk * h->dim * h->dim;
  std::vector<int> eb((size_t)h->n_el * nen * nen);
  for (int e = 0; e < h->n_el; ++e)
    for (int a = 0; a < nen; ++a) {
      int na = E[e * nen + a];
      for (int b = 0; b < nen; ++b) {
        int nb = E[e * nen + b];
        auto beg = h->h_blk_col.begin() + h->h_blk_ptr[na];
        auto end = h->h_blk_col.begin() + h->h_blk_ptr[na + 1];
        eb[((size_t)e * nen + a) * nen + b] = (int)(std::lower_bound(beg, end, nb) - h->h_blk_col.begin());
      }
    }
  h->elem_blk.upload(eb, h->stream);
  h->blk_ptr.upload(h->h_blk_ptr, h->stream);
  h->blk_col.upload(h->h_blk_col, h->stream);
  if (h->dim == 3) build_node_groups(h);
  // greedy colouring: elements of one colour share no node
  std::vector<std::vector<int>> node_el(nn);
  for (int e = 0; e < h->n_el; ++e)
    for (int a = 0; a < nen; ++a) node_el[E[e * nen + a]].push_back(e);
  std::vector<int> col(h->n_el, -1);
  int ncol = 0;
  for (int e = 0; e < h->n_el; ++e) {
    std::vector<char> used(64, 0);
    for (int a = 0; a < nen; ++a)
      for (int f : node_el[E[e * nen + a]])
        if (col[f] >= 0) used[col[f]] = 1;
    int c = 0;
    while (used[c]) ++c;
    col[e] = c;
    ncol = std::max(ncol, c + 1);
  }
  h->color_start.assign(ncol + 1, 0);
  std::vector<int> ce;
  for (int c = 0; c < ncol; ++c) {
    for (int e = 0; e < h->n_el; ++e)
      if (col[e] == c) ce.push_back(e);
    h->color_start[c + 1] = (int)ce.size();
  }
  h->color_elems.upload(ce, h->stream);
}

void build_maps(lat_ctx* h, const lat_mesh_desc* ds) {
  const int d = h->dim, nn = h->n_nodes_cell, ns = h->n_cells, nl = h->n_loc;
  const int* cn = ds->cell_nodes;
  // global node -> copies
  std::vector<int> cptr(h->n_glob_nodes + 1, 0);
  for (int64_t i = 0; i < (int64_t)ns * nn; ++i) {
    LAT_REQUIRE(cn[i] >= 0 && cn[i] < h->n_glob_nodes, LAT_EINVAL, "cell_nodes out of range");
    cptr[cn[i] + 1]++;
  }
  for (int64_t g = 0; g < h->n_glob_nodes; ++g) cptr[g + 1] += cptr[g];
  std::vector<int> cidx(cptr[h->n_glob_nodes]), fill(cptr.begin(), cptr.end() - 1);
  for (int s = 0; s < ns; ++s)
    for (int a = 0; a < nn; ++a) cidx[fill[cn[(size_t)s * nn + a]]++] = s * nn + a;  // cell order
  for (int64_t g = 0; g < h->n_glob_nodes; ++g)
    LAT_REQUIRE(cptr[g + 1] > cptr[g], LAT_EINVAL, "global node used by no cell");
  h->copy_ptr.upload(cptr, h->stream);
  h->copy_idx.upload(cidx, h->stream);
  h->h_cptr = cptr;
  h->h_cidx = cidx;
  h->h_X_ref.assign(ds->X_ref, ds->X_ref + (size_t)nn * d);
  h->h_cell_nodes.assign(cn, cn + (size_t)ns * nn);
  const uint8_t* fx = ds->dof_fixed;

  // boundary-condition classes: cells with the same set of fixed local DOFs
  std::map<std::vector<uint8_t>, int> cls;
  std::vector<int> ccls(ns);
  h->class_rep.clear();
  for (int s = 0; s < ns; ++s) {
    std::vector<uint8_t> mask(nl);
    for (int k = 0; k < nl; ++k)
      mask[k] = fx[(int64_t)cn[(size_t)s * nn + k / d] * d + k % d];
    auto it = cls.find(mask);
    if (it == cls.end()) {
      int id = (int)cls.size();
      cls[mask] = id;
      h->class_rep.push_back(s);
      ccls[s] = id;
    } else {
      ccls[s] = it->second;
    }
  }
  h->n_classes = (int)cls.size();
  h->cell_class.upload(ccls, h->stream);

}

// FETI-DP index sets for primal enrichment `level` (Section 3.3.2): level 0 takes the cell
// corners as primal nodes (Section 3.3.1); level L >= 1 adds, on every edge of the unit cell
// (the four sides in 2D, the twelve cube edges in 3D), the nodes nearest to the points
// j / 2^L (j = 1 .. 2^L - 1) of the edge, for all cells alike.
std::vector<int> primal_nodes(lat_ctx* h, int level) {
  const int d = h->dim, nn = h->n_nodes_cell;
  const std::vector<double>& X = h->h_X_ref;
  auto is01 = [](double x) { return std::fabs(x) < 1e-12 || std::fabs(x - 1.0) < 1e-12; };
  std::vector<int> prim(nn, -1);
  int np = 0;
  for (int a = 0; a < nn; ++a) {
    bool c = true;
    for (int k = 0; k < d; ++k) c = c && is01(X[(size_t)a * d + k]);
    if (c) prim[a] = np++;
  }
  LAT_REQUIRE(np == (1 << d), LAT_EINVAL, "reference cell must have a node at every cube corner");
  if (level <= 0) return prim;
  // edges: the free coordinate `axis`, the fixed coordinates taking values in {0,1}
  std::vector<int> extra;
  for (int axis = 0; axis < d; ++axis) {
    const int nfix = d - 1;
    for (int combo = 0; combo < (1 << nfix); ++combo) {
      std::vector<std::pair<double, int>> on_edge;
      for (int a = 0; a < nn; ++a) {
        if (prim[a] >= 0) continue;
        bool ok = true;
        int bit = 0;
        for (int k = 0; k < d; ++k) {
          if (k == axis) continue;
          const double want = (combo >> bit++) & 1 ? 1.0 : 0.0;
          ok = ok && std::fabs(X[(size_t)a * d + k] - want) < 1e-12;
        }
        if (ok) on_edge.push_back({X[(size_t)a * d + axis], a});
      }
      if (on_edge.empty()) continue;
      const int parts = 1 << level;
      for (int jj = 1; jj < parts; ++jj) {
        const double t = (double)jj / parts;
        int best = -1;
        double bd = 1e300;
        for (auto& pr : on_edge)
          if (std::fabs(pr.first - t) < bd - 1e-12) {
            bd = std::fabs(pr.first - t);
            best = pr.second;
          }
        if (best >= 0 && prim[best] < 0) {
          prim[best] = np++;
          extra.push_back(best);
        }
      }
    }
  }
  return prim;
}

void build_feti_impl(lat_ctx* h, int level) {
  const int d = h->dim, nn = h->n_nodes_cell, ns = h->n_cells, nl = h->n_loc;
  const int* cn = h->h_cell_nodes.data();
  const std::vector<int>& cptr = h->h_cptr;
  const std::vector<int>& cidx = h->h_cidx;
  const uint8_t* fx = h->h_dof_fixed.data();
  std::vector<int> corner = primal_nodes(h, level);
  int nc = 0;
  for (int a = 0; a < nn; ++a) nc += corner[a] >= 0;
  h->enrich_level = level;
  h->corner_of_node.upload(corner, h->stream);
  // remaining dofs ordered interior first, then the non-primal dofs on the cell boundary (the
  // dual dofs): the Gauss-Jordan sweep over the interior block then leaves the dual Schur
  // complement in the trailing block (Dirichlet interface preconditioner)
  std::vector<int> rdofs, pdofs(nc * d), rpos(nl, -1);
  auto on_boundary = [&](int a) {
    for (int k = 0; k < d; ++k) {
      double x = h->h_X_ref[(size_t)a * d + k];
      if (std::fabs(x) < 1e-12 || std::fabs(x - 1.0) < 1e-12) return true;
    }
    return false;
  };
  for (int pass = 0; pass < 2; ++pass)
    for (int a = 0; a < nn; ++a) {
      if (corner[a] >= 0 || on_boundary(a) != (pass == 1)) continue;
      for (int i = 0; i < d; ++i) {
        rpos[a * d + i] = (int)rdofs.size();
        rdofs.push_back(a * d + i);
      }
    }
  for (int a = 0; a < nn; ++a)
    if (corner[a] >= 0)
      for (int i = 0; i < d; ++i) pdofs[corner[a] * d + i] = a * d + i;
  h->n_P = nc * d;
  h->n_R = (int)rdofs.size();
  h->n_I = 0;
  for (int a = 0; a < nn; ++a)
    if (corner[a] < 0 && !on_boundary(a)) h->n_I += d;
  h->rdofs.upload(rdofs, h->stream);
  h->pdofs.upload(pdofs, h->stream);
  h->rpos.upload(rpos, h->stream);

  // free global primal DOFs, numbered by global dof
  std::vector<int64_t> pglob;
  for (int s = 0; s < ns; ++s)
    for (int a = 0; a < nn; ++a)
      if (corner[a] >= 0)
        for (int i = 0; i < d; ++i) {
          int64_t g = (int64_t)cn[(size_t)s * nn + a] * d + i;
          if (!fx[g]) pglob.push_back(g);
        }
  std::sort(pglob.begin(), pglob.end());
  pglob.erase(std::unique(pglob.begin(), pglob.end()), pglob.end());
  h->n_primal = (int64_t)pglob.size();
  std::map<int64_t, int> pmap;
  for (size_t i = 0; i < pglob.size(); ++i) pmap[pglob[i]] = (int)i;
  std::vector<int> pidx((size_t)ns * h->n_P, -1);
  std::vector<std::vector<int>> pcopies(h->n_primal);
  std::vector<uint8_t> lfix((size_t)nl * ns, 0);
  for (int s = 0; s < ns; ++s)
    for (int a = 0; a < nn; ++a)
      for (int i = 0; i < d; ++i) {
        int k = a * d + i;
        int64_t g = (int64_t)cn[(size_t)s * nn + a] * d + i;
        if (corner[a] >= 0) {
          lfix[(size_t)k * ns + s] = 1;   // primal rows are not part of the local unknowns
          if (!fx[g]) {
            int p = pmap[g];
            pidx[(size_t)s * h->n_P + corner[a] * d + i] = p;
            pcopies[p].push_back(k * ns + s);
          }
        } else if (fx[g]) {
          lfix[(size_t)k * ns + s] = 1;
        }
      }
  h->pidx.upload(pidx, h->stream);
  h->loc_fixed.upload(lfix, h->stream);
  std::vector<int> pptr(h->n_primal + 1, 0), pc;
  for (int64_t p = 0; p < h->n_primal; ++p) {
    pptr[p + 1] = pptr[p] + (int)pcopies[p].size();
    for (int v : pcopies[p]) pc.push_back(v);
  }
  h->p_copy_ptr.upload(pptr, h->stream);
  h->p_copy.upload(pc, h->stream);

  // multipliers: each free non-corner DOF with m copies gets m-1 multipliers joining
  // consecutive copies in cell order (non-redundant).  They are numbered in the order of their
  // first copy's cell-stacked entry (local DOF major, cell minor), so that the jump kernels, which
  // walk the dual entries in that order, read the multiplier vector nearly contiguously.
  std::vector<std::pair<int, int>> pairs;   // (entry of the + copy, entry of the - copy)
  std::map<int, int> mult;                  // dual entry -> multiplicity of its node
  for (int64_t g = 0; g < h->n_glob_nodes; ++g) {
    int m = cptr[g + 1] - cptr[g];
    if (m < 2) continue;
    int first = cidx[cptr[g]];
    if (corner[first % nn] >= 0) continue;
    for (int i = 0; i < d; ++i) {
      if (fx[g * d + i]) continue;
      for (int c = 0; c < m - 1; ++c) {
        int ca = cidx[cptr[g] + c], cb = cidx[cptr[g] + c + 1];
        int ea = ((ca % nn) * d + i) * ns + ca / nn;
        int eb = ((cb % nn) * d + i) * ns + cb / nn;
        pairs.push_back({ea, eb});
        mult[ea] = m;
        mult[eb] = m;
      }
    }
  }
  std::sort(pairs.begin(), pairs.end());
  std::vector<int> lp, lm;
  std::map<int, std::pair<int, int>> dual;  // local entry -> (l1, l2) signed (l+1)
  std::map<int, double> dscale;
  for (const auto& pr2 : pairs) {
    const int l = (int)lp.size();
    lp.push_back(pr2.first);
    lm.push_back(pr2.second);
    auto put = [&](int e, int v) {
      auto& pr = dual[e];
      if (pr.first == 0) pr.first = v; else pr.second = v;
      dscale[e] = 1.0 / mult[e];
    };
    put(pr2.first, l + 1);
    put(pr2.second, -(l + 1));
  }
  h->n_lambda = (int64_t)lp.size();
  h->lam_p.upload(lp, h->stream);
  h->lam_m.upload(lm, h->stream);
  std::vector<int> de, d1, d2;
  std::vector<double> dsc;
  for (auto& kv : dual) {
    de.push_back(kv.first);
    d1.push_back(kv.second.first);
    d2.push_back(kv.second.second);
    dsc.push_back(dscale[kv.first]);
  }
  h->n_dual = (int64_t)de.size();
  // per (dual DOF position, cell) the signed multipliers of the copy and its scale: the
  // interface products of the tensor-core path read B^T lambda from it directly
  {
    const int nI = h->n_I, nD = h->n_R - h->n_I;
    std::vector<int2> lk((size_t)nD * ns, make_int2(0, 0));
    std::vector<float> lsc((size_t)nD * ns, 0.f);
    for (size_t q = 0; q < de.size(); ++q) {
      const int e = de[q], kl = e / ns, sc = e % ns;
      const int gk = rpos[kl] - nI;
      if (gk < 0) continue;   // a dual entry is a remaining, non-interior DOF
      lk[(size_t)gk * ns + sc] = make_int2(d1[q], d2[q]);
      lsc[(size_t)gk * ns + sc] = (float)dsc[q];
    }
    h->dual_lk.upload(lk, h->stream);
    h->dual_lsc.upload(lsc, h->stream);
  }
  h->dual_entry.upload(de, h->stream);
  h->dual_l1.upload(d1, h->stream);
  h->dual_l2.upload(d2, h->stream);
  h->dual_scale.upload(dsc, h->stream);
  h->n_krylov = (int64_t)nl * ns + h->n_primal + h->n_lambda;

  // coarse matrix entries (p, q) and their contributions (s, i, j), deterministic order
  std::map<std::pair<int, int>, std::vector<int>> ent;
  const int nP = h->n_P;
  for (int s = 0; s < ns; ++s)
    for (int i = 0; i < nP; ++i) {
      int p = pidx[(size_t)s * nP + i];
      if (p < 0) continue;
      for (int j = 0; j < nP; ++j) {
        int q = pidx[(size_t)s * nP + j];
        if (q < 0) continue;
        ent[{p, q}].push_back((s * nP + i) * nP + j);
      }
    }
  std::vector<int> crow, ccol, cptr2(1, 0), csrc;
  for (auto& kv : ent) {
    crow.push_back(kv.first.first);
    ccol.push_back(kv.first.second);
    for (int v : kv.second) csrc.push_back(v);
    cptr2.push_back((int)csrc.size());
  }
  h->coarse_row.upload(crow, h->stream);
  h->coarse_col.upload(ccol, h->stream);
  h->coarse_ptr.upload(cptr2, h->stream);
  h->coarse_src.upload(csrc, h->stream);

  // block-tridiagonal structure of the coarse matrix: a primal node belongs to the highest (or
  // the lowest) cell layer along the load axis among the cells that contain it; of the two
  // assignments the one with the smaller largest block is kept (a clamped face then adds no
  // DOFs to its layer, so the blocks come out of equal size)
  h->coarse_blocked = false;
  if (!h->h_cell_layer.empty() && h->n_primal > 0) {
    struct Blocking {
      std::vector<int> pb, pos;
      int N = 0, m = 0;
    };
    auto blocking = [&](bool highest) {
      std::vector<int> node_blk(h->n_glob_nodes, -1);
      for (int s = 0; s < ns; ++s)
        for (int a = 0; a < nn; ++a)
          if (corner[a] >= 0) {
            int& b = node_blk[cn[(size_t)s * nn + a]];
            const int l = (int)h->h_cell_layer[s];
            b = b < 0 ? l : (highest ? std::max(b, l) : std::min(b, l));
          }
      Blocking B;
      B.pb.resize(h->n_primal);
      for (int64_t p = 0; p < h->n_primal; ++p) B.pb[p] = node_blk[pglob[p] / d];
      std::vector<int> ub(B.pb);
      std::sort(ub.begin(), ub.end());
      ub.erase(std::unique(ub.begin(), ub.end()), ub.end());
      for (auto& b : B.pb) b = (int)(std::lower_bound(ub.begin(), ub.end(), b) - ub.begin());
      B.N = (int)ub.size();
      std::vector<int> cnt(B.N, 0);
      B.pos.resize(h->n_primal);
      for (int64_t p = 0; p < h->n_primal; ++p) B.pos[p] = cnt[B.pb[p]]++;
      B.m = *std::max_element(cnt.begin(), cnt.end());
      return B;
    };
    Blocking hi = blocking(true), lo = blocking(false);
    const Blocking& B = lo.m < hi.m ? lo : hi;
    // blocks padded to a multiple of 4 (identity on the padding): 16-byte rows for the sweeps
    // in FP64 and FP32
    const int N = B.N, m = (B.m + 3) & ~3;
    bool tri = N >= 2;
    std::vector<int64_t> dest(crow.size(), -1);
    const size_t mm = (size_t)m * m;
    for (size_t e = 0; e < crow.size() && tri; ++e) {
      const int bi = B.pb[crow[e]], bj = B.pb[ccol[e]];
      if (std::abs(bi - bj) > 1) tri = false;
      else if (bi == bj) dest[e] = (int64_t)(bi * mm + (size_t)B.pos[crow[e]] * m + B.pos[ccol[e]]);
      else if (bj == bi + 1) dest[e] = (int64_t)((N + bi) * mm + (size_t)B.pos[crow[e]] * m + B.pos[ccol[e]]);
    }
    // worth it when the blocks are much smaller than the whole coarse problem
    if (tri && (int64_t)m * 4 <= h->n_primal) {
      std::vector<int> perm((size_t)N * m, -1);
      for (int64_t p = 0; p < h->n_primal; ++p) perm[(size_t)B.pb[p] * m + B.pos[p]] = (int)p;
      h->cb_n = N;
      h->cb_m = m;
      h->cb_dest.upload(dest, h->stream);
      h->cb_perm.upload(perm, h->stream);
      h->coarse_blocked = true;
    }
  }
}

__global__ void k_predictor(int64_t n, double load, const double* __restrict__ up,
                            const double* __restrict__ up2, const double* __restrict__ aff,
                            const double* __restrict__ dir, const uint8_t* __restrict__ fixed,
                            double* __restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v;
  if (up == nullptr) v = load * aff[i];
  else v = 2.0 * up[i] - (up2 ? up2[i] : 0.0);
  if (fixed[i]) v = load * dir[i];
  out[i] = v;
}

__global__ void k_gather(int n_cells, int n_loc, int dim, int nn, const int* __restrict__ cell_nodes,
                         const double* __restrict__ u, double* __restrict__ x) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  int k = blockIdx.y;
  if (s >= n_cells) return;
  int a = k / dim, i = k - a * dim;
  x[(size_t)k * n_cells + s] = u[(int64_t)cell_nodes[(size_t)s * nn + a] * dim + i];
}

__global__ void k_set_mu(int n, double mu, const double* __restrict__ th, double* __restrict__ out) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) out[s] = mu * th[s];
}

}  // namespace

void build_feti(lat_ctx* h, int level) { build_feti_impl(h, level); }

static thread_local std::string g_setup_err;

extern "C" lat_status lattice_setup(const lat_mesh_desc* ds, lat_precision prec, void* stream,
                                    lat_handle* out) {
  if (!ds || !out) return LAT_EINVAL;
  lat_ctx* h = new lat_ctx();
  lat_status st = guard(h, [&] {
    LAT_REQUIRE(ds->dim == 2 || ds->dim == 3, LAT_EINVAL, "dim must be 2 or 3");
    LAT_REQUIRE(ds->n_cells > 0 && ds->n_nodes_cell > 0 && ds->n_el_cell > 0 && ds->n_glob_nodes > 0,
                LAT_EINVAL, "empty lattice");
    LAT_REQUIRE(ds->X_ref && ds->elems && ds->cell_nodes && ds->dof_fixed && ds->dirichlet_unit &&
                    ds->affine_unit, LAT_EINVAL, "missing lattice array");
    LAT_REQUIRE(prec >= LAT_FP64 && prec <= LAT_MIXED_BF16, LAT_EINVAL, "bad precision");
    LAT_REQUIRE((int64_t)ds->n_cells * ds->n_nodes_cell * ds->dim < (int64_t)1 << 31, LAT_EINVAL,
                "lattice too large for 32-bit local indexing");
    h->dim = ds->dim;
    h->nen = 1 << ds->dim;
    h->n_cells = ds->n_cells;
    h->n_nodes_cell = ds->n_nodes_cell;
    h->n_el = ds->n_el_cell;
    h->n_loc = ds->n_nodes_cell * ds->dim;
    h->n_glob_nodes = ds->n_glob_nodes;
    h->n_dof = ds->n_glob_nodes * ds->dim;
    h->mu = ds->mu;
    h->lam = ds->lam;
    h->prec = prec;
    h->stream = (cudaStream_t)stream;
    const char* vb = std::getenv("LATTICE_VERBOSE");
    h->verbose = vb && vb[0] == '1';
    int dev = 0;
    LAT_CUDA(cudaGetDevice(&dev));
    LAT_CUDA(cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev));
    for (int64_t i = 0; i < (int64_t)h->n_el * h->nen; ++i)
      LAT_REQUIRE(ds->elems[i] >= 0 && ds->elems[i] < h->n_nodes_cell, LAT_EINVAL, "elems out of range");
    std::vector<int> el(ds->elems, ds->elems + (size_t)h->n_el * h->nen);
    h->elems.upload(el, h->stream);
    build_geometry(h, ds->X_ref, ds->elems);
    build_pattern_and_colors(h, ds->elems);
    std::vector<int> cnv(ds->cell_nodes, ds->cell_nodes + (size_t)h->n_cells * h->n_nodes_cell);
    h->cell_nodes.upload(cnv, h->stream);
    h->h_dof_fixed.assign(ds->dof_fixed, ds->dof_fixed + h->n_dof);
    h->dof_fixed.upload(h->h_dof_fixed, h->stream);
    h->dir_unit.upload(std::vector<double>(ds->dirichlet_unit, ds->dirichlet_unit + h->n_dof), h->stream);
    h->aff_unit.upload(std::vector<double>(ds->affine_unit, ds->affine_unit + h->n_dof), h->stream);
    if (ds->cell_layer) h->h_cell_layer.assign(ds->cell_layer, ds->cell_layer + h->n_cells);
    build_maps(h, ds);
    build_feti_impl(h, 0);
    h->h_mu_scale.assign(h->n_cells, 1.0);
    if (ds->mu_scale) h->h_mu_scale.assign(ds->mu_scale, ds->mu_scale + h->n_cells);
    DBuf<double> th;
    th.upload(h->h_mu_scale, h->stream);
    h->mu_cell.ensure(h->n_cells);
    LAT_LAUNCH(h, k_set_mu<<<div_up(h->n_cells, 256), 256, 0, h->stream>>>(h->n_cells, h->mu, th.p, h->mu_cell.p));
    LAT_CHECK_LAUNCH();
    LAT_CUDA(cudaMallocHost(&h->h_pinned, 64 * sizeof(double)));
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    th.release();
  });
  if (st != LAT_OK) {
    g_setup_err = h->err;
    lattice_destroy(h);
    *out = nullptr;
    return st;
  }
  *out = h;
  return LAT_OK;
}

extern "C" lat_status lattice_destroy(lat_handle h) {
  if (!h) return LAT_OK;
  cudaStreamSynchronize(h->stream);
  drop_pcg_graph(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  // DBuf members free themselves through release(); walk them explicitly
  auto rel = [](auto& b) { b.release(); };
  rel(h->gradX[0]); rel(h->gradX[1]); rel(h->W[0]); rel(h->W[1]); rel(h->elems); rel(h->elem_blk);
  rel(h->color_elems); rel(h->blk_ptr); rel(h->blk_col); rel(h->cell_nodes); rel(h->mu_cell);
  rel(h->copy_ptr); rel(h->copy_idx); rel(h->dof_fixed); rel(h->dir_unit); rel(h->aff_unit);
  rel(h->corner_of_node); rel(h->rdofs); rel(h->pdofs); rel(h->rpos); rel(h->pidx);
  rel(h->p_copy_ptr); rel(h->p_copy); rel(h->loc_fixed); rel(h->lam_p); rel(h->lam_m);
  rel(h->dual_entry); rel(h->dual_l1); rel(h->dual_l2); rel(h->dual_scale); rel(h->dual_lk); rel(h->dual_lsc); rel(h->cell_class);
  rel(h->coarse_ptr); rel(h->coarse_src); rel(h->cb_dest); rel(h->cb_perm); rel(h->cb_A);
  rel(h->cb_Dinv); rel(h->cb_Einv); rel(h->cb_U); rel(h->cb_V); rel(h->cb_T); rel(h->cb_X); rel(h->cb_Ut); rel(h->cb_y); rel(h->cb_w); rel(h->coarse_row); rel(h->coarse_col);
  rel(h->S); rel(h->alpha); rel(h->alpha32); rel(h->Kp); rel(h->Kp32); rel(h->Kg);
  for (auto& g : h->ng) { rel(g.rows); rel(g.ucptr); rel(g.ucol); rel(g.pp); rel(g.pair_u); rel(g.perm); }
  rel(h->g_delta); rel(h->g_Z); rel(h->g_beta); rel(h->g_inf); rel(h->g_nrm2); rel(h->g_norms);
  rel(h->g_part); rel(h->g_maxres); rel(h->g_state); rel(h->g_scale);
  rel(h->f_cells); rel(h->r_glob); rel(h->minJ_cell); rel(h->T); rel(h->negJ);
  rel(h->key_of_cell); rel(h->key_slot); rel(h->perm); rel(h->seg_ptr); rel(h->tile_seg);
  rel(h->tile_c0); rel(h->key_list); rel(h->solver_int); rel(h->delta_cell); rel(h->c_cell);
  rel(h->G); rel(h->G16[0]); rel(h->G16[1]); rel(h->G16[2]); rel(h->G16[3]); rel(h->cb_U32); rel(h->cb_Ut32); rel(h->cb_Dinv32); rel(h->tile_seg_tc); rel(h->tile_c0_tc); rel(h->tP32); rel(h->Phi32); rel(h->SDD); rel(h->SDD32); rel(h->Phi); rel(h->Sloc); rel(h->G32); rel(h->Xb16); rel(h->KRP); rel(h->Coarse);
  rel(h->CoarseInv); rel(h->CoarseInv32); rel(h->pcg_ws); rel(h->tP); rel(h->gP); rel(h->xP); rel(h->x32); rel(h->y32);
  for (auto& b : h->kv_tmp) rel(b);
  rel(h->V); rel(h->Zk); rel(h->Hh); rel(h->gmres_small); rel(h->dots_part); rel(h->flag); rel(h->red_part);
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  for (auto& kv : h->ev)
    for (auto& pr : kv.second) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  delete h;
  return LAT_OK;
}

extern "C" const char* lattice_last_error(lat_handle h) {
  return h ? h->err.c_str() : g_setup_err.c_str();
}

extern "C" lat_status lattice_sizes(lat_handle h, lat_sizes* o) {
  if (!h || !o) return LAT_EINVAL;
  o->n_dof = h->n_dof;
  o->n_cells = h->n_cells;
  o->n_loc = h->n_loc;
  o->n_blocks = h->n_blk;
  o->nnz = h->nnz;
  o->n_r_local = h->n_R;
  o->n_p_local = h->n_P;
  o->n_primal = h->n_primal;
  o->n_lambda = h->n_lambda;
  o->n_krylov = h->n_krylov;
  o->n_q_full = h->nq[0] * h->n_el;
  o->n_q_reduced = h->nq[1] * h->n_el;
  o->n_i_local = h->n_I;
  o->n_coarse_blocks = h->coarse_blocked ? h->cb_n : 0;
  o->coarse_block = h->coarse_blocked ? h->cb_m : 0;
  o->coarse_block_lu = h->cb_solve ? 1 : 0;
  return LAT_OK;
}

extern "C" lat_status lattice_set_mu_scale(lat_handle h, const double* th) {
  if (!h || !th) return LAT_EINVAL;
  return guard(h, [&] {
    h->h_mu_scale.assign(th, th + h->n_cells);
    DBuf<double> t;
    t.upload(h->h_mu_scale, h->stream);
    LAT_LAUNCH(h, k_set_mu<<<div_up(h->n_cells, 256), 256, 0, h->stream>>>(h->n_cells, h->mu, t.p, h->mu_cell.p));
    LAT_CHECK_LAUNCH();
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    t.release();
  });
}

extern "C" lat_status lattice_predictor(lat_handle h, double load, const double* up,
                                        const double* up2, double* out) {
  if (!h || !out) return LAT_EINVAL;
  return guard(h, [&] {
    LAT_LAUNCH(h, k_predictor<<<div_up(h->n_dof, 256), 256, 0, h->stream>>>(h->n_dof, load, up, up2, h->aff_unit.p,
                                                             h->dir_unit.p, h->dof_fixed.p, out));
    LAT_CHECK_LAUNCH();
  });
}

extern "C" lat_status lattice_gather(lat_handle h, const double* u, double* x) {
  if (!h || !u || !x) return LAT_EINVAL;
  return guard(h, [&] {
    dim3 grid(div_up(h->n_cells, 128), h->n_loc);
    LAT_LAUNCH(h, k_gather<<<grid, 128, 0, h->stream>>>(h->n_cells, h->n_loc, h->dim, h->n_nodes_cell,
                                          h->cell_nodes.p, u, x));
    LAT_CHECK_LAUNCH();
  });
}

namespace {
const uint64_t kCkptMagic = 0x4c41544349434b50ull;  // "LATCICKP"
}

extern "C" lat_status lattice_checkpoint_save(lat_handle h, const char* path, int32_t step,
                                              double load, const double* u, const double* up) {
  if (!h || !path || !u) return LAT_EINVAL;
  return guard(h, [&] {
    std::vector<double> a(h->n_dof), b;
    LAT_CUDA(cudaMemcpyAsync(a.data(), u, h->n_dof * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (up) {
      b.resize(h->n_dof);
      LAT_CUDA(cudaMemcpyAsync(b.data(), up, h->n_dof * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    }
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    FILE* f = std::fopen(path, "wb");
    LAT_REQUIRE(f, LAT_EINVAL, std::string("cannot open ") + path);
    int64_t hdr[4] = {(int64_t)kCkptMagic, h->n_dof, step, up ? 1 : 0};
    bool ok = std::fwrite(hdr, sizeof(hdr), 1, f) == 1 && std::fwrite(&load, sizeof(double), 1, f) == 1 &&
              std::fwrite(a.data(), sizeof(double), a.size(), f) == a.size() &&
              (!up || std::fwrite(b.data(), sizeof(double), b.size(), f) == b.size());
    std::fclose(f);
    LAT_REQUIRE(ok, LAT_EINVAL, "checkpoint write failed");
  });
}

extern "C" lat_status lattice_checkpoint_load(lat_handle h, const char* path, int32_t* step,
                                              double* load, double* u, double* up) {
  if (!h || !path || !u || !step || !load) return LAT_EINVAL;
  return guard(h, [&] {
    FILE* f = std::fopen(path, "rb");
    LAT_REQUIRE(f, LAT_EINVAL, std::string("cannot open ") + path);
    int64_t hdr[4];
    bool ok = std::fread(hdr, sizeof(hdr), 1, f) == 1 && std::fread(load, sizeof(double), 1, f) == 1;
    ok = ok && hdr[0] == (int64_t)kCkptMagic && hdr[1] == h->n_dof;
    std::vector<double> a(h->n_dof), b;
    ok = ok && std::fread(a.data(), sizeof(double), a.size(), f) == a.size();
    if (ok && hdr[3]) {
      b.resize(h->n_dof);
      ok = std::fread(b.data(), sizeof(double), b.size(), f) == b.size();
    }
    std::fclose(f);
    LAT_REQUIRE(ok, LAT_EINVAL, "checkpoint does not match this lattice");
    *step = (int32_t)hdr[2];
    LAT_CUDA(cudaMemcpyAsync(u, a.data(), a.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (up) {
      if (hdr[3]) LAT_CUDA(cudaMemcpyAsync(up, b.data(), b.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
      else LAT_CUDA(cudaMemsetAsync(up, 0, h->n_dof * sizeof(double), h->stream));
    }
    LAT_CUDA(cudaStreamSynchronize(h->stream));
  });
}

extern "C" lat_status lattice_set_timing(lat_handle h, int32_t enable) {
  if (!h) return LAT_EINVAL;
  return guard(h, [&] {
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    for (auto& kv : h->ev)
      for (auto& pr : kv.second) {
        h->ev_pool.push_back(pr.first);
        h->ev_pool.push_back(pr.second);
      }
    h->ev.clear();
    LAT_REQUIRE(enable >= 0 && enable <= 2, LAT_EINVAL, "enable is 0, 1 or 2");
    h->timing = enable != 0;
    h->timing_apply_only = enable == 2;
  });
}

extern "C" lat_status lattice_kernel_time(lat_handle h, const char* name, double* total_ms, int32_t* launches) {
  if (!h || !name || !total_ms || !launches) return LAT_EINVAL;
  return guard(h, [&] {
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    double t = 0;
    int n = 0;
    auto it = h->ev.find(name);
    if (it != h->ev.end())
      for (auto& pr : it->second) {
        float ms = 0;
        LAT_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
        t += ms;
        ++n;
      }
    *total_ms = t;
    *launches = n;
  });
}

extern "C" lat_status lattice_launch_count(lat_handle h, int64_t* launches) {
  if (!h || !launches) return LAT_EINVAL;
  *launches = h->n_launch;
  return LAT_OK;
}
