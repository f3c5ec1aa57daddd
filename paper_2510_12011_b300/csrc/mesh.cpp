// Host side of the boundary: mesh ingest, P1 assembly on the mesh pattern, node ordering
// (reverse Cuthill-McKee, Section 2.2) and the SELL-C-sigma layout the device kernels read.
//
// Assembly is deterministic without atomics or a global sort: the pattern is the set of node
// pairs that share an element, and every row gathers the contributions of its incident
// elements in ascending element order, so entry (i,j) and entry (j,i) are sums of the same
// terms in the same order (K and M come out exactly symmetric).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <numeric>
#include <string>
#include <vector>

#include "tc_internal.h"

namespace tc {

static thread_local std::string g_err;

tc_status fail(tc_status st, const std::string& msg) {
  g_err = msg;
  return st;
}
void clear_error() { g_err.clear(); }
const char* last_error_cstr() { return g_err.c_str(); }

// Element geometry.  With edges e1 = x1-x0, e2 = x2-x0, e3 = x3-x0 and D = e1.(e2 x e3), the
// barycentric gradients are grad l1 = (e2 x e3)/D, grad l2 = (e3 x e1)/D, grad l3 = (e1 x e2)/D
// (the rows of the inverse of [e1 e2 e3]) and grad l0 = -(grad l1 + grad l2 + grad l3);
// the volume is |D|/6.
static inline void cross(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

static tc_status element_geometry(tc_mesh& m) {
  m.vol.assign(m.ne, 0.0);
  m.grad.assign(m.ne * 12, 0.0);
  int64_t bad = -1;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < m.ne; ++e) {
    const int32_t* t = &m.tets[e * 4];
    const double* x0 = &m.xyz[3 * (int64_t)t[0]];
    double ed[3][3];
    double lmax2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      const double* xk = &m.xyz[3 * (int64_t)t[k + 1]];
      for (int d = 0; d < 3; ++d) ed[k][d] = xk[d] - x0[d];
      lmax2 = std::max(lmax2, ed[k][0] * ed[k][0] + ed[k][1] * ed[k][1] + ed[k][2] * ed[k][2]);
    }
    double c23[3], c31[3], c12[3];
    cross(ed[1], ed[2], c23);
    cross(ed[2], ed[0], c31);
    cross(ed[0], ed[1], c12);
    const double D = ed[0][0] * c23[0] + ed[0][1] * c23[1] + ed[0][2] * c23[2];
    const double lmax3 = lmax2 * std::sqrt(lmax2);
    if (!(std::fabs(D) > 1e-12 * lmax3)) {
#pragma omp critical
      { if (bad < 0 || e < bad) bad = e; }
      continue;
    }
    double* g = &m.grad[e * 12];
    for (int d = 0; d < 3; ++d) {
      g[3 + d] = c23[d] / D;
      g[6 + d] = c31[d] / D;
      g[9 + d] = c12[d] / D;
      g[d] = -(g[3 + d] + g[6 + d] + g[9 + d]);
    }
    m.vol[e] = std::fabs(D) / 6.0;
  }
  if (bad >= 0) return fail(TC_ERR_MESH, "degenerate tetrahedron " + std::to_string(bad));
  return TC_OK;
}

static void build_incidence_and_pattern(tc_mesh& m) {
  const int64_t n = m.n;
  m.inc_ptr.assign(n + 1, 0);
  for (int64_t s = 0; s < 4 * m.ne; ++s) m.inc_ptr[m.tets[s] + 1]++;
  for (int64_t i = 0; i < n; ++i) m.inc_ptr[i + 1] += m.inc_ptr[i];
  m.inc.assign(4 * m.ne, 0);
  std::vector<int64_t> fill(m.inc_ptr.begin(), m.inc_ptr.end() - 1);
  for (int64_t s = 0; s < 4 * m.ne; ++s) m.inc[fill[m.tets[s]]++] = (int32_t)s;  // ascending e

  // pattern: sorted union of the vertices of the incident elements
  std::vector<std::vector<int32_t>> rows(n);
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n; ++i) {
    std::vector<int32_t>& r = rows[i];
    r.reserve(32);
    for (int64_t q = m.inc_ptr[i]; q < m.inc_ptr[i + 1]; ++q) {
      const int64_t e = m.inc[q] >> 2;
      for (int b = 0; b < 4; ++b) r.push_back(m.tets[e * 4 + b]);
    }
    if (r.empty()) r.push_back((int32_t)i);   // isolated node: keep its diagonal
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
  }
  Csr& p = m.pattern;
  p.n = n;
  p.row_ptr.assign(n + 1, 0);
  for (int64_t i = 0; i < n; ++i) p.row_ptr[i + 1] = p.row_ptr[i] + (int64_t)rows[i].size();
  p.col.resize(p.row_ptr[n]);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    std::copy(rows[i].begin(), rows[i].end(), p.col.begin() + p.row_ptr[i]);
}

tc_status assemble_mk(const tc_mesh& m, const double* sigma_l, const double* sigma_t,
                      int32_t n_regions, std::vector<double>& mval, std::vector<double>& kval) {
  if (!sigma_l || !sigma_t) return fail(TC_ERR_ARG, "sigma_l/sigma_t must not be NULL");
  if (n_regions <= m.max_region)
    return fail(TC_ERR_ARG, "n_regions (" + std::to_string(n_regions) +
                                ") must exceed the largest region id (" +
                                std::to_string(m.max_region) + ")");
  for (int32_t r = 0; r < n_regions; ++r)
    if (!(sigma_l[r] >= 0.0) || !(sigma_t[r] >= 0.0) || !std::isfinite(sigma_l[r]) ||
        !std::isfinite(sigma_t[r]))
      return fail(TC_ERR_ARG, "conductivities must be finite and >= 0");
  const Csr& p = m.pattern;
  const int64_t nnz = p.row_ptr[m.n];
  mval.assign(nnz, 0.0);
  kval.assign(nnz, 0.0);
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < m.n; ++i) {
    const int32_t* cb = &p.col[p.row_ptr[i]];
    const int64_t len = p.row_ptr[i + 1] - p.row_ptr[i];
    double* mr = &mval[p.row_ptr[i]];
    double* kr = &kval[p.row_ptr[i]];
    for (int64_t q = m.inc_ptr[i]; q < m.inc_ptr[i + 1]; ++q) {
      const int64_t e = m.inc[q] >> 2;
      const int a = m.inc[q] & 3;
      const double* g = &m.grad[e * 12];
      const double* f = &m.fib[e * 3];
      const double sl = sigma_l[m.region[e]], st = sigma_t[m.region[e]];
      const double v = m.vol[e];
      const double gaf = g[3 * a] * f[0] + g[3 * a + 1] * f[1] + g[3 * a + 2] * f[2];
      for (int b = 0; b < 4; ++b) {
        const int32_t j = m.tets[e * 4 + b];
        const int64_t pos = std::lower_bound(cb, cb + len, j) - cb;
        const double gbf = g[3 * b] * f[0] + g[3 * b + 1] * f[1] + g[3 * b + 2] * f[2];
        const double gab = g[3 * a] * g[3 * b] + g[3 * a + 1] * g[3 * b + 1] + g[3 * a + 2] * g[3 * b + 2];
        // grad l_a^T (st I + (sl - st) f f^T) grad l_b
        kr[pos] += v * (st * gab + (sl - st) * (gaf * gbf));
        mr[pos] += v * (a == b ? 2.0 : 1.0) / 20.0;
      }
    }
  }
  return TC_OK;
}

// ---- ordering ---------------------------------------------------------------------------

static void bfs_levels(const Csr& p, int32_t start, std::vector<int32_t>& level,
                       std::vector<int32_t>& last_level, int32_t& depth) {
  level[start] = 0;
  std::vector<int32_t> frontier{start}, touched{start};
  depth = 0;
  last_level = frontier;
  while (!frontier.empty()) {
    std::vector<int32_t> next;
    for (int32_t u : frontier)
      for (int64_t q = p.row_ptr[u]; q < p.row_ptr[u + 1]; ++q) {
        const int32_t v = p.col[q];
        if (level[v] < 0) {
          level[v] = depth + 1;
          next.push_back(v);
          touched.push_back(v);
        }
      }
    if (next.empty()) break;
    ++depth;
    last_level = next;
    frontier.swap(next);
  }
  for (int32_t t : touched) level[t] = -1;
}

void node_ordering(const Csr& p, int32_t sell_sigma, std::vector<int32_t>& perm,
                   std::vector<int64_t>* comp_start) {
  const int64_t n = p.n;
  std::vector<int32_t> deg(n);
  for (int64_t i = 0; i < n; ++i) deg[i] = (int32_t)(p.row_ptr[i + 1] - p.row_ptr[i]);
  std::vector<char> done(n, 0);
  std::vector<int32_t> level(n, -1), order;
  std::vector<int64_t> ends;   // end position of every component in the forward order
  order.reserve(n);
  for (int64_t seed = 0; seed < n; ++seed) {
    if (done[seed]) continue;
    // pseudo-peripheral start node (George & Liu): move to the smallest-degree node of the
    // last BFS level while the eccentricity grows
    int32_t start = (int32_t)seed, depth = -1;
    std::vector<int32_t> last;
    for (int round = 0; round < 8; ++round) {
      int32_t d;
      bfs_levels(p, start, level, last, d);
      if (d <= depth) break;
      depth = d;
      int32_t best = last[0];
      for (int32_t v : last)
        if (deg[v] < deg[best] || (deg[v] == deg[best] && v < best)) best = v;
      if (best == start) break;
      start = best;
    }
    // Cuthill-McKee BFS, neighbours by ascending (degree, index)
    std::deque<int32_t> queue{start};
    done[start] = 1;
    std::vector<int32_t> nb;
    while (!queue.empty()) {
      const int32_t u = queue.front();
      queue.pop_front();
      order.push_back(u);
      nb.clear();
      for (int64_t q = p.row_ptr[u]; q < p.row_ptr[u + 1]; ++q)
        if (!done[p.col[q]]) nb.push_back(p.col[q]);
      std::sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) {
        return deg[a] != deg[b] ? deg[a] < deg[b] : a < b;
      });
      for (int32_t v : nb) {
        done[v] = 1;
        queue.push_back(v);
      }
    }
    ends.push_back((int64_t)order.size());
  }
  std::reverse(order.begin(), order.end());
  // component starts in the reversed order
  std::vector<int64_t> starts;
  for (auto it = ends.rbegin(); it != ends.rend(); ++it) starts.push_back(n - *it);
  starts.push_back(n);
  if (sell_sigma > 1) {
    for (size_t c = 0; c + 1 < starts.size(); ++c)
      for (int64_t w0 = starts[c]; w0 < starts[c + 1]; w0 += sell_sigma) {
        const int64_t w1 = std::min<int64_t>(starts[c + 1], w0 + sell_sigma);
        std::stable_sort(order.begin() + w0, order.begin() + w1,
                         [&](int32_t a, int32_t b) { return deg[a] > deg[b]; });
      }
  }
  perm.swap(order);
  if (comp_start) comp_start->swap(starts);
}

void padded_ordering(const Csr& p, int32_t sell_sigma, std::vector<int32_t>& perm_ext,
                     std::vector<int64_t>& comp_rows) {
  std::vector<int32_t> perm;
  std::vector<int64_t> starts;
  node_ordering(p, sell_sigma, perm, &starts);
  const size_t nc = starts.size() - 1;
  comp_rows.assign(nc + 1, 0);
  for (size_t c = 0; c < nc; ++c) {
    const int64_t len = starts[c + 1] - starts[c];
    comp_rows[c + 1] = comp_rows[c] + (len + 31) / 32 * 32;
  }
  perm_ext.assign(comp_rows[nc], -1);
  for (size_t c = 0; c < nc; ++c)
    for (int64_t t = 0; t < starts[c + 1] - starts[c]; ++t)
      perm_ext[comp_rows[c] + t] = perm[starts[c] + t];
}

tc_status build_sell(const Csr& p, const std::vector<int32_t>& perm, Sell& s) {
  const int64_t n = (int64_t)perm.size();   // rows of the layout (dummy rows included)
  std::vector<int32_t> inv(p.n, -1);
  for (int64_t k = 0; k < n; ++k)
    if (perm[k] >= 0) inv[perm[k]] = (int32_t)k;
  auto row_len = [&](int64_t r) -> int64_t {
    const int32_t o = perm[r];
    return o < 0 ? 0 : p.row_ptr[o + 1] - p.row_ptr[o];
  };
  s.n = n;
  s.nslices = (n + 31) / 32;
  s.slice_ptr.assign(s.nslices + 1, 0);
  int64_t off = 0;
  for (int64_t sl = 0; sl < s.nslices; ++sl) {
    int64_t w = 0;
    for (int64_t r = sl * 32; r < std::min<int64_t>(n, sl * 32 + 32); ++r) w = std::max(w, row_len(r));
    off += 32 * w;
    if (off > INT32_MAX) return fail(TC_ERR_ARG, "matrix too large for 32-bit SELL offsets");
    s.slice_ptr[sl + 1] = (int32_t)off;
  }
  s.padded = off;
  s.col.assign(off, 0);
  s.src.assign(off, -1);
#pragma omp parallel for schedule(static)
  for (int64_t sl = 0; sl < s.nslices; ++sl) {
    std::vector<std::pair<int32_t, int64_t>> ent;
    const int64_t w = (s.slice_ptr[sl + 1] - s.slice_ptr[sl]) / 32;
    for (int lane = 0; lane < 32; ++lane) {
      const int64_t r = sl * 32 + lane;
      ent.clear();
      int32_t pad_col = (int32_t)std::min<int64_t>(r, n - 1);
      if (r < n && perm[r] >= 0) {
        const int32_t o = perm[r];
        for (int64_t q = p.row_ptr[o]; q < p.row_ptr[o + 1]; ++q) ent.push_back({inv[p.col[q]], q});
        std::sort(ent.begin(), ent.end());
      }
      for (int64_t j = 0; j < w; ++j) {
        const int64_t dst = s.slice_ptr[sl] + j * 32 + lane;
        if (j < (int64_t)ent.size()) {
          s.col[dst] = ent[j].first;
          s.src[dst] = ent[j].second;
        } else {
          s.col[dst] = pad_col;   // padding reads a valid, nearby entry and multiplies by 0
          s.src[dst] = -1;
        }
      }
    }
  }
  return TC_OK;
}

}  // namespace tc

using namespace tc;

extern "C" {

tc_status tc_mesh_create(const double* xyz, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                         const double* fibres, const int32_t* region, tc_mesh** out) {
  clear_error();
  if (!out) return fail(TC_ERR_ARG, "out must not be NULL");
  *out = nullptr;
  if (!xyz || !tets) return fail(TC_ERR_ARG, "xyz and tets must not be NULL");
  if (n_nodes < 4 || n_tets < 1) return fail(TC_ERR_ARG, "need at least 4 nodes and 1 tetrahedron");
  if (n_nodes > INT32_MAX - 64 || n_tets > INT32_MAX / 4)
    return fail(TC_ERR_ARG, "mesh too large for 32-bit indices");
  tc_mesh* m = new (std::nothrow) tc_mesh();
  if (!m) return fail(TC_ERR_NOMEM, "out of host memory");
  try {
    m->n = n_nodes;
    m->ne = n_tets;
    m->xyz.assign(xyz, xyz + 3 * n_nodes);
    m->tets.assign(tets, tets + 4 * n_tets);
    for (int64_t s = 0; s < 4 * n_tets; ++s)
      if (m->tets[s] < 0 || m->tets[s] >= n_nodes) {
        delete m;
        return fail(TC_ERR_MESH, "tetrahedron " + std::to_string(s / 4) + " has node index " +
                                     std::to_string(tets[s]) + " out of range");
      }
    for (int64_t i = 0; i < 3 * n_nodes; ++i)
      if (!std::isfinite(xyz[i])) {
        delete m;
        return fail(TC_ERR_MESH, "non-finite node coordinate");
      }
    m->fib.resize(3 * n_tets);
    for (int64_t e = 0; e < n_tets; ++e) {
      double f[3] = {1.0, 0.0, 0.0};
      if (fibres) {
        f[0] = fibres[3 * e];
        f[1] = fibres[3 * e + 1];
        f[2] = fibres[3 * e + 2];
      }
      const double nrm = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
      if (!(nrm > 0.0) || !std::isfinite(nrm)) {
        delete m;
        return fail(TC_ERR_MESH, "zero or non-finite fibre on element " + std::to_string(e));
      }
      for (int d = 0; d < 3; ++d) m->fib[3 * e + d] = f[d] / nrm;
    }
    m->region.assign(n_tets, 0);
    if (region) {
      for (int64_t e = 0; e < n_tets; ++e) {
        if (region[e] < 0) {
          delete m;
          return fail(TC_ERR_ARG, "negative region id");
        }
        m->region[e] = region[e];
        m->max_region = std::max(m->max_region, region[e]);
      }
    }
    tc_status st = element_geometry(*m);
    if (st != TC_OK) {
      delete m;
      return st;
    }
    build_incidence_and_pattern(*m);
  } catch (const std::bad_alloc&) {
    delete m;
    return fail(TC_ERR_NOMEM, "out of host memory");
  }
  *out = m;
  return TC_OK;
}

void tc_mesh_destroy(tc_mesh* mesh) { delete mesh; }

tc_status tc_mesh_nnz(const tc_mesh* mesh, int64_t* nnz) {
  clear_error();
  if (!mesh || !nnz) return fail(TC_ERR_ARG, "null argument");
  *nnz = mesh->pattern.row_ptr[mesh->n];
  return TC_OK;
}

tc_status tc_mesh_matrices(const tc_mesh* mesh, const double* sigma_l, const double* sigma_t,
                           int32_t n_regions, int64_t* row_ptr, int32_t* col, double* m_val,
                           double* k_val) {
  clear_error();
  if (!mesh) return fail(TC_ERR_ARG, "mesh must not be NULL");
  const Csr& p = mesh->pattern;
  if (row_ptr) std::copy(p.row_ptr.begin(), p.row_ptr.end(), row_ptr);
  if (col) std::copy(p.col.begin(), p.col.end(), col);
  if (m_val || k_val) {
    std::vector<double> mv, kv;
    try {
      tc_status st = assemble_mk(*mesh, sigma_l, sigma_t, n_regions, mv, kv);
      if (st != TC_OK) return st;
    } catch (const std::bad_alloc&) {
      return fail(TC_ERR_NOMEM, "out of host memory");
    }
    if (m_val) std::copy(mv.begin(), mv.end(), m_val);
    if (k_val) std::copy(kv.begin(), kv.end(), k_val);
  }
  return TC_OK;
}

tc_status tc_monodomain_conductivity(const double* il, const double* it, const double* el, const double* et,
                                     int32_t n, double* sl, double* st) {
  clear_error();
  if (!il || !it || !el || !et || !sl || !st || n < 1) return fail(TC_ERR_ARG, "bad conductivity arguments");
  for (int32_t r = 0; r < n; ++r)
    if (!(il[r] > 0 && it[r] > 0 && el[r] > 0 && et[r] > 0) || !std::isfinite(il[r] + it[r] + el[r] + et[r]))
      return fail(TC_ERR_ARG, "conductivities must be finite and > 0 (region " + std::to_string(r) + ")");
  for (int32_t r = 0; r < n; ++r) {
    sl[r] = il[r] * el[r] / (il[r] + el[r]);
    st[r] = it[r] * et[r] / (it[r] + et[r]);
  }
  return TC_OK;
}

tc_status tc_mesh_layout_size(const tc_mesh* mesh, int32_t* n_components, int64_t* n_internal) {
  clear_error();
  if (!mesh) return fail(TC_ERR_ARG, "mesh must not be NULL");
  std::vector<int32_t> pe;
  std::vector<int64_t> cr;
  padded_ordering(mesh->pattern, 1, pe, cr);
  if (n_components) *n_components = (int32_t)(cr.size() - 1);
  if (n_internal) *n_internal = cr.back();
  return TC_OK;
}

tc_status tc_mesh_set_sell_sigma(tc_mesh* mesh, int32_t sell_sigma) {
  clear_error();
  if (!mesh) return fail(TC_ERR_ARG, "mesh must not be NULL");
  if (sell_sigma < 1) return fail(TC_ERR_ARG, "sell_sigma must be >= 1");
  mesh->sell_sigma = sell_sigma;
  return TC_OK;
}

tc_status tc_mesh_ordering(const tc_mesh* mesh, int32_t sell_sigma, int32_t* perm,
                           int32_t* slice_width) {
  clear_error();
  if (!mesh || !perm) return fail(TC_ERR_ARG, "null argument");
  if (sell_sigma < 1) return fail(TC_ERR_ARG, "sell_sigma must be >= 1");
  std::vector<int32_t> pe;
  std::vector<int64_t> cr;
  padded_ordering(mesh->pattern, sell_sigma, pe, cr);
  int64_t k = 0;
  for (int32_t o : pe)
    if (o >= 0) perm[k++] = o;
  if (slice_width) {
    Sell s;
    tc_status st = build_sell(mesh->pattern, pe, s);
    if (st != TC_OK) return st;
    for (int64_t q = 0; q < s.nslices; ++q) slice_width[q] = (s.slice_ptr[q + 1] - s.slice_ptr[q]) / 32;
  }
  return TC_OK;
}

const char* tc_last_error(void) { return tc::last_error_cstr(); }

}  // extern "C"
