// Internal declarations shared by the host assembly (mesh.cpp) and the device path (sim.cu).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tc.h"

namespace tc {

// Thread-local error message plus status.
tc_status fail(tc_status st, const std::string& msg);
void clear_error();

// Host CSR pattern + values in the caller's node order.
struct Csr {
  int64_t n = 0;
  std::vector<int64_t> row_ptr;   // n+1
  std::vector<int32_t> col;       // nnz, sorted per row, diagonal included
};

}  // namespace tc

struct tc_mesh {
  int64_t n = 0, ne = 0;
  std::vector<double> xyz;        // n*3
  std::vector<int32_t> tets;      // ne*4
  std::vector<double> fib;        // ne*3 unit fibres
  std::vector<int32_t> region;    // ne
  int32_t max_region = 0;
  // per-element geometry (computed once at creation)
  std::vector<double> vol;        // ne
  std::vector<double> grad;       // ne*12: grad l_0..l_3 (x,y,z each)
  // node -> incident elements (element id ascending), slots e*4+a
  std::vector<int64_t> inc_ptr;   // n+1
  std::vector<int32_t> inc;       // 4*ne entries: e*4 + a (node is vertex a of element e)
  tc::Csr pattern;
  int32_t sell_sigma = 0;         // SELL row-sorting window for simulations assembled from it (0: 1024)
};

namespace tc {

// Assemble M and K on the mesh pattern (caller order).  sigma arrays are per region.
tc_status assemble_mk(const tc_mesh& m, const double* sigma_l, const double* sigma_t,
                      int32_t n_regions, std::vector<double>& mval, std::vector<double>& kval);

// Reverse Cuthill-McKee order of the pattern graph, component by component, then a stable
// descending sort of row lengths inside windows of `sell_sigma` rows that never cross a
// component.  perm[new] = old; comp_start (if not null) receives the first position of every
// connected component in that order plus n at the end.
void node_ordering(const Csr& pat, int32_t sell_sigma, std::vector<int32_t>& perm,
                   std::vector<int64_t>* comp_start = nullptr);

// Internal device order: the node ordering with every connected component padded to a multiple
// of 32 rows by inert dummy rows, so that no 32-row SELL slice holds two components.
// perm_ext[internal] = caller index or -1 (dummy); comp_rows[c] = first internal row of
// component c, comp_rows[n_comp] = internal row count.
void padded_ordering(const Csr& pat, int32_t sell_sigma, std::vector<int32_t>& perm_ext,
                     std::vector<int64_t>& comp_rows);

// SELL-C-sigma layout (C = 32) of the pattern permuted by perm (perm[new] = old, or -1 for a
// dummy row, which gets no entries).
struct Sell {
  int64_t n = 0, nslices = 0, padded = 0;
  std::vector<int32_t> slice_ptr;   // nslices+1, offsets in entries (multiples of 32)
  std::vector<int32_t> col;         // padded, new indices
  std::vector<int64_t> src;         // padded, index into the caller-order CSR value array or -1
};
tc_status build_sell(const Csr& pat, const std::vector<int32_t>& perm, Sell& out);

}  // namespace tc
