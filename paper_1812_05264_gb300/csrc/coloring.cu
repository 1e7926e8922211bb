// Welsh-Powell colouring of the atoms (Sec. II.E) for the multi-colour probe ensemble of
// Sec. II.C.3.  Host code: it runs once per geometry on the colouring graph's CSR.
//
// Welsh & Powell (The Computer Journal 10, 85 (1967)) list the vertices by non-increasing
// degree and fill one colour class at a time down the list.  A vertex is skipped for class k
// exactly when an earlier-listed neighbour already has colour k, so the result equals first-fit
// greedy in list order: each vertex takes the smallest colour none of its earlier-listed
// neighbours has.  That form costs O(n + nnz): a counting sort gives the list, and a stamp per
// colour marks the colours seen around each vertex.
#include <algorithm>
#include <vector>

#include "common.cuh"

extern "C" int tbk_welsh_powell(int32_t n_atoms, const int32_t* row_ptr, const int32_t* col,
                                int32_t* color, int32_t* n_colors) {
  TBK_API_BEGIN
  TBK_CHECK_ARG(n_atoms >= 0, "n_atoms < 0");
  TBK_CHECK_ARG(row_ptr && color && n_colors, "null pointer");
  TBK_CHECK_ARG(row_ptr[0] == 0, "row_ptr[0] != 0");
  const int32_t n = n_atoms;
  for (int32_t v = 0; v < n; ++v)
    TBK_CHECK_ARG(row_ptr[v + 1] >= row_ptr[v], "row_ptr decreases");
  const int64_t nnz = row_ptr[n];
  TBK_CHECK_ARG(nnz == 0 || col, "null col");
  for (int64_t e = 0; e < nnz; ++e)
    TBK_CHECK_ARG(col[e] >= 0 && col[e] < n, "column index out of range");

  // columns ascending within a row; degrees without self entries; every pair in both rows
  std::vector<int32_t> deg(n, 0);
  for (int32_t v = 0; v < n; ++v)
    for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      TBK_CHECK_ARG(e == row_ptr[v] || col[e] > col[e - 1], "columns not ascending within a row");
      deg[v] += col[e] != v;
    }
  {
    // the transpose, built row by row, has ascending columns too: equal arrays <=> symmetric
    std::vector<int64_t> fill(row_ptr, row_ptr + n);
    std::vector<int32_t> colT(static_cast<size_t>(nnz));
    bool fits = true;
    for (int32_t v = 0; v < n && fits; ++v)
      for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
        const int32_t u = col[e];
        if (fill[u] == row_ptr[u + 1]) { fits = false; break; }
        colT[fill[u]++] = v;
      }
    TBK_CHECK_ARG(fits && std::equal(colT.begin(), colT.end(), col), "a pair is listed in one row only");
  }

  // the list: counting sort by degree, largest first, index order within a degree
  int32_t dmax = 0;
  for (int32_t v = 0; v < n; ++v) dmax = std::max(dmax, deg[v]);
  std::vector<int64_t> start(static_cast<size_t>(dmax) + 2, 0);
  for (int32_t v = 0; v < n; ++v) ++start[dmax - deg[v] + 1];
  for (int32_t d = 0; d <= dmax; ++d) start[d + 1] += start[d];
  std::vector<int32_t> order(n);
  for (int32_t v = 0; v < n; ++v) order[start[dmax - deg[v]]++] = v;

  // first fit down the list
  std::vector<int32_t> c(n, -1);
  std::vector<int32_t> stamp(static_cast<size_t>(dmax) + 1, -1);  // colour k last seen around vertex stamp[k]
  int32_t q = 0;
  for (int32_t v : order) {
    for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      const int32_t k = c[col[e]];
      if (k >= 0) stamp[k] = v;      // a coloured neighbour is an earlier-listed one
    }
    int32_t k = 0;
    while (stamp[k] == v) ++k;       // at most deg[v] colours are taken, so k <= dmax
    c[v] = k;
    q = std::max(q, k + 1);
  }
  std::copy(c.begin(), c.end(), color);
  *n_colors = q;
  TBK_API_END
}
