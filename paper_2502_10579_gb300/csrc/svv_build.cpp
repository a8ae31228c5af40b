// svv_build.cpp -- host builder of the versioned union graph (Section 4.1):
// one edge per live edge instance, grouped by source, with a presence mask of
// ceil(S/64) words per edge (bit i = live in snapshot i).
#include <cstdint>
#include <vector>

#include "../../include/svv.h"

extern "C" svv_status svv_build_versioned_csr(uint32_t V, uint32_t S, uint64_t n_inst, const uint32_t* src,
                                              const uint32_t* dst, const uint32_t* w, const uint32_t* t_add,
                                              const uint32_t* t_del, uint64_t* row_ptr, uint32_t* col,
                                              uint32_t* weight, uint64_t* mask, uint64_t* E_out) {
  if (V == 0 || S == 0 || !row_ptr || !E_out) return SVV_EINVAL;
  if (n_inst && (!src || !dst || !w || !t_add || !t_del || !col || !weight || !mask)) return SVV_EINVAL;
  const uint32_t W = (S + 63) / 64;
  for (uint64_t k = 0; k < n_inst; ++k)
    if (src[k] >= V || dst[k] >= V || t_add[k] > S || t_del[k] > S) return SVV_EINVAL;
  for (uint32_t v = 0; v <= V; ++v) row_ptr[v] = 0;
  for (uint64_t k = 0; k < n_inst; ++k)
    if (t_add[k] < t_del[k]) row_ptr[src[k] + 1]++;
  for (uint32_t v = 0; v < V; ++v) row_ptr[v + 1] += row_ptr[v];
  std::vector<uint64_t> fill(row_ptr, row_ptr + V);
  for (uint64_t k = 0; k < n_inst; ++k) {
    if (t_add[k] >= t_del[k]) continue;
    const uint64_t p = fill[src[k]]++;
    col[p] = dst[k];
    weight[p] = w[k];
    uint64_t* m = mask + p * W;
    for (uint32_t j = 0; j < W; ++j) {
      // bits [t_add, t_del) restricted to word j
      const uint32_t lo = t_add[k] > 64 * j ? t_add[k] : 64 * j;
      const uint32_t hi = t_del[k] < 64 * j + 64 ? t_del[k] : 64 * j + 64;
      uint64_t x = 0;
      if (lo < hi) {
        const uint32_t n = hi - lo;
        x = (n == 64 ? ~0ull : ((1ull << n) - 1ull)) << (lo - 64 * j);
      }
      m[j] = x;
    }
  }
  *E_out = row_ptr[V];
  return SVV_OK;
}
