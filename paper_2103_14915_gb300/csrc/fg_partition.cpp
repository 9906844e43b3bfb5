// Host-side graph partitioning (Def. 2.1): a division of V into |P| disjoint
// vertex sets of S vertices each (the last may be smaller).
//
// RANGE keeps the caller's id order: partition j is the id range [jS, (j+1)S).
// With randomly permuted ids this is the paper's random equal-vertex split for
// social graphs (Sec. 6.1). GROW grows each partition breadth-first from the
// smallest unassigned id until it holds S vertices; on road-like graphs it
// yields compact regions with few cut edges and stands in for the METIS
// edge-cut partitioning the paper applies to road networks (Sec. 6.1). DEGREE
// orders the vertices by out-degree, highest first, so the hubs of a
// power-law graph share partitions and the arcs among them stay inside one
// (a cheap ordering in the spirit of the locality-improving orderings the
// paper's partition study discusses, Sec. 6.4). Within a GROW partition,
// vertices are ordered by original id so that a partition's state maps to
// runs of consecutive ids in the caller's query-major arrays.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "fg_internal.h"

namespace fg {

// perm[i] = original id of internal vertex i. Returns false on bad arguments.
bool partition_plan_impl(int64_t n, const int64_t *row_ptr, const int32_t *col, int method, int S,
                         int32_t *perm) {
  if (n < 1 || S < 1 || !perm) return false;
  if (method == FG_PART_RANGE) {
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    return true;
  }
  if (method == FG_PART_DEGREE) {
    if (!row_ptr) return false;
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    std::stable_sort(perm, perm + n, [&](int32_t a, int32_t b) {
      return row_ptr[a + 1] - row_ptr[a] > row_ptr[b + 1] - row_ptr[b];
    });
    return true;
  }
  if (method != FG_PART_GROW || !row_ptr || !col) return false;
  std::vector<uint8_t> assigned((size_t)n, 0);
  std::vector<int32_t> queue;
  queue.reserve((size_t)S);
  int64_t next_seed = 0, k = 0;
  while (k < n) {
    const int64_t part_begin = k;
    const int64_t part_end = std::min<int64_t>(n, k + S);
    while (k < part_end) {
      while (next_seed < n && assigned[(size_t)next_seed]) ++next_seed;
      const int32_t seed = (int32_t)next_seed;
      queue.clear();
      queue.push_back(seed);
      assigned[(size_t)seed] = 1;
      perm[k++] = seed;
      for (size_t head = 0; head < queue.size() && k < part_end; ++head) {
        const int32_t v = queue[head];
        for (int64_t e = row_ptr[v]; e < row_ptr[v + 1] && k < part_end; ++e) {
          const int32_t u = col[e];
          if (assigned[(size_t)u]) continue;
          assigned[(size_t)u] = 1;
          queue.push_back(u);
          perm[k++] = u;
        }
      }
    }
    std::sort(perm + part_begin, perm + part_end);
  }
  return true;
}

// Arcs whose endpoints fall in different partitions under perm.
int64_t cut_arcs_impl(int64_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *perm, int slog2) {
  std::vector<int32_t> part((size_t)n);
  for (int64_t i = 0; i < n; ++i) part[(size_t)perm[i]] = (int32_t)(i >> slog2);
  int64_t cut = 0;
  for (int64_t v = 0; v < n; ++v)
    for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) cut += part[(size_t)v] != part[(size_t)col[e]];
  return cut;
}

}  // namespace fg
