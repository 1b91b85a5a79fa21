// Work lists for the tensor-core kernel's explicit-list modes.
//
// Small batches cut a row tile whose k-range is longer than S k-blocks into
// chunks of at most S, so no single work item holds back the launch.  S
// depends only on N' (not on K), so the split of a given column is the same
// in every batch.  Chunks of one row tile write their accumulator pairs to
// consecutive slots; one SplitUnit per split tile tells k_split_reduce which
// slots to add.  With all_slots every row tile, split or not, leaves its
// accumulators to the reduction (the refinement step reads W itself).
#include <algorithm>
#include <cstring>
#include <vector>

#include "td_internal.h"

namespace td {

int split_chunk(int64_t nk, int64_t nkp, int bn) {
  const int64_t nm = nkp / bn;
  const int64_t per = bn / OP_KB;
  const int64_t nkb_max = ceil_div(nk, OP_KB);
  int64_t total = 0;
  for (int64_t m = 0; m < nm; ++m) total += std::min<int64_t>(per * (m + 1), nkb_max);
  int64_t S = ceil_div(total, 2 * (int64_t)tc_num_sms());
  if (S < 4) S = 4;
  return (int)S;
}

// append the items of one segment (bn-row tiles, column tiles of `cols`,
// chunk S) to the lists.  The column tiles of one (row tile, chunk) are
// emitted next to each other: the kernel hands out neighbouring items in the
// same round, so those CTAs stream the same operator chunk together and all
// but the first read it from L2 (an operator larger than L2 would otherwise
// come from HBM once per column tile).  A unit's chunks still take
// consecutive slots.
void plan_split_segment(int seg, int64_t nk, int64_t nkp, int64_t K, int bn, int S, std::vector<TcItem>& items,
                        std::vector<SplitUnit>& units, int& n_slots, bool all_slots, int cols) {
  const int nm = (int)(nkp / bn);
  const int per = bn / OP_KB;
  const int nc = (int)ceil_div(K, cols);
  const int nkb_max = (int)ceil_div(nk, OP_KB);
  for (int m = 0; m < nm; ++m) {
    const int nkb = std::min(per * (m + 1), nkb_max);
    const int nch = (nkb + S - 1) / S;
    if (nch <= 1 && !all_slots) {
      for (int c = 0; c < nc; ++c) items.push_back(TcItem{seg, m, c, nkb, 0, -1, -1});
      continue;
    }
    // chunks of exactly S k-blocks and one shorter remainder: the remainders
    // fill the gaps of the longest-first schedule
    const int unit0 = (int)units.size();
    const int slot_base = n_slots;
    for (int c = 0; c < nc; ++c) units.push_back(SplitUnit{seg, m, c, slot_base + c * nch, nch, 0});
    for (int ch = 0; ch < nch; ++ch) {
      const int kb0 = ch * S;
      for (int c = 0; c < nc; ++c)
        items.push_back(TcItem{seg, m, c, std::min(S, nkb - kb0), kb0, slot_base + c * nch + ch, unit0 + c});
    }
    n_slots += nc * nch;
  }
}

void sort_items(std::vector<TcItem>& items) {
  std::stable_sort(items.begin(), items.end(), [](const TcItem& a, const TcItem& b) { return a.nkb > b.nkb; });
}

// Segment by segment (most work first), each segment's items longest first
// with the column tiles of a row tile (or chunk) kept together.  Taken in
// this order by the dynamic schedule, the CTAs at work at any time share a
// few segments, so each segment's residual slices are read from HBM about
// once per pass of the CTAs over it and then from L2 by its other row tiles.
void sort_items_by_segment(std::vector<TcItem>& items, int nseg) {
  std::vector<int64_t> work((size_t)nseg, 0);
  for (const TcItem& it : items) work[(size_t)it.seg] += it.nkb;
  std::stable_sort(items.begin(), items.end(), [&](const TcItem& a, const TcItem& b) {
    if (a.seg != b.seg) {
      const int64_t wa = work[(size_t)a.seg], wb = work[(size_t)b.seg];
      return wa != wb ? wa > wb : a.seg < b.seg;
    }
    return a.nkb > b.nkb;
  });
}

}  // namespace td

extern "C" int td_debug_plan(const int64_t* nk, const int64_t* K, int nseg, int bn, int S, int by_segment, int* out,
                             int cap) {
  using namespace td;
  if (!nk || !K || nseg <= 0 || (bn != 256 && bn != 128 && bn != 64) || S < 1 || cap < 0) return -1;
  std::vector<TcItem> items;
  std::vector<SplitUnit> units;
  int n_slots = 0;
  for (int i = 0; i < nseg; ++i) {
    if (nk[i] < 1 || K[i] < 0) return -1;
    plan_split_segment(i, nk[i], round_up(nk[i], OP_ROWS), K[i], bn, S, items, units, n_slots, false, TC_COLS);
  }
  if (by_segment)
    sort_items_by_segment(items, nseg);
  else
    sort_items(items);
  const int n = (int)items.size();
  if (n > cap) return -n;
  for (int j = 0; j < n; ++j) {
    const TcItem& it = items[(size_t)j];
    int* r = out + 6 * (size_t)j;
    r[0] = it.seg;
    r[1] = it.m;
    r[2] = it.c;
    r[3] = it.kb0;
    r[4] = it.nkb;
    r[5] = it.slot;
  }
  return n;
}

