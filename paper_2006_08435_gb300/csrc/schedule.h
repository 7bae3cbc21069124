// Ticket order of the persistent kernels, shared by the planner (plan.cu)
// and the entry point without allocation (noalloc.cu).  Host code only; it
// writes into storage the caller provides, so neither user needs the heap.
#pragma once

#include "internal.h"

namespace fft3d {

// Work blocks of `count` grids taken in the order order[0..count) (grid
// order[i] has edge dims[order[i]]).  Plane blocks are emitted grid after
// grid; the slab block of a grid follows once at least `concurrency`
// tickets (the items resident at once) have been handed out after its last
// plane ticket, so a slab item rarely waits, or earlier when the grids
// whose planes are done but whose slabs are not yet scheduled would exceed
// `l2_budget` bytes (8 n^3 each; their intermediate must stay in L2).  The
// grids waiting for their slabs leave in the order their planes were
// emitted, so they are the positions [head, i) of `order`.  A phase is
// `phase_items` tickets (the grid's edge when 0).
//   plane_end : scratch of `count` ints (ticket after each plane block).
//   out       : receives 2 * count blocks.
// Returns the number of blocks; *total_items = tickets in all.
inline int schedule_blocks(int count, const int* dims, const int* order, int concurrency,
                           double l2_budget, int phase_items, int* plane_end, SchedBlock* out,
                           int* total_items) {
  int start = 0, nb = 0, head = 0;
  double pending = 0.0;
  auto bytes_at = [&](int i) {
    const double n = dims[order[i]];
    return 8.0 * n * n * n;
  };
  auto emit = [&](int g, int phase) {
    out[nb++] = SchedBlock{g, phase, start, dims[g]};
    start += phase_items > 0 ? phase_items : dims[g];
  };
  // slab blocks of the waiting grids before position `next`: those whose
  // planes ended `concurrency` tickets ago, and at least one if forced
  auto flush = [&](int next, bool force_one) {
    while (head < next) {
      if (start - plane_end[head] < concurrency && !force_one) break;
      force_one = false;
      pending -= bytes_at(head);
      emit(order[head], 1);
      ++head;
    }
  };
  for (int i = 0; i < count; ++i) {
    const double b = bytes_at(i);
    while (head < i && pending + b > l2_budget) flush(i, true);
    emit(order[i], 0);
    plane_end[i] = start;
    pending += b;
    flush(i + 1, false);
  }
  while (head < count) flush(count, true);
  *total_items = start;
  return nb;
}

}  // namespace fft3d
