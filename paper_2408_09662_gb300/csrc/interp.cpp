// Packs an SSA program into the instruction stream of the interpreter kernel.
//
// This is the sequential traversal of CusADi §III-A ("traversing across the
// instructions sequentially") kept for programs too large to compile: every
// thread walks the same stream, so each step is warp-uniform.  Work slots are
// re-assigned by linear scan over the schedule, so the work vector is only as
// long as the number of values live at once.
#include <algorithm>

#include "internal.h"

namespace cusadi {

bool pack_interp(const Graph& g, InterpProgram& p, std::string& err) {
  const int64_t n = (int64_t)g.nodes.size();
  std::vector<int64_t> lu = last_uses(g);
  std::vector<int64_t> slot(n, -1);
  std::vector<uint32_t> free_slots;
  int64_t n_slots = 0;
  std::vector<std::vector<int64_t>> out_rows(n);
  for (size_t r = 0; r < g.out.size(); ++r) out_rows[g.out[r]].push_back((int64_t)r);
  p.ops.clear();
  p.k.clear();
  p.in_bcast = g.in_bcast;
  p.has_reduce = false;
  auto alloc = [&]() -> uint32_t {
    if (!free_slots.empty()) { uint32_t s = free_slots.back(); free_slots.pop_back(); return s; }
    return (uint32_t)n_slots++;
  };
  auto leaf = [&](int64_t i) { return g.nodes[i].op == INPUT || g.nodes[i].op == CONST; };
  auto code = [&](int op, int f64, uint64_t aux) -> uint32_t {
    return (uint32_t)op | ((uint32_t)(f64 ? 1 : 0) << 7) | ((uint32_t)aux << 8);
  };
  const uint64_t AUX_MAX = (1u << 24) - 1;
  auto materialise = [&](int64_t i) -> bool {
    if (slot[i] >= 0) return true;
    const Node& x = g.nodes[i];
    uint32_t s = alloc();
    slot[i] = s;
    if (x.op == INPUT) {
      if ((uint64_t)x.io > AUX_MAX) { err = "too many input rows for the interpreter"; return false; }
      p.ops.push_back({code(INPUT, x.f64, (uint64_t)x.io), s, 0, (uint32_t)x.bcast});
    } else {
      if (p.k.size() > AUX_MAX) { err = "too many constants for the interpreter"; return false; }
      p.ops.push_back({code(CONST, x.f64, p.k.size()), s, 0, 0});
      p.k.push_back(x.k);
    }
    return true;
  };
  auto emit_outputs = [&](int64_t i) -> bool {
    for (int64_t r : out_rows[i]) {
      if ((uint64_t)r > AUX_MAX) { err = "too many output rows for the interpreter"; return false; }
      // a reduced (broadcast) row carries its index among the reduced rows + 1
      uint32_t red = 0;
      if (!g.out_reduce.empty() && g.out_reduce[r]) {
        p.reduce_rows.push_back(r);
        red = (uint32_t)p.reduce_rows.size();
      }
      p.has_reduce |= red != 0;
      p.ops.push_back({code(OUTPUT, 0, (uint64_t)r), 0, (uint32_t)slot[i], red});
    }
    return true;
  };
  auto release = [&](int64_t i, int64_t t) {
    if (slot[i] >= 0 && lu[i] <= t) { free_slots.push_back((uint32_t)slot[i]); slot[i] = -2; }
  };
  // outputs fed by leaves
  for (int64_t i = 0; i < n; ++i) {
    if (!leaf(i) || out_rows[i].empty()) continue;
    if (!materialise(i) || !emit_outputs(i)) return false;
    if (lu[i] <= i) release(i, n);
  }
  for (int64_t t = 0; t < n; ++t) {
    if (leaf(t)) continue;
    const Node& x = g.nodes[t];
    for (int32_t a : {x.a, x.b})
      if (a >= 0 && leaf(a) && slot[a] == -1)
        if (!materialise(a)) return false;
    uint32_t sa = x.a >= 0 ? (uint32_t)slot[x.a] : 0, sb = x.b >= 0 ? (uint32_t)slot[x.b] : 0;
    // operands whose last reader is this op give their slot back before the write
    for (int32_t a : {x.a, x.b})
      if (a >= 0 && slot[a] >= 0 && lu[a] <= t) release(a, t);
    uint32_t s = alloc();
    slot[t] = s;
    uint64_t aux = 0;
    if (x.op == FMA_CONST) {
      if (p.k.size() > AUX_MAX) { err = "too many constants for the interpreter"; return false; }
      aux = p.k.size();
      p.k.push_back(x.k);
    }
    p.ops.push_back({code(x.op, x.f64, aux), s, sa, sb});
    if (!emit_outputs(t)) return false;
    if (lu[t] <= t) release(t, t);
  }
  p.n_slots = std::max<int64_t>(n_slots, 1);
  return true;
}

}  // namespace cusadi
