// Packs an SSA program into the instruction stream of the interpreter kernel.
//
// This is the sequential traversal of CusADi §III-A ("traversing across the
// instructions sequentially") kept for programs too large to compile: every
// thread walks the same stream, so each step is warp-uniform.
//
// Work slots come in two tiers: `max_shared` slots in shared memory (one
// column per thread) and, beyond them, slots in a global workspace (one row
// per slot, instance-fastest).  Every value occupies one slot from its
// definition to its last read.  The shared tier is assigned by linear-scan
// allocation over the emission order (M. Poletto and V. Sarkar, "Linear scan
// register allocation", TOPLAS 21(5), 1999): when a value finds the shared
// slots full, whichever of it and the live shared values is read last moves
// to the global tier for its whole life, so the shared tier keeps the
// short-lived temporaries that make up most reads.  The global values are
// then packed onto as few rows as their lifetimes allow.
#include <algorithm>
#include <set>

#include "internal.h"

namespace cusadi {

bool pack_interp(const Graph& g, InterpProgram& p, std::string& err, int64_t max_shared) {
  const int64_t n = (int64_t)g.nodes.size();
  std::vector<std::vector<int64_t>> out_rows(n);
  for (size_t r = 0; r < g.out.size(); ++r) out_rows[g.out[r]].push_back((int64_t)r);
  p.ops.clear();
  p.k.clear();
  p.reduce_rows.clear();
  p.in_bcast = g.in_bcast;
  p.has_reduce = false;
  auto leaf = [&](int64_t i) { return g.nodes[i].op == INPUT || g.nodes[i].op == CONST; };
  const uint64_t AUX_MAX = (1u << 24) - 1;

  // 1. emission order: each leaf just before its first reader (leaves that
  // only feed outputs first), each op followed by the outputs it feeds.  An
  // event is (node, kind): 0 define, 1 output store of row `row`.
  struct Ev { int64_t node; int kind; int64_t row; };
  std::vector<Ev> ev;
  std::vector<int64_t> def(n, -1), end(n, -1);   // emission positions
  auto emit_def = [&](int64_t i) { def[i] = (int64_t)ev.size(); end[i] = def[i]; ev.push_back({i, 0, 0}); };
  auto read = [&](int64_t i) { end[i] = (int64_t)ev.size(); };
  auto emit_outputs = [&](int64_t i) {
    for (int64_t r : out_rows[i]) { read(i); ev.push_back({i, 1, r}); }
  };
  for (int64_t i = 0; i < n; ++i)
    if (leaf(i) && !out_rows[i].empty()) { emit_def(i); emit_outputs(i); }
  for (int64_t t = 0; t < n; ++t) {
    if (leaf(t)) continue;
    const Node& x = g.nodes[t];
    for (int32_t a : {x.a, x.b})
      if (a >= 0 && leaf(a) && def[a] < 0) emit_def(a);
    // the op reads its operands at its own position, before it writes
    const int64_t pos = (int64_t)ev.size();
    for (int32_t a : {x.a, x.b})
      if (a >= 0) end[a] = std::max(end[a], pos);
    emit_def(t);
    emit_outputs(t);
  }

  // 2. shared tier: linear scan in order of definition, intervals [def, end];
  // an operand whose last read is the op defining v may share v's slot
  std::vector<int64_t> slot(n, -1);
  std::vector<uint8_t> global(n, 0);
  {
    std::set<std::pair<int64_t, int64_t>> active;   // (end, node) in shared slots
    std::vector<int64_t> free_sh;
    int64_t next_sh = 0;
    for (const Ev& e : ev) {
      if (e.kind != 0) continue;
      const int64_t v = e.node, start = def[v];
      while (!active.empty() && active.begin()->first <= start) {
        free_sh.push_back(slot[active.begin()->second]);
        active.erase(active.begin());
      }
      if (!free_sh.empty() || next_sh < max_shared) {
        int64_t s;
        if (!free_sh.empty()) { s = free_sh.back(); free_sh.pop_back(); }
        else s = next_sh++;
        slot[v] = s;
        active.insert({end[v], v});
      } else if (!active.empty() && std::prev(active.end())->first > end[v]) {
        auto last = std::prev(active.end());          // read last: moves to the global tier
        const int64_t u = last->second;
        slot[v] = slot[u];
        slot[u] = -1;
        global[u] = 1;
        active.erase(last);
        active.insert({end[v], v});
      } else {
        global[v] = 1;
      }
    }
    p.n_shared = next_sh;
  }
  // 3. global tier: rows reused once their value is dead
  {
    std::set<std::pair<int64_t, int64_t>> active;
    std::vector<int64_t> free_gl;
    int64_t next_gl = 0;
    for (const Ev& e : ev) {
      if (e.kind != 0 || !global[e.node]) continue;
      const int64_t v = e.node;
      while (!active.empty() && active.begin()->first <= def[v]) {
        free_gl.push_back(slot[active.begin()->second]);
        active.erase(active.begin());
      }
      int64_t s;
      if (!free_gl.empty()) { s = free_gl.back(); free_gl.pop_back(); }
      else s = next_gl++;
      slot[v] = s;
      active.insert({end[v], v});
    }
    p.n_global = next_gl;
    for (int64_t v = 0; v < n; ++v)
      if (global[v]) slot[v] += p.n_shared;         // global rows follow the shared slots
  }
  p.n_slots = std::max<int64_t>(p.n_shared + p.n_global, 1);

  // 4. the stream
  auto code = [&](int op, int f64, uint64_t aux) -> uint32_t {
    return (uint32_t)op | ((uint32_t)(f64 ? 1 : 0) << 7) | ((uint32_t)aux << 8);
  };
  for (const Ev& e : ev) {
    const int64_t i = e.node;
    const Node& x = g.nodes[i];
    const uint32_t s = (uint32_t)slot[i];
    if (e.kind == 1) {
      if ((uint64_t)e.row > AUX_MAX) { err = "too many output rows for the interpreter"; return false; }
      // a reduced (broadcast) row carries its index among the reduced rows + 1
      uint32_t red = 0;
      if (!g.out_reduce.empty() && g.out_reduce[e.row]) {
        p.reduce_rows.push_back(e.row);
        red = (uint32_t)p.reduce_rows.size();
      }
      p.has_reduce |= red != 0;
      p.ops.push_back({code(OUTPUT, 0, (uint64_t)e.row), 0, s, red});
    } else if (x.op == INPUT) {
      if ((uint64_t)x.io > AUX_MAX) { err = "too many input rows for the interpreter"; return false; }
      p.ops.push_back({code(INPUT, x.f64, (uint64_t)x.io), s, 0, (uint32_t)x.bcast});
    } else if (x.op == CONST) {
      if (p.k.size() > AUX_MAX) { err = "too many constants for the interpreter"; return false; }
      p.ops.push_back({code(CONST, x.f64, p.k.size()), s, 0, 0});
      p.k.push_back(x.k);
    } else {
      uint64_t aux = 0;
      if (x.op == FMA_CONST) {
        if (p.k.size() > AUX_MAX) { err = "too many constants for the interpreter"; return false; }
        aux = p.k.size();
        p.k.push_back(x.k);
      }
      const uint32_t sa = x.a >= 0 ? (uint32_t)slot[x.a] : 0, sb = x.b >= 0 ? (uint32_t)slot[x.b] : 0;
      p.ops.push_back({code(x.op, x.f64, aux), s, sa, sb});
    }
  }
  return true;
}

}  // namespace cusadi
