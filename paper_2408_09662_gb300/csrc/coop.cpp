// Within-instance parallelism: W warps cooperate on each group of 32
// instances (lane = instance), splitting one program's ops between them.
//
// CusADi parallelises across instances only and names parallelism inside one
// expression graph as future work (§VI).  Here a list scheduler assigns every
// op to a warp (earliest finish time, with a fixed cost for a value that has
// to cross to another warp), then ops are grouped into phases: an op runs in
// the phase of its latest same-warp operand, or one phase after an operand
// produced by another warp.  Phases are separated by a CTA barrier and values
// that cross warps go through shared memory.
#include <algorithm>
#include <map>

#include "internal.h"

namespace cusadi {

namespace {

double op_cost(int op) {
  switch (op) {
    case SIN: case COS: case TAN: case ATAN: case ATAN2: case TANH: case ASIN: case ACOS:
    case SINH: case COSH: case ERF: case POW: case LOG: case HYPOT: case LOG1P: case EXPM1:
    case FMOD:
      return 24.0;
    case EXP: return 12.0;
    case DIV: case SQRT: case INV: return 8.0;
    default: return 1.0;
  }
}

}  // namespace

CoopPlan plan_coop(const Graph& g, int ways, double comm_cost) {
  const int64_t n = (int64_t)g.nodes.size();
  CoopPlan P;
  P.ways = ways;
  P.owner.assign(n, -1);
  P.phase.assign(n, 0);
  std::vector<double> finish(n, 0.0), avail(ways, 0.0);
  auto leaf = [&](int64_t i) { return g.nodes[i].op == INPUT || g.nodes[i].op == CONST; };
  for (int64_t i = 0; i < n; ++i) {
    if (leaf(i)) continue;
    const Node& x = g.nodes[i];
    int best = 0;
    double best_f = 1e300, best_start = 0;
    for (int w = 0; w < ways; ++w) {
      double start = avail[w];
      for (int32_t o : {x.a, x.b})
        if (o >= 0 && !leaf(o)) start = std::max(start, finish[o] + (P.owner[o] == w ? 0.0 : comm_cost));
      double f = start + op_cost(x.op);
      if (f < best_f - 1e-12 || (f < best_f + 1e-12 && avail[w] < avail[best])) {
        best = w;
        best_f = f;
        best_start = start;
      }
    }
    (void)best_start;
    P.owner[i] = best;
    finish[i] = best_f;
    avail[best] = best_f;
    int ph = 0;
    for (int32_t o : {x.a, x.b})
      if (o >= 0 && !leaf(o)) ph = std::max(ph, P.phase[o] + (P.owner[o] == best ? 0 : 1));
    P.phase[i] = ph;
  }
  P.n_phases = 1;
  for (int64_t i = 0; i < n; ++i)
    if (!leaf(i)) P.n_phases = std::max(P.n_phases, P.phase[i] + 1);
  return P;
}

int assign_coop_slots(const Graph& g, const CoopPlan& P, const std::vector<int>& seg_of_node,
                      int max_slots, std::vector<int>& slot, std::vector<int>& gslot,
                      int& n_gslots) {
  // Values read by another warp of the same kernel get a shared-memory slot for
  // the phases [producer phase, last such reader's phase]; a slot is free again
  // from the phase after its last reader.  When all max_slots are taken, the
  // value goes to a workspace row instead (the CTA barrier orders global
  // memory as well).  Reads from a later kernel go through the workspace.
  const int64_t n = (int64_t)g.nodes.size();
  auto leaf = [&](int64_t i) { return g.nodes[i].op == INPUT || g.nodes[i].op == CONST; };
  slot.assign(n, -1);
  gslot.assign(n, -1);
  std::vector<int> last_read(n, -1);
  for (int64_t i = 0; i < n; ++i) {
    if (leaf(i)) continue;
    const Node& x = g.nodes[i];
    for (int32_t o : {x.a, x.b})
      if (o >= 0 && !leaf(o) && P.owner[o] != P.owner[i] && seg_of_node[o] == seg_of_node[i])
        last_read[o] = std::max(last_read[o], P.phase[i]);
  }
  std::vector<std::vector<int64_t>> by_phase(P.n_phases);
  for (int64_t i = 0; i < n; ++i)
    if (last_read[i] >= 0) by_phase[P.phase[i]].push_back(i);
  std::vector<std::vector<int>> release(P.n_phases + 1), grelease(P.n_phases + 1);
  std::vector<int> free_slots, free_g;
  int slots = 0;
  n_gslots = 0;
  for (int q = 0; q < P.n_phases; ++q) {
    for (int s : release[q]) free_slots.push_back(s);
    for (int s : grelease[q]) free_g.push_back(s);
    for (int64_t i : by_phase[q]) {
      const int end = std::min(last_read[i] + 1, P.n_phases);
      if (!free_slots.empty() || slots < max_slots) {
        int s;
        if (!free_slots.empty()) { s = free_slots.back(); free_slots.pop_back(); }
        else s = slots++;
        slot[i] = s;
        release[end].push_back(s);
      } else {
        int s;
        if (!free_g.empty()) { s = free_g.back(); free_g.pop_back(); }
        else s = n_gslots++;
        gslot[i] = s;
        grelease[end].push_back(s);
      }
    }
  }
  return slots;
}

}  // namespace cusadi
