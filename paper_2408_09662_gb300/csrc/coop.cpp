// Within-instance parallelism: W warps cooperate on each group of 32
// instances (lane = instance), splitting one program's ops between them.
//
// CusADi parallelises across instances only and names parallelism inside one
// expression graph as future work (§VI).  Ops are assigned a warp and a phase;
// phases are separated by a CTA barrier, an op may read a value of its own
// warp from its own or an earlier phase and a value of another warp from an
// earlier phase (through shared memory).  Two schedulers are tried and the
// one with the lower estimated time (sum over phases of the busiest warp's
// op cost plus a barrier cost) is kept:
//  * earliest finish time: each op goes to the warp where it finishes first,
//    counting a fixed cost for a value that crosses warps; phases follow;
//  * phase packing: phases are filled one at a time, up to a target cost per
//    warp, always with the ready op of longest remaining critical path (bottom
//    level), so every warp carries about the same work between barriers.
//    Several targets are tried.
#include <algorithm>
#include <cstdlib>
#include <map>
#include <queue>

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

// a CTA barrier plus the shared-memory hand-off, in op costs (CUSADI_COOP_BARRIER_COST
// overrides it, for sweeps of the phase count against compile time and run time)
double barrier_cost() {
  static const double c = [] {
    const char* e = std::getenv("CUSADI_COOP_BARRIER_COST");
    return e ? std::max(0.0, std::atof(e)) : 6.0;
  }();
  return c;
}

bool is_leaf(const Graph& g, int64_t i) { return g.nodes[i].op == INPUT || g.nodes[i].op == CONST; }

// sum over phases of (the busiest warp's op cost + one barrier)
double estimate(const Graph& g, const CoopPlan& P) {
  std::vector<double> load((size_t)P.n_phases * P.ways, 0.0);
  for (int64_t i = 0; i < (int64_t)g.nodes.size(); ++i)
    if (!is_leaf(g, i)) load[(size_t)P.phase[i] * P.ways + P.owner[i]] += op_cost(g.nodes[i].op);
  double t = 0;
  for (int q = 0; q < P.n_phases; ++q)
    t += *std::max_element(load.begin() + (size_t)q * P.ways, load.begin() + (size_t)(q + 1) * P.ways) +
         barrier_cost();
  return t;
}

struct Ready {
  double pri;
  int64_t i;
  bool operator<(const Ready& o) const { return pri < o.pri || (pri == o.pri && i > o.i); }
};

CoopPlan plan_packed(const Graph& g, int ways, double target, const std::vector<double>& bottom,
                     const std::vector<std::vector<int64_t>>& users) {
  const int64_t n = (int64_t)g.nodes.size();
  CoopPlan P;
  P.ways = ways;
  P.owner.assign(n, -1);
  P.phase.assign(n, 0);
  std::vector<int> pending(n, 0);
  int64_t todo = 0;
  std::priority_queue<Ready> open;                        // any warp may take these
  std::vector<std::priority_queue<Ready>> mine(ways);     // need a value of this warp's phase
  std::vector<int64_t> later;                             // need values of two warps' phase
  for (int64_t i = 0; i < n; ++i) {
    if (is_leaf(g, i)) continue;
    ++todo;
    for (int32_t o : {g.nodes[i].a, g.nodes[i].b})
      if (o >= 0 && !is_leaf(g, o)) ++pending[i];
    if (pending[i] == 0) open.push({bottom[i], i});
  }
  int q = 0;
  std::vector<double> load(ways);
  std::vector<char> full(ways);
  while (todo > 0) {
    std::fill(load.begin(), load.end(), 0.0);
    std::fill(full.begin(), full.end(), 0);
    int active = ways;
    while (active > 0) {
      int w = -1;
      for (int k = 0; k < ways; ++k)
        if (!full[k] && (w < 0 || load[k] < load[w])) w = k;
      const bool has_mine = !mine[w].empty(), has_open = !open.empty();
      if (!has_mine && !has_open) { full[w] = 1; --active; continue; }
      const bool take_mine = has_mine && (!has_open || !(mine[w].top() < open.top()));
      const Ready r = take_mine ? mine[w].top() : open.top();
      const double c = op_cost(g.nodes[r.i].op);
      if (load[w] > 0 && load[w] + c > target) { full[w] = 1; --active; continue; }
      (take_mine ? mine[w] : open).pop();
      P.owner[r.i] = w;
      P.phase[r.i] = q;
      load[w] += c;
      --todo;
      for (int64_t u : users[r.i]) {
        if (--pending[u] != 0) continue;
        int same = -1;   // warp of the operands computed in this phase, -2 if two warps
        for (int32_t o : {g.nodes[u].a, g.nodes[u].b})
          if (o >= 0 && !is_leaf(g, o) && P.phase[o] == q)
            same = (same == -1 || same == P.owner[o]) ? P.owner[o] : -2;
        if (same == -1) open.push({bottom[u], u});
        else if (same >= 0) mine[same].push({bottom[u], u});
        else later.push_back(u);
      }
    }
    // what waited on this phase's values of one warp, or of two, is open next phase
    for (auto& m : mine)
      while (!m.empty()) { open.push(m.top()); m.pop(); }
    for (int64_t u : later) open.push({bottom[u], u});
    later.clear();
    ++q;
  }
  P.n_phases = std::max(q, 1);
  return P;
}

CoopPlan plan_eft(const Graph& g, int ways, double comm_cost);

}  // namespace

CoopPlan plan_coop(const Graph& g, int ways, double comm_cost) {
  const int64_t n = (int64_t)g.nodes.size();
  // bottom level: op cost on the longest path from the op to the end
  std::vector<double> bottom(n, 0.0);
  std::vector<std::vector<int64_t>> users(n);
  for (int64_t i = 0; i < n; ++i) {
    if (is_leaf(g, i)) continue;
    bottom[i] = op_cost(g.nodes[i].op);
    for (int32_t o : {g.nodes[i].a, g.nodes[i].b})
      if (o >= 0 && !is_leaf(g, o)) users[o].push_back(i);
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    if (is_leaf(g, i)) continue;
    for (int32_t o : {g.nodes[i].a, g.nodes[i].b})
      if (o >= 0 && !is_leaf(g, o)) bottom[o] = std::max(bottom[o], op_cost(g.nodes[o].op) + bottom[i]);
  }
  CoopPlan best = plan_eft(g, ways, comm_cost);
  double best_t = estimate(g, best);
  for (double target : {8.0, 16.0, 32.0, 64.0, 128.0, 256.0, 512.0}) {
    CoopPlan P = plan_packed(g, ways, target, bottom, users);
    const double t = estimate(g, P);
    if (t < best_t) { best_t = t; best = std::move(P); }
  }
  return best;
}

namespace {

CoopPlan plan_eft(const Graph& g, int ways, double comm_cost) {
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
    double best_f = 1e300;
    for (int w = 0; w < ways; ++w) {
      double start = avail[w];
      for (int32_t o : {x.a, x.b})
        if (o >= 0 && !leaf(o)) start = std::max(start, finish[o] + (P.owner[o] == w ? 0.0 : comm_cost));
      double f = start + op_cost(x.op);
      if (f < best_f - 1e-12 || (f < best_f + 1e-12 && avail[w] < avail[best])) {
        best = w;
        best_f = f;
      }
    }
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

}  // namespace

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
