// Passes over the SSA form of a program: renaming, constant folding, exact
// identities, common-subexpression and dead-code elimination, scheduling for
// register pressure, and the reverse-mode (adjoint) transform.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <queue>
#include <unordered_map>

#include "internal.h"

namespace cusadi {

// ---------------------------------------------------------------------------
// work vector -> SSA.  A slot's current value is the node that last wrote it;
// operands are resolved before the destination is rebound (Listing 2 reads
// work[1] and writes work[1] in one instruction).
// ---------------------------------------------------------------------------
Graph build_ssa(const IRFile& f) {
  Graph g;
  g.nnz_in = f.nnz_in;
  std::vector<uint8_t>& bcast = g.in_bcast;
  bcast.assign(f.nnz_in, 0);
  for (const Arg& a : f.in)
    if (a.flags & 1)
      for (uint32_t q = 0; q < a.nnz; ++q) bcast[a.offset + q] = 1;
  std::vector<int32_t> slot(f.n_work, -1);
  g.out.assign(f.nnz_out, -1);
  g.out_reduce.assign(f.nnz_out, 0);
  g.nodes.reserve(f.code.size());
  for (const IRInstr& I : f.code) {
    Node n;
    n.op = I.op;
    n.f64 = (I.flags & 1) ? 1 : 0;
    switch (I.op) {
      case OUTPUT:
        g.out[I.out] = slot[I.a];
        continue;
      case ASSIGN:
        slot[I.out] = slot[I.a];
        continue;
      case INPUT:
        n.io = I.a;
        n.bcast = bcast[I.a];
        break;
      case CONST:
        n.k = f.k[I.a];
        break;
      default:
        n.a = slot[I.a];
        if (op_arity(I.op) == 2) n.b = slot[I.b];
        if (I.op == FMA_CONST) n.k = f.k[I.c];
    }
    g.nodes.push_back(n);
    slot[I.out] = (int32_t)g.nodes.size() - 1;
  }
  return g;
}

// ---------------------------------------------------------------------------
// host evaluation for constant folding (double; float-rounded for FP32 nodes)
// ---------------------------------------------------------------------------
static double sgn(double a) { return a > 0 ? 1.0 : (a < 0 ? -1.0 : 0.0); }

static double fold(int op, double a, double b, double k) {
  switch (op) {
    case ADD: return a + b;
    case SUB: return a - b;
    case MUL: return a * b;
    case DIV: return a / b;
    case NEG: return -a;
    case EXP: return std::exp(a);
    case LOG: return std::log(a);
    case POW: return std::pow(a, b);
    case SQ: return a * a;
    case SQRT: return std::sqrt(a);
    case SIN: return std::sin(a);
    case COS: return std::cos(a);
    case TAN: return std::tan(a);
    case ATAN: return std::atan(a);
    case ATAN2: return std::atan2(a, b);
    case TANH: return std::tanh(a);
    case FABS: return std::fabs(a);
    case FMIN: return std::fmin(a, b);
    case FMAX: return std::fmax(a, b);
    case FMA_CONST: return std::fma(k, a, b);
    case IF_ELSE_ZERO: return a != 0 ? b : 0.0;
    case LT: return a < b;
    case LE: return a <= b;
    case EQ: return a == b;
    case NE: return a != b;
    case NOT: return a == 0;
    case AND: return a != 0 && b != 0;
    case OR: return a != 0 || b != 0;
    case ASIN: return std::asin(a);
    case ACOS: return std::acos(a);
    case SINH: return std::sinh(a);
    case COSH: return std::cosh(a);
    case ERF: return std::erf(a);
    case SIGN: return sgn(a);
    case FLOOR: return std::floor(a);
    case CEIL: return std::ceil(a);
    case FMOD: return std::fmod(a, b);
    case INV: return 1.0 / a;
    case HYPOT: return std::hypot(a, b);
    case LOG1P: return std::log1p(a);
    case EXPM1: return std::expm1(a);
    case COPYSIGN: return std::copysign(a, b);
  }
  return NAN;
}

namespace {
struct Key {
  uint16_t op;
  uint8_t f64, bcast;
  int32_t a, b;
  uint64_t k;
  int64_t io;
  bool operator==(const Key& o) const {
    return op == o.op && f64 == o.f64 && bcast == o.bcast && a == o.a && b == o.b && k == o.k &&
           io == o.io;
  }
};
struct KeyHash {
  size_t operator()(const Key& x) const {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
    mix(x.op | ((uint64_t)x.f64 << 16) | ((uint64_t)x.bcast << 24));
    mix((uint32_t)x.a);
    mix((uint32_t)x.b);
    mix(x.k);
    mix((uint64_t)x.io);
    return (size_t)h;
  }
};
uint64_t bits(double d) {
  uint64_t u;
  std::memcpy(&u, &d, 8);
  return u;
}
}  // namespace

// ---------------------------------------------------------------------------
// simplify: fold, exact identities, CSE, then DCE from the outputs.
// ---------------------------------------------------------------------------
void simplify(Graph& g, int dtype) {
  std::vector<Node> nn;
  nn.reserve(g.nodes.size());
  std::vector<int32_t> map(g.nodes.size(), -1);
  std::unordered_map<Key, int32_t, KeyHash> seen;
  seen.reserve(g.nodes.size() * 2);
  auto is_const = [&](int32_t i, double v) { return i >= 0 && nn[i].op == CONST && nn[i].k == v; };
  auto intern = [&](const Node& n) -> int32_t {
    Key key{n.op, n.f64, n.bcast, n.a, n.b, bits(n.k), n.io};
    auto it = seen.find(key);
    if (it != seen.end()) return it->second;
    nn.push_back(n);
    int32_t id = (int32_t)nn.size() - 1;
    seen.emplace(key, id);
    return id;
  };
  for (size_t i = 0; i < g.nodes.size(); ++i) {
    Node n = g.nodes[i];
    if (n.a >= 0) n.a = map[n.a];
    if (n.b >= 0) n.b = map[n.b];
    const bool f32 = dtype != CUSADI_F64 && !n.f64;
    if (n.op == CONST) {
      if (f32) n.k = (double)(float)n.k;
      map[i] = intern(n);
      continue;
    }
    if (n.op == INPUT) { map[i] = intern(n); continue; }
    int ar = op_arity(n.op);
    bool ca = nn[n.a].op == CONST, cb = ar == 2 ? nn[n.b].op == CONST : true;
    if (ca && cb) {
      double av = nn[n.a].k, bv = ar == 2 ? nn[n.b].k : 0.0, kv = n.k;
      if (f32) { av = (float)av; bv = (float)bv; kv = (float)kv; }
      double v = fold(n.op, av, bv, kv);
      if (f32) v = (double)(float)v;
      Node c;
      c.op = CONST;
      c.f64 = n.f64;
      c.k = v;
      map[i] = intern(c);
      continue;
    }
    // exact identities (hold for every IEEE value up to the sign of zero)
    if ((n.op == ADD && is_const(n.b, 0.0)) || (n.op == SUB && is_const(n.b, 0.0)) ||
        (n.op == MUL && is_const(n.b, 1.0)) || (n.op == DIV && is_const(n.b, 1.0))) {
      map[i] = n.a;
      continue;
    }
    if ((n.op == ADD && is_const(n.a, 0.0)) || (n.op == MUL && is_const(n.a, 1.0))) {
      map[i] = n.b;
      continue;
    }
    if (n.op == NEG && nn[n.a].op == NEG && nn[n.a].f64 == n.f64) {
      map[i] = nn[n.a].a;
      continue;
    }
    if (n.op == ASSIGN) { map[i] = n.a; continue; }
    if (op_commutative(n.op) && n.a > n.b) std::swap(n.a, n.b);
    map[i] = intern(n);
  }
  for (auto& o : g.out) o = map[o];
  // DCE
  std::vector<uint8_t> live(nn.size(), 0);
  for (int32_t o : g.out) live[o] = 1;
  for (size_t i = nn.size(); i-- > 0;) {
    if (!live[i]) continue;
    if (nn[i].a >= 0) live[nn[i].a] = 1;
    if (nn[i].b >= 0) live[nn[i].b] = 1;
  }
  std::vector<int32_t> renum(nn.size(), -1);
  std::vector<Node> out;
  out.reserve(nn.size());
  for (size_t i = 0; i < nn.size(); ++i) {
    if (!live[i]) continue;
    Node n = nn[i];
    if (n.a >= 0) n.a = renum[n.a];
    if (n.b >= 0) n.b = renum[n.b];
    renum[i] = (int32_t)out.size();
    out.push_back(n);
  }
  for (auto& o : g.out) o = renum[o];
  g.nodes.swap(out);
}

// ---------------------------------------------------------------------------
// liveness
// ---------------------------------------------------------------------------
std::vector<int64_t> last_uses(const Graph& g) {
  std::vector<int64_t> lu(g.nodes.size(), -1);
  for (size_t i = 0; i < g.nodes.size(); ++i) {
    const Node& n = g.nodes[i];
    if (n.a >= 0) lu[n.a] = std::max<int64_t>(lu[n.a], (int64_t)i);
    if (n.b >= 0) lu[n.b] = std::max<int64_t>(lu[n.b], (int64_t)i);
  }
  for (int32_t o : g.out) lu[o] = std::max<int64_t>(lu[o], o);
  return lu;
}

// Values held at once when inputs are loaded at their first use, constants are
// immediates, and each value dies at its last use.
int64_t max_live(const Graph& g) {
  const size_t n = g.nodes.size();
  std::vector<int64_t> first(n, -1), lu = last_uses(g);
  for (size_t i = 0; i < n; ++i) {
    const Node& x = g.nodes[i];
    for (int32_t o : {x.a, x.b})
      if (o >= 0 && first[o] < 0) first[o] = (int64_t)i;
  }
  std::vector<int32_t> delta(n + 1, 0);
  for (size_t i = 0; i < n; ++i) {
    const Node& x = g.nodes[i];
    if (x.op == CONST) continue;
    int64_t start = x.op == INPUT ? first[i] : (int64_t)i;
    if (start < 0) start = (int64_t)i;          // input used only as an output
    int64_t end = std::max(lu[i], start);
    delta[start] += 1;
    delta[end + 1 <= (int64_t)n ? end + 1 : n] -= 1;
  }
  int64_t cur = 0, best = 0;
  for (size_t i = 0; i < n; ++i) {
    cur += delta[i];
    best = std::max(best, cur);
  }
  return best;
}

int64_t count_ops(const Graph& g) {
  int64_t c = 0;
  for (const Node& n : g.nodes)
    if (n.op != INPUT && n.op != CONST) ++c;
  return c;
}

void op_histogram(const Graph& g, std::vector<int64_t>& h, bool f64_only) {
  h.assign(N_OPS, 0);
  for (const Node& n : g.nodes)
    if (n.op != INPUT && n.op != CONST && (!f64_only || n.f64)) h[n.op]++;
}

// ---------------------------------------------------------------------------
// scheduling: greedy list scheduling that, among ready nodes, prefers the one
// that frees the most operands (ties: the earliest in the current order).
// Inputs and constants are free to schedule (loaded at first use).
// ---------------------------------------------------------------------------
void schedule(Graph& g) {
  const int32_t n = (int32_t)g.nodes.size();
  if (n < 3) return;
  std::vector<int32_t> users_left(n, 0), deps_left(n, 0);
  std::vector<std::vector<int32_t>> users(n);
  std::vector<uint8_t> is_out(n, 0);
  for (int32_t o : g.out) is_out[o] = 1;
  for (int32_t i = 0; i < n; ++i) {
    const Node& x = g.nodes[i];
    if (x.a >= 0) { users[x.a].push_back(i); users_left[x.a]++; deps_left[i]++; }
    if (x.b >= 0 && x.b != x.a) { users[x.b].push_back(i); users_left[x.b]++; deps_left[i]++; }
  }
  auto leaf = [&](int32_t i) { return g.nodes[i].op == INPUT || g.nodes[i].op == CONST; };
  // priority: (number of operands whose last user this is) desc, position asc
  auto score = [&](int32_t i) {
    const Node& x = g.nodes[i];
    int kill = 0;
    if (x.a >= 0 && !leaf(x.a) && users_left[x.a] == 1) kill++;
    if (x.b >= 0 && x.b != x.a && !leaf(x.b) && users_left[x.b] == 1) kill++;
    // a node whose result nobody needs except an output frees itself at once
    int self = (users[i].empty()) ? 1 : 0;
    return kill * 2 + self;
  };
  using Item = std::pair<int64_t, int32_t>;  // (-(score<<32) + pos) ordering via comparator
  auto cmp = [](const Item& p, const Item& q) { return p.first > q.first || (p.first == q.first && p.second > q.second); };
  std::priority_queue<Item, std::vector<Item>, decltype(cmp)> ready(cmp);
  std::vector<int32_t> order;
  order.reserve(n);
  std::vector<uint8_t> done(n, 0);
  auto push = [&](int32_t i) { ready.push({-(int64_t)score(i) * (int64_t)n * 4 + i, i}); };
  // leaves are emitted lazily: mark as done from the start
  for (int32_t i = 0; i < n; ++i)
    if (leaf(i)) done[i] = 1;
  for (int32_t i = 0; i < n; ++i) {
    if (leaf(i)) {
      for (int32_t u : users[i]) deps_left[u]--;
    }
  }
  for (int32_t i = 0; i < n; ++i)
    if (!leaf(i) && deps_left[i] == 0) push(i);
  while (!ready.empty()) {
    Item it = ready.top();
    ready.pop();
    int32_t i = it.second;
    if (done[i]) continue;
    // scores change as users complete; re-queue stale entries
    int64_t fresh = -(int64_t)score(i) * (int64_t)n * 4 + i;
    if (fresh < it.first) { ready.push({fresh, i}); continue; }
    done[i] = 1;
    order.push_back(i);
    const Node& x = g.nodes[i];
    if (x.a >= 0) users_left[x.a]--;
    if (x.b >= 0 && x.b != x.a) users_left[x.b]--;
    for (int32_t u : users[i])
      if (--deps_left[u] == 0) push(u);
    // operands that now have one user left make that user more attractive
    for (int32_t o : {x.a, x.b})
      if (o >= 0 && !leaf(o) && users_left[o] == 1)
        for (int32_t u : users[o])
          if (!done[u] && deps_left[u] == 0) push(u);
  }
  // leaves first (their position does not matter), then the schedule
  std::vector<int32_t> perm;
  perm.reserve(n);
  for (int32_t i = 0; i < n; ++i)
    if (leaf(i)) perm.push_back(i);
  for (int32_t i : order) perm.push_back(i);
  if ((int32_t)perm.size() != n) return;  // cannot happen for a DAG; keep the old order
  std::vector<int32_t> pos(n);
  for (int32_t p = 0; p < n; ++p) pos[perm[p]] = p;
  std::vector<Node> nn(n);
  for (int32_t p = 0; p < n; ++p) {
    Node x = g.nodes[perm[p]];
    if (x.a >= 0) x.a = pos[x.a];
    if (x.b >= 0) x.b = pos[x.b];
    nn[p] = x;
  }
  for (auto& o : g.out) o = pos[o];
  g.nodes.swap(nn);
}

// ---------------------------------------------------------------------------
// reverse mode.  The adjoint of every active node is accumulated as new nodes
// appended after the forward sweep, visiting the forward nodes in reverse.
// ---------------------------------------------------------------------------
Graph adjoint_graph(const Graph& fwd) {
  Graph g;
  g.nodes = fwd.nodes;
  const int64_t nin = fwd.nnz_in, nout = (int64_t)fwd.out.size();
  g.nnz_in = nin + nout;
  g.in_bcast = fwd.in_bcast;
  g.in_bcast.resize(nin + nout, 0);
  const int32_t nf = (int32_t)fwd.nodes.size();
  std::vector<uint8_t> active(nf, 0);
  for (int32_t i = 0; i < nf; ++i) {
    const Node& x = fwd.nodes[i];
    if (x.op == INPUT) active[i] = 1;
    else if (x.op != CONST) active[i] = (x.a >= 0 && active[x.a]) || (x.b >= 0 && active[x.b]);
  }
  auto mk = [&](uint16_t op, int32_t a, int32_t b, uint8_t f64, double k = 0) {
    Node n;
    n.op = op; n.a = a; n.b = b; n.f64 = f64; n.k = k;
    g.nodes.push_back(n);
    return (int32_t)g.nodes.size() - 1;
  };
  auto cst = [&](double v, uint8_t f64) { return mk(CONST, -1, -1, f64, v); };
  std::vector<int32_t> adj(nf, -1);
  auto acc = [&](int32_t target, int32_t contrib, bool negate) {
    if (target < 0 || !active[target]) return;
    uint8_t t = fwd.nodes[target].f64;
    if (adj[target] < 0) adj[target] = negate ? mk(NEG, contrib, -1, t) : contrib;
    else adj[target] = mk(negate ? SUB : ADD, adj[target], contrib, t);
  };
  // seeds: y_bar rows are new inputs after the x rows
  for (int64_t r = 0; r < nout; ++r) {
    int32_t o = fwd.out[r];
    if (!active[o]) continue;
    Node in;
    in.op = INPUT;
    in.io = nin + r;
    in.f64 = fwd.nodes[o].f64;
    g.nodes.push_back(in);
    acc(o, (int32_t)g.nodes.size() - 1, false);
  }
  for (int32_t i = nf - 1; i >= 0; --i) {
    const int32_t gi = adj[i];
    if (gi < 0) continue;
    const Node x = fwd.nodes[i];
    if (x.op == INPUT || x.op == CONST) continue;
    const int32_t a = x.a, b = x.b, y = i;
    const uint8_t t = x.f64;
    const bool aa = a >= 0 && active[a], ab = b >= 0 && active[b];
    switch (x.op) {
      case ADD: acc(a, gi, false); acc(b, gi, false); break;
      case SUB: acc(a, gi, false); acc(b, gi, true); break;
      case MUL:
        if (aa) acc(a, mk(MUL, gi, b, t), false);
        if (ab) acc(b, mk(MUL, gi, a, t), false);
        break;
      case DIV: {
        int32_t q = mk(DIV, gi, b, t);
        acc(a, q, false);
        if (ab) acc(b, mk(MUL, q, y, t), true);
        break;
      }
      case NEG: acc(a, gi, true); break;
      case EXP: acc(a, mk(MUL, gi, y, t), false); break;
      case LOG: acc(a, mk(DIV, gi, a, t), false); break;
      case POW:
        if (aa) {
          int32_t e = mk(POW, a, mk(SUB, b, cst(1.0, t), t), t);
          acc(a, mk(MUL, gi, mk(MUL, b, e, t), t), false);
        }
        if (ab) {
          int32_t yl = mk(MUL, y, mk(LOG, a, -1, t), t);
          int32_t nz = mk(NE, y, cst(0.0, t), t);
          acc(b, mk(MUL, gi, mk(IF_ELSE_ZERO, nz, yl, t), t), false);
        }
        break;
      case SQ: acc(a, mk(MUL, gi, mk(ADD, a, a, t), t), false); break;
      case SQRT: acc(a, mk(DIV, gi, mk(ADD, y, y, t), t), false); break;
      case SIN: acc(a, mk(MUL, gi, mk(COS, a, -1, t), t), false); break;
      case COS: acc(a, mk(MUL, gi, mk(SIN, a, -1, t), t), true); break;
      case TAN: acc(a, mk(MUL, gi, mk(ADD, cst(1.0, t), mk(MUL, y, y, t), t), t), false); break;
      case ATAN: acc(a, mk(DIV, gi, mk(ADD, cst(1.0, t), mk(MUL, a, a, t), t), t), false); break;
      case ATAN2: {
        int32_t r = mk(ADD, mk(MUL, a, a, t), mk(MUL, b, b, t), t);
        int32_t q = mk(DIV, gi, r, t);
        if (aa) acc(a, mk(MUL, q, b, t), false);
        if (ab) acc(b, mk(MUL, q, a, t), true);
        break;
      }
      case TANH: acc(a, mk(MUL, gi, mk(SUB, cst(1.0, t), mk(MUL, y, y, t), t), t), false); break;
      case FABS: acc(a, mk(MUL, gi, mk(SIGN, a, -1, t), t), false); break;
      case FMIN: case FMAX: {
        // the selected operand: a if (a <= b) [fmin] / (b <= a) [fmax], or if b is NaN
        int32_t le = x.op == FMIN ? mk(LE, a, b, t) : mk(LE, b, a, t);
        int32_t c = mk(OR, le, mk(NE, b, b, t), t);
        if (aa) acc(a, mk(IF_ELSE_ZERO, c, gi, t), false);
        if (ab) acc(b, mk(IF_ELSE_ZERO, mk(NOT, c, -1, t), gi, t), false);
        break;
      }
      case FMA_CONST:
        if (aa) acc(a, mk(MUL, gi, cst(x.k, t), t), false);
        acc(b, gi, false);
        break;
      case IF_ELSE_ZERO: acc(b, mk(IF_ELSE_ZERO, a, gi, t), false); break;
      case ASIN: case ACOS: {
        int32_t s = mk(SQRT, mk(SUB, cst(1.0, t), mk(MUL, a, a, t), t), -1, t);
        acc(a, mk(DIV, gi, s, t), x.op == ACOS);
        break;
      }
      case SINH: acc(a, mk(MUL, gi, mk(COSH, a, -1, t), t), false); break;
      case COSH: acc(a, mk(MUL, gi, mk(SINH, a, -1, t), t), false); break;
      case ERF: {
        int32_t e = mk(EXP, mk(NEG, mk(MUL, a, a, t), -1, t), -1, t);
        acc(a, mk(MUL, gi, mk(MUL, cst(1.1283791670955126, t), e, t), t), false);  // 2/sqrt(pi)
        break;
      }
      case INV: acc(a, mk(MUL, gi, mk(MUL, y, y, t), t), true); break;
      case HYPOT: {
        int32_t q = mk(DIV, gi, y, t);
        if (aa) acc(a, mk(MUL, q, a, t), false);
        if (ab) acc(b, mk(MUL, q, b, t), false);
        break;
      }
      case LOG1P: acc(a, mk(DIV, gi, mk(ADD, cst(1.0, t), a, t), t), false); break;
      case EXPM1: acc(a, mk(MUL, gi, mk(ADD, y, cst(1.0, t), t), t), false); break;
      case FMOD: {
        acc(a, gi, false);
        if (ab) {
          int32_t q = mk(DIV, a, b, t);
          int32_t tr = mk(COPYSIGN, mk(FLOOR, mk(FABS, q, -1, t), -1, t), q, t);
          acc(b, mk(MUL, gi, tr, t), true);
        }
        break;
      }
      case COPYSIGN: {
        int32_t s = mk(MUL, mk(COPYSIGN, cst(1.0, t), a, t), mk(COPYSIGN, cst(1.0, t), b, t), t);
        acc(a, mk(MUL, gi, s, t), false);
        break;
      }
      default: break;  // piecewise-constant ops have zero derivative
    }
  }
  // outputs: x_bar rows
  g.out.assign(nin, -1);
  g.out_reduce.assign(nin, 0);
  std::vector<int32_t> input_node(nin, -1);
  for (int32_t i = 0; i < nf; ++i)
    if (fwd.nodes[i].op == INPUT) input_node[fwd.nodes[i].io] = i;
  for (int64_t r = 0; r < nin; ++r) {
    int32_t nd = input_node[r];
    int32_t v = (nd >= 0 && adj[nd] >= 0) ? adj[nd] : -1;
    if (v < 0) v = cst(0.0, nd >= 0 ? fwd.nodes[nd].f64 : 0);
    g.out[r] = v;
    if (fwd.in_bcast[r]) g.out_reduce[r] = 1;
  }
  return g;
}

}  // namespace cusadi
