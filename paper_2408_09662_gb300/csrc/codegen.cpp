// CUDA source generator: one straight-line kernel body per program segment.
//
// CusADi §III-A turns each instruction into one CUDA statement over a global
// work array (Listing 1, Listing 2).  Here each SSA value becomes a local
// variable, so the compiler keeps the work vector in registers; inputs are
// loaded at their first use and outputs stored right after they are computed,
// all instance-fastest so a warp touches 32 consecutive elements per row.
// Programs longer than segment_ops are split into several kernels that pass
// the values live across a cut through a workspace (same SoA layout).
//
// Launch shapes of the one-thread form: R consecutive instances per thread
// (every statement repeated per lane, rows moved as float2/float4/double2
// when the buffers allow), a register cap through the launch bounds, CTA
// barriers every few hundred ops, a register budget that moves the values
// past it to shared-memory slots, workspace rows or re-reads, and pairs of
// out-of-line math calls of the same function issued as one two-argument
// call.  The cooperative form (W warps per 32 instances, its schedule from
// plan_coop in coop.cpp) is generate_coop, further down.
#include <algorithm>
#include <cinttypes>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <sstream>

#include "internal.h"

namespace cusadi {

namespace {

std::string lit(double v, bool f64) {
  char buf[64];
  if (f64) {
    if (std::isnan(v)) return "__longlong_as_double(0x7ff8000000000000ll)";
    if (std::isinf(v)) return v > 0 ? "__longlong_as_double(0x7ff0000000000000ll)"
                                    : "__longlong_as_double((long long)0xfff0000000000000ull)";
    std::snprintf(buf, sizeof buf, "%a", v);
    return std::string("(") + buf + ")";
  }
  float f = (float)v;
  if (std::isnan(f)) return "__int_as_float(0x7fc00000)";
  if (std::isinf(f)) return f > 0 ? "__int_as_float(0x7f800000)" : "__int_as_float((int)0xff800000u)";
  std::snprintf(buf, sizeof buf, "%af", (double)f);
  return std::string("(") + buf + ")";
}

struct MathFn {
  const char* d;
  const char* f;
};

MathFn math_name(int op) {
  switch (op) {
    case EXP: return {"exp", "expf"};
    case LOG: return {"log", "logf"};
    case POW: return {"pow", "powf"};
    case SIN: return {"sin", "sinf"};
    case COS: return {"cos", "cosf"};
    case TAN: return {"tan", "tanf"};
    case ATAN: return {"atan", "atanf"};
    case ATAN2: return {"atan2", "atan2f"};
    case TANH: return {"tanh", "tanhf"};
    case ASIN: return {"asin", "asinf"};
    case ACOS: return {"acos", "acosf"};
    case SINH: return {"sinh", "sinhf"};
    case COSH: return {"cosh", "coshf"};
    case ERF: return {"erf", "erff"};
    case FMOD: return {"fmod", "fmodf"};
    case HYPOT: return {"hypot", "hypotf"};
    case LOG1P: return {"log1p", "log1pf"};
    case EXPM1: return {"expm1", "expm1f"};
    case SQRT: return {"sqrt", "sqrtf"};
    case FABS: return {"fabs", "fabsf"};
    case FMIN: return {"fmin", "fminf"};
    case FMAX: return {"fmax", "fmaxf"};
    case FLOOR: return {"floor", "floorf"};
    case CEIL: return {"ceil", "ceilf"};
    case COPYSIGN: return {"copysign", "copysignf"};
  }
  return {"?", "?"};
}

struct Gen {
  const Graph& g;
  const CodegenOptions& o;
  std::vector<int> seg_of;          // per node (leaves: -1)
  std::vector<int> last_seg;        // last segment that reads the node
  std::vector<int64_t> ws_slot;     // workspace row of values crossing a cut
  std::vector<std::vector<int64_t>> out_rows;  // per node: output rows it feeds
  std::set<std::pair<int, bool>> calls;        // (op, f64) of out-of-line math used
  std::set<std::pair<int, bool>> calls2;       // (op, f64) of the paired (two-argument) versions
  bool own_f32 = false;                        // own FP32 sin/cos/exp used

  Gen(const Graph& g_, const CodegenOptions& o_) : g(g_), o(o_) {}

  bool node_f64(int32_t i) const {
    if (o.dtype == CUSADI_F64) return true;
    if (o.dtype == CUSADI_F32) return false;
    return g.nodes[i].f64 != 0;
  }
  const char* ty(bool f64) const { return f64 ? "double" : "float"; }
  bool buf_f64() const { return o.dtype == CUSADI_F64; }
  bool ws_f64() const { return o.dtype != CUSADI_F32; }
  bool leaf(int32_t i) const { return g.nodes[i].op == INPUT || g.nodes[i].op == CONST; }
};

// Whether op is inlined at its uses (else one out-of-line function per op and
// precision, called from every use).
bool inlined(int op, int inline_math) {
  if (inline_math == 1) return true;
  if (inline_math == 2) return op == EXP || op == EXPM1 || op == LOG || op == LOG1P;
  return false;
}

// __launch_bounds__ of a kernel of `threads` threads per CTA: a register cap
// becomes the minimum number of resident CTAs per SM that leaves each thread
// at most that many registers (a plain --maxrregcount is ignored for kernels
// with launch bounds).
std::string launch_bounds(int threads, int maxrregcount) {
  std::string s = "__launch_bounds__(" + std::to_string(threads);
  if (maxrregcount > 0) s += ", " + std::to_string(std::max(1, 65536 / (threads * maxrregcount)));
  return s + ")";
}

std::string call_name(int op, bool f64, bool inl) {
  MathFn m = math_name(op);
  if (inl) return f64 ? m.d : m.f;
  return std::string("cs_") + m.d + (f64 ? "_d" : "_f");
}

// The engine's own single-precision sin, cos and exp (FP32 ops when the
// library's are not inlined): Cody & Waite argument reduction with an FMA per
// step and near-minimax polynomials; constants from csrc/gen_math_coeffs.py.
// sin/cos take the fast path for |x| <= 128 * pi/2, where the 17-bit leading
// parts of pi/2 make j * part exact; anything else (and inf/NaN) goes to the
// library function.  Branch-free apart from that rare fallback.
bool own_f32_math(int op) { return op == SIN || op == COS || op == EXP; }

const char* kOwnMathF32 = R"(static __device__ __noinline__ float cs_sin_slow(float a) { return sinf(a); }
static __device__ __noinline__ float cs_cos_slow(float a) { return cosf(a); }
static __device__ __forceinline__ void cs_sincos_core(float x, float& s, float& c, int& q) {
  const float j = rintf(x * 0x1.45f306p-1f);
  float r = fmaf(-j, 0x1.922p+0f, x);
  r = fmaf(-j, -0x1.2aefp-18f, r);
  r = fmaf(-j, 0x1.68c234p-39f, r);
  q = (int)j;
  const float t = r * r;
  s = fmaf(r * t, fmaf(t, fmaf(t, -0x1.9943ep-13f, 0x1.11073ap-7f), -0x1.555546p-3f), r);
  c = fmaf(t, fmaf(t, fmaf(t, fmaf(t, 0x1.99169ep-16f, -0x1.6c07f2p-10f), 0x1.55553cp-5f), -0x1p-1f), 1.0f);
}
static __device__ __forceinline__ float cs_own_sin_f(float x) {
  if (!(fabsf(x) <= 201.0f)) return cs_sin_slow(x);
  float s, c; int q;
  cs_sincos_core(x, s, c, q);
  const float v = (q & 1) ? c : s;
  return (q & 2) ? -v : v;
}
static __device__ __forceinline__ float cs_own_cos_f(float x) {
  if (!(fabsf(x) <= 201.0f)) return cs_cos_slow(x);
  float s, c; int q;
  cs_sincos_core(x, s, c, q);
  const float v = (q & 1) ? s : c;
  return ((q + 1) & 2) ? -v : v;
}
static __device__ __forceinline__ float cs_own_exp_f(float x) {
  const float xc = x < -104.0f ? -104.0f : (x > 89.0f ? 89.0f : x);
  const float k = rintf(xc * 0x1.715476p+0f);
  float r = fmaf(-k, 0x1.62e4p-1f, xc);
  r = fmaf(-k, 0x1.7f7d1cp-20f, r);
  float p = fmaf(r, 0x1.6a2448p-10f, 0x1.1239d4p-7f);
  p = fmaf(r, p, 0x1.5558f2p-5f);
  p = fmaf(r, p, 0x1.555492p-3f);
  p = fmaf(r, p, 0x1.fffffcp-2f);
  p = fmaf(r * r, p, r) + 1.0f;
  const int ki = (int)k, k1 = ki >> 1, k2 = ki - k1;
  return (p * __int_as_float((k1 + 127) << 23)) * __int_as_float((k2 + 127) << 23);
}
)";

// Own math as generated: mode 1 inlines sin/cos/exp at every use, mode 2 makes
// them out-of-line functions (one copy of the code, a call per use).
std::string own_math_source(int mode) {
  std::string t = kOwnMathF32;
  if (mode == 2) {
    const std::string a = "__forceinline__ float cs_own_", b = "__noinline__ float cs_own_";
    for (size_t p = t.find(a); p != std::string::npos; p = t.find(a, p + b.size())) t.replace(p, a.size(), b);
  }
  return t;
}

// Accesses of NL consecutive instances of one row by one thread (NL = 2 or 4):
// one vector load/store when `full` (the caller checked alignment and that all
// NL instances are inside the batch), else one element at a time, the lanes
// past the batch's end reading lane 0's element and storing nothing.
const char* kLaneAccess = R"(template <typename T> struct cs_vec2;
template <> struct cs_vec2<float> { typedef float2 t; };
template <> struct cs_vec2<double> { typedef double2 t; };
template <typename T>
static __device__ __forceinline__ void cs_ld2(const T* __restrict__ p, bool full, int m, T& a, T& b) {
  if (full) { const typename cs_vec2<T>::t v = *reinterpret_cast<const typename cs_vec2<T>::t*>(p); a = v.x; b = v.y; }
  else { a = p[0]; b = m > 1 ? p[1] : a; }
}
template <typename T>
static __device__ __forceinline__ void cs_st2(T* __restrict__ p, bool full, int m, T a, T b) {
  if (full) { typename cs_vec2<T>::t v; v.x = a; v.y = b; *reinterpret_cast<typename cs_vec2<T>::t*>(p) = v; }
  else { p[0] = a; if (m > 1) p[1] = b; }
}
static __device__ __forceinline__ void cs_ld4(const float* __restrict__ p, bool full, int m, float& a, float& b,
                                              float& c, float& d) {
  if (full) { const float4 v = *reinterpret_cast<const float4*>(p); a = v.x; b = v.y; c = v.z; d = v.w; }
  else { a = p[0]; b = m > 1 ? p[1] : a; c = m > 2 ? p[2] : a; d = m > 3 ? p[3] : a; }
}
static __device__ __forceinline__ void cs_st4(float* __restrict__ p, bool full, int m, float a, float b, float c,
                                              float d) {
  if (full) *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
  else { p[0] = a; if (m > 1) p[1] = b; if (m > 2) p[2] = c; if (m > 3) p[3] = d; }
}
static __device__ __forceinline__ void cs_ld4(const double* __restrict__ p, bool full, int m, double& a, double& b,
                                              double& c, double& d) {
  if (full) { cs_ld2(p, true, 2, a, b); cs_ld2(p + 2, true, 2, c, d); }
  else { a = p[0]; b = m > 1 ? p[1] : a; c = m > 2 ? p[2] : a; d = m > 3 ? p[3] : a; }
}
static __device__ __forceinline__ void cs_st4(double* __restrict__ p, bool full, int m, double a, double b,
                                              double c, double d) {
  if (full) { cs_st2(p, true, 2, a, b); cs_st2(p + 2, true, 2, c, d); }
  else { p[0] = a; if (m > 1) p[1] = b; if (m > 2) p[2] = c; if (m > 3) p[3] = d; }
}
)";

// C expression of one op with operand expressions A, B in precision f.
std::string op_expr(Gen& G, const Node& x, bool f, const std::string& A, const std::string& B,
                    const CodegenOptions& o) {
  const char* T = G.ty(f);
  std::string Z = std::string("(") + T + ")0", One = std::string("(") + T + ")1";
  std::string e;
  MathFn m = math_name(x.op);
  const char* mn = f ? m.d : m.f;
  switch (x.op) {
    case ADD: e = A + " + " + B; break;
    case SUB: e = A + " - " + B; break;
    case MUL: e = A + " * " + B; break;
    case DIV: e = A + " / " + B; break;
    case NEG: e = "-" + A; break;
    case SQ: e = A + " * " + A; break;
    case INV: e = One + " / " + A; break;
    case SQRT: case FABS: case FLOOR: case CEIL: e = std::string(mn) + "(" + A + ")"; break;
    case FMIN: case FMAX: case COPYSIGN: e = std::string(mn) + "(" + A + ", " + B + ")"; break;
    case FMA_CONST: e = std::string(f ? "fma(" : "fmaf(") + lit(x.k, f) + ", " + A + ", " + B + ")"; break;
    case IF_ELSE_ZERO: e = "(" + A + " != " + Z + " ? " + B + " : " + Z + ")"; break;
    case LT: e = "(" + A + " < " + B + " ? " + One + " : " + Z + ")"; break;
    case LE: e = "(" + A + " <= " + B + " ? " + One + " : " + Z + ")"; break;
    case EQ: e = "(" + A + " == " + B + " ? " + One + " : " + Z + ")"; break;
    case NE: e = "(" + A + " != " + B + " ? " + One + " : " + Z + ")"; break;
    case NOT: e = "(" + A + " == " + Z + " ? " + One + " : " + Z + ")"; break;
    case AND: e = "((" + A + " != " + Z + " && " + B + " != " + Z + ") ? " + One + " : " + Z + ")"; break;
    case OR: e = "((" + A + " != " + Z + " || " + B + " != " + Z + ") ? " + One + " : " + Z + ")"; break;
    case SIGN: e = "(" + A + " > " + Z + " ? " + One + " : (" + A + " < " + Z + " ? -" + One + " : " + Z + "))"; break;
    default:
      if (!f && o.inline_math != 1 && o.own_math && own_f32_math(x.op)) {
        G.own_f32 = true;
        e = std::string(x.op == SIN ? "cs_own_sin_f(" : (x.op == COS ? "cs_own_cos_f(" : "cs_own_exp_f(")) + A + ")";
      } else if (op_call(x.op)) {
        const bool inl = inlined(x.op, o.inline_math);
        if (!inl) G.calls.insert({x.op, f});
        e = call_name(x.op, f, inl) + "(" + A + (op_arity(x.op) == 2 ? ", " + B : "") + ")";
      } else {
        e = "/* unsupported op */ " + Z;
      }
  }
  return e;
}

}  // namespace

std::string finish_source(CodegenResult& R, const std::string& prefix, const char* tin,
                          const char* tw);

CodegenResult generate(const Graph& g, const CodegenOptions& o) {
  CodegenResult R;
  Gen G(g, o);
  const int64_t n = (int64_t)g.nodes.size();
  G.seg_of.assign(n, -1);
  G.last_seg.assign(n, -1);
  G.out_rows.assign(n, {});
  for (size_t r = 0; r < g.out.size(); ++r) G.out_rows[g.out[r]].push_back((int64_t)r);

  // segment cuts by op count
  std::vector<std::pair<int64_t, int64_t>> segs;
  {
    int64_t start = 0, ops = 0;
    for (int64_t i = 0; i < n; ++i) {
      if (G.leaf(i)) continue;
      if (o.segment_ops > 0 && ops >= o.segment_ops) {
        segs.push_back({start, i});
        start = i;
        ops = 0;
      }
      ++ops;
    }
    segs.push_back({start, n});
  }
  const int nseg = (int)segs.size();
  for (int s = 0; s < nseg; ++s)
    for (int64_t i = segs[s].first; i < segs[s].second; ++i)
      if (!G.leaf(i)) G.seg_of[i] = s;
  for (int64_t i = 0; i < n; ++i) {
    const Node& x = g.nodes[i];
    if (G.leaf(i)) continue;
    for (int32_t a : {x.a, x.b})
      if (a >= 0 && !G.leaf(a)) G.last_seg[a] = std::max(G.last_seg[a], G.seg_of[i]);
  }
  // workspace rows for values read in a later segment; a row is free again for
  // values defined after the segment of its last reader
  G.ws_slot.assign(n, -1);
  {
    std::vector<std::vector<int64_t>> release(nseg + 1);
    std::vector<int64_t> free_rows;
    int64_t rows = 0;
    for (int s = 0; s < nseg; ++s) {
      for (int64_t r : release[s > 0 ? s - 1 : nseg]) free_rows.push_back(r);
      if (s > 0) release[s - 1].clear();
      for (int64_t i = segs[s].first; i < segs[s].second; ++i) {
        if (G.leaf(i) || G.last_seg[i] <= s) continue;
        int64_t r;
        if (!free_rows.empty()) { r = free_rows.back(); free_rows.pop_back(); }
        else r = rows++;
        G.ws_slot[i] = r;
        release[G.last_seg[i]].push_back(r);
      }
    }
    R.ws_rows = rows;
  }
  for (uint8_t f : g.out_reduce) R.has_reduce |= (f != 0);
  std::vector<int64_t> reduce_k(g.out_reduce.size(), -1);
  for (size_t r = 0; r < g.out_reduce.size(); ++r)
    if (g.out_reduce[r]) {
      reduce_k[r] = (int64_t)R.reduce_rows.size();
      R.reduce_rows.push_back((int64_t)r);
    }

  const char* tin = G.buf_f64() ? "double" : "float";
  const char* tw = G.ws_f64() ? "double" : "float";
  // Register budget (spill_values > 0, one instance per thread): per segment, a
  // linear scan over the values' live ranges in statement order keeps at most
  // spill_values of them in registers; when a value finds the budget full,
  // whichever of it and the live register values is read last leaves the
  // registers for its whole life (M. Poletto and V. Sarkar, "Linear scan
  // register allocation", TOPLAS 1999).  An input or a value carried from an
  // earlier kernel is then re-read from its buffer at each use; a computed value
  // is stored once to a shared-memory slot (spill_shared_kb per CTA), or beyond
  // those to a workspace row, and re-read at each use.  Accesses go through
  // volatile pointers so that the compiler does not keep the value in a register.
  enum { SP_REG = 0, SP_SMEM = 1, SP_WS = 2, SP_RELOAD = 3 };
  // where each value lives in the segment being generated (a value carried into
  // a later segment is placed afresh there)
  std::vector<uint8_t> sp_kind(n, SP_REG);
  std::vector<int64_t> sp_idx(n, -1);
  const bool spill = o.spill_values > 0 && !o.device_fn && std::max(1, o.inst_per_thread) == 1;
  const int64_t sp_cap_sm = (int64_t)o.spill_shared_kb * 1024 / ((int64_t)o.block * (G.ws_f64() ? 8 : 4));
  const int64_t sp_ws_base = R.ws_rows;   // spill rows follow the carried rows
  // fills sp_kind / sp_idx for segment s; returns (shared slots, workspace rows) used
  auto spill_segment = [&](int s) -> std::pair<int64_t, int64_t> {
    std::fill(sp_kind.begin(), sp_kind.end(), (uint8_t)SP_REG);
    std::fill(sp_idx.begin(), sp_idx.end(), (int64_t)-1);
    // positions: materialised operands of op i at 2i, its result at 2i + 1
    std::vector<int64_t> def(n, -1), end(n, -1), order;
    for (int64_t i = segs[s].first; i < segs[s].second; ++i) {
      if (G.leaf(i)) continue;
      const Node& x = g.nodes[i];
      for (int32_t a : {x.a, x.b}) {
        if (a < 0 || g.nodes[a].op == CONST) continue;
        const bool outside = g.nodes[a].op == INPUT || G.seg_of[a] != s;
        if (outside && def[a] < 0) { def[a] = 2 * i; order.push_back(a); }
        end[a] = std::max(end[a], 2 * i + 1);
      }
      def[i] = 2 * i + 1;
      end[i] = std::max(end[i], def[i]);
      order.push_back(i);
    }
    std::set<std::pair<int64_t, int64_t>> active;   // (end, value) in registers
    std::vector<int64_t> spilled;
    for (int64_t v : order) {
      while (!active.empty() && active.begin()->first <= def[v]) active.erase(active.begin());
      if ((int64_t)active.size() < o.spill_values) { active.insert({end[v], v}); continue; }
      auto last = std::prev(active.end());
      if (last->first > end[v]) {
        spilled.push_back(last->second);
        active.erase(last);
        active.insert({end[v], v});
      } else {
        spilled.push_back(v);
      }
    }
    // memory slots of the spilled computed values: shared first, then workspace rows
    std::sort(spilled.begin(), spilled.end(), [&](int64_t a, int64_t c) { return def[a] < def[c]; });
    std::set<std::pair<int64_t, int64_t>> live_sm, live_ws;   // (end, slot)
    std::vector<int64_t> free_sm, free_ws;
    int64_t next_sm = 0, next_ws = 0;
    for (int64_t v : spilled) {
      if (def[v] % 2 == 0) { sp_kind[v] = SP_RELOAD; continue; }   // input / carried value
      while (!live_sm.empty() && live_sm.begin()->first <= def[v]) { free_sm.push_back(live_sm.begin()->second); live_sm.erase(live_sm.begin()); }
      while (!live_ws.empty() && live_ws.begin()->first <= def[v]) { free_ws.push_back(live_ws.begin()->second); live_ws.erase(live_ws.begin()); }
      int64_t k;
      if (!free_sm.empty() || next_sm < sp_cap_sm) {
        if (!free_sm.empty()) { k = free_sm.back(); free_sm.pop_back(); } else k = next_sm++;
        sp_kind[v] = SP_SMEM; sp_idx[v] = k; live_sm.insert({end[v], k});
      } else {
        if (!free_ws.empty()) { k = free_ws.back(); free_ws.pop_back(); } else k = next_ws++;
        sp_kind[v] = SP_WS; sp_idx[v] = sp_ws_base + k; live_ws.insert({end[v], k});
      }
    }
    return {next_sm, next_ws};
  };
  if (spill) {   // sizes: the most any segment needs (the segments run one after the other)
    int64_t sm = 0, ws = 0;
    for (int s = 0; s < nseg; ++s) {
      auto u = spill_segment(s);
      sm = std::max(sm, u.first);
      ws = std::max(ws, u.second);
    }
    R.ws_rows += ws;
    R.smem_bytes = sm * o.block * (G.ws_f64() ? 8 : 4);
  }
  // Lanes: a kernel thread evaluates NL consecutive instances i .. i + NL - 1,
  // op by op in turn; their inputs and outputs move as one vector access when
  // the buffers allow it.  A kernel thread past the end of the batch still runs
  // (CTA barriers need it) on the last thread's instances, storing nothing.
  const int NL = o.device_fn ? 1 : std::max(1, o.inst_per_thread);
  const bool clamped = o.adjoint || NL > 1 || (o.sync_every > 0 && !o.device_fn);
  R.inst_per_thread = NL;
  auto vname = [&](int64_t i, int r) {
    return NL == 1 ? "v" + std::to_string(i) : "v" + std::to_string(i) + "_" + std::to_string(r);
  };
  // a comma-separated list of the NL lane names of node i
  auto lanes = [&](int64_t i) {
    std::string l;
    for (int r = 0; r < NL; ++r) l += (r ? ", " : "") + vname(i, r);
    return l;
  };

  // Paired calls: an out-of-line unary math call (sin, cos, exp, ...) is issued
  // together with a later call of the same function whose argument is already
  // computed, as one call of a two-argument version: half the call overhead, and
  // the two evaluations inside it are independent work the compiler can overlap.
  const bool pairing = o.pair_calls > 0 && NL == 1 && !spill && o.inline_math != 1;
  auto pairable = [&](int64_t i) {
    const Node& x = g.nodes[i];
    if (G.leaf(i) || !op_call(x.op) || op_arity(x.op) != 1 || inlined(x.op, o.inline_math)) return false;
    return !( !G.node_f64((int32_t)i) && o.own_math && own_f32_math(x.op));
  };
  std::vector<int64_t> partner(n, -1);
  std::vector<uint8_t> hoisted(n, 0);
  for (int s = 0; s < nseg; ++s) {
    if (spill) spill_segment(s);
    if (pairing) {
      for (int64_t i = segs[s].first; i < segs[s].second; ++i) {
        if (!pairable(i) || hoisted[i]) continue;
        const int64_t lim = std::min<int64_t>(segs[s].second, i + 1 + o.pair_calls);
        for (int64_t j = i + 1; j < lim; ++j) {
          if (!pairable(j) || hoisted[j] || partner[j] >= 0 || g.nodes[j].op != g.nodes[i].op ||
              G.node_f64((int32_t)j) != G.node_f64((int32_t)i))
            continue;
          const int32_t a = g.nodes[j].a;   // available at i: a leaf, carried in, or computed before i
          if (!(G.leaf(a) || G.seg_of[a] != s || a < i)) continue;
          partner[i] = j;
          hoisted[j] = 1;
          break;
        }
      }
    }
    std::ostringstream body;
    std::vector<uint8_t> have(n, 0);   // leaf or ws value materialised in this segment
    std::vector<uint8_t> decl_buf(n, 0);  // lanes declared with the buffer's type, not the op's
    G.calls.clear();
    G.calls2.clear();
    G.own_f32 = false;
    auto operand = [&](int32_t i, bool want_f64, int r) -> std::string {
      const Node& x = g.nodes[i];
      bool f = G.node_f64(i);
      if (x.op == CONST) return lit(x.k, want_f64);
      if (spill && sp_kind[i] != SP_REG) {
        // read at each use from where the value lives
        const char* W2 = G.ty(want_f64);
        if (sp_kind[i] == SP_SMEM)
          return std::string("((") + W2 + ")cs_sp[" + std::to_string(sp_idx[i]) + " * blockDim.x])";
        if (sp_kind[i] == SP_WS)
          return std::string("((") + W2 + ")Wv[" + std::to_string(sp_idx[i]) + "ll * ldw])";
        if (x.op == INPUT) {
          const bool second = o.split >= 0 && x.io >= o.split;
          const int64_t row = second ? x.io - o.split : x.io;
          const std::string base = second ? (x.bcast ? "X2b" : "X2") : (x.bcast ? "Xb" : "X");
          return std::string("((") + W2 + ")((const volatile " + tin + "*)" + base + ")[" + std::to_string(row) +
                 (second ? "ll * ldx2])" : "ll * ldx])");
        }
        return std::string("((") + W2 + ")Wv[" + std::to_string(G.ws_slot[i]) + "ll * ldw])";
      }
      if (x.op == INPUT) {
        if (!have[i]) {
          have[i] = 1;
          const bool second = o.split >= 0 && x.io >= o.split;
          const int64_t row = second ? x.io - o.split : x.io;
          const std::string src = std::string(second ? (x.bcast ? "X2b[" : "X2[") : (x.bcast ? "Xb[" : "X[")) +
                                  std::to_string(row) + (second ? "ll * ldx2]" : "ll * ldx]");
          if (NL == 1 || x.bcast) {
            // a broadcast row holds one value for every instance: all lanes share it
            body << "  const " << G.ty(f) << " v" << i << " = (" << G.ty(f) << ")" << src << ";\n";
          } else {
            decl_buf[i] = 1;
            body << "  " << tin << " " << lanes(i) << ";\n"
                 << "  cs_ld" << NL << "(&" << src << ", full, m, " << lanes(i) << ");\n";
          }
        }
        std::string name = (NL == 1 || x.bcast) ? "v" + std::to_string(i) : vname(i, r);
        const bool df = decl_buf[i] ? G.buf_f64() : f;
        if (df != want_f64) return std::string("(") + G.ty(want_f64) + ")" + name;
        return name;
      }
      if (G.seg_of[i] != s) {
        if (!have[i]) {
          have[i] = 1;
          if (NL == 1) {
            body << "  const " << G.ty(f) << " v" << i << " = (" << G.ty(f) << ")W["
                 << G.ws_slot[i] << "ll * ldw];\n";
          } else {
            decl_buf[i] = 1;   // workspace columns are padded to 32: always whole vectors
            body << "  " << tw << " " << lanes(i) << ";\n"
                 << "  cs_ld" << NL << "(&W[" << G.ws_slot[i] << "ll * ldw], true, " << NL << ", "
                 << lanes(i) << ");\n";
          }
        }
      }
      const bool df = decl_buf[i] ? G.ws_f64() : f;
      if (df != want_f64) return std::string("(") + G.ty(want_f64) + ")" + vname(i, r);
      return vname(i, r);
    };
    // stores of output row r of node i (values v[lane])
    auto store_out = [&](int64_t r, const std::vector<std::string>& v) {
      if (o.adjoint) {
        for (int l = 0; l < NL; ++l) {
          const std::string guard = NL == 1 ? "active" : "active && m > " + std::to_string(l);
          const std::string off = NL == 1 ? "" : " + " + std::to_string(l);
          const std::string plain = "if (" + guard + ") { " + tin + "* p_ = &Y[" + std::to_string(r) +
                                    "ll * ldy" + off + "]; *p_ = acc ? *p_ + (" + tin + ")" + v[l] + " : (" +
                                    tin + ")" + v[l] + "; }";
          if (g.out_reduce[r]) {
            // the instance's term goes to the workspace (a coalesced store); the
            // finishing kernel sums each such row over the instances
            body << "  if (reduce) {\n    if (" << guard << ") Wp[" << reduce_k[r] << "ll * ldw" << off
                 << "] = (" << tw << ")" << v[l] << ";\n  } else " << plain << "\n";
          } else {
            body << "  " << plain << "\n";
          }
        }
      } else if (NL == 1) {
        body << "  " << (clamped ? "if (active) " : "") << "Y[" << r << "ll * ldy] = (" << tin << ")" << v[0] << ";\n";
      } else {
        body << "  if (active) cs_st" << NL << "(&Y[" << r << "ll * ldy], full, m";
        for (int l = 0; l < NL; ++l) body << ", (" << tin << ")" << v[l];
        body << ");\n";
      }
      if (o.debug_checks && !o.device_fn)   // count non-finite results (cusadi_debug_count)
        for (int l = 0; l < NL; ++l)
          body << "  if (active" << (NL == 1 ? "" : " && m > " + std::to_string(l)) << " && !isfinite((double)("
               << v[l] << "))) atomicAdd(&cs_dbg, 1u);\n";
    };
    auto lane_values = [&](int64_t i, bool f) {
      std::vector<std::string> v;
      for (int l = 0; l < NL; ++l) v.push_back(G.leaf(i) ? operand((int32_t)i, f, l) : vname(i, l));
      return v;
    };
    // outputs fed directly by inputs or constants are written by segment 0
    if (s == 0) {
      for (int64_t i = 0; i < n; ++i) {
        if (!G.leaf(i) || G.out_rows[i].empty()) continue;
        std::vector<std::string> v = lane_values(i, G.node_f64((int32_t)i));
        for (int64_t r : G.out_rows[i]) store_out(r, v);
      }
    }
    int64_t since_sync = 0;
    for (int64_t i = segs[s].first; i < segs[s].second; ++i) {
      if (G.leaf(i)) continue;
      const Node& x = g.nodes[i];
      const bool f = G.node_f64((int32_t)i);
      const char* T = G.ty(f);
      if (pairing && partner[i] >= 0) {
        const int64_t j = partner[i];
        std::string A = operand(x.a, f, 0), Aj = operand(g.nodes[j].a, f, 0);
        G.calls2.insert({x.op, f});
        MathFn m = math_name(x.op);
        body << "  const " << T << "2 p" << i << " = cs_" << m.d << "2" << (f ? "_d" : "_f") << "(" << A
             << ", " << Aj << ");\n"
             << "  const " << T << " v" << i << " = p" << i << ".x;\n"
             << "  const " << T << " v" << j << " = p" << i << ".y;\n";
      } else if (!(pairing && hoisted[i])) {    // a hoisted op was computed with its partner
        for (int l = 0; l < NL; ++l) {
          std::string A = x.a >= 0 ? operand(x.a, f, l) : "";
          std::string B = x.b >= 0 ? operand(x.b, f, l) : "";
          body << "  const " << T << " " << vname(i, l) << " = " << op_expr(G, x, f, A, B, o) << ";\n";
        }
      }
      if (spill && sp_kind[i] == SP_SMEM)
        body << "  cs_sp[" << sp_idx[i] << " * blockDim.x] = (" << tw << ")v" << i << ";\n";
      else if (spill && sp_kind[i] == SP_WS)
        body << "  Wv[" << sp_idx[i] << "ll * ldw] = (" << tw << ")v" << i << ";\n";
      if (G.ws_slot[i] >= 0) {
        if (NL == 1) {
          body << "  if (active) W[" << G.ws_slot[i] << "ll * ldw] = (" << tw << ")v" << i << ";\n";
        } else {
          body << "  if (active) cs_st" << NL << "(&W[" << G.ws_slot[i] << "ll * ldw], true, " << NL;
          for (int l = 0; l < NL; ++l) body << ", (" << tw << ")" << vname(i, l);
          body << ");\n";
        }
      }
      if (!G.out_rows[i].empty()) {
        std::vector<std::string> v = lane_values(i, f);
        for (int64_t r : G.out_rows[i]) store_out(r, v);
      }
      if (o.sync_every > 0 && !o.device_fn && ++since_sync >= o.sync_every) {
        body << "  __syncthreads();\n";
        since_sync = 0;
      }
    }

    std::ostringstream src;
    src << "// Generated straight-line kernel: segment " << s << " of " << nseg
        << (o.adjoint ? " (adjoint)" : "") << ", dtype "
        << (o.dtype == CUSADI_F64 ? "f64" : (o.dtype == CUSADI_F32 ? "f32" : "mixed"));
    if (NL > 1) src << ", " << NL << " instances per thread";
    if (o.sync_every > 0 && !o.device_fn) src << ", CTA barrier every " << o.sync_every << " ops";
    src << "\n";
    if (NL > 1) src << kLaneAccess;
    if (G.own_f32) src << own_math_source(o.own_math);
    if (o.debug_checks && !o.device_fn) src << "__device__ unsigned int cs_dbg;   // non-finite results\n";
    {
      for (auto& c : G.calls) {
        MathFn m = math_name(c.first);
        const char* t = c.second ? "double" : "float";
        bool bin = op_arity(c.first) == 2;
        src << "static __device__ __noinline__ " << t << " " << call_name(c.first, c.second, false) << "("
            << t << " a" << (bin ? std::string(", ") + t + " b" : "") << ") { return "
            << (c.second ? m.d : m.f) << "(a" << (bin ? ", b" : "") << "); }\n";
      }
      for (auto& c : G.calls2) {   // two independent evaluations per call
        MathFn m = math_name(c.first);
        const char* t = c.second ? "double" : "float";
        const char* fn = c.second ? m.d : m.f;
        src << "static __device__ __noinline__ " << t << "2 cs_" << m.d << "2" << (c.second ? "_d" : "_f")
            << "(" << t << " a, " << t << " b) { " << t << "2 r; r.x = " << fn << "(a); r.y = " << fn
            << "(b); return r; }\n";
      }
    }
    std::string name = o.prefix + "_" + std::to_string(s);
    if (o.device_fn) {
      // one instance per call; the caller owns the index and the bounds check
      src << "extern \"C\" __device__ void " << name << "(\n"
          << "    const " << tin << "* __restrict__ X, long long ldx, const " << tin
          << "* __restrict__ X2, long long ldx2, " << tin
          << "* __restrict__ Y, long long ldy,\n    " << tw
          << "* __restrict__ W, long long ldw, long long i) {\n"
          << "  const bool active = true;\n  const int acc = 0, reduce = 0;\n"
          << "  const " << tin << "* __restrict__ Xb = X;\n"
          << "  const " << tin << "* __restrict__ X2b = X2;\n"
          << "  " << tin << "* __restrict__ Yb = Y;\n"
          << "  X += i; X2 += i; Y += i; W += i;\n"
          << "  (void)Xb; (void)X2b; (void)Yb; (void)W; (void)ldw; (void)ldx2; (void)acc; (void)reduce; (void)active;\n"
          << body.str() << "}\n";
      Segment S;
      S.begin = segs[s].first;
      S.end = segs[s].second;
      S.name = name;
      S.source = src.str();
      R.segs.push_back(std::move(S));
      continue;
    }
    src << "extern \"C\" __global__ void " << launch_bounds(o.block, o.maxrregcount) << " " << name << "(\n"
        << "    const " << tin << "* __restrict__ X, long long ldx, const " << tin
        << "* __restrict__ X2, long long ldx2, " << tin
        << "* __restrict__ Y, long long ldy,\n    long long N, " << tw
        << "* __restrict__ W, long long ldw, int acc, int reduce, int vec) {\n";
    if (NL == 1) {
      src << "  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;\n";
      if (clamped) {
        src << "  const bool active = i0 < N;\n"
            << "  const long long i = active ? i0 : N - 1;\n";
      } else {
        src << "  if (i0 >= N) return;\n  const bool active = true;\n  const long long i = i0;\n";
      }
    } else {
      // m: instances of this thread inside the batch; full: whole vector accesses
      src << "  const long long i0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * " << NL << ";\n"
          << "  const bool active = i0 < N;\n"
          << "  const long long i = active ? i0 : (N - 1) / " << NL << " * " << NL << ";\n"
          << "  const int m = N - i < " << NL << " ? (int)(N - i) : " << NL << ";\n"
          << "  const bool full = vec != 0 && m == " << NL << ";\n";
    }
    src << "  const " << tin << "* __restrict__ Xb = X;\n"
        << "  const " << tin << "* __restrict__ X2b = X2;\n"
        << "  " << tin << "* __restrict__ Yb = Y;\n";
    if (spill)   // values kept out of registers: shared slots and workspace rows, never cached
      src << "  extern __shared__ __align__(16) unsigned char cs_smem[];\n"
          << "  volatile " << tw << "* const cs_sp = reinterpret_cast<volatile " << tw
          << "*>(cs_smem) + threadIdx.x;\n"
          << "  volatile " << tw << "* const Wv = W + i;\n"
          << "  (void)cs_sp; (void)Wv;\n";
    if (o.adjoint && R.has_reduce)
      src << "  " << tw << "* __restrict__ Wp = W + " << R.ws_rows << "ll * ldw + i;  // reduced-row terms\n";
    src << "  X += i; X2 += i; Y += i; W += i;\n"
        << "  (void)Xb; (void)X2b; (void)Yb; (void)W; (void)ldw; (void)ldx2; (void)acc; (void)reduce; (void)active; (void)vec;\n"
        << body.str() << "}\n";
    Segment S;
    S.begin = segs[s].first;
    S.end = segs[s].second;
    S.name = name;
    S.source = src.str();
    R.segs.push_back(std::move(S));
  }
  if (R.has_reduce) R.segs[0].source += finish_source(R, o.prefix, tin, tw);
  return R;
}

// One CTA per reduced row adds the row's N per-instance terms in a fixed order
// (strided per thread, then a tree), so the sum is the same on every run; it
// then writes, or adds to, the row's column 0.
std::string finish_source(CodegenResult& R, const std::string& prefix, const char* tin,
                          const char* tw) {
  {
    std::ostringstream z;
    R.finish_kernel = prefix + "_finish";
    z << "static __device__ const long long cs_reduce_row[] = {";
    for (size_t k = 0; k < R.reduce_rows.size(); ++k) z << (k ? ", " : "") << R.reduce_rows[k];
    z << "};\n"
      << "extern \"C\" __global__ void __launch_bounds__(512) " << R.finish_kernel << "(const " << tw
      << "* __restrict__ W, long long ldw, long long N, " << tin << "* __restrict__ Y, long long ldy, "
      << "int accumulate) {\n"
      << "  __shared__ " << tw << " s_[512];\n"
      << "  const " << tw << "* __restrict__ P = W + (" << R.ws_rows << "ll + blockIdx.x) * ldw;\n"
      << "  " << tw << " a = 0;\n"
      << "  for (long long j = threadIdx.x; j < N; j += 512) a += P[j];\n"
      << "  s_[threadIdx.x] = a;\n"
      << "  __syncthreads();\n"
      << "  for (int d = 256; d > 0; d >>= 1) {\n"
      << "    if ((int)threadIdx.x < d) s_[threadIdx.x] += s_[threadIdx.x + d];\n"
      << "    __syncthreads();\n"
      << "  }\n"
      << "  if (threadIdx.x == 0) {\n"
      << "    " << tin << "* p = &Y[cs_reduce_row[blockIdx.x] * ldy];\n"
      << "    *p = (" << tin << ")(accumulate ? (" << tw << ")*p + s_[0] : s_[0]);\n"
      << "  }\n}\n";
    return z.str();
  }
}

}  // namespace cusadi

namespace cusadi {

// Cooperative kernels: the CTA's warps split one program; lane l of every warp
// works on instance 32 * blockIdx.x + l.  The code is laid out phase by phase:
// one `if (warp == w)` block per warp with work in that phase, then a
// __syncthreads() at function scope, so every thread executes the same barrier
// instructions.  (Per-warp regions with a non-aligned barrier.sync gave wrong
// results at 6-8 warps with ~160 KB of shared slots on GB300, so that layout
// is not used.)  Values read by another warp are staged in shared memory
// (overflow: workspace rows); values a warp needs in a later phase are
// declared at function scope.
CodegenResult generate_coop(const Graph& g, const CodegenOptions& o, const CoopPlan& plan) {
  CodegenResult R;
  Gen G(g, o);
  const int64_t n = (int64_t)g.nodes.size();
  const int W = plan.ways;
  const int NG = o.device_fn ? 1 : std::max(1, o.coop_groups);   // groups of 32 instances per CTA
  G.out_rows.assign(n, {});
  for (size_t r = 0; r < g.out.size(); ++r) G.out_rows[g.out[r]].push_back((int64_t)r);
  // segments: runs of whole phases of at most ~segment_ops ops
  std::vector<int64_t> ops_in_phase(plan.n_phases, 0);
  for (int64_t i = 0; i < n; ++i)
    if (!G.leaf(i)) ops_in_phase[plan.phase[i]]++;
  std::vector<std::pair<int, int>> segs;  // [first phase, last phase + 1)
  {
    int start = 0;
    int64_t acc = 0;
    for (int q = 0; q < plan.n_phases; ++q) {
      if (o.segment_ops > 0 && acc > 0 && acc + ops_in_phase[q] > o.segment_ops) {
        segs.push_back({start, q});
        start = q;
        acc = 0;
      }
      acc += ops_in_phase[q];
    }
    segs.push_back({start, plan.n_phases});
  }
  const int nseg = (int)segs.size();
  std::vector<int> seg_of_phase(plan.n_phases, 0);
  for (int s = 0; s < nseg; ++s)
    for (int q = segs[s].first; q < segs[s].second; ++q) seg_of_phase[q] = s;
  G.seg_of.assign(n, -1);
  G.last_seg.assign(n, -1);
  for (int64_t i = 0; i < n; ++i)
    if (!G.leaf(i)) G.seg_of[i] = seg_of_phase[plan.phase[i]];
  for (int64_t i = 0; i < n; ++i) {
    if (G.leaf(i)) continue;
    const Node& x = g.nodes[i];
    for (int32_t a : {x.a, x.b})
      if (a >= 0 && !G.leaf(a)) G.last_seg[a] = std::max(G.last_seg[a], G.seg_of[i]);
  }
  std::vector<int> slot, gslot;
  int n_gslots = 0;
  const bool sm64 = o.dtype != CUSADI_F32;
  // shared-memory budget for cross-warp values (CUSADI_COOP_SHARED_KB overrides
  // it, so tests can force the workspace overflow path on small programs)
  int budget_kb = o.coop_shared_kb;
  if (const char* e = std::getenv("CUSADI_COOP_SHARED_KB")) budget_kb = std::max(0, std::atoi(e));
  const int max_slots = (int)((budget_kb * 1024) / (32 * (sm64 ? 8 : 4)));
  const int n_slots = assign_coop_slots(g, plan, G.seg_of, max_slots, slot, gslot, n_gslots);
  // workspace rows for values crossing kernels (same interval reuse as generate)
  G.ws_slot.assign(n, -1);
  {
    std::vector<std::vector<int64_t>> release(nseg + 1);
    std::vector<int64_t> free_rows;
    int64_t rows = 0;
    std::vector<std::vector<int64_t>> defs(nseg);
    for (int64_t i = 0; i < n; ++i)
      if (!G.leaf(i)) defs[G.seg_of[i]].push_back(i);
    for (int s = 0; s < nseg; ++s) {
      if (s > 0) {
        for (int64_t r : release[s - 1]) free_rows.push_back(r);
        release[s - 1].clear();
      }
      for (int64_t i : defs[s]) {
        if (G.last_seg[i] <= s) continue;
        int64_t r;
        if (!free_rows.empty()) { r = free_rows.back(); free_rows.pop_back(); }
        else r = rows++;
        G.ws_slot[i] = r;
        release[G.last_seg[i]].push_back(r);
      }
    }
    R.ws_rows = rows;
  }
  // cross-warp values that did not fit in shared memory use rows after those
  const int64_t g_base = R.ws_rows;
  R.ws_rows += n_gslots;
  const char* tin = G.buf_f64() ? "double" : "float";
  const char* tw = G.ws_f64() ? "double" : "float";
  const bool sm_f64 = sm64;  // shared slots hold the widest type in use
  const char* tsm = sm_f64 ? "double" : "float";
  // adjoint outputs: accumulate or overwrite; a reduced (broadcast) row's term
  // goes to its workspace row, summed over the instances by the finishing kernel
  for (uint8_t f : g.out_reduce) R.has_reduce |= (f != 0);
  std::vector<int64_t> reduce_k(g.out_reduce.size(), -1);
  for (size_t r = 0; r < g.out_reduce.size(); ++r)
    if (g.out_reduce[r]) {
      reduce_k[r] = (int64_t)R.reduce_rows.size();
      R.reduce_rows.push_back((int64_t)r);
    }
  auto store_out = [&](std::ostringstream& body, int64_t r, const std::string& v) {
    if (o.debug_checks && !o.device_fn)   // count non-finite results (cusadi_debug_count)
      body << "    if (active && !isfinite((double)(" << v << "))) atomicAdd(&cs_dbg, 1u);\n";
    if (!o.adjoint) {
      body << "    if (active) Y[" << r << "ll * ldy] = (" << tin << ")" << v << ";\n";
      return;
    }
    const std::string plain = std::string("if (active) { ") + tin + "* p_ = &Y[" + std::to_string(r) +
                              "ll * ldy]; *p_ = acc ? *p_ + (" + tin + ")" + v + " : (" + tin + ")" + v + "; }";
    if (!g.out_reduce[r]) {
      body << "    " << plain << "\n";
      return;
    }
    body << "    if (reduce) { if (active) Wp[" << reduce_k[r] << "ll * ldw] = (" << tw << ")" << v
         << "; } else " << plain << "\n";
  };
  // nodes per (segment, warp, phase) in topological order
  for (int s = 0; s < nseg; ++s) {
    std::vector<std::vector<std::vector<int64_t>>> work(W, std::vector<std::vector<int64_t>>(segs[s].second - segs[s].first));
    for (int64_t i = 0; i < n; ++i)
      if (!G.leaf(i) && G.seg_of[i] == s) work[plan.owner[i]][plan.phase[i] - segs[s].first].push_back(i);
    std::ostringstream regions;
    G.calls.clear();
    G.own_f32 = false;
    const int nph_seg = segs[s].second - segs[s].first;
    // phase-major layout: every warp reaches the same __syncthreads() (aligned
    // barrier); a value used by its own warp in a later phase is declared once
    // at function scope, everything else is local to its phase block
    std::vector<int> last_own_phase(n, -1);
    for (int64_t i = 0; i < n; ++i) {
      if (G.leaf(i) || G.seg_of[i] != s) continue;
      const Node& x = g.nodes[i];
      for (int32_t a : {x.a, x.b})
        if (a >= 0 && !G.leaf(a) && G.seg_of[a] == s && plan.owner[a] == plan.owner[i])
          last_own_phase[a] = std::max(last_own_phase[a], plan.phase[i]);
    }
    std::ostringstream decls;
    std::vector<std::ostringstream> phase_code(nph_seg);
    std::vector<std::vector<std::string>> phase_warp(nph_seg, std::vector<std::string>(W));
    for (int w = 0; w < W; ++w) {
      std::ostringstream body;
      std::vector<uint8_t> have(n, 0);
      auto operand = [&](int32_t i, bool want_f64) -> std::string {
        const Node& x = g.nodes[i];
        bool f = G.node_f64(i);
        if (x.op == CONST) return lit(x.k, want_f64);
        // a value this warp loads (input, another warp's value, an earlier
        // kernel's value) gets its own name; in the phase-major layout it is
        // declared at function scope because later phases may use it again
        const bool loaded = x.op == INPUT || G.seg_of[i] != s || plan.owner[i] != w;
        std::string name = "v" + std::to_string(i) + (loaded ? "_" + std::to_string(w) : "");
        if (!have[i]) {
          std::string lhs;
          if (loaded) {
            decls << "  " << G.ty(f) << " " << name << ";\n";
            lhs = "    " + name;
          } else {
            lhs = std::string("    const ") + G.ty(f) + " " + name;
          }
          if (x.op == INPUT) {
            const bool second = o.split >= 0 && x.io >= o.split;   // adjoint: y_bar rows
            const int64_t row = second ? x.io - o.split : x.io;
            body << lhs << " = (" << G.ty(f) << ")"
                 << (second ? (x.bcast ? "X2b[" : "X2[") : (x.bcast ? "Xb[" : "X[")) << row
                 << (second ? "ll * ldx2];\n" : "ll * ldx];\n");
          } else if (G.seg_of[i] != s) {
            body << lhs << " = (" << G.ty(f) << ")W[" << G.ws_slot[i] << "ll * ldw];\n";
          } else if (plan.owner[i] != w) {
            if (slot[i] >= 0)
              body << lhs << " = (" << G.ty(f) << ")cs_x[" << slot[i] << " * 32 + lane];\n";
            else
              body << lhs << " = (" << G.ty(f) << ")W[" << g_base + gslot[i] << "ll * ldw];\n";
          }
          have[i] = 1;
        }
        if (f != want_f64) return std::string("(") + G.ty(want_f64) + ")" + name;
        return name;
      };
      const int nph = nph_seg;
      for (int q = 0; q < nph; ++q) {
        for (int64_t i : work[w][q]) {
          const Node& x = g.nodes[i];
          const bool f = G.node_f64((int32_t)i);
          const char* T = G.ty(f);
          std::string A = x.a >= 0 ? operand(x.a, f) : "";
          std::string B = x.b >= 0 ? operand(x.b, f) : "";
          const bool persists = plan.phase[i] < last_own_phase[i];
          if (persists) {
            decls << "  " << T << " v" << i << ";\n";
            body << "    v" << i << " = " << op_expr(G, x, f, A, B, o) << ";\n";
          } else {
            body << "    const " << T << " v" << i << " = " << op_expr(G, x, f, A, B, o) << ";\n";
          }
          have[i] = 1;
          if (slot[i] >= 0) body << "    cs_x[" << slot[i] << " * 32 + lane] = (" << tsm << ")v" << i << ";\n";
          if (gslot[i] >= 0) body << "    if (active) W[" << g_base + gslot[i] << "ll * ldw] = (" << tw << ")v" << i << ";\n";
          if (G.ws_slot[i] >= 0) body << "    if (active) W[" << G.ws_slot[i] << "ll * ldw] = (" << tw << ")v" << i << ";\n";
          for (int64_t r : G.out_rows[i]) store_out(body, r, "v" + std::to_string(i));
        }
        phase_warp[q][w] = body.str();
        body.str("");
        body.clear();
      }
      if (s == 0 && w == 0) {
        // outputs fed directly by inputs or constants
        for (int64_t i = 0; i < n; ++i) {
          if (!G.leaf(i) || G.out_rows[i].empty()) continue;
          std::string v = operand((int32_t)i, G.node_f64((int32_t)i));
          for (int64_t r : G.out_rows[i]) store_out(body, r, v);
        }
      }
      if (!body.str().empty()) phase_warp[nph - 1][w] += body.str();
    }
    {
      regions << decls.str();
      for (int q = 0; q < nph_seg; ++q) {
        bool first = true;
        for (int w = 0; w < W; ++w) {
          if (phase_warp[q][w].empty()) continue;
          regions << (first ? "  if (warp == " : "  else if (warp == ") << w << ") {\n" << phase_warp[q][w] << "  }\n";
          first = false;
        }
        if (q + 1 < nph_seg) regions << "  __syncthreads();\n";
      }
    }
    std::ostringstream src;
    src << "// Generated cooperative kernel: segment " << s << " of " << nseg << ", " << W
        << " warps per 32 instances, " << (segs[s].second - segs[s].first) << " phases\n";
    if (G.own_f32) src << own_math_source(o.own_math);
    if (o.debug_checks && !o.device_fn) src << "__device__ unsigned int cs_dbg;   // non-finite results\n";
    {
      for (auto& c : G.calls) {
        MathFn m = math_name(c.first);
        const char* t = c.second ? "double" : "float";
        bool bin = op_arity(c.first) == 2;
        src << "static __device__ __noinline__ " << t << " " << call_name(c.first, c.second, false) << "("
            << t << " a" << (bin ? std::string(", ") + t + " b" : "") << ") { return "
            << (c.second ? m.d : m.f) << "(a" << (bin ? ", b" : "") << "); }\n";
      }
    }
    std::string name = o.prefix + "_" + std::to_string(s);
    if (o.device_fn) {
      // one group of 32 instances (first .. first + count - 1) per call, made
      // by every thread of the calling CTA of 32 * W threads (the barriers
      // need all of them); the barrier on entry orders this segment after the
      // previous one's workspace writes and shared-slot reads
      src << "extern \"C\" __device__ void " << name << "(\n"
          << "    const " << tin << "* __restrict__ X, long long ldx, " << tin
          << "* __restrict__ Y, long long ldy, " << tw << "* __restrict__ W, long long ldw,\n"
          << "    long long first, int count, unsigned char* __restrict__ cs_smem) {\n"
          << "  " << tsm << "* __restrict__ cs_x = reinterpret_cast<" << tsm << "*>(cs_smem);\n"
          << "  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;\n"
          << "  const bool active = lane < count;\n"
          << "  const long long i = first + (active ? lane : count - 1);\n"
          << "  const " << tin << "* __restrict__ Xb = X;\n"
          << "  X += i; Y += i; W += i;\n"
          << "  (void)Xb; (void)W; (void)ldw; (void)cs_x;\n"
          << "  __syncthreads();\n"
          << regions.str() << "}\n";
      Segment S;
      S.begin = segs[s].first;
      S.end = segs[s].second;
      S.name = name;
      S.source = src.str();
      R.segs.push_back(std::move(S));
      continue;
    }
    // NG groups of 32 instances per CTA: warp w of every group runs role w % W
    // on group w / W, each group with its own block of shared slots
    src << "extern \"C\" __global__ void " << launch_bounds(32 * W * NG, o.maxrregcount) << " " << name << "(\n"
        << "    const " << tin << "* __restrict__ X, long long ldx, const " << tin
        << "* __restrict__ X2, long long ldx2, " << tin << "* __restrict__ Y, long long ldy,\n    long long N, "
        << tw << "* __restrict__ W, long long ldw, int acc, int reduce, int vec) {\n"
        << "  extern __shared__ __align__(16) unsigned char cs_smem[];\n"
        << "  const int lane = threadIdx.x & 31, warp = (threadIdx.x >> 5) % " << W
        << ", grp = (threadIdx.x >> 5) / " << W << ";\n"
        << "  " << tsm << "* __restrict__ cs_x = reinterpret_cast<" << tsm << "*>(cs_smem) + grp * "
        << std::max(n_slots, 1) * 32 << ";\n"
        << "  const long long i0 = ((long long)blockIdx.x * " << NG << " + grp) * 32 + lane;\n"
        << "  const bool active = i0 < N;\n"
        << "  const long long i = active ? i0 : N - 1;\n"
        << "  const " << tin << "* __restrict__ Xb = X;\n"
        << "  const " << tin << "* __restrict__ X2b = X2;\n";
    if (R.has_reduce) src << "  " << tw << "* __restrict__ Wp = W + " << R.ws_rows << "ll * ldw + i;  // reduced-row terms\n";
    src << "  X += i; X2 += i; Y += i; W += i;\n"
        << "  (void)Xb; (void)X2b; (void)ldx2; (void)W; (void)ldw; (void)acc; (void)reduce; (void)cs_x; (void)vec;\n"
        << regions.str() << "}\n";
    Segment S;
    S.begin = segs[s].first;
    S.end = segs[s].second;
    S.name = name;
    S.source = src.str();
    R.segs.push_back(std::move(S));
  }
  R.coop_ways = W;
  R.coop_groups = NG;
  R.smem_bytes = (int64_t)NG * std::max(n_slots, 1) * 32 * (sm_f64 ? 8 : 4);
  if (R.has_reduce && !o.device_fn) R.segs[0].source += finish_source(R, o.prefix, tin, tw);
  return R;
}

}  // namespace cusadi
