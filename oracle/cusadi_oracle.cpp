// Oracle: plain, slow, sequential CPU interpreter of the straight-line program IR.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
// CPU-baseline leg may load this library.  It shares no code with the CUDA path:
// it has its own parser, its own op semantics and its own reverse sweep.
//
// What it computes (CusADi §III-A): a function is a work vector plus a list of
// instructions (operation id, input slots, output slot) that are evaluated by
// traversing the list in order, one instance at a time.  Each instruction reads
// its operands before it writes its result, so slots can be reused in place
// (Listing 2).  Only the structural non-zeros of the inputs and outputs are
// read and written (§II-A).  Instances are independent; they are split over
// std::threads in contiguous chunks.
//
// Arithmetic is IEEE double with the host libm, built with -ffp-contract=off so
// that every operation rounds once, as the instruction list states.  Modes:
//   0  FP64: every value is a double.
//   1  FP32 emulation: inputs, constants and every result are rounded to float;
//      each operation is computed in double from float operands and rounded
//      once (exact for + - * / sqrt since 53 >= 2*24 + 2).
//   2  mixed emulation: as mode 1, except that instructions tagged FP64 (flag
//      bit 0) take their operands unrounded and keep a double result.
//
// Reverse mode (CusADi §II-A names algorithmic differentiation as the reason
// for building on CasADi): textbook adjoint sweep over a full tape of operand
// values, x_bar = J^T y_bar per instance.
//
// Rounding bound: the first-order forward error bound of straight-line code,
// sum_t |d y_k / d v_t| * eps_t * |v_t| over the instructions t, with eps_t the
// relative error of instruction t (Higham, Accuracy and Stability of Numerical
// Algorithms, 2nd ed., §3.1 and Ch. 3's running error analysis).  It is computed
// with one reverse sweep per output.
//
// Monte Carlo arithmetic (D. S. Parker, "Monte Carlo Arithmetic: exploiting
// randomness in floating-point arithmetic", UCLA CSD-970002, 1997): the program
// is evaluated in FP64 with each instruction's result multiplied by
// (1 + eps_t * xi), xi uniform in [-1, 1), eps_t the same per-instruction
// relative error as in the rounding bound.  The spread of a few such runs around
// the unperturbed value estimates how far another evaluation with rounding
// errors of that size can land, including the nonlinear effects that a
// first-order bound leaves out (a perturbed operand at a stationary point of
// exp(-a^2), for instance).  Only FP32-sized perturbations (u = 2^-24) are
// offered: double carries them with 29 bits to spare, whereas perturbations of
// FP64 size would be lost in double's own rounding (1 + 2^-53 xi rounds to one
// of three values).  xi comes from a counter-based generator: the
// SplitMix64 output function (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014) applied to a key made of the
// seed, the instance and the instruction index.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <thread>
#include <vector>
#include <algorithm>

namespace {

enum OracleOp : int {
  O_INPUT = 0, O_OUTPUT, O_CONST, O_ASSIGN, O_ADD, O_SUB, O_MUL, O_DIV, O_NEG, O_EXP,
  O_LOG, O_POW, O_SQ, O_SQRT, O_SIN, O_COS, O_TAN, O_ATAN, O_ATAN2, O_TANH, O_FABS,
  O_FMIN, O_FMAX, O_FMA_CONST, O_IF_ELSE_ZERO, O_LT, O_LE, O_EQ, O_NE, O_NOT, O_AND,
  O_OR, O_ASIN, O_ACOS, O_SINH, O_COSH, O_ERF, O_SIGN, O_FLOOR, O_CEIL, O_FMOD, O_INV,
  O_HYPOT, O_LOG1P, O_EXPM1, O_COPYSIGN, O_COUNT
};

struct OInstr {
  int op;
  int flags;
  uint32_t out, a, b, c;
};

struct OArg {
  uint32_t nrow, ncol, nnz, flags;
};

struct OProgram {
  uint32_t n_work = 0;
  std::vector<OArg> in, out;
  std::vector<OInstr> code;
  std::vector<double> k;
  std::vector<uint32_t> in_row;     // stacked input nz -> argument broadcast flag
  uint32_t nnz_in = 0, nnz_out = 0;
  std::vector<uint8_t> in_bcast;    // per stacked input nz
};

struct Reader {
  const uint8_t* p;
  size_t n, off = 0;
  bool ok = true;
  uint32_t u32() {
    if (off + 4 > n) { ok = false; return 0; }
    uint32_t v = (uint32_t)p[off] | ((uint32_t)p[off + 1] << 8) | ((uint32_t)p[off + 2] << 16) |
                 ((uint32_t)p[off + 3] << 24);
    off += 4;
    return v;
  }
  uint16_t u16() {
    if (off + 2 > n) { ok = false; return 0; }
    uint16_t v = (uint16_t)(p[off] | (p[off + 1] << 8));
    off += 2;
    return v;
  }
  double f64() {
    if (off + 8 > n) { ok = false; return 0; }
    uint64_t v = 0;
    for (int i = 7; i >= 0; --i) v = (v << 8) | p[off + i];
    off += 8;
    double d;
    std::memcpy(&d, &v, 8);
    return d;
  }
  void skip(size_t m) {
    if (off + m > n) ok = false; else off += m;
  }
};

int arity(int op) {
  switch (op) {
    case O_INPUT: case O_CONST: case O_OUTPUT: return 0;
    case O_ADD: case O_SUB: case O_MUL: case O_DIV: case O_POW: case O_ATAN2: case O_FMIN:
    case O_FMAX: case O_FMA_CONST: case O_IF_ELSE_ZERO: case O_LT: case O_LE: case O_EQ:
    case O_NE: case O_AND: case O_OR: case O_FMOD: case O_HYPOT: case O_COPYSIGN: return 2;
    default: return 1;
  }
}

// Returns 0 on success, a positive code naming the first problem otherwise.
int parse(const uint8_t* buf, size_t n, OProgram& P) {
  Reader r{buf, n};
  if (n < 4 || std::memcmp(buf, "CSDI", 4) != 0) return 1;
  r.skip(4);
  uint32_t ver = r.u32();
  if (ver != 1) return 2;
  P.n_work = r.u32();
  uint32_t n_in = r.u32(), n_out = r.u32(), n_instr = r.u32(), n_const = r.u32();
  r.u32();
  if (!r.ok) return 3;
  for (uint32_t i = 0; i < n_in + n_out; ++i) {
    OArg a;
    a.nrow = r.u32(); a.ncol = r.u32(); a.nnz = r.u32(); a.flags = r.u32();
    uint32_t nl = r.u32();
    r.skip(nl);
    r.skip(4ull * (a.nrow + 1ull));
    r.skip(4ull * a.nnz);
    if (!r.ok) return 4;
    (i < n_in ? P.in : P.out).push_back(a);
  }
  for (auto& a : P.in) {
    for (uint32_t j = 0; j < a.nnz; ++j) P.in_bcast.push_back((a.flags & 1) ? 1 : 0);
    P.nnz_in += a.nnz;
  }
  for (auto& a : P.out) P.nnz_out += a.nnz;
  P.code.resize(n_instr);
  for (uint32_t t = 0; t < n_instr; ++t) {
    OInstr& I = P.code[t];
    I.op = r.u16(); I.flags = r.u16();
    I.out = r.u32(); I.a = r.u32(); I.b = r.u32(); I.c = r.u32();
  }
  P.k.resize(n_const);
  for (uint32_t t = 0; t < n_const; ++t) P.k[t] = r.f64();
  if (!r.ok) return 5;
  // semantic checks the interpreter relies on
  std::vector<int> written(P.nnz_out, 0);
  std::vector<uint8_t> defined(P.n_work, 0);
  for (auto& I : P.code) {
    if (I.op < 0 || I.op >= O_COUNT) return 6;
    int ar = arity(I.op);
    if (I.op == O_OUTPUT) {
      if (I.out >= P.nnz_out || I.a >= P.n_work || !defined[I.a]) return 7;
      written[I.out]++;
      continue;
    }
    if (I.out >= P.n_work) return 8;
    if (I.op == O_INPUT && I.a >= P.nnz_in) return 9;
    if (I.op == O_CONST && I.a >= n_const) return 10;
    if (I.op == O_FMA_CONST && I.c >= n_const) return 10;
    if (I.op != O_INPUT && I.op != O_CONST) {
      if (I.a >= P.n_work || !defined[I.a]) return 11;
      if (ar == 2 && (I.b >= P.n_work || !defined[I.b])) return 11;
    }
    defined[I.out] = 1;
  }
  for (int w : written)
    if (w != 1) return 12;
  return 0;
}

inline double rf(double v) { return (double)(float)v; }

double sgn(double a) { return a > 0 ? 1.0 : (a < 0 ? -1.0 : 0.0); }

double apply(int op, double a, double b, double kc) {
  switch (op) {
    case O_ASSIGN: return a;
    case O_ADD: return a + b;
    case O_SUB: return a - b;
    case O_MUL: return a * b;
    case O_DIV: return a / b;
    case O_NEG: return -a;
    case O_EXP: return std::exp(a);
    case O_LOG: return std::log(a);
    case O_POW: return std::pow(a, b);
    case O_SQ: return a * a;
    case O_SQRT: return std::sqrt(a);
    case O_SIN: return std::sin(a);
    case O_COS: return std::cos(a);
    case O_TAN: return std::tan(a);
    case O_ATAN: return std::atan(a);
    case O_ATAN2: return std::atan2(a, b);
    case O_TANH: return std::tanh(a);
    case O_FABS: return std::fabs(a);
    case O_FMIN: return std::fmin(a, b);
    case O_FMAX: return std::fmax(a, b);
    case O_FMA_CONST: return std::fma(kc, a, b);
    case O_IF_ELSE_ZERO: return a != 0.0 ? b : 0.0;
    case O_LT: return a < b ? 1.0 : 0.0;
    case O_LE: return a <= b ? 1.0 : 0.0;
    case O_EQ: return a == b ? 1.0 : 0.0;
    case O_NE: return a != b ? 1.0 : 0.0;
    case O_NOT: return a == 0.0 ? 1.0 : 0.0;
    case O_AND: return (a != 0.0 && b != 0.0) ? 1.0 : 0.0;
    case O_OR: return (a != 0.0 || b != 0.0) ? 1.0 : 0.0;
    case O_ASIN: return std::asin(a);
    case O_ACOS: return std::acos(a);
    case O_SINH: return std::sinh(a);
    case O_COSH: return std::cosh(a);
    case O_ERF: return std::erf(a);
    case O_SIGN: return sgn(a);
    case O_FLOOR: return std::floor(a);
    case O_CEIL: return std::ceil(a);
    case O_FMOD: return std::fmod(a, b);
    case O_INV: return 1.0 / a;
    case O_HYPOT: return std::hypot(a, b);
    case O_LOG1P: return std::log1p(a);
    case O_EXPM1: return std::expm1(a);
    case O_COPYSIGN: return std::copysign(a, b);
  }
  return NAN;
}

// Evaluate one instance into w (and optionally record a tape of a, b, result).
void run_instance(const OProgram& P, const double* x, int64_t ld_x, int64_t i, double* y,
                  int64_t ld_y, int mode, double* w, double* tape) {
  for (size_t t = 0; t < P.code.size(); ++t) {
    const OInstr& I = P.code[t];
    const bool f32 = (mode == 1) || (mode == 2 && !(I.flags & 1));
    double res, va = 0, vb = 0;
    switch (I.op) {
      case O_INPUT: {
        int64_t col = P.in_bcast[I.a] ? 0 : i;
        res = x[(int64_t)I.a * ld_x + col];
        if (mode != 0) res = rf(res);  // the float buffer holds the rounded input
        break;
      }
      case O_CONST:
        res = P.k[I.a];
        if (f32) res = rf(res);
        break;
      case O_OUTPUT: {
        double v = w[I.a];
        if (mode != 0) v = rf(v);
        if (y) y[(int64_t)I.out * ld_y + i] = v;
        if (tape) { tape[3 * t] = v; tape[3 * t + 1] = 0; tape[3 * t + 2] = v; }
        continue;
      }
      default: {
        va = w[I.a];
        vb = arity(I.op) == 2 ? w[I.b] : 0.0;
        double kc = I.op == O_FMA_CONST ? P.k[I.c] : 0.0;
        if (f32) { va = rf(va); vb = rf(vb); kc = rf(kc); }
        res = apply(I.op, va, vb, kc);
        if (f32) res = rf(res);
      }
    }
    if (tape) { tape[3 * t] = va; tape[3 * t + 1] = vb; tape[3 * t + 2] = res; }
    w[I.out] = res;
  }
}

// Partial derivatives of instruction t's result with respect to operands a, b.
void partials(const OInstr& I, const OProgram& P, double a, double b, double y, double& da,
              double& db) {
  da = 0; db = 0;
  switch (I.op) {
    case O_ASSIGN: da = 1; break;
    case O_ADD: da = 1; db = 1; break;
    case O_SUB: da = 1; db = -1; break;
    case O_MUL: da = b; db = a; break;
    case O_DIV: da = 1.0 / b; db = -a / (b * b); break;
    case O_NEG: da = -1; break;
    case O_EXP: da = y; break;
    case O_LOG: da = 1.0 / a; break;
    case O_POW:
      da = b * std::pow(a, b - 1.0);
      db = (y == 0.0) ? 0.0 : y * std::log(a);
      break;
    case O_SQ: da = 2 * a; break;
    case O_SQRT: da = 0.5 / y; break;
    case O_SIN: da = std::cos(a); break;
    case O_COS: da = -std::sin(a); break;
    case O_TAN: da = 1 + y * y; break;
    case O_ATAN: da = 1.0 / (1 + a * a); break;
    case O_ATAN2: { double r = a * a + b * b; da = b / r; db = -a / r; break; }
    case O_TANH: da = 1 - y * y; break;
    case O_FABS: da = sgn(a); break;
    case O_FMIN: if (a <= b || std::isnan(b)) da = 1; else db = 1; break;
    case O_FMAX: if (a >= b || std::isnan(b)) da = 1; else db = 1; break;
    case O_FMA_CONST: da = P.k[I.c]; db = 1; break;
    case O_IF_ELSE_ZERO: db = (a != 0.0) ? 1.0 : 0.0; break;
    case O_ASIN: da = 1.0 / std::sqrt(1 - a * a); break;
    case O_ACOS: da = -1.0 / std::sqrt(1 - a * a); break;
    case O_SINH: da = std::cosh(a); break;
    case O_COSH: da = std::sinh(a); break;
    case O_ERF: da = 2.0 / std::sqrt(M_PI) * std::exp(-a * a); break;
    case O_INV: da = -y * y; break;
    case O_HYPOT: da = a / y; db = b / y; break;
    case O_LOG1P: da = 1.0 / (1 + a); break;
    case O_EXPM1: da = y + 1; break;
    case O_FMOD: da = 1; db = -std::trunc(a / b); break;
    case O_COPYSIGN: da = (std::signbit(a) == std::signbit(b)) ? 1.0 : -1.0; break;
    default: break;  // comparisons, logic, sign, floor, ceil: zero almost everywhere
  }
}

// Reverse sweep over the tape of one instance.  wb: slot adjoints (zeroed on
// entry).  Either accumulates x_bar (xb != nullptr) or, when eps != nullptr,
// returns sum_t |adjoint of v_t| * eps_t * |v_t|.
double reverse_instance(const OProgram& P, const double* tape, const double* ybar_i,
                        double* wb, double* xb_i, const double* eps) {
  double bound = 0;
  for (size_t tt = P.code.size(); tt-- > 0;) {
    const OInstr& I = P.code[tt];
    if (I.op == O_OUTPUT) { wb[I.a] += ybar_i[I.out]; continue; }
    double g = wb[I.out];
    wb[I.out] = 0;
    if (eps) bound += std::fabs(g) * eps[tt] * std::fabs(tape[3 * tt + 2]);
    if (g == 0.0) continue;
    if (I.op == O_INPUT) { if (xb_i) xb_i[I.a] += g; continue; }
    if (I.op == O_CONST) continue;
    double da, db;
    partials(I, P, tape[3 * tt], tape[3 * tt + 1], tape[3 * tt + 2], da, db);
    if (da != 0.0) wb[I.a] += g * da;
    if (db != 0.0) wb[I.b] += g * db;
  }
  return bound;
}

template <class F>
void parallel_for(int64_t N, int n_threads, F f) {
  if (n_threads <= 0) n_threads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (N < n_threads) n_threads = (int)std::max<int64_t>(1, N);
  if (n_threads == 1) { f(0, N); return; }
  std::vector<std::thread> th;
  int64_t chunk = (N + n_threads - 1) / n_threads;
  for (int t = 0; t < n_threads; ++t) {
    int64_t lo = t * chunk, hi = std::min<int64_t>(N, lo + chunk);
    if (lo >= hi) break;
    th.emplace_back([=, &f] { f(lo, hi); });
  }
  for (auto& x : th) x.join();
}

// Maximum error in ulps of each operation: index 0 for the GPU's FP64 math,
// 1 for its FP32 math (CUDA C Programming Guide, "Mathematical Functions"
// appendix, maximum ulp error tables; correctly rounded operations are 0.5).
double ulp_gpu(int op, bool f32) {
  switch (op) {
    case O_EXP: return f32 ? 2 : 1;
    case O_LOG: return f32 ? 1 : 1;
    case O_POW: return f32 ? 4 : 2;
    case O_SIN: case O_COS: return f32 ? 2 : 2;
    case O_TAN: return f32 ? 4 : 2;
    case O_ATAN: return f32 ? 2 : 2;
    case O_ATAN2: return f32 ? 3 : 2;
    case O_TANH: return f32 ? 2 : 2;
    case O_ASIN: case O_ACOS: return f32 ? 4 : 2;
    case O_SINH: return f32 ? 3 : 2;
    case O_COSH: return f32 ? 2 : 1;
    case O_ERF: return f32 ? 2 : 2;
    case O_HYPOT: return f32 ? 3 : 1;
    case O_LOG1P: return f32 ? 1 : 1;
    case O_EXPM1: return f32 ? 1 : 1;
    default: return 0.5;
  }
}


// Relative error eps_t of each instruction for the rounding bound and for
// Monte Carlo arithmetic.
// kind 0: eps_t bounds |GPU FP64 - oracle FP64| (GPU ulp table + up to 2 ulp for
//         the host libm, u = 2^-53 per correctly rounded op on each side).
// kind 1: eps_t bounds |GPU FP32 - exact| (u = 2^-24, GPU FP32 ulp table,
//         plus the rounding of inputs and constants to float).
std::vector<double> op_eps(const OProgram& P, int kind) {
  const size_t n = P.code.size();
  std::vector<double> eps(n, 0.0);
  for (size_t t = 0; t < n; ++t) {
    const OInstr& I = P.code[t];
    if (kind == 0) {
      const double u = std::ldexp(1.0, -53);
      if (I.op == O_INPUT || I.op == O_CONST || I.op == O_OUTPUT || I.op == O_ASSIGN) eps[t] = 0;
      else if (ulp_gpu(I.op, false) > 0.5) eps[t] = 2 * u * ulp_gpu(I.op, false) + 4 * u;  // host <= 2 ulp
      else eps[t] = 2 * u;  // correctly rounded on both sides
    } else {
      const double u = std::ldexp(1.0, -24);
      if (I.op == O_OUTPUT || I.op == O_ASSIGN) eps[t] = 0;
      else if (I.op == O_INPUT || I.op == O_CONST) eps[t] = u;
      else eps[t] = 2 * u * ulp_gpu(I.op, true);
    }
  }
  return eps;
}

// SplitMix64's output function of a 64-bit key.
inline uint64_t splitmix64_mix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Uniform in [-1, 1) for (seed, instance i, instruction t).
inline double mca_xi(uint64_t seed, int64_t i, size_t t) {
  uint64_t key = splitmix64_mix(seed) ^ (((uint64_t)i << 32) | (uint64_t)(t & 0xffffffffu));
  uint64_t z = splitmix64_mix(key);
  return (double)(z >> 11) * std::ldexp(1.0, -52) - 1.0;
}

}  // namespace

extern "C" {

struct orc_prog { OProgram P; };

int orc_load(const void* ir, size_t nbytes, orc_prog** out) {
  auto* h = new orc_prog;
  int rc = parse((const uint8_t*)ir, nbytes, h->P);
  if (rc) { delete h; *out = nullptr; return rc; }
  *out = h;
  return 0;
}

void orc_free(orc_prog* h) { delete h; }

void orc_info(orc_prog* h, int64_t* nnz_in, int64_t* nnz_out, int64_t* n_instr,
              int64_t* n_work) {
  *nnz_in = h->P.nnz_in; *nnz_out = h->P.nnz_out;
  *n_instr = (int64_t)h->P.code.size(); *n_work = h->P.n_work;
}

// x: [nnz_in x ld_x] doubles (broadcast rows read at column 0); y: [nnz_out x ld_y].
int orc_eval(orc_prog* h, const double* x, int64_t ld_x, double* y, int64_t ld_y, int64_t N,
             int mode, int n_threads) {
  const OProgram& P = h->P;
  if (mode < 0 || mode > 2) return 1;
  parallel_for(N, n_threads, [&](int64_t lo, int64_t hi) {
    std::vector<double> w(std::max<uint32_t>(P.n_work, 1));
    for (int64_t i = lo; i < hi; ++i) run_instance(P, x, ld_x, i, y, ld_y, mode, w.data(), nullptr);
  });
  return 0;
}

// x_bar[k, i] = sum_j y_bar[j, i] * d y_j / d x_k at instance i (FP64).
// Broadcast inputs get per-instance adjoints in their own columns; reduce them
// over instances yourself.
int orc_adjoint(orc_prog* h, const double* x, int64_t ld_x, const double* ybar, int64_t ld_yb,
                double* xbar, int64_t ld_xb, int64_t N, int n_threads) {
  const OProgram& P = h->P;
  parallel_for(N, n_threads, [&](int64_t lo, int64_t hi) {
    std::vector<double> w(std::max<uint32_t>(P.n_work, 1)), wb(w.size());
    std::vector<double> tape(3 * P.code.size() + 1), yb(P.nnz_out), xb(P.nnz_in);
    for (int64_t i = lo; i < hi; ++i) {
      run_instance(P, x, ld_x, i, nullptr, 0, 0, w.data(), tape.data());
      for (uint32_t j = 0; j < P.nnz_out; ++j) yb[j] = ybar[(int64_t)j * ld_yb + i];
      std::fill(wb.begin(), wb.end(), 0.0);
      std::fill(xb.begin(), xb.end(), 0.0);
      reverse_instance(P, tape.data(), yb.data(), wb.data(), xb.data(), nullptr);
      for (uint32_t k = 0; k < P.nnz_in; ++k) xbar[(int64_t)k * ld_xb + i] = xb[k];
    }
  });
  return 0;
}

// Per output k and instance i: B[k, i] = sum_t |d y_k / d v_t| * eps_t * |v_t|,
// eps_t from op_eps (kind 0: FP64 GPU vs oracle; kind 1: FP32 GPU vs exact).
int orc_rounding_bound(orc_prog* h, const double* x, int64_t ld_x, double* B, int64_t ld_b,
                       int64_t N, int kind, int n_threads) {
  const OProgram& P = h->P;
  const size_t n = P.code.size();
  const std::vector<double> eps = op_eps(P, kind);
  parallel_for(N, n_threads, [&](int64_t lo, int64_t hi) {
    std::vector<double> w(std::max<uint32_t>(P.n_work, 1)), wb(w.size());
    std::vector<double> tape(3 * n + 1), yb(P.nnz_out, 0.0);
    for (int64_t i = lo; i < hi; ++i) {
      run_instance(P, x, ld_x, i, nullptr, 0, 0, w.data(), tape.data());
      for (uint32_t k = 0; k < P.nnz_out; ++k) {
        std::fill(wb.begin(), wb.end(), 0.0);
        yb[k] = 1.0;
        B[(int64_t)k * ld_b + i] = reverse_instance(P, tape.data(), yb.data(), wb.data(), nullptr,
                                                    eps.data());
        yb[k] = 0.0;
      }
    }
  });
  return 0;
}

// Monte Carlo arithmetic run `seed` at FP32 sizes: FP64 evaluation in which
// every instruction's result and every stored output is multiplied by
// (1 + eps_t * xi), eps_t from op_eps(kind 1) (u for outputs) and
// xi = mca_xi(seed, i, t).  Only kind 1 is accepted.
int orc_eval_perturbed(orc_prog* h, const double* x, int64_t ld_x, double* y, int64_t ld_y,
                       int64_t N, int kind, uint64_t seed, int n_threads) {
  const OProgram& P = h->P;
  if (kind != 1) return 1;
  const std::vector<double> eps = op_eps(P, kind);
  const double u_out = std::ldexp(1.0, -24);
  parallel_for(N, n_threads, [&](int64_t lo, int64_t hi) {
    std::vector<double> w(std::max<uint32_t>(P.n_work, 1));
    for (int64_t i = lo; i < hi; ++i) {
      for (size_t t = 0; t < P.code.size(); ++t) {
        const OInstr& I = P.code[t];
        double res;
        if (I.op == O_INPUT) {
          res = x[(int64_t)I.a * ld_x + (P.in_bcast[I.a] ? 0 : i)];
        } else if (I.op == O_CONST) {
          res = P.k[I.a];
        } else if (I.op == O_OUTPUT) {
          double v = w[I.a];
          v *= 1.0 + u_out * mca_xi(seed, i, t);
          y[(int64_t)I.out * ld_y + i] = v;
          continue;
        } else {
          double va = w[I.a], vb = arity(I.op) == 2 ? w[I.b] : 0.0;
          res = apply(I.op, va, vb, I.op == O_FMA_CONST ? P.k[I.c] : 0.0);
        }
        if (eps[t] > 0) res *= 1.0 + eps[t] * mca_xi(seed, i, t);
        w[I.out] = res;
      }
    }
  });
  return 0;
}

}  // extern "C"
