// Program file reader and validator (the work-vector + instruction-list form
// of CusADi §III-A, with sparse argument patterns as in §II-A).
#include <cstring>

#include "internal.h"

namespace cusadi {

int op_arity(int op) {
  switch (op) {
    case INPUT: case CONST: case OUTPUT: return 0;
    case ADD: case SUB: case MUL: case DIV: case POW: case ATAN2: case FMIN: case FMAX:
    case FMA_CONST: case IF_ELSE_ZERO: case LT: case LE: case EQ: case NE: case AND: case OR:
    case FMOD: case HYPOT: case COPYSIGN:
      return 2;
    default:
      return 1;
  }
}

bool op_commutative(int op) {
  switch (op) {
    case ADD: case MUL: case FMIN: case FMAX: case EQ: case NE: case AND: case OR: case HYPOT:
      return true;
    default:
      return false;
  }
}

bool op_call(int op) {
  switch (op) {
    case EXP: case LOG: case POW: case SIN: case COS: case TAN: case ATAN: case ATAN2:
    case TANH: case ASIN: case ACOS: case SINH: case COSH: case ERF: case FMOD: case HYPOT:
    case LOG1P: case EXPM1:
      return true;
    default:
      return false;
  }
}

const char* op_name(int op) {
  static const char* names[] = {
      "INPUT", "OUTPUT", "CONST", "ASSIGN", "ADD", "SUB", "MUL", "DIV", "NEG", "EXP", "LOG",
      "POW", "SQ", "SQRT", "SIN", "COS", "TAN", "ATAN", "ATAN2", "TANH", "FABS", "FMIN",
      "FMAX", "FMA_CONST", "IF_ELSE_ZERO", "LT", "LE", "EQ", "NE", "NOT", "AND", "OR", "ASIN",
      "ACOS", "SINH", "COSH", "ERF", "SIGN", "FLOOR", "CEIL", "FMOD", "INV", "HYPOT", "LOG1P",
      "EXPM1", "COPYSIGN"};
  return (op >= 0 && op < N_OPS) ? names[op] : "?";
}

namespace {
struct In {
  const uint8_t* p;
  size_t n, off;
  bool ok;
  bool need(size_t m) {
    if (!ok || m > n - off) ok = false;
    return ok;
  }
  uint32_t u32() {
    if (!need(4)) return 0;
    uint32_t v;
    std::memcpy(&v, p + off, 4);  // little-endian hosts only (x86_64, aarch64)
    off += 4;
    return v;
  }
  uint16_t u16() {
    if (!need(2)) return 0;
    uint16_t v;
    std::memcpy(&v, p + off, 2);
    off += 2;
    return v;
  }
  double f64() {
    if (!need(8)) return 0;
    double v;
    std::memcpy(&v, p + off, 8);
    off += 8;
    return v;
  }
};
}  // namespace

bool parse_ir(const uint8_t* p, size_t n, IRFile& f, std::string& err) {
  In r{p, n, 0, true};
  if (n < 32 || std::memcmp(p, "CSDI", 4) != 0) { err = "bad magic or truncated header"; return false; }
  r.off = 4;
  uint32_t ver = r.u32();
  if (ver != 1) { err = "unsupported IR version " + std::to_string(ver); return false; }
  f.n_work = r.u32();
  uint32_t n_in = r.u32(), n_out = r.u32(), n_instr = r.u32(), n_const = r.u32();
  r.u32();
  if ((uint64_t)n_in + n_out > (1u << 20)) { err = "too many arguments"; return false; }
  for (uint32_t j = 0; j < n_in + n_out; ++j) {
    Arg a;
    a.nrow = r.u32(); a.ncol = r.u32(); a.nnz = r.u32(); a.flags = r.u32();
    uint32_t nl = r.u32();
    if (!r.need(nl)) break;
    a.name.assign((const char*)p + r.off, nl);
    r.off += nl;
    if (!r.need(4ull * (a.nrow + 1ull) + 4ull * a.nnz)) break;
    a.rowptr.resize(a.nrow + 1);
    for (auto& v : a.rowptr) v = r.u32();
    a.col.resize(a.nnz);
    for (auto& v : a.col) v = r.u32();
    // CSR consistency
    if (a.rowptr[0] != 0 || a.rowptr[a.nrow] != a.nnz) { err = "argument " + std::to_string(j) + ": bad row pointers"; return false; }
    for (uint32_t i = 0; i < a.nrow; ++i) {
      if (a.rowptr[i] > a.rowptr[i + 1]) { err = "argument " + std::to_string(j) + ": row pointers decrease"; return false; }
      for (uint32_t q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q) {
        if (a.col[q] >= a.ncol) { err = "argument " + std::to_string(j) + ": column out of range"; return false; }
        if (q > a.rowptr[i] && a.col[q] <= a.col[q - 1]) { err = "argument " + std::to_string(j) + ": columns not strictly increasing"; return false; }
      }
    }
    if (j >= n_in && (a.flags & 1)) { err = "outputs cannot be broadcast"; return false; }
    if (j < n_in) { a.offset = f.nnz_in; f.nnz_in += a.nnz; f.in.push_back(std::move(a)); }
    else { a.offset = f.nnz_out; f.nnz_out += a.nnz; f.out.push_back(std::move(a)); }
  }
  if (!r.ok) { err = "truncated argument table"; return false; }
  if (!r.need(20ull * n_instr + 8ull * n_const)) { err = "truncated instruction list"; return false; }
  f.code.resize(n_instr);
  for (auto& I : f.code) {
    I.op = r.u16(); I.flags = r.u16();
    I.out = r.u32(); I.a = r.u32(); I.b = r.u32(); I.c = r.u32();
  }
  f.k.resize(n_const);
  for (auto& v : f.k) v = r.f64();
  if (r.off != n) { err = "trailing bytes after the constant pool"; return false; }

  // semantics: operands defined before use, indices in range, outputs written once
  std::vector<uint8_t> defined(f.n_work, 0);
  std::vector<uint32_t> written(f.nnz_out, 0);
  for (size_t t = 0; t < f.code.size(); ++t) {
    const IRInstr& I = f.code[t];
    auto bad = [&](const char* what) {
      err = "instruction " + std::to_string(t) + " (" + op_name(I.op) + "): " + what;
      return false;
    };
    if (I.op >= N_OPS) return bad("unknown op code");
    if (I.op == OUTPUT) {
      if (I.out >= f.nnz_out) return bad("output row out of range");
      if (I.a >= f.n_work || !defined[I.a]) return bad("reads an undefined slot");
      written[I.out]++;
      continue;
    }
    if (I.out >= f.n_work) return bad("destination slot out of range");
    if (I.op == INPUT) {
      if (I.a >= f.nnz_in) return bad("input row out of range");
    } else if (I.op == CONST) {
      if (I.a >= n_const) return bad("constant index out of range");
    } else {
      if (I.a >= f.n_work || !defined[I.a]) return bad("reads an undefined slot");
      if (op_arity(I.op) == 2 && (I.b >= f.n_work || !defined[I.b])) return bad("reads an undefined slot");
      if (I.op == FMA_CONST && I.c >= n_const) return bad("constant index out of range");
      if (I.op != ASSIGN) f.n_ops++;
    }
    defined[I.out] = 1;
  }
  for (size_t r2 = 0; r2 < written.size(); ++r2)
    if (written[r2] != 1) { err = "output row " + std::to_string(r2) + " written " + std::to_string(written[r2]) + " times"; return false; }
  return true;
}

}  // namespace cusadi
