// Internal declarations of libcusadi: IR, SSA graph, passes, code generation.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda.h>

#include "cusadi.h"

namespace cusadi {

// Op codes of the program file (numbering is this project's own; the op set
// follows the atomic operations CusADi §II-A and Listing 1 name).
enum Op : uint16_t {
  INPUT = 0, OUTPUT, CONST, ASSIGN, ADD, SUB, MUL, DIV, NEG, EXP, LOG, POW, SQ, SQRT, SIN,
  COS, TAN, ATAN, ATAN2, TANH, FABS, FMIN, FMAX, FMA_CONST, IF_ELSE_ZERO, LT, LE, EQ, NE,
  NOT, AND, OR, ASIN, ACOS, SINH, COSH, ERF, SIGN, FLOOR, CEIL, FMOD, INV, HYPOT, LOG1P,
  EXPM1, COPYSIGN, N_OPS
};

int op_arity(int op);            // slot operands: 0 (INPUT/CONST/OUTPUT), 1 or 2
bool op_commutative(int op);
bool op_call(int op);            // evaluated through an out-of-line math function
const char* op_name(int op);

struct Arg {
  uint32_t nrow = 0, ncol = 0, nnz = 0, flags = 0;
  std::string name;
  std::vector<uint32_t> rowptr, col;
  int64_t offset = 0;            // first stacked row
};

struct IRInstr {
  uint16_t op, flags;
  uint32_t out, a, b, c;
};

struct IRFile {
  uint32_t n_work = 0;
  std::vector<Arg> in, out;
  std::vector<IRInstr> code;
  std::vector<double> k;
  int64_t nnz_in = 0, nnz_out = 0, n_ops = 0;
};

// Parses and validates; on failure returns false with a message.
bool parse_ir(const uint8_t* p, size_t n, IRFile& f, std::string& err);

// SSA node.  Operands refer to earlier nodes.
struct Node {
  uint16_t op = CONST;
  uint8_t f64 = 0;               // FP64 tag (mixed precision)
  uint8_t bcast = 0;             // INPUT from a broadcast row
  int32_t a = -1, b = -1;
  double k = 0;                  // CONST value, FMA_CONST literal
  int64_t io = 0;                // INPUT: stacked input row
};

struct Graph {
  std::vector<Node> nodes;       // topological order = evaluation order
  std::vector<int32_t> out;      // node of each stacked output row
  std::vector<uint8_t> out_reduce;  // per output row: summed over instances (adjoint)
  std::vector<uint8_t> in_bcast;    // per stacked input row: broadcast
  int64_t nnz_in = 0;
};

Graph build_ssa(const IRFile& f);
// Constant folding, exact identities, CSE, DCE.  Renumbers nodes.
void simplify(Graph& g, int dtype);
// Reorders nodes to lower the number of simultaneously live values.
void schedule(Graph& g);
// Reverse-mode transform: inputs [x (nnz_in rows); y_bar (nnz_out rows)],
// outputs x_bar (nnz_in rows); broadcast x rows are marked out_reduce.
Graph adjoint_graph(const Graph& g);

// last_use[i]: position of the last reader (or output store) of node i, -1 if none.
std::vector<int64_t> last_uses(const Graph& g);
int64_t max_live(const Graph& g);
int64_t count_ops(const Graph& g);
void op_histogram(const Graph& g, std::vector<int64_t>& h, bool f64_only = false);

// --- code generation -------------------------------------------------------
struct Segment {
  int64_t begin = 0, end = 0;    // node positions [begin, end)
  std::string name;
  std::string source;
};

struct CodegenResult {
  std::vector<Segment> segs;
  int64_t ws_rows = 0;           // workspace rows (values carried between segments)
  bool has_reduce = false;
  // reduced rows (adjoint): each instance writes its term to workspace row
  // ws_rows + k (instance-indexed columns); the finish kernel adds each row's
  // terms in a fixed order
  std::vector<int64_t> reduce_rows;
  std::string finish_kernel;
  int coop_ways = 0;             // > 0: cooperative kernels, 32 * coop_ways threads per group
  int coop_groups = 1;           // groups of 32 instances per CTA (cooperative kernels)
  int inst_per_thread = 1;       // consecutive instances per thread (one-thread kernels)
  int64_t smem_bytes = 0;        // dynamic shared memory per CTA (cooperative kernels)
};

struct CodegenOptions {
  int dtype = CUSADI_F64;
  int block = 128;
  int64_t segment_ops = 40000;
  int inline_math = 0;           // 1: inline every math function; 2: inline the short
                                 // ones (exp, expm1, log, log1p), call the rest
  int maxrregcount = 0;          // > 0: registers per thread the launch bounds allow
  int own_math = 0;              // own FP32 sin/cos/exp instead of library calls:
                                 // 1 inlined, 2 out-of-line functions
  int inst_per_thread = 1;       // one-thread kernels: R consecutive instances per thread
  int sync_every = 0;            // one-thread kernels: a CTA barrier every this many ops
  int coop_groups = 1;           // cooperative kernels: groups of 32 instances per CTA
  int spill_values = 0;          // one-thread kernels: > 0 keeps at most this many values
                                 // live in registers, the rest in shared memory / workspace
  int spill_shared_kb = 96;      // shared memory per CTA for those values
  int pair_calls = 0;            // one-thread kernels: > 0 evaluates two calls of the same
                                 // out-of-line math function at once, the second hoisted
                                 // from at most this many ops later
  bool adjoint = false;
  int64_t split = -1;            // input rows >= split come from the second buffer
  bool device_fn = false;        // emit relocatable __device__ functions of one instance
                                 // (cooperative: of one group of 32, called by the whole CTA)
  int coop_shared_kb = 160;      // shared memory for cross-warp values (cooperative)
  bool debug_checks = false;     // count non-finite stored values in the module's cs_dbg
  std::string prefix = "cs_fwd";
};

CodegenResult generate(const Graph& g, const CodegenOptions& o);

// --- within-instance parallelism ----------------------------------------------
struct CoopPlan {
  int ways = 1;                  // warps cooperating on one group of 32 instances
  std::vector<int> owner;        // per node: warp computing it (-1: input/constant)
  std::vector<int> phase;        // per node: barrier-separated phase
  int n_phases = 1;
};
CoopPlan plan_coop(const Graph& g, int ways, double comm_cost);
// Shared-memory slots (at most max_slots; overflow to workspace rows gslot) of
// the values read by another warp of the same kernel (seg_of_node: kernel of
// each node); returns the shared slot count.
int assign_coop_slots(const Graph& g, const CoopPlan& P, const std::vector<int>& seg_of_node,
                      int max_slots, std::vector<int>& slot, std::vector<int>& gslot,
                      int& n_gslots);
// Kernels of W = ways warps per CTA, 32 instances per CTA (forward only).
CodegenResult generate_coop(const Graph& g, const CodegenOptions& o, const CoopPlan& plan);

// --- interpreter stream -------------------------------------------------------
// code = op | f64 << 7 | bcast << 6 ... packed per instruction (see kernels.cu)
struct IOp {
  uint32_t code;   // bits 0..6 op, bit 7 f64 tag, bits 8..31 aux (input row / const / output row)
  uint32_t out;    // destination slot (OUTPUT: unused)
  uint32_t a, b;   // operand slots
};

struct InterpProgram {
  std::vector<IOp> ops;
  std::vector<double> k;
  std::vector<uint8_t> in_bcast;
  int64_t n_slots = 0;             // n_shared + n_global (at least 1)
  int64_t n_shared = 0;            // slots 0 .. n_shared - 1: shared memory
  int64_t n_global = 0;            // slots n_shared ..: rows of the global workspace
  bool has_reduce = false;
  std::vector<int64_t> reduce_rows;   // output rows summed over instances (adjoint)
};

// At most max_shared slots go to shared memory (interp.cpp: linear scan).
bool pack_interp(const Graph& g, InterpProgram& p, std::string& err, int64_t max_shared);
// Shared-memory slots per thread of the interpreter kernel for a budget in KB.
int interp_shared_slots(int dtype, int shared_kb);

// launchers implemented in kernels.cu.  Input rows >= split are read from X2
// (row - split); returns a cudaError_t value.
int launch_interp(const IOp* ops, int64_t n_ops, const double* k, int dtype, const void* X,
                  int64_t ldx, const void* X2, int64_t ldx2, int64_t split, void* Y, int64_t ldy,
                  int64_t N, void* W, int64_t ldw, int64_t n_shared, int acc, int reduce,
                  void* Wr, int64_t ldr, void* stream);
// fixed-order sums of the reduced rows' per-instance terms (row k of Wr, k <
// n_rows) into column 0 of output rows rows[k]
int launch_reduce_finish(int dtype, const void* Wr, int64_t ldr, int64_t N, const int64_t* rows,
                         int64_t n_rows, void* Y, int64_t ldy, int accumulate, void* stream);
// S[r] (+)= sum over the N instances of row r of Y, rows 0..rows-1, in a fixed
// order; dtype CUSADI_F64 sums doubles, otherwise floats.
int launch_sum_rows(int dtype, const void* Y, int64_t ldy, int64_t rows, int64_t N, void* S,
                    int accumulate, void* stream);
// dense copy of one output argument (kernels.cu); returns a cudaError_t value
int launch_densify(int dtype, const void* y, int64_t ldy, int64_t off, const int32_t* map,
                   int64_t n_dense, void* dense, int64_t ldd, int64_t N, int sms, void* stream);

// runtime.cpp: NVRTC compile with the in-memory and on-disk content-hash cache
bool compile_nvrtc(const std::string& src, const std::string& name,
                   const std::vector<std::string>& opts, const char* cache_dir, std::string& cubin,
                   std::string& log);

// Driver-API entry points, fetched through the runtime so that the library
// does not link libcuda (it must load on machines without a GPU driver).
struct Driver {
  CUresult (*moduleLoadData)(CUmodule*, const void*) = nullptr;
  CUresult (*moduleGetFunction)(CUfunction*, CUmodule, const char*) = nullptr;
  CUresult (*moduleUnload)(CUmodule) = nullptr;
  CUresult (*launchKernel)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                           unsigned, CUstream, void**, void**) = nullptr;
  CUresult (*occupancy)(int*, CUfunction, int, size_t) = nullptr;
  CUresult (*funcGetAttribute)(int*, CUfunction_attribute, CUfunction) = nullptr;
  CUresult (*funcSetAttribute)(CUfunction, CUfunction_attribute, int) = nullptr;
  CUresult (*moduleGetGlobal)(CUdeviceptr*, size_t*, CUmodule, const char*) = nullptr;
  bool ok = false;
};
const Driver& driver();

// runtime.cpp: records msg as this thread's last error and returns s
cusadi_status report(cusadi_status s, const std::string& msg);
// runtime.cpp: forward evaluation using `scratch` as the workspace, loading nothing
cusadi_status eval_in_scratch(cusadi_fn fn, const void* in, int64_t ld_in, void* out,
                              int64_t ld_out, int64_t N, void* scratch, size_t scratch_bytes,
                              cusadi_stream stream);

}  // namespace cusadi
