/*
 * cusadi.h -- C ABI of the batched straight-line-program engine (libcusadi.so).
 *
 * The engine evaluates ONE closed-form symbolic function -- a work vector plus
 * an ordered list of scalar instructions (CusADi §III-A: each instruction has
 * an operation id, input slot(s) and an output slot, and the function is
 * evaluated by traversing the list in order) -- across N independent
 * instances on the GPU.  Only structural non-zeros of the sparse inputs and
 * outputs are read and written (§II-A).  Data stays on the GPU: every pointer
 * passed to the evaluation calls is a device pointer (§III intro: inputs and
 * outputs are stored only on the GPU), except the host buffers of
 * cusadi_eval_host, which copies them in and out itself.
 *
 * Layout of every batched buffer: instance-fastest ("SoA").  Row k of
 * instance i lives at  buf[k * ld + i]  with ld >= N (elements, not bytes).
 * The rows of a function's input buffer are the non-zeros of all its input
 * arguments stacked in argument order (cusadi_arg_info gives each argument's
 * first row); likewise for outputs.  An input argument flagged BROADCAST holds
 * one value per non-zero shared by every instance: only column 0 of its rows
 * is read.
 *
 * Element type of the buffers: double for CUSADI_F64, float for CUSADI_F32
 * and CUSADI_MIXED.
 *
 * Errors: every call returns a cusadi_status.  Argument errors are detected on
 * the host before anything is launched; cusadi_last_error() then returns a
 * message for the calling thread.  Evaluation calls are asynchronous on the
 * given stream.  The first call of a function on a device loads its kernels
 * (allocates, synchronises); after that they neither synchronise the host nor
 * allocate device memory.
 *
 * Threading: a cusadi_fn is immutable after cusadi_load and may be used from
 * several host threads and streams at once, provided the workspaces differ.
 */
#ifndef CUSADI_H
#define CUSADI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CUSADI_ABI_VERSION 1

typedef struct cusadi_fn_s* cusadi_fn;        /* one loaded function (library-owned) */
typedef struct cusadi_batch_s* cusadi_batch;  /* several functions, one launch */
typedef void* cusadi_stream;                  /* a cudaStream_t / CUstream (NULL = legacy) */

typedef enum {
  CUSADI_OK = 0,
  CUSADI_E_INVALID_ARG = 1,  /* a pointer, size, stride or option is unusable */
  CUSADI_E_INVALID_IR = 2,   /* the program file is malformed or inconsistent */
  CUSADI_E_COMPILE = 3,      /* NVRTC rejected the generated source */
  CUSADI_E_CUDA = 4,         /* a CUDA runtime/driver call failed */
  CUSADI_E_OOM = 5,          /* host allocation failed */
  CUSADI_E_TIMEOUT = 6,      /* a bounded wait ran out */
  CUSADI_E_UNSUPPORTED = 7   /* valid request this build does not implement */
} cusadi_status;

typedef enum { CUSADI_F64 = 0, CUSADI_F32 = 1, CUSADI_MIXED = 2 } cusadi_dtype;

/* Evaluation path.  COMPILED: generated straight-line CUDA kernels (one
 * instance per thread, values in registers).  INTERP: one precompiled kernel
 * that walks a packed instruction stream (no compile time; for programs too
 * large to compile).  AUTO picks COMPILED up to compile_limit_ops, and the
 * interpreter when the program is larger or NVRTC fails on it. */
typedef enum { CUSADI_PATH_AUTO = 0, CUSADI_PATH_COMPILED = 1, CUSADI_PATH_INTERP = 2 } cusadi_path;

typedef struct {
  int32_t dtype;              /* cusadi_dtype                                     (F64) */
  int32_t path;               /* cusadi_path                                      (AUTO) */
  int64_t compile_limit_ops;  /* AUTO compiles programs with at most this many ops (300000) */
  int64_t segment_ops;        /* compiled programs are split into kernels of at most this
                                 many ops, compiled in parallel                  (40000) */
  int32_t block;              /* threads per block of compiled kernels, multiple of 32 (128) */
  int32_t maxrregcount;       /* register cap for compiled kernels (enforced through their
                                 launch bounds: at least 65536 / (CTA threads * cap)
                                 resident CTAs per SM), 0 = compiler's choice */
  int32_t fmad;               /* 1: let the compiler contract a*b+c into fma     (1) */
  int32_t compile_threads;    /* parallel NVRTC compiles, 0 = all host cores */
  int32_t schedule;           /* 1: reorder ops to lower register pressure       (1) */
  int32_t inline_math;        /* 1: inline every math function (slow compile); 2: inline the
                                 short ones (exp, expm1, log, log1p) and call the rest;
                                 0: every transcendental is an out-of-line call    (0) */
  int32_t adjoint;            /* 1: build the adjoint kernels at load; 0: at the first call
                                 that needs them (cusadi_adjoint and friends)   (0) */
  int32_t ways;               /* 2..16: within-instance parallelism on the compiled path
                                 (forward and adjoint kernels): `ways` warps split each
                                 program across a group of 32 instances (small batches,
                                 few-instance long programs; at large batches it can also
                                 win: time it); 0: one instance per thread          (0) */
  int32_t own_math;           /* FP32 sin/cos/exp: 0 the library's (out-of-line calls),
                                 1 the engine's own (<= 2 ulp) inlined, 2 the engine's
                                 own as out-of-line functions                      (0) */
  int32_t debug_checks;       /* 1: compiled kernels count every non-finite value they
                                 store (NaN, +-inf) in a device counter that
                                 cusadi_debug_count reads; 0: no checks            (0) */
  int32_t inst_per_thread;    /* 1, 2 or 4: consecutive instances evaluated by each thread
                                 of the one-thread-per-instance kernels (ways = 0), op by
                                 op in turn (more independent work per thread, more
                                 registers); their inputs and outputs move as one
                                 float2/float4/double2 access when the buffers allow it
                                 (16-byte aligned base, ld a multiple of it)         (1) */
  int32_t coop_groups;        /* 1..8: groups of 32 instances per CTA of the cooperative
                                 kernels (ways > 1): 32 * ways * coop_groups threads
                                 per CTA; warps of one role in one CTA run the same
                                 code together                                      (1) */
  int32_t sync_every;         /* one-thread-per-instance kernels: a CTA-wide barrier
                                 after every this many ops, so the CTA's warps stay in
                                 the same stretch of a long kernel's code (instruction
                                 cache reuse); 0: no barriers                       (0) */
  int32_t interp_shared_kb;   /* interpreter path: shared memory per 128-thread CTA for the
                                 work slots, in KB (0..200); the slots of the values that
                                 do not fit, chosen by linear scan as the ones read
                                 last, live in the workspace; more shared memory
                                 means fewer resident CTAs, which costs more than the
                                 slots gain beyond ~48 KB on GB300                 (48) */
  int32_t spill_values;       /* one-thread-per-instance kernels (ways = 0, inst_per_thread
                                 = 1): > 0 keeps at most this many values live in
                                 registers; linear scan over their live ranges moves the
                                 value read last out of the registers for its whole life,
                                 to a shared-memory slot, a workspace row beyond those,
                                 or (inputs, carried values) a re-read of its buffer at
                                 each use.  0: the compiler allocates registers    (0) */
  int32_t spill_shared_kb;    /* shared memory per CTA for those values, KB (0..200) (96) */
  int32_t pair_calls;         /* one-thread-per-instance kernels: > 0 issues an out-of-line
                                 unary math call (sin, cos, exp, ...) together with a later
                                 call of the same function, at most this many ops ahead,
                                 whose argument is already computed: one call of a
                                 two-argument version evaluating both.  0: one call per
                                 op                                                 (0) */
  const char* cache_dir;      /* directory for compiled kernels, NULL = in-memory only */
} cusadi_options;

typedef struct {
  int32_t n_in, n_out;        /* argument counts */
  int64_t nnz_in, nnz_out;    /* stacked non-zero rows of the input / output buffers */
  int64_t n_instr;            /* instructions in the program file */
  int64_t n_work;             /* work-vector length in the program file */
  int64_t n_ops_ir;           /* arithmetic instructions in the program file */
  int64_t n_ops;              /* arithmetic ops evaluated per instance after the passes */
  int64_t n_slots;            /* values live at once after scheduling (work slots) */
  int32_t path;               /* CUSADI_PATH_COMPILED or CUSADI_PATH_INTERP */
  int32_t n_segments;         /* kernels per evaluation on the compiled path */
  int32_t dtype;              /* cusadi_dtype */
  int32_t n_bcast_in;         /* input rows flagged broadcast */
  double compile_seconds;     /* wall time spent generating and compiling at load */
} cusadi_fn_info;

typedef struct {
  uint32_t nrow, ncol, nnz;   /* shape and non-zero count of the sparse argument */
  uint32_t flags;             /* bit 0: broadcast (inputs only) */
  int64_t row_offset;         /* first row of this argument in the stacked buffer */
  const uint32_t* rowptr;     /* CSR row pointers [nrow + 1], owned by the function */
  const uint32_t* col;        /* CSR column indices [nnz], owned by the function */
  const char* name;           /* owned by the function */
} cusadi_arg;

/* Adjoint flags. */
#define CUSADI_ADJ_ACCUMULATE 1u        /* add into in_bar instead of overwriting it */
#define CUSADI_ADJ_REDUCE_BROADCAST 2u  /* sum broadcast inputs' adjoints over instances
                                           into column 0 of their rows */
#define CUSADI_ADJ_ACCUMULATE_BROADCAST 4u  /* with REDUCE_BROADCAST: add the sums into column 0
                                               (other rows are still overwritten) */

/* Fills *opt with the defaults quoted above. */
void cusadi_default_options(cusadi_options* opt);

/* Parses and validates a program (the binary IR of §III-A), runs the passes
 * (SSA renaming, constant folding, common-subexpression and dead-code
 * elimination, scheduling for register pressure) and prepares the chosen
 * path: on the compiled path it generates sm_103a CUDA source and compiles it
 * with NVRTC (cached by content hash); on the interpreter path it packs the
 * instruction stream.  Device modules are loaded lazily, on the first
 * evaluation on each device.  `ir` is copied; the caller keeps it.
 * opt may be NULL (defaults).  Errors: INVALID_ARG, INVALID_IR, COMPILE, OOM. */
cusadi_status cusadi_load(const void* ir, size_t nbytes, const cusadi_options* opt,
                          cusadi_fn* out);

/* Releases a function and its device modules (call with no evaluation of it
 * in flight). */
void cusadi_free(cusadi_fn fn);

/* Sizes of a loaded function: its argument counts and stacked non-zeros, the
 * work-vector length and instruction count of the program file (§III-A: a
 * function is a work vector plus n_instructions instructions), and what the
 * passes and the chosen path made of it.  out is written by the library.
 * Errors: INVALID_ARG for a NULL fn or out. */
cusadi_status cusadi_info(cusadi_fn fn, cusadi_fn_info* out);

/* Description of input (is_output = 0) or output argument `index`: shape,
 * flags, first row in the stacked buffer and the argument's sparsity pattern
 * (§II-A: CasADi functions compute only the structural non-zeros of sparse
 * matrices; here the pattern is stored as CSR).  The pointers in *out belong to
 * the function and live as long as it does.  Errors: INVALID_ARG for a NULL fn
 * or out, or an index out of range. */
cusadi_status cusadi_arg_info(cusadi_fn fn, int is_output, int index, cusadi_arg* out);

/* counts[op] = number of ops with that IR op code evaluated per instance, for
 * op < n: the instruction count by which §IV sizes its benchmark functions,
 * split by operation so that a roofline can weight each op by its cost.
 * which: 0 forward kernels, 1 adjoint kernels, 2 / 3 the same but only ops
 * tagged FP64 (those a MIXED function evaluates in double).  counts (n
 * entries) is owned by the caller.  Errors: INVALID_ARG for a NULL fn or
 * counts, n < 0 or which outside 0..3; building the adjoint (which = 1, 3) can
 * also return COMPILE. */
cusadi_status cusadi_op_counts(cusadi_fn fn, int which, int64_t* counts, int n);

/* Bytes of device workspace one evaluation of N instances needs.  CusADi keeps
 * the whole work vector of every instance in global memory (§III-A, Listing
 * 2); here values live in registers and only those carried between the
 * kernels of a long program get workspace rows ([rows x round_up(N, 32)]),
 * plus, for the adjoint, one row of per-instance terms for every broadcast
 * input (0 when neither applies).  The caller allocates it, 256-byte aligned,
 * and owns it.  Returns 0 for a NULL fn, N <= 0, or an adjoint that fails to
 * build. */
size_t cusadi_workspace_bytes(cusadi_fn fn, int64_t N, int adjoint);

/* y = f(x) for N instances: every instance runs the function's instructions
 * in order (§III-A; Listing 2 evaluates one instance per GPU thread, here
 * one thread or, with ways > 1, one group of warps per 32 instances) and
 * writes only the non-zeros of its outputs.  in: [nnz_in x ld_in], out: [nnz_out x ld_out]
 * device buffers of the dtype's element type; ld_in, ld_out >= N (an input
 * buffer whose rows are all broadcast may use ld_in >= 1).  workspace: at least
 * cusadi_workspace_bytes(fn, N, 0) bytes, or NULL when that is 0.  N = 0 is a
 * no-op.  The first call on a device loads the device module (not capturable
 * in a CUDA graph); later calls only launch kernels on `stream`.  Calls that
 * may overlap on the GPU (different streams) need workspaces of their own:
 * the kernels write the workspace. */
cusadi_status cusadi_eval(cusadi_fn fn, const void* in, int64_t ld_in, void* out,
                          int64_t ld_out, int64_t N, void* workspace, cusadi_stream stream);

/* Reverse mode: in_bar = J(x)^T out_bar per instance, J = d out / d in
 * (§II-A: CasADi expressions are differentiable by algorithmic
 * differentiation; here the reverse sweep is itself a straight-line program,
 * generated at load and evaluated like the forward one).
 * out_bar: [nnz_out x ld_ob]; in_bar: [nnz_in x ld_ib].  With
 * CUSADI_ADJ_REDUCE_BROADCAST, broadcast input rows receive the sum over
 * instances in column 0: each instance writes its term to the workspace and
 * a second kernel adds each row's terms in a fixed order, so the result has
 * the same bits on every run (compiled and interpreter paths alike).  Without
 * the flag they receive per-instance values.
 * Without CUSADI_ADJ_ACCUMULATE the written entries are overwritten, except the
 * reduced rows under CUSADI_ADJ_ACCUMULATE_BROADCAST (gradient accumulation of
 * a shared parameter over many calls, e.g. the steps of a rollout).
 * workspace: cusadi_workspace_bytes(fn, N, 1) bytes. */
cusadi_status cusadi_adjoint(cusadi_fn fn, const void* in, int64_t ld_in, const void* out_bar,
                             int64_t ld_ob, void* in_bar, int64_t ld_ib, int64_t N,
                             uint32_t flags, void* workspace, cusadi_stream stream);

/* cusadi_adjoint (reverse mode, §II-A) with the sums over instances of the
 * broadcast inputs' adjoints (the gradient of a parameter shared by every
 * instance, such as the feedback gain of a differentiable rollout) written to
 * a vector of their own instead of column 0 of in_bar: shared_bar[row] for every
 * broadcast input row `row` (shared_bar has nnz_in entries of the dtype's
 * element type; other entries are left alone).  Broadcast rows of in_bar are
 * not written.  The reduction is always on (passing
 * CUSADI_ADJ_REDUCE_BROADCAST is an INVALID_ARG); with
 * CUSADI_ADJ_ACCUMULATE_BROADCAST the sums are added to shared_bar, so one
 * vector collects a shared parameter's gradient over many calls whose in_bar
 * buffers differ (the steps of a rollout ping-ponging two buffers).  Same
 * fixed summation order, hence the same bits on every run, as cusadi_adjoint.
 * Other arguments, ownership and errors as for cusadi_adjoint; INVALID_ARG
 * also for a NULL shared_bar. */
cusadi_status cusadi_adjoint_shared(cusadi_fn fn, const void* in, int64_t ld_in, const void* out_bar,
                                    int64_t ld_ob, void* in_bar, int64_t ld_ib, void* shared_bar,
                                    int64_t N, uint32_t flags, void* workspace,
                                    cusadi_stream stream);

/* sums[r] = sum over the N instances of row r of y, for r < rows (with
 * accumulate != 0: sums[r] += that sum): a batched objective such as the
 * total loss of a rollout over its environments.  y: [rows x ld_y] device
 * buffer, ld_y >= N; sums: `rows` device elements; double for CUSADI_F64,
 * float for CUSADI_F32 and CUSADI_MIXED; both owned by the caller.  One
 * kernel on `stream`, summing each row in a fixed order (per-thread strided
 * sums, then a tree), so the result has the same bits on every run.  N = 0
 * writes zeros (or leaves sums unchanged when accumulating).  The paper has
 * no counterpart: it keeps such reductions in PyTorch (§III-B).  Errors:
 * INVALID_ARG for an unknown dtype, rows outside 0..65535, N < 0, NULL
 * buffers or ld_y < N, checked before any CUDA call; CUDA if the launch
 * fails. */
cusadi_status cusadi_sum_instances(int32_t dtype, const void* y, int64_t ld_y, int64_t rows,
                                   int64_t N, void* sums, int32_t accumulate, cusadi_stream stream);

/* Size of the static scratch region behind cusadi_eval_noalloc, in bytes. */
#define CUSADI_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)

/* cusadi_eval for callers that cannot allocate device memory.  The paper has
 * no counterpart.  Some callers are not allowed to allocate once they run: a
 * real-time control loop calling the MPC every tick under a no-allocation rule
 * (allocation can block for an unbounded time), or a plugin running inside a
 * host application that owns all device memory and gives the plugin only its
 * input and output buffers.
 *
 * Same arguments and results as cusadi_eval minus the workspace: the
 * workspace is a file-scope device array of CUSADI_NOALLOC_SCRATCH_BYTES that
 * every GPU which loads this library keeps until the process exits.  The call
 * allocates nothing: it calls no cudaMalloc/cudaFree and no allocating library
 * routine.  Set-up: the first call on a device looks up the array's device
 * address there (cudaGetSymbolAddress, once per device), so make that first
 * call before any stream capture; the function's kernels must already be
 * loaded on the device, which any earlier cusadi_eval of it does (otherwise
 * INVALID_ARG).  Evaluations whose workspace exceeds the scratch size
 * (cusadi_workspace_bytes(fn, N, 0) > CUSADI_NOALLOC_SCRATCH_BYTES) are
 * rejected with INVALID_ARG; evaluate fewer instances per call.  Every call
 * shares the one array and it keeps the last call's contents; nothing in it
 * needs to start at zero (each value is written before it is read), but calls
 * that overlap on the GPU (different streams, or several threads) race on it. */
cusadi_status cusadi_eval_noalloc(cusadi_fn fn, const void* in, int64_t ld_in, void* out,
                                  int64_t ld_out, int64_t N, cusadi_stream stream);

/* y = f(x) from and to host memory: the evaluation with data transfer that
 * §IV times against the CPU (Fig. 3 reports speedups with and without it).
 * The instance range is cut into chunks; chunk c's inputs are copied in,
 * evaluated and copied out on streams of the library's own (one copy-in, one
 * copy-out and one compute stream per chunk, ordered by events), so the
 * copies of one chunk overlap the kernels of the others.
 *
 * in_host: [nnz_in x ld_in] and out_host: [nnz_out x ld_out] host buffers of
 * the dtype's element type, instance-fastest as for cusadi_eval (ld_in >= N,
 * or >= 1 when every input row is broadcast; ld_out >= N).  Page-locked host
 * memory (cudaHostAlloc / cudaHostRegister) is needed for the copies to run
 * asynchronously and overlap; pageable memory gives the same results, slower.
 * dev_in: [nnz_in x N] and dev_out: [nnz_out x N] device staging buffers with
 * leading dimension exactly N, owned by the caller; workspace as for
 * cusadi_eval(N) (each chunk uses its own columns of it).  chunks: the number
 * of pieces (0 = two from N = 16,384 on, else one); each piece is a multiple
 * of 32 instances (128 on the interpreter path).
 *
 * Asynchronous like cusadi_eval: the copies and kernels start after the work
 * already queued on `stream`, and `stream` waits for all of them, so a
 * synchronize (or an event) on `stream` makes out_host valid; the host
 * buffers must stay valid until then.  Calls on one function are enqueued one
 * at a time (a mutex) and share its streams.  Errors: INVALID_ARG for
 * NULL buffers, short leading dimensions, a missing workspace or chunks < 0,
 * checked before any CUDA call; CUSADI_E_CUDA when a copy or launch fails. */
cusadi_status cusadi_eval_host(cusadi_fn fn, const void* in_host, int64_t ld_in, void* out_host,
                               int64_t ld_out, int64_t N, void* dev_in, void* dev_out,
                               void* workspace, int32_t chunks, cusadi_stream stream);

/* Debug: the number of non-finite values (NaN, +-inf) the function's kernels
 * stored on the current device since the previous call, and the counter reset
 * to 0.  Needs a function loaded with debug_checks = 1 on the compiled path
 * (INVALID_ARG otherwise, checked before any CUDA call; UNSUPPORTED on the
 * interpreter path).  Synchronises the device (a debugging call, not for the
 * hot loop).  Kernels count values that they write to outputs (and, for an
 * adjoint, to the reduction workspace); a function never evaluated on the
 * device reads 0. */
cusadi_status cusadi_debug_count(cusadi_fn fn, uint64_t* count);

/* Output argument `arg` as a dense matrix per instance.  The engine reads and
 * writes only structural non-zeros (§II-A: sparse CasADi matrices, Listing 2
 * stores nnz entries); this scatters one argument of an evaluation result for
 * a caller that wants the full nrow x ncol block (a PyTorch tensor, §III-B).
 * y: [nnz_out x ld_y] as cusadi_eval wrote it; dense: [nrow*ncol x ld_d],
 * entry (r, c) of instance i at dense[(r*ncol + c)*ld_d + i], structural zeros
 * written as 0; both device buffers of the dtype's element type, owned by the
 * caller; ld_y, ld_d >= N.  The first call for an argument on a device
 * uploads an nrow*ncol index map (it allocates and synchronises: make it
 * before any stream capture); later calls launch one kernel on `stream`.
 * Errors: INVALID_ARG for a bad index, NULL buffers or short leading
 * dimensions, checked before any CUDA call. */
cusadi_status cusadi_densify(cusadi_fn fn, int arg, const void* y, int64_t ld_y, void* dense,
                             int64_t ld_d, int64_t N, cusadi_stream stream);

/* ---- batched launch of several programs ------------------------------------
 * CusADi puts all operations of a function into one kernel to save launch
 * overhead (§III-A, end).  A batch carries that over to several functions of
 * uneven size, each over its own fixed instance count: every program is
 * compiled as relocatable one-instance device functions and linked (nvJitLink)
 * with a persistent scheduler kernel.  Its CTAs repeatedly take the next tile
 * (one program, `block` consecutive instances) from an atomic ticket; tiles are
 * ordered longest program first, so the few-instance long programs start at
 * once and the short ones fill the GPU around them.  The launch (ticket reset +
 * kernel) is captured once per device in a CUDA graph and replayed.  The same
 * link also has one plain kernel per program (CUSADI_BATCH_PLAIN), so the two
 * modes run identical per-instance code and give bit-identical results.
 *
 * With ways = W > 1, programs with at most 8,192 instances and at least 20,000
 * ops (after the passes) become satellites: each is compiled on its own as a
 * cooperative kernel, W warps splitting the program over each group of 32
 * instances (parallelism inside one expression graph, which CusADi leaves to
 * future work, §VI), and the batch's graph runs them on parallel branches
 * beside the scheduler kernel, started first.  Such a long program with few
 * instances then stops setting the length of the launch.  Its plain mode
 * launches the same cooperative kernels. */
#define CUSADI_BATCH_PERSISTENT 0  /* one graph launch: satellites + scheduler kernel */
#define CUSADI_BATCH_PLAIN 1       /* one kernel launch per program (segment), in order */

/* Compiles and links n programs (irs[j] of nbytes[j] bytes) for N[j]
 * instances each.  opt: dtype, block (32, 64 or 128: instances per tile),
 * maxrregcount, fmad, schedule, segment_ops, compile_threads, cache_dir, and
 * ways (0, or 2..16 warps per group of the satellite kernels); path and
 * compile_limit_ops are ignored (always compiled).  n <= 32.  Errors:
 * INVALID_ARG, INVALID_IR, COMPILE, OOM. */
cusadi_status cusadi_batch_create(const void* const* irs, const size_t* nbytes, const int64_t* N,
                                  int n, const cusadi_options* opt, cusadi_batch* out);
void cusadi_batch_free(cusadi_batch b);

/* Device workspace one evaluation needs (all programs' segment carries). */
size_t cusadi_batch_workspace_bytes(cusadi_batch b);

/* Evaluates every program: in[j] / out[j] are [nnz_in_j x ld_in[j]] and
 * [nnz_out_j x ld_out[j]] device buffers (ld >= N[j]) as for cusadi_eval.
 * mode: CUSADI_BATCH_PERSISTENT or CUSADI_BATCH_PLAIN.  The first call on a
 * device loads the modules and uploads the tile table (allocates; not
 * capturable); the first persistent call captures the graph.  Later calls
 * only copy the buffer table when it changed (a few hundred bytes; with
 * satellites the graph is then captured again, since their launches carry
 * the buffers' addresses) and launch.  The buffer table and the tile
 * counter belong to the batch (one per device), so calls on one batch must not
 * overlap on the GPU: issue them on one stream, or order them with events. */
cusadi_status cusadi_batch_eval(cusadi_batch b, const void* const* in, const int64_t* ld_in,
                                void* const* out, const int64_t* ld_out, void* workspace,
                                int mode, cusadi_stream stream);

/* Selects the tile size (32, 64 or 128 instances = threads per CTA) of the
 * persistent launch; the link holds all three.  INVALID_ARG for other sizes. */
cusadi_status cusadi_batch_set_block(cusadi_batch b, int block);

/* Tile count, threads per CTA, persistent grid size (0 before the first
 * evaluation on this device) and the linked kernel's registers per thread. */
cusadi_status cusadi_batch_info(cusadi_batch b, int64_t* n_tiles, int32_t* block, int32_t* grid,
                                int32_t* registers);

/* counts[op] = number of ops with that IR op code that program `prog` of the
 * batch evaluates per instance (after the passes), for op < n; the weights of
 * a roofline count (as cusadi_op_counts for one function).  INVALID_ARG for a
 * NULL batch or counts, or prog outside [0, n_programs). */
cusadi_status cusadi_batch_op_counts(cusadi_batch b, int prog, int64_t* counts, int n);

/* Waits for all work queued on `stream` with a time limit: OK once it is done,
 * TIMEOUT if it is still running after timeout_seconds (the work is left
 * running; call again to keep waiting), CUDA if the stream reports an error.
 * Polls; never blocks in the driver. */
cusadi_status cusadi_stream_wait(cusadi_stream stream, double timeout_seconds);

/* Writes the generated CUDA source of kernel `segment` (adjoint = 1: of the
 * adjoint kernels) into buf (NUL-terminated, truncated to *len bytes); sets *len
 * to the full size + 1.  UNSUPPORTED on the interpreter path. */
cusadi_status cusadi_source(cusadi_fn fn, int adjoint, int segment, char* buf, size_t* len);

/* Human-readable name of a status, and the last error message of this thread. */
const char* cusadi_status_string(cusadi_status s);
const char* cusadi_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CUSADI_H */
