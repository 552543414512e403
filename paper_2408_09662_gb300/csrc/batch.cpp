// Batched launch of several straight-line programs in one persistent kernel.
//
// CusADi evaluates all operations of one function in a single kernel to save
// launch overhead (§III-A, end).  Here several functions of uneven length and
// instance count share one launch: each program is compiled as relocatable
// one-instance device functions, linked with a scheduler kernel whose CTAs
// take tiles (program, consecutive instances) from an atomic ticket in
// longest-program-first order, and the launch is replayed from a CUDA graph.
// Long programs with few instances ("satellites", with ways > 1) run instead
// as cooperative kernels of their own, W warps per group of 32 instances, on
// parallel branches of the same graph, started before the scheduler kernel.
#include <cuda.h>
#include <cuda_runtime.h>
#include <nvJitLink.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <sstream>
#include <thread>

#include "internal.h"

using namespace cusadi;

namespace {

constexpr int kVariants = 3;
constexpr int kBlocks[kVariants] = {32, 64, 128};
constexpr int kMaxProgs = 32;

struct BTile {
  int32_t prog;
  int32_t count;
  int64_t first;
};

struct BArg {
  const void* X;
  long long ldx;
  void* Y;
  long long ldy;
  void* W;
  long long ldw;
};

struct BatchProg {
  IRFile ir;
  Graph g;
  CodegenResult cg;              // one-instance device functions (linked, scheduler tiles)
  std::vector<std::string> bins;
  CodegenResult scg;             // satellite: standalone cooperative kernels
  std::vector<std::string> sbins;
  bool sat = false;
  int64_t N = 0, n_ops = 0;
  size_t ws_off = 0;
  int64_t ldw = 0;
};

// Satellites: a program with few instances and many ops would set the length
// of the persistent launch (its tiles are the longest chains), so with
// ways = W > 1 it runs as its own cooperative kernel, W warps splitting the
// program over each group of 32 instances (within-instance parallelism), in a
// module of its own (not linked with the scheduler, so it does not raise the
// scheduler's register count), concurrently with the scheduler kernel.
// Which programs: at most 8,192 instances and at least 20,000 ops (after the
// passes): then the one-thread tiles of the program hold fewer warps than the
// GPU has SMs while each runs for as long as a whole many-instance program.
constexpr int64_t kSatMaxN = 8192, kSatMinOps = 20000;

struct BatchDev {
  bool ready = false;
  CUmodule mod = nullptr;
  CUfunction persist[kVariants] = {};
  std::vector<CUfunction> plain;
  int grid[kVariants] = {};
  void* d_tiles[kVariants] = {};
  unsigned* d_ticket = nullptr;
  BArg* d_args = nullptr;
  std::vector<BArg> last;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec[kVariants] = {};
  bool captured = false;                     // exec[] hold the current buffers' launches
  // satellites (per program; empty for scheduler programs)
  std::vector<CUmodule> sat_mods;
  std::vector<std::vector<CUfunction>> sat_fn;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
};

cusadi_status bfail(cusadi_status s, const std::string& m) { return report(s, m); }

}  // namespace

struct cusadi_batch_s {
  cusadi_options opt;
  std::string cache_dir;
  std::vector<BatchProg> progs;
  std::string linked;
  std::vector<BTile> tiles[kVariants];
  int variant = 2;
  size_t ws_bytes = 0;
  int n_sat = 0;                 // programs run as satellites
  int registers = 0;
  std::mutex mu;
  std::map<int, BatchDev> dev;
};

namespace {

const char* tname(bool f64) { return f64 ? "double" : "float"; }

std::string scheduler_source(const cusadi_batch_s& b) {
  const bool f64io = b.opt.dtype == CUSADI_F64, f64w = b.opt.dtype != CUSADI_F32;
  const char* T = tname(f64io);
  const char* TW = tname(f64w);
  std::ostringstream s;
  s << "// Generated batch scheduler: " << b.progs.size() << " programs\n"
    << "struct BArg { const " << T << "* X; long long ldx; " << T << "* Y; long long ldy; " << TW
    << "* W; long long ldw; };\n"
    << "struct BTile { int prog; int count; long long first; };\n";
  for (size_t p = 0; p < b.progs.size(); ++p)
    for (auto& seg : b.progs[p].cg.segs)
      s << "extern \"C\" __device__ void " << seg.name << "(const " << T << "* __restrict__, long long, const "
        << T << "* __restrict__, long long, " << T << "* __restrict__, long long, " << TW
        << "* __restrict__, long long, long long);\n";
  s << "static __device__ __forceinline__ void cs_run(const BArg* __restrict__ A, int p, long long i) {\n"
    << "  switch (p) {\n";
  for (size_t p = 0; p < b.progs.size(); ++p) {
    if (b.progs[p].sat) continue;
    s << "    case " << p << ": {\n      const BArg a = A[" << p << "];\n";
    for (auto& seg : b.progs[p].cg.segs)
      s << "      " << seg.name << "(a.X, a.ldx, a.X, a.ldx, a.Y, a.ldy, a.W, a.ldw, i);\n";
    s << "      break;\n    }\n";
  }
  s << "  }\n}\n";
  for (int v = 0; v < kVariants; ++v) {
    const int B = kBlocks[v];
    s << "extern \"C\" __global__ void __launch_bounds__(" << B << ") cs_batch_" << B
      << "(const BTile* __restrict__ tiles, int n_tiles, unsigned int* ticket,\n"
      << "    const BArg* __restrict__ A) {\n"
      << "  __shared__ int s_t;\n"
      << "  for (;;) {\n"
      << "    if (threadIdx.x == 0) s_t = (int)atomicAdd(ticket, 1u);\n"
      << "    __syncthreads();\n"
      << "    const int t = s_t;\n"
      << "    __syncthreads();\n"
      << "    if (t >= n_tiles) return;\n"
      << "    const BTile tl = tiles[t];\n"
      << "    if ((int)threadIdx.x < tl.count) cs_run(A, tl.prog, tl.first + threadIdx.x);\n"
      << "  }\n}\n";
  }
  for (size_t p = 0; p < b.progs.size(); ++p) {
    if (b.progs[p].sat) continue;
    s << "extern \"C\" __global__ void __launch_bounds__(128) cs_plain_" << p
      << "(const BArg* __restrict__ A, long long N) {\n"
      << "  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;\n"
      << "  if (i < N) cs_run(A, " << p << ", i);\n}\n";
  }
  return s.str();
}

bool link(const std::vector<std::string>& objs, const cusadi_options& o, std::string& out,
          std::string& log) {
  std::vector<std::string> opts = {"-arch=sm_103a"};
  if (o.maxrregcount > 0) opts.push_back("-maxrregcount=" + std::to_string(o.maxrregcount));
  std::vector<const char*> c;
  for (auto& x : opts) c.push_back(x.c_str());
  nvJitLinkHandle h;
  if (nvJitLinkCreate(&h, (uint32_t)c.size(), c.data()) != NVJITLINK_SUCCESS) {
    log = "nvJitLinkCreate failed";
    return false;
  }
  bool ok = true;
  for (size_t i = 0; i < objs.size() && ok; ++i)
    ok = nvJitLinkAddData(h, NVJITLINK_INPUT_CUBIN, objs[i].data(), objs[i].size(),
                          ("obj" + std::to_string(i)).c_str()) == NVJITLINK_SUCCESS;
  if (ok) ok = nvJitLinkComplete(h) == NVJITLINK_SUCCESS;
  if (!ok) {
    size_t n = 0;
    nvJitLinkGetErrorLogSize(h, &n);
    log.resize(n + 1);
    if (n) nvJitLinkGetErrorLog(h, &log[0]);
  } else {
    size_t n = 0;
    nvJitLinkGetLinkedCubinSize(h, &n);
    out.resize(n);
    nvJitLinkGetLinkedCubin(h, &out[0]);
  }
  nvJitLinkDestroy(&h);
  return ok;
}

cusadi_status batch_device(cusadi_batch b, BatchDev** out) {
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return bfail(CUSADI_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ce));
  std::lock_guard<std::mutex> lk(b->mu);
  BatchDev& d = b->dev[dev];
  if (d.ready) { *out = &d; return CUSADI_OK; }
  if ((ce = cudaFree(nullptr)) != cudaSuccess) return bfail(CUSADI_E_CUDA, cudaGetErrorString(ce));
  const Driver& D = driver();
  if (!D.ok) return bfail(CUSADI_E_CUDA, "CUDA driver entry points unavailable");
  CUresult r = D.moduleLoadData(&d.mod, b->linked.data());
  if (r != CUDA_SUCCESS) return bfail(CUSADI_E_CUDA, "cuModuleLoadData failed: " + std::to_string(r));
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int v = 0; v < kVariants; ++v) {
    std::string nm = "cs_batch_" + std::to_string(kBlocks[v]);
    if ((r = D.moduleGetFunction(&d.persist[v], d.mod, nm.c_str())) != CUDA_SUCCESS)
      return bfail(CUSADI_E_CUDA, "missing " + nm);
    int per_sm = 0;
    D.occupancy(&per_sm, d.persist[v], kBlocks[v], 0);
    const int64_t nt = (int64_t)b->tiles[v].size();
    // with satellites, the scheduler kernel takes the SMs in proportion to its
    // share of the work (ops x instances), so the satellites find SMs free
    // whichever of them the GPU starts first
    int64_t sm_share = sms;
    if (b->n_sat > 0) {
      double reg = 0, sat = 0;
      for (const BatchProg& P : b->progs) (P.sat ? sat : reg) += (double)P.n_ops * (double)P.N;
      sm_share = std::max<int64_t>(1, (int64_t)std::llround(sms * reg / std::max(reg + sat, 1.0)));
    }
    d.grid[v] = (int)std::max<int64_t>(1, std::min<int64_t>(sm_share * std::max(per_sm, 1), nt));
    size_t tb = std::max<size_t>(1, b->tiles[v].size()) * sizeof(BTile);
    if ((ce = cudaMalloc(&d.d_tiles[v], tb)) != cudaSuccess) return bfail(CUSADI_E_CUDA, cudaGetErrorString(ce));
    if (!b->tiles[v].empty())
      cudaMemcpy(d.d_tiles[v], b->tiles[v].data(), b->tiles[v].size() * sizeof(BTile), cudaMemcpyHostToDevice);
  }
  d.plain.assign(b->progs.size(), nullptr);
  d.sat_fn.assign(b->progs.size(), {});
  for (size_t p = 0; p < b->progs.size(); ++p) {
    const BatchProg& P = b->progs[p];
    if (!P.sat) {
      std::string nm = "cs_plain_" + std::to_string(p);
      if ((r = D.moduleGetFunction(&d.plain[p], d.mod, nm.c_str())) != CUDA_SUCCESS)
        return bfail(CUSADI_E_CUDA, "missing " + nm);
      continue;
    }
    for (size_t k = 0; k < P.sbins.size(); ++k) {
      CUmodule m;
      if ((r = D.moduleLoadData(&m, P.sbins[k].data())) != CUDA_SUCCESS)
        return bfail(CUSADI_E_CUDA, "cuModuleLoadData (satellite) failed: " + std::to_string(r));
      d.sat_mods.push_back(m);
      CUfunction f;
      if ((r = D.moduleGetFunction(&f, m, P.scg.segs[k].name.c_str())) != CUDA_SUCCESS)
        return bfail(CUSADI_E_CUDA, "missing " + P.scg.segs[k].name);
      if (P.scg.smem_bytes > 48 * 1024 &&
          (r = D.funcSetAttribute(f, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)P.scg.smem_bytes)) != CUDA_SUCCESS)
        return bfail(CUSADI_E_CUDA, "cuFuncSetAttribute failed: " + std::to_string(r));
      d.sat_fn[p].push_back(f);
    }
  }
  if ((ce = cudaMalloc((void**)&d.d_ticket, 256)) != cudaSuccess) return bfail(CUSADI_E_CUDA, cudaGetErrorString(ce));
  if ((ce = cudaMalloc((void**)&d.d_args, kMaxProgs * sizeof(BArg))) != cudaSuccess)
    return bfail(CUSADI_E_CUDA, cudaGetErrorString(ce));
  if ((ce = cudaStreamCreateWithFlags(&d.cap, cudaStreamNonBlocking)) != cudaSuccess)
    return bfail(CUSADI_E_CUDA, cudaGetErrorString(ce));
  if (b->n_sat > 0) {
    if ((ce = cudaEventCreateWithFlags(&d.fork, cudaEventDisableTiming)) != cudaSuccess)
      return bfail(CUSADI_E_CUDA, cudaGetErrorString(ce));
    for (int k = 0; k < b->n_sat; ++k) {
      cudaStream_t st;
      cudaEvent_t ev;
      if ((ce = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess)
        return bfail(CUSADI_E_CUDA, cudaGetErrorString(ce));
      d.side.push_back(st);
      if ((ce = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
        return bfail(CUSADI_E_CUDA, cudaGetErrorString(ce));
      d.join.push_back(ev);
    }
  }
  d.ready = true;
  *out = &d;
  return CUSADI_OK;
}

// Launches satellite p's kernels (one per segment, in order) on `st`.
cusadi_status launch_satellite(cusadi_batch b, BatchDev& d, size_t p, const BArg& a, cudaStream_t st) {
  const BatchProg& P = b->progs[p];
  const void* X = a.X;
  void* Y = a.Y;
  void* W = a.W;
  long long ldx = a.ldx, ldy = a.ldy, n = P.N, ldw = a.ldw;
  int acc = 0, reduce = 0, vec = 0;
  for (CUfunction f : d.sat_fn[p]) {
    void* args[] = {(void*)&X, &ldx, (void*)&X, &ldx, &Y, &ldy, &n, &W, &ldw, &acc, &reduce, &vec};
    CUresult r = driver().launchKernel(f, (unsigned)((P.N + 31) / 32), 1, 1, 32u * (unsigned)P.scg.coop_ways, 1, 1,
                                       (unsigned)P.scg.smem_bytes, (CUstream)st, args, nullptr);
    if (r != CUDA_SUCCESS) return bfail(CUSADI_E_CUDA, "cuLaunchKernel (satellite) failed: " + std::to_string(r));
  }
  return CUSADI_OK;
}

// One graph per tile size: reset the ticket; fork the satellites onto side
// streams (their kernels carry the buffers' addresses, so a change of buffers
// re-captures); run the scheduler kernel; join.
cusadi_status capture_graphs(cusadi_batch b, BatchDev& d, const std::vector<BArg>& args) {
  for (int v = 0; v < kVariants; ++v)
    if (d.exec[v]) { cudaGraphExecDestroy(d.exec[v]); d.exec[v] = nullptr; }
  d.captured = false;
  const Driver& D = driver();
  for (int v = 0; v < kVariants; ++v) {
    cudaGraph_t g;
    cudaError_t ce = cudaStreamBeginCapture(d.cap, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) return bfail(CUSADI_E_CUDA, cudaGetErrorString(ce));
    bool ok = cudaMemsetAsync(d.d_ticket, 0, sizeof(unsigned), d.cap) == cudaSuccess;
    if (b->n_sat > 0) ok = ok && cudaEventRecord(d.fork, d.cap) == cudaSuccess;
    std::vector<size_t> sats;                        // longest first
    for (size_t p = 0; p < b->progs.size(); ++p)
      if (b->progs[p].sat) sats.push_back(p);
    std::stable_sort(sats.begin(), sats.end(),
                     [&](size_t a, size_t c) { return b->progs[a].n_ops > b->progs[c].n_ops; });
    int k = 0;
    for (size_t p : sats) {
      if (!ok) break;
      ok = cudaStreamWaitEvent(d.side[k], d.fork, 0) == cudaSuccess &&
           launch_satellite(b, d, p, args[p], d.side[k]) == CUSADI_OK &&
           cudaEventRecord(d.join[k], d.side[k]) == cudaSuccess;
      ++k;
    }
    int nt = (int)b->tiles[v].size();
    CUresult r = CUDA_SUCCESS;
    if (ok && nt > 0) {
      void* kargs[] = {&d.d_tiles[v], &nt, &d.d_ticket, &d.d_args};
      r = D.launchKernel(d.persist[v], (unsigned)d.grid[v], 1, 1, (unsigned)kBlocks[v], 1, 1, 0u,
                         (CUstream)d.cap, kargs, nullptr);
    }
    for (int j = 0; ok && j < k; ++j) ok = cudaStreamWaitEvent(d.cap, d.join[j], 0) == cudaSuccess;
    ce = cudaStreamEndCapture(d.cap, &g);
    if (!ok || r != CUDA_SUCCESS || ce != cudaSuccess)
      return bfail(CUSADI_E_CUDA, "capturing the batch launch failed");
    ce = cudaGraphInstantiate(&d.exec[v], g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return bfail(CUSADI_E_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ce));
  }
  d.captured = true;
  return CUSADI_OK;
}

}  // namespace

extern "C" {

cusadi_status cusadi_batch_create(const void* const* irs, const size_t* nbytes, const int64_t* N,
                                  int n, const cusadi_options* opt, cusadi_batch* out) {
  if (!out) return bfail(CUSADI_E_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n <= 0 || n > kMaxProgs || !irs || !nbytes || !N)
    return bfail(CUSADI_E_INVALID_ARG, "need 1..32 programs with sizes and instance counts");
  std::unique_ptr<cusadi_batch_s> b(new cusadi_batch_s);
  cusadi_default_options(&b->opt);
  if (opt) b->opt = *opt;
  cusadi_options& o = b->opt;
  if (o.cache_dir) b->cache_dir = o.cache_dir;
  o.cache_dir = nullptr;
  if (o.dtype < 0 || o.dtype > 2) return bfail(CUSADI_E_INVALID_ARG, "dtype must be F64, F32 or MIXED");
  if (o.maxrregcount < 0 || o.maxrregcount > 255) return bfail(CUSADI_E_INVALID_ARG, "maxrregcount must be in [0, 255]");
  b->variant = -1;
  for (int v = 0; v < kVariants; ++v)
    if (o.block == kBlocks[v]) b->variant = v;
  if (b->variant < 0) return bfail(CUSADI_E_INVALID_ARG, "batch block must be 32, 64 or 128");
  if (o.ways < 0 || o.ways == 1 || o.ways > 16)
    return bfail(CUSADI_E_INVALID_ARG, "batch ways must be 0 or 2..16");
  b->progs.resize(n);
  const size_t elt_ws = o.dtype == CUSADI_F32 ? 4 : 8;
  try {
    for (int p = 0; p < n; ++p) {
      if (!irs[p] || nbytes[p] == 0 || N[p] < 1 || N[p] > ((int64_t)1 << 31))
        return bfail(CUSADI_E_INVALID_ARG, "program " + std::to_string(p) + ": empty or bad instance count");
      BatchProg& P = b->progs[p];
      std::string err;
      if (!parse_ir((const uint8_t*)irs[p], nbytes[p], P.ir, err))
        return bfail(CUSADI_E_INVALID_IR, "program " + std::to_string(p) + ": " + err);
      P.g = build_ssa(P.ir);
      simplify(P.g, o.dtype);
      if (o.schedule) schedule(P.g);
      P.n_ops = count_ops(P.g);
      P.N = N[p];
    }
    for (int p = 0; p < n; ++p)
      if (o.ways > 1 && b->progs[p].N <= kSatMaxN && b->progs[p].n_ops >= kSatMinOps) {
        b->progs[p].sat = true;
        ++b->n_sat;
      }
    for (int p = 0; p < n; ++p) {
      BatchProg& P = b->progs[p];
      CodegenOptions co;
      co.dtype = o.dtype;
      co.segment_ops = o.segment_ops;
      co.inline_math = o.inline_math;
      co.own_math = o.own_math;
      co.device_fn = true;
      co.prefix = "cs_b" + std::to_string(p);
      if (!P.sat) {
        P.cg = generate(P.g, co);
      } else {
        // standalone kernels: W warps per group of 32 instances, one group per CTA
        CodegenOptions cc = co;
        cc.device_fn = false;
        cc.prefix = "cs_bs" + std::to_string(p);
        cc.maxrregcount = o.maxrregcount;
        P.scg = generate_coop(P.g, cc, plan_coop(P.g, o.ways, 8.0));
      }
      P.ldw = (P.N + 31) / 32 * 32;
      b->ws_bytes = (b->ws_bytes + 255) / 256 * 256;
      P.ws_off = b->ws_bytes;
      b->ws_bytes += (size_t)std::max(P.cg.ws_rows, P.scg.ws_rows) * P.ldw * elt_ws;
    }
  } catch (const std::bad_alloc&) {
    return bfail(CUSADI_E_OOM, "out of host memory");
  }
  // compile every segment (all programs) in parallel, then the scheduler, then link
  struct Job {
    const std::string* src; const std::string* name; std::string* bin; std::string log; bool ok;
    bool standalone = false;    // a satellite kernel: its own module, not relocatable
  };
  std::vector<std::string> sched(1);
  std::string sched_src = scheduler_source(*b), sched_name = "cs_batch_sched";
  std::vector<Job> jobs;
  for (auto& P : b->progs) {
    P.bins.assign(P.cg.segs.size(), std::string());
    for (size_t s = 0; s < P.cg.segs.size(); ++s)
      jobs.push_back({&P.cg.segs[s].source, &P.cg.segs[s].name, &P.bins[s], "", false});
    P.sbins.assign(P.scg.segs.size(), std::string());
    for (size_t s = 0; s < P.scg.segs.size(); ++s)
      jobs.push_back({&P.scg.segs[s].source, &P.scg.segs[s].name, &P.sbins[s], "", false, true});
  }
  jobs.push_back({&sched_src, &sched_name, &sched[0], "", false});
  std::vector<std::string> opts = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo",
                                   "-DNDEBUG", "--relocatable-device-code=true"};
  opts.push_back(o.fmad ? "--fmad=true" : "--fmad=false");
  if (o.maxrregcount > 0) opts.push_back("--maxrregcount=" + std::to_string(o.maxrregcount));
  std::vector<std::string> sopts;
  for (auto& x : opts)
    if (x != "--relocatable-device-code=true") sopts.push_back(x);
  // biggest first, so the longest compile starts at once
  std::vector<size_t> order(jobs.size());
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](size_t a, size_t c) { return jobs[a].src->size() > jobs[c].src->size(); });
  int nt = o.compile_threads > 0 ? o.compile_threads : (int)std::max(1u, std::thread::hardware_concurrency());
  nt = std::min<int>(nt, (int)jobs.size());
  std::atomic<size_t> next{0};
  const char* cache = b->cache_dir.empty() ? nullptr : b->cache_dir.c_str();
  auto work = [&] {
    for (size_t k; (k = next.fetch_add(1)) < order.size();) {
      Job& j = jobs[order[k]];
      j.ok = compile_nvrtc(*j.src, *j.name, j.standalone ? sopts : opts, cache, *j.bin, j.log);
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) th.emplace_back(work);
  for (auto& t : th) t.join();
  for (auto& j : jobs)
    if (!j.ok) return bfail(CUSADI_E_COMPILE, "NVRTC failed on " + *j.name + ": " + j.log.substr(0, 4000));
  std::vector<std::string> objs;
  for (auto& P : b->progs) {
    for (auto& x : P.bins) objs.push_back(x);
  }
  objs.push_back(sched[0]);
  std::string log;
  if (!link(objs, o, b->linked, log)) return bfail(CUSADI_E_COMPILE, "nvJitLink failed: " + log.substr(0, 4000));
  // tile tables, longest program first
  std::vector<int> byops(n);
  std::iota(byops.begin(), byops.end(), 0);
  std::stable_sort(byops.begin(), byops.end(), [&](int a, int c) { return b->progs[a].n_ops > b->progs[c].n_ops; });
  for (int v = 0; v < kVariants; ++v)
    for (int p : byops) {
      if (b->progs[p].sat) continue;
      const int64_t t = kBlocks[v];
      for (int64_t f = 0; f < b->progs[p].N; f += t)
        b->tiles[v].push_back({p, (int32_t)std::min<int64_t>(t, b->progs[p].N - f), f});
    }
  *out = b.release();
  return CUSADI_OK;
}

void cusadi_batch_free(cusadi_batch b) {
  if (!b) return;
  for (auto& kv : b->dev) {
    BatchDev& d = kv.second;
    if (cudaSetDevice(kv.first) != cudaSuccess) continue;
    for (int v = 0; v < kVariants; ++v) {
      if (d.exec[v]) cudaGraphExecDestroy(d.exec[v]);
      if (d.d_tiles[v]) cudaFree(d.d_tiles[v]);
    }
    if (d.d_ticket) cudaFree(d.d_ticket);
    if (d.d_args) cudaFree(d.d_args);
    if (d.cap) cudaStreamDestroy(d.cap);
    for (cudaStream_t st : d.side) cudaStreamDestroy(st);
    for (cudaEvent_t ev : d.join) cudaEventDestroy(ev);
    if (d.fork) cudaEventDestroy(d.fork);
    if (d.mod && driver().ok) driver().moduleUnload(d.mod);
    for (CUmodule m : d.sat_mods)
      if (driver().ok) driver().moduleUnload(m);
  }
  delete b;
}

size_t cusadi_batch_workspace_bytes(cusadi_batch b) { return b ? b->ws_bytes : 0; }

cusadi_status cusadi_batch_set_block(cusadi_batch b, int block) {
  if (!b) return bfail(CUSADI_E_INVALID_ARG, "NULL batch");
  for (int v = 0; v < kVariants; ++v)
    if (block == kBlocks[v]) {
      b->variant = v;
      return CUSADI_OK;
    }
  return bfail(CUSADI_E_INVALID_ARG, "batch block must be 32, 64 or 128");
}

cusadi_status cusadi_batch_eval(cusadi_batch b, const void* const* in, const int64_t* ld_in,
                                void* const* out, const int64_t* ld_out, void* workspace,
                                int mode, cusadi_stream stream) {
  if (!b || !in || !ld_in || !out || !ld_out) return bfail(CUSADI_E_INVALID_ARG, "NULL argument");
  if (mode != CUSADI_BATCH_PERSISTENT && mode != CUSADI_BATCH_PLAIN)
    return bfail(CUSADI_E_INVALID_ARG, "unknown batch mode");
  if (b->ws_bytes > 0 && !workspace)
    return bfail(CUSADI_E_INVALID_ARG, "this batch needs a workspace (cusadi_batch_workspace_bytes)");
  const size_t n = b->progs.size();
  std::vector<BArg> args(n);
  for (size_t p = 0; p < n; ++p) {
    const BatchProg& P = b->progs[p];
    if ((P.ir.nnz_in > 0 && (!in[p] || ld_in[p] < P.N)) || (P.ir.nnz_out > 0 && (!out[p] || ld_out[p] < P.N)))
      return bfail(CUSADI_E_INVALID_ARG, "program " + std::to_string(p) + ": missing buffer or ld < N");
    args[p] = {in[p], (long long)ld_in[p], out[p], (long long)ld_out[p],
               (char*)workspace + P.ws_off, (long long)P.ldw};
  }
  BatchDev* d;
  cusadi_status s = batch_device(b, &d);
  if (s != CUSADI_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  bool same = d->last.size() == n;
  for (size_t p = 0; same && p < n; ++p) same = std::memcmp(&d->last[p], &args[p], sizeof(BArg)) == 0;
  if (!same) {
    // pageable source: the call returns once the bytes are staged, so `args` may go away
    cudaError_t ce = cudaMemcpyAsync(d->d_args, args.data(), n * sizeof(BArg), cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) return bfail(CUSADI_E_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(ce));
    d->last = args;
    if (b->n_sat > 0) d->captured = false;   // the satellites' launches carry the addresses
  }
  if (mode == CUSADI_BATCH_PERSISTENT) {
    if (!d->captured) {
      std::lock_guard<std::mutex> lk(b->mu);
      s = capture_graphs(b, *d, args);
      if (s != CUSADI_OK) return s;
    }
    cudaError_t ce = cudaGraphLaunch(d->exec[b->variant], st);
    if (ce != cudaSuccess) return bfail(CUSADI_E_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(ce));
    return CUSADI_OK;
  }
  for (size_t p = 0; p < n; ++p) {
    if (b->progs[p].sat) {
      s = launch_satellite(b, *d, p, args[p], st);
      if (s != CUSADI_OK) return s;
      continue;
    }
    long long N = b->progs[p].N;
    void* a[] = {&d->d_args, &N};
    CUresult r = driver().launchKernel(d->plain[p], (unsigned)((N + 127) / 128), 1, 1, 128, 1, 1, 0u,
                                       (CUstream)st, a, nullptr);
    if (r != CUDA_SUCCESS) return bfail(CUSADI_E_CUDA, "cuLaunchKernel failed: " + std::to_string(r));
  }
  return CUSADI_OK;
}

cusadi_status cusadi_batch_info(cusadi_batch b, int64_t* n_tiles, int32_t* block, int32_t* grid,
                                int32_t* registers) {
  if (!b) return bfail(CUSADI_E_INVALID_ARG, "NULL batch");
  if (n_tiles) *n_tiles = (int64_t)b->tiles[b->variant].size();
  if (block) *block = kBlocks[b->variant];
  if (grid) {
    *grid = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
      std::lock_guard<std::mutex> lk(b->mu);
      auto it = b->dev.find(dev);
      if (it != b->dev.end() && it->second.ready) *grid = it->second.grid[b->variant];
    }
  }
  if (registers) {
    *registers = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
      std::lock_guard<std::mutex> lk(b->mu);
      auto it = b->dev.find(dev);
      if (it != b->dev.end() && it->second.ready && driver().funcGetAttribute)
        driver().funcGetAttribute(registers, CU_FUNC_ATTRIBUTE_NUM_REGS,
                                  it->second.persist[b->variant]);
    }
  }
  return CUSADI_OK;
}

cusadi_status cusadi_batch_op_counts(cusadi_batch b, int prog, int64_t* counts, int n) {
  if (!b || !counts || n < 0) return bfail(CUSADI_E_INVALID_ARG, "NULL argument");
  if (prog < 0 || prog >= (int)b->progs.size())
    return bfail(CUSADI_E_INVALID_ARG, "program index out of range");
  std::vector<int64_t> h;
  op_histogram(b->progs[prog].g, h);
  for (int i = 0; i < n; ++i) counts[i] = i < (int)h.size() ? h[i] : 0;
  return CUSADI_OK;
}

}  // extern "C"
