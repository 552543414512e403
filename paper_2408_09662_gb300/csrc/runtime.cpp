// Runtime and C ABI of libcusadi: load (parse, passes, code generation, NVRTC
// compile with a content-hash cache), lazy per-device module loading, and the
// asynchronous evaluation calls.  Compiling generated code once and calling it
// from PyTorch on GPU-resident tensors is the CusADi workflow (§III-A end,
// §III-B); here the compile happens at load time through NVRTC instead of an
// offline toolkit run.
#include <cuda.h>
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <thread>
#include <unordered_map>

#include "internal.h"

using namespace cusadi;

namespace {

thread_local std::string t_last_error;

cusadi_status fail(cusadi_status s, const std::string& msg) {
  t_last_error = msg;
  return s;
}

uint64_t fnv1a(const void* p, size_t n, uint64_t h = 1469598103934665603ull) {
  const uint8_t* b = (const uint8_t*)p;
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

std::mutex g_cache_mu;
std::unordered_map<uint64_t, std::string> g_cubins;  // content hash -> cubin

}  // namespace

namespace cusadi {

bool compile_nvrtc(const std::string& src, const std::string& name,
                   const std::vector<std::string>& opts, const char* cache_dir, std::string& cubin,
                   std::string& log) {
  int vmaj = 0, vmin = 0;
  nvrtcVersion(&vmaj, &vmin);
  uint64_t h = fnv1a(src.data(), src.size());
  for (auto& o : opts) h = fnv1a(o.data(), o.size() + 1, h);
  h = fnv1a(&vmaj, sizeof vmaj, h);
  h = fnv1a(&vmin, sizeof vmin, h);
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_cubins.find(h);
    if (it != g_cubins.end()) { cubin = it->second; return true; }
  }
  char hex[32];
  std::snprintf(hex, sizeof hex, "%016llx", (unsigned long long)h);
  std::string path = cache_dir && *cache_dir ? std::string(cache_dir) + "/cs_" + hex + ".cubin" : "";
  if (!path.empty()) {
    std::ifstream f(path, std::ios::binary);
    if (f) {
      std::ostringstream ss;
      ss << f.rdbuf();
      cubin = ss.str();
      if (!cubin.empty()) {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        g_cubins[h] = cubin;
        return true;
      }
    }
  }
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), (name + ".cu").c_str(), 0, nullptr, nullptr) !=
      NVRTC_SUCCESS) {
    log = "nvrtcCreateProgram failed";
    return false;
  }
  std::vector<const char*> o;
  for (auto& s : opts) o.push_back(s.c_str());
  nvrtcResult rc = nvrtcCompileProgram(prog, (int)o.size(), o.data());
  size_t ls = 0;
  nvrtcGetProgramLogSize(prog, &ls);
  if (ls > 1) {
    log.resize(ls);
    nvrtcGetProgramLog(prog, &log[0]);
  }
  if (rc != NVRTC_SUCCESS) {
    log = std::string(nvrtcGetErrorString(rc)) + ": " + log;
    nvrtcDestroyProgram(&prog);
    return false;
  }
  size_t cs = 0;
  nvrtcGetCUBINSize(prog, &cs);
  cubin.resize(cs);
  nvrtcGetCUBIN(prog, &cubin[0]);
  nvrtcDestroyProgram(&prog);
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_cubins[h] = cubin;
  }
  if (!path.empty()) {
    std::string tmp = path + ".tmp" + std::to_string((unsigned long long)std::hash<std::thread::id>()(std::this_thread::get_id()));
    std::ofstream f(tmp, std::ios::binary);
    if (f) {
      f.write(cubin.data(), (std::streamsize)cubin.size());
      f.close();
      std::rename(tmp.c_str(), path.c_str());
    }
  }
  return true;
}

const Driver& driver() {
  static Driver d;
  static std::once_flag once;
  std::call_once(once, [] {
    auto get = [](const char* sym, void** fp) {
      cudaDriverEntryPointQueryResult q;
      return cudaGetDriverEntryPointByVersion(sym, fp, 12000, cudaEnableDefault, &q) ==
                 cudaSuccess &&
             q == cudaDriverEntryPointSuccess && *fp != nullptr;
    };
    d.ok = get("cuModuleLoadData", (void**)&d.moduleLoadData) &&
           get("cuModuleGetFunction", (void**)&d.moduleGetFunction) &&
           get("cuModuleUnload", (void**)&d.moduleUnload) &&
           get("cuLaunchKernel", (void**)&d.launchKernel) &&
           get("cuOccupancyMaxActiveBlocksPerMultiprocessor", (void**)&d.occupancy) &&
           get("cuFuncGetAttribute", (void**)&d.funcGetAttribute) &&
           get("cuFuncSetAttribute", (void**)&d.funcSetAttribute) &&
           get("cuModuleGetGlobal", (void**)&d.moduleGetGlobal);
  });
  return d;
}

}  // namespace cusadi

namespace {

struct DevState {
  bool fwd_ready = false, adj_ready = false;
  int sms = 0;                       // streaming multiprocessors of the device
  std::vector<CUmodule> mods;
  std::vector<CUfunction> fwd, adj;
  CUfunction adj_finish = nullptr;   // fixed-order sum of the reduced rows' per-instance terms
  void* d_ops_fwd = nullptr;
  double* d_k_fwd = nullptr;
  void* d_ops_adj = nullptr;
  double* d_k_adj = nullptr;
  int64_t* d_reduce_rows = nullptr;  // interpreter adjoint: rows summed over instances
  // host-buffer evaluation: a copy-in and a copy-out stream, one compute
  // stream per chunk, and the events that order them (created on first use)
  cudaStream_t h_in = nullptr, h_out = nullptr;
  std::vector<cudaStream_t> h_comp;
  std::map<int, int32_t*> dense_map;  // output argument -> dense index map (device)
  std::vector<cudaEvent_t> hev;
};

// One compiled or packed evaluation direction (forward or adjoint).
struct Direction {
  Graph g;
  int64_t n_ops = 0, n_slots = 0;
  std::vector<int64_t> hist, hist_f64;
  CodegenResult cg;
  std::vector<std::string> bins;
  InterpProgram ip;
};

}  // namespace

struct cusadi_fn_s {
  cusadi_options opt;
  std::string cache_dir;
  IRFile ir;
  int path = CUSADI_PATH_COMPILED;
  Direction fwd;
  std::mutex adj_mu;
  bool adj_built = false;
  cusadi_status adj_status = CUSADI_OK;
  std::string adj_error;
  Direction adj;
  double compile_seconds = 0;
  std::string compile_fallback;   // why AUTO fell back to the interpreter, if it did
  std::mutex dev_mu;
  std::map<int, DevState> dev;
  std::mutex host_mu;             // serialises the enqueue of host-buffer evaluations
};

namespace {

std::vector<std::string> nvrtc_options(const cusadi_options& o) {
  std::vector<std::string> v = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo",
                                "-DNDEBUG"};
  v.push_back(o.fmad ? "--fmad=true" : "--fmad=false");
  if (o.maxrregcount > 0) v.push_back("--maxrregcount=" + std::to_string(o.maxrregcount));
  return v;
}

// Host-side fault injection for tests: CUSADI_INJECT=compile makes every
// NVRTC compile of this process fail (nothing on the GPU is involved).
bool injected(const char* what) {
  const char* e = std::getenv("CUSADI_INJECT");
  return e && std::strstr(e, what) != nullptr;
}

cusadi_status compile_direction(cusadi_fn fn, Direction& d, bool adjoint) {
  CodegenOptions co;
  co.dtype = fn->opt.dtype;
  co.block = fn->opt.block;
  co.segment_ops = fn->opt.segment_ops;
  co.inline_math = fn->opt.inline_math;
  co.maxrregcount = fn->opt.maxrregcount;
  co.own_math = fn->opt.own_math;
  co.debug_checks = fn->opt.debug_checks != 0;
  co.inst_per_thread = fn->opt.ways > 1 ? 1 : fn->opt.inst_per_thread;
  co.sync_every = fn->opt.ways > 1 ? 0 : fn->opt.sync_every;
  co.coop_groups = fn->opt.coop_groups;
  co.spill_values = fn->opt.ways > 1 ? 0 : fn->opt.spill_values;
  co.spill_shared_kb = fn->opt.spill_shared_kb;
  co.pair_calls = fn->opt.ways > 1 ? 0 : fn->opt.pair_calls;
  co.adjoint = adjoint;
  co.split = adjoint ? fn->ir.nnz_in : -1;
  static const char* tag[] = {"f64", "f32", "mixed"};
  co.prefix = std::string(adjoint ? "cs_adj_" : "cs_fwd_") + tag[fn->opt.dtype];
  if (fn->opt.ways > 1) {
    co.prefix = std::string(adjoint ? "cs_coopadj" : "cs_coop") + std::to_string(fn->opt.ways) + "_" +
                tag[fn->opt.dtype];
    CoopPlan plan = plan_coop(d.g, fn->opt.ways, 8.0);
    // the CTA's groups share the shared-memory budget
    co.coop_shared_kb = std::min(co.coop_shared_kb, 200 / std::max(1, co.coop_groups));
    d.cg = generate_coop(d.g, co, plan);
    if (d.cg.smem_bytes > 200 * 1024)   // cannot happen: overflow goes to the workspace
      return fail(CUSADI_E_UNSUPPORTED, "cooperative plan needs too much shared memory");
  } else {
    d.cg = generate(d.g, co);
  }
  const size_t ns = d.cg.segs.size();
  d.bins.assign(ns, std::string());
  std::vector<std::string> logs(ns);
  std::vector<uint8_t> ok(ns, 0);
  auto opts = nvrtc_options(fn->opt);
  int nt = fn->opt.compile_threads > 0 ? fn->opt.compile_threads
                                       : (int)std::max(1u, std::thread::hardware_concurrency());
  nt = (int)std::min<size_t>((size_t)nt, ns);
  std::atomic<size_t> next{0};
  auto work = [&]() {
    for (size_t s; (s = next.fetch_add(1)) < ns;)
      ok[s] = compile_nvrtc(d.cg.segs[s].source, d.cg.segs[s].name, opts,
                            fn->cache_dir.empty() ? nullptr : fn->cache_dir.c_str(), d.bins[s],
                            logs[s]);
  };
  if (nt <= 1) work();
  else {
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t) th.emplace_back(work);
    for (auto& t : th) t.join();
  }
  if (injected("compile")) return fail(CUSADI_E_COMPILE, "NVRTC failure injected (CUSADI_INJECT=compile)");
  for (size_t s = 0; s < ns; ++s)
    if (!ok[s]) return fail(CUSADI_E_COMPILE, "NVRTC failed on " + d.cg.segs[s].name + ": " + logs[s].substr(0, 4000));
  return CUSADI_OK;
}

cusadi_status prepare_direction(cusadi_fn fn, Direction& d, bool adjoint) {
  simplify(d.g, fn->opt.dtype);
  if (fn->opt.schedule) schedule(d.g);
  d.n_ops = count_ops(d.g);
  d.n_slots = max_live(d.g);
  op_histogram(d.g, d.hist);
  op_histogram(d.g, d.hist_f64, true);
  if (fn->path == CUSADI_PATH_COMPILED) {
    cusadi_status s = compile_direction(fn, d, adjoint);
    // AUTO falls back to the interpreter kernel when the compiler fails
    if (s != CUSADI_E_COMPILE || fn->opt.path != CUSADI_PATH_AUTO || adjoint) return s;
    fn->compile_fallback = t_last_error;
    fn->path = CUSADI_PATH_INTERP;
  }
  std::string err;
  if (!pack_interp(d.g, d.ip, err, interp_shared_slots(fn->opt.dtype, fn->opt.interp_shared_kb)))
    return fail(CUSADI_E_UNSUPPORTED, err);
  d.n_slots = d.ip.n_slots;
  return CUSADI_OK;
}

cusadi_status ensure_adjoint(cusadi_fn fn) {
  std::lock_guard<std::mutex> lk(fn->adj_mu);
  if (fn->adj_built) {
    if (fn->adj_status != CUSADI_OK) t_last_error = fn->adj_error;
    return fn->adj_status;
  }
  auto t0 = std::chrono::steady_clock::now();
  fn->adj.g = adjoint_graph(fn->fwd.g);
  fn->adj_status = prepare_direction(fn, fn->adj, true);
  if (fn->adj_status != CUSADI_OK) fn->adj_error = t_last_error;
  fn->compile_seconds +=
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  fn->adj_built = true;
  return fn->adj_status;
}

cusadi_status cuda_fail(const char* what, int code) {
  return fail(CUSADI_E_CUDA, std::string(what) + " failed with code " + std::to_string(code));
}

// Loads the direction's modules (or uploads its instruction stream) on the
// current device.  Called with fn->dev_mu held.
cusadi_status load_on_device(cusadi_fn fn, DevState& ds, bool adjoint) {
  cudaError_t ce = cudaFree(nullptr);  // makes the device's primary context current
  if (ce != cudaSuccess) return fail(CUSADI_E_CUDA, std::string("CUDA init: ") + cudaGetErrorString(ce));
  if (!driver().ok) return fail(CUSADI_E_CUDA, "CUDA driver entry points unavailable");
  if (ds.sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&ds.sms, cudaDevAttrMultiProcessorCount, dev);
  }
  Direction& d = adjoint ? fn->adj : fn->fwd;
  if (fn->path == CUSADI_PATH_INTERP) {
    void* ops = nullptr;
    double* k = nullptr;
    size_t ob = std::max<size_t>(d.ip.ops.size(), 1) * sizeof(IOp);
    size_t kb = std::max<size_t>(d.ip.k.size(), 1) * sizeof(double);
    if ((ce = cudaMalloc(&ops, ob)) != cudaSuccess) return cuda_fail("cudaMalloc", ce);
    if ((ce = cudaMalloc((void**)&k, kb)) != cudaSuccess) { cudaFree(ops); return cuda_fail("cudaMalloc", ce); }
    if (!d.ip.ops.empty()) cudaMemcpy(ops, d.ip.ops.data(), d.ip.ops.size() * sizeof(IOp), cudaMemcpyHostToDevice);
    if (!d.ip.k.empty()) cudaMemcpy(k, d.ip.k.data(), d.ip.k.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (adjoint && !d.ip.reduce_rows.empty()) {
      const size_t rb = d.ip.reduce_rows.size() * sizeof(int64_t);
      if ((ce = cudaMalloc((void**)&ds.d_reduce_rows, rb)) != cudaSuccess) return cuda_fail("cudaMalloc", ce);
      cudaMemcpy(ds.d_reduce_rows, d.ip.reduce_rows.data(), rb, cudaMemcpyHostToDevice);
    }
    if ((ce = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail("upload", ce);
    (adjoint ? ds.d_ops_adj : ds.d_ops_fwd) = ops;
    (adjoint ? ds.d_k_adj : ds.d_k_fwd) = k;
  } else {
    std::vector<CUfunction>& fs = adjoint ? ds.adj : ds.fwd;
    fs.clear();
    for (size_t s = 0; s < d.bins.size(); ++s) {
      CUmodule m;
      CUresult r = driver().moduleLoadData(&m, d.bins[s].data());
      if (r != CUDA_SUCCESS) return cuda_fail("cuModuleLoadData", r);
      ds.mods.push_back(m);
      CUfunction f;
      r = driver().moduleGetFunction(&f, m, d.cg.segs[s].name.c_str());
      if (r != CUDA_SUCCESS) return cuda_fail("cuModuleGetFunction", r);
      if (d.cg.smem_bytes > 48 * 1024) {
        r = driver().funcSetAttribute(f, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)d.cg.smem_bytes);
        if (r != CUDA_SUCCESS) return cuda_fail("cuFuncSetAttribute", r);
      }
      fs.push_back(f);
      if (s == 0 && adjoint && d.cg.has_reduce) {
        r = driver().moduleGetFunction(&ds.adj_finish, m, d.cg.finish_kernel.c_str());
        if (r != CUDA_SUCCESS) return cuda_fail("cuModuleGetFunction", r);
      }
    }
  }
  (adjoint ? ds.adj_ready : ds.fwd_ready) = true;
  return CUSADI_OK;
}

cusadi_status device_state(cusadi_fn fn, bool adjoint, DevState** out) {
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return fail(CUSADI_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ce));
  std::lock_guard<std::mutex> lk(fn->dev_mu);
  DevState& ds = fn->dev[dev];
  if (!(adjoint ? ds.adj_ready : ds.fwd_ready)) {
    cusadi_status s = load_on_device(fn, ds, adjoint);
    if (s != CUSADI_OK) return s;
  }
  *out = &ds;
  return CUSADI_OK;
}

size_t elt_io(int dtype) { return dtype == CUSADI_F64 ? 8 : 4; }
size_t elt_ws(int dtype) { return dtype == CUSADI_F32 ? 4 : 8; }
int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

int64_t interp_ldw(int64_t N) { return round_up(std::max<int64_t>(N, 1), 128); }

size_t direction_ws(cusadi_fn fn, const Direction& d, int64_t N) {
  if (N <= 0) return 0;
  if (fn->path == CUSADI_PATH_INTERP)   // global work slots (if any), then reduced-row terms
    return ((size_t)d.ip.n_global * interp_ldw(N) +
            d.ip.reduce_rows.size() * (size_t)round_up(N, 32)) * elt_ws(fn->opt.dtype);
  // rows carried between kernels, then (adjoint) one row of per-instance terms per reduced row
  return ((size_t)d.cg.ws_rows + d.cg.reduce_rows.size()) * round_up(N, 32) * elt_ws(fn->opt.dtype);
}

bool all_bcast(const Graph& g, int64_t rows) {
  for (int64_t r = 0; r < rows; ++r)
    if (r >= (int64_t)g.in_bcast.size() || !g.in_bcast[r]) return false;
  return true;
}

// ldw > 0: the workspace's leading dimension when W points into a larger
// workspace (a chunk of a bigger batch); otherwise the one for N instances.
cusadi_status run(cusadi_fn fn, Direction& d, DevState& ds, bool adjoint, const void* X,
                  int64_t ldx, const void* X2, int64_t ldx2, void* Y, int64_t ldy, int64_t N,
                  void* W, int acc, int reduce, cusadi_stream stream, int64_t ldw = 0) {
  if (fn->path == CUSADI_PATH_INTERP) {
    const int64_t lw = ldw > 0 ? ldw : interp_ldw(N);
    void* Wr = (W && !d.ip.reduce_rows.empty())
                   ? (void*)((char*)W + (size_t)d.ip.n_global * lw *
                                            elt_ws(fn->opt.dtype))
                   : nullptr;
    int rc = launch_interp((const IOp*)(adjoint ? ds.d_ops_adj : ds.d_ops_fwd),
                           (int64_t)d.ip.ops.size(), adjoint ? ds.d_k_adj : ds.d_k_fwd,
                           fn->opt.dtype, X, ldx, X2 ? X2 : X, ldx2, adjoint ? fn->ir.nnz_in : (int64_t)1 << 40,
                           Y, ldy, N, W, lw, d.ip.n_shared, acc, reduce, Wr, round_up(N, 32), stream);
    if (rc != 0) return fail(CUSADI_E_CUDA, std::string("interpreter launch: ") + cudaGetErrorString((cudaError_t)rc));
    return CUSADI_OK;
  }
  const std::vector<CUfunction>& fs = adjoint ? ds.adj : ds.fwd;
  // small batches: shrink the CTA (in warps) until every SM gets one, since a
  // straight-line kernel's throughput per SM does not depend on how many CTAs
  // share it but idle SMs are lost (N = 4096 at 128 threads fills 32 of 152)
  const int64_t NL = std::max(1, d.cg.inst_per_thread);
  const int64_t threads = (N + NL - 1) / NL;
  unsigned block = (unsigned)fn->opt.block;
  if (fn->opt.sync_every <= 0)
    while (block > 32 && ds.sms > 0 && (threads + block - 1) / block < ds.sms) block = (block / 2 + 31) / 32 * 32;
  unsigned grid = (unsigned)((threads + block - 1) / block);
  unsigned smem = (unsigned)d.cg.smem_bytes;   // register-budget spill slots (sized for opt.block)
  if (d.cg.coop_ways > 0) {   // W warps per group of 32 instances, G groups per CTA
    const int G = std::max(1, d.cg.coop_groups);
    block = 32u * (unsigned)d.cg.coop_ways * (unsigned)G;
    grid = (unsigned)((N + 32 * G - 1) / (32 * G));
    smem = (unsigned)d.cg.smem_bytes;
  }
  // whole-vector accesses of NL consecutive instances: every buffer a vector
  // touches starts on a multiple of the vector and its rows are a whole number
  // of vectors apart
  int vec = 0;
  if (NL > 1) {
    const size_t elt = elt_io(fn->opt.dtype);
    const size_t a = std::min<size_t>(16, (size_t)NL * elt);
    auto ok = [&](const void* p, int64_t ld) {
      return p == nullptr || ((uintptr_t)p % a == 0 && ((size_t)ld * elt) % a == 0);
    };
    vec = ok(X, ldx) && ok(X2, ldx2) && ok(Y, ldy) ? 1 : 0;
  }
  long long lx = ldx, lx2 = ldx2, ly = ldy, n = N, lw = ldw > 0 ? ldw : round_up(N, 32);
  const void* x2 = X2 ? X2 : X;
  for (size_t s = 0; s < fs.size(); ++s) {
    void* args[] = {(void*)&X, &lx, (void*)&x2, &lx2, &Y, &ly, &n, &W, &lw, &acc, &reduce, &vec};
    CUresult r = driver().launchKernel(fs[s], grid, 1, 1, block, 1, 1, smem, (CUstream)stream, args, nullptr);
    if (r != CUDA_SUCCESS) return cuda_fail("cuLaunchKernel", r);
  }
  return CUSADI_OK;
}

}  // namespace

namespace cusadi {

cusadi_status report(cusadi_status s, const std::string& msg) { return fail(s, msg); }

// Forward evaluation with a caller-supplied scratch region used as the
// workspace.  Loads nothing: the function's kernels must already be on the
// current device.  Used by the allocation-free entry point.
cusadi_status eval_in_scratch(cusadi_fn fn, const void* in, int64_t ld_in, void* out,
                              int64_t ld_out, int64_t N, void* scratch, size_t scratch_bytes,
                              cusadi_stream stream) {
  if (!fn) return fail(CUSADI_E_INVALID_ARG, "fn is NULL");
  if (N < 0) return fail(CUSADI_E_INVALID_ARG, "N must be >= 0");
  if (N == 0 || fn->ir.nnz_out == 0) return CUSADI_OK;
  if (N > ((int64_t)1 << 40)) return fail(CUSADI_E_INVALID_ARG, "N too large");
  if (fn->ir.nnz_in > 0) {
    if (!in) return fail(CUSADI_E_INVALID_ARG, "in is NULL");
    int64_t need = all_bcast(fn->fwd.g, fn->ir.nnz_in) ? 1 : N;
    if (ld_in < need) return fail(CUSADI_E_INVALID_ARG, "ld_in smaller than N");
  }
  if (!out) return fail(CUSADI_E_INVALID_ARG, "out is NULL");
  if (ld_out < N) return fail(CUSADI_E_INVALID_ARG, "ld_out smaller than N");
  const size_t need = direction_ws(fn, fn->fwd, N);
  if (need > scratch_bytes)
    return fail(CUSADI_E_INVALID_ARG,
                "this evaluation needs " + std::to_string(need) + " bytes of scratch; the static "
                "scratch region holds " + std::to_string(scratch_bytes) +
                " bytes (evaluate fewer instances per call)");
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return fail(CUSADI_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ce));
  DevState* ds = nullptr;
  {
    std::lock_guard<std::mutex> lk(fn->dev_mu);
    auto it = fn->dev.find(dev);
    if (it != fn->dev.end() && it->second.fwd_ready) ds = &it->second;
  }
  if (!ds)
    return fail(CUSADI_E_INVALID_ARG,
                "the function's kernels are not loaded on this device yet: call cusadi_eval "
                "once on it first (loading them allocates device memory)");
  return run(fn, fn->fwd, *ds, false, in, ld_in, nullptr, 0, out, ld_out, N,
             need > 0 ? scratch : nullptr, 0, 0, stream);
}

}  // namespace cusadi

extern "C" {

void cusadi_default_options(cusadi_options* o) {
  if (!o) return;
  o->dtype = CUSADI_F64;
  o->path = CUSADI_PATH_AUTO;
  o->compile_limit_ops = 300000;
  o->segment_ops = 40000;
  o->block = 128;
  o->maxrregcount = 0;
  o->fmad = 1;
  o->compile_threads = 0;
  o->schedule = 1;
  o->inline_math = 0;
  o->adjoint = 0;
  o->own_math = 0;
  o->ways = 0;
  o->debug_checks = 0;
  o->inst_per_thread = 1;
  o->coop_groups = 1;
  o->sync_every = 0;
  o->interp_shared_kb = 48;
  o->spill_values = 0;
  o->spill_shared_kb = 96;
  o->pair_calls = 0;
  o->cache_dir = nullptr;
}

const char* cusadi_status_string(cusadi_status s) {
  switch (s) {
    case CUSADI_OK: return "ok";
    case CUSADI_E_INVALID_ARG: return "invalid argument";
    case CUSADI_E_INVALID_IR: return "invalid program";
    case CUSADI_E_COMPILE: return "compilation failed";
    case CUSADI_E_CUDA: return "CUDA error";
    case CUSADI_E_OOM: return "out of host memory";
    case CUSADI_E_TIMEOUT: return "timeout";
    case CUSADI_E_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* cusadi_last_error(void) { return t_last_error.c_str(); }

cusadi_status cusadi_load(const void* ir, size_t nbytes, const cusadi_options* opt,
                          cusadi_fn* out) {
  if (!out) return fail(CUSADI_E_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!ir || nbytes == 0) return fail(CUSADI_E_INVALID_ARG, "empty program");
  std::unique_ptr<cusadi_fn_s> fn;
  try {
    fn.reset(new cusadi_fn_s);
  } catch (...) {
    return fail(CUSADI_E_OOM, "allocation failed");
  }
  cusadi_default_options(&fn->opt);
  if (opt) fn->opt = *opt;
  cusadi_options& o = fn->opt;
  if (o.dtype < 0 || o.dtype > 2) return fail(CUSADI_E_INVALID_ARG, "dtype must be F64, F32 or MIXED");
  if (o.path < 0 || o.path > 2) return fail(CUSADI_E_INVALID_ARG, "unknown path");
  if (o.block <= 0) o.block = 128;
  if (o.block % 32 != 0 || o.block > 1024) return fail(CUSADI_E_INVALID_ARG, "block must be a multiple of 32 in [32, 1024]");
  if (o.maxrregcount < 0 || o.maxrregcount > 255) return fail(CUSADI_E_INVALID_ARG, "maxrregcount must be in [0, 255]");
  if (o.compile_limit_ops <= 0) o.compile_limit_ops = 300000;
  if (o.ways < 0 || o.ways > 16 || o.ways == 1) return fail(CUSADI_E_INVALID_ARG, "ways must be 0 or 2..16");
  if (o.own_math < 0 || o.own_math > 2) return fail(CUSADI_E_INVALID_ARG, "own_math must be 0, 1 or 2");
  if (o.inline_math < 0 || o.inline_math > 2) return fail(CUSADI_E_INVALID_ARG, "inline_math must be 0, 1 or 2");
  if (o.inst_per_thread <= 0) o.inst_per_thread = 1;
  if (o.inst_per_thread != 1 && o.inst_per_thread != 2 && o.inst_per_thread != 4)
    return fail(CUSADI_E_INVALID_ARG, "inst_per_thread must be 1, 2 or 4");
  if (o.coop_groups <= 0) o.coop_groups = 1;
  if (o.coop_groups > 8) return fail(CUSADI_E_INVALID_ARG, "coop_groups must be in 1..8");
  if (o.ways > 1 && 32 * o.ways * o.coop_groups > 1024)
    return fail(CUSADI_E_INVALID_ARG, "32 * ways * coop_groups must not exceed 1024 threads");
  if (o.sync_every < 0) return fail(CUSADI_E_INVALID_ARG, "sync_every must be >= 0");
  if (o.interp_shared_kb < 0 || o.interp_shared_kb > 200)
    return fail(CUSADI_E_INVALID_ARG, "interp_shared_kb must be in [0, 200]");
  if (o.spill_values < 0) return fail(CUSADI_E_INVALID_ARG, "spill_values must be >= 0");
  if (o.pair_calls < 0) return fail(CUSADI_E_INVALID_ARG, "pair_calls must be >= 0");
  if (o.spill_shared_kb < 0 || o.spill_shared_kb > 200)
    return fail(CUSADI_E_INVALID_ARG, "spill_shared_kb must be in [0, 200]");
  if (o.cache_dir) fn->cache_dir = o.cache_dir;
  o.cache_dir = nullptr;  // the caller's string is not kept
  auto t0 = std::chrono::steady_clock::now();
  try {
    std::string err;
    if (!parse_ir((const uint8_t*)ir, nbytes, fn->ir, err)) return fail(CUSADI_E_INVALID_IR, err);
    fn->fwd.g = build_ssa(fn->ir);
    // decide the path on the simplified size
    Graph probe = fn->fwd.g;
    simplify(probe, o.dtype);
    int64_t ops = count_ops(probe);
    if (o.path == CUSADI_PATH_INTERP || (o.path == CUSADI_PATH_AUTO && ops > o.compile_limit_ops))
      fn->path = CUSADI_PATH_INTERP;
    else
      fn->path = CUSADI_PATH_COMPILED;
    cusadi_status s = prepare_direction(fn.get(), fn->fwd, false);
    if (s != CUSADI_OK) return s;
    fn->compile_seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (o.adjoint) {
      s = ensure_adjoint(fn.get());
      if (s != CUSADI_OK) return s;
    }
  } catch (const std::bad_alloc&) {
    return fail(CUSADI_E_OOM, "out of host memory during load");
  }
  *out = fn.release();
  return CUSADI_OK;
}

void cusadi_free(cusadi_fn fn) {
  if (!fn) return;
  for (auto& kv : fn->dev) {
    DevState& ds = kv.second;
    if (cudaSetDevice(kv.first) == cudaSuccess) {
      for (CUmodule m : ds.mods) if (driver().ok) driver().moduleUnload(m);
      if (ds.d_ops_fwd) cudaFree(ds.d_ops_fwd);
      if (ds.d_k_fwd) cudaFree(ds.d_k_fwd);
      if (ds.d_ops_adj) cudaFree(ds.d_ops_adj);
      if (ds.d_k_adj) cudaFree(ds.d_k_adj);
      if (ds.d_reduce_rows) cudaFree(ds.d_reduce_rows);
      if (ds.h_in) cudaStreamDestroy(ds.h_in);
      if (ds.h_out) cudaStreamDestroy(ds.h_out);
      for (cudaStream_t st : ds.h_comp) cudaStreamDestroy(st);
      for (auto& m : ds.dense_map) cudaFree(m.second);
      for (cudaEvent_t e : ds.hev) cudaEventDestroy(e);
    }
  }
  delete fn;
}

cusadi_status cusadi_info(cusadi_fn fn, cusadi_fn_info* o) {
  if (!fn || !o) return fail(CUSADI_E_INVALID_ARG, "NULL argument");
  std::memset(o, 0, sizeof *o);
  o->n_in = (int32_t)fn->ir.in.size();
  o->n_out = (int32_t)fn->ir.out.size();
  o->nnz_in = fn->ir.nnz_in;
  o->nnz_out = fn->ir.nnz_out;
  o->n_instr = (int64_t)fn->ir.code.size();
  o->n_work = fn->ir.n_work;
  o->n_ops_ir = fn->ir.n_ops;
  o->n_ops = fn->fwd.n_ops;
  o->n_slots = fn->fwd.n_slots;
  o->path = fn->path;
  o->n_segments = fn->path == CUSADI_PATH_COMPILED ? (int32_t)fn->fwd.cg.segs.size() : 0;
  o->dtype = fn->opt.dtype;
  int32_t nb = 0;
  for (uint8_t b : fn->fwd.g.in_bcast) nb += b;
  o->n_bcast_in = nb;
  o->compile_seconds = fn->compile_seconds;
  return CUSADI_OK;
}

cusadi_status cusadi_arg_info(cusadi_fn fn, int is_output, int index, cusadi_arg* out) {
  if (!fn || !out) return fail(CUSADI_E_INVALID_ARG, "NULL argument");
  const std::vector<Arg>& v = is_output ? fn->ir.out : fn->ir.in;
  if (index < 0 || index >= (int)v.size()) return fail(CUSADI_E_INVALID_ARG, "argument index out of range");
  const Arg& a = v[index];
  out->nrow = a.nrow;
  out->ncol = a.ncol;
  out->nnz = a.nnz;
  out->flags = a.flags;
  out->row_offset = a.offset;
  out->rowptr = a.rowptr.data();
  out->col = a.col.data();
  out->name = a.name.c_str();
  return CUSADI_OK;
}

cusadi_status cusadi_op_counts(cusadi_fn fn, int which, int64_t* counts, int n) {
  if (!fn || !counts || n < 0) return fail(CUSADI_E_INVALID_ARG, "NULL argument");
  if (which < 0 || which > 3) return fail(CUSADI_E_INVALID_ARG, "which must be 0..3");
  const bool adjoint = (which & 1) != 0, f64_only = (which & 2) != 0;
  if (adjoint) {
    cusadi_status s = ensure_adjoint(fn);
    if (s != CUSADI_OK) return s;
  }
  const Direction& d = adjoint ? fn->adj : fn->fwd;
  const std::vector<int64_t>& h = f64_only ? d.hist_f64 : d.hist;
  for (int i = 0; i < n; ++i) counts[i] = i < (int)h.size() ? h[i] : 0;
  return CUSADI_OK;
}

size_t cusadi_workspace_bytes(cusadi_fn fn, int64_t N, int adjoint) {
  if (!fn || N <= 0) return 0;
  if (adjoint) {
    if (ensure_adjoint(fn) != CUSADI_OK) return 0;
    return direction_ws(fn, fn->adj, N);
  }
  return direction_ws(fn, fn->fwd, N);
}

cusadi_status cusadi_eval(cusadi_fn fn, const void* in, int64_t ld_in, void* out, int64_t ld_out,
                          int64_t N, void* workspace, cusadi_stream stream) {
  if (!fn) return fail(CUSADI_E_INVALID_ARG, "fn is NULL");
  if (N < 0) return fail(CUSADI_E_INVALID_ARG, "N must be >= 0");
  if (N == 0) return CUSADI_OK;
  if (N > ((int64_t)1 << 40)) return fail(CUSADI_E_INVALID_ARG, "N too large");
  if (fn->ir.nnz_in > 0) {
    if (!in) return fail(CUSADI_E_INVALID_ARG, "in is NULL");
    int64_t need = all_bcast(fn->fwd.g, fn->ir.nnz_in) ? 1 : N;
    if (ld_in < need) return fail(CUSADI_E_INVALID_ARG, "ld_in smaller than N");
  }
  if (fn->ir.nnz_out > 0) {
    if (!out) return fail(CUSADI_E_INVALID_ARG, "out is NULL");
    if (ld_out < N) return fail(CUSADI_E_INVALID_ARG, "ld_out smaller than N");
  } else {
    return CUSADI_OK;
  }
  if (direction_ws(fn, fn->fwd, N) > 0 && !workspace)
    return fail(CUSADI_E_INVALID_ARG, "this function needs a workspace (cusadi_workspace_bytes)");
  DevState* ds;
  cusadi_status s = device_state(fn, false, &ds);
  if (s != CUSADI_OK) return s;
  return run(fn, fn->fwd, *ds, false, in, ld_in, nullptr, 0, out, ld_out, N, workspace, 0, 0, stream);
}

cusadi_status cusadi_debug_count(cusadi_fn fn, uint64_t* count) {
  if (!fn || !count) return fail(CUSADI_E_INVALID_ARG, "NULL argument");
  *count = 0;
  if (!fn->opt.debug_checks) return fail(CUSADI_E_INVALID_ARG, "function loaded without debug_checks");
  if (fn->path == CUSADI_PATH_INTERP)
    return fail(CUSADI_E_UNSUPPORTED, "debug checks exist on the compiled path only");
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return cuda_fail("cudaGetDevice", ce);
  std::lock_guard<std::mutex> lk(fn->dev_mu);
  auto it = fn->dev.find(dev);
  if (it == fn->dev.end()) return CUSADI_OK;          // never evaluated here
  if ((ce = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail("cudaDeviceSynchronize", ce);
  for (CUmodule m : it->second.mods) {
    CUdeviceptr p = 0;
    size_t bytes = 0;
    if (driver().moduleGetGlobal(&p, &bytes, m, "cs_dbg") != CUDA_SUCCESS || bytes != sizeof(unsigned)) continue;
    unsigned v = 0;
    if ((ce = cudaMemcpy(&v, (const void*)p, sizeof v, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail("cudaMemcpy", ce);
    if ((ce = cudaMemset((void*)p, 0, sizeof v)) != cudaSuccess) return cuda_fail("cudaMemset", ce);
    *count += v;
  }
  return CUSADI_OK;
}

cusadi_status cusadi_densify(cusadi_fn fn, int arg, const void* y, int64_t ld_y, void* dense,
                             int64_t ld_d, int64_t N, cusadi_stream stream) {
  if (!fn) return fail(CUSADI_E_INVALID_ARG, "fn is NULL");
  if (arg < 0 || arg >= (int)fn->ir.out.size()) return fail(CUSADI_E_INVALID_ARG, "output index out of range");
  if (N < 0) return fail(CUSADI_E_INVALID_ARG, "N must be >= 0");
  const Arg& a = fn->ir.out[arg];
  const int64_t n_dense = (int64_t)a.nrow * a.ncol;
  if (N == 0 || n_dense == 0) return CUSADI_OK;
  if (!y || !dense) return fail(CUSADI_E_INVALID_ARG, "NULL buffer");
  if (ld_y < N || ld_d < N) return fail(CUSADI_E_INVALID_ARG, "leading dimension smaller than N");
  DevState* ds;
  cusadi_status st = device_state(fn, false, &ds);
  if (st != CUSADI_OK) return st;
  int32_t* map = nullptr;
  {
    std::lock_guard<std::mutex> lk(fn->dev_mu);
    auto it = ds->dense_map.find(arg);
    if (it != ds->dense_map.end()) {
      map = it->second;
    } else {
      std::vector<int32_t> h(n_dense, -1);
      for (int64_t r = 0; r < a.nrow; ++r)
        for (int64_t p = a.rowptr[r]; p < a.rowptr[r + 1]; ++p) h[r * a.ncol + a.col[p]] = (int32_t)p;
      cudaError_t ce = cudaMalloc((void**)&map, h.size() * sizeof(int32_t));
      if (ce != cudaSuccess) return cuda_fail("cudaMalloc", ce);
      if ((ce = cudaMemcpy(map, h.data(), h.size() * sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess) {
        cudaFree(map);
        return cuda_fail("cudaMemcpy", ce);
      }
      ds->dense_map[arg] = map;
    }
  }
  int rc = launch_densify(fn->opt.dtype, y, ld_y, a.offset, map, n_dense, dense, ld_d, N, ds->sms, stream);
  if (rc != 0) return fail(CUSADI_E_CUDA, std::string("densify launch: ") + cudaGetErrorString((cudaError_t)rc));
  return CUSADI_OK;
}

static int32_t host_chunks(int64_t N) {
  // two chunks from 16,384 instances: half the copy time hides behind the
  // other chunk's kernels, and each chunk still fills the GPU (more, smaller
  // concurrent launches were measured to slow some programs down)
  return N >= 16384 ? 2 : 1;
}

cusadi_status cusadi_eval_host(cusadi_fn fn, const void* in_host, int64_t ld_in, void* out_host,
                               int64_t ld_out, int64_t N, void* dev_in, void* dev_out,
                               void* workspace, int32_t chunks, cusadi_stream stream) {
  if (!fn) return fail(CUSADI_E_INVALID_ARG, "fn is NULL");
  if (N < 0) return fail(CUSADI_E_INVALID_ARG, "N must be >= 0");
  if (chunks < 0) return fail(CUSADI_E_INVALID_ARG, "chunks must be >= 0");
  if (N == 0 || fn->ir.nnz_out == 0) return CUSADI_OK;
  if (N > ((int64_t)1 << 40)) return fail(CUSADI_E_INVALID_ARG, "N too large");
  const int64_t nin = fn->ir.nnz_in, nout = fn->ir.nnz_out;
  const Graph& g = fn->fwd.g;
  if (nin > 0) {
    if (!in_host) return fail(CUSADI_E_INVALID_ARG, "in_host is NULL");
    if (!dev_in) return fail(CUSADI_E_INVALID_ARG, "dev_in is NULL");
    int64_t need = all_bcast(g, nin) ? 1 : N;
    if (ld_in < need) return fail(CUSADI_E_INVALID_ARG, "ld_in smaller than N");
  }
  if (!out_host) return fail(CUSADI_E_INVALID_ARG, "out_host is NULL");
  if (!dev_out) return fail(CUSADI_E_INVALID_ARG, "dev_out is NULL");
  if (ld_out < N) return fail(CUSADI_E_INVALID_ARG, "ld_out smaller than N");
  if (direction_ws(fn, fn->fwd, N) > 0 && !workspace)
    return fail(CUSADI_E_INVALID_ARG, "this function needs a workspace (cusadi_workspace_bytes)");
  DevState* ds;
  cusadi_status st = device_state(fn, false, &ds);
  if (st != CUSADI_OK) return st;

  // every chunk's kernels get a stream of their own, so a chunk starts as soon
  // as its inputs are in and its CTAs fill the SMs that the previous chunks'
  // tails leave free.  Each chunk uses its own columns of the workspace (the
  // interpreter writes whole 128-thread blocks of columns, hence its grain).
  const int64_t grain = fn->path == CUSADI_PATH_INTERP ? 128 : 32;
  const int64_t C = std::min<int64_t>(chunks > 0 ? chunks : host_chunks(N), (N + grain - 1) / grain);
  const int64_t chunk = round_up((N + C - 1) / C, grain);
  const int64_t n_chunks = (N + chunk - 1) / chunk;
  const size_t elt = elt_io(fn->opt.dtype);
  const int64_t ldw = fn->path == CUSADI_PATH_INTERP ? interp_ldw(N) : round_up(N, 32);
  std::lock_guard<std::mutex> lk(fn->host_mu);
  cudaError_t ce;
  for (cudaStream_t* h : {&ds->h_in, &ds->h_out})
    if (!*h && (ce = cudaStreamCreateWithFlags(h, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail("cudaStreamCreateWithFlags", ce);
  while (ds->h_comp.size() < (size_t)n_chunks) {
    cudaStream_t h;
    if ((ce = cudaStreamCreateWithFlags(&h, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail("cudaStreamCreateWithFlags", ce);
    ds->h_comp.push_back(h);
  }
  const size_t n_ev = 2 * (size_t)n_chunks + 2;
  while (ds->hev.size() < n_ev) {
    cudaEvent_t e;
    if ((ce = cudaEventCreateWithFlags(&e, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail("cudaEventCreateWithFlags", ce);
    ds->hev.push_back(e);
  }
  cudaStream_t s_in = ds->h_in, s_out = ds->h_out;
  cudaEvent_t ev_start = ds->hev[0], ev_end = ds->hev[1];
  // everything already queued on the caller's stream happens first
  if ((ce = cudaEventRecord(ev_start, (cudaStream_t)stream)) != cudaSuccess) return cuda_fail("cudaEventRecord", ce);
  std::vector<cudaStream_t> all = {s_in, s_out};
  all.insert(all.end(), ds->h_comp.begin(), ds->h_comp.begin() + n_chunks);
  for (cudaStream_t h : all)
    if ((ce = cudaStreamWaitEvent(h, ev_start, 0)) != cudaSuccess) return cuda_fail("cudaStreamWaitEvent", ce);
  const char* hin = (const char*)in_host;
  char* din = (char*)dev_in;
  for (int64_t c = 0; c < n_chunks; ++c) {
    const int64_t s0 = c * chunk, n = std::min(chunk, N - s0);
    cudaEvent_t ev_in = ds->hev[2 + 2 * c], ev_comp = ds->hev[3 + 2 * c];
    // inputs: runs of consecutive rows; a broadcast row's value goes to the
    // chunk's first column, where the kernel (given the chunk's base) reads it
    for (int64_t r0 = 0; r0 < nin;) {
      const bool bc = r0 < (int64_t)g.in_bcast.size() && g.in_bcast[r0];
      int64_t r1 = r0 + 1;
      while (r1 < nin && (r1 < (int64_t)g.in_bcast.size() && g.in_bcast[r1]) == bc) ++r1;
      ce = cudaMemcpy2DAsync(din + ((size_t)r0 * N + s0) * elt, (size_t)N * elt,
                             hin + ((size_t)r0 * ld_in + (bc ? 0 : s0)) * elt, (size_t)ld_in * elt,
                             (bc ? 1 : (size_t)n) * elt, (size_t)(r1 - r0), cudaMemcpyHostToDevice, s_in);
      if (ce != cudaSuccess) return cuda_fail("cudaMemcpy2DAsync (inputs)", ce);
      r0 = r1;
    }
    cudaStream_t s_comp = ds->h_comp[c];
    if ((ce = cudaEventRecord(ev_in, s_in)) != cudaSuccess) return cuda_fail("cudaEventRecord", ce);
    if ((ce = cudaStreamWaitEvent(s_comp, ev_in, 0)) != cudaSuccess) return cuda_fail("cudaStreamWaitEvent", ce);
    void* wc = workspace ? (void*)((char*)workspace + (size_t)s0 * elt_ws(fn->opt.dtype)) : nullptr;
    st = run(fn, fn->fwd, *ds, false, din + (size_t)s0 * elt, N, nullptr, 0,
             (char*)dev_out + (size_t)s0 * elt, N, n, wc, 0, 0, (cusadi_stream)s_comp, ldw);
    if (st != CUSADI_OK) return st;
    if ((ce = cudaEventRecord(ev_comp, s_comp)) != cudaSuccess) return cuda_fail("cudaEventRecord", ce);
    if ((ce = cudaStreamWaitEvent(s_out, ev_comp, 0)) != cudaSuccess) return cuda_fail("cudaStreamWaitEvent", ce);
    ce = cudaMemcpy2DAsync((char*)out_host + (size_t)s0 * elt, (size_t)ld_out * elt,
                           (const char*)dev_out + (size_t)s0 * elt, (size_t)N * elt, (size_t)n * elt,
                           (size_t)nout, cudaMemcpyDeviceToHost, s_out);
    if (ce != cudaSuccess) return cuda_fail("cudaMemcpy2DAsync (outputs)", ce);
  }
  // the copy-out stream has waited for every chunk's kernels, and each of
  // those for its copy-in, so its last event covers the whole evaluation
  if ((ce = cudaEventRecord(ev_end, s_out)) != cudaSuccess) return cuda_fail("cudaEventRecord", ce);
  if ((ce = cudaStreamWaitEvent((cudaStream_t)stream, ev_end, 0)) != cudaSuccess)
    return cuda_fail("cudaStreamWaitEvent", ce);
  return CUSADI_OK;
}

}  // extern "C"

namespace {

// Reverse mode with the broadcast rows' sums written to shared_bar[row] when
// shared_bar is given (else to column 0 of in_bar's broadcast rows).
cusadi_status adjoint_impl(cusadi_fn fn, const void* in, int64_t ld_in, const void* out_bar,
                           int64_t ld_ob, void* in_bar, int64_t ld_ib, void* shared_bar, int64_t N,
                           uint32_t flags, void* workspace, cusadi_stream stream) {
  if (!fn) return fail(CUSADI_E_INVALID_ARG, "fn is NULL");
  if (N < 0) return fail(CUSADI_E_INVALID_ARG, "N must be >= 0");
  if (flags & ~(CUSADI_ADJ_ACCUMULATE | CUSADI_ADJ_REDUCE_BROADCAST | CUSADI_ADJ_ACCUMULATE_BROADCAST))
    return fail(CUSADI_E_INVALID_ARG, "unknown adjoint flags");
  cusadi_status s = ensure_adjoint(fn);
  if (s != CUSADI_OK) return s;
  if (N == 0 || fn->ir.nnz_in == 0) return CUSADI_OK;
  if (!in || !in_bar) return fail(CUSADI_E_INVALID_ARG, "in / in_bar is NULL");
  const bool reduce = (flags & CUSADI_ADJ_REDUCE_BROADCAST) != 0;
  int64_t need = all_bcast(fn->fwd.g, fn->ir.nnz_in) ? 1 : N;
  if (ld_in < need) return fail(CUSADI_E_INVALID_ARG, "ld_in smaller than N");
  if (fn->ir.nnz_out > 0 && (!out_bar || ld_ob < N)) return fail(CUSADI_E_INVALID_ARG, "out_bar missing or ld_ob smaller than N");
  if (ld_ib < (reduce && all_bcast(fn->fwd.g, fn->ir.nnz_in) ? 1 : N)) return fail(CUSADI_E_INVALID_ARG, "ld_ib smaller than N");
  if (direction_ws(fn, fn->adj, N) > 0 && !workspace)
    return fail(CUSADI_E_INVALID_ARG, "this function needs a workspace (cusadi_workspace_bytes)");
  DevState* ds;
  s = device_state(fn, true, &ds);
  if (s != CUSADI_OK) return s;
  const int acc = (flags & CUSADI_ADJ_ACCUMULATE) ? 1 : 0;
  const bool has_reduce = fn->path == CUSADI_PATH_INTERP ? fn->adj.ip.has_reduce : fn->adj.cg.has_reduce;
  const bool acc_bcast = acc || (flags & CUSADI_ADJ_ACCUMULATE_BROADCAST);
  // destination of the broadcast rows' sums: element `row` of shared_bar, or
  // column 0 of row `row` of in_bar
  void* sum_dst = shared_bar ? shared_bar : in_bar;
  const int64_t sum_ld = shared_bar ? 1 : ld_ib;
  s = run(fn, fn->adj, *ds, true, in, ld_in, out_bar, ld_ob, in_bar, ld_ib, N, workspace, acc,
          reduce ? 1 : 0, stream);
  if (s != CUSADI_OK || !reduce || !has_reduce) return s;
  // the kernels left each reduced row's per-instance terms in the workspace;
  // sum them in a fixed order (the same bits on every run)
  if (fn->path == CUSADI_PATH_INTERP) {
    const InterpProgram& ip = fn->adj.ip;
    const size_t off = (size_t)ip.n_global * interp_ldw(N) *
                       elt_ws(fn->opt.dtype);
    int rc = launch_reduce_finish(fn->opt.dtype, (char*)workspace + off, round_up(N, 32), N, ds->d_reduce_rows,
                                  (int64_t)ip.reduce_rows.size(), sum_dst, sum_ld, acc_bcast ? 1 : 0,
                                  stream);
    if (rc != 0) return fail(CUSADI_E_CUDA, std::string("reduction launch: ") + cudaGetErrorString((cudaError_t)rc));
    return CUSADI_OK;
  }
  long long lw = round_up(N, 32), n = N, ly = sum_ld;
  int accumulate = acc_bcast ? 1 : 0;
  void* args[] = {&workspace, &lw, &n, &sum_dst, &ly, &accumulate};
  CUresult r = driver().launchKernel(ds->adj_finish, (unsigned)fn->adj.cg.reduce_rows.size(), 1, 1, 512, 1, 1,
                                     0, (CUstream)stream, args, nullptr);
  if (r != CUDA_SUCCESS) return cuda_fail("cuLaunchKernel", r);
  return CUSADI_OK;
}

}  // namespace

extern "C" {

cusadi_status cusadi_adjoint(cusadi_fn fn, const void* in, int64_t ld_in, const void* out_bar,
                             int64_t ld_ob, void* in_bar, int64_t ld_ib, int64_t N,
                             uint32_t flags, void* workspace, cusadi_stream stream) {
  return adjoint_impl(fn, in, ld_in, out_bar, ld_ob, in_bar, ld_ib, nullptr, N, flags, workspace,
                      stream);
}

cusadi_status cusadi_adjoint_shared(cusadi_fn fn, const void* in, int64_t ld_in, const void* out_bar,
                                    int64_t ld_ob, void* in_bar, int64_t ld_ib, void* shared_bar,
                                    int64_t N, uint32_t flags, void* workspace,
                                    cusadi_stream stream) {
  if (!shared_bar) return fail(CUSADI_E_INVALID_ARG, "shared_bar is NULL");
  if (flags & CUSADI_ADJ_REDUCE_BROADCAST)
    return fail(CUSADI_E_INVALID_ARG, "cusadi_adjoint_shared always reduces: do not pass "
                                      "CUSADI_ADJ_REDUCE_BROADCAST");
  return adjoint_impl(fn, in, ld_in, out_bar, ld_ob, in_bar, ld_ib, shared_bar, N,
                      flags | CUSADI_ADJ_REDUCE_BROADCAST, workspace, stream);
}

cusadi_status cusadi_sum_instances(int32_t dtype, const void* y, int64_t ld_y, int64_t rows,
                                   int64_t N, void* sums, int32_t accumulate, cusadi_stream stream) {
  if (dtype < CUSADI_F64 || dtype > CUSADI_MIXED) return fail(CUSADI_E_INVALID_ARG, "unknown dtype");
  if (rows < 0 || N < 0) return fail(CUSADI_E_INVALID_ARG, "rows and N must be >= 0");
  if (rows == 0) return CUSADI_OK;
  if (rows > 65535) return fail(CUSADI_E_INVALID_ARG, "at most 65,535 rows per call");
  if (!sums || (N > 0 && !y)) return fail(CUSADI_E_INVALID_ARG, "y / sums is NULL");
  if (N > 0 && ld_y < N) return fail(CUSADI_E_INVALID_ARG, "ld_y smaller than N");
  int rc = launch_sum_rows(dtype, y, ld_y, rows, N, sums, accumulate ? 1 : 0, stream);
  if (rc != 0) return fail(CUSADI_E_CUDA, std::string("sum launch: ") + cudaGetErrorString((cudaError_t)rc));
  return CUSADI_OK;
}

cusadi_status cusadi_stream_wait(cusadi_stream stream, double timeout_seconds) {
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaStreamQuery((cudaStream_t)stream);
    if (e == cudaSuccess) return CUSADI_OK;
    if (e != cudaErrorNotReady) return fail(CUSADI_E_CUDA, std::string("cudaStreamQuery: ") + cudaGetErrorString(e));
    double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (dt >= timeout_seconds)
      return fail(CUSADI_E_TIMEOUT, "work on the stream still running after " + std::to_string(timeout_seconds) + " s");
    std::this_thread::sleep_for(std::chrono::microseconds(dt < 1e-3 ? 10 : 200));
  }
}

cusadi_status cusadi_source(cusadi_fn fn, int adjoint, int segment, char* buf, size_t* len) {
  if (!fn || !len) return fail(CUSADI_E_INVALID_ARG, "NULL argument");
  if (fn->path != CUSADI_PATH_COMPILED) return fail(CUSADI_E_UNSUPPORTED, "interpreted function has no source");
  if (adjoint) {
    cusadi_status s = ensure_adjoint(fn);
    if (s != CUSADI_OK) return s;
  }
  const Direction& d = adjoint ? fn->adj : fn->fwd;
  if (segment < 0 || segment >= (int)d.cg.segs.size()) return fail(CUSADI_E_INVALID_ARG, "segment out of range");
  const std::string& src = d.cg.segs[segment].source;
  if (buf && *len > 0) {
    size_t n = std::min(*len - 1, src.size());
    std::memcpy(buf, src.data(), n);
    buf[n] = 0;
  }
  *len = src.size() + 1;
  return CUSADI_OK;
}

}  // extern "C"
