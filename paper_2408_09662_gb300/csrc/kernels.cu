// Interpreter kernel: one thread per instance walks a packed instruction
// stream (the sequential traversal of CusADi §III-A), for programs that are too
// large to compile.  Every thread reads the same instruction at the same time,
// so the switch below never diverges within a warp.  The work vector lives in
// shared memory (slot-major, one column per thread: conflict-free) when it
// fits, else in a global workspace in the instance-fastest layout.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <type_traits>

#include "internal.h"

namespace cusadi {
namespace {

constexpr int kInterpBlock = 128;   // threads per CTA of the interpreter kernel

template <typename T>
__device__ __forceinline__ T eval_op(uint32_t op, T a, T b, T k) {
  const T Z = T(0), O = T(1);
  switch (op) {
    case ADD: return a + b;
    case SUB: return a - b;
    case MUL: return a * b;
    case DIV: return a / b;
    case NEG: return -a;
    case EXP: return exp(a);
    case LOG: return log(a);
    case POW: return pow(a, b);
    case SQ: return a * a;
    case SQRT: return sqrt(a);
    case SIN: return sin(a);
    case COS: return cos(a);
    case TAN: return tan(a);
    case ATAN: return atan(a);
    case ATAN2: return atan2(a, b);
    case TANH: return tanh(a);
    case FABS: return fabs(a);
    case FMIN: return fmin(a, b);
    case FMAX: return fmax(a, b);
    case FMA_CONST: return fma(k, a, b);
    case IF_ELSE_ZERO: return a != Z ? b : Z;
    case LT: return a < b ? O : Z;
    case LE: return a <= b ? O : Z;
    case EQ: return a == b ? O : Z;
    case NE: return a != b ? O : Z;
    case NOT: return a == Z ? O : Z;
    case AND: return (a != Z && b != Z) ? O : Z;
    case OR: return (a != Z || b != Z) ? O : Z;
    case ASIN: return asin(a);
    case ACOS: return acos(a);
    case SINH: return sinh(a);
    case COSH: return cosh(a);
    case ERF: return erf(a);
    case SIGN: return a > Z ? O : (a < Z ? -O : Z);
    case FLOOR: return floor(a);
    case CEIL: return ceil(a);
    case FMOD: return fmod(a, b);
    case INV: return O / a;
    case HYPOT: return hypot(a, b);
    case LOG1P: return log1p(a);
    case EXPM1: return expm1(a);
    case COPYSIGN: return copysign(a, b);
    case ASSIGN: return a;
  }
  return Z;
}

// B: buffer element type; S: work-slot type; MIXED: per-op precision tags.
// Slots below n_shared live in shared memory (slot-major, one column per
// thread: conflict-free), the others in the global workspace (row s - n_shared,
// instance-fastest); every slot index in the stream is warp-uniform, so the
// tier test never diverges.
template <typename B, typename S, bool MIXED>
__global__ void __launch_bounds__(kInterpBlock) interp_kernel(
    const uint4* __restrict__ ops, long long n_ops, const double* __restrict__ K,
    const B* __restrict__ X, long long ldx, const B* __restrict__ X2, long long ldx2,
    long long split, B* __restrict__ Y, long long ldy, long long N, S* __restrict__ W,
    long long ldw, unsigned n_shared, int acc, int reduce, S* __restrict__ Wr, long long ldr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = i0 < N;
  const long long ix = active ? i0 : N - 1;  // inactive lanes read a valid column
  S* const sm = reinterpret_cast<S*>(smem_raw) + threadIdx.x;
  S* const gm = W + i0;                      // columns up to the grid's end exist (ldw)
  auto at = [&](unsigned s) -> S& {
    return s < n_shared ? sm[(size_t)s * kInterpBlock] : gm[(long long)(s - n_shared) * ldw];
  };
  for (long long t = 0; t < n_ops; ++t) {
    const uint4 o = __ldg(&ops[t]);
    const uint32_t op = o.x & 127u;
    const long long aux = (long long)(o.x >> 8);
    if (op == INPUT) {
      const long long col = o.w ? 0 : ix;
      at(o.y) = aux < split ? (S)X[aux * ldx + col] : (S)X2[(aux - split) * ldx2 + col];
      continue;
    }
    if (op == CONST) {
      at(o.y) = (S)K[aux];
      continue;
    }
    if (op == OUTPUT) {
      const S v = at(o.z);
      if (o.w && reduce) {   // reduced row o.w - 1: the instance's term, summed later
        if (active) Wr[(long long)(o.w - 1) * ldr + i0] = v;
      } else if (active) {
        B* p = &Y[aux * ldy + i0];
        *p = acc ? *p + (B)v : (B)v;
      }
      continue;
    }
    const S a = at(o.z), b = at(o.w);
    const double kd = op == FMA_CONST ? K[aux] : 0.0;
    S r;
    if (!MIXED || ((o.x >> 7) & 1u)) {
      r = eval_op<S>(op, a, b, (S)kd);
    } else {
      r = (S)eval_op<float>(op, (float)a, (float)b, (float)kd);
    }
    at(o.y) = r;
  }
}

template <typename B, typename S, bool MIXED>
int launch(const IOp* ops, int64_t n_ops, const double* k, const void* X, int64_t ldx,
           const void* X2, int64_t ldx2, int64_t split, void* Y, int64_t ldy, int64_t N, void* W,
           int64_t ldw, int64_t n_shared, int acc, int reduce, void* Wr, int64_t ldr,
           cudaStream_t st) {
  auto kern = interp_kernel<B, S, MIXED>;
  size_t smem = (size_t)n_shared * kInterpBlock * sizeof(S);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
  }
  long long grid = (N + kInterpBlock - 1) / kInterpBlock;
  kern<<<(unsigned)grid, kInterpBlock, smem, st>>>(reinterpret_cast<const uint4*>(ops), n_ops, k,
                                                    (const B*)X, ldx, (const B*)X2, ldx2, split, (B*)Y,
                                                    ldy, N, (S*)W, ldw, (unsigned)n_shared, acc, reduce,
                                                    (S*)Wr, ldr);
  return (int)cudaGetLastError();
}

// One CTA per reduced row: strided per-thread sums, then a tree, always in the
// same order, so the result has the same bits on every run.
template <typename B, typename S>
__global__ void __launch_bounds__(512) reduce_finish_kernel(const S* __restrict__ Wr, long long ldr,
                                                            long long N, const int64_t* __restrict__ rows,
                                                            B* __restrict__ Y, long long ldy, int accumulate) {
  __shared__ S s_[512];
  const S* __restrict__ P = Wr + (long long)blockIdx.x * ldr;
  S a = 0;
  for (long long j = threadIdx.x; j < N; j += 512) a += P[j];
  s_[threadIdx.x] = a;
  __syncthreads();
  for (int d = 256; d > 0; d >>= 1) {
    if ((int)threadIdx.x < d) s_[threadIdx.x] += s_[threadIdx.x + d];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    B* p = &Y[rows[blockIdx.x] * ldy];
    *p = (B)(accumulate ? (S)*p + s_[0] : s_[0]);
  }
}

// One CTA per row of Y: S[r] = sum over j < N of Y[r * ldy + j], in the same
// order as reduce_finish_kernel (strided per-thread sums, then a tree).
template <typename T>
__global__ void __launch_bounds__(512) sum_rows_kernel(const T* __restrict__ Y, long long ldy,
                                                       long long N, T* __restrict__ S,
                                                       int accumulate) {
  __shared__ T s_[512];
  const T* __restrict__ P = Y + (long long)blockIdx.x * ldy;
  T a = 0;
  for (long long j = threadIdx.x; j < N; j += 512) a += P[j];
  s_[threadIdx.x] = a;
  __syncthreads();
  for (int d = 256; d > 0; d >>= 1) {
    if ((int)threadIdx.x < d) s_[threadIdx.x] += s_[threadIdx.x + d];
    __syncthreads();
  }
  if (threadIdx.x == 0) S[blockIdx.x] = accumulate ? S[blockIdx.x] + s_[0] : s_[0];
}

}  // namespace

int interp_shared_slots(int dtype, int shared_kb) {
  const size_t elt = dtype == CUSADI_F32 ? 4 : 8;
  return (int)(((size_t)std::max(0, shared_kb) * 1024) / (kInterpBlock * elt));
}

int launch_interp(const IOp* ops, int64_t n_ops, const double* k, int dtype, const void* X,
                  int64_t ldx, const void* X2, int64_t ldx2, int64_t split, void* Y, int64_t ldy,
                  int64_t N, void* W, int64_t ldw, int64_t n_shared, int acc, int reduce,
                  void* Wr, int64_t ldr, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == CUSADI_F64)
    return launch<double, double, false>(ops, n_ops, k, X, ldx, X2, ldx2, split, Y, ldy, N, W, ldw, n_shared, acc, reduce, Wr, ldr, st);
  if (dtype == CUSADI_F32)
    return launch<float, float, false>(ops, n_ops, k, X, ldx, X2, ldx2, split, Y, ldy, N, W, ldw, n_shared, acc, reduce, Wr, ldr, st);
  return launch<float, double, true>(ops, n_ops, k, X, ldx, X2, ldx2, split, Y, ldy, N, W, ldw, n_shared, acc, reduce, Wr, ldr, st);
}

// Dense copy of one sparse output argument: dense[k * ldd + i] = y[(off +
// map[k]) * ldy + i] where map[k] >= 0 (a structural non-zero), else 0.  k
// runs over the nrow * ncol entries (row-major); the grid covers (k, i) with
// instances fastest so loads and stores are coalesced.
template <typename T>
__global__ void __launch_bounds__(256) densify_kernel(const T* __restrict__ y, int64_t ldy,
                                                      int64_t off, const int32_t* __restrict__ map,
                                                      int64_t n_dense, T* __restrict__ dense,
                                                      int64_t ldd, int64_t N) {
  const int64_t total = n_dense * N;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t / N, i = t - k * N;
    const int32_t src = map[k];
    dense[k * ldd + i] = src >= 0 ? y[(off + src) * ldy + i] : T(0);
  }
}

int launch_densify(int dtype, const void* y, int64_t ldy, int64_t off, const int32_t* map,
                   int64_t n_dense, void* dense, int64_t ldd, int64_t N, int sms, void* stream) {
  const int64_t total = n_dense * N;
  const int64_t blocks = std::min<int64_t>((total + 255) / 256, (int64_t)std::max(sms, 1) * 8);
  if (blocks <= 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == CUSADI_F64)
    densify_kernel<double><<<(unsigned)blocks, 256, 0, st>>>((const double*)y, ldy, off, map, n_dense,
                                                           (double*)dense, ldd, N);
  else
    densify_kernel<float><<<(unsigned)blocks, 256, 0, st>>>((const float*)y, ldy, off, map, n_dense,
                                                          (float*)dense, ldd, N);
  return (int)cudaGetLastError();
}

int launch_reduce_finish(int dtype, const void* Wr, int64_t ldr, int64_t N, const int64_t* rows,
                         int64_t n_rows, void* Y, int64_t ldy, int accumulate, void* stream) {
  if (n_rows <= 0 || N <= 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == CUSADI_F64)
    reduce_finish_kernel<double, double><<<(unsigned)n_rows, 512, 0, st>>>(
        (const double*)Wr, ldr, N, rows, (double*)Y, ldy, accumulate);
  else if (dtype == CUSADI_F32)
    reduce_finish_kernel<float, float><<<(unsigned)n_rows, 512, 0, st>>>(
        (const float*)Wr, ldr, N, rows, (float*)Y, ldy, accumulate);
  else
    reduce_finish_kernel<float, double><<<(unsigned)n_rows, 512, 0, st>>>(
        (const double*)Wr, ldr, N, rows, (float*)Y, ldy, accumulate);
  return (int)cudaGetLastError();
}

int launch_sum_rows(int dtype, const void* Y, int64_t ldy, int64_t rows, int64_t N, void* S,
                    int accumulate, void* stream) {
  if (rows <= 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == CUSADI_F64)
    sum_rows_kernel<double><<<(unsigned)rows, 512, 0, st>>>((const double*)Y, ldy, N, (double*)S,
                                                            accumulate);
  else
    sum_rows_kernel<float><<<(unsigned)rows, 512, 0, st>>>((const float*)Y, ldy, N, (float*)S,
                                                           accumulate);
  return (int)cudaGetLastError();
}

}  // namespace cusadi
