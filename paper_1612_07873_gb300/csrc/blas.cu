// Level-1 vector kernels of the solvers (Sec. 7.1: GCR, MR, setup
// iteration).  Scalars stay on the device: a reduction writes one complex
// double per right-hand side into a row of ctx->scalars and the following
// update kernel reads it, so smoothers and orthogonalisation never wait on
// the host.
// Reductions are two-stage with a grid that depends only on the length,
// so results are bitwise reproducible run to run.
#include <type_traits>

#include "kernels.cuh"

namespace gbmg {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxRedBlocks = 1024;

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Reduction grid: one block per 4096 elements, at most one full wave of
// the reduction kernel (per_sm resident blocks of 256 threads: 4 for the
// kernels of <= 64 registers a thread); a second, partly filled wave would
// leave SMs idle at the end.  The grid depends only on the length and the
// device.
int red_blocks(size_t n, int per_sm = 4) {
  static const int sms = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1)
      return kMaxRedBlocks / 4;
    return v;
  }();
  const int cap = per_sm * sms < kMaxRedBlocks ? per_sm * sms : kMaxRedBlocks;
  long long b = (long long)((n + 4095) / 4096);
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return int(b);
}
int ew_blocks(size_t n) {
  long long b = (long long)((n + kThreads - 1) / kThreads);
  if (b > 152 * 64) b = 152 * 64;
  if (b < 1) b = 1;
  return int(b);
}
// batched element-wise grid: (blocks per vector, vector)
dim3 ew_grid_b(size_t n, int nvec) {
  long long b = (long long)((n + kThreads - 1) / kThreads);
  long long cap = (152 * 64 + nvec - 1) / nvec;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return dim3(unsigned(b), unsigned(nvec));
}

__device__ __forceinline__ double2 block_sum(double2 v, double2* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    v = (l < nw) ? sh[l] : make_double2(0.0, 0.0);
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
  }
  return v;
}

// Per-thread partial sums run in the arithmetic type T: FP32 when both
// operands are FP32 (FP64 issue is scarce on GB300), FP64 otherwise; the
// per-thread partials are combined in FP64.
template <typename Ra, typename Rb>
using acc_t = typename std::conditional<std::is_same<Ra, float>::value &&
                                            std::is_same<Rb, float>::value,
                                        float, double>::type;

// ---- Solver kernels.  Every vector argument holds nr right-hand sides back
// to back (rhs v at offset v * n); blockIdx.y is the right-hand side and
// per-RHS scalars are read from a row S[v] of the scalar table.

// Grid-stride loop over [0, n) that hands each thread's elements to
// body(i, k) round-robin over kAcc independent accumulators k (a fixed
// assignment, so sums stay bitwise reproducible): a single accumulator
// chains every multiply-add on the previous one, and an FP64 chain of that
// kind runs far below GB300's FP64 issue rate.
constexpr int kAcc = 4;
template <typename F>
__device__ __forceinline__ void grid_loop_acc(size_t n, F&& body) {
  const size_t stride = size_t(gridDim.x) * blockDim.x;
  size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x;
  for (; i + (kAcc - 1) * stride < n; i += kAcc * stride) {
#pragma unroll
    for (int k = 0; k < kAcc; ++k) body(i + k * stride, k);
  }
  for (; i < n; i += stride) body(i, 0);
}

// NORM: a == b, only the real part |a|^2 is formed (half the multiply-adds,
// which matters where they are FP64)
template <typename Ra, typename Rb, typename T, bool NORM = false>
__global__ void k_dot_partial(const cpx<Ra>* __restrict__ a, const cpx<Rb>* __restrict__ b,
                              size_t n, double2* __restrict__ part) {
  __shared__ double2 sh[32];
  a += size_t(blockIdx.y) * n;
  b += size_t(blockIdx.y) * n;
  cpx<T> acc[kAcc];
#pragma unroll
  for (int k = 0; k < kAcc; ++k) acc[k] = cpx<T>(T(0), T(0));
  grid_loop_acc(n, [&](size_t i, int k) {
    if constexpr (NORM) {
      const cpx<T> x(a[i]);
      acc[k].re = fma(x.re, x.re, fma(x.im, x.im, acc[k].re));
    } else {
      cmac_conj(acc[k], cpx<T>(a[i]), cpx<T>(b[i]));
    }
  });
  const cpx<T> t = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  double2 d = block_sum(make_double2(double(t.re), double(t.im)), sh);
  if (threadIdx.x == 0) part[size_t(blockIdx.y) * gridDim.x + blockIdx.x] = d;
}

// FP64-accurate inner products of FP32 vectors without the FP64 pipe, whose
// issue rate on GB300 would make them several times slower than reading
// the vectors.  Each product is split exactly, a b = p + e (p rounded,
// e = fma(a, b, -p)); the running sum is an unevaluated pair hi + lo of
// floats (about 48 significant bits), updated with Knuth's TwoSum, which
// returns the rounding error of a float addition exactly, and renormalised
// (Dekker's Fast2Sum) after every element.  The rounding-explicit
// intrinsics keep the compiler from contracting these sums into FMAs, which
// would break the exact error terms.  Per-thread pairs are combined in FP64.
__device__ __forceinline__ void ff_mac(float& hi, float& lo, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  const float s = __fadd_rn(hi, p);
  const float v = __fsub_rn(s, hi);
  const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, v)), __fsub_rn(p, v));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(t, e));
}
__device__ __forceinline__ void ff_renorm(float& hi, float& lo) {
  const float s = __fadd_rn(hi, lo);
  lo = __fsub_rn(lo, __fsub_rn(s, hi));
  hi = s;
}

// W = 1: one complex number per access; W = 2: 16-byte loads of two (the
// vectors 16-byte aligned, n even)
template <bool NORM, int W>
__global__ void k_dot_partial_ff(const cpx<float>* __restrict__ a, const cpx<float>* __restrict__ b,
                                 size_t n, double2* __restrict__ part) {
  __shared__ double2 sh[32];
  a += size_t(blockIdx.y) * n;
  b += size_t(blockIdx.y) * n;
  float rh[kAcc], rl[kAcc], ih[kAcc], il[kAcc];
#pragma unroll
  for (int k = 0; k < kAcc; ++k) rh[k] = rl[k] = ih[k] = il[k] = 0.f;
  auto term = [&](cpx<float> x, cpx<float> y, int k) {
    if constexpr (NORM) {
      ff_mac(rh[k], rl[k], x.re, x.re);
      ff_mac(rh[k], rl[k], x.im, x.im);
    } else {
      ff_mac(rh[k], rl[k], x.re, y.re);  // conj(x) y
      ff_mac(rh[k], rl[k], x.im, y.im);
      ff_mac(ih[k], il[k], x.re, y.im);
      ff_mac(ih[k], il[k], -x.im, y.re);
      ff_renorm(ih[k], il[k]);
    }
    ff_renorm(rh[k], rl[k]);
  };
  if constexpr (W == 2) {
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const float4* b4 = reinterpret_cast<const float4*>(b);
    grid_loop_acc(n / 2, [&](size_t i, int k) {
      const float4 x = a4[i];
      const float4 y = NORM ? x : b4[i];
      term(cpx<float>(x.x, x.y), cpx<float>(y.x, y.y), k);
      term(cpx<float>(x.z, x.w), cpx<float>(y.z, y.w), k);
    });
  } else {
    grid_loop_acc(n, [&](size_t i, int k) { term(a[i], NORM ? a[i] : b[i], k); });
  }
  double re = 0.0, im = 0.0;
#pragma unroll
  for (int k = 0; k < kAcc; ++k) {
    re += double(rh[k]) + double(rl[k]);
    im += double(ih[k]) + double(il[k]);
  }
  double2 d = block_sum(make_double2(re, im), sh);
  if (threadIdx.x == 0) part[size_t(blockIdx.y) * gridDim.x + blockIdx.x] = d;
}

// ---- block Gram-Schmidt: m <= kCgs vectors X[j] (nr right-hand sides each,
// back to back) against y in one pass.
struct VecList {
  const void* p[kCgs];
};

// partial <X[j], y> per block at part[(v m + j) * gridDim.x + block].  FF:
// float-float sums of exact products (FP32 operands, FP64-accurate);
// otherwise sums in acc_t<R, R>.  Each j is its own accumulation chain.
template <typename R, bool FF>
__global__ void __launch_bounds__(256, 2) k_dot_multi(VecList X, const cpx<R>* __restrict__ y, int m, size_t n,
                            double2* __restrict__ part) {
  using T = acc_t<R, R>;
  __shared__ double2 sh[32];
  const int v = blockIdx.y;
  const size_t off = size_t(v) * n;
  y += off;
  cpx<T> acc[kCgs];
  float rh[kCgs], rl[kCgs], ih[kCgs], il[kCgs];
#pragma unroll
  for (int j = 0; j < kCgs; ++j) {
    acc[j] = cpx<T>(T(0), T(0));
    rh[j] = rl[j] = ih[j] = il[j] = 0.f;
  }
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    const cpx<R> yi = y[i];
#pragma unroll
    for (int j = 0; j < kCgs; ++j)
      if (j < m) {
        const cpx<R> xj = static_cast<const cpx<R>*>(X.p[j])[off + i];
        if constexpr (FF) {
          ff_mac(rh[j], rl[j], xj.re, yi.re);  // conj(x) y
          ff_mac(rh[j], rl[j], xj.im, yi.im);
          ff_mac(ih[j], il[j], xj.re, yi.im);
          ff_mac(ih[j], il[j], -xj.im, yi.re);
          ff_renorm(rh[j], rl[j]);
          ff_renorm(ih[j], il[j]);
        } else {
          cmac_conj(acc[j], cpx<T>(xj), cpx<T>(yi));
        }
      }
  }
#pragma unroll
  for (int j = 0; j < kCgs; ++j)
    if (j < m) {  // m is uniform: every thread takes the same branches
      double2 d;
      if constexpr (FF)
        d = make_double2(double(rh[j]) + double(rl[j]), double(ih[j]) + double(il[j]));
      else
        d = make_double2(double(acc[j].re), double(acc[j].im));
      d = block_sum(d, sh);
      if (threadIdx.x == 0) part[(size_t(v) * m + j) * gridDim.x + blockIdx.x] = d;
      __syncthreads();
    }
}

// The float-float form of k_dot_multi for a compile-time count M of
// vectors, 16-byte loads of two complex numbers (16-byte aligned vectors, n
// even): registers grow with M only, so small blocks keep many warps and
// loads in flight.
template <int M>
__global__ void __launch_bounds__(256) k_dot_multi_ff(VecList X, const cpx<float>* __restrict__ y,
                                                      size_t n, double2* __restrict__ part) {
  __shared__ double2 sh[32];
  const int v = blockIdx.y;
  const size_t off2 = size_t(v) * (n / 2);
  const float4* y4 = reinterpret_cast<const float4*>(y) + off2;
  float rh[M], rl[M], ih[M], il[M];
#pragma unroll
  for (int j = 0; j < M; ++j) rh[j] = rl[j] = ih[j] = il[j] = 0.f;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n / 2;
       i += size_t(gridDim.x) * blockDim.x) {
    const float4 yv = y4[i];
    float4 xv[M];
#pragma unroll
    for (int j = 0; j < M; ++j) xv[j] = (reinterpret_cast<const float4*>(X.p[j]) + off2)[i];
#pragma unroll
    for (int j = 0; j < M; ++j) {
      ff_mac(rh[j], rl[j], xv[j].x, yv.x);  // conj(x) y, first complex number
      ff_mac(rh[j], rl[j], xv[j].y, yv.y);
      ff_mac(ih[j], il[j], xv[j].x, yv.y);
      ff_mac(ih[j], il[j], -xv[j].y, yv.x);
      ff_mac(rh[j], rl[j], xv[j].z, yv.z);  // second
      ff_mac(rh[j], rl[j], xv[j].w, yv.w);
      ff_mac(ih[j], il[j], xv[j].z, yv.w);
      ff_mac(ih[j], il[j], -xv[j].w, yv.z);
      ff_renorm(rh[j], rl[j]);
      ff_renorm(ih[j], il[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < M; ++j) {
    double2 d = make_double2(double(rh[j]) + double(rl[j]), double(ih[j]) + double(il[j]));
    d = block_sum(d, sh);
    if (threadIdx.x == 0) part[(size_t(v) * M + j) * gridDim.x + blockIdx.x] = d;
    __syncthreads();
  }
}

// row r = v m + j of the partials -> S[j][v] (slot stride kMaxNrhs)
__global__ void k_reduce_final_multi(const double2* __restrict__ part, int nparts, int m,
                                     double2* __restrict__ S) {
  __shared__ double2 sh[32];
  const double2* src = part + size_t(blockIdx.x) * nparts;
  double2 acc = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    acc.x += src[i].x;
    acc.y += src[i].y;
  }
  acc = block_sum(acc, sh);
  const int v = blockIdx.x / m, j = blockIdx.x - v * m;
  if (threadIdx.x == 0) S[size_t(j) * kMaxNrhs + v] = acc;
}

// y += sign sum_j S[j][v] X[j]
template <typename R>
__global__ void k_axpy_multi(cpx<R>* __restrict__ y, VecList X, int m, size_t n,
                             const double2* __restrict__ S, double sign) {
  using T = acc_t<R, R>;
  const int v = blockIdx.y;
  const size_t off = size_t(v) * n;
  cpx<T> a[kCgs];
#pragma unroll
  for (int j = 0; j < kCgs; ++j) {
    const double2 s = j < m ? S[size_t(j) * kMaxNrhs + v] : make_double2(0.0, 0.0);
    a[j] = cpx<T>(T(sign * s.x), T(sign * s.y));
  }
  y += off;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    cpx<T> yy(y[i]);
#pragma unroll
    for (int j = 0; j < kCgs; ++j)
      if (j < m) cmac(yy, a[j], cpx<T>(static_cast<const cpx<R>*>(X.p[j])[off + i]));
    y[i] = cpx<R>(yy);
  }
}

// k_axpy_multi for FP32 vectors with a compile-time count M, 16-byte loads
// of two complex numbers (16-byte aligned vectors, n even)
template <int M>
__global__ void __launch_bounds__(256) k_axpy_multi_w2(cpx<float>* __restrict__ y, VecList X,
                                                       size_t n, const double2* __restrict__ S,
                                                       double sign) {
  const int v = blockIdx.y;
  const size_t off2 = size_t(v) * (n / 2);
  float ar[M], ai[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const double2 s = S[size_t(j) * kMaxNrhs + v];
    ar[j] = float(sign * s.x);
    ai[j] = float(sign * s.y);
  }
  float4* y4 = reinterpret_cast<float4*>(y) + off2;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n / 2;
       i += size_t(gridDim.x) * blockDim.x) {
    float4 yy = y4[i];
    float4 xv[M];
#pragma unroll
    for (int j = 0; j < M; ++j) xv[j] = (reinterpret_cast<const float4*>(X.p[j]) + off2)[i];
#pragma unroll
    for (int j = 0; j < M; ++j) {  // yy += a_j x_j, two complex numbers
      yy.x = fmaf(ar[j], xv[j].x, fmaf(-ai[j], xv[j].y, yy.x));
      yy.y = fmaf(ar[j], xv[j].y, fmaf(ai[j], xv[j].x, yy.y));
      yy.z = fmaf(ar[j], xv[j].z, fmaf(-ai[j], xv[j].w, yy.z));
      yy.w = fmaf(ar[j], xv[j].w, fmaf(ai[j], xv[j].z, yy.w));
    }
    y4[i] = yy;
  }
}

// <p, r> and |p|^2 in one pass; partials at part[(2 v + k) * gridDim.x + block]
template <typename Ra, typename Rb>
__global__ void k_dot2_partial_b(const cpx<Ra>* __restrict__ p, const cpx<Rb>* __restrict__ r,
                                 size_t n, double2* __restrict__ part) {
  using T = acc_t<Ra, Rb>;
  __shared__ double2 sh[32];
  p += blockIdx.y * n;
  r += blockIdx.y * n;
  cpx<T> pr_k[kAcc];
  T pp_k[kAcc];
#pragma unroll
  for (int k = 0; k < kAcc; ++k) {
    pr_k[k] = cpx<T>(T(0), T(0));
    pp_k[k] = T(0);
  }
  grid_loop_acc(n, [&](size_t i, int k) {
    cpx<T> x(p[i]), y(r[i]);
    cmac_conj(pr_k[k], x, y);
    pp_k[k] = fma(x.re, x.re, fma(x.im, x.im, pp_k[k]));
  });
  const cpx<T> a_pr = (pr_k[0] + pr_k[1]) + (pr_k[2] + pr_k[3]);
  const T a_pp = (pp_k[0] + pp_k[1]) + (pp_k[2] + pp_k[3]);
  double2 pr = block_sum(make_double2(double(a_pr.re), double(a_pr.im)), sh);
  __syncthreads();
  double2 pp = block_sum(make_double2(double(a_pp), 0.0), sh);
  if (threadIdx.x == 0) {
    const size_t base = size_t(blockIdx.y) * 2 * gridDim.x;
    part[base + blockIdx.x] = pr;
    part[base + gridDim.x + blockIdx.x] = pp;
  }
}

// out[b] = sum of the nparts partials of row b (one block per row)
__global__ void k_reduce_final_b(const double2* __restrict__ part, int nparts,
                                 double2* __restrict__ out) {
  __shared__ double2 sh[32];
  const double2* src = part + size_t(blockIdx.x) * nparts;
  double2 acc = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    acc.x += src[i].x;
    acc.y += src[i].y;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = acc;
}

// rows (2 v, 2 v + 1) of the dot2 partials into A[v] and B[v]
__global__ void k_reduce_final_pair(const double2* __restrict__ part, int nparts,
                                    double2* __restrict__ A, double2* __restrict__ B) {
  __shared__ double2 sh[32];
  const double2* src = part + size_t(blockIdx.x) * nparts;
  double2 acc = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    acc.x += src[i].x;
    acc.y += src[i].y;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) (blockIdx.x & 1 ? B : A)[blockIdx.x >> 1] = acc;
}

// Per-RHS scalar of an update, formed once per warp (lane 0, broadcast):
// FP64 division and square root are slow on GB300, so they stay out of the
// per-element work.
__device__ __forceinline__ double2 warp_bcast(double2 v) {
  v.x = __shfl_sync(0xffffffffu, v.x, 0);
  v.y = __shfl_sync(0xffffffffu, v.y, 0);
  return v;
}

template <typename Ry, typename Rx>
__global__ void k_copy(cpx<Ry>* __restrict__ y, const cpx<Rx>* __restrict__ x, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    y[i] = cpx<Ry>(x[i]);
}

// y += a x with a host constant
template <typename Ry, typename Rx>
__global__ void k_axpy(cpx<Ry>* __restrict__ y, const cpx<Rx>* __restrict__ x, size_t n,
                       double are, double aim) {
  using T = acc_t<Ry, Rx>;
  const cpx<T> at(cpx<double>(are, aim));
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    cpx<T> yy(y[i]);
    cmac(yy, at, cpx<T>(x[i]));
    y[i] = cpx<Ry>(yy);
  }
}

// y_v += sign S[v] x_v
template <typename Ry, typename Rx>
__global__ void k_axpy_s(cpx<Ry>* __restrict__ y, const cpx<Rx>* __restrict__ x, size_t n,
                         const double2* __restrict__ S, double sign) {
  using T = acc_t<Ry, Rx>;
  const int v = blockIdx.y;
  const cpx<T> at(T(sign * S[v].x), T(sign * S[v].y));
  y += size_t(v) * n;
  x += size_t(v) * n;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    cpx<T> yy(y[i]);
    cmac(yy, at, cpx<T>(x[i]));
    y[i] = cpx<Ry>(yy);
  }
}

template <typename Ro, typename Rb, typename Ra>
__global__ void k_sub(cpx<Ro>* __restrict__ o, const cpx<Rb>* __restrict__ b,
                      const cpx<Ra>* __restrict__ ax, size_t n) {
  using T = acc_t<Ro, acc_t<Rb, Ra>>;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    o[i] = cpx<Ro>(cpx<T>(b[i]) - cpx<T>(ax[i]));
}

// x_v += a_v r_v ; r_v -= a_v p_v  with a_v = omega PR[v] / PP[v].re
template <typename R>
__global__ void k_mr_update(cpx<R>* __restrict__ x, cpx<R>* __restrict__ r,
                            const cpx<R>* __restrict__ p, size_t n,
                            const double2* __restrict__ PR, const double2* __restrict__ PP,
                            double omega) {
  const int v = blockIdx.y;
  double2 a = make_double2(0.0, 0.0);
  if ((threadIdx.x & 31) == 0) {
    const double den = PP[v].x;
    if (den > 0.0) {
      const double f = omega / den;
      a = make_double2(f * PR[v].x, f * PR[v].y);
    }
  }
  a = warp_bcast(a);
  const cpx<R> ar(R(a.x), R(a.y));
  x += size_t(v) * n;
  r += size_t(v) * n;
  p += size_t(v) * n;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    cpx<R> ri = r[i], xi = x[i];
    cmac(xi, ar, ri);
    cmac(ri, -ar, p[i]);
    x[i] = xi;
    r[i] = ri;
  }
}

// a_v, b_v *= 1 / sqrt(S[v].re)   (b may be null)
template <typename Ra, typename Rb>
__global__ void k_scale_invnorm(cpx<Ra>* __restrict__ a, cpx<Rb>* __restrict__ b, size_t n,
                                const double2* __restrict__ S) {
  const int v = blockIdx.y;
  double2 sv = make_double2(0.0, 0.0);
  if ((threadIdx.x & 31) == 0) sv.x = S[v].x > 0.0 ? 1.0 / sqrt(S[v].x) : 0.0;
  sv = warp_bcast(sv);
  const Ra sa = Ra(sv.x);
  const Rb sb = Rb(sv.x);
  a += size_t(v) * n;
  if (b) b += size_t(v) * n;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    a[i] = sa * a[i];
    if (b) b[i] = sb * b[i];
  }
}

// x_v += S[v] z_v ; r_v -= S[v] w_v.  With FP32 directions z, w the products
// are formed in FP32 (they carry the precision of z and w, no more) and only
// the sums run in the precision of x and r; x and r receive the same scalar.
template <typename Rx, typename Rz>
__global__ void k_gcr_update(cpx<Rx>* __restrict__ x, cpx<Rx>* __restrict__ r,
                             const cpx<Rz>* __restrict__ z, const cpx<Rz>* __restrict__ w,
                             size_t n, const double2* __restrict__ S) {
  using T = typename std::conditional<std::is_same<Rz, float>::value, float, double>::type;
  const int v = blockIdx.y;
  const cpx<T> a(T(S[v].x), T(S[v].y));
  x += size_t(v) * n;
  r += size_t(v) * n;
  z += size_t(v) * n;
  w += size_t(v) * n;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    cpx<Rx> xi = x[i], ri = r[i];
    if constexpr (std::is_same<T, float>::value) {
      xi += cpx<Rx>(a * cpx<T>(z[i]));
      ri -= cpx<Rx>(a * cpx<T>(w[i]));
    } else {
      cmac(xi, cpx<Rx>(a), cpx<Rx>(z[i]));
      cmac(ri, -cpx<Rx>(a), cpx<Rx>(w[i]));
    }
    x[i] = xi;
    r[i] = ri;
  }
}

// ---- BF16 vectors (the 16-bit fine-level smoother): storage BF16, all
// arithmetic FP32, per-thread sums FP32 and cross-thread sums FP64
__device__ __forceinline__ cpx<float> h2f(bf16c v) { return StoreTraits<bf16c>::load(v); }

// W = 1: one complex number per access; W = 4: 16-byte words of four BF16
// complex numbers (both vectors 16-byte aligned, n a multiple of 4)
template <int W>
__global__ void k_copy_to16(bf16c* __restrict__ y, const cpx<float>* __restrict__ x, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n / W;
       i += size_t(gridDim.x) * blockDim.x) {
    if constexpr (W == 4) {
      const float4* x4 = reinterpret_cast<const float4*>(x) + 2 * i;
      const float4 a = x4[0], b = x4[1];
      uint4 o;
      bf16c* oc = reinterpret_cast<bf16c*>(&o);
      oc[0] = StoreTraits<bf16c>::pack(cpx<float>(a.x, a.y));
      oc[1] = StoreTraits<bf16c>::pack(cpx<float>(a.z, a.w));
      oc[2] = StoreTraits<bf16c>::pack(cpx<float>(b.x, b.y));
      oc[3] = StoreTraits<bf16c>::pack(cpx<float>(b.z, b.w));
      reinterpret_cast<uint4*>(y)[i] = o;
    } else {
      y[i] = StoreTraits<bf16c>::pack(x[i]);
    }
  }
}
template <int W>
__global__ void k_copy_from16(cpx<float>* __restrict__ y, const bf16c* __restrict__ x, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n / W;
       i += size_t(gridDim.x) * blockDim.x) {
    if constexpr (W == 4) {
      const uint4 w = reinterpret_cast<const uint4*>(x)[i];
      const bf16c* wc = reinterpret_cast<const bf16c*>(&w);
      const cpx<float> c0 = h2f(wc[0]), c1 = h2f(wc[1]), c2 = h2f(wc[2]), c3 = h2f(wc[3]);
      float4* y4 = reinterpret_cast<float4*>(y) + 2 * i;
      y4[0] = make_float4(c0.re, c0.im, c1.re, c1.im);
      y4[1] = make_float4(c2.re, c2.im, c3.re, c3.im);
    } else {
      y[i] = h2f(x[i]);
    }
  }
}

// W = 1: one complex number per access; W = 4: 16-byte loads of four (the
// vectors 16-byte aligned, n a multiple of 4)
template <int W>
__global__ void k_dot2_partial_h(const bf16c* __restrict__ p, const bf16c* __restrict__ r,
                                 size_t n, double2* __restrict__ part) {
  __shared__ double2 sh[32];
  p += blockIdx.y * n;
  r += blockIdx.y * n;
  cpx<float> pr_k[kAcc];
  float pp_k[kAcc];
#pragma unroll
  for (int k = 0; k < kAcc; ++k) {
    pr_k[k] = cpx<float>(0.f, 0.f);
    pp_k[k] = 0.f;
  }
  auto term = [&](bf16c xp, bf16c yr, int k) {
    const cpx<float> x = h2f(xp), y = h2f(yr);
    cmac_conj(pr_k[k], x, y);
    pp_k[k] = fmaf(x.re, x.re, fmaf(x.im, x.im, pp_k[k]));
  };
  if constexpr (W == 4) {
    const uint4* p4 = reinterpret_cast<const uint4*>(p);
    const uint4* r4 = reinterpret_cast<const uint4*>(r);
    grid_loop_acc(n / 4, [&](size_t i, int k) {
      const uint4 wp = p4[i], wr = r4[i];
#pragma unroll
      for (int j = 0; j < 4; ++j)
        term(reinterpret_cast<const bf16c*>(&wp)[j], reinterpret_cast<const bf16c*>(&wr)[j], k);
    });
  } else {
    grid_loop_acc(n, [&](size_t i, int k) { term(p[i], r[i], k); });
  }
  const cpx<float> a_pr = (pr_k[0] + pr_k[1]) + (pr_k[2] + pr_k[3]);
  const float a_pp = (pp_k[0] + pp_k[1]) + (pp_k[2] + pp_k[3]);
  double2 pr = block_sum(make_double2(double(a_pr.re), double(a_pr.im)), sh);
  __syncthreads();
  double2 pp = block_sum(make_double2(double(a_pp), 0.0), sh);
  if (threadIdx.x == 0) {
    const size_t base = size_t(blockIdx.y) * 2 * gridDim.x;
    part[base + blockIdx.x] = pr;
    part[base + gridDim.x + blockIdx.x] = pp;
  }
}

template <int W>
__global__ void k_mr_update_h(bf16c* __restrict__ x, bf16c* __restrict__ r,
                              const bf16c* __restrict__ p, size_t n,
                              const double2* __restrict__ PR, const double2* __restrict__ PP,
                              double omega) {
  const int v = blockIdx.y;
  double2 a = make_double2(0.0, 0.0);
  if ((threadIdx.x & 31) == 0) {
    const double den = PP[v].x;
    if (den > 0.0) {
      const double f = omega / den;
      a = make_double2(f * PR[v].x, f * PR[v].y);
    }
  }
  a = warp_bcast(a);
  const cpx<float> ar(float(a.x), float(a.y));
  x += size_t(v) * n;
  r += size_t(v) * n;
  p += size_t(v) * n;
  auto upd = [&](bf16c& xs, bf16c& rs, bf16c ps) {
    cpx<float> ri = h2f(rs), xi = h2f(xs);
    cmac(xi, ar, ri);
    cmac(ri, -ar, h2f(ps));
    xs = StoreTraits<bf16c>::pack(xi);
    rs = StoreTraits<bf16c>::pack(ri);
  };
  if constexpr (W == 4) {
    uint4* x4 = reinterpret_cast<uint4*>(x);
    uint4* r4 = reinterpret_cast<uint4*>(r);
    const uint4* p4 = reinterpret_cast<const uint4*>(p);
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n / 4;
         i += size_t(gridDim.x) * blockDim.x) {
      uint4 wx = x4[i], wr = r4[i];
      const uint4 wp = p4[i];
#pragma unroll
      for (int j = 0; j < 4; ++j)
        upd(reinterpret_cast<bf16c*>(&wx)[j], reinterpret_cast<bf16c*>(&wr)[j],
            reinterpret_cast<const bf16c*>(&wp)[j]);
      x4[i] = wx;
      r4[i] = wr;
    }
  } else {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
         i += size_t(gridDim.x) * blockDim.x)
      upd(x[i], r[i], p[i]);
  }
}

// ---- batched forms for the setup sweeps (nvec vectors back to back;
// blockIdx.y is the vector)
// x_v -= (B[2v] / B[2v+1].re) t_v
template <typename R>
__global__ void k_sweep_update_b(cpx<R>* __restrict__ x, const cpx<R>* __restrict__ t, size_t n,
                                 const double2* __restrict__ B) {
  const int v = blockIdx.y;
  double2 a = make_double2(0.0, 0.0);
  if ((threadIdx.x & 31) == 0) {
    const double den = B[2 * v + 1].x;
    if (den > 0.0) {
      const double inv = 1.0 / den;
      a = make_double2(-B[2 * v].x * inv, -B[2 * v].y * inv);
    }
  }
  a = warp_bcast(a);
  const cpx<R> ar(R(a.x), R(a.y));
  x += size_t(v) * n;
  t += size_t(v) * n;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    cpx<R> xi = x[i];
    cmac(xi, ar, t[i]);
    x[i] = xi;
  }
}

// x_v /= sqrt(B[2v+1].re)
template <typename R>
__global__ void k_normalise_b(cpx<R>* __restrict__ x, size_t n, const double2* __restrict__ B) {
  const int v = blockIdx.y;
  double2 s = make_double2(0.0, 0.0);
  if ((threadIdx.x & 31) == 0) {
    const double nn = B[2 * v + 1].x;
    s.x = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
  }
  s = warp_bcast(s);
  const R sr = R(s.x);
  x += size_t(v) * n;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    x[i] = sr * x[i];
}

// [nvec][n] <-> [n][nvec] layout change of complex vectors
template <typename R>
__global__ void k_transpose(cpx<R>* __restrict__ out, const cpx<R>* __restrict__ in, size_t n,
                            int nvec, int to_interleaved) {
  const size_t total = n * nvec;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total;
       i += size_t(gridDim.x) * blockDim.x) {
    if (to_interleaved) {  // out[e][v] = in[v][e], i enumerates out
      const size_t e = i / nvec;
      const int v = int(i - e * nvec);
      out[i] = in[size_t(v) * n + e];
    } else {               // out[v][e] = in[e][v], i enumerates out
      const int v = int(i / n);
      const size_t e = i - size_t(v) * n;
      out[i] = in[e * nvec + v];
    }
  }
}

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC11), used to draw the
// random initial null-vector guesses on the device.
__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint2 key) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int i = 0; i < 10; ++i) {
    uint32_t hi0 = __umulhi(M0, ctr.x), lo0 = M0 * ctr.x;
    uint32_t hi1 = __umulhi(M1, ctr.z), lo1 = M1 * ctr.z;
    ctr = make_uint4(hi1 ^ ctr.y ^ key.x, lo1, hi0 ^ ctr.w ^ key.y, lo0);
    key.x += W0;
    key.y += W1;
  }
  return ctr;
}

template <typename R>
__global__ void k_gaussian(cpx<R>* __restrict__ v, size_t n, uint64_t seed, uint64_t offset) {
  uint2 key = make_uint2(uint32_t(seed), uint32_t(seed >> 32));
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    uint64_t c = offset + i;
    uint4 r = philox4x32_10(make_uint4(uint32_t(c), uint32_t(c >> 32), 0x6A09E667u, 0), key);
    // Box-Muller on two uniforms in (0, 1], in the output precision
    const R u1 = (R(r.x) + R(1)) * R(2.3283064365386963e-10);
    const R u2 = R(r.y) * R(2.3283064365386963e-10);
    const R rad = sqrt(R(-2) * log(u1));
    R s, co;
    sincospi(R(2) * u2, &s, &co);
    v[i] = cpx<R>(rad * co, rad * s);
  }
}

// row of slot `slot`: the nr per-RHS values S[slot][v]
double2* srow(mg_ctx* c, int slot) { return c->scalars.as<double2>() + size_t(slot) * kMaxNrhs; }

double2* partials(mg_ctx* c, size_t count) {
  const size_t need = count * sizeof(double2);
  if (c->red_partials.bytes < need) c->red_partials.alloc(need);
  return c->red_partials.as<double2>();
}

void check_nr(const Vec& v) {
  GB_REQUIRE(v.nr >= 1 && v.nr <= kMaxNrhs, MG_ERR_ARG, "more right-hand sides than supported");
}

}  // namespace

#define GB_DISPATCH1(prec, R, ...)                      \
  do {                                                  \
    if ((prec) == MG_F64) {                             \
      using R = double;                                 \
      __VA_ARGS__;                                      \
    } else {                                            \
      using R = float;                                  \
      __VA_ARGS__;                                      \
    }                                                   \
  } while (0)

#define GB_DISPATCH2(pa, Ra, pb, Rb, ...)                    \
  GB_DISPATCH1(pa, Ra, GB_DISPATCH1(pb, Rb, __VA_ARGS__))

void blas_zero(mg_ctx* c, Vec v, cudaStream_t st) {
  GB_CHECK(cudaMemsetAsync(v.p, 0, v.total() * prec_bytes_complex(v.prec), st));
}

void blas_copy(mg_ctx* c, Vec d, Vec s, cudaStream_t st) {
  GB_REQUIRE(d.total() == s.total(), MG_ERR_ARG, "copy: length mismatch");
  if (d.prec != s.prec && (d.prec == MG_BF16 || s.prec == MG_BF16)) {
    GB_REQUIRE(d.prec == MG_F32 || s.prec == MG_F32, MG_ERR_ARG, "copy: BF16 <-> FP32 only");
    const size_t n = d.total();
    const bool w4 = n % 4 == 0 && aligned16(d.p) && aligned16(s.p);
    if (d.prec == MG_BF16) {
      if (w4)
        k_copy_to16<4><<<ew_blocks(n / 4), kThreads, 0, st>>>((bf16c*)d.p,
                                                              (const cpx<float>*)s.p, n);
      else
        k_copy_to16<1><<<ew_blocks(n), kThreads, 0, st>>>((bf16c*)d.p, (const cpx<float>*)s.p,
                                                          n);
    } else {
      if (w4)
        k_copy_from16<4><<<ew_blocks(n / 4), kThreads, 0, st>>>((cpx<float>*)d.p,
                                                                (const bf16c*)s.p, n);
      else
        k_copy_from16<1><<<ew_blocks(n), kThreads, 0, st>>>((cpx<float>*)d.p,
                                                            (const bf16c*)s.p, n);
    }
    GB_LAUNCH_CHECK();
    c->launches++;
    return;
  }
  if (d.prec == s.prec) {
    GB_CHECK(cudaMemcpyAsync(d.p, s.p, d.total() * prec_bytes_complex(d.prec),
                             cudaMemcpyDeviceToDevice, st));
    return;
  }
  GB_DISPATCH2(d.prec, Ry, s.prec, Rx,
               (k_copy<Ry, Rx><<<ew_blocks(d.total()), kThreads, 0, st>>>(
                   (cpx<Ry>*)d.p, (const cpx<Rx>*)s.p, d.total())));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void blas_axpy_host(mg_ctx* c, Vec y, Vec x, double are, double aim, cudaStream_t st) {
  GB_REQUIRE(y.total() == x.total(), MG_ERR_ARG, "axpy: length mismatch");
  GB_DISPATCH2(y.prec, Ry, x.prec, Rx,
               (k_axpy<Ry, Rx><<<ew_blocks(y.total()), kThreads, 0, st>>>(
                   (cpx<Ry>*)y.p, (const cpx<Rx>*)x.p, y.total(), are, aim)));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void blas_axpy_slot(mg_ctx* c, Vec y, Vec x, int slot, double sign, cudaStream_t st) {
  check_nr(y);
  GB_REQUIRE(y.n == x.n && y.nr == x.nr, MG_ERR_ARG, "axpy: shape mismatch");
  GB_DISPATCH2(y.prec, Ry, x.prec, Rx,
               (k_axpy_s<Ry, Rx><<<ew_grid_b(y.n, y.nr), kThreads, 0, st>>>(
                   (cpx<Ry>*)y.p, (const cpx<Rx>*)x.p, y.n, srow(c, slot), sign)));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void blas_sub(mg_ctx* c, Vec o, Vec b, Vec ax, cudaStream_t st) {
  GB_REQUIRE(o.total() == b.total() && b.total() == ax.total(), MG_ERR_ARG,
             "sub: length mismatch");
  GB_DISPATCH1(o.prec, Ro,
               GB_DISPATCH2(b.prec, Rb, ax.prec, Ra,
                            (k_sub<Ro, Rb, Ra><<<ew_blocks(o.total()), kThreads, 0, st>>>(
                                (cpx<Ro>*)o.p, (const cpx<Rb>*)b.p, (const cpx<Ra>*)ax.p,
                                o.total()))));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void blas_dot(mg_ctx* c, Vec a, Vec b, int slot, cudaStream_t st, bool fp64_partials) {
  check_nr(a);
  GB_REQUIRE(a.n == b.n && a.nr == b.nr, MG_ERR_ARG, "dot: shape mismatch");
  const int nb = red_blocks(a.n);
  double2* part = partials(c, size_t(nb) * a.nr);
  const dim3 grid(nb, a.nr);
  const bool norm = a.p == b.p && a.prec == b.prec;
  const bool ff = fp64_partials && a.prec == MG_F32 && b.prec == MG_F32;
  const bool w2 = a.n % 2 == 0 && aligned16(a.p) && aligned16(b.p);
  if (ff) {
    const auto* pa = (const cpx<float>*)a.p;
    const auto* pb = (const cpx<float>*)b.p;
    if (norm && w2)
      k_dot_partial_ff<true, 2><<<grid, kThreads, 0, st>>>(pa, pa, a.n, part);
    else if (norm)
      k_dot_partial_ff<true, 1><<<grid, kThreads, 0, st>>>(pa, pa, a.n, part);
    else if (w2)
      k_dot_partial_ff<false, 2><<<grid, kThreads, 0, st>>>(pa, pb, a.n, part);
    else
      k_dot_partial_ff<false, 1><<<grid, kThreads, 0, st>>>(pa, pb, a.n, part);
  } else if (norm && fp64_partials) {
    GB_DISPATCH1(a.prec, Ra,
                 (k_dot_partial<Ra, Ra, double, true><<<grid, kThreads, 0, st>>>(
                     (const cpx<Ra>*)a.p, (const cpx<Ra>*)a.p, a.n, part)));
  } else if (norm) {
    GB_DISPATCH1(a.prec, Ra,
                 (k_dot_partial<Ra, Ra, acc_t<Ra, Ra>, true><<<grid, kThreads, 0, st>>>(
                     (const cpx<Ra>*)a.p, (const cpx<Ra>*)a.p, a.n, part)));
  } else if (fp64_partials) {
    GB_DISPATCH2(a.prec, Ra, b.prec, Rb,
                 (k_dot_partial<Ra, Rb, double><<<grid, kThreads, 0, st>>>(
                     (const cpx<Ra>*)a.p, (const cpx<Rb>*)b.p, a.n, part)));
  } else {
    GB_DISPATCH2(a.prec, Ra, b.prec, Rb,
                 (k_dot_partial<Ra, Rb, acc_t<Ra, Rb>><<<grid, kThreads, 0, st>>>(
                     (const cpx<Ra>*)a.p, (const cpx<Rb>*)b.p, a.n, part)));
  }
  GB_LAUNCH_CHECK();
  k_reduce_final_b<<<a.nr, 256, 0, st>>>(part, nb, srow(c, slot));
  GB_LAUNCH_CHECK();
  c->launches += 2;
}

void blas_norm2(mg_ctx* c, Vec a, int slot, cudaStream_t st, bool fp64_partials) {
  blas_dot(c, a, a, slot, st, fp64_partials);
}

void blas_dot2(mg_ctx* c, Vec p, Vec r, int s_pr, int s_pp, cudaStream_t st) {
  check_nr(p);
  GB_REQUIRE(p.n == r.n && p.nr == r.nr, MG_ERR_ARG, "dot2: shape mismatch");
  const int nb = red_blocks(p.n);
  double2* part = partials(c, size_t(nb) * 2 * p.nr);
  if (p.prec == MG_BF16 || r.prec == MG_BF16) {
    GB_REQUIRE(p.prec == MG_BF16 && r.prec == MG_BF16, MG_ERR_ARG, "dot2: precision mix");
    if (p.n % 4 == 0 && aligned16(p.p) && aligned16(r.p))
      k_dot2_partial_h<4><<<dim3(nb, p.nr), kThreads, 0, st>>>((const bf16c*)p.p,
                                                               (const bf16c*)r.p, p.n, part);
    else
      k_dot2_partial_h<1><<<dim3(nb, p.nr), kThreads, 0, st>>>((const bf16c*)p.p,
                                                               (const bf16c*)r.p, p.n, part);
  } else {
    GB_DISPATCH2(p.prec, Ra, r.prec, Rb,
                 (k_dot2_partial_b<Ra, Rb><<<dim3(nb, p.nr), kThreads, 0, st>>>(
                     (const cpx<Ra>*)p.p, (const cpx<Rb>*)r.p, p.n, part)));
  }
  GB_LAUNCH_CHECK();
  k_reduce_final_pair<<<2 * p.nr, 256, 0, st>>>(part, nb, srow(c, s_pr), srow(c, s_pp));
  GB_LAUNCH_CHECK();
  c->launches += 2;
}

void blas_mr_update(mg_ctx* c, Vec x, Vec r, Vec p, int s_pr, int s_pp, double omega,
                    cudaStream_t st) {
  check_nr(x);
  GB_REQUIRE(x.prec == r.prec && r.prec == p.prec, MG_ERR_ARG, "mr_update: precision mix");
  if (x.prec == MG_BF16) {
    if (x.n % 4 == 0 && aligned16(x.p) && aligned16(r.p) && aligned16(p.p))
      k_mr_update_h<4><<<ew_grid_b(x.n / 4, x.nr), kThreads, 0, st>>>(
          (bf16c*)x.p, (bf16c*)r.p, (const bf16c*)p.p, x.n, srow(c, s_pr), srow(c, s_pp), omega);
    else
      k_mr_update_h<1><<<ew_grid_b(x.n, x.nr), kThreads, 0, st>>>(
          (bf16c*)x.p, (bf16c*)r.p, (const bf16c*)p.p, x.n, srow(c, s_pr), srow(c, s_pp), omega);
    GB_LAUNCH_CHECK();
    c->launches++;
    return;
  }
  GB_DISPATCH1(x.prec, R,
               (k_mr_update<R><<<ew_grid_b(x.n, x.nr), kThreads, 0, st>>>(
                   (cpx<R>*)x.p, (cpx<R>*)r.p, (const cpx<R>*)p.p, x.n, srow(c, s_pr),
                   srow(c, s_pp), omega)));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void blas_scale_invnorm(mg_ctx* c, Vec a, Vec b, int slot, cudaStream_t st) {
  check_nr(a);
  GB_DISPATCH2(a.prec, Ra, b.prec, Rb,
               (k_scale_invnorm<Ra, Rb><<<ew_grid_b(a.n, a.nr), kThreads, 0, st>>>(
                   (cpx<Ra>*)a.p, (cpx<Rb>*)b.p, a.n, srow(c, slot))));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void blas_gcr_update(mg_ctx* c, Vec x, Vec r, Vec z, Vec w, int slot, cudaStream_t st) {
  check_nr(x);
  GB_REQUIRE(x.prec == r.prec && z.prec == w.prec, MG_ERR_ARG, "gcr_update: precision mix");
  GB_DISPATCH2(x.prec, Rx, z.prec, Rz,
               (k_gcr_update<Rx, Rz><<<ew_grid_b(x.n, x.nr), kThreads, 0, st>>>(
                   (cpx<Rx>*)x.p, (cpx<Rx>*)r.p, (const cpx<Rz>*)z.p, (const cpx<Rz>*)w.p, x.n,
                   srow(c, slot))));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void blas_read_slot(mg_ctx* c, int slot, int nr, double* out_re, cudaStream_t st) {
  GB_REQUIRE(nr >= 1 && nr <= kMaxNrhs, MG_ERR_ARG, "read_slot: bad count");
  GB_CHECK(cudaMemcpyAsync(c->h_scalars, srow(c, slot), sizeof(double2) * nr,
                           cudaMemcpyDeviceToHost, st));
  GB_CHECK(cudaStreamSynchronize(st));
  for (int v = 0; v < nr; ++v) out_re[v] = c->h_scalars[2 * v];
}

void blas_dot_multi(mg_ctx* c, const Vec* X, int m, Vec y, int slot, cudaStream_t st,
                    bool fp64_partials) {
  check_nr(y);
  GB_REQUIRE(m >= 1 && m <= kCgs && slot + m <= SC_COUNT, MG_ERR_ARG, "dot_multi: bad count");
  VecList L{};
  for (int j = 0; j < m; ++j) {
    GB_REQUIRE(X[j].n == y.n && X[j].nr == y.nr && X[j].prec == y.prec, MG_ERR_ARG,
               "dot_multi: shape mismatch");
    L.p[j] = X[j].p;
  }
  bool w2 = y.prec == MG_F32 && fp64_partials && y.n % 2 == 0 && aligned16(y.p);
  for (int j = 0; j < m; ++j) w2 = w2 && aligned16(X[j].p);
  // resident blocks per SM from the registers a thread: k_dot_multi <= 128;
  // k_dot_multi_ff<M> <= 64 up to M = 6, <= 80 up to M = 8, <= 128 beyond
  const int nb = red_blocks(y.n, !w2 ? 2 : m <= 6 ? 4 : m <= 8 ? 3 : 2);
  double2* part = partials(c, size_t(nb) * m * y.nr);
  const dim3 grid(nb, y.nr);
  const auto* yp = (const cpx<float>*)y.p;
  if (w2) {
    switch (m) {
      case 1: k_dot_multi_ff<1><<<grid, kThreads, 0, st>>>(L, yp, y.n, part); break;
      case 2: k_dot_multi_ff<2><<<grid, kThreads, 0, st>>>(L, yp, y.n, part); break;
      case 3: k_dot_multi_ff<3><<<grid, kThreads, 0, st>>>(L, yp, y.n, part); break;
      case 4: k_dot_multi_ff<4><<<grid, kThreads, 0, st>>>(L, yp, y.n, part); break;
      case 5: k_dot_multi_ff<5><<<grid, kThreads, 0, st>>>(L, yp, y.n, part); break;
      case 6: k_dot_multi_ff<6><<<grid, kThreads, 0, st>>>(L, yp, y.n, part); break;
      case 7: k_dot_multi_ff<7><<<grid, kThreads, 0, st>>>(L, yp, y.n, part); break;
      case 8: k_dot_multi_ff<8><<<grid, kThreads, 0, st>>>(L, yp, y.n, part); break;
      case 9: k_dot_multi_ff<9><<<grid, kThreads, 0, st>>>(L, yp, y.n, part); break;
      default: k_dot_multi_ff<10><<<grid, kThreads, 0, st>>>(L, yp, y.n, part); break;
    }
  } else if (y.prec == MG_F32 && fp64_partials)
    k_dot_multi<float, true><<<grid, kThreads, 0, st>>>(L, yp, m, y.n, part);
  else
    GB_DISPATCH1(y.prec, R,
                 (k_dot_multi<R, false><<<grid, kThreads, 0, st>>>(L, (const cpx<R>*)y.p, m,
                                                                  y.n, part)));
  GB_LAUNCH_CHECK();
  k_reduce_final_multi<<<m * y.nr, 256, 0, st>>>(part, nb, m, srow(c, slot));
  GB_LAUNCH_CHECK();
  c->launches += 2;
}

void blas_axpy_multi(mg_ctx* c, Vec y, const Vec* X, int m, int slot, double sign,
                     cudaStream_t st) {
  check_nr(y);
  GB_REQUIRE(m >= 1 && m <= kCgs && slot + m <= SC_COUNT, MG_ERR_ARG, "axpy_multi: bad count");
  VecList L{};
  for (int j = 0; j < m; ++j) {
    GB_REQUIRE(X[j].n == y.n && X[j].nr == y.nr && X[j].prec == y.prec, MG_ERR_ARG,
               "axpy_multi: shape mismatch");
    L.p[j] = X[j].p;
  }
  bool w2 = y.prec == MG_F32 && y.n % 2 == 0 && aligned16(y.p);
  for (int j = 0; j < m; ++j) w2 = w2 && aligned16(X[j].p);
  if (w2) {
    const dim3 grid = ew_grid_b(y.n / 2, y.nr);
    auto* yp = (cpx<float>*)y.p;
    const double2* S = srow(c, slot);
    switch (m) {
      case 1: k_axpy_multi_w2<1><<<grid, kThreads, 0, st>>>(yp, L, y.n, S, sign); break;
      case 2: k_axpy_multi_w2<2><<<grid, kThreads, 0, st>>>(yp, L, y.n, S, sign); break;
      case 3: k_axpy_multi_w2<3><<<grid, kThreads, 0, st>>>(yp, L, y.n, S, sign); break;
      case 4: k_axpy_multi_w2<4><<<grid, kThreads, 0, st>>>(yp, L, y.n, S, sign); break;
      case 5: k_axpy_multi_w2<5><<<grid, kThreads, 0, st>>>(yp, L, y.n, S, sign); break;
      case 6: k_axpy_multi_w2<6><<<grid, kThreads, 0, st>>>(yp, L, y.n, S, sign); break;
      case 7: k_axpy_multi_w2<7><<<grid, kThreads, 0, st>>>(yp, L, y.n, S, sign); break;
      case 8: k_axpy_multi_w2<8><<<grid, kThreads, 0, st>>>(yp, L, y.n, S, sign); break;
      case 9: k_axpy_multi_w2<9><<<grid, kThreads, 0, st>>>(yp, L, y.n, S, sign); break;
      default: k_axpy_multi_w2<10><<<grid, kThreads, 0, st>>>(yp, L, y.n, S, sign); break;
    }
  } else {
    GB_DISPATCH1(y.prec, R,
                 (k_axpy_multi<R><<<ew_grid_b(y.n, y.nr), kThreads, 0, st>>>(
                     (cpx<R>*)y.p, L, m, y.n, srow(c, slot), sign)));
  }
  GB_LAUNCH_CHECK();
  c->launches++;
}

void blas_read_slot_c(mg_ctx* c, int slot, double out[2], cudaStream_t st) {
  GB_CHECK(cudaMemcpyAsync(c->h_scalars, srow(c, slot), sizeof(double2),
                           cudaMemcpyDeviceToHost, st));
  GB_CHECK(cudaStreamSynchronize(st));
  out[0] = c->h_scalars[0];
  out[1] = c->h_scalars[1];
}

void blas_dot2_batched(mg_ctx* c, Vec p, Vec r, int nvec, cudaStream_t st) {
  GB_REQUIRE(nvec >= 1 && nvec <= 64, MG_ERR_ARG, "dot2_batched: nvec out of range");
  const int nb = red_blocks(p.n);
  const size_t need = size_t(nvec) * 2 * nb * sizeof(double2);
  if (c->batch_partials.bytes < need) c->batch_partials.alloc(need);
  double2* part = c->batch_partials.as<double2>();
  dim3 grid(nb, nvec);
  GB_DISPATCH2(p.prec, Ra, r.prec, Rb,
               (k_dot2_partial_b<Ra, Rb><<<grid, kThreads, 0, st>>>(
                   (const cpx<Ra>*)p.p, (const cpx<Rb>*)r.p, p.n, part)));
  GB_LAUNCH_CHECK();
  k_reduce_final_b<<<2 * nvec, 256, 0, st>>>(part, nb, c->batch_scalars.as<double2>());
  GB_LAUNCH_CHECK();
  c->launches += 2;
}

void blas_sweep_update_batched(mg_ctx* c, Vec x, Vec t, int nvec, cudaStream_t st) {
  GB_REQUIRE(x.prec == t.prec, MG_ERR_ARG, "sweep_update_batched: precision mix");
  GB_DISPATCH1(x.prec, R,
               (k_sweep_update_b<R><<<ew_grid_b(x.n, nvec), kThreads, 0, st>>>(
                   (cpx<R>*)x.p, (const cpx<R>*)t.p, x.n, c->batch_scalars.as<double2>())));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void blas_normalise_batched(mg_ctx* c, Vec x, int nvec, cudaStream_t st) {
  // |x_v|^2 into the second slot of each vector's pair
  blas_dot2_batched(c, x, x, nvec, st);
  GB_DISPATCH1(x.prec, R,
               (k_normalise_b<R><<<ew_grid_b(x.n, nvec), kThreads, 0, st>>>(
                   (cpx<R>*)x.p, x.n, c->batch_scalars.as<double2>())));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void blas_transpose(mg_ctx* c, Vec out, Vec in, int nvec, bool to_interleaved, cudaStream_t st) {
  GB_REQUIRE(out.prec == in.prec && out.n == in.n, MG_ERR_ARG, "transpose: mismatch");
  GB_DISPATCH1(out.prec, R,
               (k_transpose<R><<<ew_blocks(out.n * nvec), kThreads, 0, st>>>(
                   (cpx<R>*)out.p, (const cpx<R>*)in.p, out.n, nvec, to_interleaved ? 1 : 0)));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void blas_gaussian(mg_ctx* c, Vec v, uint64_t seed, uint64_t offset, cudaStream_t st) {
  GB_DISPATCH1(v.prec, R,
               (k_gaussian<R><<<ew_blocks(v.n), kThreads, 0, st>>>((cpx<R>*)v.p, v.n, seed,
                                                                    offset)));
  GB_LAUNCH_CHECK();
  c->launches++;
}

int read_status(mg_ctx* c, cudaStream_t st) {
  int h = 0;
  GB_CHECK(cudaMemcpyAsync(&h, c->status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  GB_CHECK(cudaStreamSynchronize(st));
  return h;
}

void clear_status(mg_ctx* c, cudaStream_t st) {
  GB_CHECK(cudaMemsetAsync(c->status.p, 0, c->status.bytes, st));
}

}  // namespace gbmg
