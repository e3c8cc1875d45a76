// Level-1 vector kernels of the solvers (Sec. VI-A: GCR, MR, setup
// iteration).  Scalars stay on the device: a reduction writes a complex
// double into a slot of ctx->scalars and the following update kernel reads
// it, so smoothers and orthogonalisation never wait on the host.
// Reductions are two-stage with a grid that depends only on the length,
// so results are bitwise reproducible run to run.
#include <type_traits>

#include "kernels.cuh"

namespace gbmg {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxRedBlocks = 1024;

int red_blocks(size_t n) {
  long long b = (long long)((n + 4095) / 4096);
  if (b < 1) b = 1;
  if (b > kMaxRedBlocks) b = kMaxRedBlocks;
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

template <typename Ra, typename Rb, typename T>
__global__ void k_dot_partial(const cpx<Ra>* __restrict__ a, const cpx<Rb>* __restrict__ b,
                              size_t n, double2* __restrict__ part) {
  __shared__ double2 sh[32];
  cpx<T> acc(T(0), T(0));
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    cmac_conj(acc, cpx<T>(a[i]), cpx<T>(b[i]));
  double2 d = block_sum(make_double2(double(acc.re), double(acc.im)), sh);
  if (threadIdx.x == 0) part[blockIdx.x] = d;
}

template <typename Ra, typename Rb>
__global__ void k_dot2_partial(const cpx<Ra>* __restrict__ p, const cpx<Rb>* __restrict__ r,
                               size_t n, double2* __restrict__ part, int stride) {
  using T = acc_t<Ra, Rb>;
  __shared__ double2 sh[32];
  cpx<T> a_pr(T(0), T(0));
  T a_pp = T(0);
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    cpx<T> x(p[i]), y(r[i]);
    cmac_conj(a_pr, x, y);
    a_pp = fma(x.re, x.re, fma(x.im, x.im, a_pp));
  }
  double2 pr = block_sum(make_double2(double(a_pr.re), double(a_pr.im)), sh);
  __syncthreads();
  double2 pp = block_sum(make_double2(double(a_pp), 0.0), sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = pr;
    part[stride + blockIdx.x] = pp;
  }
}

__global__ void k_reduce_final(const double2* __restrict__ part, int nparts, double2* out) {
  __shared__ double2 sh[32];
  double2 acc = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    acc.x += part[i].x;
    acc.y += part[i].y;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = acc;
}

template <typename Ry, typename Rx>
__global__ void k_copy(cpx<Ry>* __restrict__ y, const cpx<Rx>* __restrict__ x, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    y[i] = cpx<Ry>(x[i]);
}

template <typename Ry, typename Rx>
__global__ void k_axpy(cpx<Ry>* __restrict__ y, const cpx<Rx>* __restrict__ x, size_t n,
                       double are, double aim, const double2* __restrict__ S, int slot,
                       double sign) {
  using T = acc_t<Ry, Rx>;
  cpx<double> a(are, aim);
  if (S) a = cpx<double>(sign * S[slot].x, sign * S[slot].y);
  const cpx<T> at(a);
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

// x += a r ; r -= a p  with a = omega S[spr] / S[spp].re
template <typename R>
__global__ void k_mr_update(cpx<R>* __restrict__ x, cpx<R>* __restrict__ r,
                            const cpx<R>* __restrict__ p, size_t n, const double2* S, int spr,
                            int spp, double omega) {
  double den = S[spp].x;
  cpx<double> a(0.0, 0.0);
  if (den > 0.0) a = cpx<double>(omega * S[spr].x / den, omega * S[spr].y / den);
  cpx<R> ar(R(a.re), R(a.im));
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    cpx<R> ri = r[i], xi = x[i];
    cmac(xi, ar, ri);
    cmac(ri, -ar, p[i]);
    x[i] = xi;
    r[i] = ri;
  }
}

template <typename Ra, typename Rb>
__global__ void k_scale_invnorm(cpx<Ra>* __restrict__ a, cpx<Rb>* __restrict__ b, size_t n,
                                const double2* S, int slot) {
  const double s = S[slot].x > 0.0 ? 1.0 / sqrt(S[slot].x) : 0.0;
  const Ra sa = Ra(s);
  const Rb sb = Rb(s);
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    a[i] = sa * a[i];
    if (b) b[i] = sb * b[i];
  }
}

// x += a z ; r -= a w.  With FP32 directions z, w the products a z and a w
// are formed in FP32 (they carry the precision of z and w, no more) and only
// the sums run in the precision of x and r; x and r receive the same a.
template <typename Rx, typename Rz>
__global__ void k_gcr_update(cpx<Rx>* __restrict__ x, cpx<Rx>* __restrict__ r,
                             const cpx<Rz>* __restrict__ z, const cpx<Rz>* __restrict__ w,
                             size_t n, const double2* S, int slot) {
  using T = typename std::conditional<std::is_same<Rz, float>::value, float, double>::type;
  const cpx<T> a(T(S[slot].x), T(S[slot].y));
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

// x -= (S[qt] / S[qq].re) t
template <typename R>
__global__ void k_sweep_update(cpx<R>* __restrict__ x, const cpx<R>* __restrict__ t, size_t n,
                               const double2* S, int sqt, int sqq) {
  double den = S[sqq].x;
  cpx<double> a(0.0, 0.0);
  if (den > 0.0) a = cpx<double>(-S[sqt].x / den, -S[sqt].y / den);
  cpx<R> ar(R(a.re), R(a.im));
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    cpx<R> xi = x[i];
    cmac(xi, ar, t[i]);
    x[i] = xi;
  }
}

// ---- batched forms over nvec vectors stored back to back (vector v at
// offset v * n); blockIdx.y is the vector.
template <typename Ra, typename Rb>
__global__ void k_dot2_partial_b(const cpx<Ra>* __restrict__ p, const cpx<Rb>* __restrict__ r,
                                 size_t n, double2* __restrict__ part) {
  using T = acc_t<Ra, Rb>;
  __shared__ double2 sh[32];
  p += blockIdx.y * n;
  r += blockIdx.y * n;
  cpx<T> a_pr(T(0), T(0));
  T a_pp = T(0);
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    cpx<T> x(p[i]), y(r[i]);
    cmac_conj(a_pr, x, y);
    a_pp = fma(x.re, x.re, fma(x.im, x.im, a_pp));
  }
  double2 pr = block_sum(make_double2(double(a_pr.re), double(a_pr.im)), sh);
  __syncthreads();
  double2 pp = block_sum(make_double2(double(a_pp), 0.0), sh);
  if (threadIdx.x == 0) {
    const size_t base = size_t(blockIdx.y) * 2 * gridDim.x;
    part[base + blockIdx.x] = pr;
    part[base + gridDim.x + blockIdx.x] = pp;
  }
}

// out[2 v + k] = sum of the nparts partials of (vector v, quantity k)
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

// Per-vector scalar of the batched updates, computed once per warp (lane 0,
// broadcast): FP64 division and square root are slow on GB300, so they stay
// out of the per-element loop.
__device__ __forceinline__ double2 warp_bcast(double2 v) {
  v.x = __shfl_sync(0xffffffffu, v.x, 0);
  v.y = __shfl_sync(0xffffffffu, v.y, 0);
  return v;
}

// x_v -= (B[2v] / B[2v+1].re) t_v   (setup sweep, every vector at once;
// blockIdx.y is the vector)
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

template <typename R>
__global__ void k_normalise(cpx<R>* __restrict__ x, size_t n, const double2* S, int slot) {
  const R s = R(S[slot].x > 0.0 ? 1.0 / sqrt(S[slot].x) : 0.0);
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    x[i] = s * x[i];
}

double2* scal(mg_ctx* c) { return c->scalars.as<double2>(); }

void finish_reduction(mg_ctx* c, int nb, int slot, const double2* part, cudaStream_t st) {
  k_reduce_final<<<1, 256, 0, st>>>(part, nb, scal(c) + slot);
  GB_LAUNCH_CHECK();
  c->launches++;
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
  GB_CHECK(cudaMemsetAsync(v.p, 0, v.n * prec_bytes_complex(v.prec), st));
}

void blas_copy(mg_ctx* c, Vec d, Vec s, cudaStream_t st) {
  GB_REQUIRE(d.n == s.n, MG_ERR_ARG, "copy: length mismatch");
  if (d.prec == s.prec) {
    GB_CHECK(cudaMemcpyAsync(d.p, s.p, d.n * prec_bytes_complex(d.prec), cudaMemcpyDeviceToDevice,
                             st));
    return;
  }
  GB_DISPATCH2(d.prec, Ry, s.prec, Rx,
               (k_copy<Ry, Rx><<<ew_blocks(d.n), kThreads, 0, st>>>(
                   (cpx<Ry>*)d.p, (const cpx<Rx>*)s.p, d.n)));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void blas_axpy_host(mg_ctx* c, Vec y, Vec x, double are, double aim, cudaStream_t st) {
  GB_DISPATCH2(y.prec, Ry, x.prec, Rx,
               (k_axpy<Ry, Rx><<<ew_blocks(y.n), kThreads, 0, st>>>(
                   (cpx<Ry>*)y.p, (const cpx<Rx>*)x.p, y.n, are, aim, nullptr, 0, 1.0)));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void blas_axpy_slot(mg_ctx* c, Vec y, Vec x, int slot, double sign, cudaStream_t st) {
  GB_DISPATCH2(y.prec, Ry, x.prec, Rx,
               (k_axpy<Ry, Rx><<<ew_blocks(y.n), kThreads, 0, st>>>(
                   (cpx<Ry>*)y.p, (const cpx<Rx>*)x.p, y.n, 0.0, 0.0, scal(c), slot, sign)));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void blas_sub(mg_ctx* c, Vec o, Vec b, Vec ax, cudaStream_t st) {
  GB_REQUIRE(o.n == b.n && b.n == ax.n, MG_ERR_ARG, "sub: length mismatch");
  GB_DISPATCH1(o.prec, Ro,
               GB_DISPATCH2(b.prec, Rb, ax.prec, Ra,
                            (k_sub<Ro, Rb, Ra><<<ew_blocks(o.n), kThreads, 0, st>>>(
                                (cpx<Ro>*)o.p, (const cpx<Rb>*)b.p, (const cpx<Ra>*)ax.p, o.n))));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void blas_dot(mg_ctx* c, Vec a, Vec b, int slot, cudaStream_t st, bool fp64_partials) {
  int nb = red_blocks(a.n);
  double2* part = c->red_partials.as<double2>();
  if (fp64_partials) {
    GB_DISPATCH2(a.prec, Ra, b.prec, Rb,
                 (k_dot_partial<Ra, Rb, double><<<nb, kThreads, 0, st>>>(
                     (const cpx<Ra>*)a.p, (const cpx<Rb>*)b.p, a.n, part)));
  } else {
    GB_DISPATCH2(a.prec, Ra, b.prec, Rb,
                 (k_dot_partial<Ra, Rb, acc_t<Ra, Rb>><<<nb, kThreads, 0, st>>>(
                     (const cpx<Ra>*)a.p, (const cpx<Rb>*)b.p, a.n, part)));
  }
  GB_LAUNCH_CHECK();
  c->launches++;
  finish_reduction(c, nb, slot, part, st);
}

void blas_norm2(mg_ctx* c, Vec a, int slot, cudaStream_t st, bool fp64_partials) {
  blas_dot(c, a, a, slot, st, fp64_partials);
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

void blas_dot2(mg_ctx* c, Vec p, Vec r, int s_pr, int s_pp, cudaStream_t st) {
  int nb = red_blocks(p.n);
  double2* part = c->red_partials.as<double2>();
  GB_DISPATCH2(p.prec, Ra, r.prec, Rb,
               (k_dot2_partial<Ra, Rb><<<nb, kThreads, 0, st>>>(
                   (const cpx<Ra>*)p.p, (const cpx<Rb>*)r.p, p.n, part, kMaxRedBlocks)));
  GB_LAUNCH_CHECK();
  c->launches++;
  finish_reduction(c, nb, s_pr, part, st);
  finish_reduction(c, nb, s_pp, part + kMaxRedBlocks, st);
}

void blas_mr_update(mg_ctx* c, Vec x, Vec r, Vec p, int s_pr, int s_pp, double omega,
                    cudaStream_t st) {
  GB_REQUIRE(x.prec == r.prec && r.prec == p.prec, MG_ERR_ARG, "mr_update: precision mix");
  GB_DISPATCH1(x.prec, R,
               (k_mr_update<R><<<ew_blocks(x.n), kThreads, 0, st>>>(
                   (cpx<R>*)x.p, (cpx<R>*)r.p, (const cpx<R>*)p.p, x.n, scal(c), s_pr, s_pp,
                   omega)));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void blas_scale_invnorm(mg_ctx* c, Vec a, Vec b, int slot, cudaStream_t st) {
  GB_DISPATCH2(a.prec, Ra, b.prec, Rb,
               (k_scale_invnorm<Ra, Rb><<<ew_blocks(a.n), kThreads, 0, st>>>(
                   (cpx<Ra>*)a.p, (cpx<Rb>*)b.p, a.n, scal(c), slot)));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void blas_gcr_update(mg_ctx* c, Vec x, Vec r, Vec z, Vec w, int slot, cudaStream_t st) {
  GB_REQUIRE(x.prec == r.prec && z.prec == w.prec, MG_ERR_ARG, "gcr_update: precision mix");
  GB_DISPATCH2(x.prec, Rx, z.prec, Rz,
               (k_gcr_update<Rx, Rz><<<ew_blocks(x.n), kThreads, 0, st>>>(
                   (cpx<Rx>*)x.p, (cpx<Rx>*)r.p, (const cpx<Rz>*)z.p, (const cpx<Rz>*)w.p, x.n,
                   scal(c), slot)));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void blas_sweep_update(mg_ctx* c, Vec x, Vec t, int s_qt, int s_qq, cudaStream_t st) {
  GB_REQUIRE(x.prec == t.prec, MG_ERR_ARG, "sweep_update: precision mix");
  GB_DISPATCH1(x.prec, R,
               (k_sweep_update<R><<<ew_blocks(x.n), kThreads, 0, st>>>(
                   (cpx<R>*)x.p, (const cpx<R>*)t.p, x.n, scal(c), s_qt, s_qq)));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void blas_read_scalars(mg_ctx* c, int first, int count, double* out, cudaStream_t st) {
  GB_CHECK(cudaMemcpyAsync(c->h_scalars, scal(c) + first, sizeof(double2) * count,
                           cudaMemcpyDeviceToHost, st));
  GB_CHECK(cudaStreamSynchronize(st));
  for (int i = 0; i < 2 * count; ++i) out[i] = c->h_scalars[i];
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

void blas_normalise(mg_ctx* c, Vec x, int slot, cudaStream_t st) {
  GB_DISPATCH1(x.prec, R,
               (k_normalise<R><<<ew_blocks(x.n), kThreads, 0, st>>>((cpx<R>*)x.p, x.n, scal(c),
                                                                     slot)));
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
