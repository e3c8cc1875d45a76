// Shared device/host helpers of the CUDA library: complex arithmetic,
// storage formats, lattice geometry and error handling.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <stdexcept>
#include <string>

#include "gbmg.h"

namespace gbmg {

// ------------------------------------------------------------------ errors
struct Error : std::runtime_error {
  mg_status code;
  Error(mg_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define GB_CHECK(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      throw ::gbmg::Error(e_ == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA, \
                          std::string(#call) + ": " + cudaGetErrorString(e_));      \
  } while (0)

#define GB_REQUIRE(cond, code, msg)                    \
  do {                                                 \
    if (!(cond)) throw ::gbmg::Error((code), (msg));   \
  } while (0)

#define GB_LAUNCH_CHECK() GB_CHECK(cudaGetLastError())

// ------------------------------------------------------------------ complex
template <typename R>
struct alignas(2 * sizeof(R)) cpx {
  R re, im;
  cpx() = default;
  __host__ __device__ constexpr cpx(R r, R i = R(0)) : re(r), im(i) {}
  template <typename S>
  __host__ __device__ explicit cpx(const cpx<S>& o) : re(R(o.re)), im(R(o.im)) {}
};

template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) {
  return cpx<R>(a.re + b.re, a.im + b.im);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) {
  return cpx<R>(a.re - b.re, a.im - b.im);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a) {
  return cpx<R>(-a.re, -a.im);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
  return cpx<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) {
  return cpx<R>(s * a.re, s * a.im);
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R>& operator+=(cpx<R>& a, cpx<R> b) {
  a.re += b.re;
  a.im += b.im;
  return a;
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R>& operator-=(cpx<R>& a, cpx<R> b) {
  a.re -= b.re;
  a.im -= b.im;
  return a;
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> conj(cpx<R> a) {
  return cpx<R>(a.re, -a.im);
}
// a += b * c
template <typename R>
__host__ __device__ __forceinline__ void cmac(cpx<R>& a, cpx<R> b, cpx<R> c) {
  a.re = fma(b.re, c.re, a.re);
  a.re = fma(-b.im, c.im, a.re);
  a.im = fma(b.re, c.im, a.im);
  a.im = fma(b.im, c.re, a.im);
}
// a += conj(b) * c
template <typename R>
__host__ __device__ __forceinline__ void cmac_conj(cpx<R>& a, cpx<R> b, cpx<R> c) {
  a.re = fma(b.re, c.re, a.re);
  a.re = fma(b.im, c.im, a.re);
  a.im = fma(b.re, c.im, a.im);
  a.im = fma(-b.im, c.re, a.im);
}
// i * a
template <typename R>
__host__ __device__ __forceinline__ cpx<R> times_i(cpx<R> a) {
  return cpx<R>(-a.im, a.re);
}
template <typename R>
__host__ __device__ __forceinline__ R norm2(cpx<R> a) {
  return a.re * a.re + a.im * a.im;
}

// ------------------------------------------------------------------ storage
// Complex element types of the link store.  16-bit forms carry a per-site
// FP32 scale: value = scale * stored.
struct bf16c {
  __nv_bfloat162 v;
};
struct f16c {
  __half2 v;
};

// 16-bit fixed point: q = round(value / scale * 32767), |value| <= scale
struct i16c {
  short2 v;
};

template <typename S>
struct StoreTraits;
template <>
struct StoreTraits<cpx<double>> {
  using real = double;
  static constexpr bool scaled = false;
  __device__ static __forceinline__ cpx<double> load(cpx<double> s) { return s; }
};
template <>
struct StoreTraits<cpx<float>> {
  using real = float;
  static constexpr bool scaled = false;
  __device__ static __forceinline__ cpx<float> load(cpx<float> s) { return s; }
};
template <>
struct StoreTraits<bf16c> {
  using real = float;
  static constexpr bool scaled = true;
  __device__ static __forceinline__ cpx<float> load(bf16c s) {
    float2 f = __bfloat1622float2(s.v);
    return cpx<float>(f.x, f.y);
  }
  __device__ static __forceinline__ bf16c pack(cpx<float> c) {
    bf16c r;
    r.v = __floats2bfloat162_rn(c.re, c.im);
    return r;
  }
};
template <>
struct StoreTraits<f16c> {
  using real = float;
  static constexpr bool scaled = true;
  __device__ static __forceinline__ cpx<float> load(f16c s) {
    float2 f = __half22float2(s.v);
    return cpx<float>(f.x, f.y);
  }
  __device__ static __forceinline__ f16c pack(cpx<float> c) {
    f16c r;
    r.v = __floats2half2_rn(c.re, c.im);
    return r;
  }
};

template <>
struct StoreTraits<i16c> {
  using real = float;
  static constexpr bool scaled = true;
  __device__ static __forceinline__ cpx<float> load(i16c s) {
    return cpx<float>(float(s.v.x) * (1.f / 32767.f), float(s.v.y) * (1.f / 32767.f));
  }
  __device__ static __forceinline__ i16c pack(cpx<float> c) {
    i16c r;
    r.v.x = short(__float2int_rn(fminf(fmaxf(c.re, -1.f), 1.f) * 32767.f));
    r.v.y = short(__float2int_rn(fminf(fmaxf(c.im, -1.f), 1.f) * 32767.f));
    return r;
  }
};

inline bool prec_is16(mg_prec p) { return p == MG_BF16 || p == MG_F16 || p == MG_I16; }

inline size_t prec_bytes_complex(mg_prec p) {
  switch (p) {
    case MG_F64: return 16;
    case MG_F32: return 8;
    default: return 4;
  }
}
inline mg_prec vec_prec_of(mg_prec p) { return p == MG_F64 ? MG_F64 : MG_F32; }

// ------------------------------------------------------------------ geometry
// Site index s = x + Lx*(y + Ly*(z + Lz*t)); stencil slot d: 0 = site,
// 1 + 2mu = +mu neighbour, 2 + 2mu = -mu neighbour (periodic).
struct Geom {
  int L[4];
  int stride[4];
  int vol;
};

inline Geom make_geom(const int d[4]) {
  Geom g;
  int s = 1;
  for (int m = 0; m < 4; ++m) {
    g.L[m] = d[m];
    g.stride[m] = s;
    s *= d[m];
  }
  g.vol = s;
  return g;
}

__host__ __device__ __forceinline__ void site_coords(const Geom& g, int s, int c[4]) {
  c[0] = s % g.L[0];
  s /= g.L[0];
  c[1] = s % g.L[1];
  s /= g.L[1];
  c[2] = s % g.L[2];
  c[3] = s / g.L[2];
}

// neighbour of site s (coordinates c) in slot d
__host__ __device__ __forceinline__ int neighbour(const Geom& g, int s, const int c[4], int d) {
  if (d == 0) return s;
  int mu = (d - 1) >> 1;
  bool fwd = ((d - 1) & 1) == 0;
  if (fwd) return (c[mu] == g.L[mu] - 1) ? s - (g.L[mu] - 1) * g.stride[mu] : s + g.stride[mu];
  return (c[mu] == 0) ? s + (g.L[mu] - 1) * g.stride[mu] : s - g.stride[mu];
}

// ------------------------------------------------------------------ loads
// Streaming 16-byte load that bypasses L1 allocation (each link byte is
// used once per apply).
__device__ __forceinline__ uint4 ld_stream16(const void* p) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}

// The same load with an L2 cache policy (createpolicy): evict-last for data
// another CTA reads again soon, evict-first for data's last use.
__device__ __forceinline__ uint4 ld_stream16_hint(const void* p, uint64_t pol) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

inline int ceil_div(long long a, long long b) { return int((a + b - 1) / b); }

}  // namespace gbmg
