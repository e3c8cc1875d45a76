// Element access shared by the coarse-operator kernels (coarse.cu, the
// red-black kernels of schur.cu): a 16-byte chunk of link rows unpacked to
// FP32 / FP64 complex numbers, RPC rows per chunk.
#pragma once

#include "common.cuh"

namespace gbmg {

template <typename S>
struct Unpack;
template <>
struct Unpack<cpx<double>> {
  static constexpr int RPC = 1;
  __device__ static __forceinline__ void get(uint4 v, cpx<double> out[1]) {
    out[0] = cpx<double>(__hiloint2double(int(v.y), int(v.x)), __hiloint2double(int(v.w), int(v.z)));
  }
};
template <>
struct Unpack<cpx<float>> {
  static constexpr int RPC = 2;
  __device__ static __forceinline__ void get(uint4 v, cpx<float> out[2]) {
    out[0] = cpx<float>(__uint_as_float(v.x), __uint_as_float(v.y));
    out[1] = cpx<float>(__uint_as_float(v.z), __uint_as_float(v.w));
  }
};
template <>
struct Unpack<bf16c> {
  static constexpr int RPC = 4;
  __device__ static __forceinline__ void get(uint4 v, cpx<float> out[4]) {
    uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      out[i] = cpx<float>(__uint_as_float(w[i] << 16), __uint_as_float(w[i] & 0xffff0000u));
    }
  }
};
template <>
struct Unpack<f16c> {
  static constexpr int RPC = 4;
  __device__ static __forceinline__ void get(uint4 v, cpx<float> out[4]) {
    uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __half2 h = *reinterpret_cast<__half2*>(&w[i]);
      float2 f = __half22float2(h);
      out[i] = cpx<float>(f.x, f.y);
    }
  }
};

template <>
struct Unpack<i16c> {
  static constexpr int RPC = 4;
  __device__ static __forceinline__ void get(uint4 v, cpx<float> out[4]) {
    uint32_t w[4] = {v.x, v.y, v.z, v.w};
    const float s = 1.f / 32767.f;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      out[i] = cpx<float>(float(short(w[i] & 0xffffu)) * s, float(short(w[i] >> 16)) * s);
  }
};

constexpr int batch_of(int iters, int umax = 8) {
  for (int u = umax; u > 1; --u)
    if (iters % u == 0) return u;
  return 1;
}

}  // namespace gbmg
