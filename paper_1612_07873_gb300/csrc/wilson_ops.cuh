// Device building blocks of the Wilson-clover matrix, Eq. (2):
//   M = -1/2 sum_mu [ (1 - g_mu) (x) U_mu(x) d_{x+mu,x'} + (1 + g_mu) (x) U_mu(x-mu)^dag d_{x-mu,x'} ]
//       + (4 + m + A_x) d_{x,x'}
// in the DeGrand-Rossi chiral basis, where every gamma_mu = [[0, B],[C, 0]]
// is off-diagonal in chirality with CB = 1.  Hence
//   (1 - g) psi = [h ; -C h],  h = psi_u - B psi_l,
//   (1 + g) psi = [h ;  C h],  h = psi_u + B psi_l,
// and a hop costs one colour multiply of a 2-spinor.
// Spinor dof = spin*3 + colour; spins 0,1 (upper) are chirality 0.
#pragma once

#include "common.cuh"

namespace gbmg {

// (B_mu l) for the lower 2-spinor l = (l0, l1) of one colour.
template <int MU, typename R>
__device__ __forceinline__ void Bmul(cpx<R> l0, cpx<R> l1, cpx<R>& o0, cpx<R>& o1) {
  if constexpr (MU == 0) {         // B = i s1
    o0 = times_i(l1);
    o1 = times_i(l0);
  } else if constexpr (MU == 1) {  // B = -i s2 = [[0,-1],[1,0]]
    o0 = -l1;
    o1 = l0;
  } else if constexpr (MU == 2) {  // B = i s3
    o0 = times_i(l0);
    o1 = -times_i(l1);
  } else {                         // B = 1
    o0 = l0;
    o1 = l1;
  }
}

// (C_mu u) for the upper 2-spinor u of one colour.
template <int MU, typename R>
__device__ __forceinline__ void Cmul(cpx<R> u0, cpx<R> u1, cpx<R>& o0, cpx<R>& o1) {
  if constexpr (MU == 0) {         // C = -i s1
    o0 = -times_i(u1);
    o1 = -times_i(u0);
  } else if constexpr (MU == 1) {  // C = i s2 = [[0,1],[-1,0]]
    o0 = u1;
    o1 = -u0;
  } else if constexpr (MU == 2) {  // C = -i s3
    o0 = -times_i(u0);
    o1 = times_i(u1);
  } else {                         // C = 1
    o0 = u0;
    o1 = u1;
  }
}

// acc += -1/2 (1 - g_mu) (x) U  psi     (forward hop, U = U_mu(x))
// acc += -1/2 (1 + g_mu) (x) U^dag psi  (backward hop, U = U_mu(x - mu))
template <int MU, bool FWD, typename R>
__device__ __forceinline__ void hop_accum(const cpx<R>* __restrict__ U, const cpx<R> psi[12],
                                          cpx<R> acc[12]) {
  cpx<R> h[2][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    cpx<R> b0, b1;
    Bmul<MU>(psi[6 + k], psi[9 + k], b0, b1);
    if (FWD) {
      h[0][k] = psi[k] - b0;
      h[1][k] = psi[3 + k] - b1;
    } else {
      h[0][k] = psi[k] + b0;
      h[1][k] = psi[3 + k] + b1;
    }
  }
  cpx<R> w[2][3];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cpx<R> t(R(0), R(0));
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (FWD)
          cmac(t, U[a * 3 + b], h[s][b]);
        else
          cmac_conj(t, U[b * 3 + a], h[s][b]);  // (U^dag)_{ab} = conj(U_{ba})
      }
      w[s][a] = t;
    }
  const R half = R(0.5);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cpx<R> c0, c1;
    Cmul<MU>(w[0][a], w[1][a], c0, c1);
    acc[a] -= half * w[0][a];
    acc[3 + a] -= half * w[1][a];
    if (FWD) {
      acc[6 + a] += half * c0;
      acc[9 + a] += half * c1;
    } else {
      acc[6 + a] -= half * c0;
      acc[9 + a] -= half * c1;
    }
  }
}

// Runtime-mu dispatch of hop_accum.
template <typename R>
__device__ __forceinline__ void hop_accum_rt(int mu, bool fwd, const cpx<R>* __restrict__ U,
                                             const cpx<R> psi[12], cpx<R> acc[12]) {
  switch (mu * 2 + (fwd ? 0 : 1)) {
    case 0: hop_accum<0, true>(U, psi, acc); break;
    case 1: hop_accum<0, false>(U, psi, acc); break;
    case 2: hop_accum<1, true>(U, psi, acc); break;
    case 3: hop_accum<1, false>(U, psi, acc); break;
    case 4: hop_accum<2, true>(U, psi, acc); break;
    case 5: hop_accum<2, false>(U, psi, acc); break;
    case 6: hop_accum<3, true>(U, psi, acc); break;
    default: hop_accum<3, false>(U, psi, acc); break;
  }
}

// acc += (diag + A_x) psi with A_x stored as two packed 6x6 Hermitian blocks
// (per chirality: 6 real diagonal entries, then the 15 complex entries
// below the diagonal in row order).
template <typename R>
__device__ __forceinline__ void clover_accum(const R* __restrict__ A, R diag, const cpx<R> psi[12],
                                             cpx<R> acc[12]) {
#pragma unroll
  for (int chi = 0; chi < 2; ++chi) {
    const R* a = A + chi * 36;
    const cpx<R>* in = psi + chi * 6;
    cpx<R>* out = acc + chi * 6;
#pragma unroll
    for (int i = 0; i < 6; ++i) out[i] += (diag + a[i]) * in[i];
#pragma unroll
    for (int i = 1; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < i; ++j) {
        int k = i * (i - 1) / 2 + j;
        cpx<R> l(a[6 + 2 * k], a[7 + 2 * k]);
        cmac(out[i], l, in[j]);
        cmac_conj(out[j], l, in[i]);
      }
  }
}

// clover_accum with element k of the packed clover at A[k * stride] (a
// transposed shared-memory tile).
template <typename R>
__device__ __forceinline__ void clover_accum_strided(const R* __restrict__ A, int stride, R diag,
                                                     const cpx<R> psi[12], cpx<R> acc[12]) {
#pragma unroll
  for (int chi = 0; chi < 2; ++chi) {
    const R* a = A + chi * 36 * stride;
    const cpx<R>* in = psi + chi * 6;
    cpx<R>* out = acc + chi * 6;
#pragma unroll
    for (int i = 0; i < 6; ++i) out[i] += (diag + a[i * stride]) * in[i];
#pragma unroll
    for (int i = 1; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < i; ++j) {
        int k = i * (i - 1) / 2 + j;
        cpx<R> l(a[(6 + 2 * k) * stride], a[(7 + 2 * k) * stride]);
        cmac(out[i], l, in[j]);
        cmac_conj(out[j], l, in[i]);
      }
  }
}

// acc6 += (diag + A_chi) psi6 for one packed 6x6 Hermitian chirality block.
template <typename R>
__device__ __forceinline__ void clover_block_accum(const R* __restrict__ a, R diag,
                                                   const cpx<R> in[6], cpx<R> out[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) out[i] += (diag + a[i]) * in[i];
#pragma unroll
  for (int i = 1; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) {
      int k = i * (i - 1) / 2 + j;
      cpx<R> l(a[6 + 2 * k], a[7 + 2 * k]);
      cmac(out[i], l, in[j]);
      cmac_conj(out[j], l, in[i]);
    }
}

}  // namespace gbmg
