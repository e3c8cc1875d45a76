// Learned null-vector proposer: a three-layer nearest-neighbour-stencil
// network (the "4D convolution" of this library) that maps the links around
// a site to Nv starting vectors for the adaptive setup (Sec. 3.4 step 1
// draws them at random; the paper has no learned part).
//
//   p(x)  = cos, sin (2 pi x_mu / L_mu), mu = 0..3                  8 channels
//   f(x)  = (Re, Im) of U_mu(x)[a][b], then p(x)                 72 + 8 channels
//   h1(x) = tanh(b1 + sum_{d=0..8} W1[d] f(x + shift(d)))         -> 32
//   h2(x) = tanh(b2 + sum_{d=0..8} W2[d] h1(x + shift(d)))        -> 32
//   o(x)  = b3 + W3 [h2(x); p(x)]                                 -> 24 Nv
// The links carry no position, and the smooth low modes the setup looks for
// vary slowly across the lattice; the phases p(x) of the lowest lattice
// momenta give the network that position (as inputs of the first layer and
// directly to the output layer).
//   vector i, dof a at x: o[x][24 i + 2 a] + i o[x][24 i + 2 a + 1]
//
// Training loss, per aggregate A and chirality s with B the block of the
// predicted vectors and T the block of target (block-orthonormal) vectors:
//   l = 1 - tr(C^H G^{-1} C) / Nv,  G = B^H B + kappa |B|_F^2 I,  C = B^H T,
// kappa = 1e-5 / Nv, averaged over blocks;
//   dl/dB* = -(T A^H - B A A^H - kappa |A|_F^2 B) / Nv,  A = G^{-1} C.
// Parameters and activations are FP32 (flat: W1, b1, W2, b2, W3, b3); the
// loss and its gradient with respect to the network output are formed in
// FP64 (Gram and cross products, factorisation, gradient rows).  Weight
// gradients are per-weight sums over sites in a fixed order
// (deterministic): FP32 over 32 sites, FP64 beyond.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kernels.cuh"

struct mg_cnn {
  int nvec = 0;
  int nout = 0;
  int nparams = 0;
  int adam_t = 0;
  int vol = 0;
  gbmg::DevBuf theta, grad, m1, m2;
  gbmg::DevBuf f, h1, h2, o, go, g2, g1, blk_loss, part;
  std::string err;
};

namespace gbmg {

namespace {

constexpr int NL = 72, NP = 8;       // link and position channels
constexpr int NF = NL + NP, NH = 32;  // first-layer inputs, hidden channels
constexpr int ND = NH + NP;           // output-layer inputs [h2; p]

struct Offsets {
  int W1, b1, W2, b2, W3, b3, total;
};
Offsets offsets(int nout) {
  Offsets o;
  o.W1 = 0;
  o.b1 = o.W1 + 9 * NH * NF;
  o.W2 = o.b1 + NH;
  o.b2 = o.W2 + 9 * NH * NH;
  o.W3 = o.b2 + NH;
  o.b3 = o.W3 + nout * ND;
  o.total = o.b3 + nout;
  return o;
}

int blocks_for(size_t n) {
  long long b = (long long)((n + 255) / 256);
  if (b > 152 * 32) b = 152 * 32;
  return int(b < 1 ? 1 : b);
}

// f [V][NF] (links, then positions) and the position channels of the
// output-layer input hp [V][ND]
__global__ void k_features(float* __restrict__ f, float* __restrict__ hp,
                           const cpx<double>* __restrict__ U, Geom g) {
  const int vol = g.vol;
  const size_t total = size_t(vol) * 40;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total;
       i += size_t(gridDim.x) * blockDim.x) {
    const int x = int(i / 40), k = int(i - size_t(x) * 40);
    if (k < 36) {
      const int mu = k / 9, ab = k - mu * 9;
      const cpx<double> u = U[(size_t(mu) * vol + x) * 9 + ab];
      f[size_t(x) * NF + 2 * k] = float(u.re);
      f[size_t(x) * NF + 2 * k + 1] = float(u.im);
    } else {
      const int mu = k - 36;
      int c[4];
      site_coords(g, x, c);
      float sn, cs;
      sincospif(2.f * float(c[mu]) / float(g.L[mu]), &sn, &cs);
      f[size_t(x) * NF + NL + 2 * mu] = cs;
      f[size_t(x) * NF + NL + 2 * mu + 1] = sn;
      hp[size_t(x) * ND + NH + 2 * mu] = cs;
      hp[size_t(x) * ND + NH + 2 * mu + 1] = sn;
    }
  }
}

// out(x)[c] = tanh(b[c] + sum_d sum_k W[d][c][k] in(x + shift(d))[k]); thread (x, c);
// output rows OS floats apart
template <int CIN, int OS>
__global__ void k_conv9_tanh(float* __restrict__ out, const float* __restrict__ in,
                             const float* __restrict__ W, const float* __restrict__ b, Geom g) {
  const size_t total = size_t(g.vol) * NH;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total;
       i += size_t(gridDim.x) * blockDim.x) {
    const int x = int(i / NH), c = int(i - size_t(x) * NH);
    int cc[4];
    site_coords(g, x, cc);
    float acc = b[c];
    for (int d = 0; d < 9; ++d) {
      const float* src = in + size_t(neighbour(g, x, cc, d)) * CIN;
      const float* w = W + (size_t(d) * NH + c) * CIN;
#pragma unroll 8
      for (int k = 0; k < CIN; ++k) acc = fmaf(__ldg(w + k), src[k], acc);
    }
    out[size_t(x) * OS + c] = tanhf(acc);
  }
}

// o(x)[j] = b3[j] + sum_c W3[j][c] hp(x)[c],  hp = [h2; p]
__global__ void k_dense(float* __restrict__ o, const float* __restrict__ h2,
                        const float* __restrict__ W3, const float* __restrict__ b3, int vol,
                        int nout) {
  const size_t total = size_t(vol) * nout;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total;
       i += size_t(gridDim.x) * blockDim.x) {
    const int x = int(i / nout), j = int(i - size_t(x) * nout);
    const float* h = h2 + size_t(x) * ND;
    const float* w = W3 + size_t(j) * ND;
    float acc = b3[j];
#pragma unroll
    for (int c = 0; c < ND; ++c) acc = fmaf(__ldg(w + c), h[c], acc);
    o[i] = acc;
  }
}

// o [V][24 Nv] -> vectors [Nv][V][12] complex double
__global__ void k_to_vectors(cpx<double>* __restrict__ v, const float* __restrict__ o, int vol,
                             int nvec) {
  const size_t total = size_t(nvec) * vol * 12;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total;
       i += size_t(gridDim.x) * blockDim.x) {
    const int a = int(i % 12);
    const size_t t = i / 12;
    const int x = int(t % vol), iv = int(t / vol);
    const float* src = o + size_t(x) * 24 * nvec + 24 * iv + 2 * a;
    v[i] = cpx<double>(double(src[0]), double(src[1]));
  }
}

struct AggInfo {
  Geom fine, coarse;
  int b[4];
  int per;
};

__device__ __forceinline__ int agg_site(const AggInfo& m, int xc, int ls) {
  int cc[4];
  site_coords(m.coarse, xc, cc);
  const int l0 = ls % m.b[0];
  ls /= m.b[0];
  const int l1 = ls % m.b[1];
  ls /= m.b[1];
  const int l2 = ls % m.b[2];
  const int l3 = ls / m.b[2];
  return (cc[0] * m.b[0] + l0) + m.fine.stride[1] * (cc[1] * m.b[1] + l1) +
         m.fine.stride[2] * (cc[2] * m.b[2] + l2) + m.fine.stride[3] * (cc[3] * m.b[3] + l3);
}

constexpr int KCH = 32;  // rows per shared-memory chunk
constexpr int NVMAX = 32;

// One CTA per (aggregate, chirality) block; see the file comment.  Every
// quantity of the loss and of dl/dB is formed in FP64: B (the FP32 network
// output, exact in FP64), T (FP64), the Gram matrix G, the cross products C,
// the factorisation and the gradient rows.  Only the gradient rows written
// for the backward pass are rounded to FP32.
__global__ void __launch_bounds__(256) k_subspace_loss(
    float* __restrict__ go, float* __restrict__ blk_loss, const float* __restrict__ o,
    const cpx<double>* __restrict__ tgt, AggInfo m, int nvec, float gscale) {
  extern __shared__ unsigned char smem_raw[];
  cpx<double>* Bs = reinterpret_cast<cpx<double>*>(smem_raw);  // [KCH][nvec]
  cpx<double>* Ts = Bs + KCH * nvec;                           // [KCH][nvec]
  cpx<double>* G = Ts + KCH * nvec;                            // [nvec][nvec]
  cpx<double>* C = G + nvec * nvec;                            // [nvec][nvec]
  cpx<double>* AH = C + nvec * nvec;                           // A^H
  cpx<double>* M2 = AH + nvec * nvec;                          // A A^H
  const int blk = blockIdx.x;
  const int xc = blk >> 1, chi = blk & 1;
  const int rows = m.per * 6;
  const int nv2 = nvec * nvec;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nout = 24 * nvec;
  auto load_chunk = [&](int r0) {
    for (int k = tid; k < KCH * nvec; k += 256) {
      const int rr = k / nvec, i = k - rr * nvec, row = r0 + rr;
      cpx<double> bv(0.0, 0.0), tv(0.0, 0.0);
      if (row < rows) {
        const int ls = row / 6, a = row - ls * 6, dof = chi * 6 + a;
        const int x = agg_site(m, xc, ls);
        const float* src = o + size_t(x) * nout + 24 * i + 2 * dof;
        bv = cpx<double>(double(src[0]), double(src[1]));
        tv = tgt[(size_t(i) * m.fine.vol + x) * 12 + dof];
      }
      Bs[k] = bv;
      Ts[k] = tv;
    }
  };
  // ---- G = B^H B, C = B^H T
  constexpr int EPT = (2 * NVMAX * NVMAX + 255) / 256;
  cpx<double> acc[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) acc[e] = cpx<double>(0.0, 0.0);
  for (int r0 = 0; r0 < rows; r0 += KCH) {
    load_chunk(r0);
    __syncthreads();
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const int q = tid + 256 * e;
      if (q < 2 * nv2) {
        const int which = q / nv2, ij = q - which * nv2;
        const int i = ij / nvec, j = ij - i * nvec;
        const cpx<double>* R = which ? Ts : Bs;
        cpx<double> a_ = acc[e];
        for (int rr = 0; rr < KCH; ++rr) cmac_conj(a_, Bs[rr * nvec + i], R[rr * nvec + j]);
        acc[e] = a_;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int q = tid + 256 * e;
    if (q < 2 * nv2) {
      const int which = q / nv2, ij = q - which * nv2;
      (which ? C : G)[ij] = acc[e];
    }
  }
  __syncthreads();
  // ---- warp 0: G += kappa tr(G) I, Cholesky G = L L^H (lane i owns row i),
  // then A = G^{-1} C in place of C (lane c owns column c)
  __shared__ double a2_sh;
  if (warp == 0) {
    double trG = lane < nvec ? G[lane * nvec + lane].re : 0.0;
    for (int off = 16; off > 0; off >>= 1) trG += __shfl_xor_sync(0xffffffffu, trG, off);
    if (lane < nvec) G[lane * nvec + lane].re += 1e-5 / nvec * trG;
    __syncwarp();
    for (int j = 0; j < nvec; ++j) {  // lower triangle of G becomes L
      if (lane == j) {
        double dsum = G[j * nvec + j].re;
        for (int k = 0; k < j; ++k) dsum -= norm2(G[j * nvec + k]);
        G[j * nvec + j] = cpx<double>(sqrt(fmax(dsum, 1e-300)), 0.0);
      }
      __syncwarp();
      if (lane > j && lane < nvec) {
        const double ljj = G[j * nvec + j].re;
        cpx<double> s = G[lane * nvec + j];
        for (int k = 0; k < j; ++k) s -= G[lane * nvec + k] * conj(G[j * nvec + k]);
        G[lane * nvec + j] = (1.0 / ljj) * s;
      }
      __syncwarp();
    }
    double a2 = 0.0;
    if (lane < nvec) {  // solve L L^H a = C[:, c], c = lane
      const int c = lane;
      for (int i = 0; i < nvec; ++i) {
        cpx<double> s = C[i * nvec + c];
        for (int k = 0; k < i; ++k) s -= G[i * nvec + k] * C[k * nvec + c];
        C[i * nvec + c] = (1.0 / G[i * nvec + i].re) * s;
      }
      for (int i = nvec - 1; i >= 0; --i) {
        cpx<double> s = C[i * nvec + c];
        for (int k = i + 1; k < nvec; ++k) s -= conj(G[k * nvec + i]) * C[k * nvec + c];
        C[i * nvec + c] = (1.0 / G[i * nvec + i].re) * s;
        a2 += norm2(C[i * nvec + c]);
      }
    }
    for (int off = 16; off > 0; off >>= 1) a2 += __shfl_xor_sync(0xffffffffu, a2, off);
    if (lane == 0) a2_sh = a2;
  }
  __syncthreads();
  const double ka2 = 1e-5 / nvec * a2_sh;
  // C now holds A.  f = Re tr(C0^H A) needs the original C: it is still in
  // the accumulators of this thread's entries.
  double fpart = 0.0;
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int q = tid + 256 * e;
    if (q >= nv2 && q < 2 * nv2) {
      const int ij = q - nv2;
      fpart += acc[e].re * C[ij].re + acc[e].im * C[ij].im;
    }
  }
  // A^H and A A^H
  for (int q = tid; q < nv2; q += 256) {
    const int i = q / nvec, j = q - i * nvec;
    AH[q] = conj(C[j * nvec + i]);
    cpx<double> s(0.0, 0.0);
    for (int k = 0; k < nvec; ++k) s += C[i * nvec + k] * conj(C[j * nvec + k]);
    M2[q] = s;
  }
  // block sum of fpart
  __shared__ double red[8];
  for (int off = 16; off > 0; off >>= 1) fpart += __shfl_xor_sync(0xffffffffu, fpart, off);
  if (lane == 0) red[warp] = fpart;
  __syncthreads();
  if (tid == 0) {
    double f = 0.0;
    for (int w = 0; w < 8; ++w) f += red[w];
    blk_loss[blk] = float(1.0 - f / nvec);
  }
  // ---- gradient rows: Gamma = T A^H - B (A A^H) - kappa |A|_F^2 B;
  // dO = -2 gscale (Re, Im) Gamma
  for (int r0 = 0; r0 < rows; r0 += KCH) {
    load_chunk(r0);
    __syncthreads();
    for (int k = tid; k < KCH * nvec; k += 256) {
      const int rr = k / nvec, i = k - rr * nvec, row = r0 + rr;
      if (row >= rows) continue;
      cpx<double> gam = -ka2 * Bs[rr * nvec + i];
      for (int j = 0; j < nvec; ++j) {
        cmac(gam, Ts[rr * nvec + j], AH[j * nvec + i]);
        cmac(gam, -Bs[rr * nvec + j], M2[j * nvec + i]);
      }
      const int ls = row / 6, a = row - ls * 6, dof = chi * 6 + a;
      const int x = agg_site(m, xc, ls);
      float* dst = go + size_t(x) * nout + 24 * i + 2 * dof;
      dst[0] = float(-2.0 * gscale * gam.re);
      dst[1] = float(-2.0 * gscale * gam.im);
    }
    __syncthreads();
  }
}

// dh2(x)[c] = sum_j W3[j][c] go(x)[j], times (1 - h2^2)
__global__ void k_dense_back_in(float* __restrict__ g2, const float* __restrict__ go,
                                const float* __restrict__ W3, const float* __restrict__ h2,
                                int vol, int nout) {
  const size_t total = size_t(vol) * NH;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total;
       i += size_t(gridDim.x) * blockDim.x) {
    const int x = int(i / NH), c = int(i - size_t(x) * NH);
    const float* gx = go + size_t(x) * nout;
    float acc = 0.f;
    for (int j = 0; j < nout; ++j) acc = fmaf(__ldg(W3 + size_t(j) * ND + c), gx[j], acc);
    const float h = h2[size_t(x) * ND + c];
    g2[i] = acc * (1.f - h * h);
  }
}

// Segmented weight gradient  P[seg][d][co][k] = sum_{x in seg} gp(x)[co] in(src_d(x))[k]
// with src_d(x) = x + shift(d) (conv layers, d < 9) or x (dense layer, d = 0
// with ndir = 1).  Grid (segment, d, 32-row chunk of co); sites staged in
// shared memory 32 at a time, the 32-site partial sum formed in FP32 and
// added to an FP64 accumulator; a second kernel sums the segments in order.
constexpr int WSEG = 1024;  // sites per segment
template <int CI>
__global__ void __launch_bounds__(256) k_wgrad_seg(double* __restrict__ part,
                                                   const float* __restrict__ gp, int co_total,
                                                   const float* __restrict__ in, Geom g, int ndir) {
  __shared__ float sg[32][33];
  __shared__ float si[32][CI + 1];
  const int seg = blockIdx.x, d = blockIdx.y, co0 = blockIdx.z * 32;
  const int tid = threadIdx.x;
  constexpr int OPT = (32 * CI + 255) / 256;
  double acc[OPT];
#pragma unroll
  for (int e = 0; e < OPT; ++e) acc[e] = 0.0;
  const int x0 = seg * WSEG, x1 = min(g.vol, x0 + WSEG);
  for (int xb = x0; xb < x1; xb += 32) {
    for (int q = tid; q < 32 * 32; q += 256) {
      const int r = q >> 5, c = q & 31, x = xb + r;
      sg[r][c] = (x < x1 && co0 + c < co_total) ? gp[size_t(x) * co_total + co0 + c] : 0.f;
    }
    for (int q = tid; q < 32 * CI; q += 256) {
      const int r = q / CI, k = q - r * CI, x = xb + r;
      float v = 0.f;
      if (x < x1) {
        int src = x;
        if (ndir > 1) {
          int cc[4];
          site_coords(g, x, cc);
          src = neighbour(g, x, cc, d);
        }
        v = in[size_t(src) * CI + k];
      }
      si[r][k] = v;
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < OPT; ++e) {
      const int o = tid + 256 * e;
      if (o < 32 * CI) {
        const int c = o / CI, k = o - c * CI;
        float a = 0.f;
#pragma unroll 8
        for (int r = 0; r < 32; ++r) a = fmaf(sg[r][c], si[r][k], a);
        acc[e] += double(a);
      }
    }
    __syncthreads();
  }
  const int nseg = gridDim.x;
#pragma unroll
  for (int e = 0; e < OPT; ++e) {
    const int o = tid + 256 * e;
    if (o < 32 * CI) {
      const int c = o / CI, k = o - c * CI;
      if (co0 + c < co_total)
        part[((size_t(d) * co_total + co0 + c) * CI + k) * nseg + seg] = acc[e];
    }
  }
}

// W[i] = sum_seg part[i][seg] (FP64, rounded once);  bias[co] = sum_x gp(x)[co]
__global__ void k_wgrad_sum(float* __restrict__ W, const double* __restrict__ part, int n,
                            int nseg) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < nseg; ++q) s += part[size_t(i) * nseg + q];
    W[i] = float(s);
  }
}
__global__ void k_bias_grad(float* __restrict__ gb, const float* __restrict__ gp, int vol,
                            int co_total) {
  // one CTA per output channel, fixed-order FP64 tree over sites
  __shared__ double sh[256];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int x = threadIdx.x; x < vol; x += 256) s += double(gp[size_t(x) * co_total + c]);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) gb[c] = float(sh[0]);
}

// slot d' whose partner is the site that uses y in slot d: y = x + shift(d)  <=>  x = y - shift(d)
__device__ __forceinline__ int opposite(int d) { return d == 0 ? 0 : (((d - 1) & 1) ? d - 1 : d + 1); }

// g1(y)[k] = (1 - h1(y)^2) sum_d sum_c W2[d][c][k] gp2(y - shift(d))[c]
__global__ void k_conv9_back_in_tanh(float* __restrict__ g1, const float* __restrict__ gp2,
                                     const float* __restrict__ W2, const float* __restrict__ h1,
                                     Geom g) {
  const size_t total = size_t(g.vol) * NH;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total;
       i += size_t(gridDim.x) * blockDim.x) {
    const int y = int(i / NH), k = int(i - size_t(y) * NH);
    int cc[4];
    site_coords(g, y, cc);
    float acc = 0.f;
    for (int d = 0; d < 9; ++d) {
      const int x = neighbour(g, y, cc, opposite(d));
      const float* gx = gp2 + size_t(x) * NH;
      const float* w = W2 + size_t(d) * NH * NH + k;
#pragma unroll 8
      for (int c = 0; c < NH; ++c) acc = fmaf(__ldg(w + c * NH), gx[c], acc);
    }
    const float h = h1[i];
    g1[i] = acc * (1.f - h * h);
  }
}

__global__ void k_adam(float* __restrict__ th, float* __restrict__ m1, float* __restrict__ m2,
                       const float* __restrict__ gr, int n, float lr, float b1, float b2,
                       float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = gr[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    th[i] -= lr * (a / c1) / (sqrtf(b / c2) + 1e-8f);
  }
}

__global__ void k_init_params(float* th, int n, Offsets o, uint64_t seed) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float scale;
    if (i < o.b1) scale = rsqrtf(9.f * NF);
    else if (i < o.W2) scale = 0.f;
    else if (i < o.b2) scale = rsqrtf(9.f * NH);
    else if (i < o.W3) scale = 0.f;
    else if (i < o.b3) scale = rsqrtf(float(ND));
    else scale = 0.f;
    // splitmix64 hash -> two uniforms -> Box-Muller
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * uint64_t(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const float u1 = (float(uint32_t(z)) + 1.f) * 2.3283064e-10f;
    const float u2 = float(uint32_t(z >> 32)) * 2.3283064e-10f;
    th[i] = scale * sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
  }
}

void ensure_ws(mg_cnn* n, int vol) {
  if (n->vol == vol) return;
  n->f.alloc(size_t(vol) * NF * 4);
  n->h1.alloc(size_t(vol) * NH * 4);
  n->h2.alloc(size_t(vol) * ND * 4);
  n->o.alloc(size_t(vol) * n->nout * 4);
  n->go.alloc(size_t(vol) * n->nout * 4);
  n->g2.alloc(size_t(vol) * NH * 4);
  n->g1.alloc(size_t(vol) * NH * 4);
  n->vol = vol;
}

void forward(mg_cnn* n, const Geom& g, const void* gauge, cudaStream_t st) {
  ensure_ws(n, g.vol);
  const Offsets o = offsets(n->nout);
  const float* th = n->theta.as<float>();
  k_features<<<blocks_for(size_t(g.vol) * 40), 256, 0, st>>>(n->f.as<float>(), n->h2.as<float>(),
                                                             (const cpx<double>*)gauge, g);
  k_conv9_tanh<NF, NH><<<blocks_for(size_t(g.vol) * NH), 256, 0, st>>>(
      n->h1.as<float>(), n->f.as<float>(), th + o.W1, th + o.b1, g);
  k_conv9_tanh<NH, ND><<<blocks_for(size_t(g.vol) * NH), 256, 0, st>>>(
      n->h2.as<float>(), n->h1.as<float>(), th + o.W2, th + o.b2, g);
  k_dense<<<blocks_for(size_t(g.vol) * n->nout), 256, 0, st>>>(n->o.as<float>(), n->h2.as<float>(),
                                                               th + o.W3, th + o.b3, g.vol,
                                                               n->nout);
  GB_LAUNCH_CHECK();
}

}  // namespace

}  // namespace gbmg

using namespace gbmg;

namespace {
thread_local std::string g_cnn_error;
template <typename F>
mg_status cnn_guard(mg_cnn* n, F&& f) {
  try {
    f();
    return MG_OK;
  } catch (const Error& e) {
    if (n) n->err = e.what();
    g_cnn_error = e.what();
    set_last_error(e.what());
    return e.code;
  }
}
Geom geom_of(const int dims[4]) {
  GB_REQUIRE(dims, MG_ERR_ARG, "cnn: null dims");
  for (int m = 0; m < 4; ++m) GB_REQUIRE(dims[m] >= 1, MG_ERR_ARG, "cnn: bad lattice extent");
  return make_geom(dims);
}
}  // namespace

extern "C" {

mg_status mg_cnn_create(int nvec, uint64_t seed, mg_cnn** out) {
  if (!out) return MG_ERR_ARG;
  *out = nullptr;
  if (nvec < 1 || nvec > NVMAX) {
    set_last_error("cnn: nvec must be 1..32");
    return MG_ERR_ARG;
  }
  mg_cnn* n = new mg_cnn();
  mg_status s = cnn_guard(n, [&] {
    n->nvec = nvec;
    n->nout = 24 * nvec;
    const Offsets o = offsets(n->nout);
    n->nparams = o.total;
    n->theta.alloc(size_t(o.total) * 4);
    n->grad.alloc(size_t(o.total) * 4);
    n->m1.alloc(size_t(o.total) * 4);
    n->m2.alloc(size_t(o.total) * 4);
    GB_CHECK(cudaMemset(n->m1.p, 0, n->m1.bytes));
    GB_CHECK(cudaMemset(n->m2.p, 0, n->m2.bytes));
    GB_CHECK(cudaMemset(n->grad.p, 0, n->grad.bytes));
    k_init_params<<<blocks_for(o.total), 256>>>(n->theta.as<float>(), o.total, o, seed);
    GB_LAUNCH_CHECK();
    GB_CHECK(cudaDeviceSynchronize());
  });
  if (s != MG_OK) {
    delete n;
    return s;
  }
  *out = n;
  return MG_OK;
}

mg_status mg_cnn_destroy(mg_cnn* n) {
  if (!n) return MG_ERR_ARG;
  cudaDeviceSynchronize();
  delete n;
  return MG_OK;
}

mg_status mg_cnn_nparams(mg_cnn* n, int* count) {
  if (!n || !count) return MG_ERR_ARG;
  *count = n->nparams;
  return MG_OK;
}

mg_status mg_cnn_set_params(mg_cnn* n, const void* src_dev, size_t bytes, void* stream) {
  return cnn_guard(n, [&] {
    GB_REQUIRE(n && src_dev && bytes == size_t(n->nparams) * 4, MG_ERR_ARG, "cnn: size mismatch");
    GB_CHECK(cudaMemcpyAsync(n->theta.p, src_dev, bytes, cudaMemcpyDeviceToDevice,
                             (cudaStream_t)stream));
    n->adam_t = 0;
    GB_CHECK(cudaMemsetAsync(n->m1.p, 0, n->m1.bytes, (cudaStream_t)stream));
    GB_CHECK(cudaMemsetAsync(n->m2.p, 0, n->m2.bytes, (cudaStream_t)stream));
  });
}

mg_status mg_cnn_get_params(mg_cnn* n, void* dst_dev, size_t bytes, int which, void* stream) {
  return cnn_guard(n, [&] {
    GB_REQUIRE(n && dst_dev && bytes == size_t(n->nparams) * 4, MG_ERR_ARG, "cnn: size mismatch");
    GB_REQUIRE(which == 0 || which == 1, MG_ERR_ARG, "cnn: which must be 0 or 1");
    GB_CHECK(cudaMemcpyAsync(dst_dev, which ? n->grad.p : n->theta.p, bytes,
                             cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  });
}

mg_status mg_cnn_forward(mg_cnn* n, const int dims[4], const void* gauge_dev, void* vecs_dev,
                         void* stream) {
  return cnn_guard(n, [&] {
    GB_REQUIRE(n && gauge_dev && vecs_dev, MG_ERR_ARG, "cnn: null pointer");
    const Geom g = geom_of(dims);
    cudaStream_t st = (cudaStream_t)stream;
    forward(n, g, gauge_dev, st);
    k_to_vectors<<<blocks_for(size_t(n->nvec) * g.vol * 12), 256, 0, st>>>(
        (cpx<double>*)vecs_dev, n->o.as<float>(), g.vol, n->nvec);
    GB_LAUNCH_CHECK();
  });
}

mg_status mg_cnn_loss_grad(mg_cnn* n, const int dims[4], const int block[4], const void* gauge_dev,
                           const void* target_dev, double* loss, void* stream) {
  return cnn_guard(n, [&] {
    GB_REQUIRE(n && gauge_dev && target_dev && block, MG_ERR_ARG, "cnn: null pointer");
    const Geom g = geom_of(dims);
    int cd[4];
    for (int m = 0; m < 4; ++m) {
      GB_REQUIRE(block[m] >= 1 && dims[m] % block[m] == 0, MG_ERR_ARG,
                 "cnn: extent not divisible by block");
      cd[m] = dims[m] / block[m];
    }
    cudaStream_t st = (cudaStream_t)stream;
    forward(n, g, gauge_dev, st);
    AggInfo m;
    m.fine = g;
    m.coarse = make_geom(cd);
    for (int k = 0; k < 4; ++k) m.b[k] = block[k];
    m.per = g.vol / m.coarse.vol;
    const int nblk = 2 * m.coarse.vol;
    n->blk_loss.alloc(size_t(nblk) * 4);
    const int nv = n->nvec;
    const size_t smem = size_t(2) * KCH * nv * 16 + size_t(4) * nv * nv * 16;
    GB_CHECK(cudaFuncSetAttribute(k_subspace_loss, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(smem)));
    k_subspace_loss<<<nblk, 256, smem, st>>>(n->go.as<float>(), n->blk_loss.as<float>(),
                                              n->o.as<float>(), (const cpx<double>*)target_dev, m,
                                              nv, 1.f / (float(nv) * nblk));
    GB_LAUNCH_CHECK();
    const Offsets o = offsets(n->nout);
    float* gr = n->grad.as<float>();
    const float* th = n->theta.as<float>();
    const int nseg = (g.vol + WSEG - 1) / WSEG;
    const size_t part_elems = size_t(nseg) * std::max(9 * NH * NF, n->nout * ND);
    if (n->part.bytes < part_elems * 8) n->part.alloc(part_elems * 8);
    double* part = n->part.as<double>();
    // dense layer
    k_wgrad_seg<ND><<<dim3(nseg, 1, (n->nout + 31) / 32), 256, 0, st>>>(
        part, n->go.as<float>(), n->nout, n->h2.as<float>(), g, 1);
    k_wgrad_sum<<<blocks_for(size_t(n->nout) * ND), 256, 0, st>>>(gr + o.W3, part,
                                                                  n->nout * ND, nseg);
    k_bias_grad<<<n->nout, 256, 0, st>>>(gr + o.b3, n->go.as<float>(), g.vol, n->nout);
    k_dense_back_in<<<blocks_for(size_t(g.vol) * NH), 256, 0, st>>>(
        n->g2.as<float>(), n->go.as<float>(), th + o.W3, n->h2.as<float>(), g.vol, n->nout);
    // layer 2
    k_wgrad_seg<NH><<<dim3(nseg, 9, 1), 256, 0, st>>>(part, n->g2.as<float>(), NH,
                                                      n->h1.as<float>(), g, 9);
    k_wgrad_sum<<<blocks_for(9 * NH * NH), 256, 0, st>>>(gr + o.W2, part, 9 * NH * NH, nseg);
    k_bias_grad<<<NH, 256, 0, st>>>(gr + o.b2, n->g2.as<float>(), g.vol, NH);
    k_conv9_back_in_tanh<<<blocks_for(size_t(g.vol) * NH), 256, 0, st>>>(
        n->g1.as<float>(), n->g2.as<float>(), th + o.W2, n->h1.as<float>(), g);
    // layer 1
    k_wgrad_seg<NF><<<dim3(nseg, 9, 1), 256, 0, st>>>(part, n->g1.as<float>(), NH,
                                                      n->f.as<float>(), g, 9);
    k_wgrad_sum<<<blocks_for(9 * NH * NF), 256, 0, st>>>(gr + o.W1, part, 9 * NH * NF, nseg);
    k_bias_grad<<<NH, 256, 0, st>>>(gr + o.b1, n->g1.as<float>(), g.vol, NH);
    GB_LAUNCH_CHECK();
    if (loss) {
      std::vector<float> h(nblk);
      GB_CHECK(cudaMemcpyAsync(h.data(), n->blk_loss.p, size_t(nblk) * 4, cudaMemcpyDeviceToHost,
                               st));
      GB_CHECK(cudaStreamSynchronize(st));
      double s = 0.0;
      for (float v : h) s += v;
      *loss = s / nblk;
    }
  });
}

mg_status mg_cnn_adam_step(mg_cnn* n, float lr, void* stream) {
  return cnn_guard(n, [&] {
    GB_REQUIRE(n && lr > 0.f, MG_ERR_ARG, "cnn: bad step");
    n->adam_t++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, float(n->adam_t)), c2 = 1.f - powf(b2, float(n->adam_t));
    k_adam<<<blocks_for(n->nparams), 256, 0, (cudaStream_t)stream>>>(
        n->theta.as<float>(), n->m1.as<float>(), n->m2.as<float>(), n->grad.as<float>(),
        n->nparams, lr, b1, b2, c1, c2);
    GB_LAUNCH_CHECK();
  });
}

}  // extern "C"
