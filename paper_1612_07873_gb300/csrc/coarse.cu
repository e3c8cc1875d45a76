// Coarse-grid stencil apply of Eq. (3) and the coarse-link store.
//
//   y(s) = sum_{slot=0..8} L[s][slot] x(nbr(s, slot)),  n x n complex blocks
//
// Every link byte is used exactly once per apply, so the single-RHS apply is
// an HBM stream (about 1 flop per byte in FP32).  Internal link layout per
// site: [slot][col][row] -- a column of n rows is contiguous -- so the 9n
// "columns" of a site form one contiguous run of 9n*n complex numbers.
//
// Thread mapping of the streaming kernel (Secs. 6.1-6.4 exposed differently):
//  * one CTA per coarse site;
//  * a thread owns one 16-byte chunk of rows (RPC = 16 / sizeof(element)
//    rows: 1 in FP64, 2 in FP32, 4 in 16-bit) -> TPC = n / RPC threads span a
//    column, so consecutive threads read consecutive 16-byte chunks;
//  * CG column groups split the 9n-long dot products (stencil direction and
//    dot-product parallelism at once); the CG partial sums of every row are
//    reduced through shared memory;
//  * the 9 gathered neighbour spinors sit in shared memory (9n complex).
// 16-bit links carry one FP32 scale per site (value = scale * stored); the
// arithmetic accumulates in FP32.
#include <type_traits>

#include "coarse_ops.cuh"
#include "kernels.cuh"
#include "tune.cuh"

namespace gbmg {

namespace {

// Eq. (3), one right-hand side: y = X x + sum_{+-mu} Y_{+-mu} x(. +- mu).
template <typename S, int N, int CG>
__global__ void __launch_bounds__(CG*(N / Unpack<S>::RPC))
    k_coarse_stream(cpx<typename StoreTraits<S>::real>* __restrict__ y,
                    const cpx<typename StoreTraits<S>::real>* __restrict__ x,
                    const S* __restrict__ links, const float* __restrict__ scales, Geom g) {
  using R = typename StoreTraits<S>::real;
  constexpr int RPC = Unpack<S>::RPC;
  constexpr int TPC = N / RPC;
  constexpr int K = 9 * N;
  constexpr int NT = CG * TPC;
  constexpr int ITER = K / CG;
  constexpr int U = batch_of(ITER);
  static_assert(N % RPC == 0 && K % CG == 0, "tile shape");
  __shared__ cpx<R> xs[K];
  __shared__ cpx<R> red[CG][N];
  __shared__ int nb[9];
  const int site = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid < 9) {
    int c[4];
    site_coords(g, site, c);
    nb[tid] = neighbour(g, site, c, tid);
  }
  __syncthreads();
  for (int i = tid; i < K; i += NT) {
    int d = i / N;
    xs[i] = x[size_t(nb[d]) * N + (i - d * N)];
  }
  __syncthreads();
  const int rp = tid % TPC;
  const int cg = tid / TPC;
  cpx<R> acc[RPC];
#pragma unroll
  for (int r = 0; r < RPC; ++r) acc[r] = cpx<R>(R(0), R(0));
  const uint4* L = reinterpret_cast<const uint4*>(links) + size_t(site) * K * TPC + rp;
  for (int it = 0; it < ITER; it += U) {
    uint4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = ld_stream16(L + size_t(cg + (it + u) * CG) * TPC);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      cpx<R> e[RPC];
      Unpack<S>::get(v[u], e);
      cpx<R> xv = xs[cg + (it + u) * CG];
#pragma unroll
      for (int r = 0; r < RPC; ++r) cmac(acc[r], e[r], xv);
    }
  }
#pragma unroll
  for (int r = 0; r < RPC; ++r) red[cg][rp * RPC + r] = acc[r];
  __syncthreads();
  for (int row = tid; row < N; row += NT) {
    cpx<R> s = red[0][row];
#pragma unroll
    for (int q = 1; q < CG; ++q) s += red[q][row];
    if (StoreTraits<S>::scaled) s = R(scales[site]) * s;
    y[size_t(site) * N + row] = s;
  }
}

// Multi-RHS form of the streaming kernel for stores without a tensor-core
// path (FP32).  Element (rhs, site, dof) sits at rhs * rs + (site * n + dof)
// * ss: interleaved [site][n][nrhs] (rs = 1, ss = nrhs) or back to back
// [nrhs][site][n] (rs = V n, ss = 1).  CTA (chunk, site) applies the site's
// links to NR right-hand sides, so each link chunk read from HBM feeds
// NR x RPC complex multiply-adds.  The gathered neighbour values sit in
// shared memory as xs[k][r] (k = slot*n + col); the same buffer then holds
// the CG partial sums as red[cg][r][row].
// UM caps the 16-byte link loads a thread keeps in flight (the batch U
// divides the K / CG columns it walks); a larger batch takes registers
// from occupancy, so the autotuner picks it per shape.
// Eq. (3) on NR right-hand sides per link read.
template <typename S, int N, int CG, int NR, int UM = 4>
__global__ void __launch_bounds__(CG*(N / Unpack<S>::RPC))
    k_coarse_stream_mr(cpx<typename StoreTraits<S>::real>* __restrict__ y,
                       const cpx<typename StoreTraits<S>::real>* __restrict__ x,
                       const S* __restrict__ links, const float* __restrict__ scales, Geom g,
                       size_t rs, size_t ss) {
  using R = typename StoreTraits<S>::real;
  constexpr int RPC = Unpack<S>::RPC;
  constexpr int TPC = N / RPC;
  constexpr int K = 9 * N;
  constexpr int NT = CG * TPC;
  constexpr int ITER = K / CG;
  constexpr int U = batch_of(ITER, UM);
  constexpr int XS = K * NR, RED = CG * NR * N;
  static_assert(N % RPC == 0 && K % CG == 0 && NR % 2 == 0 && ITER % U == 0, "tile shape");
  __shared__ __align__(16) cpx<R> buf[XS > RED ? XS : RED];
  __shared__ int nb[9];
  const int chunk = blockIdx.x, site = blockIdx.y;
  const int tid = threadIdx.x;
  if (tid < 9) {
    int c[4];
    site_coords(g, site, c);
    nb[tid] = neighbour(g, site, c, tid);
  }
  __syncthreads();
  if (ss == 1) {  // back to back: read each vector's neighbour values in order
    for (int i = tid; i < XS; i += NT) {
      const int r = i / K, k = i - r * K;
      const int d = k / N;
      buf[k * NR + r] = x[size_t(chunk * NR + r) * rs + size_t(nb[d]) * N + (k - d * N)];
    }
  } else {
    for (int i = tid; i < XS; i += NT) {
      const int k = i / NR, r = i - k * NR;
      const int d = k / N;
      buf[i] = x[size_t(chunk * NR + r) * rs + (size_t(nb[d]) * N + (k - d * N)) * ss];
    }
  }
  __syncthreads();
  const int rp = tid % TPC;
  const int cg = tid / TPC;
  cpx<R> acc[NR][RPC];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int q = 0; q < RPC; ++q) acc[r][q] = cpx<R>(R(0), R(0));
  const uint4* L = reinterpret_cast<const uint4*>(links) + size_t(site) * K * TPC + rp;
  for (int it = 0; it < ITER; it += U) {
    uint4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = ld_stream16(L + size_t(cg + (it + u) * CG) * TPC);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      cpx<R> e[RPC];
      Unpack<S>::get(v[u], e);
      const cpx<R>* xk = buf + (cg + (it + u) * CG) * NR;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const cpx<R> xv = xk[r];
#pragma unroll
        for (int q = 0; q < RPC; ++q) cmac(acc[r][q], e[q], xv);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int q = 0; q < RPC; ++q) buf[(cg * NR + r) * N + rp * RPC + q] = acc[r][q];
  __syncthreads();
  const R sc = StoreTraits<S>::scaled ? R(scales[site]) : R(1);
  for (int o = tid; o < N * NR; o += NT) {
    int row, r;
    if (ss == 1) {
      r = o / N;
      row = o - r * N;
    } else {
      row = o / NR;
      r = o - row * NR;
    }
    cpx<R> sum = buf[r * N + row];
#pragma unroll
    for (int q = 1; q < CG; ++q) sum += buf[(q * NR + r) * N + row];
    y[size_t(chunk * NR + r) * rs + (size_t(site) * N + row) * ss] = sc * sum;
  }
}

// Five-block form (X and the four forward links stored): the backward
// block is rebuilt from the -mu neighbour's forward link F = Y_{+mu}(x-mu),
//   Y_{-mu}(x) v = g5 F^dag (g5 v),   g5 = diag(+1 on the first n/2 dofs, -1),
// so its output row r is the dot product of the *stored column* r of F
// (contiguous) with w = g5 v.  Forward terms stream as in k_coarse_stream
// over K = 5n columns; backward terms: thread (part = t % TPC, column
// group = t / TPC) reads chunk `part` of columns t/TPC + CG i and keeps N/CG
// partial dot products, reduced over the TPC parts through shared memory.
// The neighbour's forward block was (or will soon be) streamed by the
// neighbour's own CTA, so most of these reads hit L2: HBM traffic is 5 of
// the 9 blocks.  16-bit forms: each backward input is pre-scaled by the
// neighbour's per-site scale.
// Eq. (3) from five stored blocks, Y_{-mu}(x) = g5hat Y_{+mu}(x - mu)^dag g5hat.
template <typename S, int N, int CG>
__global__ void __launch_bounds__(CG*(N / Unpack<S>::RPC))
    k_coarse_stream5(cpx<typename StoreTraits<S>::real>* __restrict__ y,
                     const cpx<typename StoreTraits<S>::real>* __restrict__ x,
                     const S* __restrict__ links5, const float* __restrict__ scales, Geom g) {
  using R = typename StoreTraits<S>::real;
  constexpr int RPC = Unpack<S>::RPC;
  constexpr int TPC = N / RPC;
  constexpr int K = 5 * N;
  constexpr int NT = CG * TPC;
  constexpr int ITER = K / CG;
  constexpr int U = batch_of(ITER);
  constexpr int CPT = N / CG;  // backward columns per thread
  static_assert(N % RPC == 0 && K % CG == 0 && N % CG == 0, "tile shape");
  __shared__ cpx<R> xs[K];          // forward inputs: x(site), x(site + mu)
  __shared__ cpx<R> ws[4 * N];      // backward inputs: scale(site - mu) g5 x(site - mu)
  __shared__ cpx<R> red[CG][N];
  __shared__ cpx<R> redb[TPC][N];
  __shared__ int nb[9];
  const int site = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid < 9) {
    int c[4];
    site_coords(g, site, c);
    nb[tid] = neighbour(g, site, c, tid);
  }
  __syncthreads();
  for (int i = tid; i < K; i += NT) {
    const int q = i / N, col = i - q * N;  // q: 0 -> site, 1..4 -> +mu
    const int slot = q == 0 ? 0 : 2 * q - 1;
    xs[i] = x[size_t(nb[slot]) * N + col];
  }
  for (int i = tid; i < 4 * N; i += NT) {
    const int mu = i / N, col = i - mu * N;
    const int sb = nb[2 + 2 * mu];
    R f = (col < N / 2) ? R(1) : R(-1);
    if (StoreTraits<S>::scaled) f *= R(scales[sb]);
    ws[i] = f * x[size_t(sb) * N + col];
  }
  __syncthreads();
  const int rp = tid % TPC;
  const int cg = tid / TPC;
  // forward: X and Y_{+mu}(site).  The four Y_{+mu} blocks are read again
  // by the +mu neighbours' CTAs (their backward terms): kept in L2 with an
  // evict-last policy; X, read once, and the backward reads (the last use)
  // evict first.
  const uint64_t keep = l2_policy_evict_last(), drop = l2_policy_evict_first();
  cpx<R> acc[RPC];
#pragma unroll
  for (int r = 0; r < RPC; ++r) acc[r] = cpx<R>(R(0), R(0));
  const uint4* L = reinterpret_cast<const uint4*>(links5) + size_t(site) * K * TPC + rp;
  for (int it = 0; it < ITER; it += U) {
    uint4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = cg + (it + u) * CG;
      v[u] = ld_stream16_hint(L + size_t(k) * TPC, k < N ? drop : keep);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      cpx<R> e[RPC];
      Unpack<S>::get(v[u], e);
      cpx<R> xv = xs[cg + (it + u) * CG];
#pragma unroll
      for (int r = 0; r < RPC; ++r) cmac(acc[r], e[r], xv);
    }
  }
  // backward: column dot products with the -mu neighbours' forward blocks
  cpx<R> accb[CPT];
#pragma unroll
  for (int i = 0; i < CPT; ++i) accb[i] = cpx<R>(R(0), R(0));
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const uint4* F = reinterpret_cast<const uint4*>(links5) +
                     (size_t(nb[2 + 2 * mu]) * 5 + 1 + mu) * N * TPC + rp;
    uint4 v[CPT];
#pragma unroll
    for (int i = 0; i < CPT; ++i) v[i] = ld_stream16_hint(F + size_t(cg + CG * i) * TPC, drop);
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
      cpx<R> e[RPC];
      Unpack<S>::get(v[i], e);
#pragma unroll
      for (int r = 0; r < RPC; ++r) cmac_conj(accb[i], e[r], ws[mu * N + rp * RPC + r]);
    }
  }
#pragma unroll
  for (int r = 0; r < RPC; ++r) red[cg][rp * RPC + r] = acc[r];
#pragma unroll
  for (int i = 0; i < CPT; ++i) redb[rp][cg + CG * i] = accb[i];
  __syncthreads();
  const R sc = StoreTraits<S>::scaled ? R(scales[site]) : R(1);
  for (int row = tid; row < N; row += NT) {
    cpx<R> f = red[0][row];
#pragma unroll
    for (int q = 1; q < CG; ++q) f += red[q][row];
    cpx<R> b = redb[0][row];
#pragma unroll
    for (int q = 1; q < TPC; ++q) b += redb[q][row];
    const R g5 = row < N / 2 ? R(1) : R(-1);
    y[size_t(site) * N + row] = sc * f + g5 * b;
  }
}

// [V][9][n][n] (any store type) -> [V][5][n][n]: slots 0, 1, 3, 5, 7
// Five-block store of the Eq. (3) links (X and the four Y_{+mu}).
template <typename S>
__global__ void k_links_pick5(S* __restrict__ out, const S* __restrict__ in, int vol, int n) {
  const size_t per = size_t(n) * n;
  const size_t total = size_t(vol) * 5 * per;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total;
       i += size_t(gridDim.x) * blockDim.x) {
    const size_t blk = i / per, e = i - blk * per;
    const size_t site = blk / 5;
    const int q = int(blk - site * 5);
    const int slot = q == 0 ? 0 : 2 * q - 1;
    out[i] = in[(site * 9 + slot) * per + e];
  }
}

// Any n, any number of right-hand sides: one CTA per site, threads over
// (row, rhs); links are read column-wise (coalesced over rows).
// Eq. (3) for any n and any number of right-hand sides.
template <typename S>
__global__ void k_coarse_generic(cpx<typename StoreTraits<S>::real>* __restrict__ y,
                                 const cpx<typename StoreTraits<S>::real>* __restrict__ x,
                                 const S* __restrict__ links, const float* __restrict__ scales,
                                 Geom g, int n, int nrhs) {
  using R = typename StoreTraits<S>::real;
  __shared__ int nb[9];
  const int site = blockIdx.x;
  if (threadIdx.x < 9) {
    int c[4];
    site_coords(g, site, c);
    nb[threadIdx.x] = neighbour(g, site, c, threadIdx.x);
  }
  __syncthreads();
  const S* Ls = links + size_t(site) * 9 * n * n;
  const R sc = StoreTraits<S>::scaled ? R(scales[site]) : R(1);
  for (int t = threadIdx.x; t < n * nrhs; t += blockDim.x) {
    int row = t / nrhs, rhs = t - row * nrhs;
    cpx<R> acc(R(0), R(0));
    for (int d = 0; d < 9; ++d) {
      const cpx<R>* xn = x + size_t(nb[d]) * n * nrhs + rhs;
      const S* Ld = Ls + size_t(d) * n * n + row;
      for (int col = 0; col < n; ++col)
        cmac(acc, StoreTraits<S>::load(Ld[size_t(col) * n]), xn[size_t(col) * nrhs]);
    }
    y[size_t(site) * n * nrhs + t] = sc * acc;
  }
}

// ext [V][9][row][col] complex double -> internal [V][9][col][row] in R
// Eq. (3) link store: ABI layout [slot][row][col] -> internal [slot][col][row].
template <typename R>
__global__ void k_links_import(cpx<R>* __restrict__ out, const cpx<double>* __restrict__ in,
                               int vol, int n) {
  size_t total = size_t(vol) * 9 * n * n;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total;
       i += size_t(gridDim.x) * blockDim.x) {
    size_t blk = i / (size_t(n) * n);
    int rem = int(i - blk * n * n);
    int col = rem / n, row = rem - col * n;
    out[i] = cpx<R>(in[blk * n * n + size_t(row) * n + col]);
  }
}

// Eq. (3) link store: internal layout -> ABI layout.
template <typename S>
__global__ void k_links_export(cpx<double>* __restrict__ out, const S* __restrict__ in,
                               const float* __restrict__ scales, int vol, int n) {
  size_t total = size_t(vol) * 9 * n * n;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total;
       i += size_t(gridDim.x) * blockDim.x) {
    size_t blk = i / (size_t(n) * n);
    int rem = int(i - blk * n * n);
    int row = rem / n, col = rem - row * n;
    size_t site = blk / 9;
    double sc = StoreTraits<S>::scaled ? double(scales[site]) : 1.0;
    cpx<double> v(StoreTraits<S>::load(in[blk * n * n + size_t(col) * n + row]));
    out[i] = sc * v;
  }
}

// per-site scale = max |component| over the nine blocks; stored = value/scale
// Eq. (3) links in 16-bit storage with one scale per site (Sec. 4 half precision).
template <typename S>
__global__ void k_links_pack16(S* __restrict__ out, float* __restrict__ scales,
                               const cpx<float>* __restrict__ in, int n) {
  __shared__ float sh[32];
  const size_t per = size_t(9) * n * n;
  const cpx<float>* src = in + blockIdx.x * per;
  float m = 0.f;
  for (size_t i = threadIdx.x; i < per; i += blockDim.x)
    m = fmaxf(m, fmaxf(fabsf(src[i].re), fabsf(src[i].im)));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) sh[0] = m > 0.f ? m : 1.f;
  }
  __syncthreads();
  const float sc = sh[0], inv = 1.f / sc;
  if (threadIdx.x == 0) scales[blockIdx.x] = sc;
  S* dst = out + blockIdx.x * per;
  for (size_t i = threadIdx.x; i < per; i += blockDim.x)
    dst[i] = StoreTraits<S>::pack(cpx<float>(src[i].re * inv, src[i].im * inv));
}

template <typename S, int N, int CG>
void launch_stream(const Level& L, void* y, const void* x, const void* links, cudaStream_t st) {
  using R = typename StoreTraits<S>::real;
  constexpr int NT = CG * (N / Unpack<S>::RPC);
  k_coarse_stream<S, N, CG><<<L.g.vol, NT, 0, st>>>((cpx<R>*)y, (const cpx<R>*)x, (const S*)links,
                                                    L.scales.as<float>(), L.g);
}

template <typename S, int N, int CG>
void launch_stream5(const Level& L, void* y, const void* x, const void* links, cudaStream_t st) {
  using R = typename StoreTraits<S>::real;
  constexpr int NT = CG * (N / Unpack<S>::RPC);
  k_coarse_stream5<S, N, CG><<<L.g.vol, NT, 0, st>>>((cpx<R>*)y, (const cpx<R>*)x,
                                                     (const S*)links, L.scales.as<float>(), L.g);
}

// Column-group counts the autotuner chooses from: the middle one is the
// default; a count is a candidate when it divides the kernel's K.
template <typename S>
struct CgSet {
  static constexpr int RPC = Unpack<S>::RPC;
  static constexpr int c0 = RPC == 1 ? 4 : (RPC == 2 ? 8 : 16);
  static constexpr int c1 = c0 / 2;
  static constexpr int c2 = c0 * 2;
};

template <typename S, int N, bool FIVE>
void launch_cg(int cg, const Level& L, void* y, const void* x, const void* links, cudaStream_t st) {
  using CS = CgSet<S>;
  if constexpr (FIVE) {
    if (cg == CS::c1) {
      if constexpr (N % CS::c1 == 0) return launch_stream5<S, N, CS::c1>(L, y, x, links, st);
    } else if (cg == CS::c2) {
      if constexpr (N % CS::c2 == 0) return launch_stream5<S, N, CS::c2>(L, y, x, links, st);
    }
    return launch_stream5<S, N, CS::c0>(L, y, x, links, st);
  } else {
    if (cg == CS::c1) {
      if constexpr ((9 * N) % CS::c1 == 0) return launch_stream<S, N, CS::c1>(L, y, x, links, st);
    } else if (cg == CS::c2) {
      if constexpr ((9 * N) % CS::c2 == 0) return launch_stream<S, N, CS::c2>(L, y, x, links, st);
    }
    return launch_stream<S, N, CS::c0>(L, y, x, links, st);
  }
}

template <typename S, int N, bool FIVE>
void tuned_stream(const Level& L, void* y, const void* x, const void* links, cudaStream_t st) {
  using CS = CgSet<S>;
  std::vector<int> cands{CS::c0};
  // FP64 stores serve parity runs only: not tuned
  if (!std::is_same<S, cpx<double>>::value) {
    const int K = FIVE ? N : 9 * N;
    if (K % CS::c1 == 0) cands.push_back(CS::c1);
    if (K % CS::c2 == 0) cands.push_back(CS::c2);
  }
  const std::string key = std::string(FIVE ? "stream5" : "stream") + "/p" +
                          std::to_string(int(L.prec)) + "/n" + std::to_string(N) + "/v" +
                          std::to_string(L.g.vol);
  const int cg = Tuner::get().choose(key, cands, st, [&](int c) {
    launch_cg<S, N, FIVE>(c, L, y, x, links, st);
  });
  launch_cg<S, N, FIVE>(cg, L, y, x, links, st);
}

template <typename S>
bool try_stream5(const Level& L, void* y, const void* x, cudaStream_t st) {
  // FP64 stores (parity runs) keep the nine-block kernel: the five-block
  // form's reduction buffer would not fit its static shared memory
  if (std::is_same<S, cpx<double>>::value) return false;
  const void* links = L.links5.p;
  switch (L.nd) {
    case 32: tuned_stream<S, 32, true>(L, y, x, links, st); return true;
    case 48: tuned_stream<S, 48, true>(L, y, x, links, st); return true;
    case 64: tuned_stream<S, 64, true>(L, y, x, links, st); return true;
    default: return false;
  }
}

template <typename S>
bool try_stream(const Level& L, void* y, const void* x, const void* links, cudaStream_t st) {
  switch (L.nd) {
    case 16: tuned_stream<S, 16, false>(L, y, x, links, st); return true;
    case 32: tuned_stream<S, 32, false>(L, y, x, links, st); return true;
    case 48: tuned_stream<S, 48, false>(L, y, x, links, st); return true;
    case 64: tuned_stream<S, 64, false>(L, y, x, links, st); return true;
    default: return false;
  }
}

template <typename S, int N>
void launch_stream_mr(const Level& L, void* y, const void* x, const void* links, int nrhs,
                      bool blocked, cudaStream_t st) {
  using R = typename StoreTraits<S>::real;
  constexpr int CG = CgSet<S>::c0;
  constexpr int NT = CG * (N / Unpack<S>::RPC);
  const cpx<R>* xp = (const cpx<R>*)x;
  cpx<R>* yp = (cpx<R>*)y;
  const S* lp = (const S*)links;
  const size_t rs = blocked ? size_t(L.g.vol) * N : 1;
  const size_t ss = blocked ? 1 : size_t(nrhs);
  if (nrhs % 8 == 0) {
    // 8 right-hand sides per link read: the load batch is tuned (choice =
    // its cap UM; caps giving the same batch are one candidate)
    constexpr int ITER = 9 * N / CG;
    std::vector<int> cands{4};
    if (!std::is_same<S, cpx<double>>::value) {
      if (batch_of(ITER, 6) != batch_of(ITER, 4)) cands.push_back(6);
      if (batch_of(ITER, 9) != batch_of(ITER, 6) && batch_of(ITER, 9) != batch_of(ITER, 4))
        cands.push_back(9);
    }
    auto launch = [&](int um) {
      const dim3 grid(nrhs / 8, L.g.vol);
      if (um == 9)
        k_coarse_stream_mr<S, N, CG, 8, 9><<<grid, NT, 0, st>>>(yp, xp, lp, L.scales.as<float>(),
                                                                 L.g, rs, ss);
      else if (um == 6)
        k_coarse_stream_mr<S, N, CG, 8, 6><<<grid, NT, 0, st>>>(yp, xp, lp, L.scales.as<float>(),
                                                                 L.g, rs, ss);
      else
        k_coarse_stream_mr<S, N, CG, 8, 4><<<grid, NT, 0, st>>>(yp, xp, lp, L.scales.as<float>(),
                                                                 L.g, rs, ss);
    };
    const std::string key = "stream_mr/p" + std::to_string(int(L.prec)) + "/n" +
                            std::to_string(N) + "/v" + std::to_string(L.g.vol) + "/r" +
                            std::to_string(nrhs) + "/b" + std::to_string(int(blocked));
    launch(cands.size() == 1 ? cands.front() : Tuner::get().choose(key, cands, st, launch));
  } else if (nrhs % 4 == 0)
    k_coarse_stream_mr<S, N, CG, 4><<<dim3(nrhs / 4, L.g.vol), NT, 0, st>>>(
        yp, xp, lp, L.scales.as<float>(), L.g, rs, ss);
  else
    k_coarse_stream_mr<S, N, CG, 2><<<dim3(nrhs / 2, L.g.vol), NT, 0, st>>>(
        yp, xp, lp, L.scales.as<float>(), L.g, rs, ss);
}

template <typename S>
bool try_stream_mr(const Level& L, void* y, const void* x, const void* links, int nrhs,
                   bool blocked, cudaStream_t st) {
  if (nrhs % 2 != 0) return false;
  switch (L.nd) {
    case 16: launch_stream_mr<S, 16>(L, y, x, links, nrhs, blocked, st); return true;
    case 32: launch_stream_mr<S, 32>(L, y, x, links, nrhs, blocked, st); return true;
    case 48: launch_stream_mr<S, 48>(L, y, x, links, nrhs, blocked, st); return true;
    case 64: launch_stream_mr<S, 64>(L, y, x, links, nrhs, blocked, st); return true;
    default: return false;
  }
}

template <typename S>
void dispatch_apply(const Level& L, void* y, const void* x, const void* links, int nrhs,
                    cudaStream_t st) {
  using R = typename StoreTraits<S>::real;
  if (nrhs == 1 && L.slots5 && L.links5.p && try_stream5<S>(L, y, x, st)) return;
  if (nrhs == 1 && try_stream<S>(L, y, x, links, st)) return;
  if constexpr (std::is_same<S, cpx<float>>::value) {
    if (nrhs > 1 && try_stream_mr<S>(L, y, x, links, nrhs, false, st)) return;
  }
  int threads = L.nd * nrhs >= 256 ? 256 : ((L.nd * nrhs + 31) / 32) * 32;
  k_coarse_generic<S><<<L.g.vol, threads, 0, st>>>((cpx<R>*)y, (const cpx<R>*)x, (const S*)links,
                                                   L.scales.as<float>(), L.g, L.nd, nrhs);
}

}  // namespace

bool coarse_apply_multi_fast(const Level& L, int nrhs) {
  if (nrhs < 2) return false;
  if (coarse_apply_mma_supported(L, nrhs)) return true;
  return L.prec == MG_F32 && nrhs % 2 == 0 &&
         (L.nd == 16 || L.nd == 32 || L.nd == 48 || L.nd == 64);
}

void coarse_apply(mg_ctx* c, int level, void* y, const void* x, int nrhs, cudaStream_t st) {
  Level& L = c->L[level];
  GB_REQUIRE(level >= 1 && level < c->nlevels, MG_ERR_ARG, "coarse_apply: bad level");
  GB_REQUIRE(L.have_op, MG_ERR_STATE, "coarse_apply: coarse operator not built");
  GB_REQUIRE(nrhs >= 1, MG_ERR_ARG, "coarse_apply: nrhs < 1");
  GB_REQUIRE(y != x, MG_ERR_ARG, "coarse_apply: output aliases input");
  const double n = L.nd;
  const bool five = L.slots5 && L.links5.p && nrhs == 1 && L.prec != MG_F64 &&
                    (L.nd == 32 || L.nd == 48 || L.nd == 64);
  const double lbytes = double(L.g.vol) * (five ? 5 : 9) * n * n *
                        (L.prec == MG_F64 ? 16 : L.prec == MG_F32 ? 8 : 4);
  const double vbytes = double(L.g.vol) * 2 * n * nrhs * (L.vprec == MG_F64 ? 16 : 8);
  // single- and multi-RHS applies are profiled under separate names
  ProfScope ps(c->prof, st, nrhs == 1 ? "coarse_apply" : "coarse_apply_multi", level,
               lbytes + vbytes,
               8.0 * 9 * n * n * L.g.vol * nrhs);
  if (nrhs > 1 && coarse_apply_mma_supported(L, nrhs)) {
    coarse_apply_mma(c, level, y, x, nrhs, st);
    GB_LAUNCH_CHECK();
    c->launches++;
    return;
  }
  switch (L.prec) {
    case MG_F64: dispatch_apply<cpx<double>>(L, y, x, L.links.p, nrhs, st); break;
    case MG_F32: dispatch_apply<cpx<float>>(L, y, x, L.links.p, nrhs, st); break;
    case MG_BF16: dispatch_apply<bf16c>(L, y, x, L.links16.p, nrhs, st); break;
    case MG_F16: dispatch_apply<f16c>(L, y, x, L.links16.p, nrhs, st); break;
    case MG_I16: dispatch_apply<i16c>(L, y, x, L.links16.p, nrhs, st); break;
  }
  GB_LAUNCH_CHECK();
  c->launches++;
}

void coarse_apply_blocked(mg_ctx* c, int level, void* y, const void* x, int nr,
                          cudaStream_t st) {
  if (nr == 1) return coarse_apply(c, level, y, x, 1, st);
  Level& L = c->L[level];
  GB_REQUIRE(level >= 1 && level < c->nlevels, MG_ERR_ARG, "coarse_apply: bad level");
  GB_REQUIRE(L.have_op, MG_ERR_STATE, "coarse_apply: coarse operator not built");
  GB_REQUIRE(y != x, MG_ERR_ARG, "coarse_apply: output aliases input");
  const size_t n = L.vec_elems();
  const size_t vb = n * prec_bytes_complex(L.vprec);
  if (L.prec == MG_F32 && !L.slots5 && nr % 2 == 0 &&
      (L.nd == 16 || L.nd == 32 || L.nd == 48 || L.nd == 64)) {
    const double nd = L.nd;
    ProfScope ps(c->prof, st, "coarse_apply_multi", level,
                 double(L.g.vol) * 9 * nd * nd * 8 + double(nr) * 2 * double(vb),
                 8.0 * 9 * nd * nd * L.g.vol * nr);
    try_stream_mr<cpx<float>>(L, y, x, L.links.p, nr, true, st);
    GB_LAUNCH_CHECK();
    c->launches++;
    return;
  }
  if (coarse_apply_mma_supported(L, nr)) {
    // the tensor-core kernel takes the interleaved layout
    if (L.tr_in.bytes < vb * nr) L.tr_in.alloc(vb * nr);
    if (L.tr_out.bytes < vb * nr) L.tr_out.alloc(vb * nr);
    Vec vx, vi, vo, vy;
    vx.p = const_cast<void*>(x);
    vy.p = y;
    vi.p = L.tr_in.p;
    vo.p = L.tr_out.p;
    vx.prec = vy.prec = vi.prec = vo.prec = L.vprec;
    vx.n = vy.n = vi.n = vo.n = n;
    blas_transpose(c, vi, vx, nr, true, st);
    coarse_apply(c, level, vo.p, vi.p, nr, st);
    blas_transpose(c, vy, vo, nr, false, st);
    return;
  }
  for (int v = 0; v < nr; ++v)
    coarse_apply(c, level, (char*)y + v * vb, (const char*)x + v * vb, 1, st);
}

void links_pick5(mg_ctx* c, int level, cudaStream_t st) {
  Level& L = c->L[level];
  if (!L.slots5) return;
  const size_t total = size_t(L.g.vol) * 5 * L.nd * L.nd;
  int blocks = ceil_div(total, 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  switch (L.prec) {
    case MG_F64:
      L.links5.alloc(total * 16);
      k_links_pick5<cpx<double>><<<blocks, 256, 0, st>>>(L.links5.as<cpx<double>>(),
                                                         L.links.as<cpx<double>>(), L.g.vol, L.nd);
      break;
    case MG_F32:
      L.links5.alloc(total * 8);
      k_links_pick5<cpx<float>><<<blocks, 256, 0, st>>>(L.links5.as<cpx<float>>(),
                                                        L.links.as<cpx<float>>(), L.g.vol, L.nd);
      break;
    default:
      L.links5.alloc(total * 4);
      k_links_pick5<bf16c><<<blocks, 256, 0, st>>>(L.links5.as<bf16c>(), L.links16.as<bf16c>(),
                                                   L.g.vol, L.nd);
      break;
  }
  GB_LAUNCH_CHECK();
  c->launches++;
}

void links_pack16(mg_ctx* c, int level, cudaStream_t st) {
  Level& L = c->L[level];
  if (!prec_is16(L.prec)) {
    links_pick5(c, level, st);
    return;
  }
  const size_t per = size_t(9) * L.nd * L.nd;
  L.links16.alloc(per * L.g.vol * 4);
  L.scales.alloc(size_t(L.g.vol) * sizeof(float));
  if (L.prec == MG_BF16)
    k_links_pack16<bf16c><<<L.g.vol, 256, 0, st>>>(L.links16.as<bf16c>(), L.scales.as<float>(),
                                                   L.links.as<cpx<float>>(), L.nd);
  else if (L.prec == MG_F16)
    k_links_pack16<f16c><<<L.g.vol, 256, 0, st>>>(L.links16.as<f16c>(), L.scales.as<float>(),
                                                  L.links.as<cpx<float>>(), L.nd);
  else
    k_links_pack16<i16c><<<L.g.vol, 256, 0, st>>>(L.links16.as<i16c>(), L.scales.as<float>(),
                                                  L.links.as<cpx<float>>(), L.nd);
  GB_LAUNCH_CHECK();
  c->launches++;
  links_tile_mma(c, level, st);
  links_pick5(c, level, st);
}

void links_import(mg_ctx* c, int level, const void* ext, cudaStream_t st) {
  Level& L = c->L[level];
  const size_t total = size_t(L.g.vol) * 9 * L.nd * L.nd;
  L.links.alloc(total * prec_bytes_complex(L.vprec));
  int blocks = ceil_div(total, 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (L.vprec == MG_F64)
    k_links_import<double><<<blocks, 256, 0, st>>>(L.links.as<cpx<double>>(),
                                                   (const cpx<double>*)ext, L.g.vol, L.nd);
  else
    k_links_import<float><<<blocks, 256, 0, st>>>(L.links.as<cpx<float>>(),
                                                  (const cpx<double>*)ext, L.g.vol, L.nd);
  GB_LAUNCH_CHECK();
  c->launches++;
  links_pack16(c, level, st);
  L.have_op = true;
}

void links_export(mg_ctx* c, int level, void* ext, cudaStream_t st) {
  Level& L = c->L[level];
  GB_REQUIRE(L.have_op, MG_ERR_STATE, "coarse links not built");
  const size_t total = size_t(L.g.vol) * 9 * L.nd * L.nd;
  int blocks = ceil_div(total, 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  cpx<double>* o = (cpx<double>*)ext;
  const float* sc = L.scales.as<float>();
  switch (L.prec) {
    case MG_F64:
      k_links_export<cpx<double>><<<blocks, 256, 0, st>>>(o, L.links.as<cpx<double>>(), sc, L.g.vol, L.nd);
      break;
    case MG_F32:
      k_links_export<cpx<float>><<<blocks, 256, 0, st>>>(o, L.links.as<cpx<float>>(), sc, L.g.vol, L.nd);
      break;
    case MG_BF16:
      k_links_export<bf16c><<<blocks, 256, 0, st>>>(o, L.links16.as<bf16c>(), sc, L.g.vol, L.nd);
      break;
    case MG_F16:
      k_links_export<f16c><<<blocks, 256, 0, st>>>(o, L.links16.as<f16c>(), sc, L.g.vol, L.nd);
      break;
    case MG_I16:
      k_links_export<i16c><<<blocks, 256, 0, st>>>(o, L.links16.as<i16c>(), sc, L.g.vol, L.nd);
      break;
  }
  GB_LAUNCH_CHECK();
  c->launches++;
}

}  // namespace gbmg
