// Red-black (Schur complement) preconditioning on every level (Secs. 3.3
// and 7.1).  With sites split by parity (every extent even) a level's
// operator is M = A + H: A site-local (the clover diagonal 4 + m + A_x on
// the fine level, the dense block X on a coarse level), H the hops, which
// join the two parities.  On the odd sites
//   S = A_o - H_oe A_e^-1 H_eo,   b^ = b_o - H_oe A_e^-1 b_e,
// and x_e = A_e^-1 (b_e - H_eo x_o) completes a solution of M x = b.
//
// Parity vectors are compact: the site s of parity p is entry s >> 1 (the
// x extent is even, so each pair of sites 2h, 2h + 1 holds one site of each
// parity).  A_e^-1 is formed once per operator in FP64 (Gauss-Jordan with
// partial pivoting per site) and stored for the even sites only.
//
// One kernel family per operator type applies the hops of one parity with a
// fused epilogue (EoMode): H in, A^-1 H in, A xc - H in, xc - H in,
// A^-1 (xc - H in).  S costs two launches (A^-1 H on the even sites, then
// A xc - H on the odd ones).
#include "coarse_ops.cuh"
#include "kernels.cuh"
#include "wilson_ops.cuh"

namespace gbmg {

namespace {

// site of parity p at compact index h
__host__ __device__ __forceinline__ int eo_site(const Geom& g, int h, int p) {
  const int half0 = g.L[0] >> 1;
  const int row = h / half0;  // y + L1 (z + L2 t)
  const int k = h - row * half0;
  int r = row;
  const int y = r % g.L[1];
  r /= g.L[1];
  const int z = r % g.L[2];
  const int t = r / g.L[2];
  return 2 * k + ((p + y + z + t) & 1) + g.L[0] * row;
}

__device__ __forceinline__ int parity_of(const int c[4]) { return (c[0] + c[1] + c[2] + c[3]) & 1; }

// 1 / z = conj(z) / |z|^2
__device__ __forceinline__ cpx<double> crecip(cpx<double> z) { return (1.0 / norm2(z)) * conj(z); }

// ------------------------------------------------------------ fine level
// C12: links in the two-row form, third row rebuilt in registers with the
// boundary sign of the link (as in the full-lattice kernel).
// Sec. 3.3: the hops of Eq. (2) between parities, fused epilogue.
template <typename R, int MODE, bool C12>
__global__ void __launch_bounds__(128) k_wilson_eo(cpx<R>* __restrict__ out,
                                                   const cpx<R>* __restrict__ in,
                                                   const cpx<R>* __restrict__ xc,
                                                   const cpx<R>* __restrict__ U,
                                                   const R* __restrict__ A,
                                                   const R* __restrict__ Ainv, Geom g, R diag,
                                                   int p, size_t hstride, int antiperiodic) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= (g.vol >> 1)) return;
  const size_t off = size_t(blockIdx.y) * hstride;
  in += off;
  out += off;
  const int s = eo_site(g, h, p);
  int c[4];
  site_coords(g, s, c);
  cpx<R> psi[12], acc[12], u[9];
#pragma unroll
  for (int i = 0; i < 12; ++i) acc[i] = cpx<R>(R(0), R(0));
  auto load_spinor = [&](const cpx<R>* base, int hh) {
    const uint4* q = reinterpret_cast<const uint4*>(base + size_t(hh) * 12);
    constexpr int W = sizeof(cpx<R>) * 12 / 16;
    uint4 w[W];
#pragma unroll
    for (int i = 0; i < W; ++i) w[i] = __ldg(q + i);
#pragma unroll
    for (int i = 0; i < 12; ++i) psi[i] = reinterpret_cast<const cpx<R>*>(w)[i];
  };
  auto load_link = [&](size_t idx, bool neg) {
    if constexpr (C12) {
      const uint4* q = reinterpret_cast<const uint4*>(U + idx * 6);
      uint4 w[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) w[i] = __ldg(q + i);
#pragma unroll
      for (int i = 0; i < 6; ++i) u[i] = reinterpret_cast<const cpx<R>*>(w)[i];
      const R sg = neg ? R(-1) : R(1);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, cc = (a + 2) % 3;
        u[6 + a] = sg * conj(u[b] * u[3 + cc] - u[cc] * u[3 + b]);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 9; ++i) u[i] = U[idx * 9 + i];
    }
  };
  const bool tlast = antiperiodic && c[3] == g.L[3] - 1, tfirst = antiperiodic && c[3] == 0;
  const size_t V = g.vol;
#define GB_EO_HOP(MU)                                    \
  {                                                      \
    const int sf = neighbour(g, s, c, 1 + 2 * MU);       \
    load_spinor(in, sf >> 1);                            \
    load_link(MU * V + s, MU == 3 && tlast);             \
    hop_accum<MU, true>(u, psi, acc);                    \
    const int sb = neighbour(g, s, c, 2 + 2 * MU);       \
    load_spinor(in, sb >> 1);                            \
    load_link(MU * V + sb, MU == 3 && tfirst);           \
    hop_accum<MU, false>(u, psi, acc);                   \
  }
  GB_EO_HOP(0) GB_EO_HOP(1) GB_EO_HOP(2) GB_EO_HOP(3)
#undef GB_EO_HOP
  cpx<R> y[12];
  if constexpr (MODE == EO_HOP) {
#pragma unroll
    for (int i = 0; i < 12; ++i) y[i] = acc[i];
  } else if constexpr (MODE == EO_AINV_HOP) {
#pragma unroll
    for (int i = 0; i < 12; ++i) y[i] = cpx<R>(R(0), R(0));
    clover_accum(Ainv + size_t(h) * 72, R(0), acc, y);
  } else {
    load_spinor(xc + off, h);  // psi = xc at this site
    if constexpr (MODE == EO_A_XC_MINUS_HOP) {
#pragma unroll
      for (int i = 0; i < 12; ++i) y[i] = -acc[i];
      clover_accum(A + size_t(s) * 72, diag, psi, y);
    } else if constexpr (MODE == EO_XC_MINUS_HOP) {
#pragma unroll
      for (int i = 0; i < 12; ++i) y[i] = psi[i] - acc[i];
    } else {  // EO_AINV_XC_MINUS_HOP
#pragma unroll
      for (int i = 0; i < 12; ++i) {
        acc[i] = psi[i] - acc[i];
        y[i] = cpx<R>(R(0), R(0));
      }
      clover_accum(Ainv + size_t(h) * 72, R(0), acc, y);
    }
  }
  uint4* o = reinterpret_cast<uint4*>(out + size_t(h) * 12);
#pragma unroll
  for (int i = 0; i < int(sizeof(cpx<R>) * 12 / 16); ++i) o[i] = reinterpret_cast<const uint4*>(y)[i];
}

// (4 + m + A_x)^-1 for the even sites: two 6x6 Hermitian chirality blocks,
// inverted in FP64 by Gauss-Jordan with partial pivoting, stored packed as
// the clover (6 real diagonal entries, then the 15 entries below it).
// Sec. 3.3: A_e^-1 of the fine level, per even site.
template <typename Rout>
__global__ void k_clover_inverse(Rout* __restrict__ out, const double* __restrict__ clover,
                                 Geom g, double diag, int* __restrict__ status) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.vol) return;  // (even site h, chirality) = (t >> 1, t & 1)
  const int h = t >> 1, chi = t & 1;
  const int s = eo_site(g, h, 0);
  const double* a = clover + size_t(s) * 72 + chi * 36;
  cpx<double> m[6][6];
#pragma unroll
  for (int i = 0; i < 6; ++i) m[i][i] = cpx<double>(diag + a[i], 0.0);
#pragma unroll
  for (int i = 1; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) {
      const int k = i * (i - 1) / 2 + j;
      m[i][j] = cpx<double>(a[6 + 2 * k], a[7 + 2 * k]);
      m[j][i] = conj(m[i][j]);
    }
  int perm[6];
  for (int k = 0; k < 6; ++k) {
    int piv = k;
    double best = norm2(m[k][k]);
    for (int i = k + 1; i < 6; ++i)
      if (norm2(m[i][k]) > best) {
        best = norm2(m[i][k]);
        piv = i;
      }
    perm[k] = piv;
    if (!(best > 0.0)) {
      atomicOr(status, 2);
      return;
    }
    if (piv != k)
      for (int j = 0; j < 6; ++j) {
        const cpx<double> tmp = m[k][j];
        m[k][j] = m[piv][j];
        m[piv][j] = tmp;
      }
    const cpx<double> pinv = crecip(m[k][k]);
    m[k][k] = cpx<double>(1.0, 0.0);
    for (int j = 0; j < 6; ++j) m[k][j] = m[k][j] * pinv;
    for (int i = 0; i < 6; ++i) {
      if (i == k) continue;
      const cpx<double> f = m[i][k];
      for (int j = 0; j < 6; ++j) m[i][j] -= f * m[k][j];
      m[i][k] = -(f * pinv);
    }
  }
  for (int k = 5; k >= 0; --k)
    if (perm[k] != k)
      for (int i = 0; i < 6; ++i) {
        const cpx<double> tmp = m[i][k];
        m[i][k] = m[i][perm[k]];
        m[i][perm[k]] = tmp;
      }
  Rout* o = out + size_t(h) * 72 + chi * 36;
  for (int i = 0; i < 6; ++i) o[i] = Rout(m[i][i].re);
  for (int i = 1; i < 6; ++i)
    for (int j = 0; j < i; ++j) {
      const int k = i * (i - 1) / 2 + j;
      o[6 + 2 * k] = Rout(m[i][j].re);
      o[7 + 2 * k] = Rout(m[i][j].im);
    }
}

// full [V][nd] <-> compact halves [V/2][nd] (even, odd)
// Sec. 3.3: full vector -> compact parity halves.
template <typename R>
__global__ void k_eo_split(cpx<R>* __restrict__ he, cpx<R>* __restrict__ ho,
                           const cpx<R>* __restrict__ full, Geom g, int nd, size_t fstride,
                           size_t hstride) {
  const size_t n = size_t(g.vol) * nd;
  full += size_t(blockIdx.y) * fstride;
  he += size_t(blockIdx.y) * hstride;
  ho += size_t(blockIdx.y) * hstride;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    const int s = int(i / nd), a = int(i - size_t(s) * nd);
    int c[4];
    site_coords(g, s, c);
    (parity_of(c) ? ho : he)[size_t(s >> 1) * nd + a] = full[i];
  }
}

// Sec. 3.3: compact parity halves -> full vector.
template <typename R>
__global__ void k_eo_merge(cpx<R>* __restrict__ full, const cpx<R>* __restrict__ he,
                           const cpx<R>* __restrict__ ho, Geom g, int nd, size_t fstride,
                           size_t hstride) {
  const size_t n = size_t(g.vol) * nd;
  full += size_t(blockIdx.y) * fstride;
  he += size_t(blockIdx.y) * hstride;
  ho += size_t(blockIdx.y) * hstride;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    const int s = int(i / nd), a = int(i - size_t(s) * nd);
    int c[4];
    site_coords(g, s, c);
    full[i] = (parity_of(c) ? ho : he)[size_t(s >> 1) * nd + a];
  }
}

// A_e^-1 applied site by site to a compact even vector (fine level)
// Sec. 3.3: A_e^-1 applied on the even sites.
template <typename R>
__global__ void k_clover_inv_apply(cpx<R>* __restrict__ out, const cpx<R>* __restrict__ in,
                                   const R* __restrict__ Ainv, int vh, size_t hstride) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= vh) return;
  const size_t off = size_t(blockIdx.y) * hstride + size_t(h) * 12;
  cpx<R> x[12], y[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    x[i] = in[off + i];
    y[i] = cpx<R>(R(0), R(0));
  }
  clover_accum(Ainv + size_t(h) * 72, R(0), x, y);
#pragma unroll
  for (int i = 0; i < 12; ++i) out[off + i] = y[i];
}

// ------------------------------------------------------------ coarse levels
// out_h = sum_k cols[k] xs[k] over K columns of N rows (column-major, the
// link layout [col][row]); work item (rp, cg) streams 16-byte row chunk rp
// of columns cg, cg + CG, ...; the CG partial sums meet in `red`; the result
// (times `scale`) lands in res[0..N).  The CTA's threads loop over the
// CG * N / RPC work items, so one CTA serves element types of different
// widths (16-bit links and FP32 X_e^-1).  Ends with a CTA barrier.
template <typename S, int N, int CG, int K>
__device__ __forceinline__ void stream_cols(const S* __restrict__ cols,
                                            const cpx<typename StoreTraits<S>::real>* xs,
                                            cpx<typename StoreTraits<S>::real>* red,
                                            cpx<typename StoreTraits<S>::real>* res,
                                            typename StoreTraits<S>::real scale) {
  using R = typename StoreTraits<S>::real;
  constexpr int RPC = Unpack<S>::RPC;
  constexpr int TPC = N / RPC;
  constexpr int NT = CG * TPC;
  constexpr int ITER = K / CG;
  constexpr int U = batch_of(ITER, 8);
  static_assert(K % CG == 0 && N % RPC == 0, "tile shape");
  const int tid = threadIdx.x;
  for (int item = tid; item < NT; item += blockDim.x) {
    const int rp = item % TPC, cg = item / TPC;
    cpx<R> acc[RPC];
#pragma unroll
    for (int r = 0; r < RPC; ++r) acc[r] = cpx<R>(R(0), R(0));
    const uint4* L = reinterpret_cast<const uint4*>(cols) + rp;
    for (int it = 0; it < ITER; it += U) {
      uint4 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = ld_stream16(L + size_t(cg + (it + u) * CG) * TPC);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        cpx<R> e[RPC];
        Unpack<S>::get(v[u], e);
        const cpx<R> xv = xs[cg + (it + u) * CG];
#pragma unroll
        for (int r = 0; r < RPC; ++r) cmac(acc[r], e[r], xv);
      }
    }
#pragma unroll
    for (int r = 0; r < RPC; ++r) red[cg * N + rp * RPC + r] = acc[r];
  }
  __syncthreads();
  for (int row = tid; row < N; row += blockDim.x) {
    cpx<R> s = red[row];
#pragma unroll
    for (int q = 1; q < CG; ++q) s += red[q * N + row];
    res[row] = scale * s;
  }
  __syncthreads();
}

// Coarse hops of one parity with the fused epilogues.  CTA per compact site
// h (blockIdx.x) and right-hand side (blockIdx.y).  S: the level's link
// store (with per-site scales for 16-bit stores); Xinv: A_e^-1 = X_e^-1 as
// [V/2][col][row] in the vector precision.
// Sec. 3.3: the hops of Eq. (3) between parities, fused epilogue.
template <typename S, int N, int CG, int MODE>
__global__ void __launch_bounds__(CG*(N / Unpack<S>::RPC))
    k_coarse_eo(cpx<typename StoreTraits<S>::real>* __restrict__ out,
                const cpx<typename StoreTraits<S>::real>* __restrict__ in,
                const cpx<typename StoreTraits<S>::real>* __restrict__ xc,
                const S* __restrict__ links, const float* __restrict__ scales,
                const cpx<typename StoreTraits<S>::real>* __restrict__ Xinv, Geom g, int p,
                size_t hstride) {
  using R = typename StoreTraits<S>::real;
  constexpr int RPC = Unpack<S>::RPC;
  constexpr int NT = CG * (N / RPC);
  __shared__ cpx<R> xs[8 * N];
  __shared__ cpx<R> red[CG * N];
  __shared__ cpx<R> v1[N], v2[N];
  __shared__ int nb[9];
  const int h = blockIdx.x, tid = threadIdx.x;
  const size_t off = size_t(blockIdx.y) * hstride;
  in += off;
  out += off;
  const int s = eo_site(g, h, p);
  if (tid < 9) {
    int c[4];
    site_coords(g, s, c);
    nb[tid] = neighbour(g, s, c, tid) >> 1;
  }
  __syncthreads();
  for (int i = tid; i < 8 * N; i += NT) {
    const int d = i / N;
    xs[i] = in[size_t(nb[1 + d]) * N + (i - d * N)];
  }
  if constexpr (MODE != EO_HOP && MODE != EO_AINV_HOP)
    for (int i = tid; i < N; i += NT) v2[i] = xc[off + size_t(h) * N + i];
  __syncthreads();
  const R sc = StoreTraits<S>::scaled ? R(scales[s]) : R(1);
  const S* site_links = links + size_t(s) * 9 * N * N;
  // v1 = H in: the eight hop blocks are columns N .. 9N of the site's block
  stream_cols<S, N, CG, 8 * N>(site_links + size_t(N) * N, xs, red, v1, sc);
  if constexpr (MODE == EO_HOP) {
    for (int i = tid; i < N; i += NT) out[size_t(h) * N + i] = v1[i];
  } else if constexpr (MODE == EO_AINV_HOP) {
    stream_cols<cpx<R>, N, CG, N>(Xinv + size_t(h) * N * N, v1, red, v2, R(1));
    for (int i = tid; i < N; i += NT) out[size_t(h) * N + i] = v2[i];
  } else if constexpr (MODE == EO_A_XC_MINUS_HOP) {
    // X xc with the site block (slot 0)
    stream_cols<S, N, CG, N>(site_links, v2, red, xs, sc);
    for (int i = tid; i < N; i += NT) out[size_t(h) * N + i] = xs[i] - v1[i];
  } else if constexpr (MODE == EO_XC_MINUS_HOP) {
    for (int i = tid; i < N; i += NT) out[size_t(h) * N + i] = v2[i] - v1[i];
  } else {  // EO_AINV_XC_MINUS_HOP
    for (int i = tid; i < N; i += NT) v1[i] = v2[i] - v1[i];
    __syncthreads();
    stream_cols<cpx<R>, N, CG, N>(Xinv + size_t(h) * N * N, v1, red, v2, R(1));
    for (int i = tid; i < N; i += NT) out[size_t(h) * N + i] = v2[i];
  }
}

// X_e^-1 per even site: the dense site block (slot 0, internal [col][row],
// vector precision) inverted in FP64 by Gauss-Jordan with partial pivoting
// in shared memory; written as [V/2][col][row].  status bit 2: singular.
// Sec. 3.3: X_e^-1 of a coarse level, per even site.
template <typename R>
__global__ void k_site_inverse(cpx<R>* __restrict__ out, const cpx<R>* __restrict__ links,
                               Geom g, int n, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<double>* a = reinterpret_cast<cpx<double>*>(smem_raw);  // [row][col], n x n
  cpx<double>* fcol = a + n * n;
  __shared__ int perm[64];
  __shared__ int piv_sh;
  __shared__ cpx<double> pinv_sh;
  const int h = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const int s = eo_site(g, h, 0);
  const cpx<R>* X = links + size_t(s) * 9 * n * n;  // slot 0, [col][row]
  for (int i = tid; i < n * n; i += T) {
    const int col = i / n, row = i - col * n;
    a[row * n + col] = cpx<double>(X[i]);
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      int piv = k;
      double best = norm2(a[k * n + k]);
      for (int i = k + 1; i < n; ++i)
        if (norm2(a[i * n + k]) > best) {
          best = norm2(a[i * n + k]);
          piv = i;
        }
      piv_sh = best > 0.0 ? piv : -1;
      perm[k] = piv;
    }
    __syncthreads();
    const int piv = piv_sh;
    if (piv < 0) {
      if (tid == 0) atomicOr(status, 2);
      return;  // uniform: every thread read the same piv_sh
    }
    if (piv != k)
      for (int j = tid; j < n; j += T) {
        const cpx<double> t = a[k * n + j];
        a[k * n + j] = a[piv * n + j];
        a[piv * n + j] = t;
      }
    __syncthreads();
    if (tid == 0) {
      pinv_sh = crecip(a[k * n + k]);
      a[k * n + k] = cpx<double>(1.0, 0.0);
    }
    __syncthreads();
    const cpx<double> pinv = pinv_sh;
    for (int j = tid; j < n; j += T) a[k * n + j] = a[k * n + j] * pinv;
    for (int i = tid; i < n; i += T) fcol[i] = i == k ? cpx<double>(0.0, 0.0) : a[i * n + k];
    __syncthreads();
    for (int e = tid; e < n * n; e += T) {
      const int i = e / n, j = e - i * n;
      if (i == k) continue;
      if (j == k)
        a[e] = -(fcol[i] * pinv);
      else
        a[e] -= fcol[i] * a[k * n + j];
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    const int pk = perm[k];
    if (pk != k)
      for (int i = tid; i < n; i += T) {
        const cpx<double> t = a[i * n + k];
        a[i * n + k] = a[i * n + pk];
        a[i * n + pk] = t;
      }
    __syncthreads();
  }
  cpx<R>* o = out + size_t(h) * n * n;
  for (int i = tid; i < n * n; i += T) {
    const int col = i / n, row = i - col * n;
    o[i] = cpx<R>(a[row * n + col]);
  }
}

// out_h = X_e^-1 in_h on a compact even vector (CTA per site and RHS)
// Sec. 3.3: X_e^-1 applied on the even sites.
template <typename R, int N, int CG>
__global__ void __launch_bounds__(CG*(N / Unpack<cpx<R>>::RPC))
    k_coarse_xinv(cpx<R>* __restrict__ out, const cpx<R>* __restrict__ in,
                  const cpx<R>* __restrict__ Xinv, size_t hstride) {
  constexpr int NT = CG * (N / Unpack<cpx<R>>::RPC);
  __shared__ cpx<R> xs[N], res[N];
  __shared__ cpx<R> red[CG * N];
  const int h = blockIdx.x;
  const size_t off = size_t(blockIdx.y) * hstride + size_t(h) * N;
  for (int i = threadIdx.x; i < N; i += NT) xs[i] = in[off + i];
  __syncthreads();
  stream_cols<cpx<R>, N, CG, N>(Xinv + size_t(h) * N * N, xs, red, res, R(1));
  for (int i = threadIdx.x; i < N; i += NT) out[off + i] = res[i];
}

template <typename R, int N>
void launch_xinv(const Level& L, Vec out, Vec in, cudaStream_t st) {
  constexpr int CG = Unpack<cpx<R>>::RPC == 1 ? 4 : 8;
  constexpr int NT = CG * (N / Unpack<cpx<R>>::RPC);
  k_coarse_xinv<R, N, CG><<<dim3(unsigned(L.g.vol / 2), unsigned(in.nr)), NT, 0, st>>>(
      (cpx<R>*)out.p, (const cpx<R>*)in.p, L.xinv.as<cpx<R>>(), in.n);
}

template <typename S, int N, int MODE>
void launch_coarse_eo(const Level& L, const void* links, Vec out, Vec in, const void* xc, int p,
                      cudaStream_t st) {
  using R = typename StoreTraits<S>::real;
  constexpr int CG = Unpack<S>::RPC == 1 ? 4 : 8;
  constexpr int NT = CG * (N / Unpack<S>::RPC);
  const dim3 grid(unsigned(L.g.vol / 2), unsigned(in.nr));
  k_coarse_eo<S, N, CG, MODE><<<grid, NT, 0, st>>>(
      (cpx<R>*)out.p, (const cpx<R>*)in.p, (const cpx<R>*)xc, (const S*)links,
      L.scales.as<float>(), L.xinv.as<cpx<R>>(), L.g, p, in.n);
}

template <typename S, int MODE>
bool coarse_eo_n(const Level& L, const void* links, Vec out, Vec in, const void* xc, int p,
                 cudaStream_t st) {
  switch (L.nd) {
    case 16: launch_coarse_eo<S, 16, MODE>(L, links, out, in, xc, p, st); return true;
    case 32: launch_coarse_eo<S, 32, MODE>(L, links, out, in, xc, p, st); return true;
    case 48: launch_coarse_eo<S, 48, MODE>(L, links, out, in, xc, p, st); return true;
    case 64: launch_coarse_eo<S, 64, MODE>(L, links, out, in, xc, p, st); return true;
    default: return false;
  }
}

template <int MODE>
void coarse_eo(const Level& L, Vec out, Vec in, const void* xc, int p, cudaStream_t st) {
  bool ok = false;
  switch (L.prec) {
    case MG_F64: ok = coarse_eo_n<cpx<double>, MODE>(L, L.links.p, out, in, xc, p, st); break;
    case MG_F32: ok = coarse_eo_n<cpx<float>, MODE>(L, L.links.p, out, in, xc, p, st); break;
    case MG_BF16: ok = coarse_eo_n<bf16c, MODE>(L, L.links16.p, out, in, xc, p, st); break;
    case MG_F16: ok = coarse_eo_n<f16c, MODE>(L, L.links16.p, out, in, xc, p, st); break;
    case MG_I16: ok = coarse_eo_n<i16c, MODE>(L, L.links16.p, out, in, xc, p, st); break;
  }
  GB_REQUIRE(ok, MG_ERR_ARG, "red-black: unsupported coarse dof count");
}

template <int MODE>
void fine_eo(mg_ctx* c, Vec out, Vec in, const void* xc, int p, cudaStream_t st) {
  Level& L = c->L[0];
  const dim3 grid(ceil_div(L.g.vol / 2, 128), unsigned(in.nr));
  const int ap = c->p.t_antiperiodic;
  if (L.vprec == MG_F64)
    k_wilson_eo<double, MODE, false><<<grid, 128, 0, st>>>(
        (cpx<double>*)out.p, (const cpx<double>*)in.p, (const cpx<double>*)xc,
        L.gauge64.as<cpx<double>>(), L.clover64.as<double>(), L.ainv.as<double>(), L.g, L.diag,
        p, in.n, ap);
  else if (L.gauge12_ok)  // two-row links: a third fewer link bytes, read twice per S
    k_wilson_eo<float, MODE, true><<<grid, 128, 0, st>>>(
        (cpx<float>*)out.p, (const cpx<float>*)in.p, (const cpx<float>*)xc,
        L.gauge12.as<cpx<float>>(), L.clover32.as<float>(), L.ainv.as<float>(), L.g,
        float(L.diag), p, in.n, ap);
  else
    k_wilson_eo<float, MODE, false><<<grid, 128, 0, st>>>(
        (cpx<float>*)out.p, (const cpx<float>*)in.p, (const cpx<float>*)xc,
        L.gauge32.as<cpx<float>>(), L.clover32.as<float>(), L.ainv.as<float>(), L.g,
        float(L.diag), p, in.n, ap);
}

}  // namespace

bool schur_supported(const mg_ctx* c, int level) {
  const Level& L = c->L[level];
  for (int m = 0; m < 4; ++m)
    if (L.g.L[m] % 2) return false;
  if (level == 0) return true;
  return L.nd == 16 || L.nd == 32 || L.nd == 48 || L.nd == 64;
}

void schur_prepare(mg_ctx* c, int level, cudaStream_t st) {
  Level& L = c->L[level];
  L.have_schur = false;
  if (!schur_supported(c, level)) return;
  const int vh = L.g.vol / 2;
  clear_status(c, st);
  if (level == 0) {
    const size_t n = size_t(vh) * 72;
    if (L.vprec == MG_F64) {
      L.ainv.alloc(n * sizeof(double));
      k_clover_inverse<double><<<ceil_div(L.g.vol, 128), 128, 0, st>>>(
          L.ainv.as<double>(), L.clover64.as<double>(), L.g, L.diag, c->status.as<int>());
    } else {
      L.ainv.alloc(n * sizeof(float));
      k_clover_inverse<float><<<ceil_div(L.g.vol, 128), 128, 0, st>>>(
          L.ainv.as<float>(), L.clover64.as<double>(), L.g, L.diag, c->status.as<int>());
    }
  } else {
    GB_REQUIRE(L.have_op && L.links.p, MG_ERR_STATE, "red-black: coarse operator missing");
    const int n = L.nd;
    const size_t smem = (size_t(n) * n + n) * sizeof(cpx<double>);
    L.xinv.alloc(size_t(vh) * n * n * prec_bytes_complex(L.vprec));
    if (L.vprec == MG_F64) {
      GB_CHECK(cudaFuncSetAttribute(k_site_inverse<double>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
      k_site_inverse<double><<<vh, 256, smem, st>>>(L.xinv.as<cpx<double>>(),
                                                    L.links.as<cpx<double>>(), L.g, n,
                                                    c->status.as<int>());
    } else {
      GB_CHECK(cudaFuncSetAttribute(k_site_inverse<float>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
      k_site_inverse<float><<<vh, 256, smem, st>>>(L.xinv.as<cpx<float>>(),
                                                   L.links.as<cpx<float>>(), L.g, n,
                                                   c->status.as<int>());
    }
  }
  GB_LAUNCH_CHECK();
  c->launches++;
  if (read_status(c, st) & 2)
    throw Error(MG_ERR_NUMERICAL, "red-black: singular site-local block");
  L.have_schur = true;
}

void eo_apply(mg_ctx* c, int level, int mode, Vec out, Vec in, const void* xc, int p,
              cudaStream_t st) {
  const Level& L = c->L[level];
  GB_REQUIRE(L.have_schur, MG_ERR_STATE, "red-black operator not prepared");
  if (level == 0) {
    switch (mode) {
      case EO_HOP: fine_eo<EO_HOP>(c, out, in, xc, p, st); break;
      case EO_AINV_HOP: fine_eo<EO_AINV_HOP>(c, out, in, xc, p, st); break;
      case EO_A_XC_MINUS_HOP: fine_eo<EO_A_XC_MINUS_HOP>(c, out, in, xc, p, st); break;
      case EO_XC_MINUS_HOP: fine_eo<EO_XC_MINUS_HOP>(c, out, in, xc, p, st); break;
      default: fine_eo<EO_AINV_XC_MINUS_HOP>(c, out, in, xc, p, st); break;
    }
  } else {
    switch (mode) {
      case EO_HOP: coarse_eo<EO_HOP>(L, out, in, xc, p, st); break;
      case EO_AINV_HOP: coarse_eo<EO_AINV_HOP>(L, out, in, xc, p, st); break;
      case EO_A_XC_MINUS_HOP: coarse_eo<EO_A_XC_MINUS_HOP>(L, out, in, xc, p, st); break;
      case EO_XC_MINUS_HOP: coarse_eo<EO_XC_MINUS_HOP>(L, out, in, xc, p, st); break;
      default: coarse_eo<EO_AINV_XC_MINUS_HOP>(L, out, in, xc, p, st); break;
    }
  }
  GB_LAUNCH_CHECK();
  c->launches++;
}

void eo_split(mg_ctx* c, int level, Vec he, Vec ho, Vec full, cudaStream_t st) {
  const Level& L = c->L[level];
  const dim3 grid(ceil_div(full.n, 256) > 152 * 16 ? 152 * 16 : ceil_div(full.n, 256),
                  unsigned(full.nr));
  if (full.prec == MG_F64)
    k_eo_split<double><<<grid, 256, 0, st>>>((cpx<double>*)he.p, (cpx<double>*)ho.p,
                                             (const cpx<double>*)full.p, L.g, L.nd, full.n, he.n);
  else
    k_eo_split<float><<<grid, 256, 0, st>>>((cpx<float>*)he.p, (cpx<float>*)ho.p,
                                            (const cpx<float>*)full.p, L.g, L.nd, full.n, he.n);
  GB_LAUNCH_CHECK();
  c->launches++;
}

void eo_merge(mg_ctx* c, int level, Vec full, Vec he, Vec ho, cudaStream_t st) {
  const Level& L = c->L[level];
  const dim3 grid(ceil_div(full.n, 256) > 152 * 16 ? 152 * 16 : ceil_div(full.n, 256),
                  unsigned(full.nr));
  if (full.prec == MG_F64)
    k_eo_merge<double><<<grid, 256, 0, st>>>((cpx<double>*)full.p, (const cpx<double>*)he.p,
                                             (const cpx<double>*)ho.p, L.g, L.nd, full.n, he.n);
  else
    k_eo_merge<float><<<grid, 256, 0, st>>>((cpx<float>*)full.p, (const cpx<float>*)he.p,
                                            (const cpx<float>*)ho.p, L.g, L.nd, full.n, he.n);
  GB_LAUNCH_CHECK();
  c->launches++;
}

// t_e = A_e^-1 x_e
void eo_ainv(mg_ctx* c, int level, Vec out, Vec in, cudaStream_t st) {
  const Level& L = c->L[level];
  GB_REQUIRE(L.have_schur, MG_ERR_STATE, "red-black operator not prepared");
  if (level == 0) {
    const dim3 grid(ceil_div(L.g.vol / 2, 128), unsigned(in.nr));
    if (L.vprec == MG_F64)
      k_clover_inv_apply<double><<<grid, 128, 0, st>>>((cpx<double>*)out.p,
                                                       (const cpx<double>*)in.p,
                                                       L.ainv.as<double>(), L.g.vol / 2, in.n);
    else
      k_clover_inv_apply<float><<<grid, 128, 0, st>>>((cpx<float>*)out.p,
                                                      (const cpx<float>*)in.p,
                                                      L.ainv.as<float>(), L.g.vol / 2, in.n);
    GB_LAUNCH_CHECK();
    c->launches++;
  } else {
    bool ok = false;
    if (L.vprec == MG_F64) {
      switch (L.nd) {
        case 16: launch_xinv<double, 16>(L, out, in, st); ok = true; break;
        case 32: launch_xinv<double, 32>(L, out, in, st); ok = true; break;
        case 48: launch_xinv<double, 48>(L, out, in, st); ok = true; break;
        case 64: launch_xinv<double, 64>(L, out, in, st); ok = true; break;
      }
    } else {
      switch (L.nd) {
        case 16: launch_xinv<float, 16>(L, out, in, st); ok = true; break;
        case 32: launch_xinv<float, 32>(L, out, in, st); ok = true; break;
        case 48: launch_xinv<float, 48>(L, out, in, st); ok = true; break;
        case 64: launch_xinv<float, 64>(L, out, in, st); ok = true; break;
      }
    }
    GB_REQUIRE(ok, MG_ERR_ARG, "red-black: unsupported coarse dof count");
    GB_LAUNCH_CHECK();
    c->launches++;
  }
}

}  // namespace gbmg
