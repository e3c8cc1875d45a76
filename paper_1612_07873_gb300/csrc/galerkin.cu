// Galerkin coarse operator, Sec. 3.4 step 4:  M_hat = P^dag M P, stored as
// the nine blocks of Eq. (3) per coarse site.
//
// For coarse site xc and slot d:
//   d != 0:  Y_d(xc) = sum_{x in A(xc), hop x->x+d leaves A} P(x)^dag H_d(x) P(x+d)
//   d == 0:  X(xc)   = sum_{x in A(xc)} P(x)^dag [ D(x) P(x) + sum_{d' inside A} H_d'(x) P(x+d') ]
// with H_d the fine operator's block in slot d and P(x) the nf x 2Nv local
// prolongator (column (s, j) = null vector j on the chirality-s dofs).
// A hop x -> x+mu leaves A exactly when x_mu mod b_mu = b_mu - 1 (x - mu:
// when x_mu mod b_mu = 0), also when the coarse extent is 1.
//
// One CTA per (xc, d).  Per fine site x it builds T = (term) P in shared
// memory and accumulates P(x)^dag T into per-thread output registers.
// Fine level (Wilson-clover, nf = 12): each term applies a spin-projected
// hop; terms go to separate shared slices and are summed in a fixed order,
// so the result is deterministic.  Coarse level: T is a dense product with
// the level's link blocks.
#include "async_copy.cuh"
#include "kernels.cuh"
#include "wilson_ops.cuh"

namespace gbmg {

namespace {

struct AggGeom {
  Geom fine, coarse;
  int b[4];
  int per;
};

__device__ __forceinline__ int fine_site(const AggGeom& m, int xc, int ls, int lc[4]) {
  int cc[4];
  site_coords(m.coarse, xc, cc);
  lc[0] = ls % m.b[0];
  ls /= m.b[0];
  lc[1] = ls % m.b[1];
  ls /= m.b[1];
  lc[2] = ls % m.b[2];
  lc[3] = ls / m.b[2];
  return (cc[0] * m.b[0] + lc[0]) + m.fine.stride[1] * (cc[1] * m.b[1] + lc[1]) +
         m.fine.stride[2] * (cc[2] * m.b[2] + lc[2]) + m.fine.stride[3] * (cc[3] * m.b[3] + lc[3]);
}

__device__ __forceinline__ bool leaves(const AggGeom& m, const int lc[4], int d) {
  int mu = (d - 1) >> 1;
  bool fwd = ((d - 1) & 1) == 0;
  return fwd ? (lc[mu] == m.b[mu] - 1) : (lc[mu] == 0);
}

template <typename R>
struct WilsonOp {
  static constexpr bool wilson = true;
  const cpx<R>* U;   // [4][V][9]
  const R* A;        // [V][72]
  R diag;
};

template <typename R>
struct CoarseOp {
  static constexpr bool wilson = false;
  const cpx<R>* links;  // [V][9][col][row]
};

// MAXO: output elements per thread (>= (2Nv)^2 / blockDim).  TILE > 0: the
// 256 threads form a 16 x 16 grid, thread (ty, tx) owning output rows
// ty*TILE.. and columns tx*TILE.. (2Nv = 16 TILE, MAXO = TILE^2), so that a
// shared-memory load of P(x) or T feeds TILE complex MACs.
// Sec. 3.4 step 4: P^dag M P into the nine blocks of Eq. (3).
template <typename R, typename Rout, typename Op, int MAXO, int TILE>
__global__ void __launch_bounds__(256) k_galerkin(Op op, const cpx<R>* __restrict__ Vp, AggGeom m,
                                                  int nf, int nv, cpx<Rout>* __restrict__ out) {
  extern __shared__ unsigned char smem_raw[];
  const int n2 = 2 * nv;
  const int halff = nf / 2;
  cpx<R>* sV = reinterpret_cast<cpx<R>*>(smem_raw);  // [nf][nv]
  cpx<R>* sT = sV + nf * nv;                          // [nf][n2]
  cpx<R>* sSl = sT + nf * n2;                         // Wilson: [9][12][n2] term slices
  __shared__ int s_nb[9];
  __shared__ int s_act[9];

  const int xc = blockIdx.x;
  const int d = blockIdx.y;
  const int tid = threadIdx.x, T = blockDim.x;

  cpx<R> acc[MAXO];
#pragma unroll
  for (int k = 0; k < MAXO; ++k) acc[k] = cpx<R>(R(0), R(0));

  for (int ls = 0; ls < m.per; ++ls) {
    int lc[4];
    const int x = fine_site(m, xc, ls, lc);
    if (d != 0 && !leaves(m, lc, d)) continue;  // uniform over the CTA
    __syncthreads();
    if (tid < 9) {
      int c[4];
      site_coords(m.fine, x, c);
      s_nb[tid] = neighbour(m.fine, x, c, tid);
      // active terms: slot d alone for a face hop; for X the diagonal and every
      // hop that stays inside the aggregate
      s_act[tid] = (d != 0) ? (tid == d) : (tid == 0 || !leaves(m, lc, tid));
    }
    for (int k = tid; k < nf * nv; k += T) sV[k] = Vp[size_t(x) * nf * nv + k];
    __syncthreads();

    if constexpr (Op::wilson) {
      // items (term e, column c): slice e, column c = H_e(x) P_c(x + e)
      for (int it = tid; it < 9 * n2; it += T) {
        const int e = it / n2, col = it - e * n2;
        if (!s_act[e]) continue;
        const int sp = col / nv, j = col - sp * nv;
        const cpx<R>* src = Vp + size_t(s_nb[e]) * 12 * nv + j;
        cpx<R> psi[12], o[12];
#pragma unroll
        for (int a = 0; a < 12; ++a) {
          psi[a] = ((a / 6) == sp) ? src[a * nv] : cpx<R>(R(0), R(0));
          o[a] = cpx<R>(R(0), R(0));
        }
        if (e == 0) {
          clover_accum(op.A + size_t(x) * 72, op.diag, psi, o);
        } else {
          const int mu = (e - 1) >> 1;
          const bool fwd = ((e - 1) & 1) == 0;
          const int ls_ = fwd ? x : s_nb[e];
          hop_accum_rt(mu, fwd, op.U + (size_t(mu) * m.fine.vol + ls_) * 9, psi, o);
        }
#pragma unroll
        for (int a = 0; a < 12; ++a) sSl[(e * 12 + a) * n2 + col] = o[a];
      }
      __syncthreads();
      for (int k = tid; k < 12 * n2; k += T) {
        cpx<R> s(R(0), R(0));
        for (int e = 0; e < 9; ++e)
          if (s_act[e]) s += sSl[e * 12 * n2 + k];
        sT[k] = s;
      }
    } else {
      // T[a][c] = sum_e sum_{b in chi(c)} H_e(x)[a][b] P(x+e)[b][j]
      for (int it = tid; it < nf * n2; it += T) {
        const int col = it / nf, a = it - col * nf;
        const int sp = col / nv, j = col - sp * nv;
        cpx<R> s(R(0), R(0));
        for (int e = 0; e < 9; ++e) {
          if (!s_act[e]) continue;
          const cpx<R>* H = op.links + (size_t(x) * 9 + e) * nf * nf + a;
          const cpx<R>* src = Vp + size_t(s_nb[e]) * nf * nv + j;
          for (int b = sp * halff; b < (sp + 1) * halff; ++b)
            cmac(s, H[size_t(b) * nf], src[size_t(b) * nv]);
        }
        sT[a * n2 + col] = s;
      }
    }
    __syncthreads();

    // acc[(s,i),(s',j)] += sum_{a in chi s} conj(P(x)[a][i]) T[a][(s',j)]
    if constexpr (TILE > 0) {
      const int r0 = (tid >> 4) * TILE, c0 = (tid & 15) * TILE;
      const int s = r0 / nv, i0 = r0 - s * nv;
      for (int a = s * halff; a < (s + 1) * halff; ++a) {
        cpx<R> pv[TILE], tv[TILE];
#pragma unroll
        for (int u = 0; u < TILE; ++u) {
          pv[u] = sV[a * nv + i0 + u];
          tv[u] = sT[a * n2 + c0 + u];
        }
#pragma unroll
        for (int u = 0; u < TILE; ++u)
#pragma unroll
          for (int w = 0; w < TILE; ++w) cmac_conj(acc[u * TILE + w], pv[u], tv[w]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < MAXO; ++k) {
        const int o = tid + k * T;
        if (o < n2 * n2) {
          const int row = o / n2, col = o - row * n2;
          const int s = row / nv, i = row - s * nv;
          cpx<R> a_ = acc[k];
          for (int a = s * halff; a < (s + 1) * halff; ++a)
            cmac_conj(a_, sV[a * nv + i], sT[a * n2 + col]);
          acc[k] = a_;
        }
      }
    }
  }
  // internal layout [xc][d][col][row]
  cpx<Rout>* dst = out + (size_t(xc) * 9 + d) * n2 * n2;
  if constexpr (TILE > 0) {
    const int r0 = (tid >> 4) * TILE, c0 = (tid & 15) * TILE;
#pragma unroll
    for (int u = 0; u < TILE; ++u)
#pragma unroll
      for (int w = 0; w < TILE; ++w)
        dst[size_t(c0 + w) * n2 + r0 + u] = cpx<Rout>(acc[u * TILE + w]);
  } else {
#pragma unroll
    for (int k = 0; k < MAXO; ++k) {
      const int o = tid + k * T;
      if (o < n2 * n2) {
        const int row = o / n2, col = o - row * n2;
        dst[size_t(col) * n2 + row] = cpx<Rout>(acc[k]);
      }
    }
  }
}

// four consecutive complex numbers from a 16-byte aligned address
__device__ __forceinline__ void load4c(const cpx<float>* p, cpx<float> v[4]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  v[0] = cpx<float>(a.x, a.y);
  v[1] = cpx<float>(a.z, a.w);
  v[2] = cpx<float>(b.x, b.y);
  v[3] = cpx<float>(b.z, b.w);
}
__device__ __forceinline__ void load4c(const cpx<double>* p, cpx<double> v[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p) + k);
    v[k] = cpx<double>(a.x, a.y);
  }
}

template <int E>
struct TermIdx {
  static constexpr int value = E;
};

// Column j of chirality SP of T(x) = sum_e H_e(x) P(x + e) at the fine
// Wilson-clover level, for output block d: the single hop d for Y_d; for X
// the clover block of chirality SP, then the eight hops (each applied when
// it stays inside the aggregate), with the next hop's P entries and link
// loaded before the current hop is applied.  P(x + e) of the column lives
// on chirality SP only, so the other six spinor entries are zero.
template <int SP, typename R>
__device__ __forceinline__ void t_column(const WilsonOp<R>& op, const cpx<R>* __restrict__ Vp,
                                         int vol, int nv, int x, const int* nbk, const int* ak,
                                         int d, int j, cpx<R> o[12]) {
  auto load_v = [&](int y, cpx<R> v[6]) {
    const cpx<R>* src = Vp + (size_t(y) * 12 + 6 * SP) * nv + j;
#pragma unroll
    for (int a = 0; a < 6; ++a) v[a] = src[a * nv];
  };
  auto load_u = [&](int mu, int ls, cpx<R> u[9]) {
    const cpx<R>* U = op.U + (size_t(mu) * vol + ls) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = U[k];
  };
  auto spinor = [&](const cpx<R> v[6], cpx<R> psi[12]) {
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      psi[6 * SP + a] = v[a];
      psi[6 * (1 - SP) + a] = cpx<R>(R(0), R(0));
    }
  };
#pragma unroll
  for (int a = 0; a < 12; ++a) o[a] = cpx<R>(R(0), R(0));
  if (d != 0) {
    const int mu = (d - 1) >> 1;
    const bool fwd = ((d - 1) & 1) == 0;
    cpx<R> v[6], u[9], psi[12];
    load_v(nbk[d], v);
    load_u(mu, fwd ? x : nbk[d], u);
    spinor(v, psi);
    hop_accum_rt(mu, fwd, u, psi, o);
    return;
  }
  {
    // the column lives on chirality SP: only that clover block acts
    cpx<R> v[6];
    load_v(x, v);
    clover_block_accum(op.A + size_t(x) * 72 + 36 * SP, op.diag, v, o + 6 * SP);
  }
  cpx<R> v[6], u[9];
  load_v(nbk[1], v);
  load_u(0, x, u);
  auto step = [&](auto ic) {
    constexpr int E = decltype(ic)::value;
    constexpr int MU = (E - 1) >> 1;
    constexpr bool FWD = ((E - 1) & 1) == 0;
    cpx<R> vn[6], un[9];
    if constexpr (E < 8) {
      // hop E + 1: direction E / 2, forward when E is even
      load_v(nbk[E + 1], vn);
      load_u(E >> 1, (E & 1) == 0 ? x : nbk[E + 1], un);
    }
    if (ak[E]) {
      cpx<R> psi[12];
      spinor(v, psi);
      hop_accum<MU, FWD>(u, psi, o);
    }
    if constexpr (E < 8) {
#pragma unroll
      for (int a = 0; a < 6; ++a) v[a] = vn[a];
#pragma unroll
      for (int k = 0; k < 9; ++k) u[k] = un[k];
    }
  };
  step(TermIdx<1>{});
  step(TermIdx<2>{});
  step(TermIdx<3>{});
  step(TermIdx<4>{});
  step(TermIdx<5>{});
  step(TermIdx<6>{});
  step(TermIdx<7>{});
  step(TermIdx<8>{});
}

// Chunked form of the same product for 2Nv = 16 TILE: the fine sites that
// contribute to (xc, d) -- every site of the aggregate for X, the sites on
// the face d leaves through for Y_d -- are processed CH at a time.  Per
// chunk the CTA stages P(x) of the CH sites, then every thread computes
// columns of T(x) = sum_e H_e(x) P(x + e) for (site, column) items (all the
// terms of one item in one thread, so no per-term slices are needed), then
// the 16 x 16 thread grid accumulates P(x)^dag T(x) over the chunk's
// K = CH x nf / 2 values of each chirality in TILE x TILE register tiles.
// Three block barriers per chunk instead of three per fine site; the
// contributing sites are enumerated from their index (no serial list).
// P(x) of the chunk's sites (contiguous rows of the prolongator) arrives by
// bulk copies issued before the T products, so the copies overlap them;
// the contraction waits on the copies' mbarrier (bounded: on a timeout the
// CTA records it in *err and leaves).
template <typename R, typename Rout, typename Op, int TILE>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1)
    k_galerkin_chunk(Op op, const cpx<R>* __restrict__ Vp,
                                                        AggGeom m, int nf, int nv, int CH,
                                                        cpx<Rout>* __restrict__ out,
                                                        int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t vbar;
  const int n2 = 2 * nv;
  const int halff = nf / 2;
  cpx<R>* sV = reinterpret_cast<cpx<R>*>(smem_raw);  // [CH][nf][nv]
  cpx<R>* sT = sV + size_t(CH) * nf * nv;             // [CH][nf][n2]
  int* s_x = reinterpret_cast<int*>(sT + size_t(CH) * nf * n2);  // [CH] fine site
  int* s_nb = s_x + CH;                                          // [CH][9] partners
  int* s_act = s_nb + 9 * CH;                                    // [CH][9] active terms
  const int xc = blockIdx.x;
  const int d = blockIdx.y;
  const int tid = threadIdx.x;
  // contributing fine sites: every site of the aggregate for X (d = 0);
  // for Y_d the face that d leaves through (x_mu = b_mu - 1 forward, 0
  // backward), enumerated over the other three coordinates in order
  const int dmu = d > 0 ? (d - 1) >> 1 : 0;
  const bool dfwd = d > 0 && ((d - 1) & 1) == 0;
  // (a select, not m.b[dmu]: a kernel-parameter array indexed at run time
  // would be copied to the stack)
  const int bmu = dmu == 0 ? m.b[0] : dmu == 1 ? m.b[1] : dmu == 2 ? m.b[2] : m.b[3];
  const int cnt = d == 0 ? m.per : m.per / bmu;
  auto contrib_ls = [&](int q) {
    if (d == 0) return q;
    int lc[4];
#pragma unroll
    for (int nu = 0; nu < 4; ++nu) {
      if (nu == dmu) {
        lc[nu] = dfwd ? m.b[nu] - 1 : 0;
      } else {
        lc[nu] = q % m.b[nu];
        q /= m.b[nu];
      }
    }
    return lc[0] + m.b[0] * (lc[1] + m.b[1] * (lc[2] + m.b[2] * lc[3]));
  };
  const int r0 = (tid >> 4) * TILE, c0 = (tid & 15) * TILE;
  const int srow = r0 / nv, i0 = r0 - srow * nv;
  cpx<R> acc[TILE * TILE];
#pragma unroll
  for (int k = 0; k < TILE * TILE; ++k) acc[k] = cpx<R>(R(0), R(0));
  if (tid == 0) {
    mbar_init(&vbar, 1);
    fence_mbar_init();
  }
  const uint32_t pbytes = uint32_t(nf) * uint32_t(nv) * uint32_t(sizeof(cpx<R>));
  uint32_t vphase = 0;

  for (int k0 = 0; k0 < cnt; k0 += CH) {
    const int nk = min(CH, cnt - k0);
    __syncthreads();  // the previous chunk's tiles are consumed
    // one thread per chunk site: the site, its partner across each term and
    // whether the term contributes to this block
    if (tid < nk) {
      int lc[4], c[4];
      const int x = fine_site(m, xc, contrib_ls(k0 + tid), lc);
      site_coords(m.fine, x, c);
      s_x[tid] = x;
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        s_nb[tid * 9 + e] = neighbour(m.fine, x, c, e);
        s_act[tid * 9 + e] = (d != 0) ? (e == d) : (e == 0 || !leaves(m, lc, e));
      }
    }
    __syncthreads();
    if (tid == 0) {
      // the previous chunk's reads of sV are ordered before the copies that
      // overwrite it
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&vbar, uint32_t(nk) * pbytes);
      for (int sk = 0; sk < nk; ++sk)
        bulk_g2s_plain(sV + size_t(sk) * nf * nv, Vp + size_t(s_x[sk]) * nf * nv, pbytes, &vbar);
    }
    if constexpr (Op::wilson) {
      // items (chirality sp, chunk site, column j within sp), sp slowest so
      // a warp's items share sp: T[site][.][sp nv + j] = sum_e H_e P_col(x + e)
      for (int it = tid; it < nk * n2; it += 256) {
        const int sp = it / (nk * nv);
        const int rem = it - sp * nk * nv;
        const int sk = rem / nv, j = rem - sk * nv;
        const int col = sp * nv + j;
        cpx<R> o[12];
        if (sp == 0)
          t_column<0>(op, Vp, m.fine.vol, nv, s_x[sk], s_nb + sk * 9, s_act + sk * 9, d, j, o);
        else
          t_column<1>(op, Vp, m.fine.vol, nv, s_x[sk], s_nb + sk * 9, s_act + sk * 9, d, j, o);
#pragma unroll
        for (int a = 0; a < 12; ++a) sT[(size_t(sk) * 12 + a) * n2 + col] = o[a];
      }
    } else if (nf % 4 == 0 && nv % 4 == 0) {
      // T[site][a][col] = sum_e sum_{b in chi(col)} H_e(x)[a][b] P(x+e)[b][j]
      // in register tiles of 4 rows a x 4 columns j of one chirality: per
      // (term, b) 16-byte loads of rows a0..a0+3 of H_e's column b (the
      // [col][row] store keeps them contiguous) and of columns j0..j0+3 of
      // P(x+e)'s row b, then 16 complex MACs.  Items (site, chirality, j
      // tile, a tile), a tile fastest: a warp's H loads are one contiguous
      // run, its P loads shared.
      const int atn = nf / 4, jtn = nv / 4;
      const int per_site = 2 * atn * jtn;
      for (int it = tid; it < nk * per_site; it += 256) {
        const int sk = it / per_site;
        int rem = it - sk * per_site;
        const int at = rem % atn;
        rem /= atn;
        const int jt = rem % jtn, sp = rem / jtn;
        const int a0 = 4 * at, j0 = 4 * jt;
        const int x = s_x[sk];
        cpx<R> t[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int w = 0; w < 4; ++w) t[u][w] = cpx<R>(R(0), R(0));
        for (int e = 0; e < 9; ++e) {
          if (!s_act[sk * 9 + e]) continue;
          const cpx<R>* H = op.links + (size_t(x) * 9 + e) * nf * nf + a0;
          const cpx<R>* src = Vp + size_t(s_nb[sk * 9 + e]) * nf * nv + j0;
#pragma unroll 2
          for (int b = sp * halff; b < (sp + 1) * halff; ++b) {
            cpx<R> h[4], q[4];
            load4c(H + size_t(b) * nf, h);
            load4c(src + size_t(b) * nv, q);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int w = 0; w < 4; ++w) cmac(t[u][w], h[u], q[w]);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int w = 0; w < 4; ++w)
            sT[(size_t(sk) * nf + a0 + u) * n2 + sp * nv + j0 + w] = t[u][w];
      }
    } else {
      // T[site][a][col] = sum_e sum_{b in chi(col)} H_e(x)[a][b] P(x+e)[b][j]
      for (int it = tid; it < nk * nf * n2; it += 256) {
        const int sk = it / (nf * n2), rem = it - sk * nf * n2;
        const int col = rem / nf, a = rem - col * nf;
        const int sp = col / nv, j = col - sp * nv;
        const int x = s_x[sk];
        cpx<R> t(R(0), R(0));
        for (int e = 0; e < 9; ++e) {
          if (!s_act[sk * 9 + e]) continue;
          const cpx<R>* H = op.links + (size_t(x) * 9 + e) * nf * nf + a;
          const cpx<R>* src = Vp + size_t(s_nb[sk * 9 + e]) * nf * nv + j;
          for (int b = sp * halff; b < (sp + 1) * halff; ++b)
            cmac(t, H[size_t(b) * nf], src[size_t(b) * nv]);
        }
        sT[(size_t(sk) * nf + a) * n2 + col] = t;
      }
    }
    __syncthreads();
    if (!mbar_wait(&vbar, vphase)) {
      // the copies did not land within the budget: record it, give them a
      // second bounded wait and leave
      if (tid == 0) {
        atomicOr(err, 1);
        mbar_wait(&vbar, vphase);
      }
      return;
    }
    vphase ^= 1u;
    // acc[(s,i),(s',j)] += sum_{site, a in chi s} conj(P(x)[a][i]) T(x)[a][(s',j)]
    for (int sk = 0; sk < nk; ++sk) {
      const cpx<R>* Vk = sV + size_t(sk) * nf * nv;
      const cpx<R>* Tk = sT + size_t(sk) * nf * n2;
#pragma unroll 2
      for (int a = srow * halff; a < (srow + 1) * halff; ++a) {
        cpx<R> pv[TILE], tv[TILE];
#pragma unroll
        for (int u = 0; u < TILE; ++u) {
          pv[u] = Vk[a * nv + i0 + u];
          tv[u] = Tk[a * n2 + c0 + u];
        }
#pragma unroll
        for (int u = 0; u < TILE; ++u)
#pragma unroll
          for (int w = 0; w < TILE; ++w) cmac_conj(acc[u * TILE + w], pv[u], tv[w]);
      }
    }
  }
  // internal layout [xc][d][col][row]
  cpx<Rout>* dst = out + (size_t(xc) * 9 + d) * n2 * n2;
#pragma unroll
  for (int u = 0; u < TILE; ++u)
#pragma unroll
    for (int w = 0; w < TILE; ++w)
      dst[size_t(c0 + w) * n2 + r0 + u] = cpx<Rout>(acc[u * TILE + w]);
}

template <typename R, typename Rout, typename Op>
void launch_galerkin(const Op& op, const cpx<R>* Vp, const AggGeom& m, int nf, int nv,
                     cpx<Rout>* out, int* err, cudaStream_t st) {
  const int n2 = 2 * nv;
  size_t smem = size_t(nf) * nv * sizeof(cpx<R>) + size_t(nf) * n2 * sizeof(cpx<R>);
  if (Op::wilson) smem += size_t(9) * 12 * n2 * sizeof(cpx<R>);
  dim3 grid(m.coarse.vol, 9);
  const int per_thread = (n2 * n2 + 255) / 256;
  auto go = [&](auto kern) {
    GB_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    kern<<<grid, 256, smem, st>>>(op, Vp, m, nf, nv, out);
  };
  // chunked kernel: as many fine sites per chunk (up to 16) as two CTAs per
  // SM leave room for
  // (the chunked kernel bulk-copies rows of Vp: 16-byte aligned)
  if ((n2 == 32 || n2 == 48 || n2 == 64) && reinterpret_cast<uintptr_t>(Vp) % 16 == 0) {
    const size_t per_site = (size_t(nf) * nv + size_t(nf) * n2) * sizeof(cpx<R>) + 19 * sizeof(int);
    const size_t budget = 110 * 1024;
    int CH = int(budget / per_site);
    if (CH > 16) CH = 16;
    if (CH < 1) CH = 1;
    const size_t csm = size_t(CH) * per_site;
    auto goc = [&](auto kern) {
      GB_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(csm)));
      kern<<<grid, 256, csm, st>>>(op, Vp, m, nf, nv, CH, out, err);
    };
    if (n2 == 32)
      goc(k_galerkin_chunk<R, Rout, Op, 2>);
    else if (n2 == 48)
      goc(k_galerkin_chunk<R, Rout, Op, 3>);
    else
      goc(k_galerkin_chunk<R, Rout, Op, 4>);
  } else if (per_thread <= 4)
    go(k_galerkin<R, Rout, Op, 4, 0>);
  else if (per_thread <= 9)
    go(k_galerkin<R, Rout, Op, 9, 0>);
  else if (per_thread <= 16)
    go(k_galerkin<R, Rout, Op, 16, 0>);
  else if (per_thread <= 36)
    go(k_galerkin<R, Rout, Op, 36, 0>);
  else
    throw Error(MG_ERR_ARG, "galerkin: too many null vectors (2Nv > 96)");
  GB_LAUNCH_CHECK();
}

}  // namespace

void galerkin_build(mg_ctx* c, int level, cudaStream_t st) {
  Level& F = c->L[level];
  Level& C = c->L[level + 1];
  GB_REQUIRE(F.have_V, MG_ERR_STATE, "build_coarse: null vectors not set");
  GB_REQUIRE(level == 0 || F.have_op, MG_ERR_STATE, "build_coarse: level operator missing");
  AggGeom m;
  m.fine = F.g;
  m.coarse = C.g;
  for (int i = 0; i < 4; ++i) m.b[i] = F.block[i];
  m.per = F.g.vol / C.g.vol;
  const int nf = F.nd, nv = F.nvec;
  const size_t total = size_t(C.g.vol) * 9 * C.nd * C.nd;
  C.links.alloc(total * prec_bytes_complex(C.vprec));
  // arithmetic per fine site: the P^dag T contractions (8 n2 nv nf flop
  // each) of X and of the exit-face Y blocks (1 + sum_mu 2 / b_mu per site),
  // and the T = H P columns: at the Wilson-clover level the clover block of
  // the column's chirality (270 flop) and eight hops (204 flop each), at a
  // coarse level nine dense nf x nf/2 blocks (36 nf^2 flop)
  double blocks = 1.0;
  for (int mu = 0; mu < 4; ++mu) blocks += 2.0 / F.block[mu];
  const double n2d = 2.0 * nv;
  const double tcol = level == 0 ? 270.0 + 8.0 * 204.0 : 36.0 * nf * nf;
  const double flops = double(F.g.vol) * (blocks * 8.0 * n2d * nv * nf + n2d * tcol);
  ProfScope ps(c->prof, st, "galerkin", level, double(F.g.vol) * nf * nv * 16.0, flops);
  int* err = c->status.as<int>() + 1;
  if (F.vprec == MG_F64) {
    GB_REQUIRE(C.vprec == MG_F64, MG_ERR_ARG, "FP64 level above an FP32 level is not supported");
    if (level == 0) {
      WilsonOp<double> op{F.gauge64.as<cpx<double>>(), F.clover64.as<double>(), F.diag};
      launch_galerkin<double, double>(op, F.Vp.as<cpx<double>>(), m, nf, nv,
                                      C.links.as<cpx<double>>(), err, st);
    } else {
      CoarseOp<double> op{F.links.as<cpx<double>>()};
      launch_galerkin<double, double>(op, F.Vp.as<cpx<double>>(), m, nf, nv,
                                      C.links.as<cpx<double>>(), err, st);
    }
  } else {
    GB_REQUIRE(C.vprec == MG_F32, MG_ERR_ARG, "FP64 level above an FP32 level is not supported");
    if (level == 0) {
      WilsonOp<float> op{F.gauge32.as<cpx<float>>(), F.clover32.as<float>(), float(F.diag)};
      launch_galerkin<float, float>(op, F.Vp.as<cpx<float>>(), m, nf, nv, C.links.as<cpx<float>>(),
                                    err, st);
    } else {
      CoarseOp<float> op{F.links.as<cpx<float>>()};
      launch_galerkin<float, float>(op, F.Vp.as<cpx<float>>(), m, nf, nv, C.links.as<cpx<float>>(),
                                    err, st);
    }
  }
  c->launches++;
  links_pack16(c, level + 1, st);
  C.have_op = true;
}

}  // namespace gbmg
