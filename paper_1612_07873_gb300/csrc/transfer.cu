// Null-vector block orthonormalisation (Sec. 3.4 step 3 with the chiral
// split of its footnote) and the transfer operators of Sec. 6.6.
//
// For aggregate A and chirality s the (|A| * nd/2) x Nv block of chirality-s
// components is orthonormalised column by column by Gram-Schmidt at FP64
// accuracy in float-float arithmetic on the FP32 pipe (projection repeated
// when the first one cancels more than half of the column's squared norm;
// see k_block_qr).  Rows are ordered (site of A in
// lexicographic order, dof of chirality s).  The prolongator column (s, i)
// is vector i of the result restricted to chirality s; coarse dof = s*Nv + i.
//
// Transfer layout Vp: [fine site][dof][Nv] in the level's vector precision,
// so the Nv coefficients of one fine dof are contiguous.
#include <mutex>

#include <type_traits>

#include "kernels.cuh"
#include "tune.cuh"

namespace gbmg {

namespace {

struct AggMap {
  Geom fine, coarse;
  int b[4];
  int per;  // fine sites per aggregate
};

__host__ __device__ __forceinline__ int agg_of(const AggMap& m, const int c[4]) {
  return (c[0] / m.b[0]) + m.coarse.stride[1] * (c[1] / m.b[1]) +
         m.coarse.stride[2] * (c[2] / m.b[2]) + m.coarse.stride[3] * (c[3] / m.b[3]);
}
__host__ __device__ __forceinline__ int local_of(const AggMap& m, const int c[4]) {
  int l0 = c[0] % m.b[0], l1 = c[1] % m.b[1], l2 = c[2] % m.b[2], l3 = c[3] % m.b[3];
  return l0 + m.b[0] * (l1 + m.b[1] * (l2 + m.b[2] * l3));
}
// fine site of local index ls inside aggregate xc
__host__ __device__ __forceinline__ int fine_of(const AggMap& m, int xc, int ls) {
  int cc[4], c[4];
  site_coords(m.coarse, xc, cc);
  c[0] = cc[0] * m.b[0] + ls % m.b[0];
  ls /= m.b[0];
  c[1] = cc[1] * m.b[1] + ls % m.b[1];
  ls /= m.b[1];
  c[2] = cc[2] * m.b[2] + ls % m.b[2];
  c[3] = cc[3] * m.b[3] + ls / m.b[2];
  return c[0] + m.fine.stride[1] * c[1] + m.fine.stride[2] * c[2] + m.fine.stride[3] * c[3];
}

AggMap make_map(const Level& f, const Level& c) {
  AggMap m;
  m.fine = f.g;
  m.coarse = c.g;
  for (int i = 0; i < 4; ++i) m.b[i] = f.block[i];
  m.per = f.g.vol / c.g.vol;
  return m;
}

// ---------------------------------------------------------------------------
// Float-float complex numbers: value = (rh + rl) + i (ih + il) with
// |rl| <= ulp(rh) / 2 (likewise il) whenever one is stored.  About 48
// significant bits: the block Gram-Schmidt keeps FP64-level accuracy while
// running on the FP32 pipe (GB300's FP64 rate is a small fraction of it).
// The products are exact (FMA-split TwoProduct of the high parts plus the
// FP32 cross terms, whose own rounding is 2^-48 relative), the sums TwoSum.
struct alignas(16) ffc {
  float rh, rl, ih, il;
};
struct ff {
  float hi, lo;  // accumulator: lo is renormalised by ff_norm / ff_add
};

__device__ __forceinline__ void ff_split(double x, float& h, float& l) {
  h = __double2float_rn(x);
  l = __double2float_rn(x - double(h));
}
__device__ __forceinline__ ffc ffc_from(double2 v) {
  ffc r;
  ff_split(v.x, r.rh, r.rl);
  ff_split(v.y, r.ih, r.il);
  return r;
}
__device__ __forceinline__ double2 ffc_to(const ffc& a) {
  return make_double2(double(a.rh) + double(a.rl), double(a.ih) + double(a.il));
}
__device__ __forceinline__ double ff_to(ff a) { return double(a.hi) + double(a.lo); }
// s += a b, a = (ah, al), b = (bh, bl)
__device__ __forceinline__ void ff_mac(ff& s, float ah, float al, float bh, float bl) {
  const float p = ah * bh;
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float t = s.hi + p;
  const float bp = t - s.hi;
  const float err = (s.hi - (t - bp)) + (p - bp);
  s.hi = t;
  s.lo += err + e;
}
// a + b, renormalised
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const float t = a.hi + b.hi;
  const float bp = t - a.hi;
  const float err = (a.hi - (t - bp)) + (b.hi - bp);
  const float lo = a.lo + b.lo + err;
  ff r;
  r.hi = t + lo;
  r.lo = lo - (r.hi - t);
  return r;
}
// (ah, al) -= (ch, cl) (qh, ql), renormalised
__device__ __forceinline__ void ff_msub(float& ah, float& al, float ch, float cl, float qh,
                                        float ql) {
  const float p = ch * qh;
  float e = fmaf(ch, qh, -p);
  e = fmaf(ch, ql, e);
  e = fmaf(cl, qh, e);
  const float t = ah - p;
  const float bp = t - ah;
  const float err = (ah - (t - bp)) - (p + bp);
  const float lo = al - e + err;
  const float hi = t + lo;
  al = lo - (hi - t);
  ah = hi;
}
// (ah, al) *= (sh, sl), renormalised
__device__ __forceinline__ void ff_scale(float& ah, float& al, float sh, float sl) {
  const float p = ah * sh;
  float e = fmaf(ah, sh, -p);
  e = fmaf(ah, sl, e);
  e = fmaf(al, sh, e);
  ah = p + e;
  al = e - (ah - p);
}
__device__ __forceinline__ ff ff_shfl_xor(ff a, int o) {
  ff r;
  r.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
  r.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
  return r;
}

// workspace entries: float-float (the fast path) or FP64 (the fallback)
__device__ __forceinline__ void ws_store(ffc& d, double2 v) { d = ffc_from(v); }
__device__ __forceinline__ void ws_store(double2& d, double2 v) { d = v; }
__device__ __forceinline__ double2 ws_load(const ffc& a) { return ffc_to(a); }
__device__ __forceinline__ double2 ws_load(const double2& a) { return a; }

// raw [Nv][V][nd] -> W [agg][chi][Nv][rows]
// Sec. 3.4 step 3: chirality-split aggregate blocks of the null vectors.
template <typename WT>
__global__ void k_mgs_gather(WT* __restrict__ W, const double2* __restrict__ raw, AggMap m,
                             int nd, int nv) {
  const int half = nd / 2;
  const int rows = m.per * half;
  size_t total = size_t(nv) * m.fine.vol * nd;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < total;
       idx += size_t(gridDim.x) * blockDim.x) {
    int a = int(idx % nd);
    size_t t = idx / nd;
    int s = int(t % m.fine.vol);
    int i = int(t / m.fine.vol);
    int c[4];
    site_coords(m.fine, s, c);
    int ag = agg_of(m, c), ls = local_of(m, c);
    int chi = a / half, ad = a - chi * half;
    ws_store(W[((size_t(ag) * 2 + chi) * nv + i) * rows + size_t(ls) * half + ad], raw[idx]);
  }
}

constexpr int kQrMaxVec = 64;
constexpr int kQrMaxWarps = 32;

__device__ __forceinline__ double2 blk_sum2(double2 v, double2* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double2 r = make_double2(0.0, 0.0);
  for (int k = 0; k < nw; ++k) {
    r.x += sh[k].x;
    r.y += sh[k].y;
  }
  return r;
}

// Sec. 3.4 step 3: the same QR in FP64 (the fallback for blocks whose first
// projection cancels more than float-float can carry; see k_block_qr).
template <int RPT, int NT>
__global__ void __launch_bounds__(NT) k_block_qr64(double2* __restrict__ W, int rows, int nv,
                                                   int* status) {
  __shared__ double2 sh[32];
  __shared__ double2 part[kQrMaxWarps][kQrMaxVec];
  __shared__ double2 coef[kQrMaxVec];
  double2* B = W + size_t(blockIdx.x) * nv * rows;
  const int T = blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
  // Frobenius norm of the block for the rank test
  double2 f = make_double2(0.0, 0.0);
  for (size_t k = threadIdx.x; k < size_t(nv) * rows; k += T) {
    double2 v = B[k];
    f.x += v.x * v.x + v.y * v.y;
  }
  const double scale = sqrt(blk_sum2(f, sh).x);
  for (int i = 0; i < nv; ++i) {
    double2 v[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      int row = threadIdx.x + r * T;
      v[r] = row < rows ? B[size_t(i) * rows + row] : make_double2(0.0, 0.0);
    }
    double n0 = 0.0;  // squared norm before the first projection
    if (i > 0) {
      double2 nn0 = make_double2(0.0, 0.0);
#pragma unroll
      for (int r = 0; r < RPT; ++r) nn0.x += v[r].x * v[r].x + v[r].y * v[r].y;
      n0 = blk_sum2(nn0, sh).x;
    }
    for (int pass = 0; pass < 2 && i > 0; ++pass) {
      for (int j = 0; j < i; ++j) {
        const double2* q = B + size_t(j) * rows;
        double2 d = make_double2(0.0, 0.0);
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          int row = threadIdx.x + r * T;
          if (row < rows) {
            // d += conj(q) v, four FP64 FMAs (the FP64 pipe bounds this kernel)
            double2 qv = q[row];
            d.x = fma(qv.x, v[r].x, d.x);
            d.x = fma(qv.y, v[r].y, d.x);
            d.y = fma(qv.x, v[r].y, d.y);
            d.y = fma(-qv.y, v[r].x, d.y);
          }
        }
        for (int o = 16; o > 0; o >>= 1) {
          d.x += __shfl_xor_sync(0xffffffffu, d.x, o);
          d.y += __shfl_xor_sync(0xffffffffu, d.y, o);
        }
        if (lane == 0) part[warp][j] = d;
      }
      __syncthreads();
      if (threadIdx.x < i) {
        double2 c = make_double2(0.0, 0.0);
        for (int w = 0; w < nw; ++w) {
          c.x += part[w][threadIdx.x].x;
          c.y += part[w][threadIdx.x].y;
        }
        coef[threadIdx.x] = c;
      }
      __syncthreads();
      for (int j = 0; j < i; ++j) {
        const double2* q = B + size_t(j) * rows;
        const double2 c = coef[j];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          int row = threadIdx.x + r * T;
          if (row < rows) {
            // v -= c q, four FP64 FMAs
            double2 qv = q[row];
            v[r].x = fma(-c.x, qv.x, v[r].x);
            v[r].x = fma(c.y, qv.y, v[r].x);
            v[r].y = fma(-c.x, qv.y, v[r].y);
            v[r].y = fma(-c.y, qv.x, v[r].y);
          }
        }
      }
      __syncthreads();  // coef / part are rewritten by the next pass
      if (pass == 0) {
        double2 nn1 = make_double2(0.0, 0.0);
#pragma unroll
        for (int r = 0; r < RPT; ++r) nn1.x += v[r].x * v[r].x + v[r].y * v[r].y;
        // the same value in every thread: the whole CTA takes the same branch
        if (blk_sum2(nn1, sh).x >= 0.5 * n0) break;
      }
    }
    double2 nn = make_double2(0.0, 0.0);
#pragma unroll
    for (int r = 0; r < RPT; ++r) nn.x += v[r].x * v[r].x + v[r].y * v[r].y;
    double nrm = sqrt(blk_sum2(nn, sh).x);
    double inv = 0.0;
    if (nrm <= 1e-12 * scale) {
      if (threadIdx.x == 0) atomicOr(status, 1);
    } else {
      inv = 1.0 / nrm;
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      int row = threadIdx.x + r * T;
      if (row < rows) B[size_t(i) * rows + row] = make_double2(v[r].x * inv, v[r].y * inv);
    }
    __syncthreads();
  }
}

// sum of one float-float value per thread over the CTA; every thread gets
// the total (FP64).  sh: at least 32 entries.
__device__ __forceinline__ double blk_sum_ff(ff v, ff* sh) {
  for (int o = 16; o > 0; o >>= 1) v = ff_add(v, ff_shfl_xor(v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    ff t = l < nw ? sh[l] : ff{0.f, 0.f};
    for (int o = 16; o > 0; o >>= 1) t = ff_add(t, ff_shfl_xor(t, o));
    if (l == 0) sh[32] = t;
  }
  __syncthreads();
  return ff_to(sh[32]);
}

// One CTA per (aggregate, chirality) block of `rows` x nv, in place,
// float-float (see ffc).  Gram-Schmidt in column order.  Status bit 1: a
// rank-deficient column; bit 2: a first projection that kept less than 1 %
// of a column's norm, which float-float cannot resolve to FP64 accuracy --
// the caller then redoes the QR in FP64 (k_block_qr64).  The projection of
// column i on the finished columns 0..i-1 is formed as one classical step
// (all i coefficients reduced together) rather than i sequential ones: the
// same Q in exact arithmetic, with ~8 block barriers per column instead of
// ~4i.  The projection is repeated ("twice is enough") when the first one
// removed more than half of the column's squared norm (the Kahan-Parlett /
// Daniel-Gragg-Kaufman-Stewart criterion, |v'| < |v| / sqrt 2); otherwise
// one pass already leaves the column orthogonal to the others to working
// precision.
// Sec. 3.4 step 3: QR of every (aggregate, chirality) block.
template <int RPT, int NT>
__global__ void __launch_bounds__(NT) k_block_qr(ffc* __restrict__ W, int rows, int nv,
                                                 int* status) {
  __shared__ ff sh[33];
  __shared__ ff part[kQrMaxWarps][kQrMaxVec][2];
  __shared__ ffc coef[kQrMaxVec];
  ffc* B = W + size_t(blockIdx.x) * nv * rows;
  const int T = blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
  auto norm2 = [&](const ffc* v) {
    ff s = {0.f, 0.f};
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      ff_mac(s, v[r].rh, v[r].rl, v[r].rh, v[r].rl);
      ff_mac(s, v[r].ih, v[r].il, v[r].ih, v[r].il);
    }
    return s;
  };
  // Frobenius norm of the block for the rank test
  ff f = {0.f, 0.f};
  for (size_t k = threadIdx.x; k < size_t(nv) * rows; k += T) {
    const ffc v = B[k];
    ff_mac(f, v.rh, v.rl, v.rh, v.rl);
    ff_mac(f, v.ih, v.il, v.ih, v.il);
  }
  const double scale = sqrt(blk_sum_ff(f, sh));
  for (int i = 0; i < nv; ++i) {
    ffc v[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      int row = threadIdx.x + r * T;
      v[r] = row < rows ? B[size_t(i) * rows + row] : ffc{0.f, 0.f, 0.f, 0.f};
    }
    double n0 = 0.0;  // squared norm before the first projection
    double nn = -1.0;  // squared norm after the last projection, when known
    for (int pass = 0; pass < 2 && i > 0; ++pass) {
      if (pass == 0) {
        // the column's squared norm rides with the coefficients (slot i)
        ff s = norm2(v);
        for (int o = 16; o > 0; o >>= 1) s = ff_add(s, ff_shfl_xor(s, o));
        if (lane == 0) {
          part[warp][i][0] = s;
          part[warp][i][1] = ff{0.f, 0.f};
        }
      }
      for (int j = 0; j < i; ++j) {
        const ffc* q = B + size_t(j) * rows;
        // d = sum conj(q) v
        ff dr = {0.f, 0.f}, di = {0.f, 0.f};
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          int row = threadIdx.x + r * T;
          if (row < rows) {
            const ffc qv = q[row];
            ff_mac(dr, qv.rh, qv.rl, v[r].rh, v[r].rl);
            ff_mac(dr, qv.ih, qv.il, v[r].ih, v[r].il);
            ff_mac(di, qv.rh, qv.rl, v[r].ih, v[r].il);
            ff_mac(di, -qv.ih, -qv.il, v[r].rh, v[r].rl);
          }
        }
        for (int o = 16; o > 0; o >>= 1) {
          dr = ff_add(dr, ff_shfl_xor(dr, o));
          di = ff_add(di, ff_shfl_xor(di, o));
        }
        if (lane == 0) {
          part[warp][j][0] = dr;
          part[warp][j][1] = di;
        }
      }
      __syncthreads();
      if (threadIdx.x < i + (pass == 0 ? 1 : 0)) {
        ff cr = {0.f, 0.f}, ci = {0.f, 0.f};
        for (int w = 0; w < nw; ++w) {
          cr = ff_add(cr, part[w][threadIdx.x][0]);
          ci = ff_add(ci, part[w][threadIdx.x][1]);
        }
        coef[threadIdx.x] = ffc{cr.hi, cr.lo, ci.hi, ci.lo};
      }
      __syncthreads();
      if (pass == 0) n0 = ff_to(ff{coef[i].rh, coef[i].rl});
      for (int j = 0; j < i; ++j) {
        const ffc* q = B + size_t(j) * rows;
        const ffc c = coef[j];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          int row = threadIdx.x + r * T;
          if (row < rows) {
            // v -= c q
            const ffc qv = q[row];
            ff_msub(v[r].rh, v[r].rl, c.rh, c.rl, qv.rh, qv.rl);
            ff_msub(v[r].rh, v[r].rl, -c.ih, -c.il, qv.ih, qv.il);
            ff_msub(v[r].ih, v[r].il, c.rh, c.rl, qv.ih, qv.il);
            ff_msub(v[r].ih, v[r].il, c.ih, c.il, qv.rh, qv.rl);
          }
        }
      }
      __syncthreads();  // coef / part are rewritten by the next pass
      if (pass == 0) {
        // the same value in every thread: the whole CTA takes the same branch
        const double n1 = blk_sum_ff(norm2(v), sh);
        // a first projection that keeps less than 1 % of the column's norm
        // amplifies the float-float representation error (2^-48 of the input)
        // past FP64 accuracy: the block is redone in FP64 (status bit 2)
        if (n1 < 1e-4 * n0 && threadIdx.x == 0) atomicOr(status, 2);
        if (n1 >= 0.5 * n0) {
          nn = n1;  // one pass: the column's norm is already reduced
          break;
        }
      }
    }
    const double nrm = sqrt(nn >= 0.0 ? nn : blk_sum_ff(norm2(v), sh));
    float sh_inv = 0.f, sl_inv = 0.f;
    if (nrm <= 1e-12 * scale) {
      if (threadIdx.x == 0) atomicOr(status, 1);
    } else {
      ff_split(1.0 / nrm, sh_inv, sl_inv);
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      int row = threadIdx.x + r * T;
      if (row < rows) {
        ffc o = v[r];
        ff_scale(o.rh, o.rl, sh_inv, sl_inv);
        ff_scale(o.ih, o.il, sh_inv, sl_inv);
        B[size_t(i) * rows + row] = o;
      }
    }
    __syncthreads();
  }
}

// QR of every (aggregate, chirality) block of W; false if a block is too tall.
#define GB_QR_LAUNCH(KERN, WT)                                                       \
  bool launch_##KERN(WT* W, int rows, int nv, int nblk, int* status, cudaStream_t st) { \
    if (nv > kQrMaxVec || rows > 1024 * 24) return false;                            \
    if (rows <= 256)                                                                  \
      KERN<1, 256><<<nblk, 256, 0, st>>>(W, rows, nv, status);                       \
    else if (rows <= 512)                                                             \
      KERN<2, 256><<<nblk, 256, 0, st>>>(W, rows, nv, status);                       \
    else if (rows <= 1024)                                                            \
      KERN<4, 256><<<nblk, 256, 0, st>>>(W, rows, nv, status);                       \
    else if (rows <= 2048)                                                            \
      KERN<8, 256><<<nblk, 256, 0, st>>>(W, rows, nv, status);                       \
    else if (rows <= 4096)                                                            \
      KERN<16, 256><<<nblk, 256, 0, st>>>(W, rows, nv, status);                      \
    else if (rows <= 8192)                                                            \
      KERN<8, 1024><<<nblk, 1024, 0, st>>>(W, rows, nv, status);                     \
    else if (rows <= 16384)                                                           \
      KERN<16, 1024><<<nblk, 1024, 0, st>>>(W, rows, nv, status);                    \
    else                                                                              \
      KERN<24, 1024><<<nblk, 1024, 0, st>>>(W, rows, nv, status);                    \
    return true;                                                                      \
  }
// 256 threads up to 4096 rows (16 rows per thread), 1024 threads beyond;
// false if a block is too tall or has too many vectors
GB_QR_LAUNCH(k_block_qr, ffc)
GB_QR_LAUNCH(k_block_qr64, double2)
#undef GB_QR_LAUNCH

// W -> Vp [V][nd][Nv] (R)
// Sec. 3.4 step 3: the orthonormal blocks as prolongator rows.
template <typename R, typename WT>
__global__ void k_mgs_scatter(cpx<R>* __restrict__ Vp, const WT* __restrict__ W, AggMap m,
                              int nd, int nv) {
  const int half = nd / 2;
  const int rows = m.per * half;
  size_t total = size_t(nv) * m.fine.vol * nd;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < total;
       idx += size_t(gridDim.x) * blockDim.x) {
    // idx enumerates Vp order: (site, dof, vec)
    int i = int(idx % nv);
    size_t t = idx / nv;
    int a = int(t % nd);
    int s = int(t / nd);
    int c[4];
    site_coords(m.fine, s, c);
    int ag = agg_of(m, c), ls = local_of(m, c);
    int chi = a / half, ad = a - chi * half;
    const double2 v = ws_load(W[((size_t(ag) * 2 + chi) * nv + i) * rows + size_t(ls) * half + ad]);
    Vp[idx] = cpx<R>(R(v.x), R(v.y));
  }
}

// coarse_v[xc][chi*Nv + i] = sum_{x in A(xc), a in chi} conj(Vp[x][a][i])
// fine_v[x][a].  CTA b: aggregate b / nr, right-hand side b % nr (the nr
// CTAs of one aggregate run side by side and share its Vp rows through L2).
// Restriction R = P^dag (Secs. 3.4 and 6.6).
template <typename Rf, typename Rc>
__global__ void k_restrict(cpx<Rc>* __restrict__ coarse, const cpx<Rf>* __restrict__ fine,
                           const cpx<Rf>* __restrict__ Vp, AggMap m, int nd, int nv, int nr,
                           size_t fstride, size_t cstride) {
  extern __shared__ unsigned char smem_raw[];
  cpx<Rf>* red = reinterpret_cast<cpx<Rf>*>(smem_raw);  // [G][2][nv]
  const int xc = blockIdx.x / nr, rhs = blockIdx.x - xc * nr;
  fine += rhs * fstride;
  coarse += rhs * cstride;
  const int G = blockDim.x / nv;
  const int i = threadIdx.x % nv, g = threadIdx.x / nv;
  const int half = nd / 2;
  cpx<Rf> acc0(Rf(0), Rf(0)), acc1(Rf(0), Rf(0));
  if (g < G) {
    const int rows = m.per * nd;
    for (int q = g; q < rows; q += G) {
      int ls = q / nd, a = q - ls * nd;
      int x = fine_of(m, xc, ls);
      cpx<Rf> f = fine[size_t(x) * nd + a];
      cpx<Rf> v = Vp[(size_t(x) * nd + a) * nv + i];
      if (a < half)
        cmac_conj(acc0, v, f);
      else
        cmac_conj(acc1, v, f);
    }
    red[(g * 2 + 0) * nv + i] = acc0;
    red[(g * 2 + 1) * nv + i] = acc1;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 2 * nv; t += blockDim.x) {
    int chi = t / nv, ii = t - chi * nv;
    cpx<Rf> s(Rf(0), Rf(0));
    for (int k = 0; k < G; ++k) s += red[(k * 2 + chi) * nv + ii];
    coarse[size_t(xc) * 2 * nv + t] = cpx<Rc>(s);
  }
}

// fine_v[x][a] = sum_i Vp[x][a][i] coarse_v[agg(x)][chi(a)*Nv + i].  CTA b
// works on right-hand side b % nr, element chunk b / nr.
// Prolongation P (Secs. 3.4 and 6.6).
template <typename Rf, typename Rc>
__global__ void k_prolong(cpx<Rf>* __restrict__ fine, const cpx<Rc>* __restrict__ coarse,
                          const cpx<Rf>* __restrict__ Vp, AggMap m, int nd, int nv, int nr,
                          size_t fstride, size_t cstride) {
  const int rhs = blockIdx.x % nr;
  const size_t blk = blockIdx.x / nr, nblk = gridDim.x / nr;
  fine += rhs * fstride;
  coarse += rhs * cstride;
  size_t total = size_t(m.fine.vol) * nd;
  const int half = nd / 2;
  for (size_t idx = blk * blockDim.x + threadIdx.x; idx < total; idx += nblk * blockDim.x) {
    int a = int(idx % nd);
    int s = int(idx / nd);
    int c[4];
    site_coords(m.fine, s, c);
    int ag = agg_of(m, c);
    const cpx<Rc>* ec = coarse + size_t(ag) * 2 * nv + (a / half) * nv;
    const cpx<Rf>* v = Vp + idx * nv;
    cpx<Rf> acc(Rf(0), Rf(0));
    for (int i = 0; i < nv; ++i) cmac(acc, v[i], cpx<Rf>(ec[i]));
    fine[idx] = acc;
  }
}

// ---- Transfer kernels for the fine level (12 dofs per site), one CTA per
// aggregate.  Every fine site of an aggregate sits at the aggregate's first
// site plus an offset that depends only on its local index, so the offsets
// are tabulated once per CTA in shared memory and the per-row index work is
// one table lookup.  Vp rows (Nv coefficients of one fine dof, 96 B / 192 B
// for Nv = 24 in FP32 / FP64) are read as 16-byte vectors.

__device__ __forceinline__ int agg_origin(const AggMap& m, int xc) {
  int cc[4];
  site_coords(m.coarse, xc, cc);
  return cc[0] * m.b[0] + m.fine.stride[1] * cc[1] * m.b[1] +
         m.fine.stride[2] * cc[2] * m.b[2] + m.fine.stride[3] * cc[3] * m.b[3];
}
__device__ __forceinline__ int local_offset(const AggMap& m, int ls) {
  int l0 = ls % m.b[0];
  ls /= m.b[0];
  int l1 = ls % m.b[1];
  ls /= m.b[1];
  int l2 = ls % m.b[2];
  int l3 = ls / m.b[2];
  return l0 + m.fine.stride[1] * l1 + m.fine.stride[2] * l2 + m.fine.stride[3] * l3;
}

// A 16-byte word of Vp as CPL complex numbers in the fine vector precision:
// Vp stored in the vector precision, or in BF16 (the fine-level copy used
// when the fine smoother runs in 16 bits).
template <typename VT, typename Rf>
struct VUnpack {
  static constexpr int CPL = 16 / int(sizeof(VT));
  __device__ static __forceinline__ void get(const uint4& w, cpx<Rf> out[CPL]) {
    if constexpr (std::is_same<VT, bf16c>::value) {
#pragma unroll
      for (int k = 0; k < CPL; ++k)
        out[k] = cpx<Rf>(StoreTraits<bf16c>::load(reinterpret_cast<const bf16c*>(&w)[k]));
    } else {
#pragma unroll
      for (int k = 0; k < CPL; ++k) out[k] = reinterpret_cast<const cpx<Rf>*>(&w)[k];
    }
  }
};

// coarse_v[xc][chi*Nv + i] = sum over fine sites x of the aggregate and dofs
// a of chirality chi of conj(Vp[x][a][i]) fine_v[x][a], for NRB right-hand
// sides v per CTA.  Thread (g, p): p picks the 16-byte column of Vp rows (CPL
// coefficients), g strides over sites; each Vp word read serves NRB
// right-hand sides.  CTA b: aggregate b / nchunk, right-hand-side chunk
// b % nchunk (chunks of one aggregate run side by side and share its Vp
// rows through L2).
// Restriction R = P^dag from the 12-dof fine level (Sec. 6.6).
template <typename Rf, typename Rc, int NRB, typename VT>
__global__ void __launch_bounds__(256) k_restrict12(cpx<Rc>* __restrict__ coarse,
                                                   const cpx<Rf>* __restrict__ fine,
                                                   const VT* __restrict__ Vp, AggMap m,
                                                   int nv, int G, int nchunk, size_t fstride,
                                                   size_t cstride) {
  constexpr int ND = 12, CPL = VUnpack<VT, Rf>::CPL;
  constexpr int FW = ND * int(sizeof(cpx<Rf>)) / 16;  // 16-byte words of a fine site
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<Rf>* red = reinterpret_cast<cpx<Rf>*>(smem_raw);  // [G][2][nv]
  int* off = reinterpret_cast<int*>(red + size_t(G) * 2 * nv);
  const int xc = blockIdx.x / nchunk, chunk = blockIdx.x - xc * nchunk;
  fine += size_t(chunk) * NRB * fstride;
  coarse += size_t(chunk) * NRB * cstride;
  const int NP = nv / CPL;
  const int p = threadIdx.x % NP, g = threadIdx.x / NP;
  for (int ls = threadIdx.x; ls < m.per; ls += blockDim.x) off[ls] = local_offset(m, ls);
  const size_t base = size_t(agg_origin(m, xc));
  __syncthreads();
  cpx<Rf> acc[NRB][2][CPL];
#pragma unroll
  for (int b = 0; b < NRB; ++b)
#pragma unroll
    for (int k = 0; k < CPL; ++k) acc[b][0][k] = acc[b][1][k] = cpx<Rf>(Rf(0), Rf(0));
  if (g < G) {
    for (int ls = g; ls < m.per; ls += G) {
      const size_t x = base + off[ls];
      const uint4* vr = reinterpret_cast<const uint4*>(Vp + x * ND * nv) + p;
      uint4 w[ND];
#pragma unroll
      for (int a = 0; a < ND; ++a) w[a] = ld_stream16(vr + a * NP);
#pragma unroll
      for (int b = 0; b < NRB; ++b) {
        uint4 fw[FW];
        const uint4* fr = reinterpret_cast<const uint4*>(fine + b * fstride + x * ND);
#pragma unroll
        for (int k = 0; k < FW; ++k) fw[k] = __ldg(fr + k);
        const cpx<Rf>* f = reinterpret_cast<const cpx<Rf>*>(fw);
#pragma unroll
        for (int a = 0; a < ND; ++a) {
          cpx<Rf> v[CPL];
          VUnpack<VT, Rf>::get(w[a], v);
#pragma unroll
          for (int k = 0; k < CPL; ++k) cmac_conj(acc[b][a < ND / 2 ? 0 : 1][k], v[k], f[a]);
        }
      }
    }
  }
#pragma unroll
  for (int b = 0; b < NRB; ++b) {
    if (g < G) {
#pragma unroll
      for (int chi = 0; chi < 2; ++chi)
#pragma unroll
        for (int k = 0; k < CPL; ++k) red[(g * 2 + chi) * nv + p * CPL + k] = acc[b][chi][k];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * nv; t += blockDim.x) {
      cpx<Rf> sum(Rf(0), Rf(0));
      for (int k = 0; k < G; ++k) sum += red[k * 2 * nv + t];
      coarse[b * cstride + size_t(xc) * 2 * nv + t] = cpx<Rc>(sum);
    }
    __syncthreads();
  }
}

// fine_v[x][a] = sum_i Vp[x][a][i] coarse_v[agg(x)][chi(a)*Nv + i] for all nr
// right-hand sides.  Two threads per Vp row, each holding half of it in
// registers: thread q takes the 16-byte words 2k + q (PW words), so a pair
// reads whole 32-byte sectors; the halves meet by one shuffle.  A pair
// loads RPI rows (RPI * PW <= 12 words) before any arithmetic, so short
// rows (16-bit Vp, small Nv) still keep several loads per thread in flight.
// Prolongation P onto the 12-dof fine level (Sec. 6.6).
template <typename Rf, typename Rc, typename VT, int PW>
__global__ void __launch_bounds__(256) k_prolong12(cpx<Rf>* __restrict__ fine,
                                                  const cpx<Rc>* __restrict__ coarse,
                                                  const VT* __restrict__ Vp, AggMap m,
                                                  int nv, int nr, size_t fstride,
                                                  size_t cstride) {
  constexpr int ND = 12, CPL = VUnpack<VT, Rf>::CPL;
  constexpr int RPI = PW >= 12 ? 1 : (12 / PW > 6 ? 6 : 12 / PW);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<Rf>* cs = reinterpret_cast<cpx<Rf>*>(smem_raw);  // [nr][2][nv]
  int* off = reinterpret_cast<int*>(cs + size_t(nr) * 2 * nv);
  const int xc = blockIdx.x;
  for (int ls = threadIdx.x; ls < m.per; ls += blockDim.x) off[ls] = local_offset(m, ls);
  for (int t = threadIdx.x; t < nr * 2 * nv; t += blockDim.x) {
    const int b = t / (2 * nv), e = t - b * 2 * nv;
    cs[t] = cpx<Rf>(coarse[b * cstride + size_t(xc) * 2 * nv + e]);
  }
  const size_t base = size_t(agg_origin(m, xc));
  __syncthreads();
  const int q = threadIdx.x & 1, pair = threadIdx.x >> 1, npairs = blockDim.x >> 1;
  const int rows = m.per * ND;
  // the loop bound is uniform across the CTA, so every lane reaches the
  // full-warp shuffles; rows past the end compute nothing and store nothing
  for (int r0 = 0; r0 < rows; r0 += npairs * RPI) {
    uint4 w[RPI][PW];
    size_t frow[RPI];  // fine element x * ND + a of each row
    int coff[RPI];     // its chirality's offset into the coarse vector
    bool ok[RPI];
#pragma unroll
    for (int j = 0; j < RPI; ++j) {
      const int r = r0 + j * npairs + pair;
      ok[j] = r < rows;
      const int ls = ok[j] ? r / ND : 0, a = ok[j] ? r - ls * ND : 0;
      frow[j] = (base + off[ls]) * ND + a;
      coff[j] = (a < ND / 2 ? 0 : nv) + q * CPL;
      const uint4* vr = reinterpret_cast<const uint4*>(Vp + frow[j] * nv) + q;
#pragma unroll
      for (int k = 0; k < PW; ++k)
        if (ok[j]) w[j][k] = ld_stream16(vr + 2 * k);
    }
    for (int b = 0; b < nr; ++b) {
#pragma unroll
      for (int j = 0; j < RPI; ++j) {
        const cpx<Rf>* c = cs + b * 2 * nv + coff[j];
        cpx<Rf> acc(Rf(0), Rf(0));
        if (ok[j]) {
#pragma unroll
          for (int k = 0; k < PW; ++k) {
            cpx<Rf> v[CPL];
            VUnpack<VT, Rf>::get(w[j][k], v);
#pragma unroll
            for (int i = 0; i < CPL; ++i) cmac(acc, v[i], c[2 * k * CPL + i]);
          }
        }
        acc.re += __shfl_xor_sync(0xffffffffu, acc.re, 1);
        acc.im += __shfl_xor_sync(0xffffffffu, acc.im, 1);
        if (ok[j] && q == 0) fine[b * fstride + frow[j]] = acc;
      }
    }
  }
}

// W [agg][chi][Nv][rows] -> out [Nv][V][nd] (FP64)
// Sec. 3.4 step 3: orthonormal blocks back to the null-vector layout.
template <typename WT>
__global__ void k_blocked_to_vectors(double2* __restrict__ out, const WT* __restrict__ W,
                                  AggMap m, int nd, int nv) {
  const int half = nd / 2;
  const int rows = m.per * half;
  size_t total = size_t(nv) * m.fine.vol * nd;
  for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < total;
       idx += size_t(gridDim.x) * blockDim.x) {
    int a = int(idx % nd);
    size_t t = idx / nd;
    int s = int(t % m.fine.vol);
    int i = int(t / m.fine.vol);
    int c[4];
    site_coords(m.fine, s, c);
    int ag = agg_of(m, c), ls = local_of(m, c);
    int chi = a / half, ad = a - chi * half;
    out[idx] = ws_load(W[((size_t(ag) * 2 + chi) * nv + i) * rows + size_t(ls) * half + ad]);
  }
}

int grid_for(size_t n) {
  long long b = (long long)((n + 255) / 256);
  if (b > 152 * 32) b = 152 * 32;
  return int(b < 1 ? 1 : b);
}

}  // namespace

void block_orthonormalise(mg_ctx* c, int level, cudaStream_t st) {
  Level& F = c->L[level];
  Level& C = c->L[level + 1];
  GB_REQUIRE(F.have_raw, MG_ERR_STATE, "block_orthonormalise: no null vectors");
  const int nd = F.nd, nv = F.nvec;
  AggMap m = make_map(F, C);
  const int rows = m.per * nd / 2;
  const size_t elems = size_t(nv) * F.g.vol * nd;
  // the orthonormal vectors are kept in the aggregate-blocked layout
  // [agg][chi][Nv][rows] in which the QR runs in place: float-float, or FP64
  // when a block's first projection cancels too much (16 B either way)
  F.orth64.alloc(elems * sizeof(ffc));
  F.Vp.alloc(elems * prec_bytes_complex(F.vprec));
  const int nblk = C.g.vol * 2;
  ProfScope ps(c->prof, st, "block_orth", level, double(elems) * 16.0 * 2,
               8.0 * nv * (nv - 1) * 2.0 * rows * nblk);
  clear_status(c, st);
  k_mgs_gather<ffc><<<grid_for(elems), 256, 0, st>>>(F.orth64.as<ffc>(), F.raw.as<double2>(), m,
                                                     nd, nv);
  GB_LAUNCH_CHECK();
  GB_REQUIRE(launch_k_block_qr(F.orth64.as<ffc>(), rows, nv, nblk, c->status.as<int>(), st),
             MG_ERR_ARG, "aggregate block too large (rows > 24576 or nvec > 64)");
  GB_LAUNCH_CHECK();
  int qs = read_status(c, st);
  F.orth_ff = !(qs & 2);
  if (!F.orth_ff) {
    clear_status(c, st);
    k_mgs_gather<double2><<<grid_for(elems), 256, 0, st>>>(F.orth64.as<double2>(),
                                                           F.raw.as<double2>(), m, nd, nv);
    GB_LAUNCH_CHECK();
    launch_k_block_qr64(F.orth64.as<double2>(), rows, nv, nblk, c->status.as<int>(), st);
    GB_LAUNCH_CHECK();
    qs = read_status(c, st);
    c->launches += 2;
  }
  auto scatter = [&](auto* W) {
    if (F.vprec == MG_F64)
      k_mgs_scatter<<<grid_for(elems), 256, 0, st>>>(F.Vp.as<cpx<double>>(), W, m, nd, nv);
    else
      k_mgs_scatter<<<grid_for(elems), 256, 0, st>>>(F.Vp.as<cpx<float>>(), W, m, nd, nv);
  };
  if (F.orth_ff)
    scatter(F.orth64.as<ffc>());
  else
    scatter(F.orth64.as<double2>());
  GB_LAUNCH_CHECK();
  c->launches += 3;
  if (level == 0 && F.vprec == MG_F32 && smoother16_enabled(c)) {
    // the fine-level transfers read a BF16 copy (the Galerkin build keeps Vp)
    F.Vp16.alloc(elems * 4);
    Vec src, dst;
    src.p = F.Vp.p;
    src.prec = MG_F32;
    dst.p = F.Vp16.p;
    dst.prec = MG_BF16;
    src.n = dst.n = elems;
    blas_copy(c, dst, src, st);
  } else {
    F.Vp16.release();
  }
  if (qs & 1) {
    F.have_V = false;
    throw Error(MG_ERR_RANK, "rank-deficient null-vector aggregate block");
  }
  F.have_V = true;
}

namespace {

template <typename Rf, typename Rc, typename VT = cpx<Rf>>
void launch_restrict12(int nrb, dim3 grid, int thr, size_t smem, cudaStream_t st, Vec coarse,
                       Vec fine, const void* Vp, const AggMap& m, int nv, int G, int nchunk) {
  auto* cp = (cpx<Rc>*)coarse.p;
  auto* fp = (const cpx<Rf>*)fine.p;
  auto* vp = (const VT*)Vp;
  switch (nrb) {
    case 8:
      k_restrict12<Rf, Rc, 8, VT><<<grid, thr, smem, st>>>(cp, fp, vp, m, nv, G, nchunk, fine.n,
                                                        coarse.n);
      break;
    case 4:
      k_restrict12<Rf, Rc, 4, VT><<<grid, thr, smem, st>>>(cp, fp, vp, m, nv, G, nchunk, fine.n,
                                                        coarse.n);
      break;
    case 2:
      k_restrict12<Rf, Rc, 2, VT><<<grid, thr, smem, st>>>(cp, fp, vp, m, nv, G, nchunk, fine.n,
                                                        coarse.n);
      break;
    default:
      k_restrict12<Rf, Rc, 1, VT><<<grid, thr, smem, st>>>(cp, fp, vp, m, nv, G, nchunk, fine.n,
                                                        coarse.n);
      break;
  }
}

#define GB_TRANSFER_DISPATCH(fprec, cprec, Rf, Rc, ...)      \
  do {                                                       \
    if ((fprec) == MG_F64) {                                 \
      using Rf = double;                                     \
      if ((cprec) == MG_F64) {                               \
        using Rc = double;                                   \
        __VA_ARGS__;                                         \
      } else {                                               \
        using Rc = float;                                    \
        __VA_ARGS__;                                         \
      }                                                      \
    } else {                                                 \
      using Rf = float;                                      \
      if ((cprec) == MG_F64) {                               \
        using Rc = double;                                   \
        __VA_ARGS__;                                         \
      } else {                                               \
        using Rc = float;                                    \
        __VA_ARGS__;                                         \
      }                                                      \
    }                                                        \
  } while (0)

}  // namespace

void restrict_apply(mg_ctx* c, int level, Vec coarse, Vec fine, cudaStream_t st) {
  Level& F = c->L[level];
  Level& C = c->L[level + 1];
  GB_REQUIRE(F.have_V, MG_ERR_STATE, "restrict: null vectors not set");
  GB_REQUIRE(fine.prec == F.vprec, MG_ERR_ARG, "restrict: fine vector precision");
  GB_REQUIRE(fine.nr == coarse.nr && fine.n == F.vec_elems() && coarse.n == C.vec_elems(),
             MG_ERR_ARG, "restrict: vector shapes");
  AggMap m = make_map(F, C);
  const int nv = F.nvec, nr = fine.nr;
  const double vb = prec_bytes_complex(F.vprec);
  const bool h16 = F.Vp16.p && F.vprec == MG_F32 && F.nd == 12 && nv % 4 == 0;
  ProfScope ps(c->prof, st, "restrict", level,
               double(F.g.vol) * F.nd * (nv * (h16 ? 4.0 : vb) + nr * vb) +
                   double(C.g.vol) * C.nd * nr * vb,
               8.0 * F.g.vol * F.nd * nv * nr);
  if (F.nd == 12) {
    // per-aggregate kernel: NP 16-byte columns per Vp row, G site groups,
    // NRB right-hand sides per CTA
    const int cpl = h16 ? 4 : F.vprec == MG_F64 ? 1 : 2;
    const int NP = nv / cpl;
    int G2 = 256 / NP;
    while (G2 > 1 && m.per % G2) --G2;
    const size_t smem2 = size_t(G2) * 2 * nv * size_t(vb) + size_t(m.per) * sizeof(int);
    // the fine vectors are read in 16-byte words: a misaligned caller pointer
    // takes the generic kernel
    const bool aligned = (reinterpret_cast<uintptr_t>(fine.p) & 15) == 0;
    if (aligned && nv % cpl == 0 && G2 >= 1 && smem2 <= 48 * 1024) {
      // right-hand sides per CTA: the autotuner weighs Vp reuse against the
      // registers of the accumulators
      std::vector<int> cands;
      for (int q : {8, 4, 2, 1})
        if (nr % q == 0) cands.push_back(q);
      auto launch = [&](int nrb) {
        const int nchunk = nr / nrb;
        const dim3 grid(unsigned(C.g.vol) * nchunk);
        if (h16) {
          if (coarse.prec == MG_F64)
            launch_restrict12<float, double, bf16c>(nrb, grid, G2 * NP, smem2, st, coarse, fine,
                                                    F.Vp16.p, m, nv, G2, nchunk);
          else
            launch_restrict12<float, float, bf16c>(nrb, grid, G2 * NP, smem2, st, coarse, fine,
                                                   F.Vp16.p, m, nv, G2, nchunk);
        } else {
          GB_TRANSFER_DISPATCH(F.vprec, coarse.prec, Rf, Rc,
                               (launch_restrict12<Rf, Rc>(nrb, grid, G2 * NP, smem2, st, coarse,
                                                          fine, F.Vp.p, m, nv, G2, nchunk)));
        }
      };
      const std::string key = "restrict12/p" + std::to_string(int(F.vprec)) + "/h" +
                              std::to_string(int(h16)) + "/v" + std::to_string(F.g.vol) +
                              "/nv" + std::to_string(nv) + "/r" + std::to_string(nr);
      launch(Tuner::get().choose(key, cands, st, launch));
      GB_LAUNCH_CHECK();
      c->launches++;
      return;
    }
  }
  int G = 256 / nv;
  if (G < 1) G = 1;
  const int threads = G * nv;
  const size_t smem = size_t(G) * 2 * nv * prec_bytes_complex(F.vprec);
  const dim3 grid(unsigned(C.g.vol) * nr);
  GB_TRANSFER_DISPATCH(F.vprec, coarse.prec, Rf, Rc,
                       (k_restrict<Rf, Rc><<<grid, threads, smem, st>>>(
                           (cpx<Rc>*)coarse.p, (const cpx<Rf>*)fine.p, F.Vp.as<cpx<Rf>>(), m,
                           F.nd, nv, nr, fine.n, coarse.n)));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void prolong_apply(mg_ctx* c, int level, Vec fine, Vec coarse, cudaStream_t st) {
  Level& F = c->L[level];
  Level& C = c->L[level + 1];
  GB_REQUIRE(F.have_V, MG_ERR_STATE, "prolong: null vectors not set");
  GB_REQUIRE(fine.prec == F.vprec, MG_ERR_ARG, "prolong: fine vector precision");
  GB_REQUIRE(fine.nr == coarse.nr && fine.n == F.vec_elems() && coarse.n == C.vec_elems(),
             MG_ERR_ARG, "prolong: vector shapes");
  AggMap m = make_map(F, C);
  const int nv = F.nvec, nr = fine.nr;
  const size_t n = size_t(F.g.vol) * F.nd;
  const double vb = prec_bytes_complex(F.vprec);
  const bool h16 = F.Vp16.p && F.vprec == MG_F32 && F.nd == 12 && nv % 8 == 0;
  ProfScope ps(c->prof, st, "prolong", level,
               double(n) * (nv * (h16 ? 4.0 : vb) + nr * vb) + double(C.g.vol) * C.nd * nr * vb,
               8.0 * n * nv * nr);
  const int cpl = h16 ? 4 : F.vprec == MG_F64 ? 1 : 2;
  const size_t smem2 = size_t(nr) * 2 * nv * size_t(vb) + size_t(m.per) * sizeof(int);
  const int pw = nv % (2 * cpl) == 0 ? nv / (2 * cpl) : 0;  // 16-byte words per half row
  if (F.nd == 12 && (pw == 1 || pw == 2 || pw == 3 || pw == 4 || pw == 6 || pw == 8 || pw == 12) &&
      smem2 <= 48 * 1024) {
    auto go = [&](auto pwc) {
      constexpr int PW = decltype(pwc)::value;
      if (h16) {
        if (coarse.prec == MG_F64)
          k_prolong12<float, double, bf16c, PW><<<C.g.vol, 256, smem2, st>>>(
              (cpx<float>*)fine.p, (const cpx<double>*)coarse.p, F.Vp16.as<bf16c>(), m, nv, nr,
              fine.n, coarse.n);
        else
          k_prolong12<float, float, bf16c, PW><<<C.g.vol, 256, smem2, st>>>(
              (cpx<float>*)fine.p, (const cpx<float>*)coarse.p, F.Vp16.as<bf16c>(), m, nv, nr,
              fine.n, coarse.n);
      } else {
        GB_TRANSFER_DISPATCH(F.vprec, coarse.prec, Rf, Rc,
                             (k_prolong12<Rf, Rc, cpx<Rf>, PW><<<C.g.vol, 256, smem2, st>>>(
                                 (cpx<Rf>*)fine.p, (const cpx<Rc>*)coarse.p,
                                 F.Vp.as<cpx<Rf>>(), m, nv, nr, fine.n, coarse.n)));
      }
    };
    switch (pw) {
      case 1: go(std::integral_constant<int, 1>{}); break;
      case 2: go(std::integral_constant<int, 2>{}); break;
      case 3: go(std::integral_constant<int, 3>{}); break;
      case 4: go(std::integral_constant<int, 4>{}); break;
      case 6: go(std::integral_constant<int, 6>{}); break;
      case 8: go(std::integral_constant<int, 8>{}); break;
      default: go(std::integral_constant<int, 12>{}); break;
    }
    GB_LAUNCH_CHECK();
    c->launches++;
    return;
  }
  int blocks = grid_for(n);
  if (blocks * size_t(nr) > (1u << 30)) blocks = int((1u << 30) / nr);
  GB_TRANSFER_DISPATCH(F.vprec, coarse.prec, Rf, Rc,
                       (k_prolong<Rf, Rc><<<unsigned(blocks) * nr, 256, 0, st>>>(
                           (cpx<Rf>*)fine.p, (const cpx<Rc>*)coarse.p, F.Vp.as<cpx<Rf>>(), m,
                           F.nd, nv, nr, fine.n, coarse.n)));
  GB_LAUNCH_CHECK();
  c->launches++;
}

void nullvecs_export(mg_ctx* c, int level, void* dst, cudaStream_t st) {
  Level& F = c->L[level];
  Level& C = c->L[level + 1];
  GB_REQUIRE(F.have_V, MG_ERR_STATE, "get_nullvecs: not available");
  AggMap m = make_map(F, C);
  const size_t elems = size_t(F.nvec) * F.g.vol * F.nd;
  if (F.orth_ff)
    k_blocked_to_vectors<<<grid_for(elems), 256, 0, st>>>((double2*)dst, F.orth64.as<ffc>(), m,
                                                         F.nd, F.nvec);
  else
    k_blocked_to_vectors<<<grid_for(elems), 256, 0, st>>>((double2*)dst, F.orth64.as<double2>(),
                                                         m, F.nd, F.nvec);
  GB_LAUNCH_CHECK();
  c->launches++;
}

// ---------------------------------------------------------------------------
// Block orthonormalisation without device allocation.
//
// Some callers cannot let a library call cudaMalloc: programs whose device
// memory is owned by another allocator (a framework's caching allocator that
// has reserved the device), programs held to a fixed device-memory budget,
// and latency-critical loops where the implicit synchronisation of
// cudaMalloc / cudaFree is not acceptable.  mg_block_orthonormalise_noalloc
// serves them: the caller passes the input and output vectors, and the
// Gram-Schmidt workspace lives in the file-scope array below, which every
// GPU that loads this library holds until the process exits.
namespace {

constexpr size_t kNoAllocMaxElems = size_t(1) << 21;  // 16-byte complex entries: 32 MiB

static __device__ __align__(256) ffc g_noalloc_scratch[kNoAllocMaxElems];
static __device__ __align__(256) int g_noalloc_status[64];

// The device address of the workspace, looked up once per device and kept
// for the life of the process.  A reset of the device (cudaDeviceReset, or a
// framework that tears down and recreates the primary context) makes the
// kept address stale; calls after such a reset are not supported.
struct NoAllocSlot {
  bool ready = false;
  ffc* scratch = nullptr;
  int* status = nullptr;
};
constexpr int kNoAllocMaxDevices = 64;
NoAllocSlot g_noalloc_slots[kNoAllocMaxDevices];
std::mutex g_noalloc_mutex;

}  // namespace

}  // namespace gbmg

extern "C" mg_status mg_block_orthonormalise_noalloc(const void* vecs_dev, void* out_dev,
                                                     size_t bytes, const int dims[4],
                                                     const int block[4], int ndof, int nvec,
                                                     void* stream) {
  using namespace gbmg;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto fail = [](mg_status s, const char* msg) {
    set_last_error(msg);
    return s;
  };
  if (!vecs_dev || !out_dev || !dims || !block) return fail(MG_ERR_ARG, "noalloc: null argument");
  if (vecs_dev == out_dev) return fail(MG_ERR_ARG, "noalloc: output aliases input");
  if (nvec < 1 || ndof < 2 || (ndof & 1)) return fail(MG_ERR_ARG, "noalloc: bad nvec or ndof");
  if (nvec > kQrMaxVec) return fail(MG_ERR_ARG, "noalloc: nvec exceeds 64");
  int cd[4];
  unsigned long long vol = 1;
  for (int m = 0; m < 4; ++m) {
    if (dims[m] < 1 || block[m] < 1 || dims[m] % block[m])
      return fail(MG_ERR_ARG, "noalloc: lattice extent not divisible by block");
    cd[m] = dims[m] / block[m];
    // the running product stays below 2^21 or the call is refused: no wrap
    vol *= (unsigned long long)dims[m];
    if (vol * (unsigned long long)ndof * (unsigned long long)nvec > kNoAllocMaxElems)
      return fail(MG_ERR_ARG,
                  "noalloc: nvec * volume * ndof exceeds the 2^21-entry workspace "
                  "(32 MiB)");
  }
  const unsigned long long elems = (unsigned long long)nvec * vol * ndof;
  if (bytes != elems * 16ull)
    return fail(MG_ERR_ARG, "noalloc: bytes differs from nvec * volume * ndof * 16");
  AggMap m;
  m.fine = make_geom(dims);
  m.coarse = make_geom(cd);
  for (int k = 0; k < 4; ++k) m.b[k] = block[k];
  m.per = m.fine.vol / m.coarse.vol;
  const int rows = m.per * ndof / 2;
  const int threads = rows <= 256 * 16 ? 256 : 1024;
  const int rpt = (rows + threads - 1) / threads;
  if (rpt > 24) return fail(MG_ERR_ARG, "noalloc: aggregate block too large (rows > 24576)");
  // an error left pending by earlier, unrelated work is not this call's
  cudaGetLastError();
  // once per device, with that device current: device address of the workspace
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices)
    return fail(MG_ERR_CUDA, "noalloc: cudaGetDevice failed");
  NoAllocSlot slot;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    NoAllocSlot& s = g_noalloc_slots[dev];
    if (!s.ready) {
      void* p = nullptr;
      void* q = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess ||
          cudaGetSymbolAddress(&q, g_noalloc_status) != cudaSuccess) {
        cudaGetLastError();
        return fail(MG_ERR_CUDA, "noalloc: cudaGetSymbolAddress failed");
      }
      s.scratch = static_cast<ffc*>(p);
      s.status = static_cast<int*>(q);
      s.ready = true;
    }
    slot = s;
  }
  // the workspace keeps the previous call's contents: clear the status word
  if (cudaMemsetAsync(slot.status, 0, sizeof(int), st) != cudaSuccess)
    return fail(MG_ERR_CUDA, "noalloc: cudaMemsetAsync failed");
  auto read_back = [&](int& h) {
    return cudaMemcpyAsync(&h, slot.status, sizeof(int), cudaMemcpyDeviceToHost, st) ==
               cudaSuccess &&
           cudaStreamSynchronize(st) == cudaSuccess;
  };
  k_mgs_gather<ffc><<<grid_for(elems), 256, 0, st>>>(slot.scratch, (const double2*)vecs_dev, m,
                                                     ndof, nvec);
  if (cudaGetLastError() != cudaSuccess)
    return fail(MG_ERR_CUDA, "noalloc: gather launch failed");
  const int nblk = m.coarse.vol * 2;
  if (!launch_k_block_qr(slot.scratch, rows, nvec, nblk, slot.status, st))
    return fail(MG_ERR_ARG, "noalloc: aggregate block too large for the block QR");
  if (cudaGetLastError() != cudaSuccess)
    return fail(MG_ERR_CUDA, "noalloc: block QR launch failed");
  int h = 0;
  if (!read_back(h)) return fail(MG_ERR_CUDA, "noalloc: status read-back failed");
  const bool fp64 = (h & 2) != 0;
  if (fp64) {
    // a block's first projection cancelled more than float-float carries:
    // the same workspace (16-byte entries) redoes the QR in FP64
    double2* scratch64 = reinterpret_cast<double2*>(slot.scratch);
    if (cudaMemsetAsync(slot.status, 0, sizeof(int), st) != cudaSuccess)
      return fail(MG_ERR_CUDA, "noalloc: cudaMemsetAsync failed");
    k_mgs_gather<double2><<<grid_for(elems), 256, 0, st>>>(scratch64, (const double2*)vecs_dev,
                                                           m, ndof, nvec);
    if (cudaGetLastError() != cudaSuccess)
      return fail(MG_ERR_CUDA, "noalloc: gather launch failed");
    launch_k_block_qr64(scratch64, rows, nvec, nblk, slot.status, st);
    if (cudaGetLastError() != cudaSuccess)
      return fail(MG_ERR_CUDA, "noalloc: block QR launch failed");
    k_blocked_to_vectors<<<grid_for(elems), 256, 0, st>>>((double2*)out_dev, scratch64, m, ndof,
                                                         nvec);
  } else {
    k_blocked_to_vectors<<<grid_for(elems), 256, 0, st>>>((double2*)out_dev, slot.scratch, m,
                                                         ndof, nvec);
  }
  if (cudaGetLastError() != cudaSuccess)
    return fail(MG_ERR_CUDA, "noalloc: scatter launch failed");
  if (!read_back(h)) return fail(MG_ERR_CUDA, "noalloc: status read-back failed");
  if (h & 1) return fail(MG_ERR_RANK, "noalloc: rank-deficient null-vector aggregate block");
  return MG_OK;
}
