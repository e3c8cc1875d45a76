// Fine-level MR smoother in 16-bit storage (Sec. 7.1: the finest level's MR
// smoother runs in half precision): the smoother's vectors and a copy of the
// Wilson-clover operator (two-row or full links, clover) are stored as BF16
// complex numbers (FP32 exponent range, so the shrinking residuals of late
// outer iterations need no rescaling); all arithmetic runs in FP32.  The
// outer FP64 GCR and the rest of the K-cycle are unchanged.
#include "kernels.cuh"
#include "tune.cuh"
#include "wilson_ops.cuh"

namespace gbmg {

namespace {

__device__ __forceinline__ cpx<float> ld16(bf16c v) { return StoreTraits<bf16c>::load(v); }
__device__ __forceinline__ bf16c st16(cpx<float> v) { return StoreTraits<bf16c>::pack(v); }

// two-row (LC = 6) or full (LC = 9) FP32 links -> BF16; FP32 clover -> BF16
// Eq. (2) links in BF16 for the 16-bit fine smoother (Sec. 7.1).
template <int LC>
__global__ void k_links_to16(bf16c* __restrict__ out, const cpx<float>* __restrict__ in,
                             size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n * LC;
       i += size_t(gridDim.x) * blockDim.x)
    out[i] = st16(in[i]);
}
// Eq. (2) clover in BF16 for the 16-bit fine smoother (Sec. 7.1).
__global__ void k_clover_to16(__nv_bfloat16* __restrict__ out, const float* __restrict__ in,
                              size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    out[i] = __float2bfloat16_rn(in[i]);
}

// out = M in on 16-bit vectors; one thread per site, CTAs vector-fastest
// (as the FP32 kernel).  LC = 6: two-row links, third row rebuilt with the
// boundary sign of the link.  MINB: minimum resident CTAs per SM promised
// to the compiler (0: none), which sets its register budget and with it how
// far ahead of the arithmetic it can issue the neighbour loads.
// Eq. (2) on BF16 vectors: the fine smoother of Sec. 7.1.
template <int LC, int MINB>
__global__ void __launch_bounds__(128, MINB) k_wilson16(bf16c* __restrict__ out,
                                                  const bf16c* __restrict__ in,
                                                  const bf16c* __restrict__ U,
                                                  const __nv_bfloat16* __restrict__ A, Geom g,
                                                  float diag, size_t vstride, int nvec,
                                                  int antiperiodic) {
  const int vec = blockIdx.x % nvec;
  const int s = (blockIdx.x / nvec) * blockDim.x + threadIdx.x;
  if (s >= g.vol) return;
  in += vec * vstride;
  out += vec * vstride;
  int c[4];
  site_coords(g, s, c);
  cpx<float> psi[12], acc[12], u[9];
  auto load_spinor = [&](int site) {
    const uint4* q = reinterpret_cast<const uint4*>(in + size_t(site) * 12);
    uint4 w[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) w[i] = __ldg(q + i);
#pragma unroll
    for (int i = 0; i < 12; ++i) psi[i] = ld16(reinterpret_cast<const bf16c*>(w)[i]);
  };
  const bool tlast = antiperiodic && c[3] == g.L[3] - 1, tfirst = antiperiodic && c[3] == 0;
  auto load_link = [&](size_t idx, bool neg) {
    const unsigned* q = reinterpret_cast<const unsigned*>(U + idx * LC);
#pragma unroll
    for (int e = 0; e < LC; ++e) {
      const unsigned wv = __ldg(q + e);
      u[e] = ld16(*reinterpret_cast<const bf16c*>(&wv));
    }
    if constexpr (LC == 6) {
      const float sg = neg ? -1.f : 1.f;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int b = (r + 1) % 3, cc = (r + 2) % 3;
        u[6 + r] = sg * conj(u[b] * u[3 + cc] - u[cc] * u[3 + b]);
      }
    }
  };
  load_spinor(s);
#pragma unroll
  for (int i = 0; i < 12; ++i) acc[i] = cpx<float>(0.f, 0.f);
  {
    const uint4* q = reinterpret_cast<const uint4*>(A + size_t(s) * 72);
    uint4 w[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) w[i] = __ldg(q + i);
    const __nv_bfloat16* a = reinterpret_cast<const __nv_bfloat16*>(w);
    // (diag + A) psi per chirality block, entries converted on use
#pragma unroll
    for (int chi = 0; chi < 2; ++chi) {
      const __nv_bfloat16* ab = a + chi * 36;
      const cpx<float>* x = psi + chi * 6;
      cpx<float>* y = acc + chi * 6;
#pragma unroll
      for (int i = 0; i < 6; ++i) y[i] += (diag + __bfloat162float(ab[i])) * x[i];
#pragma unroll
      for (int i = 1; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < i; ++j) {
          const int k = i * (i - 1) / 2 + j;
          const cpx<float> l(__bfloat162float(ab[6 + 2 * k]), __bfloat162float(ab[7 + 2 * k]));
          cmac(y[i], l, x[j]);
          cmac_conj(y[j], l, x[i]);
        }
    }
  }
  const size_t V = g.vol;
#define GB_HOP16(MU)                                     \
  {                                                      \
    const int sf = neighbour(g, s, c, 1 + 2 * MU);       \
    load_spinor(sf);                                     \
    load_link(MU * V + s, MU == 3 && tlast);             \
    hop_accum<MU, true>(u, psi, acc);                    \
    const int sb = neighbour(g, s, c, 2 + 2 * MU);       \
    load_spinor(sb);                                     \
    load_link(MU * V + sb, MU == 3 && tfirst);           \
    hop_accum<MU, false>(u, psi, acc);                   \
  }
  GB_HOP16(0) GB_HOP16(1) GB_HOP16(2) GB_HOP16(3)
#undef GB_HOP16
  bf16c o[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) o[i] = st16(acc[i]);
  uint4* dst = reinterpret_cast<uint4*>(out + size_t(s) * 12);
#pragma unroll
  for (int i = 0; i < 3; ++i) dst[i] = reinterpret_cast<const uint4*>(o)[i];
}

}  // namespace

bool smoother16_enabled(const mg_ctx* c) {
  return c->p.prec_smoother == MG_BF16 && c->L[0].prec == MG_F32;
}

void smoother16_prepare(mg_ctx* c, cudaStream_t st) {
  Level& L = c->L[0];
  if (!smoother16_enabled(c)) return;
  const size_t nl = size_t(4) * L.g.vol;
  int blocks = ceil_div(nl * 9, 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (L.gauge12_ok) {
    L.gauge16.alloc(nl * 6 * sizeof(bf16c));
    k_links_to16<6><<<blocks, 256, 0, st>>>(L.gauge16.as<bf16c>(), L.gauge12.as<cpx<float>>(),
                                            nl);
  } else {
    L.gauge16.alloc(nl * 9 * sizeof(bf16c));
    k_links_to16<9><<<blocks, 256, 0, st>>>(L.gauge16.as<bf16c>(), L.gauge32.as<cpx<float>>(),
                                            nl);
  }
  GB_LAUNCH_CHECK();
  const size_t nc = size_t(L.g.vol) * 72;
  L.clover16.alloc(nc * sizeof(__nv_bfloat16));
  k_clover_to16<<<blocks, 256, 0, st>>>(L.clover16.as<__nv_bfloat16>(), L.clover32.as<float>(),
                                        nc);
  GB_LAUNCH_CHECK();
  c->launches += 2;
}

void wilson16_apply(mg_ctx* c, Vec out, Vec in, cudaStream_t st) {
  Level& L = c->L[0];
  GB_REQUIRE(out.prec == MG_BF16 && in.prec == MG_BF16, MG_ERR_ARG,
             "16-bit smoother: BF16 vectors expected");
  GB_REQUIRE(L.gauge16.p && L.clover16.p, MG_ERR_STATE, "16-bit smoother operator not built");
  const int nvec = in.nr;
  const dim3 grid(ceil_div(L.g.vol, 128) * nvec);
  const size_t vs = size_t(L.g.vol) * 12;
  // algorithmic bytes per site: 16-bit spinor in + out per vector, links and
  // clover once
  const double bytes = double(L.g.vol) * (96.0 * nvec + (L.gauge12_ok ? 4 * 24.0 : 4 * 36.0) +
                                          144.0);
  ProfScope ps(c->prof, st, "wilson_clover16", 0, bytes, double(nvec) * L.g.vol * 1824.0);
  auto* o = (bf16c*)out.p;
  auto* i = (const bf16c*)in.p;
  const bf16c* U = L.gauge16.as<bf16c>();
  const __nv_bfloat16* A = L.clover16.as<__nv_bfloat16>();
  const float dg = float(L.diag);
  const int ap = c->p.t_antiperiodic;
  // autotuned register budget: minimum CTAs per SM 0 (none), 3, 4 or 6
  auto launch = [&](int q) {
    if (L.gauge12_ok) {
      switch (q) {
        case 3: k_wilson16<6, 3><<<grid, 128, 0, st>>>(o, i, U, A, L.g, dg, vs, nvec, ap); break;
        case 4: k_wilson16<6, 4><<<grid, 128, 0, st>>>(o, i, U, A, L.g, dg, vs, nvec, ap); break;
        case 6: k_wilson16<6, 6><<<grid, 128, 0, st>>>(o, i, U, A, L.g, dg, vs, nvec, ap); break;
        default: k_wilson16<6, 0><<<grid, 128, 0, st>>>(o, i, U, A, L.g, dg, vs, nvec, ap); break;
      }
    } else {
      switch (q) {
        case 3: k_wilson16<9, 3><<<grid, 128, 0, st>>>(o, i, U, A, L.g, dg, vs, nvec, ap); break;
        case 4: k_wilson16<9, 4><<<grid, 128, 0, st>>>(o, i, U, A, L.g, dg, vs, nvec, ap); break;
        case 6: k_wilson16<9, 6><<<grid, 128, 0, st>>>(o, i, U, A, L.g, dg, vs, nvec, ap); break;
        default: k_wilson16<9, 0><<<grid, 128, 0, st>>>(o, i, U, A, L.g, dg, vs, nvec, ap); break;
      }
    }
  };
  const std::string key = "wilson16/v" + std::to_string(L.g.vol) + "/n" + std::to_string(nvec) +
                          "/c" + std::to_string(int(L.gauge12_ok));
  launch(Tuner::get().choose(key, {0, 3, 4, 6}, st, launch));
  GB_LAUNCH_CHECK();
  c->launches++;
}

}  // namespace gbmg
