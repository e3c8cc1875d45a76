// Domain-decomposed coarse apply with a one-site halo (Sec. 6.5).
//
// The coarse lattice of one level is cut into P0 x P1 x P2 x P3 equal
// sub-domains ("ranks", lexicographic with x fastest).  Each rank holds the
// links of its own sites and its own spinor; a hop that leaves the
// sub-domain reads the neighbour's spinor from a halo buffer of the rank.
// Per apply:
//   1. pack   -- ONE kernel per rank copies the spinor on every face it
//                shares with another rank (all dimensions at once) into the
//                rank's send buffer;
//   2. exchange -- each face segment is copied into the receiving rank's own
//                halo buffer (peer-to-peer into the receiver's memory on a
//                multi-GPU machine; device-to-device copies when every rank
//                lives on this GPU, as here);
//   3. apply  -- the stencil of Eq. (3) on the rank's sites, hops across the
//                sub-domain boundary served from the halo buffer.
// Only the spinor is exchanged, n complex numbers per face site, against
// 9 n^2 link elements of work per site (the paper's O(n) vs O(n^2) point).
//
// Face f = 2 mu + s of a rank (only for mu with P_mu > 1):
//   send face 2mu   = sites at local x_mu = 0        -> rank r - mu, recv 2mu
//   send face 2mu+1 = sites at local x_mu = l_mu - 1 -> rank r + mu, recv 2mu+1
//   recv face 2mu   = the +mu neighbours of the sites at x_mu = l_mu - 1
//   recv face 2mu+1 = the -mu neighbours of the sites at x_mu = 0
// Face sites are ordered lexicographically over the other three local
// coordinates (lowest direction fastest), the same order on both sides.
#include <string>
#include <vector>

#include "coarse_ops.cuh"
#include "kernels.cuh"

namespace gbmg {

struct HaloGeom {
  Geom local;           // sub-domain extents
  int P[4];             // ranks per direction
  int face_off[8];      // first face site of face f in the send / recv buffer
  int face_sites[8];    // sites of face f (0 when P_mu == 1)
  int halo_sites;       // sum of face_sites
};

// index of the face site of local coordinates c on a face of direction mu
__host__ __device__ __forceinline__ int face_index(const Geom& l, const int c[4], int mu) {
  int q = 0, stride = 1;
  for (int k = 0; k < 4; ++k) {
    if (k == mu) continue;
    q += c[k] * stride;
    stride *= l.L[k];
  }
  return q;
}

// local site of face index q on face side (0: x_mu = 0, 1: x_mu = l_mu - 1)
__host__ __device__ __forceinline__ int face_site(const Geom& l, int mu, int side, int q) {
  int c[4];
  for (int k = 0; k < 4; ++k) {
    if (k == mu) continue;
    c[k] = q % l.L[k];
    q /= l.L[k];
  }
  c[mu] = side ? l.L[mu] - 1 : 0;
  return c[0] + l.stride[1] * c[1] + l.stride[2] * c[2] + l.stride[3] * c[3];
}

HaloGeom make_halo_geom(const int gdims[4], const int P[4]) {
  HaloGeom h;
  int ld[4];
  for (int m = 0; m < 4; ++m) {
    ld[m] = gdims[m] / P[m];
    h.P[m] = P[m];
  }
  h.local = make_geom(ld);
  int off = 0;
  for (int f = 0; f < 8; ++f) {
    const int mu = f >> 1;
    h.face_off[f] = off;
    h.face_sites[f] = P[mu] > 1 ? h.local.vol / ld[mu] : 0;
    off += h.face_sites[f];
  }
  h.halo_sites = off;
  return h;
}

void rank_coords(const int P[4], int r, int rc[4]) {
  for (int m = 0; m < 4; ++m) {
    rc[m] = r % P[m];
    r /= P[m];
  }
}

int rank_of(const int P[4], const int rc[4]) {
  int r = 0, s = 1;
  for (int m = 0; m < 4; ++m) {
    r += ((rc[m] % P[m] + P[m]) % P[m]) * s;
    s *= P[m];
  }
  return r;
}

namespace {

// every face of one rank's spinor into its send buffer: one launch, all
// dimensions (thread per (face site, dof) element)
template <typename R>
__global__ void k_halo_pack(cpx<R>* __restrict__ send, const cpx<R>* __restrict__ x, HaloGeom h,
                            int n) {
  const size_t total = size_t(h.halo_sites) * n;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total;
       i += size_t(gridDim.x) * blockDim.x) {
    const int hs = int(i / n), dof = int(i - size_t(hs) * n);
    int f = 0;
#pragma unroll
    for (int k = 1; k < 8; ++k)
      if (h.face_sites[k] > 0 && hs >= h.face_off[k]) f = k;
    const int s = face_site(h.local, f >> 1, f & 1, hs - h.face_off[f]);
    send[i] = x[size_t(s) * n + dof];
  }
}

// local site <-> global site (vector scatter / gather and link import)
__device__ __forceinline__ int global_site(const Geom& gl, const Geom& l, const int rc[4],
                                           int s) {
  int c[4];
  site_coords(l, s, c);
  return (rc[0] * l.L[0] + c[0]) + gl.stride[1] * (rc[1] * l.L[1] + c[1]) +
         gl.stride[2] * (rc[2] * l.L[2] + c[2]) + gl.stride[3] * (rc[3] * l.L[3] + c[3]);
}

struct RankPos {
  int rc[4];
};

// words per site copied between a global per-site array and a rank's local one
__global__ void k_halo_sites_copy(uint32_t* __restrict__ dst, const uint32_t* __restrict__ src,
                                  Geom gl, Geom l, RankPos rp, size_t words, int to_global) {
  const size_t total = size_t(l.vol) * words;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total;
       i += size_t(gridDim.x) * blockDim.x) {
    const int s = int(i / words);
    const size_t w = i - size_t(s) * words;
    const size_t g = size_t(global_site(gl, l, rp.rc, s)) * words + w;
    if (to_global)
      dst[g] = src[i];
    else
      dst[i] = src[g];
  }
}

// Eq. (3) on the sites of one rank.  The gather of the nine partner spinors
// takes a hop that leaves the sub-domain from the halo buffer; the link
// stream is the one of the single-domain kernel (one CTA per site, threads
// over 16-byte row chunks, CG column groups).
template <typename S, int N, int CG>
__global__ void __launch_bounds__(CG*(N / Unpack<S>::RPC))
    k_coarse_halo(cpx<typename StoreTraits<S>::real>* __restrict__ y,
                  const cpx<typename StoreTraits<S>::real>* __restrict__ x,
                  const cpx<typename StoreTraits<S>::real>* __restrict__ recv,
                  const S* __restrict__ links, const float* __restrict__ scales, HaloGeom h) {
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
  __shared__ const cpx<R>* src[9];
  const int site = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid < 9) {
    int c[4];
    site_coords(h.local, site, c);
    const cpx<R>* p;
    if (tid == 0) {
      p = x + size_t(site) * N;
    } else {
      const int mu = (tid - 1) >> 1;
      const bool fwd = ((tid - 1) & 1) == 0;
      const bool leaves = h.P[mu] > 1 && (fwd ? c[mu] == h.local.L[mu] - 1 : c[mu] == 0);
      if (leaves) {
        const int f = 2 * mu + (fwd ? 0 : 1);
        p = recv + size_t(h.face_off[f] + face_index(h.local, c, mu)) * N;
      } else {
        p = x + size_t(neighbour(h.local, site, c, tid)) * N;
      }
    }
    src[tid] = p;
  }
  __syncthreads();
  for (int i = tid; i < K; i += NT) {
    const int d = i / N;
    xs[i] = src[d][i - d * N];
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
      const cpx<R> xv = xs[cg + (it + u) * CG];
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

template <typename S, int N>
void launch_halo(void* y, const void* x, const void* recv, const void* links,
                 const float* scales, const HaloGeom& h, cudaStream_t st) {
  using R = typename StoreTraits<S>::real;
  constexpr int RPC = Unpack<S>::RPC;
  constexpr int CG = RPC == 1 ? 4 : (RPC == 2 ? 8 : 16);
  constexpr int NT = CG * (N / RPC);
  k_coarse_halo<S, N, CG><<<h.local.vol, NT, 0, st>>>((cpx<R>*)y, (const cpx<R>*)x,
                                                       (const cpx<R>*)recv, (const S*)links,
                                                       scales, h);
}

template <typename S>
bool dispatch_halo(int n, void* y, const void* x, const void* recv, const void* links,
                   const float* scales, const HaloGeom& h, cudaStream_t st) {
  switch (n) {
    case 16: launch_halo<S, 16>(y, x, recv, links, scales, h, st); return true;
    case 32: launch_halo<S, 32>(y, x, recv, links, scales, h, st); return true;
    case 48: launch_halo<S, 48>(y, x, recv, links, scales, h, st); return true;
    case 64: launch_halo<S, 64>(y, x, recv, links, scales, h, st); return true;
    default: return false;
  }
}

int grid_of(size_t n) {
  long long b = (long long)((n + 255) / 256);
  if (b > 152 * 32) b = 152 * 32;
  return int(b < 1 ? 1 : b);
}

}  // namespace

}  // namespace gbmg

struct mg_halo {
  mg_ctx* ctx = nullptr;
  int level = 0;
  int n = 0;
  mg_prec prec = MG_F64;   // link store
  mg_prec vprec = MG_F64;  // spinor precision
  gbmg::Geom global{};
  gbmg::HaloGeom h{};
  int nranks = 0;
  std::vector<std::unique_ptr<gbmg::DevBuf>> links, scales, send, recv;
  long long launches = 0;
};

using namespace gbmg;

namespace {

thread_local std::string g_halo_error;

template <typename F>
mg_status halo_guard(F&& f) {
  try {
    f();
    return MG_OK;
  } catch (const Error& e) {
    g_halo_error = e.what();
    set_last_error(e.what());
    return e.code;
  }
}

void check_plan_args(const int dims[4], const int procs[4]) {
  GB_REQUIRE(dims && procs, MG_ERR_ARG, "halo: null dims or procs");
  long long nr = 1;
  for (int m = 0; m < 4; ++m) {
    GB_REQUIRE(dims[m] >= 1 && procs[m] >= 1 && dims[m] % procs[m] == 0, MG_ERR_ARG,
               "halo: every extent must be a positive multiple of its rank count");
    nr *= procs[m];
    GB_REQUIRE(nr <= 4096, MG_ERR_ARG, "halo: at most 4096 sub-domains");
  }
}

size_t store_bytes(mg_prec p) { return p == MG_F64 ? 16 : p == MG_F32 ? 8 : 4; }

}  // namespace

extern "C" {

mg_status mg_halo_plan(const int dims[4], const int procs[4], int rank, int send_to[8],
                       int recv_from[8], int face_offset[8], int face_sites[8]) {
  return halo_guard([&] {
    check_plan_args(dims, procs);
    GB_REQUIRE(send_to && recv_from && face_offset && face_sites, MG_ERR_ARG,
               "halo: null output array");
    const int nr = procs[0] * procs[1] * procs[2] * procs[3];
    GB_REQUIRE(rank >= 0 && rank < nr, MG_ERR_ARG, "halo: rank out of range");
    const HaloGeom h = make_halo_geom(dims, procs);
    int rc[4];
    rank_coords(procs, rank, rc);
    for (int f = 0; f < 8; ++f) {
      const int mu = f >> 1;
      face_offset[f] = h.face_off[f];
      face_sites[f] = h.face_sites[f];
      if (h.face_sites[f] == 0) {
        send_to[f] = recv_from[f] = -1;
        continue;
      }
      int lo[4] = {rc[0], rc[1], rc[2], rc[3]}, hi[4] = {rc[0], rc[1], rc[2], rc[3]};
      lo[mu] -= 1;
      hi[mu] += 1;
      // send face 2mu (x_mu = 0) goes down, 2mu+1 (x_mu = l - 1) goes up; the
      // recv face of the same index comes from the opposite neighbour
      send_to[f] = (f & 1) ? rank_of(procs, hi) : rank_of(procs, lo);
      recv_from[f] = (f & 1) ? rank_of(procs, lo) : rank_of(procs, hi);
    }
  });
}

mg_status mg_halo_face_sites(const int local_dims[4], int mu, int side, int* sites) {
  return halo_guard([&] {
    GB_REQUIRE(local_dims && sites, MG_ERR_ARG, "halo: null argument");
    GB_REQUIRE(mu >= 0 && mu < 4 && (side == 0 || side == 1), MG_ERR_ARG,
               "halo: bad direction or side");
    for (int m = 0; m < 4; ++m)
      GB_REQUIRE(local_dims[m] >= 1, MG_ERR_ARG, "halo: bad local extent");
    const Geom l = make_geom(local_dims);
    const int nf = l.vol / l.L[mu];
    for (int q = 0; q < nf; ++q) sites[q] = face_site(l, mu, side, q);
  });
}

mg_status mg_halo_create(mg_ctx* ctx, int level, const int procs[4], mg_halo** out,
                         void* stream) {
  if (out) *out = nullptr;
  mg_halo* hp = new mg_halo();
  mg_status s = halo_guard([&] {
    GB_REQUIRE(ctx && out, MG_ERR_ARG, "halo: null context or output");
    GB_REQUIRE(level >= 1 && level < ctx->nlevels, MG_ERR_ARG, "halo: level must be coarse");
    const Level& L = ctx->L[level];
    GB_REQUIRE(L.have_op, MG_ERR_STATE, "halo: coarse operator not built");
    GB_REQUIRE(L.nd == 16 || L.nd == 32 || L.nd == 48 || L.nd == 64, MG_ERR_ARG,
               "halo: n must be 16, 32, 48 or 64");
    check_plan_args(L.g.L, procs);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    hp->ctx = ctx;
    hp->level = level;
    hp->n = L.nd;
    hp->prec = L.prec;
    hp->vprec = L.vprec;
    hp->global = L.g;
    hp->h = make_halo_geom(L.g.L, procs);
    hp->nranks = procs[0] * procs[1] * procs[2] * procs[3];
    const size_t lvol = size_t(hp->h.local.vol);
    const size_t es = store_bytes(L.prec);
    const size_t link_words = size_t(9) * L.nd * L.nd * es / 4;
    const void* gl_links = prec_is16(L.prec) ? L.links16.p : L.links.p;
    GB_REQUIRE(gl_links, MG_ERR_STATE, "halo: level has no link store");
    for (int r = 0; r < hp->nranks; ++r) {
      RankPos rp;
      rank_coords(procs, r, rp.rc);
      auto lk = std::make_unique<DevBuf>();
      lk->alloc(lvol * link_words * 4);
      k_halo_sites_copy<<<grid_of(lvol * link_words), 256, 0, st>>>(
          lk->as<uint32_t>(), (const uint32_t*)gl_links, L.g, hp->h.local, rp, link_words, 0);
      GB_LAUNCH_CHECK();
      auto sc = std::make_unique<DevBuf>();
      if (prec_is16(L.prec)) {
        sc->alloc(lvol * 4);
        k_halo_sites_copy<<<grid_of(lvol), 256, 0, st>>>(
            sc->as<uint32_t>(), L.scales.as<uint32_t>(), L.g, hp->h.local, rp, 1, 0);
        GB_LAUNCH_CHECK();
        hp->launches++;
      }
      auto sb = std::make_unique<DevBuf>(), rb = std::make_unique<DevBuf>();
      const size_t hb = size_t(hp->h.halo_sites) * L.nd * prec_bytes_complex(L.vprec);
      if (hb) {
        sb->alloc(hb);
        rb->alloc(hb);
      }
      hp->links.push_back(std::move(lk));
      hp->scales.push_back(std::move(sc));
      hp->send.push_back(std::move(sb));
      hp->recv.push_back(std::move(rb));
      hp->launches++;
    }
    GB_CHECK(cudaStreamSynchronize(st));
  });
  if (s != MG_OK) {
    delete hp;
    return s;
  }
  *out = hp;
  return MG_OK;
}

mg_status mg_halo_destroy(mg_halo* h) {
  if (!h) return MG_ERR_ARG;
  cudaDeviceSynchronize();
  delete h;
  return MG_OK;
}

mg_status mg_halo_info(mg_halo* hp, int* nranks, int local_dims[4], int* halo_sites,
                       size_t* halo_bytes) {
  return halo_guard([&] {
    GB_REQUIRE(hp, MG_ERR_ARG, "halo: null handle");
    if (nranks) *nranks = hp->nranks;
    if (local_dims)
      for (int m = 0; m < 4; ++m) local_dims[m] = hp->h.local.L[m];
    if (halo_sites) *halo_sites = hp->h.halo_sites;
    if (halo_bytes) *halo_bytes = size_t(hp->h.halo_sites) * hp->n * prec_bytes_complex(hp->vprec);
  });
}

mg_status mg_halo_scatter(mg_halo* hp, int rank, void* local_dev, const void* global_dev,
                          int to_global, void* stream) {
  return halo_guard([&] {
    GB_REQUIRE(hp && local_dev && global_dev, MG_ERR_ARG, "halo: null argument");
    GB_REQUIRE(rank >= 0 && rank < hp->nranks, MG_ERR_ARG, "halo: rank out of range");
    GB_REQUIRE(local_dev != global_dev, MG_ERR_ARG, "halo: local vector aliases the global one");
    RankPos rp;
    rank_coords(hp->h.P, rank, rp.rc);
    const size_t words = size_t(hp->n) * prec_bytes_complex(hp->vprec) / 4;
    const size_t total = size_t(hp->h.local.vol) * words;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (to_global)
      k_halo_sites_copy<<<grid_of(total), 256, 0, st>>>((uint32_t*)global_dev,
                                                        (const uint32_t*)local_dev, hp->global,
                                                        hp->h.local, rp, words, 1);
    else
      k_halo_sites_copy<<<grid_of(total), 256, 0, st>>>((uint32_t*)local_dev,
                                                        (const uint32_t*)global_dev, hp->global,
                                                        hp->h.local, rp, words, 0);
    GB_LAUNCH_CHECK();
    hp->launches++;
  });
}

mg_status mg_halo_pack(mg_halo* hp, int rank, const void* local_dev, void* stream) {
  return halo_guard([&] {
    GB_REQUIRE(hp && local_dev, MG_ERR_ARG, "halo: null argument");
    GB_REQUIRE(rank >= 0 && rank < hp->nranks, MG_ERR_ARG, "halo: rank out of range");
    if (hp->h.halo_sites == 0) return;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t total = size_t(hp->h.halo_sites) * hp->n;
    if (hp->vprec == MG_F64)
      k_halo_pack<double><<<grid_of(total), 256, 0, st>>>(
          hp->send[rank]->as<cpx<double>>(), (const cpx<double>*)local_dev, hp->h, hp->n);
    else
      k_halo_pack<float><<<grid_of(total), 256, 0, st>>>(
          hp->send[rank]->as<cpx<float>>(), (const cpx<float>*)local_dev, hp->h, hp->n);
    GB_LAUNCH_CHECK();
    hp->launches++;
  });
}

mg_status mg_halo_exchange(mg_halo* hp, void* stream) {
  return halo_guard([&] {
    GB_REQUIRE(hp, MG_ERR_ARG, "halo: null handle");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t sb = size_t(hp->n) * prec_bytes_complex(hp->vprec);
    int send_to[8], recv_from[8], off[8], fs[8];
    for (int r = 0; r < hp->nranks; ++r) {
      GB_REQUIRE(mg_halo_plan(hp->global.L, hp->h.P, r, send_to, recv_from, off, fs) == MG_OK,
                 MG_ERR_ARG, "halo: plan failed");
      for (int f = 0; f < 8; ++f) {
        if (fs[f] == 0) continue;
        // rank r's send face f lands in the same face of rank send_to[f]
        char* dst = static_cast<char*>(hp->recv[send_to[f]]->p) + size_t(off[f]) * sb;
        const char* src = static_cast<const char*>(hp->send[r]->p) + size_t(off[f]) * sb;
        GB_CHECK(cudaMemcpyAsync(dst, src, size_t(fs[f]) * sb, cudaMemcpyDeviceToDevice, st));
      }
    }
  });
}

mg_status mg_halo_apply(mg_halo* hp, int rank, void* y_local, const void* x_local,
                        void* stream) {
  return halo_guard([&] {
    GB_REQUIRE(hp && y_local && x_local, MG_ERR_ARG, "halo: null argument");
    GB_REQUIRE(rank >= 0 && rank < hp->nranks, MG_ERR_ARG, "halo: rank out of range");
    GB_REQUIRE(y_local != x_local, MG_ERR_ARG, "halo: output aliases input");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const void* lk = hp->links[rank]->p;
    const void* rv = hp->recv[rank]->p;
    const float* sc = hp->scales[rank]->as<float>();
    bool ok = false;
    switch (hp->prec) {
      case MG_F64: ok = dispatch_halo<cpx<double>>(hp->n, y_local, x_local, rv, lk, sc, hp->h, st); break;
      case MG_F32: ok = dispatch_halo<cpx<float>>(hp->n, y_local, x_local, rv, lk, sc, hp->h, st); break;
      case MG_BF16: ok = dispatch_halo<bf16c>(hp->n, y_local, x_local, rv, lk, sc, hp->h, st); break;
      case MG_F16: ok = dispatch_halo<f16c>(hp->n, y_local, x_local, rv, lk, sc, hp->h, st); break;
      case MG_I16: ok = dispatch_halo<i16c>(hp->n, y_local, x_local, rv, lk, sc, hp->h, st); break;
    }
    GB_REQUIRE(ok, MG_ERR_ARG, "halo: unsupported n");
    GB_LAUNCH_CHECK();
    hp->launches++;
  });
}

mg_status mg_halo_buffers(mg_halo* hp, int rank, void** send_dev, void** recv_dev) {
  return halo_guard([&] {
    GB_REQUIRE(hp && send_dev && recv_dev, MG_ERR_ARG, "halo: null argument");
    GB_REQUIRE(rank >= 0 && rank < hp->nranks, MG_ERR_ARG, "halo: rank out of range");
    *send_dev = hp->send[rank]->p;
    *recv_dev = hp->recv[rank]->p;
  });
}

long long mg_halo_launch_count(mg_halo* hp) { return hp ? hp->launches : -1; }

}  // extern "C"
