// Multi-right-hand-side coarse apply of Eq. (3) on the 5th-generation
// tensor cores (tcgen05, FP16/BF16 operands, FP32 accumulators in TMEM).
//
// For one coarse site the apply of nrhs vectors is a complex GEMM
//   Y[m][j] = sum_{slot d} sum_k L_d[m][k] X(nbr_d)[k][j],   m, k < n, j < nrhs.
// It is run as a real GEMM D = A B^T per site with K = 2n per slot:
//   B_d[m][2k + c] = (re, im) of L_d[m][k]   (the link rows, K-major),
//   A_d[j][2k]     =  Re X[k][j],  A_d[j][2k + 1] = -Im X[k][j]   (row j  -> Re Y[.][j])
//   A_d[nrhs+j][2k] = Im X[k][j],  A_d[nrhs+j][2k+1] = Re X[k][j] (row nrhs+j -> Im Y[.][j])
// so D[j][m] = Re Y[m][j] and D[nrhs + j][m] = Im Y[m][j].  M = 128 rows
// (2 nrhs <= 128, the rest zero), N = n, accumulated over the 9 slots.
//
// Data flow per site: for each slot the CTA copies the slot's links (stored
// in HBM already in the canonical K-major core-matrix order, no swizzle) and
// builds the spinor operand in shared memory, double-buffered; one thread
// issues the 2n/16 MMAs of the slot and commits them to the buffer's
// mbarrier.  After the 9 slots the four warps read their 32 TMEM lanes,
// exchange real/imaginary rows through shared memory and store Y coalesced.
// Every mbarrier wait is bounded: on timeout the kernel records an error
// word, waits (bounded) for its MMAs, frees its TMEM and returns.
//
// Two kernels do this: k_coarse_mma (register-staged operands, two
// buffers, the whole CTA in step) and k_coarse_mma_ws (warp-specialised:
// bulk copies of the links and of the neighbour spinors into a load ring,
// separate converting, MMA and epilogue warps).  The autotuner picks the
// kernel, the stage granularity and the ring depths (or the CTAs per SM)
// per shape.
#include "async_copy.cuh"
#include "kernels.cuh"
#include "tune.cuh"

namespace gbmg {

namespace {

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 32 lanes x 16 consecutive FP32 columns
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor, K-major, no swizzle: 8-row x 16-byte
// core matrices; lbo = bytes between K-adjacent core matrices, sbo = bytes
// between M/N-adjacent ones.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= uint64_t((saddr >> 4) & 0x3FFFu);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;  // descriptor version of the sm_100 family; no swizzle
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, A and B both F16 or
// both BF16, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N, bool bf16) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
         (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// byte offset of element (row, k) in a K-major, no-swizzle operand of
// `kcols` K elements (16-bit): core matrices [row/8][k/8] of 128 bytes
__host__ __device__ __forceinline__ uint32_t core_off(int row, int k, int kcols) {
  return uint32_t(((row >> 3) * (kcols >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

template <bool BF16>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  if constexpr (BF16) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  } else {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
}

// One lattice of a batched launch; the launch walks the concatenated site
// list of all lattices (global site gs belongs to the last lattice whose
// site0 <= gs).  Passed by value, so a launch carries no host-side state and
// can be captured into a CUDA graph.
constexpr int kMaxBatch = 8;
struct MmaLattice {
  const uint4* links;
  const float* scales;
  const cpx<float>* x;
  cpx<float>* y;
  // x already in the 16-bit operand layout, [site][half][core(row, k)]
  // (pre-converted launches only; written by k_spinor_tile_mma)
  unsigned char* xc;
  Geom g;
  int site0;
};
struct MmaBatch {
  MmaLattice lat[kMaxBatch];
  int count;
  int total;
  // fault injection (host-set, for tests of the timeout path): every CTA
  // first waits on a barrier that nothing arrives at, before any MMA
  int stall;
};

// Eq. (3) on nrhs right-hand sides: a complex GEMM per coarse site.
template <bool BF16, int N>
__global__ void __launch_bounds__(128) k_coarse_mma(const MmaBatch batch, int nrhs,
                                                    int* __restrict__ err) {
  // a pipeline stage is half a stencil slot: N/2 complex link columns, i.e.
  // KS = N real K values; 18 stages per site
  constexpr int KS = N;                     // real K of one stage
  constexpr int A_BYTES = 128 * KS * 2;     // spinor operand, M = 128 rows
  constexpr int B_BYTES = N * KS * 2;       // link operand, N rows
  constexpr uint32_t LBO = 128;
  constexpr uint32_t SBO = (KS / 8) * 128;
  constexpr int NST = 18;                   // stages per site
  constexpr uint32_t IDESC = mma_idesc(128, N, BF16);
  constexpr uint32_t TMEM_COLS = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t mbar[3];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int nb_sh[9];
  __shared__ int abort_sh;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // buffers: A0 A1 B0 B1
#define ABUF(b) (smem + (b) * A_BYTES)
#define BBUF(b) (smem + 2 * A_BYTES + (b) * B_BYTES)

  if (warp == 0) {
    tmem_alloc(&tmem_base_sh, TMEM_COLS);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    mbar_init(&mbar[2], 1);  // the injected stall's barrier; never arrived at
    fence_mbar_init();
    abort_sh = 0;
  }
  // both spinor buffers start at zero: rows >= 2 nrhs stay zero throughout
  for (int i = tid; i < 2 * A_BYTES / 16; i += 128)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  // per buffer b: bit b of `parity` = mbarrier phase to wait for, bit b of
  // `pending` = MMAs committed on that buffer not yet waited for
  uint32_t parity = 0u, pending = 0u;
  bool ok = true;
  if (batch.stall) {
    if (tid == 0 && !mbar_wait(&mbar[2], 0u)) abort_sh = 1;
    __syncthreads();
    ok = !abort_sh;
  }

  // Operands of one slot are fetched into registers by fully unrolled,
  // independent loads (every load of the slot in flight at once); slot d+1
  // is fetched while slot d's barrier and MMAs run.
  MmaLattice cur = batch.lat[0];  // lattice of the site being processed
  // Spinor staging: the (N/2) x nrhs complex values of a stage are cut into
  // tiles of 4 columns k x 8 right-hand sides j; warp w stages tiles w, w+4,
  // ...  Lane l takes j = 8 jt + (l & 7), k = 4 kt + (l >> 3), so the 32
  // 4-byte stores of a warp fill one 8-row x 16-byte core matrix: 32
  // different banks.  The right-hand-side tile count is rounded up to a
  // power of two (tiles past nrhs stage nothing) so the mapping is shifts.
  constexpr int XPT = N / 4;                        // tiles per warp (nrhs <= 64)
  constexpr int BPT = (B_BYTES / 16 + 127) / 128;   // 16-byte link chunks per thread
  cpx<float> xr[XPT];
  uint4 br[BPT];
  const int nx = N * nrhs;          // spinor elements of one site
  const int nxs = (N / 2) * nrhs;   // spinor elements of one stage
  const int jsh = nrhs <= 8 ? 0 : nrhs <= 16 ? 1 : nrhs <= 32 ? 2 : 3;  // log2 of the tile count
  auto tile_jk = [&](int u, int& j, int& k) {
    const int t = warp + 4 * u;
    j = 8 * (t & ((1 << jsh) - 1)) + (lane & 7);
    k = 4 * (t >> jsh) + (lane >> 3);
    return k < N / 2 && j < nrhs;
  };
  auto fetch = [&](int site, int st) {
    const int d = st >> 1, h = st & 1;
    const cpx<float>* xs = cur.x + size_t(nb_sh[d]) * nx + size_t(h) * nxs;
    const uint4* src = cur.links + (size_t(site) * NST + st) * (B_BYTES / 16);
#pragma unroll
    for (int u = 0; u < BPT; ++u) {
      const int i = tid + 128 * u;
      if (i < B_BYTES / 16) br[u] = ld_stream16(src + i);
    }
#pragma unroll
    for (int u = 0; u < XPT; ++u) {
      int j, k;
      if (tile_jk(u, j, k)) xr[u] = xs[k * nrhs + j];
    }
  };
  auto stage = [&](int b) {
    uint4* dstB = reinterpret_cast<uint4*>(BBUF(b));
#pragma unroll
    for (int u = 0; u < BPT; ++u) {
      const int i = tid + 128 * u;
      if (i < B_BYTES / 16) dstB[i] = br[u];
    }
    unsigned char* A = ABUF(b);
#pragma unroll
    for (int u = 0; u < XPT; ++u) {
      int j, k;  // k: complex column within the stage, j: right-hand side
      if (tile_jk(u, j, k)) {
        const cpx<float> v = xr[u];
        *reinterpret_cast<uint32_t*>(A + core_off(j, 2 * k, KS)) = pack2<BF16>(v.re, -v.im);
        *reinterpret_cast<uint32_t*>(A + core_off(nrhs + j, 2 * k, KS)) = pack2<BF16>(v.im, v.re);
      }
    }
  };

  for (int gs = blockIdx.x; gs < batch.total && ok; gs += gridDim.x) {
    int li = 0;
#pragma unroll
    for (int q = 1; q < kMaxBatch; ++q)
      if (q < batch.count && batch.lat[q].site0 <= gs) li = q;
    cur = batch.lat[li];
    const int site = gs - cur.site0;
    if (tid < 9) {
      int c[4];
      site_coords(cur.g, site, c);
      nb_sh[tid] = neighbour(cur.g, site, c, tid);
    }
    __syncthreads();
    fetch(site, 0);
    for (int d = 0; d < NST; ++d) {
      const int b = d & 1;
      if (pending & (1u << b)) {  // the MMAs that read this buffer two slots ago
        if (tid == 0 && !mbar_wait(&mbar[b], (parity >> b) & 1u)) abort_sh = 1;
        __syncthreads();
        if (abort_sh) {
          ok = false;
          break;
        }
        parity ^= 1u << b;
        pending &= ~(1u << b);
      }
      stage(b);
      if (d < NST - 1) fetch(site, d + 1);
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(ABUF(b)), b0 = smem_u32(BBUF(b));
#pragma unroll
        for (int kk = 0; kk < KS / 16; ++kk)
          mma_f16(tmem, smem_desc(a0 + kk * 256, LBO, SBO), smem_desc(b0 + kk * 256, LBO, SBO),
                  IDESC, (d > 0 || kk > 0) ? 1u : 0u);
        mma_commit(&mbar[b]);
      }
      pending |= 1u << b;
    }
    if (!ok) break;
    for (int b = 0; b < 2; ++b)
      if (pending & (1u << b)) {
        if (tid == 0 && !mbar_wait(&mbar[b], (parity >> b) & 1u)) abort_sh = 1;
        __syncthreads();
        if (abort_sh) {
          ok = false;
          break;
        }
        parity ^= 1u << b;
        pending &= ~(1u << b);
      }
    if (!ok) break;
    tc_fence_after();
    // TMEM lanes 32w..32w+31 = rows of D, staged as FP32 [row][N + 1] (the
    // odd row stride keeps both the row-per-lane stores and the column reads
    // below free of bank conflicts) over the spinor buffers and, for 2 nrhs
    // = 128, the first 512 bytes of the idle link buffer: 128 (N + 1) 4 <=
    // 2 A_BYTES + B_BYTES for N = 32, 48, 64
    constexpr int CS = N + 1;
    static_assert(128 * CS * 4 <= 2 * A_BYTES + B_BYTES, "epilogue staging fits");
    float* Cs = reinterpret_cast<float*>(smem);
    const int row = 32 * warp + lane;
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + (uint32_t(32 * warp) << 16) + uint32_t(c0), v);
      if (row < 2 * nrhs) {
#pragma unroll
        for (int q = 0; q < 16; ++q) Cs[row * CS + c0 + q] = v[q];
      }
    }
    tc_fence_before();
    __syncthreads();
    const float sc = cur.scales[site];
    cpx<float>* ys = cur.y + size_t(site) * nx;
    for (int e = tid; e < nx; e += 128) {
      const int m = e / nrhs, j = e - m * nrhs;
      ys[e] = cpx<float>(sc * Cs[j * CS + m], sc * Cs[(nrhs + j) * CS + m]);
    }
    __syncthreads();
    // restore the zero rows >= 2 nrhs of both spinor buffers
    for (int b = 0; b < 2; ++b) {
      uint4* z = reinterpret_cast<uint4*>(ABUF(b) + 2 * nrhs * KS * 2);
      for (int i = tid; i < (128 - 2 * nrhs) * KS * 2 / 16; i += 128) z[i] = make_uint4(0, 0, 0, 0);
    }
  }
  if (!ok) {
    // let any MMAs still in flight finish (bounded) before TMEM is freed
    if (tid == 0) {
      for (int b = 0; b < 2; ++b)
        if (pending & (1u << b)) mbar_wait(&mbar[b], (parity >> b) & 1u);
      atomicOr(err, 1);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
#undef ABUF
#undef BBUF
}

// ---------------------------------------------------------------------------
// Warp-specialised, pipelined form of the same GEMM (persistent, one to
// three CTAs per SM, 320 threads each).  A pipeline stage is KH half slots of one stencil slot
// (KH = 2: the whole slot, K = 2n; KH = 1: half of it, K = n).  Both inputs
// of a stage are contiguous in global memory and arrive by bulk copies
// (cp.async.bulk) into an SL-deep load ring: the stage's links (the tiled
// store, L2 evict-first) and the rows of the neighbour's FP32 spinor the
// stage needs.  Four warps convert the spinor rows into the 16-bit MMA
// operand in shared memory (an SA-deep operand ring), each warp a whole
// stage (stage q: warp q mod 4), so four stages convert at once, and
//   warps 0-3  convert (x(nbr) -> the real and imaginary rows of right-
//              hand side j: rows j and nrhs + j, or 2j and 2j + 1 when IL)
//   warps 4-7  epilogue: their TMEM lane quarter -> y; IL: in registers,
//              the two rows of a right-hand side paired by a lane shuffle;
//              otherwise staged as FP32 rows in shared memory
//   warp 8     lane 0 issues the bulk copies
//   warp 9     lane 0 issues the MMAs of each stage and commits them
// Barriers: load_full (copy bytes) and load_empty (the stage's MMAs and
// its converting warp done) per load slot; a_full (the converting warp)
// and a_empty (MMAs done) per operand slot; acc_full (MMAs of the
// site done) and acc_empty (the four epilogue warps) per accumulator (two
// TMEM buffers of n columns, so the epilogue of one site overlaps the MMAs
// of the next).  The A operand keeps only its 2 nrhs used rows; the MMA's
// rows beyond them (M = 128) read whatever follows in shared memory and
// produce accumulator rows that are never read.  Every wait is bounded; on
// a timeout (or the injected stall) every role stops, the copy issuer waits
// for its copies in flight, the MMA issuer for its MMAs, and TMEM is freed.
// PC: x arrives already converted (k_spinor_tile_mma, one streaming pass
// before the launch); the copy issuer bulk-copies each stage's operand rows
// into the operand ring beside its links, the converting warps idle, and
// one barrier pair per ring slot (SA = SL) carries both.
constexpr int kWsThreads = 320;
constexpr int kWsMaxStages = 8;

__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity,
                                              volatile int* abort_flag, int* err) {
  constexpr uint64_t kBudgetNs = 1000000000ull;
  if (mbar_try_wait(bar, parity)) return true;  // the common case: no timer read
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if ((it & 255u) == 255u && global_ns() - t0 > kBudgetNs) {
      *abort_flag = 1;
      atomicOr(err, 1);
      return false;
    }
  }
}

// Shared-memory layout of the pipelined kernel: [A ring][link ring][spinor
// ring][epilogue rows (split rows only)]; the A ring comes first, so the MMA
// rows beyond 2 nrhs of its last half slot read up to 256 n bytes past it
// inside the rings that follow.
struct WsLayout {
  uint32_t xh, ab, lb, rb, a_off, l_off, r_off, c_off, total;
};
__host__ __device__ inline WsLayout ws_layout(int N, int KH, int nrhs, int SL, int SA, bool IL,
                                              bool PC) {
  WsLayout w;
  w.xh = uint32_t(4 * nrhs * N);                 // A operand bytes of a half slot
  w.ab = uint32_t(KH) * w.xh;                    // A operand bytes of a stage
  w.lb = uint32_t(KH) * uint32_t(2 * N * N);     // link bytes of a stage
  // spinor bytes of a stage (none when the operand arrives pre-converted)
  w.rb = PC ? 0u : uint32_t(KH) * uint32_t((N / 2) * nrhs * 8);
  w.a_off = 0;
  w.l_off = uint32_t(SA) * w.ab;
  w.r_off = w.l_off + uint32_t(SL) * w.lb;
  w.c_off = w.r_off + uint32_t(SL) * w.rb;
  // split rows: the epilogue stages the accumulator rows, FP32 [2 nrhs][n + 1]
  const uint32_t cs = IL ? 0u : (uint32_t(2 * nrhs * (N + 1) * 4) + 15u) / 16u * 16u;
  w.total = w.c_off + cs;
  return w;
}

template <bool BF16, int N, int KH, bool IL, bool PC>
__global__ void __launch_bounds__(kWsThreads, 3)
    k_coarse_mma_ws(const MmaBatch batch, int nrhs, int SL, int SA, int* __restrict__ err) {
  constexpr int NST = 18 / KH;                         // stages per site
  constexpr int HB = 2 * N * N;                        // link bytes of a half slot
  constexpr uint32_t LBO = 128, SBO = (N / 8) * 128;  // K extent N per half, both operands
  constexpr uint32_t IDESC = mma_idesc(128, N, BF16);
  constexpr uint32_t TMEM_COLS = 128;                  // accumulators at columns 0 and 64
  constexpr int CS = N + 1;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t load_full[kWsMaxStages], load_empty[kWsMaxStages];
  __shared__ uint64_t a_full[kWsMaxStages], a_empty[kWsMaxStages];
  __shared__ uint64_t acc_full[2], acc_empty[2], fin, stall_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_sh;
  __shared__ int epi_ok;
  // ring depths the host guarantees: 4 or 8 (multiples of the converting
  // warps, see the converter) -- any other value would break the phase rule
  if ((SL != 4 && SL != 8) || (SA != 4 && SA != 8)) {
    if (threadIdx.x == 0) atomicOr(err, 1);
    return;
  }
  // pre-converted operands travel with the links: one ring, SA == SL
  if ((SL != 4 && SL != 8) || (SA != 4 && SA != 8) || (PC && SA != SL)) {
    if (threadIdx.x == 0) atomicOr(err, 1);
    return;
  }
  const WsLayout lay = ws_layout(N, KH, nrhs, SL, SA, IL, PC);
  unsigned char* aring = smem + lay.a_off;
  unsigned char* lring = smem + lay.l_off;
  unsigned char* rring = smem + lay.r_off;
  float* Cs = reinterpret_cast<float*>(smem + lay.c_off);  // split rows only
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    tmem_alloc(&tmem_base_sh, TMEM_COLS);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int q = 0; q < SL; ++q) {
      mbar_init(&load_full[q], 1);
      mbar_init(&load_empty[q], PC ? 1 : 2);  // the MMA commit (+ the converting warp)
    }
    for (int q = 0; q < SA; ++q) {
      mbar_init(&a_full[q], 1);
      mbar_init(&a_empty[q], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(&fin, 1);
    mbar_init(&stall_bar, 1);  // the injected stall's barrier; never arrived at
    fence_mbar_init();
    abort_sh = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  if (batch.stall) {
    if (tid == 0 && !mbar_wait(&stall_bar, 0u)) {
      abort_sh = 1;
      atomicOr(err, 1);
    }
    __syncthreads();
  }
  auto lattice_of_site = [&](int gs) {
    int li = 0;
#pragma unroll
    for (int q = 1; q < kMaxBatch; ++q)
      if (q < batch.count && batch.lat[q].site0 <= gs) li = q;
    return li;
  };

  if (warp < 4 && PC) {
    // the operand arrives pre-converted: the converting warps idle
  } else if (warp < 4) {
    // ---- convert: warp w converts stages w, w + 4, ...  SL and SA are
    // multiples of 4, so every ring slot is always served by the same warp:
    // when the warp waits for a slot's phase k, it has itself waited for
    // phase k - 1 (the slot's previous use), so the parity test of
    // mbarrier.try_wait cannot match a phase two back.  Element (k, j) of a
    // half slot, k < N / 2 complex columns, j < nrhs; lane l takes
    // j = 8 jt + (l & 7), k = 4 kt + (l >> 3), so the warp's 32 four-byte
    // stores fill one 8-row x 16-byte core matrix.  The right-hand-side tile
    // count is rounded up to a power of two (tiles past nrhs convert
    // nothing) so the mapping is shifts; the tile values of a batch are all
    // read before any is written.
    const int jsh = nrhs <= 8 ? 0 : nrhs <= 16 ? 1 : nrhs <= 32 ? 2 : 3;
    const int ntiles = (N / 8) << jsh;  // tiles of a half slot
    const int jl = lane & 7, kl0 = lane >> 3;
    uint32_t q = 0;
    for (int gs = blockIdx.x; gs < batch.total && !abort_sh; gs += gridDim.x) {
      for (int d = 0; d < NST; ++d, ++q) {
        if (int(q & 3u) != warp) continue;
        const uint32_t sl = q % uint32_t(SL), lph = (q / uint32_t(SL)) & 1u;
        const uint32_t sa = q % uint32_t(SA), aph = (q / uint32_t(SA)) & 1u;
        if (!wait_or_abort(&load_full[sl], lph, &abort_sh, err)) break;
        if (!wait_or_abort(&a_empty[sa], aph ^ 1u, &abort_sh, err)) break;
        const cpx<float>* __restrict__ xr =
            reinterpret_cast<const cpx<float>*>(rring + size_t(sl) * lay.rb);
        unsigned char* __restrict__ A = aring + size_t(sa) * lay.ab;
#pragma unroll
        for (int h = 0; h < KH; ++h) {
          unsigned char* Ah = A + h * lay.xh;
          const cpx<float>* xh = xr + h * (N / 2) * nrhs;
          for (int t0 = 0; t0 < ntiles; t0 += 8) {
            cpx<float> v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int t = t0 + u;
              const int j = 8 * (t & ((1 << jsh) - 1)) + jl, k = 4 * (t >> jsh) + kl0;
              if (t < ntiles && j < nrhs) v[u] = xh[k * nrhs + j];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int t = t0 + u;
              const int j = 8 * (t & ((1 << jsh) - 1)) + jl, k = 4 * (t >> jsh) + kl0;
              if (t < ntiles && j < nrhs) {
                const int rre = IL ? 2 * j : j, rim = IL ? 2 * j + 1 : nrhs + j;
                *reinterpret_cast<uint32_t*>(Ah + core_off(rre, 2 * k, N)) =
                    pack2<BF16>(v[u].re, -v[u].im);
                *reinterpret_cast<uint32_t*>(Ah + core_off(rim, 2 * k, N)) =
                    pack2<BF16>(v[u].im, v[u].re);
              }
            }
          }
        }
        // every lane's operand writes made visible to the tensor core, then
        // one arrival: the spinor rows are read, the operand is ready
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&a_full[sa]);
          mbar_arrive(&load_empty[sl]);
        }
      }
    }
  } else if (warp < 8 && IL) {
    // ---- epilogue, interleaved rows: warp ew reads TMEM lanes 32 ew..
    // (accumulator rows); row 2j holds Re Y[.][j], row 2j + 1 Im Y[.][j], so
    // lanes l and l ^ 1 exchange their columns and each writes every other
    // m of its pair -- no staging rows, no barrier between the warps
    const int ew = warp - 4;
    const int row = 32 * ew + lane;
    const int j = row >> 1, part = row & 1;
    uint32_t it = 0;
    for (int gs = blockIdx.x; gs < batch.total; gs += gridDim.x, ++it) {
      const uint32_t b = it & 1u, ph = (it >> 1) & 1u;
      if (!wait_or_abort(&acc_full[b], ph, &abort_sh, err)) break;
      tc_fence_after();
      const MmaLattice& cur = batch.lat[lattice_of_site(gs)];
      const int site = gs - cur.site0;
      const float sc = cur.scales[site];
      cpx<float>* ys = cur.y + size_t(site) * N * nrhs;
      if (32 * ew < 2 * nrhs) {  // warp-uniform: the warp holds live rows
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 16) {
          float v[16];
          tmem_ld16(tmem + (uint32_t(32 * ew) << 16) + b * 64u + uint32_t(c0), v);
#pragma unroll
          for (int q = 0; q < 16; q += 2) {
            // part 0 writes m = c0 + q, part 1 writes m = c0 + q + 1
            const float mine = part ? v[q + 1] : v[q];
            const float give = part ? v[q] : v[q + 1];
            const float other = __shfl_xor_sync(0xffffffffu, give, 1);
            const int m = c0 + q + part;
            if (row < 2 * nrhs)
              ys[size_t(m) * nrhs + j] =
                  part ? cpx<float>(sc * other, sc * mine) : cpx<float>(sc * mine, sc * other);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
    }
  } else if (warp < 8) {
    // ---- epilogue, split rows (row j = Re Y[.][j], row nrhs + j = Im):
    // TMEM -> FP32 rows in shared memory -> y, all four warps storing
    const int e = tid - 128, ew = e >> 5;
    uint32_t it = 0;
    for (int gs = blockIdx.x; gs < batch.total; gs += gridDim.x, ++it) {
      const uint32_t b = it & 1u, ph = (it >> 1) & 1u;
      if (e == 0) epi_ok = wait_or_abort(&acc_full[b], ph, &abort_sh, err) ? 1 : 0;
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (!epi_ok) break;
      tc_fence_after();
      const MmaLattice& cur = batch.lat[lattice_of_site(gs)];
      const int site = gs - cur.site0;
      const int row = 32 * ew + lane;
      if (32 * ew < 2 * nrhs) {
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 16) {
          float v[16];
          tmem_ld16(tmem + (uint32_t(32 * ew) << 16) + b * 64u + uint32_t(c0), v);
          if (row < 2 * nrhs) {
#pragma unroll
            for (int q2 = 0; q2 < 16; ++q2) Cs[row * CS + c0 + q2] = v[q2];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
      asm volatile("bar.sync 1, 128;" ::: "memory");
      const float sc = cur.scales[site];
      cpx<float>* ys = cur.y + size_t(site) * N * nrhs;
      for (int q2 = e; q2 < N * nrhs; q2 += 128) {
        const int m = q2 / nrhs, jj = q2 - m * nrhs;
        ys[q2] = cpx<float>(sc * Cs[jj * CS + m], sc * Cs[(nrhs + jj) * CS + m]);
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
    }
  } else if (warp == 8) {
    // ---- bulk copies: the stage's links and the neighbour's spinor rows
    if (lane == 0) {
      const uint64_t pol = policy_evict_first(), pol_x = policy_evict_last();
      // a pre-converted launch may start while the pre-pass that writes its
      // operand is still running (programmatic dependent launch): wait for
      // that grid's completion and memory before the first copy (a no-op
      // when the launch has no such predecessor)
      if (PC) asm volatile("griddepcontrol.wait;" ::: "memory");
      uint32_t q = 0;
      bool go = true;
      for (int gs = blockIdx.x; gs < batch.total && go && !abort_sh; gs += gridDim.x) {
        const MmaLattice& cur = batch.lat[lattice_of_site(gs)];
        const int site = gs - cur.site0;
        int c[4];
        site_coords(cur.g, site, c);
        const unsigned char* lsrc =
            reinterpret_cast<const unsigned char*>(cur.links) + size_t(site) * 18 * HB;
        for (int d = 0; d < NST; ++d) {
          const uint32_t sl = q % uint32_t(SL), ph = (q / uint32_t(SL)) & 1u;
          if (!wait_or_abort(&load_empty[sl], ph ^ 1u, &abort_sh, err)) {
            go = false;
            break;
          }
          const int slot = (d * KH) >> 1, h0 = (d * KH) & 1;
          const int nb = neighbour(cur.g, site, c, slot);
          if (PC) {
            // the stage's operand rows, already converted: straight into
            // the operand ring (SA == SL, so slot sl)
            const unsigned char* asrc =
                cur.xc + size_t(nb) * 2 * lay.xh + size_t(h0) * lay.xh;
            mbar_arrive_expect_tx(&load_full[sl], lay.lb + lay.ab);
            bulk_g2s(lring + size_t(sl) * lay.lb, lsrc + size_t(d) * lay.lb, lay.lb,
                     &load_full[sl], pol);
            bulk_g2s(aring + size_t(sl) * lay.ab, asrc, lay.ab, &load_full[sl], pol_x);
          } else {
            const cpx<float>* xsrc =
                cur.x + size_t(nb) * N * nrhs + size_t(h0) * (N / 2) * nrhs;
            mbar_arrive_expect_tx(&load_full[sl], lay.lb + lay.rb);
            bulk_g2s(lring + size_t(sl) * lay.lb, lsrc + size_t(d) * lay.lb, lay.lb,
                     &load_full[sl], pol);
            bulk_g2s(rring + size_t(sl) * lay.rb, xsrc, lay.rb, &load_full[sl], pol_x);
          }
          ++q;
        }
      }
      // copies still in flight land before the CTA's shared memory goes away
      const uint32_t first = q > uint32_t(SL) ? q - uint32_t(SL) : 0u;
      for (uint32_t r = first; r < q; ++r)
        mbar_wait(&load_full[r % uint32_t(SL)], (r / uint32_t(SL)) & 1u);
    }
  } else {
    // ---- MMA issue
    if (lane == 0) {
      uint32_t q = 0, it = 0;
      bool issued = false, go = true;
      for (int gs = blockIdx.x; gs < batch.total && go && !abort_sh; gs += gridDim.x, ++it) {
        const uint32_t b = it & 1u, ph = (it >> 1) & 1u;
        if (!wait_or_abort(&acc_empty[b], ph ^ 1u, &abort_sh, err)) break;
        tc_fence_after();
        const uint32_t dt = tmem + b * 64u;
        for (int d = 0; d < NST; ++d, ++q) {
          const uint32_t sl = q % uint32_t(SL), lph = (q / uint32_t(SL)) & 1u;
          const uint32_t sa = q % uint32_t(SA), aph = (q / uint32_t(SA)) & 1u;
          if (!wait_or_abort(&load_full[sl], lph, &abort_sh, err) ||
              (!PC && !wait_or_abort(&a_full[sa], aph, &abort_sh, err))) {
            go = false;
            break;
          }
          tc_fence_after();
          // descriptors of the stage's first K step; a step of 256 bytes
          // adds 16 to the start-address field (addresses stay below 256 KB)
          const uint64_t da = smem_desc(smem_u32(aring + size_t(sa) * lay.ab), LBO, SBO);
          const uint64_t db = smem_desc(smem_u32(lring + size_t(sl) * lay.lb), LBO, SBO);
#pragma unroll
          for (int h = 0; h < KH; ++h)
#pragma unroll
            for (int kk = 0; kk < N / 16; ++kk)
              mma_f16(dt, da + uint64_t((h * lay.xh + kk * 256) >> 4),
                      db + uint64_t((h * HB + kk * 256) >> 4), IDESC,
                      (d > 0 || h > 0 || kk > 0) ? 1u : 0u);
          mma_commit(&load_empty[sl]);
          if (!PC) mma_commit(&a_empty[sa]);
          issued = true;
        }
        if (!go) break;
        mma_commit(&acc_full[b]);
      }
      if (issued) {  // every MMA issued has completed before TMEM is freed
        mma_commit(&fin);
        mbar_wait(&fin, 0u);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// x [site][n][nrhs] (FP32) -> the pipelined kernel's 16-bit A operand,
// [site][half h][core(row, k)]: half h holds complex columns h n/2 .. of
// x's n rows, each right-hand side j as two operand rows (re, -im) and
// (im, re) -- rows j and nrhs + j, or 2j and 2j + 1 when IL -- exactly the
// tile the converting warps would build in shared memory.  A thread takes
// one right-hand side j and four complex columns (one 16-byte row of a core
// matrix in each of its two rows): four loads coalesced over j, two 16-byte
// stores; two items in flight per thread; sites in descending order.
template <bool BF16, int N, bool IL>
__global__ void __launch_bounds__(256) k_spinor_tile_mma(const MmaBatch batch, int nrhs) {
  // the apply launched after this pass may begin its set-up now; it reads
  // the operand only after this grid has completed
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  constexpr int KT = N / 8;  // 4-column groups of a half slot
  const size_t items = size_t(batch.total) * 2 * KT * nrhs;
  const size_t xh = size_t(4) * nrhs * N;
  const size_t stride = size_t(gridDim.x) * blockDim.x;
  for (size_t e0 = size_t(blockIdx.x) * blockDim.x + threadIdx.x; e0 < items; e0 += 2 * stride) {
    cpx<float> v[2][4];
    unsigned char* dst[2];
    int jj[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (e0 + u * stride >= items) {
        dst[u] = nullptr;
        continue;
      }
      // last sites first: the first sites the apply reads are the ones
      // written last, still in L2 when it starts
      const size_t e = items - 1 - (e0 + u * stride);
      const size_t r = e / unsigned(nrhs);
      const int j = int(e - r * unsigned(nrhs));
      const size_t r2 = r / KT;
      const int kt = int(r - r2 * KT);
      const int h = int(r2 & 1), gs = int(r2 >> 1);
      int li = 0;
#pragma unroll
      for (int q = 1; q < kMaxBatch; ++q)
        if (q < batch.count && batch.lat[q].site0 <= gs) li = q;
      const MmaLattice& cur = batch.lat[li];
      const int site = gs - cur.site0;
      const cpx<float>* src = cur.x + (size_t(site) * N + h * (N / 2) + 4 * kt) * nrhs + j;
#pragma unroll
      for (int c = 0; c < 4; ++c) v[u][c] = src[c * nrhs];
      dst[u] = cur.xc + size_t(site) * 2 * xh + size_t(h) * xh + size_t(kt) * 128;
      jj[u] = j;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (!dst[u]) continue;
      const int j = jj[u];
      const int rre = IL ? 2 * j : j, rim = IL ? 2 * j + 1 : nrhs + j;
      uint4 a, b;
      a.x = pack2<BF16>(v[u][0].re, -v[u][0].im);
      a.y = pack2<BF16>(v[u][1].re, -v[u][1].im);
      a.z = pack2<BF16>(v[u][2].re, -v[u][2].im);
      a.w = pack2<BF16>(v[u][3].re, -v[u][3].im);
      b.x = pack2<BF16>(v[u][0].im, v[u][0].re);
      b.y = pack2<BF16>(v[u][1].im, v[u][1].re);
      b.z = pack2<BF16>(v[u][2].im, v[u][2].re);
      b.w = pack2<BF16>(v[u][3].im, v[u][3].re);
      // core_off(row, 8 kt, N) = ((row / 8) KT + kt) 128 + (row % 8) 16
      *reinterpret_cast<uint4*>(dst[u] + size_t(rre >> 3) * KT * 128 + (rre & 7) * 16) = a;
      *reinterpret_cast<uint4*>(dst[u] + size_t(rim >> 3) * KT * 128 + (rim & 7) * 16) = b;
    }
  }
}

// FP32 internal links [V][9][col k][row m] (unscaled) -> tiled 16-bit MMA
// operand [V][9][core(m, 2k)] scaled by the per-site scale.
// Eq. (3) links tiled as the tensor-core B operand.
template <bool BF16>
__global__ void k_links_tile_mma(uint32_t* __restrict__ out, const cpx<float>* __restrict__ in,
                                 const float* __restrict__ scales, int vol, int n) {
  const size_t total = size_t(vol) * 9 * n * n;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total;
       i += size_t(gridDim.x) * blockDim.x) {
    const size_t blk = i / (size_t(n) * n);
    const int rem = int(i - blk * n * n);
    const int k = rem / n, m = rem - k * n;  // internal [col k][row m]
    const size_t site = blk / 9;
    const int d = int(blk - site * 9);
    const int h = k / (n / 2), kl = k - h * (n / 2);  // half of the slot, column within it
    const size_t stage = site * 18 + size_t(d) * 2 + h;
    const float inv = 1.f / scales[site];
    const cpx<float> v = in[i];
    const size_t words = size_t(n) * n * 2 / 4;  // 32-bit words per (site, stage)
    out[stage * words + core_off(m, 2 * kl, n) / 4] = pack2<BF16>(v.re * inv, v.im * inv);
  }
}

// A launch shape of the pipelined kernel: stage granularity KH (half slots
// per stage), load-ring depth SL and operand-ring depth SA, as the tuner
// choice 1000 + 100 KH + 10 SL + SA; 0 if its shared memory exceeds `limit`
// or the MMA rows past the last operand stage would leave the allocation.
bool ws_fits(int N, int KH, int nrhs, int SL, int SA, bool IL, bool PC, size_t limit) {
  const WsLayout w = ws_layout(N, KH, nrhs, SL, SA, IL, PC);
  const size_t reach = size_t(SA - 1) * w.ab + size_t(KH - 1) * w.xh + size_t(256) * N;
  return w.total <= limit && reach <= w.total;
}

// Pre-converted operand buffers of a context: the newest is the largest;
// the ones it replaced stay allocated, so a CUDA graph captured with one
// stays valid for the context's lifetime.
using XcPool = std::vector<std::unique_ptr<DevBuf>>;

template <bool BF16, int N>
void launch_mma_batch(int* err, const MmaBatch& batch, int nrhs, cudaStream_t st, bool tune,
                      XcPool* pool) {
  constexpr int KS = N;
  const int smem = 2 * (128 * KS * 2) + 2 * (N * KS * 2);
  auto kern = k_coarse_mma<BF16, N>;
  GB_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  GB_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  // CTAs per SM from the kernel's own footprint: shared memory (dynamic +
  // static + 1 KB reserved per CTA) and registers; TMEM allows 8 x 64 columns
  int sms = 0, dev = 0, smem_sm = 0, regs_sm = 0, optin = 0;
  GB_CHECK(cudaGetDevice(&dev));
  GB_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  GB_CHECK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  GB_CHECK(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
  GB_CHECK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  GB_CHECK(cudaFuncGetAttributes(&fa, kern));
  int per_sm = smem_sm / int(smem + fa.sharedSizeBytes + 1024);
  const int by_regs = regs_sm / (((fa.numRegs + 7) / 8) * 8 * 128);
  if (by_regs < per_sm) per_sm = by_regs;
  if (per_sm > 8) per_sm = 8;
  if (per_sm < 1) per_sm = 1;
  cudaFuncAttributes fw;
  GB_CHECK(cudaFuncGetAttributes(&fw, k_coarse_mma_ws<BF16, N, 2, false, false>));
  const size_t ws_limit = size_t(optin) - fw.sharedSizeBytes;
  // the pipelined kernel bulk-copies spinor rows: every lattice's x must
  // start on a 16-byte boundary (n nrhs 8-byte rows keep the rest aligned)
  bool aligned = true;
  for (int i = 0; i < batch.count; ++i)
    aligned = aligned && (reinterpret_cast<uintptr_t>(batch.lat[i].x) % 16 == 0) &&
              (reinterpret_cast<uintptr_t>(batch.lat[i].links) % 16 == 0);
  // A pre-converted launch needs a buffer of the batch's operand tiles (as
  // large as x); it is offered only when one exists or can be made now (not
  // while the stream is being captured).
  const size_t xc_bytes = size_t(batch.total) * size_t(8) * nrhs * N;
  unsigned char* xc = nullptr;
  if (pool && aligned) {
    if (!pool->empty() && pool->back()->bytes >= xc_bytes) {
      xc = pool->back()->as<unsigned char>();
    } else {
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      GB_CHECK(cudaStreamIsCapturing(st, &cs));
      if (cs == cudaStreamCaptureStatusNone) {
        try {
          auto b = std::make_unique<DevBuf>();
          b->alloc(xc_bytes);
          pool->push_back(std::move(b));
          xc = pool->back()->as<unsigned char>();
        } catch (const Error&) {
          cudaGetLastError();  // no room: offer no pre-converted launch
        }
      }
    }
  }
  MmaBatch pbatch = batch;
  for (int i = 0; i < pbatch.count; ++i)
    pbatch.lat[i].xc = xc ? xc + size_t(pbatch.lat[i].site0) * 8 * nrhs * N : nullptr;
  // Autotuned launch shape: choice 100000 PC + 10000 IL + 1000 cps + 100 KH
  // + 10 SL + SA is the pipelined kernel with cps persistent CTAs per SM (KH
  // half slots per stage, SL-deep load ring, SA-deep operand ring, IL = 1:
  // interleaved accumulator rows and the register epilogue, 0: split rows
  // staged through shared memory; PC = 1: the operand pre-converted by
  // k_spinor_tile_mma and bulk-copied with the links, SA = SL); choice
  // q <= 8 the register-staged kernel with q resident CTAs per SM.
  std::vector<int> cands;
  for (int PC : {0, 1}) {
    if (!aligned || (PC && !xc)) continue;
    for (int IL : {0, 1})
      for (int cps : {1, 2, 3}) {
        // shared memory of one SM split between cps CTAs (1 KB reserved each)
        const size_t lim = std::min(ws_limit, size_t(smem_sm) / cps - 1024 - fw.sharedSizeBytes);
        // ring depths are multiples of the four converting warps (see the
        // kernel's comment on barrier phases)
        for (int KH : {2, 1})
          for (int SA : {4, 8})
            for (int SL : {8, 4})
              if ((!PC || SA == SL) && ws_fits(N, KH, nrhs, SL, SA, IL != 0, PC != 0, lim))
                cands.push_back(100000 * PC + 10000 * IL + 1000 * cps + 100 * KH + 10 * SL + SA);
      }
  }
  cands.push_back(per_sm);
  if (per_sm > 1) cands.push_back(1);
  auto launch = [&](int q) {
    if (q > 1000) {
      const bool PC = q >= 100000, IL = (q / 10000) % 10 == 1;
      const int cps = (q / 1000) % 10, KH = (q / 100) % 10, SL = (q / 10) % 10, SA = q % 10;
      const size_t sm = ws_layout(N, KH, nrhs, SL, SA, IL, PC).total;
      int grid = sms * cps;
      if (grid > batch.total) grid = batch.total;
      if (PC) {
        const size_t items = size_t(batch.total) * 2 * (N / 8) * nrhs;
        size_t blocks = (items + 511) / 512;
        if (blocks > size_t(sms) * 8) blocks = size_t(sms) * 8;
        if (IL)
          k_spinor_tile_mma<BF16, N, true><<<int(blocks), 256, 0, st>>>(pbatch, nrhs);
        else
          k_spinor_tile_mma<BF16, N, false><<<int(blocks), 256, 0, st>>>(pbatch, nrhs);
      }
      auto go = [&](auto kern) {
        GB_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)));
        if (PC) {
          // programmatic dependent launch on the pre-pass: the apply's CTAs
          // set up (TMEM, barriers) while the pre-pass drains; the copy
          // issuer waits for the pre-pass before reading its operand
          cudaLaunchConfig_t cfg = {};
          cfg.gridDim = dim3(grid);
          cfg.blockDim = dim3(kWsThreads);
          cfg.dynamicSmemBytes = sm;
          cfg.stream = st;
          cudaLaunchAttribute at[1];
          at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
          at[0].val.programmaticStreamSerializationAllowed = 1;
          cfg.attrs = at;
          cfg.numAttrs = 1;
          GB_CHECK(cudaLaunchKernelEx(&cfg, kern, pbatch, nrhs, SL, SA, err));
        } else {
          kern<<<grid, kWsThreads, sm, st>>>(pbatch, nrhs, SL, SA, err);
        }
      };
      const int form = (KH == 2 ? 4 : 0) + (IL ? 2 : 0) + (PC ? 1 : 0);
      switch (form) {
        case 0: go(k_coarse_mma_ws<BF16, N, 1, false, false>); break;
        case 1: go(k_coarse_mma_ws<BF16, N, 1, false, true>); break;
        case 2: go(k_coarse_mma_ws<BF16, N, 1, true, false>); break;
        case 3: go(k_coarse_mma_ws<BF16, N, 1, true, true>); break;
        case 4: go(k_coarse_mma_ws<BF16, N, 2, false, false>); break;
        case 5: go(k_coarse_mma_ws<BF16, N, 2, false, true>); break;
        case 6: go(k_coarse_mma_ws<BF16, N, 2, true, false>); break;
        default: go(k_coarse_mma_ws<BF16, N, 2, true, true>); break;
      }
      return;
    }
    int grid = sms * q;
    if (grid > batch.total) grid = batch.total;
    kern<<<grid, 128, smem, st>>>(batch, nrhs, err);
  };
  if (!tune || batch.stall) {
    launch(cands.front());
    return;
  }
  const std::string key = std::string("mma2/") + (BF16 ? "bf16" : "f16") + "/n" +
                          std::to_string(N) + "/r" + std::to_string(nrhs) + "/v" +
                          std::to_string(batch.total) + "/b" + std::to_string(batch.count);
  launch(Tuner::get().choose(key, cands, st, launch));
}

int take_injected_stall(mg_ctx* c) {
  if (c->inject_mma_stall <= 0) return 0;
  --c->inject_mma_stall;
  return 1;
}

MmaLattice lattice_of(const Level& L, void* y, const void* x) {
  MmaLattice m;
  m.links = L.links_mma.as<uint4>();
  m.scales = L.scales.as<float>();
  m.x = (const cpx<float>*)x;
  m.y = (cpx<float>*)y;
  m.g = L.g;
  m.site0 = 0;
  return m;
}

template <bool BF16, int N>
void launch_mma(mg_ctx* c, const Level& L, void* y, const void* x, int nrhs, cudaStream_t st) {
  MmaBatch b{};
  b.lat[0] = lattice_of(L, y, x);
  b.count = 1;
  b.total = L.g.vol;
  b.stall = take_injected_stall(c);
  launch_mma_batch<BF16, N>(c->status.as<int>() + 1, b, nrhs, st, true, &c->mma_xc);
}

}  // namespace

bool coarse_apply_mma_supported(const Level& L, int nrhs) {
  return (L.prec == MG_BF16 || L.prec == MG_F16) && L.links_mma.p && nrhs >= 2 && nrhs <= 64 &&
         nrhs % 4 == 0 && (L.nd == 32 || L.nd == 48 || L.nd == 64);
}

void coarse_apply_mma(mg_ctx* c, int level, void* y, const void* x, int nrhs, cudaStream_t st) {
  Level& L = c->L[level];
  const bool bf16 = L.prec == MG_BF16;
  switch (L.nd) {
    case 32: bf16 ? launch_mma<true, 32>(c, L, y, x, nrhs, st) : launch_mma<false, 32>(c, L, y, x, nrhs, st); break;
    case 48: bf16 ? launch_mma<true, 48>(c, L, y, x, nrhs, st) : launch_mma<false, 48>(c, L, y, x, nrhs, st); break;
    default: bf16 ? launch_mma<true, 64>(c, L, y, x, nrhs, st) : launch_mma<false, 64>(c, L, y, x, nrhs, st); break;
  }
}

void links_tile_mma(mg_ctx* c, int level, cudaStream_t st) {
  Level& L = c->L[level];
  if (!(L.prec == MG_BF16 || L.prec == MG_F16) || L.nd % 16) return;
  const size_t total = size_t(L.g.vol) * 9 * L.nd * L.nd;
  L.links_mma.alloc(total * 4);
  int blocks = ceil_div(total, 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (L.prec == MG_BF16)
    k_links_tile_mma<true><<<blocks, 256, 0, st>>>(L.links_mma.as<uint32_t>(),
                                                   L.links.as<cpx<float>>(), L.scales.as<float>(),
                                                   L.g.vol, L.nd);
  else
    k_links_tile_mma<false><<<blocks, 256, 0, st>>>(L.links_mma.as<uint32_t>(),
                                                    L.links.as<cpx<float>>(), L.scales.as<float>(),
                                                    L.g.vol, L.nd);
  GB_LAUNCH_CHECK();
  c->launches++;
}

}  // namespace gbmg

extern "C" mg_status mg_coarse_apply_multi(mg_ctx* const* ctxs, const int* levels,
                                           void* const* y, const void* const* x, int count,
                                           int nrhs, void* stream) {
  using namespace gbmg;
  try {
    GB_REQUIRE(ctxs && levels && y && x && count >= 1 && count <= kMaxBatch, MG_ERR_ARG,
               "coarse_apply_multi: 1..8 lattices with non-null arrays");
    MmaBatch b{};
    int n = 0;
    mg_prec prec = MG_F64;
    for (int i = 0; i < count; ++i) {
      mg_ctx* c = ctxs[i];
      GB_REQUIRE(c && levels[i] >= 1 && levels[i] < c->nlevels, MG_ERR_ARG,
                 "coarse_apply_multi: bad context or level");
      const Level& L = c->L[levels[i]];
      GB_REQUIRE(L.have_op, MG_ERR_STATE, "coarse_apply_multi: coarse operator not built");
      GB_REQUIRE(coarse_apply_mma_supported(L, nrhs), MG_ERR_ARG,
                 "coarse_apply_multi: needs BF16/FP16 links, n in {32,48,64}, nrhs 4..64 (x4)");
      GB_REQUIRE(i == 0 || (L.nd == n && L.prec == prec), MG_ERR_ARG,
                 "coarse_apply_multi: all lattices need the same n and precision");
      GB_REQUIRE(y[i] && x[i] && y[i] != x[i], MG_ERR_ARG, "coarse_apply_multi: bad vectors");
      n = L.nd;
      prec = L.prec;
      b.lat[i] = lattice_of(L, y[i], x[i]);
      b.lat[i].site0 = b.total;
      b.total += L.g.vol;
    }
    b.count = count;
    b.stall = take_injected_stall(ctxs[0]);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* err = ctxs[0]->status.as<int>() + 1;
    const bool bf16 = prec == MG_BF16;
    switch (n) {
      case 32: bf16 ? launch_mma_batch<true, 32>(err, b, nrhs, st, true, &ctxs[0]->mma_xc) : launch_mma_batch<false, 32>(err, b, nrhs, st, true, &ctxs[0]->mma_xc); break;
      case 48: bf16 ? launch_mma_batch<true, 48>(err, b, nrhs, st, true, &ctxs[0]->mma_xc) : launch_mma_batch<false, 48>(err, b, nrhs, st, true, &ctxs[0]->mma_xc); break;
      default: bf16 ? launch_mma_batch<true, 64>(err, b, nrhs, st, true, &ctxs[0]->mma_xc) : launch_mma_batch<false, 64>(err, b, nrhs, st, true, &ctxs[0]->mma_xc); break;
    }
    GB_LAUNCH_CHECK();
    for (int i = 0; i < count; ++i) ctxs[i]->launches += (i == 0);
    return MG_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    if (ctxs && count >= 1 && ctxs[0]) ctxs[0]->err = e.what();
    return e.code;
  }
}
