// Internal state of an mg_ctx: per-level operators, null vectors, solver
// workspace, kernel timing.  Host-side only.
#pragma once

#include <memory>
#include <string>
#include <vector>

#include "common.cuh"

namespace gbmg {

// Owning device allocation.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  void alloc(size_t n) {
    if (n == bytes && p) return;
    release();
    if (n == 0) return;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      throw Error(MG_ERR_OOM, "cudaMalloc of " + std::to_string(n) + " bytes failed");
    }
    bytes = n;
  }
  template <typename T>
  T* as() const { return static_cast<T*>(p); }
};

// One recorded launch of an instrumented kernel class.
struct ProfRecord {
  std::string name;
  int level;
  cudaEvent_t start, stop;
  double bytes, flops;
};

struct Profiler {
  bool on = false;
  std::vector<ProfRecord> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get();
  void clear();
  ~Profiler();
};

// Scoped timer: records start at construction, stop at destruction.
struct ProfScope {
  Profiler* prof;
  cudaStream_t st;
  ProfRecord rec;
  bool active;
  ProfScope(Profiler& p, cudaStream_t s, const char* name, int level, double bytes, double flops);
  ~ProfScope();
};

struct Level {
  int index = 0;
  Geom g{};
  int nd = 0;                  // dofs per site
  mg_prec prec = MG_F64;       // operator storage precision
  mg_prec vprec = MG_F64;      // vector precision (F64 or F32)

  // fine operator (level 0): gauge [4][V][9] complex with the t boundary
  // sign folded into the last slice; clover [V][2][36] packed Hermitian.
  DevBuf gauge64, gauge32, clover64, clover32;
  // FP32 links compressed to their first two rows [mu][V][6] complex; the
  // third row is rebuilt as conj(row0 x row1) (times the boundary sign),
  // valid when the field is special unitary to FP32 precision (checked at
  // import: gauge12_ok)
  DevBuf gauge12;
  bool gauge12_ok = false;
  // FP32 links in the 8-real form [mu][V][8] (Sec. 4 gauge compression):
  // a2, a3, b1 of U = [[a1 a2 a3][b1 b2 b3][c1 c2 c3]] and the phases of a1,
  // c1, without the boundary sign (the kernel applies it); eligible when
  // the rebuilt links deviate from the FP64 field by less than 1e-6 root-
  // mean-square and 1e-3 at most (gauge8_ok); both deviations are kept
  DevBuf gauge8;
  bool gauge8_ok = false;
  double gauge8_maxdev = 0.0, gauge8_rmsdev = 0.0;
  // BF16 copy of the operator for a 16-bit fine-level smoother: links
  // ([mu][V][6] two-row when gauge12_ok, else [mu][V][9]) and clover [V][72]
  DevBuf gauge16, clover16;
  double diag = 0.0;           // 4 + m

  // coarse operator (level >= 1): internal layout [V][9][col][row] in vprec;
  // 16-bit store + per-site scale when prec is BF16/F16.
  DevBuf links, links16, scales;
  DevBuf links_mma;            // 16-bit links tiled as the tensor-core operand
  DevBuf tr_in, tr_out;        // interleaved copies for multi-RHS tensor-core applies
  bool slots5 = false;         // single-RHS apply from 5 stored blocks
  DevBuf links5;               // [V][5][col][row]: slots 0, 1, 3, 5, 7 in the store type
  bool have_op = false;

  // coarsening to level + 1
  int nvec = 0;
  int block[4] = {1, 1, 1, 1};
  DevBuf raw;                  // FP64 [Nv][V][nd] raw null vectors
  DevBuf orth64;               // block-orthonormalised, [agg][chi][Nv][rows], 16-byte
                               // complex entries: float-float (orth_ff) or FP64
  bool orth_ff = true;
  DevBuf Vp;                   // vprec [V][nd][Nv] (transfer operator layout)
  DevBuf Vp16;                 // BF16 copy of Vp for the fine-level transfers (16-bit smoother)

  // red-black preconditioning: A_e^-1 on the even sites (fine: packed
  // Hermitian 6x6 chirality blocks, [V/2][72] reals; coarse: [V/2][col][row]
  // complex), both in the vector precision
  DevBuf ainv, xinv;
  bool have_schur = false;
  bool have_raw = false, have_V = false;

  size_t vec_elems() const { return size_t(g.vol) * nd; }
  size_t vec_bytes() const { return vec_elems() * prec_bytes_complex(vprec); }
};

// Scalars that solver kernels exchange through device memory: SC_COUNT
// slots, each with one complex double per right-hand side.
enum ScalarSlot {
  SC_CGS = 32,  // first slot of the block Gram-Schmidt coefficients (10 per level)
  SC_COUNT = 96
};
constexpr int kMaxNrhs = MG_MAX_NRHS;

}  // namespace gbmg

struct mg_ctx {
  mg_params p{};
  int nlevels = 0;
  gbmg::Level L[MG_MAX_LEVELS];
  std::string err;
  gbmg::Profiler prof;
  long long launches = 0;
  int inject_mma_stall = 0;     // fault injection: stalled tensor-core launches to come
  // tensor-core operand tiles of multi-RHS coarse applies (pre-converted x);
  // grown by appending, earlier buffers kept for graphs captured with them
  std::vector<std::unique_ptr<gbmg::DevBuf>> mma_xc;
  // reductions: per-block partials and final scalars (complex double)
  gbmg::DevBuf red_partials;   // [2][nrhs][max_blocks] double2
  gbmg::DevBuf scalars;        // [SC_COUNT][kMaxNrhs] double2
  gbmg::DevBuf status;         // device status words (int)
  gbmg::DevBuf batch_partials; // batched reductions: [nvec][2][blocks] double2
  gbmg::DevBuf batch_scalars;  // batched reductions: [2 * 64] double2
  double* h_scalars = nullptr; // pinned host mirror
  // solver workspace (allocated on first solve)
  struct SolverWS;
  std::unique_ptr<SolverWS> ws;
  mg_ctx();
  ~mg_ctx();
};
