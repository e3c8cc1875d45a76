// Host-side launchers of the library's kernels (one translation unit per
// group: blas.cu, wilson.cu, coarse.cu, transfer.cu, galerkin.cu).
#pragma once

#include "context.cuh"

namespace gbmg {

// nr device vectors of n complex numbers each, stored back to back (vector
// v at offset v * n), in precision prec (F64 or F32).  Element-wise kernels
// treat them as one vector of n * nr numbers; reductions and scalar updates
// act per vector, with per-vector scalars.
struct Vec {
  void* p = nullptr;
  mg_prec prec = MG_F64;
  size_t n = 0;
  int nr = 1;
  size_t total() const { return n * size_t(nr); }
};

// ---------------------------------------------------------------- blas.cu
// Device scalars live in ctx->scalars as complex doubles: slot s holds one
// value per right-hand side, S[s][v] (kMaxNrhs per slot).
void blas_zero(mg_ctx* c, Vec v, cudaStream_t st);
void blas_copy(mg_ctx* c, Vec dst, Vec src, cudaStream_t st);        // converts precision
void blas_axpy_host(mg_ctx* c, Vec y, Vec x, double are, double aim, cudaStream_t st);
// y_v += sign * S[slot][v] * x_v
void blas_axpy_slot(mg_ctx* c, Vec y, Vec x, int slot, double sign, cudaStream_t st);
// out = b - ax
void blas_sub(mg_ctx* c, Vec out, Vec b, Vec ax, cudaStream_t st);
// S[slot][v] = <a_v, b_v> = sum conj(a_v) b_v
// fp64_partials: per-thread partial sums in FP64 even for FP32 data (the
// outer GCR's orthogonalisation); otherwise FP32 data sums per thread in FP32
void blas_dot(mg_ctx* c, Vec a, Vec b, int slot, cudaStream_t st, bool fp64_partials = false);
void blas_norm2(mg_ctx* c, Vec a, int slot, cudaStream_t st, bool fp64_partials = false);
// S[s_pr][v] = <p_v, r_v>, S[s_pp][v] = <p_v, p_v> in one pass
void blas_dot2(mg_ctx* c, Vec p, Vec r, int s_pr, int s_pp, cudaStream_t st);
// MR step per vector: a = omega S[s_pr]/S[s_pp].re ; x += a r ; r -= a p
void blas_mr_update(mg_ctx* c, Vec x, Vec r, Vec p, int s_pr, int s_pp, double omega,
                    cudaStream_t st);
// a_v *= 1/sqrt(S[slot][v].re), b_v likewise
void blas_scale_invnorm(mg_ctx* c, Vec a, Vec b, int slot, cudaStream_t st);
// x_v += S[slot][v] z_v ; r_v -= S[slot][v] w_v
void blas_gcr_update(mg_ctx* c, Vec x, Vec r, Vec z, Vec w, int slot, cudaStream_t st);
// real parts of S[slot][0..nr) to the host (synchronises st)
// Block (classical) Gram-Schmidt against m <= kCgs vectors X[j] in one
// pass each: S[slot + j] = <X[j], y> (FP64-accurate when fp64_partials;
// see blas_dot), then y += sign sum_j S[slot + j] X[j].
constexpr int kCgs = 10;  // GCR(10) needs at most 9
void blas_dot_multi(mg_ctx* c, const Vec* X, int m, Vec y, int slot, cudaStream_t st,
                    bool fp64_partials);
void blas_axpy_multi(mg_ctx* c, Vec y, const Vec* X, int m, int slot, double sign,
                     cudaStream_t st);
void blas_read_slot(mg_ctx* c, int slot, int nr, double* out_re, cudaStream_t st);
// both parts of right-hand side 0's value in `slot` (synchronises)
void blas_read_slot_c(mg_ctx* c, int slot, double out[2], cudaStream_t st);
// Setup sweeps: nvec vectors of length p.n back to back, scalars in
// ctx->batch_scalars: B[2v] = <p_v, r_v>, B[2v+1] = |p_v|^2
void blas_dot2_batched(mg_ctx* c, Vec p, Vec r, int nvec, cudaStream_t st);
// x_v -= (B[2v] / B[2v+1]) t_v
void blas_sweep_update_batched(mg_ctx* c, Vec x, Vec t, int nvec, cudaStream_t st);
// x_v /= |x_v|
void blas_normalise_batched(mg_ctx* c, Vec x, int nvec, cudaStream_t st);
// nvec vectors of out.n elements: [nvec][n] -> [n][nvec] (to_interleaved) or back
void blas_transpose(mg_ctx* c, Vec out, Vec in, int nvec, bool to_interleaved, cudaStream_t st);
// complex Gaussian (Re, Im iid N(0,1)) from a counter-based Philox4x32-10
void blas_gaussian(mg_ctx* c, Vec v, uint64_t seed, uint64_t offset, cudaStream_t st);
// a device status word check (host reads it; synchronises)
int read_status(mg_ctx* c, cudaStream_t st);
void clear_status(mg_ctx* c, cudaStream_t st);

// ---------------------------------------------------------------- wilson.cu
// Build the fine operator of level 0 from the external gauge field.
void fine_operator_build(mg_ctx* c, const void* gauge_ext, cudaStream_t st);
// out = M in on `nvec` vectors (stride vstride complex elements apart)
void wilson_apply(mg_ctx* c, Vec out, Vec in, int nvec, cudaStream_t st);

// ---------------------------------------------------------------- coarse.cu
// nrhs > 1: vectors interleaved [site][n][nrhs] (the public layout)
void coarse_apply(mg_ctx* c, int level, void* y, const void* x, int nrhs, cudaStream_t st);
// nr vectors back to back [nr][site][n] (the solver's layout)
void coarse_apply_blocked(mg_ctx* c, int level, void* y, const void* x, int nr,
                          cudaStream_t st);
void links_import(mg_ctx* c, int level, const void* ext, cudaStream_t st);
void links_export(mg_ctx* c, int level, void* ext, cudaStream_t st);
void links_pack16(mg_ctx* c, int level, cudaStream_t st);

// ---------------------------------------------------------------- coarse_mma.cu
bool coarse_apply_mma_supported(const Level& L, int nrhs);
// true when an nrhs-vector coarse apply of level L runs a multi-RHS kernel
// (tensor cores for 16-bit stores, the FP32 multi-RHS stream for FP32)
bool coarse_apply_multi_fast(const Level& L, int nrhs);
void coarse_apply_mma(mg_ctx* c, int level, void* y, const void* x, int nrhs, cudaStream_t st);
void links_tile_mma(mg_ctx* c, int level, cudaStream_t st);

// ---------------------------------------------------------------- transfer.cu
void block_orthonormalise(mg_ctx* c, int level, cudaStream_t st);
// block-orthonormal null vectors of `level` into dst [Nv][V][nd] complex double
void nullvecs_export(mg_ctx* c, int level, void* dst, cudaStream_t st);
void restrict_apply(mg_ctx* c, int level, Vec coarse, Vec fine, cudaStream_t st);
void prolong_apply(mg_ctx* c, int level, Vec fine, Vec coarse, cudaStream_t st);

// ---------------------------------------------------------------- schur.cu
// Red-black preconditioning (compact parity vectors: site s at s >> 1).
// Hops of one parity with a fused epilogue; out and xc on parity p, in on
// the other parity:
enum EoMode {
  EO_HOP = 0,                // out = H in
  EO_AINV_HOP = 1,           // out = A^-1 H in            (p even)
  EO_A_XC_MINUS_HOP = 2,     // out = A xc - H in
  EO_XC_MINUS_HOP = 3,       // out = xc - H in
  EO_AINV_XC_MINUS_HOP = 4,  // out = A^-1 (xc - H in)     (p even)
};
bool schur_supported(const mg_ctx* c, int level);
// A_e^-1 of the level's operator (FP64 inversion); throws on a singular block
void schur_prepare(mg_ctx* c, int level, cudaStream_t st);
void eo_apply(mg_ctx* c, int level, int mode, Vec out, Vec in, const void* xc, int p,
              cudaStream_t st);
// full [nr][V][nd] <-> compact halves [nr][V/2][nd]
void eo_split(mg_ctx* c, int level, Vec he, Vec ho, Vec full, cudaStream_t st);
void eo_merge(mg_ctx* c, int level, Vec full, Vec he, Vec ho, cudaStream_t st);
// out_e = A_e^-1 in_e
void eo_ainv(mg_ctx* c, int level, Vec out, Vec in, cudaStream_t st);

// ---------------------------------------------------------------- smoother16.cu
// 16-bit fine-level smoother (params.prec_smoother = MG_BF16, FP32 fine level)
bool smoother16_enabled(const mg_ctx* c);
void smoother16_prepare(mg_ctx* c, cudaStream_t st);
// out = M in on BF16 vectors (in.nr vectors back to back)
void wilson16_apply(mg_ctx* c, Vec out, Vec in, cudaStream_t st);

// ---------------------------------------------------------------- galerkin.cu
void galerkin_build(mg_ctx* c, int level, cudaStream_t st);

// ---------------------------------------------------------------- solver.cu
void level_apply(mg_ctx* c, int level, Vec out, Vec in, cudaStream_t st);
void setup_sweeps(mg_ctx* c, int level, const void* init, cudaStream_t st);
void gcr_solve(mg_ctx* c, void* x, const void* b, double tol, int maxiter, mg_solve_stats* stats,
               cudaStream_t st);
// nr right-hand sides back to back; stats: nr records or null
void gcr_solve_multi(mg_ctx* c, void* x, const void* b, int nr, double tol, int maxiter,
                     mg_solve_stats* stats, cudaStream_t st);

// message returned by mg_last_error(NULL) for calls without a context
void set_last_error(const char* msg);

inline Vec level_vec(const Level& L, void* p) {
  Vec v;
  v.p = p;
  v.prec = L.vprec;
  v.n = L.vec_elems();
  return v;
}

}  // namespace gbmg
