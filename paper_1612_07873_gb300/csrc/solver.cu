// Adaptive setup iteration (Sec. 3.4 step 1) and the K-cycle multigrid
// solver of Sec. 7.1: flexible GCR(nkrylov) on the fine and intermediate
// levels, preconditioned by the next level; MR pre/post smoothing; GCR on
// the coarsest level.
//
// Precision: the outer GCR keeps x and r in FP64 and recomputes the true
// residual b - M x with the FP64 fine operator at every restart; its Krylov
// vectors, the K-cycle and all coarse levels run in each level's vector
// precision.  Inner products accumulate in FP64.  Scalars (MR and GCR
// coefficients) stay on the device; the host reads one residual norm per
// right-hand side per GCR step to decide convergence.
//
// Several right-hand sides: every vector of the solver holds nr right-hand
// sides back to back and every step acts on all of them at once (one
// batched kernel per step, per-RHS scalars), so the fine operator's links,
// the prolongator and the coarse links are read once per step for all nr.
// A GCR loop ends when every right-hand side meets its tolerance.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "kernels.cuh"

struct mg_ctx::SolverWS {
  struct LevelWS {
    std::vector<std::unique_ptr<gbmg::DevBuf>> Z, W;
    gbmg::DevBuf r, x, rhs, tmp, kres, mrx, mrr, mrp;
    gbmg::DevBuf eo1, eo2, eo3;  // red-black: each holds two compact parity halves
    gbmg::DevBuf s16x, s16r, s16p;  // 16-bit fine-level smoother (BF16 vectors)
    gbmg::DevBuf r64, tmp64;     // level 0 only
  };
  LevelWS lv[MG_MAX_LEVELS];
  int nk = 0;
  int nr = 0;  // right-hand sides the buffers hold
};

mg_ctx::mg_ctx() = default;

mg_ctx::~mg_ctx() {
  ws.reset();
  if (h_scalars) cudaFreeHost(h_scalars);
}

namespace gbmg {

namespace {

// scalar slots per level
inline int slot(int level, int k) { return level * 8 + k; }
enum { S_BETA = 0, S_NRM = 1, S_ALPHA = 2, S_R = 3, S_PR = 4, S_PP = 5 };

Vec vbuf(DevBuf& b, mg_prec p, size_t n, int nr = 1) {
  Vec v;
  v.p = b.p;
  v.prec = p;
  v.n = n;
  v.nr = nr;
  return v;
}

void ensure(DevBuf& b, size_t bytes) {
  if (b.bytes != bytes) b.alloc(bytes);
}

// solver buffers for nr right-hand sides (reallocated when nr changes)
void ensure_ws(mg_ctx* c, int nr) {
  if (!c->ws) c->ws.reset(new mg_ctx::SolverWS());
  auto& ws = *c->ws;
  const int nk = c->p.gcr_nkrylov;
  for (int l = 0; l < c->nlevels; ++l) {
    Level& L = c->L[l];
    auto& w = ws.lv[l];
    const size_t vb = L.vec_bytes() * nr;
    if (int(w.Z.size()) != nk) {
      w.Z.clear();
      w.W.clear();
      for (int k = 0; k < nk; ++k) {
        w.Z.emplace_back(new DevBuf());
        w.W.emplace_back(new DevBuf());
      }
    }
    for (int k = 0; k < nk; ++k) {
      ensure(*w.Z[k], vb);
      ensure(*w.W[k], vb);
    }
    ensure(w.r, vb);
    ensure(w.x, vb);
    ensure(w.rhs, vb);
    ensure(w.tmp, vb);
    ensure(w.kres, vb);
    ensure(w.mrx, vb);
    ensure(w.mrr, vb);
    ensure(w.mrp, vb);
    if (c->p.red_black && L.have_schur) {
      ensure(w.eo1, vb);
      ensure(w.eo2, vb);
      ensure(w.eo3, vb);
    }
    if (l == 0) {
      ensure(w.r64, L.vec_elems() * 16 * nr);
      ensure(w.tmp64, L.vec_elems() * 16 * nr);
      if (smoother16_enabled(c)) {
        ensure(w.s16x, L.vec_elems() * 4 * nr);
        ensure(w.s16r, L.vec_elems() * 4 * nr);
        ensure(w.s16p, L.vec_elems() * 4 * nr);
      }
    }
  }
  ws.nk = nk;
  ws.nr = nr;
}

// real parts of slot s for the nr right-hand sides
std::vector<double> read_slot(mg_ctx* c, int s, int nr, cudaStream_t st) {
  std::vector<double> v(nr);
  blas_read_slot(c, s, nr, v.data(), st);
  return v;
}

// x = MR_k(b) from a zero guess.  res (optional, level precision, not b):
// receives the smoother's own residual b - A x, which MR keeps up to date.
void mr_smooth(mg_ctx* c, int l, Vec x, Vec b, cudaStream_t st, const Vec* res = nullptr) {
  auto& w = c->ws->lv[l];
  Level& L = c->L[l];
  if (l == 0 && smoother16_enabled(c)) {
    // the same MR steps on BF16 vectors with the BF16 copy of the operator
    Vec x16 = vbuf(w.s16x, MG_BF16, L.vec_elems(), x.nr);
    Vec r16 = vbuf(w.s16r, MG_BF16, L.vec_elems(), x.nr);
    Vec p16 = vbuf(w.s16p, MG_BF16, L.vec_elems(), x.nr);
    blas_zero(c, x16, st);
    blas_copy(c, r16, b, st);
    for (int k = 0; k < c->p.mr_iters; ++k) {
      wilson16_apply(c, p16, r16, st);
      blas_dot2(c, p16, r16, slot(l, S_PR), slot(l, S_PP), st);
      blas_mr_update(c, x16, r16, p16, slot(l, S_PR), slot(l, S_PP), c->p.mr_omega, st);
    }
    blas_copy(c, x, x16, st);
    if (res) blas_copy(c, *res, r16, st);
    return;
  }
  Vec r = res ? *res : vbuf(w.mrr, L.vprec, L.vec_elems(), x.nr);
  Vec p = vbuf(w.mrp, L.vprec, L.vec_elems(), x.nr);
  blas_zero(c, x, st);
  blas_copy(c, r, b, st);
  for (int k = 0; k < c->p.mr_iters; ++k) {
    level_apply(c, l, p, r, st);
    blas_dot2(c, p, r, slot(l, S_PR), slot(l, S_PP), st);
    blas_mr_update(c, x, r, p, slot(l, S_PR), slot(l, S_PP), c->p.mr_omega, st);
  }
}

// compact parity half k (0 or 1) of a full-size buffer holding nr vectors:
// [nr][V/2][nd] at byte offset k * (buffer bytes / 2)
Vec half(DevBuf& b, const Level& L, int k, int nr) {
  Vec v;
  v.prec = L.vprec;
  v.n = L.vec_elems() / 2;
  v.nr = nr;
  v.p = static_cast<char*>(b.p) + size_t(k) * (L.vec_bytes() / 2) * nr;
  return v;
}

// out_o = S in_o = A_o in_o - H_oe A_e^-1 H_eo in_o; tmp_e: a compact even vector
void schur_apply(mg_ctx* c, int l, Vec out, Vec in, Vec tmp, cudaStream_t st) {
  eo_apply(c, l, EO_AINV_HOP, tmp, in, nullptr, 0, st);
  eo_apply(c, l, EO_A_XC_MINUS_HOP, out, tmp, in.p, 1, st);
}

// z = approximate M^-1 r through the Schur system (Secs. 3.3, 7.1):
// b^ = r_o - H_oe A_e^-1 r_e, x_o = MR_k(S, b^), z_e = A_e^-1 (r_e - H_eo x_o).
// res (optional): the full residual r - M z, which is zero on the even
// sites (z_e solves the even rows exactly) and b^ - S x_o, the MR
// residual, on the odd ones.
void schur_smooth(mg_ctx* c, int l, Vec z, Vec r, cudaStream_t st, const Vec* res = nullptr) {
  auto& w = c->ws->lv[l];
  Level& L = c->L[l];
  const int nr = z.nr;
  Vec he = half(w.eo1, L, 0, nr), ho = half(w.eo1, L, 1, nr);
  Vec ht = half(w.eo2, L, 0, nr), hx = half(w.eo2, L, 1, nr);
  Vec hr = half(w.mrr, L, 0, nr), hp = half(w.mrp, L, 0, nr);
  eo_split(c, l, he, ho, r, st);
  eo_ainv(c, l, ht, he, st);
  eo_apply(c, l, EO_XC_MINUS_HOP, hr, ht, ho.p, 1, st);  // MR residual starts at b^
  blas_zero(c, hx, st);
  for (int k = 0; k < c->p.mr_iters; ++k) {
    schur_apply(c, l, hp, hr, ht, st);
    blas_dot2(c, hp, hr, slot(l, S_PR), slot(l, S_PP), st);
    blas_mr_update(c, hx, hr, hp, slot(l, S_PR), slot(l, S_PP), c->p.mr_omega, st);
  }
  eo_apply(c, l, EO_AINV_XC_MINUS_HOP, ht, hx, he.p, 0, st);
  eo_merge(c, l, z, ht, hx, st);
  if (res) {
    blas_zero(c, he, st);
    eo_merge(c, l, *res, he, hr, st);
  }
}

struct GcrOut {
  int iters = 0;
  int restarts = 0;
  bool converged = false;
  std::vector<double> rel;     // final relative residual per right-hand side
  std::vector<int> conv_iter;  // step at which each right-hand side met tol
};

void kcycle(mg_ctx* c, int l, Vec z, Vec r, cudaStream_t st, mg_solve_stats* stats);

// Flexible GCR at level l on x.nr right-hand sides.  x, b: level-0 -> FP64;
// inner levels -> vprec.  stats: one record per right-hand side (or null);
// level totals go to stats[0].
// schur: solve S x_o = b^ on compact odd vectors (no preconditioner).
GcrOut gcr(mg_ctx* c, int l, Vec x, Vec b, bool precond, double tol, int maxiter,
           cudaStream_t st, mg_solve_stats* stats, bool record, bool schur = false) {
  auto& w = c->ws->lv[l];
  Level& L = c->L[l];
  const size_t n = schur ? L.vec_elems() / 2 : L.vec_elems();
  const int nr = x.nr;
  const bool outer = (l == 0);
  Vec r = outer ? vbuf(w.r64, MG_F64, n, nr) : vbuf(w.r, L.vprec, n, nr);
  Vec rK = vbuf(w.r, L.vprec, n, nr);  // residual in level precision (outer level)
  Vec tmp = outer ? vbuf(w.tmp64, MG_F64, n, nr) : vbuf(w.tmp, L.vprec, n, nr);
  Vec etmp;
  if (schur) etmp = half(w.eo3, L, 0, nr);
  auto op = [&](Vec o, Vec i) {
    if (schur)
      schur_apply(c, l, o, i, etmp, st);
    else
      level_apply(c, l, o, i, st);
  };
  GcrOut out;
  out.rel.assign(nr, 0.0);
  out.conv_iter.assign(nr, -1);
  blas_norm2(c, b, slot(l, S_R), st);
  const std::vector<double> b2 = read_slot(c, slot(l, S_R), nr, st);
  blas_zero(c, x, st);
  std::vector<double> tol2(nr);
  bool any = false;
  for (int v = 0; v < nr; ++v) {
    GB_REQUIRE(std::isfinite(b2[v]), MG_ERR_NUMERICAL, "gcr: non-finite right-hand side");
    tol2[v] = tol * tol * b2[v];
    any = any || b2[v] > 0.0;
    if (!(b2[v] > 0.0)) out.conv_iter[v] = 0;
  }
  if (!any) {
    out.converged = true;
    return out;
  }
  blas_copy(c, r, b, st);
  const int nk = c->ws->nk;
  // true when every right-hand side meets its tolerance; records the step
  // at which each first did
  auto check = [&](const std::vector<double>& r2) {
    bool all = true;
    for (int v = 0; v < nr; ++v) {
      GB_REQUIRE(std::isfinite(r2[v]), MG_ERR_NUMERICAL, "gcr: non-finite residual");
      out.rel[v] = b2[v] > 0.0 ? std::sqrt(r2[v] / b2[v]) : 0.0;
      if (r2[v] <= tol2[v]) {
        if (out.conv_iter[v] < 0) out.conv_iter[v] = out.iters;
      } else {
        all = false;
      }
    }
    return all;
  };
  while (true) {
    bool done = false;
    for (int k = 0; k < nk; ++k) {
      Vec Zk = vbuf(*w.Z[k], L.vprec, n, nr), Wk = vbuf(*w.W[k], L.vprec, n, nr);
      if (precond) {
        if (outer && r.prec != L.vprec) {
          blas_copy(c, rK, r, st);
          kcycle(c, l, Zk, rK, st, stats);
        } else {
          kcycle(c, l, Zk, r, st, stats);
        }
      } else {
        blas_copy(c, Zk, r, st);
      }
      op(Wk, Zk);
      // block (classical) Gram-Schmidt against the previous W_j, up to kCgs
      // per pass: all beta_j = <W_j, W_k> in one pass over the vectors,
      // then one update of W_k and one of Z_k
      for (int j0 = 0; j0 < k; j0 += kCgs) {
        const int m = std::min(kCgs, k - j0);
        Vec Ws[kCgs], Zs[kCgs];
        for (int j = 0; j < m; ++j) {
          Ws[j] = vbuf(*w.W[j0 + j], L.vprec, n, nr);
          Zs[j] = vbuf(*w.Z[j0 + j], L.vprec, n, nr);
        }
        const int cs = SC_CGS + kCgs * l;
        blas_dot_multi(c, Ws, m, Wk, cs, st, outer);
        blas_axpy_multi(c, Wk, Ws, m, cs, -1.0, st);
        blas_axpy_multi(c, Zk, Zs, m, cs, -1.0, st);
      }
      blas_norm2(c, Wk, slot(l, S_NRM), st, outer);
      blas_scale_invnorm(c, Wk, Zk, slot(l, S_NRM), st);
      blas_dot(c, Wk, r, slot(l, S_ALPHA), st);
      blas_gcr_update(c, x, r, Zk, Wk, slot(l, S_ALPHA), st);
      blas_norm2(c, r, slot(l, S_R), st);
      const std::vector<double> r2 = read_slot(c, slot(l, S_R), nr, st);
      out.iters++;
      done = check(r2);
      if (record && stats)
        for (int v = 0; v < nr; ++v)
          if (stats[v].history_len < 512) stats[v].history[stats[v].history_len++] = out.rel[v];
      if (done || out.iters >= maxiter) break;
    }
    if (done || out.iters >= maxiter) {
      out.converged = done;
      break;
    }
    // restart: true residual
    op(tmp, x);
    blas_sub(c, r, b, tmp, st);
    out.restarts++;
    blas_norm2(c, r, slot(l, S_R), st);
    if (check(read_slot(c, slot(l, S_R), nr, st))) {
      out.converged = true;
      break;
    }
  }
  if (stats) stats[0].level_iters[l] += out.iters;
  return out;
}

void kcycle(mg_ctx* c, int l, Vec z, Vec r, cudaStream_t st, mg_solve_stats* stats) {
  auto& w = c->ws->lv[l];
  Level& L = c->L[l];
  const size_t n = L.vec_elems();
  const int nr = z.nr;
  Vec tmp = vbuf(w.tmp, L.vprec, n, nr), kres = vbuf(w.kres, L.vprec, n, nr);
  Vec mrx = vbuf(w.mrx, L.vprec, n, nr);
  const int nl = l + 1;
  Level& C = c->L[nl];
  auto& wc = c->ws->lv[nl];
  Vec rc = vbuf(wc.rhs, C.vprec, C.vec_elems(), nr), ec = vbuf(wc.x, C.vprec, C.vec_elems(), nr);
  const bool rb = c->p.red_black && L.have_schur;
  auto smooth = [&](Vec out, Vec in, const Vec* res) {
    if (rb)
      schur_smooth(c, l, out, in, st, res);
    else
      mr_smooth(c, l, out, in, st, res);
  };
  // pre-smooth; the smoother hands back kres = r - A z from its own
  // residual recurrence (equal to the recomputed residual in exact
  // arithmetic), which saves an operator apply per cycle
  smooth(z, r, &kres);
  // coarse-grid correction
  restrict_apply(c, l, rc, kres, st);
  if (nl == c->nlevels - 1) {
    if (c->p.red_black && C.have_schur) {
      // coarsest solve on the Schur system, then the even sites
      Vec he = half(wc.eo1, C, 0, nr), hb = half(wc.eo1, C, 1, nr);
      Vec ht = half(wc.eo2, C, 0, nr), hx = half(wc.eo2, C, 1, nr);
      eo_split(c, nl, he, hx, rc, st);
      eo_ainv(c, nl, ht, he, st);
      eo_apply(c, nl, EO_XC_MINUS_HOP, hb, ht, hx.p, 1, st);
      gcr(c, nl, hx, hb, false, c->p.coarse_tol, c->p.coarse_maxiter, st, stats, false, true);
      eo_apply(c, nl, EO_AINV_XC_MINUS_HOP, ht, hx, he.p, 0, st);
      eo_merge(c, nl, ec, ht, hx, st);
    } else {
      gcr(c, nl, ec, rc, false, c->p.coarse_tol, c->p.coarse_maxiter, st, stats, false);
    }
  } else {
    gcr(c, nl, ec, rc, true, c->p.inner_tol, c->p.inner_maxiter, st, stats, false);
  }
  prolong_apply(c, l, tmp, ec, st);
  blas_axpy_host(c, z, tmp, 1.0, 0.0, st);
  // post-smooth
  level_apply(c, l, tmp, z, st);
  blas_sub(c, kres, r, tmp, st);
  smooth(mrx, kres, nullptr);
  blas_axpy_host(c, z, mrx, 1.0, 0.0, st);
}

}  // namespace

void level_apply(mg_ctx* c, int level, Vec out, Vec in, cudaStream_t st) {
  GB_REQUIRE(out.nr == in.nr, MG_ERR_ARG, "level_apply: shape mismatch");
  if (level == 0)
    wilson_apply(c, out, in, in.nr, st);
  else
    coarse_apply_blocked(c, level, out.p, in.p, in.nr, st);
}

void setup_sweeps(mg_ctx* c, int l, const void* init, cudaStream_t st) {
  Level& L = c->L[l];
  const int nv = L.nvec;
  const size_t n = L.vec_elems();
  GB_REQUIRE(nv <= 64, MG_ERR_ARG, "setup: at most 64 null vectors");
  L.raw.alloc(size_t(nv) * n * 16);
  // all nv vectors back to back: X[v] at offset v * n
  DevBuf xb, tb, qb;
  const size_t bytes = size_t(nv) * n * prec_bytes_complex(L.vprec);
  xb.alloc(bytes);
  tb.alloc(bytes);
  qb.alloc(bytes);
  Vec X = vbuf(xb, L.vprec, n), T = vbuf(tb, L.vprec, n), Q = vbuf(qb, L.vprec, n);
  Vec Xall = vbuf(xb, L.vprec, n * nv);
  Vec raw = vbuf(L.raw, MG_F64, n * nv);
  if (init) {
    Vec in;
    in.p = const_cast<void*>(init);
    in.prec = MG_F64;
    in.n = n * nv;
    blas_copy(c, Xall, in, st);
  } else {
    // element (v, j) draws counter v * n + j
    blas_gaussian(c, Xall, c->p.seed + 0x9E3779B97F4A7C15ull * uint64_t(l + 1), 0, st);
  }
  // coarse levels apply the operator to all vectors at once (interleaved
  // [site][dof][vec] operand layout): on the tensor cores for 16-bit stores,
  // with the FP32 multi-RHS stream for FP32 stores
  DevBuf ib, ob;
  const bool mrhs = l > 0 && coarse_apply_multi_fast(L, nv);
  if (mrhs) {
    ib.alloc(bytes);
    ob.alloc(bytes);
  }
  auto apply_all = [&](Vec out, Vec in) {
    if (l == 0) {
      wilson_apply(c, out, in, nv, st);
    } else if (mrhs) {
      Vec vi = vbuf(ib, L.vprec, n), vo = vbuf(ob, L.vprec, n);
      blas_transpose(c, vi, in, nv, true, st);
      coarse_apply(c, l, vo.p, vi.p, nv, st);
      blas_transpose(c, out, vo, nv, false, st);
    } else {
      const size_t vb = n * prec_bytes_complex(L.vprec);
      for (int v = 0; v < nv; ++v)
        coarse_apply(c, l, (char*)out.p + v * vb, (const char*)in.p + v * vb, 1, st);
    }
  };
  // minimal-residual steps on A x = 0 for every vector at once:
  //   t = A x,  q = A t,  x <- x - (<q, t> / <q, q>) t
  for (int k = 0; k < c->p.setup_sweeps; ++k) {
    apply_all(T, X);
    apply_all(Q, T);
    blas_dot2_batched(c, Q, T, nv, st);
    blas_sweep_update_batched(c, X, T, nv, st);
  }
  blas_normalise_batched(c, X, nv, st);
  blas_copy(c, raw, Xall, st);
  L.have_raw = true;
  L.have_V = false;
  GB_CHECK(cudaStreamSynchronize(st));
}

void gcr_solve_multi(mg_ctx* c, void* xp, const void* bp, int nr, double tol, int maxiter,
                     mg_solve_stats* stats, cudaStream_t st) {
  GB_REQUIRE(nr >= 1 && nr <= kMaxNrhs, MG_ERR_ARG, "solve: nrhs out of range");
  for (int l = 0; l + 1 < c->nlevels; ++l) {
    GB_REQUIRE(c->L[l].have_V, MG_ERR_STATE, "solve: null vectors of a level missing");
    GB_REQUIRE(c->L[l + 1].have_op, MG_ERR_STATE, "solve: coarse operator missing");
  }
  ensure_ws(c, nr);
  auto t0 = std::chrono::steady_clock::now();
  std::vector<mg_solve_stats> local(nr);
  mg_solve_stats* s = stats ? stats : local.data();
  for (int v = 0; v < nr; ++v) s[v] = mg_solve_stats{};
  Level& L = c->L[0];
  const size_t n = L.vec_elems();
  Vec x, b;
  x.p = xp;
  x.prec = MG_F64;
  x.n = n;
  x.nr = nr;
  b.p = const_cast<void*>(bp);
  b.prec = MG_F64;
  b.n = n;
  b.nr = nr;
  GcrOut o = gcr(c, 0, x, b, true, tol, maxiter, st, s, true);
  // true residual of the returned x, in FP64
  auto& w = c->ws->lv[0];
  Vec tmp = vbuf(w.tmp64, MG_F64, n, nr), r = vbuf(w.r64, MG_F64, n, nr);
  level_apply(c, 0, tmp, x, st);
  blas_sub(c, r, b, tmp, st);
  blas_norm2(c, r, slot(0, S_R), st);
  const std::vector<double> r2 = read_slot(c, slot(0, S_R), nr, st);
  blas_norm2(c, b, slot(0, S_R), st);
  const std::vector<double> b2 = read_slot(c, slot(0, S_R), nr, st);
  const double secs =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int v = 0; v < nr; ++v) {
    s[v].iters = o.conv_iter[v] >= 0 ? o.conv_iter[v] : o.iters;
    s[v].restarts = o.restarts;
    if (v > 0)
      for (int l = 0; l < MG_MAX_LEVELS; ++l) s[v].level_iters[l] = s[0].level_iters[l];
    s[v].true_residual = b2[v] > 0 ? std::sqrt(r2[v] / b2[v]) : 0.0;
    s[v].seconds = secs;
  }
  if (!o.converged) throw Error(MG_ERR_NOT_CONVERGED, "gcr: maxiter reached before tolerance");
}

void gcr_solve(mg_ctx* c, void* xp, const void* bp, double tol, int maxiter,
               mg_solve_stats* stats, cudaStream_t st) {
  gcr_solve_multi(c, xp, bp, 1, tol, maxiter, stats, st);
}

}  // namespace gbmg
