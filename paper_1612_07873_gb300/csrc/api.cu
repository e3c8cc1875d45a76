// extern "C" entry points of libgbmg.so (declared in include/gbmg.h):
// argument checks, context lifecycle, error reporting, kernel timing.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kernels.cuh"
#include "tune.cuh"

using namespace gbmg;

namespace {
thread_local std::string g_last_error;

mg_status fail(mg_ctx* c, mg_status s, const std::string& m) {
  if (c) c->err = m;
  g_last_error = m;
  return s;
}

template <typename F>
mg_status guarded(mg_ctx* c, F&& f) {
  if (!c) return fail(nullptr, MG_ERR_ARG, "null context");
  try {
    f();
    c->err.clear();
    return MG_OK;
  } catch (const Error& e) {
    return fail(c, e.code, e.what());
  } catch (const std::exception& e) {
    return fail(c, MG_ERR_CUDA, e.what());
  }
}

cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

void check_level(mg_ctx* c, int level, int lo, int hi) {
  GB_REQUIRE(level >= lo && level <= hi && level < c->nlevels, MG_ERR_ARG,
             "level " + std::to_string(level) + " out of range");
}
}  // namespace

// ------------------------------------------------------------------ profiler
namespace gbmg {
void set_last_error(const char* msg) { g_last_error = msg; }

cudaEvent_t Profiler::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  GB_CHECK(cudaEventCreate(&e));
  return e;
}
void Profiler::clear() {
  for (auto& r : recs) {
    pool.push_back(r.start);
    pool.push_back(r.stop);
  }
  recs.clear();
}
Profiler::~Profiler() {
  clear();
  for (auto e : pool) cudaEventDestroy(e);
}
// Every scope is also an NVTX range ("<kernel class> L<level>"), visible to
// Nsight tools whether or not the event timing is enabled.
ProfScope::ProfScope(Profiler& p, cudaStream_t s, const char* name, int level, double bytes,
                     double flops)
    : prof(&p), st(s), active(p.on) {
  char label[64];
  std::snprintf(label, sizeof(label), "%s L%d", name, level);
  nvtxRangePushA(label);
  if (!active) return;
  rec.name = name;
  rec.level = level;
  rec.bytes = bytes;
  rec.flops = flops;
  rec.start = p.get();
  rec.stop = p.get();
  cudaEventRecord(rec.start, st);
}
ProfScope::~ProfScope() {
  nvtxRangePop();
  if (!active) return;
  cudaEventRecord(rec.stop, st);
  prof->recs.push_back(rec);
}
}  // namespace gbmg

// ------------------------------------------------------------------ C ABI
extern "C" {

void mg_default_params(mg_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->t_antiperiodic = 1;
  p->mass = 0.0;
  p->csw = 1.0;
  p->nlevels = 2;
  p->setup_sweeps = 10;
  p->seed = 1;
  p->prec_fine = MG_F64;
  p->prec_coarse = MG_F64;
  p->mr_iters = 4;
  p->mr_omega = 1.0;
  p->gcr_nkrylov = 10;
  p->inner_tol = 0.25;
  p->inner_maxiter = 10;
  p->coarse_tol = 0.1;
  p->coarse_maxiter = 100;
  p->link_slots = 9;
  p->red_black = 0;
  p->prec_smoother = MG_F32;
}

mg_status mg_create(const mg_params* p, const void* gauge_dev, mg_ctx** out) {
  if (!p || !out) return fail(nullptr, MG_ERR_ARG, "mg_create: null argument");
  *out = nullptr;
  if (!gauge_dev) return fail(nullptr, MG_ERR_ARG, "mg_create: null gauge field");
  if (p->nlevels < 2 || p->nlevels > MG_MAX_LEVELS)
    return fail(nullptr, MG_ERR_ARG, "mg_create: nlevels must be 2..4");
  if (p->prec_fine != MG_F64 && p->prec_fine != MG_F32)
    return fail(nullptr, MG_ERR_ARG, "mg_create: prec_fine must be F64 or F32");
  if (p->prec_coarse < MG_F64 || p->prec_coarse > MG_I16)
    return fail(nullptr, MG_ERR_ARG, "mg_create: bad prec_coarse");
  if (p->gcr_nkrylov < 1 || p->gcr_nkrylov > 64 || p->mr_iters < 0)
    return fail(nullptr, MG_ERR_ARG, "mg_create: bad solver parameters");
  int dims[4];
  long long vol = 1;
  for (int m = 0; m < 4; ++m) {
    dims[m] = p->dims[m];
    if (dims[m] < 1) return fail(nullptr, MG_ERR_ARG, "mg_create: lattice extent < 1");
    vol *= dims[m];
  }
  if (vol > (1ll << 30)) return fail(nullptr, MG_ERR_ARG, "mg_create: lattice too large");
  mg_ctx* c = new mg_ctx();
  try {
    c->p = *p;
    c->nlevels = p->nlevels;
    for (int l = 0; l < c->nlevels; ++l) {
      Level& L = c->L[l];
      L.index = l;
      if (l == 0) {
        L.g = make_geom(dims);
        L.nd = 12;
        L.prec = p->prec_fine;
      } else {
        Level& F = c->L[l - 1];
        int cd[4];
        for (int m = 0; m < 4; ++m) {
          int b = p->block[l - 1][m];
          GB_REQUIRE(b >= 1 && F.g.L[m] % b == 0, MG_ERR_ARG,
                     "extent " + std::to_string(F.g.L[m]) + " of level " + std::to_string(l - 1) +
                         " not divisible by block " + std::to_string(b));
          cd[m] = F.g.L[m] / b;
          F.block[m] = b;
        }
        GB_REQUIRE(p->nvec[l - 1] >= 1 && p->nvec[l - 1] <= 48, MG_ERR_ARG,
                   "nvec must be 1..48");
        F.nvec = p->nvec[l - 1];
        L.g = make_geom(cd);
        L.nd = 2 * F.nvec;
        L.prec = p->prec_coarse;
        GB_REQUIRE(p->link_slots == 0 || p->link_slots == 9 || p->link_slots == 5, MG_ERR_ARG,
                   "link_slots must be 9 or 5");
        L.slots5 = p->link_slots == 5;
        GB_REQUIRE(!(prec_is16(L.prec) && (L.nd % 4)), MG_ERR_ARG,
                   "16-bit coarse links need an even number of null vectors");
      }
      L.vprec = vec_prec_of(L.prec);
    }
    GB_REQUIRE(!(c->L[0].vprec == MG_F32 && c->L[1].vprec == MG_F64), MG_ERR_ARG,
               "FP64 coarse levels need an FP64 fine level");
    c->red_partials.alloc(size_t(2) * 1024 * kMaxNrhs * sizeof(double2));
    c->scalars.alloc(size_t(SC_COUNT) * kMaxNrhs * sizeof(double2));
    c->status.alloc(64);
    c->batch_scalars.alloc(2 * 64 * sizeof(double2));
    GB_CHECK(cudaMallocHost(&c->h_scalars, size_t(kMaxNrhs) * sizeof(double2)));
    GB_CHECK(cudaMemset(c->scalars.p, 0, c->scalars.bytes));
    GB_CHECK(cudaMemset(c->status.p, 0, c->status.bytes));
    GB_REQUIRE(p->prec_smoother == MG_F32 || p->prec_smoother == MG_F64 ||
                   (p->prec_smoother == MG_BF16 && p->prec_fine == MG_F32),
               MG_ERR_ARG, "prec_smoother: MG_F32, or MG_BF16 with an FP32 fine level");
    fine_operator_build(c, gauge_dev, 0);
    if (p->red_black) schur_prepare(c, 0, 0);
    smoother16_prepare(c, 0);
    GB_CHECK(cudaDeviceSynchronize());
  } catch (const Error& e) {
    delete c;
    return fail(nullptr, e.code, e.what());
  } catch (const std::exception& e) {
    delete c;
    return fail(nullptr, MG_ERR_CUDA, e.what());
  }
  *out = c;
  return MG_OK;
}

mg_status mg_destroy(mg_ctx* c) {
  if (!c) return MG_ERR_ARG;
  cudaDeviceSynchronize();
  delete c;
  return MG_OK;
}

mg_status mg_setup_nullvecs(mg_ctx* c, int level, const void* init, void* stream) {
  return guarded(c, [&] {
    check_level(c, level, 0, c->nlevels - 2);
    GB_REQUIRE(level == 0 || c->L[level].have_op, MG_ERR_STATE,
               "setup_nullvecs: operator of this level not built");
    setup_sweeps(c, level, init, S(stream));
    block_orthonormalise(c, level, S(stream));
  });
}

mg_status mg_set_nullvecs(mg_ctx* c, int level, const void* vecs, void* stream) {
  return guarded(c, [&] {
    check_level(c, level, 0, c->nlevels - 2);
    GB_REQUIRE(vecs, MG_ERR_ARG, "set_nullvecs: null pointer");
    Level& L = c->L[level];
    const size_t bytes = size_t(L.nvec) * L.vec_elems() * 16;
    L.raw.alloc(bytes);
    GB_CHECK(cudaMemcpyAsync(L.raw.p, vecs, bytes, cudaMemcpyDeviceToDevice, S(stream)));
    L.have_raw = true;
    block_orthonormalise(c, level, S(stream));
  });
}

mg_status mg_get_nullvecs(mg_ctx* c, int level, int kind, void* dst, size_t bytes, void* stream) {
  return guarded(c, [&] {
    check_level(c, level, 0, c->nlevels - 2);
    Level& L = c->L[level];
    const size_t need = size_t(L.nvec) * L.vec_elems() * 16;
    GB_REQUIRE(dst && bytes == need, MG_ERR_ARG, "get_nullvecs: size mismatch");
    GB_REQUIRE(kind == 0 || kind == 1, MG_ERR_ARG, "get_nullvecs: kind must be 0 or 1");
    if (kind == 0) {
      GB_REQUIRE(L.have_raw, MG_ERR_STATE, "get_nullvecs: not available");
      GB_CHECK(cudaMemcpyAsync(dst, L.raw.p, need, cudaMemcpyDeviceToDevice, S(stream)));
    } else {
      nullvecs_export(c, level, dst, S(stream));
    }
  });
}

mg_status mg_build_coarse(mg_ctx* c, int level, void* stream) {
  return guarded(c, [&] {
    check_level(c, level, 0, c->nlevels - 2);
    galerkin_build(c, level, S(stream));
    if (c->p.red_black) schur_prepare(c, level + 1, S(stream));
  });
}

mg_status mg_coarse_apply(mg_ctx* c, int level, void* y, const void* x, int nrhs, void* stream) {
  return guarded(c, [&] {
    check_level(c, level, 1, c->nlevels - 1);
    GB_REQUIRE(x && y, MG_ERR_ARG, "coarse_apply: null vector");
    const size_t bytes = c->L[level].vec_bytes() * size_t(nrhs > 0 ? nrhs : 1);
    const char* xa = (const char*)x;
    const char* ya = (const char*)y;
    GB_REQUIRE(ya + bytes <= xa || xa + bytes <= ya, MG_ERR_ARG,
               "coarse_apply: input and output overlap");
    coarse_apply(c, level, y, x, nrhs, S(stream));
  });
}

mg_status mg_apply(mg_ctx* c, int level, void* y, const void* x, void* stream) {
  return guarded(c, [&] {
    check_level(c, level, 0, c->nlevels - 1);
    GB_REQUIRE(x && y, MG_ERR_ARG, "apply: null vector");
    Level& L = c->L[level];
    level_apply(c, level, level_vec(L, y), level_vec(L, const_cast<void*>(x)), S(stream));
  });
}

mg_status mg_wilson_clover_apply(mg_ctx* c, void* out, const void* in, void* stream) {
  return guarded(c, [&] {
    GB_REQUIRE(in && out, MG_ERR_ARG, "wilson_clover_apply: null vector");
    Level& L = c->L[0];
    wilson_apply(c, level_vec(L, out), level_vec(L, const_cast<void*>(in)), 1, S(stream));
  });
}

mg_status mg_wilson_clover_apply_multi(mg_ctx* c, void* out, const void* in, int nrhs,
                                       void* stream) {
  return guarded(c, [&] {
    GB_REQUIRE(in && out, MG_ERR_ARG, "wilson_clover_apply_multi: null vector");
    GB_REQUIRE(nrhs >= 1 && nrhs <= 64, MG_ERR_ARG, "wilson_clover_apply_multi: bad nrhs");
    Level& L = c->L[0];
    const size_t bytes = L.vec_bytes() * size_t(nrhs);
    const char* a = (const char*)in;
    const char* b = (const char*)out;
    GB_REQUIRE(a + bytes <= b || b + bytes <= a, MG_ERR_ARG,
               "wilson_clover_apply_multi: output overlaps input");
    wilson_apply(c, level_vec(L, out), level_vec(L, const_cast<void*>(in)), nrhs, S(stream));
  });
}

mg_status mg_wilson_clover_apply_bf16(mg_ctx* c, void* out, const void* in, int nrhs,
                                      void* stream) {
  return guarded(c, [&] {
    GB_REQUIRE(in && out && in != out, MG_ERR_ARG, "wilson_clover_apply_bf16: bad vectors");
    GB_REQUIRE(nrhs >= 1 && nrhs <= 64, MG_ERR_ARG, "wilson_clover_apply_bf16: bad nrhs");
    GB_REQUIRE(smoother16_enabled(c), MG_ERR_STATE, "wilson_clover_apply_bf16: no 16-bit smoother");
    Level& L = c->L[0];
    Vec vo, vi;
    vo.p = out;
    vi.p = const_cast<void*>(in);
    vo.prec = vi.prec = MG_BF16;
    vo.n = vi.n = L.vec_elems();
    vo.nr = vi.nr = nrhs;
    wilson16_apply(c, vo, vi, S(stream));
  });
}

mg_status mg_restrict(mg_ctx* c, int level, void* coarse, const void* fine, void* stream) {
  return guarded(c, [&] {
    check_level(c, level, 0, c->nlevels - 2);
    GB_REQUIRE(coarse && fine, MG_ERR_ARG, "restrict: null vector");
    restrict_apply(c, level, level_vec(c->L[level + 1], coarse),
                   level_vec(c->L[level], const_cast<void*>(fine)), S(stream));
  });
}

mg_status mg_prolong(mg_ctx* c, int level, void* fine, const void* coarse, void* stream) {
  return guarded(c, [&] {
    check_level(c, level, 0, c->nlevels - 2);
    GB_REQUIRE(coarse && fine, MG_ERR_ARG, "prolong: null vector");
    prolong_apply(c, level, level_vec(c->L[level], fine),
                  level_vec(c->L[level + 1], const_cast<void*>(coarse)), S(stream));
  });
}

mg_status mg_gcr_solve(mg_ctx* c, void* x, const void* b, double tol, int maxiter,
                       mg_solve_stats* stats, void* stream) {
  return guarded(c, [&] {
    GB_REQUIRE(x && b && x != b, MG_ERR_ARG, "gcr_solve: bad vectors");
    GB_REQUIRE(tol > 0 && maxiter > 0, MG_ERR_ARG, "gcr_solve: bad tol/maxiter");
    gcr_solve(c, x, b, tol, maxiter, stats, S(stream));
  });
}

mg_status mg_gcr_solve_multi(mg_ctx* c, void* x, const void* b, int nrhs, double tol,
                             int maxiter, mg_solve_stats* stats, void* stream) {
  return guarded(c, [&] {
    GB_REQUIRE(x && b && x != b, MG_ERR_ARG, "gcr_solve_multi: bad vectors");
    GB_REQUIRE(nrhs >= 1 && nrhs <= MG_MAX_NRHS, MG_ERR_ARG, "gcr_solve_multi: bad nrhs");
    GB_REQUIRE(tol > 0 && maxiter > 0, MG_ERR_ARG, "gcr_solve_multi: bad tol/maxiter");
    gcr_solve_multi(c, x, b, nrhs, tol, maxiter, stats, S(stream));
  });
}

mg_status mg_tune_set(const char* key, int choice) {
  if (!key) {
    set_last_error("tune_set: null key");
    return MG_ERR_ARG;
  }
  gbmg::Tuner::get().set(key, choice);
  return MG_OK;
}

int mg_tune_get(const char* key) { return key ? gbmg::Tuner::get().get(key) : -1; }

int mg_tune_report(const char* key, int* choices, float* ms, int max) {
  if (!key) return -1;
  const auto t = gbmg::Tuner::get().report(key);
  const int n = int(t.size());
  for (int i = 0; i < n && i < max; ++i) {
    if (choices) choices[i] = t[i].first;
    if (ms) ms[i] = t[i].second;
  }
  return n;
}

mg_status mg_schur_apply(mg_ctx* c, int level, void* y, const void* x, int nrhs, void* stream) {
  return guarded(c, [&] {
    check_level(c, level, 0, c->nlevels - 1);
    Level& L = c->L[level];
    GB_REQUIRE(x && y && x != y, MG_ERR_ARG, "schur_apply: bad vectors");
    GB_REQUIRE(nrhs >= 1 && nrhs <= MG_MAX_NRHS, MG_ERR_ARG, "schur_apply: bad nrhs");
    GB_REQUIRE(L.have_schur, MG_ERR_STATE, "schur_apply: level has no red-black form");
    Vec vx, vy, vt;
    vx.p = const_cast<void*>(x);
    vy.p = y;
    vx.prec = vy.prec = vt.prec = L.vprec;
    vx.n = vy.n = vt.n = L.vec_elems() / 2;
    vx.nr = vy.nr = vt.nr = nrhs;
    DevBuf tmp;
    tmp.alloc(L.vec_bytes() / 2 * nrhs);
    vt.p = tmp.p;
    eo_apply(c, level, EO_AINV_HOP, vt, vx, nullptr, 0, S(stream));
    eo_apply(c, level, EO_A_XC_MINUS_HOP, vy, vt, x, 1, S(stream));
    GB_CHECK(cudaStreamSynchronize(S(stream)));
  });
}

// ---- checkpoint of the setup: the block-orthonormal null vectors of every
// coarsening and the coarse links of every coarse level.  File: one JSON
// header line (format, lattice, blocks, nvec, precisions, seed, the byte
// count of every record, FNV-1a 64 checksum of the payload), then the raw
// little-endian records: for l = 0 .. nlevels-2 the null vectors
// [Nv][V][nd] complex double of level l, then the links [V][9][n][n]
// complex double of level l + 1.
namespace {

uint64_t fnv1a(const unsigned char* p, size_t n, uint64_t h) {
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

std::string header_json(const mg_ctx* c, const std::vector<size_t>& sizes, uint64_t sum) {
  std::string j = "{\"format\": \"gbmg-setup-1\", \"dims\": [";
  for (int m = 0; m < 4; ++m) j += std::to_string(c->p.dims[m]) + (m < 3 ? ", " : "]");
  j += ", \"nlevels\": " + std::to_string(c->nlevels) + ", \"blocks\": [";
  for (int l = 0; l + 1 < c->nlevels; ++l) {
    j += "[";
    for (int m = 0; m < 4; ++m) j += std::to_string(c->p.block[l][m]) + (m < 3 ? ", " : "]");
    j += l + 2 < c->nlevels ? ", " : "";
  }
  j += "], \"nvec\": [";
  for (int l = 0; l + 1 < c->nlevels; ++l)
    j += std::to_string(c->p.nvec[l]) + (l + 2 < c->nlevels ? ", " : "");
  j += "], \"prec_fine\": " + std::to_string(int(c->p.prec_fine)) +
       ", \"prec_coarse\": " + std::to_string(int(c->p.prec_coarse)) +
       ", \"seed\": " + std::to_string(c->p.seed) + ", \"records\": [";
  for (size_t i = 0; i < sizes.size(); ++i)
    j += std::to_string(sizes[i]) + (i + 1 < sizes.size() ? ", " : "");
  j += "], \"fnv1a64\": \"" + std::to_string(sum) + "\"}\n";
  return j;
}

}  // namespace

mg_status mg_save(mg_ctx* c, const char* path) {
  return guarded(c, [&] {
    GB_REQUIRE(path, MG_ERR_ARG, "save: null path");
    std::vector<std::vector<unsigned char>> recs;
    for (int l = 0; l + 1 < c->nlevels; ++l) {
      Level& F = c->L[l];
      Level& C = c->L[l + 1];
      GB_REQUIRE(F.have_V && C.have_op, MG_ERR_STATE, "save: setup of every level required");
      const size_t nb = size_t(F.nvec) * F.vec_elems() * 16;
      const size_t lb = size_t(C.g.vol) * 9 * C.nd * C.nd * 16;
      DevBuf tmp;
      tmp.alloc(nb > lb ? nb : lb);
      recs.emplace_back(nb);
      nullvecs_export(c, l, tmp.p, 0);
      GB_CHECK(cudaMemcpy(recs.back().data(), tmp.p, nb, cudaMemcpyDeviceToHost));
      recs.emplace_back(lb);
      links_export(c, l + 1, tmp.p, 0);
      GB_CHECK(cudaMemcpy(recs.back().data(), tmp.p, lb, cudaMemcpyDeviceToHost));
    }
    uint64_t sum = 1469598103934665603ull;
    std::vector<size_t> sizes;
    for (auto& r : recs) {
      sum = fnv1a(r.data(), r.size(), sum);
      sizes.push_back(r.size());
    }
    FILE* f = std::fopen(path, "wb");
    GB_REQUIRE(f, MG_ERR_ARG, "save: cannot open the file");
    const std::string h = header_json(c, sizes, sum);
    bool ok = std::fwrite(h.data(), 1, h.size(), f) == h.size();
    for (auto& r : recs) ok = ok && std::fwrite(r.data(), 1, r.size(), f) == r.size();
    ok = (std::fclose(f) == 0) && ok;
    GB_REQUIRE(ok, MG_ERR_ARG, "save: write failed");
  });
}

mg_status mg_load(mg_ctx* c, const char* path) {
  return guarded(c, [&] {
    GB_REQUIRE(path, MG_ERR_ARG, "load: null path");
    FILE* f = std::fopen(path, "rb");
    GB_REQUIRE(f, MG_ERR_ARG, "load: cannot open the file");
    std::string h;
    for (int ch; (ch = std::fgetc(f)) != EOF && ch != '\n';) h.push_back(char(ch));
    std::vector<size_t> want;
    for (int l = 0; l + 1 < c->nlevels; ++l) {
      want.push_back(size_t(c->L[l].nvec) * c->L[l].vec_elems() * 16);
      const Level& C = c->L[l + 1];
      want.push_back(size_t(C.g.vol) * 9 * C.nd * C.nd * 16);
    }
    // the header must describe this context (lattice, levels, blocks, nvec,
    // precisions; the seed may differ): compare with the one it would write
    const std::string key_seed = ", \"seed\": ", key_sum = ", \"fnv1a64\": \"";
    const std::string key_rec = "\"records\": [";
    const std::string mine = header_json(c, want, 0);
    const size_t cut = mine.find(key_seed), at = h.find(key_sum);
    const size_t r0 = mine.find(key_rec) + key_rec.size();
    const std::string records = key_rec + mine.substr(r0, mine.find(']', r0) + 1 - r0);
    bool match = at != std::string::npos && h.size() > at + key_sum.size() + 2 &&
                 h.compare(0, cut, mine, 0, cut) == 0 && h.find(records) != std::string::npos;
    uint64_t sum_file = 0;
    if (match) {
      const std::string digits = h.substr(at + key_sum.size(), h.size() - at - key_sum.size() - 2);
      match = !digits.empty() && digits.find_first_not_of("0123456789") == std::string::npos;
      if (match) sum_file = std::strtoull(digits.c_str(), nullptr, 10);
    }
    if (!match) std::fclose(f);
    GB_REQUIRE(match, MG_ERR_ARG, "load: file does not match the context's lattice and setup");
    std::vector<std::vector<unsigned char>> recs;
    uint64_t sum = 1469598103934665603ull;
    bool ok = true;
    for (size_t n : want) {
      recs.emplace_back(n);
      ok = ok && std::fread(recs.back().data(), 1, n, f) == n;
      if (ok) sum = fnv1a(recs.back().data(), n, sum);
    }
    std::fclose(f);
    GB_REQUIRE(ok, MG_ERR_ARG, "load: file truncated");
    GB_REQUIRE(sum == sum_file, MG_ERR_ARG, "load: checksum mismatch");
    for (int l = 0; l + 1 < c->nlevels; ++l) {
      Level& F = c->L[l];
      const auto& nvr = recs[2 * l];
      F.raw.alloc(nvr.size());
      GB_CHECK(cudaMemcpy(F.raw.p, nvr.data(), nvr.size(), cudaMemcpyHostToDevice));
      F.have_raw = true;
      block_orthonormalise(c, l, 0);
      const auto& lr = recs[2 * l + 1];
      DevBuf tmp;
      tmp.alloc(lr.size());
      GB_CHECK(cudaMemcpy(tmp.p, lr.data(), lr.size(), cudaMemcpyHostToDevice));
      links_import(c, l + 1, tmp.p, 0);
      if (c->p.red_black) schur_prepare(c, l + 1, 0);
      GB_CHECK(cudaDeviceSynchronize());
    }
  });
}

mg_status mg_get_coarse_links(mg_ctx* c, int level, void* dst, size_t bytes, void* stream) {
  return guarded(c, [&] {
    check_level(c, level, 1, c->nlevels - 1);
    Level& L = c->L[level];
    GB_REQUIRE(dst && bytes == size_t(L.g.vol) * 9 * L.nd * L.nd * 16, MG_ERR_ARG,
               "get_coarse_links: size mismatch");
    links_export(c, level, dst, S(stream));
  });
}

mg_status mg_set_coarse_links(mg_ctx* c, int level, const void* src, size_t bytes, void* stream) {
  return guarded(c, [&] {
    check_level(c, level, 1, c->nlevels - 1);
    Level& L = c->L[level];
    GB_REQUIRE(src && bytes == size_t(L.g.vol) * 9 * L.nd * L.nd * 16, MG_ERR_ARG,
               "set_coarse_links: size mismatch");
    links_import(c, level, src, S(stream));
    if (c->p.red_black) schur_prepare(c, level, S(stream));
  });
}

mg_status mg_level_info(mg_ctx* c, int level, int dims[4], int* volume, int* ndof, int* vprec) {
  return guarded(c, [&] {
    check_level(c, level, 0, c->nlevels - 1);
    Level& L = c->L[level];
    if (dims)
      for (int m = 0; m < 4; ++m) dims[m] = L.g.L[m];
    if (volume) *volume = L.g.vol;
    if (ndof) *ndof = L.nd;
    if (vprec) *vprec = int(L.vprec);
  });
}

mg_status mg_gauge_compression(mg_ctx* c, int* forms, double* max_dev8, double* rms_dev8) {
  return guarded(c, [&] {
    const Level& L = c->L[0];
    if (forms) *forms = (L.gauge12_ok ? 1 : 0) | (L.gauge8_ok ? 2 : 0);
    if (max_dev8) *max_dev8 = L.gauge8_maxdev;
    if (rms_dev8) *rms_dev8 = L.gauge8_rmsdev;
  });
}

mg_status mg_profile_enable(mg_ctx* c, int on) {
  return guarded(c, [&] { c->prof.on = on != 0; });
}

mg_status mg_profile_reset(mg_ctx* c) {
  return guarded(c, [&] {
    for (auto& r : c->prof.recs) GB_CHECK(cudaEventSynchronize(r.stop));
    c->prof.clear();
  });
}

mg_status mg_profile_query(mg_ctx* c, const char* name, int level, int* launches, double* ms,
                           double* bytes, double* flops) {
  return guarded(c, [&] {
    GB_REQUIRE(name, MG_ERR_ARG, "profile_query: null name");
    int n = 0;
    double t = 0, b = 0, f = 0;
    for (auto& r : c->prof.recs) {
      if (r.name != name || (level >= 0 && r.level != level)) continue;
      GB_CHECK(cudaEventSynchronize(r.stop));
      float e = 0.f;
      GB_CHECK(cudaEventElapsedTime(&e, r.start, r.stop));
      ++n;
      t += e;
      b += r.bytes;
      f += r.flops;
    }
    if (launches) *launches = n;
    if (ms) *ms = t;
    if (bytes) *bytes = b;
    if (flops) *flops = f;
  });
}

mg_status mg_set_setup_sweeps(mg_ctx* c, int sweeps) {
  return guarded(c, [&] {
    GB_REQUIRE(sweeps >= 0 && sweeps <= 100000, MG_ERR_ARG, "setup sweeps out of range");
    c->p.setup_sweeps = sweeps;
  });
}

mg_status mg_device_status(mg_ctx* c, void* stream) {
  return guarded(c, [&] {
    int h[2] = {0, 0};
    GB_CHECK(cudaMemcpyAsync(h, c->status.p, sizeof(h), cudaMemcpyDeviceToHost, S(stream)));
    GB_CHECK(cudaStreamSynchronize(S(stream)));
    if (h[1]) {
      GB_CHECK(cudaMemsetAsync(c->status.as<int>() + 1, 0, sizeof(int), S(stream)));
      GB_CHECK(cudaStreamSynchronize(S(stream)));
      throw Error(MG_ERR_TIMEOUT, "a bounded device wait timed out (tensor-core coarse apply, tiled fine operator or Galerkin build)");
    }
  });
}

mg_status mg_inner_product(mg_ctx* c, int level, const void* a, const void* b, mg_prec prec,
                           int fp64, double* out, void* stream) {
  return guarded(c, [&] {
    check_level(c, level, 0, c->nlevels - 1);
    GB_REQUIRE(a && b && out, MG_ERR_ARG, "inner_product: null pointer");
    GB_REQUIRE(prec == MG_F32 || prec == MG_F64, MG_ERR_ARG,
               "inner_product: FP32 or FP64 vectors");
    const size_t n = c->L[level].vec_elems();
    Vec va{const_cast<void*>(a), prec, n, 1}, vb{const_cast<void*>(b), prec, n, 1};
    const int slot = level * 8 + 7;  // the solvers use slots 0..5 of each level
    // the kernels GCR uses: norms by blas_dot, products of two vectors by
    // the block Gram-Schmidt reduction
    if (a == b)
      blas_dot(c, va, va, slot, S(stream), fp64 != 0);
    else
      blas_dot_multi(c, &va, 1, vb, slot, S(stream), fp64 != 0);
    blas_read_slot_c(c, slot, out, S(stream));
  });
}

mg_status mg_inject_fault(mg_ctx* c, const char* what, int count) {
  return guarded(c, [&] {
    GB_REQUIRE(what && count >= 0 && count <= 1000, MG_ERR_ARG, "inject_fault: bad arguments");
    GB_REQUIRE(std::string(what) == "coarse_mma_wait", MG_ERR_ARG,
               "inject_fault: unknown fault (known: coarse_mma_wait)");
    c->inject_mma_stall = count;
  });
}

long long mg_launch_count(mg_ctx* c) { return c ? c->launches : 0; }

const char* mg_status_string(mg_status s) {
  switch (s) {
    case MG_OK: return "ok";
    case MG_ERR_ARG: return "invalid argument";
    case MG_ERR_CUDA: return "CUDA error";
    case MG_ERR_OOM: return "out of device memory";
    case MG_ERR_STATE: return "call out of order";
    case MG_ERR_NOT_CONVERGED: return "solver did not converge";
    case MG_ERR_NUMERICAL: return "numerical breakdown";
    case MG_ERR_TIMEOUT: return "device wait timed out";
    case MG_ERR_RANK: return "rank-deficient null-vector block";
  }
  return "unknown status";
}

const char* mg_last_error(mg_ctx* c) { return c ? c->err.c_str() : g_last_error.c_str(); }

}  // extern "C"
