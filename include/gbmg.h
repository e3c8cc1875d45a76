/*
 * gbmg.h -- C ABI of libgbmg.so: adaptive-multigrid coarse-grid operator
 * (stencil apply and Galerkin construction) for the Wilson-clover Dirac
 * matrix, on one NVIDIA GB300 (sm_103a).
 *
 * Method: Clark et al., "Accelerating Lattice QCD Multigrid on GPUs Using
 * Fine-Grained Parallelization" (SC16).  Eq. (1) is the linear system
 * M x = b, Eq. (2) the fine Wilson-clover matrix, Sec. 3.4 the adaptive
 * setup (null vectors, aggregates, chiral split, block QR, Galerkin
 * product), Eq. (3) the coarse operator, Sec. 6 the coarse stencil
 * kernel, Sec. 6.6 the transfer operators, Sec. 7.1 the K-cycle solver.
 *
 * Conventions shared by every call
 * --------------------------------
 * Lattice site index  s = x + Lx*(y + Ly*(z + Lz*t)), directions mu = 0..3
 *                     for x, y, z, t; periodic, optionally antiperiodic in t
 *                     for the fine fermion field.
 * Fine spinor         [site][spin 4][colour 3] complex   (12 complex / site)
 *                     in the DeGrand-Rossi chiral basis, gamma_5 =
 *                     diag(1, 1, -1, -1): spins {0,1} = chirality 0.
 * Coarse spinor       [site][dof] complex, dof = s*Nv + c, s the chirality
 *                     (Sec. 6.2), 2*Nv dofs per site.
 * Multi-RHS spinor    [site][dof][rhs] complex (mg_coarse_apply, nrhs > 1);
 *                     the multi-RHS solve and fine apply take the vectors
 *                     back to back instead, [rhs][site][dof].
 * Complex numbers     interleaved (re, im).
 * Gauge field         [mu][site][3][3] complex double (row-major SU(3)).
 * Coarse links        [site][slot 0..8][row][col] complex double, the
 *                     nine blocks of Eq. (3): slot 0 = X (the dense site-
 *                     diagonal block), slot 1+2mu = Y_{+mu} acting on
 *                     x(site + mu), slot 2+2mu = Y_{-mu} acting on
 *                     x(site - mu):  y(s) = sum_slot L[s][slot] x(nbr).
 * Null vectors        [vec][site][dof] complex double.
 *
 * Vector precision.  Level l works in "vector precision" F64 when its
 * operator precision is MG_F64 and F32 otherwise (also for the 16-bit
 * link forms, whose arithmetic accumulates in FP32).  Vector arguments of
 * mg_apply / mg_coarse_apply / mg_restrict / mg_prolong /
 * mg_wilson_clover_apply are complex numbers in that precision
 * (complex128 or complex64).  mg_gcr_solve always takes complex128.
 *
 * Memory.  Pointers named *_dev are device pointers owned by the caller
 * (e.g. PyTorch tensors); the library reads or writes them only inside the
 * call, stream-ordered on `stream` (a cudaStream_t passed as void*; NULL is
 * the legacy default stream).  Everything the context holds (copies of the
 * gauge field, clover term, null vectors, coarse links, solver workspace)
 * is allocated by the library and freed by mg_destroy.
 *
 * Errors.  Every call returns an mg_status; mg_last_error(ctx) gives a
 * human-readable reason.  No call exits, traps or falls back to the CPU.
 */
#ifndef GBMG_H
#define GBMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MG_MAX_LEVELS 4
#define MG_MAX_NRHS 32   /* right-hand sides of one mg_gcr_solve_multi call */

typedef enum {
  MG_OK = 0,
  MG_ERR_ARG = -1,           /* invalid argument (sizes, pointers, levels)      */
  MG_ERR_CUDA = -2,          /* a CUDA runtime call failed                       */
  MG_ERR_OOM = -3,           /* device allocation failed                         */
  MG_ERR_STATE = -4,         /* call out of order (e.g. apply before build)      */
  MG_ERR_NOT_CONVERGED = -5, /* solver hit maxiter; stats are still filled       */
  MG_ERR_NUMERICAL = -6,     /* NaN/Inf or a zero denominator in a solver        */
  MG_ERR_TIMEOUT = -7,       /* a bounded device wait gave up                    */
  MG_ERR_RANK = -8           /* a null-vector aggregate block is rank deficient  */
} mg_status;

/* MG_I16: 16-bit fixed point (re, im) pairs, value = site scale * q / 32767,
 * the paper's "half" storage (Sec. 4).                                 */
typedef enum { MG_F64 = 0, MG_F32 = 1, MG_BF16 = 2, MG_F16 = 3, MG_I16 = 4 } mg_prec;

typedef struct mg_ctx mg_ctx;

/* Problem and solver parameters.  Eq. (2): dims, mass m, csw, boundary;
 * Sec. 3.4: blocks (aggregate extents), nvec (null vectors), setup
 * sweeps; Sec. 7.1: GCR Krylov size, MR smoother, inner tolerances.      */
typedef struct {
  int dims[4];                      /* fine lattice extents Lx, Ly, Lz, Lt          */
  int t_antiperiodic;               /* 1: antiperiodic fermion boundary in t        */
  double mass;                      /* m of Eq. (2)                                  */
  double csw;                       /* clover coefficient of A_x                    */
  int nlevels;                      /* 2..MG_MAX_LEVELS (fine level included)       */
  int block[MG_MAX_LEVELS][4];      /* aggregate extents of coarsening l -> l+1     */
  int nvec[MG_MAX_LEVELS];          /* null vectors of coarsening l -> l+1          */
  int setup_sweeps;                 /* minimal-residual sweeps on M x = 0           */
  uint64_t seed;                    /* device Gaussian x0 when none is passed       */
  mg_prec prec_fine;                /* MG_F64 or MG_F32                             */
  mg_prec prec_coarse;              /* MG_F64, MG_F32, MG_BF16, MG_F16, MG_I16 links */
  int mr_iters;                     /* MR pre- and post-smoothing steps (4)         */
  double mr_omega;                  /* MR relaxation (1.0)                          */
  int gcr_nkrylov;                  /* GCR Krylov space size (10)                   */
  double inner_tol;                 /* intermediate-level GCR tolerance (0.25)      */
  int inner_maxiter;                /* intermediate-level GCR iteration cap (10)    */
  double coarse_tol;                /* coarsest-level GCR tolerance (0.1)           */
  int coarse_maxiter;               /* coarsest-level GCR iteration cap (100)       */
  int link_slots;                   /* coarse link store: 9 (all blocks of Eq. 3) or
                                       5 (X and Y_{+mu}; Y_{-mu}(x) is rebuilt as
                                       g5 Y_{+mu}(x-mu)^dag g5 inside the apply) */
  int red_black;                    /* 1: red-black (Schur complement) preconditioning
                                       on every level with all extents even (Secs.
                                       3.3, 7.1): MR smoothing on the Schur system
                                       S = A_o - H_oe A_e^-1 H_eo and the coarsest
                                       GCR on S; 0: off (default)                  */
  mg_prec prec_smoother;            /* fine-level MR smoother storage: MG_F32 (the
                                       fine level's own) or MG_BF16 (Sec. 7.1: the
                                       finest smoother in 16 bits; vectors and a copy
                                       of the operator in BF16, FP32 arithmetic;
                                       needs an FP32 fine level)                   */
} mg_params;

typedef struct {
  int iters;                        /* outer GCR steps                              */
  int restarts;                     /* true-residual recomputations                 */
  int level_iters[MG_MAX_LEVELS];   /* GCR steps summed per level (0 = outer)       */
  double true_residual;             /* |b - M x| / |b| in FP64 at return            */
  double seconds;                   /* wall time of the call                        */
  int history_len;                  /* entries written to history                   */
  double history[512];              /* |r_k| / |b| after each outer step            */
} mg_solve_stats;

/* Fill *p with the defaults listed in the comments of mg_params (dims and
 * blocks are zero and must be set).                                        */
void mg_default_params(mg_params* p);

/* Create a context.  gauge_dev: [4][V][3][3] complex double, read once and
 * copied (with the t boundary sign folded into the last time slice) into
 * the fine operator, which also computes the clover term A_x on the device.
 * Fails with MG_ERR_ARG if an extent is not divisible by its block.        */
mg_status mg_create(const mg_params* params, const void* gauge_dev, mg_ctx** out);
mg_status mg_destroy(mg_ctx* ctx);

/* Sec. 3.4 steps 1-3 for the coarsening level -> level+1: starting from
 * init_dev ([nvec][V_l][nd_l] complex double; NULL draws Gaussian x0 on the
 * device from params.seed) run setup_sweeps minimal-residual steps on
 * A_l x = 0 in the level's vector precision, normalise every vector, then
 * block-orthonormalise (chiral split, modified Gram-Schmidt done twice,
 * FP64) per aggregate.  MG_ERR_RANK on a rank-deficient block.             */
mg_status mg_setup_nullvecs(mg_ctx* ctx, int level, const void* init_dev, void* stream);

/* Take the raw null vectors from vecs_dev ([nvec][V_l][nd_l] complex
 * double) instead of running the sweeps, then block-orthonormalise.       */
mg_status mg_set_nullvecs(mg_ctx* ctx, int level, const void* vecs_dev, void* stream);

/* Copy null vectors out: kind 0 = raw (after sweeps), 1 = block-
 * orthonormalised (the prolongator columns).  [nvec][V_l][nd_l] complex
 * double; bytes must equal that size.                                      */
mg_status mg_get_nullvecs(mg_ctx* ctx, int level, int kind, void* dst_dev, size_t bytes,
                          void* stream);

/* Sec. 3.4 step 4: Galerkin product P^dag A_l P of level l, stored as the
 * nine blocks of Eq. (3) per coarse site of level l+1 (X and Y_{+-mu}),
 * in prec_coarse.  Requires the null vectors of level l.                   */
mg_status mg_build_coarse(mg_ctx* ctx, int level, void* stream);

/* Eq. (3) on coarse level `level` >= 1:  y = X x + sum_mu Y_{+mu} x(.+mu)
 * + Y_{-mu} x(.-mu).  nrhs = 1: x, y [V][n]; nrhs > 1: [V][n][nrhs].
 * x and y are device arrays in the level's vector precision and must not
 * overlap.                                                                 */
mg_status mg_coarse_apply(mg_ctx* ctx, int level, void* y_dev, const void* x_dev, int nrhs,
                          void* stream);

/* Eq. (3) with nrhs right-hand sides on `count` (1..8) coarse operators of
 * possibly different lattices -- level levels[i] of ctxs[i], all with the
 * same n and 16-bit (BF16/FP16) links -- in ONE persistent tensor-core
 * launch that walks the concatenated site lists.  y[i], x[i]: device arrays
 * [V_i][n][nrhs] complex float, nrhs a multiple of 4 up to 64.  The call
 * enqueues a single kernel with no host-side state, so it can be captured
 * into a CUDA graph (make one uncaptured call first: it tunes the launch).
 * Errors of the bounded device waits go to ctxs[0] (mg_device_status).     */
mg_status mg_coarse_apply_multi(mg_ctx* const* ctxs, const int* levels, void* const* y_dev,
                                const void* const* x_dev, int count, int nrhs, void* stream);

/* The level-l operator on one vector: Eq. (2) for l = 0, Eq. (3) above.    */
mg_status mg_apply(mg_ctx* ctx, int level, void* y_dev, const void* x_dev, void* stream);

/* Eq. (2): out = M in on the fine lattice, vectors in the fine vector
 * precision.                                                               */
mg_status mg_wilson_clover_apply(mg_ctx* ctx, void* out_dev, const void* in_dev, void* stream);

/* The same on nrhs vectors at once, [nrhs][site][12] back to back
 * (1 <= nrhs <= 64); out must not overlap in.  One launch: the links and
 * clover of a site serve all nrhs vectors (the launch policy is autotuned). */
mg_status mg_wilson_clover_apply_multi(mg_ctx* ctx, void* out_dev, const void* in_dev, int nrhs,
                                       void* stream);

/* The operator of the 16-bit fine-level smoother (params.prec_smoother =
 * MG_BF16): out = M in on BF16 complex vectors ([nrhs][site][12] pairs of
 * bfloat16 (re, im)), with the BF16 copy of the links and clover and FP32
 * arithmetic.  MG_ERR_STATE when the context has no 16-bit smoother.      */
mg_status mg_wilson_clover_apply_bf16(mg_ctx* ctx, void* out_dev, const void* in_dev, int nrhs,
                                      void* stream);

/* Sec. 6.6 transfer operators between level l and l+1 (vector precision of
 * each level):  coarse = P^dag fine  (restrict),  fine = P coarse (prolong). */
mg_status mg_restrict(mg_ctx* ctx, int level, void* coarse_dev, const void* fine_dev,
                      void* stream);
mg_status mg_prolong(mg_ctx* ctx, int level, void* fine_dev, const void* coarse_dev,
                     void* stream);

/* Sec. 7.1: flexible GCR on the fine level, preconditioned by the K-cycle,
 * to |b - M x| <= tol |b| (true residual, FP64).  x_dev, b_dev: fine
 * vectors, complex double.  Synchronises `stream` for convergence checks.
 * Returns MG_ERR_NOT_CONVERGED at maxiter (x holds the last iterate).      */
mg_status mg_gcr_solve(mg_ctx* ctx, void* x_dev, const void* b_dev, double tol, int maxiter,
                       mg_solve_stats* stats, void* stream);

/* The same solve for nrhs right-hand sides at once (1 <= nrhs <=
 * MG_MAX_NRHS).  x_dev, b_dev: nrhs fine vectors back to back,
 * [nrhs][site][12] complex double.  Every step of the method runs on all
 * right-hand sides in one batched launch with per-RHS scalars, so the
 * fine links, the prolongators and the coarse links are read once per step
 * for all of them (the coarse applies of FP32 and 16-bit levels run
 * multi-RHS kernels; the 16-bit ones on the tensor cores).  The iteration
 * stops when every right-hand side meets tol.  stats: an array of nrhs
 * records or NULL; record v holds the step at which right-hand side v met
 * tol (iters), its true residual and history; level_iters and seconds are
 * totals of the call.  The solver workspace grows with nrhs (about 30 fine
 * vectors per right-hand side).                                            */
mg_status mg_gcr_solve_multi(mg_ctx* ctx, void* x_dev, const void* b_dev, int nrhs, double tol,
                             int maxiter, mg_solve_stats* stats, void* stream);

/* Red-black preconditioning (Secs. 3.3, 7.1; params.red_black = 1, every
 * extent of the level even): y_o = S x_o with S = A_o - H_oe A_e^-1 H_eo the
 * Schur complement of level l's operator on the odd sites.  Compact parity
 * vectors: the odd site s is entry s >> 1, [nrhs][V/2][ndof] in the level's
 * vector precision.  MG_ERR_STATE if the level has no red-black form.      */
mg_status mg_schur_apply(mg_ctx* ctx, int level, void* y_dev, const void* x_dev, int nrhs,
                         void* stream);

/* Coarse links of level l >= 1 in the external layout (see top), complex
 * double, bytes = V_l * 9 * n_l^2 * 16.  set replaces the operator of the
 * level (for apply-only use), converting to prec_coarse.  With
 * link_slots = 5 the apply uses only slots 0, 1, 3, 5, 7 and rebuilds the
 * backward blocks, so set links should satisfy that relation (Galerkin
 * links do).                                                               */
mg_status mg_get_coarse_links(mg_ctx* ctx, int level, void* dst_dev, size_t bytes, void* stream);
mg_status mg_set_coarse_links(mg_ctx* ctx, int level, const void* src_dev, size_t bytes,
                              void* stream);

/* Geometry of level l: extents, volume, dofs per site, vector precision. */
mg_status mg_level_info(mg_ctx* ctx, int level, int dims[4], int* volume, int* ndof,
                        int* vec_prec);

/* Compressed link forms of the FP32 fine operator (Sec. 4): bit 0 of
 * *forms = the two-row (12-real) form is eligible, bit 1 = the 8-real form
 * (a2, a3, b1 and the phases of a1, c1; the other entries rebuilt from
 * unit rows and columns and det U = 1) is eligible.  *max_dev8 and
 * *rms_dev8: the largest and the root-mean-square |U_rebuilt - U| over the
 * entries of every link, FP32 rebuild against the FP64 field.  The 8-real
 * form is eligible when the root-mean-square is below 1e-6 and the largest
 * below 1e-3 (the rebuild divides by 1 - |a1|^2, which is small on the
 * rare links close to a diagonal matrix); both forms are launch
 * policies of mg_wilson_clover_apply that the autotuner may pick.  Zeros
 * for an FP64 fine level.                                                  */
mg_status mg_gauge_compression(mg_ctx* ctx, int* forms, double* max_dev8, double* rms_dev8);

/* Device-side timing of the library's own kernels.  When enabled, every
 * launch of kernel class `name` ("coarse_apply" for single right-hand
 * sides, "coarse_apply_multi" for nrhs > 1, "wilson_clover", "galerkin",
 * "restrict", "prolong", "block_orth") on level
 * `level` is bracketed by CUDA events on its stream.  query() sums the
 * durations (waiting for them) and the algorithmic bytes and flops the
 * launches moved; level -1 sums all levels.  reset() clears the record.   */
mg_status mg_profile_enable(mg_ctx* ctx, int on);
mg_status mg_profile_reset(mg_ctx* ctx);
mg_status mg_profile_query(mg_ctx* ctx, const char* name, int level, int* launches,
                           double* total_ms, double* bytes, double* flops);

/* Checkpoint of the setup (the setup is amortised over many solves, Sec.
 * 7.1): mg_save writes the block-orthonormal null vectors of every
 * coarsening and the links of every coarse level to `path` (one JSON
 * header line with lattice, blocks, nvec, precisions, seed, record sizes
 * and an FNV-1a 64 checksum, then raw little-endian complex doubles);
 * MG_ERR_STATE unless every level is set up.  mg_load restores them into a
 * context created with the same lattice, blocks, nvec and precisions
 * (MG_ERR_ARG on a mismatch, a short file or a bad checksum): the
 * prolongators are rebuilt from the vectors and the coarse operators taken
 * from the file, so a solve can follow without setup sweeps or Galerkin
 * builds.                                                                  */
mg_status mg_save(mg_ctx* ctx, const char* path);
mg_status mg_load(mg_ctx* ctx, const char* path);

/* Launch-policy autotuner (process-wide).  The first call of a tuned kernel
 * for a shape times its candidate policies and keeps the fastest; keys name
 * the kernel and shape, e.g. "wilson/v<volume>/n<vectors>/c<0|1>".
 * mg_tune_set pins `choice` for `key` (a choice that is not a candidate of
 * a later call is ignored there; choice < 0 removes the entry so the next
 * call tunes again); mg_tune_get returns the entry or -1.  The environment
 * variable GBMG_TUNE=0 turns timing off (first candidate) and
 * GBMG_TUNE_CACHE=<file> keeps choices across processes.  The paper's
 * autotuning of launch parameters (Secs. 4 and 6) is the model.                  */
mg_status mg_tune_set(const char* key, int choice);
int mg_tune_get(const char* key);
/* The candidates that the last tuning of `key` timed, with milliseconds per
 * launch: fills up to `max` entries of choices / ms (either may be NULL) and
 * returns the number of candidates (0 if the key was never tuned in this
 * process, -1 for a NULL key).                                             */
int mg_tune_report(const char* key, int* choices, float* ms, int max);

/* Block orthonormalisation that allocates no device memory.  The paper has
 * no counterpart: this entry point exists for callers that cannot let a
 * library call cudaMalloc -- programs whose device memory belongs to another
 * allocator (e.g. a framework's caching allocator that reserved the device),
 * programs under a fixed device-memory budget, and latency-critical loops
 * that cannot take the implicit synchronisation of cudaMalloc / cudaFree.
 * It computes what mg_set_nullvecs + mg_get_nullvecs(kind 1) compute:
 * vecs_dev [nvec][V][ndof] complex double (V = dims[0]*..*dims[3], ndof even,
 * first half of the dofs = chirality 0) is orthonormalised per aggregate
 * (extents `block`) and chirality into out_dev (same layout, must not
 * overlap vecs_dev).  `bytes` is the size of each of the two arrays and must
 * equal nvec * V * ndof * 16 (MG_ERR_ARG otherwise).  No context is needed;
 * dims and block are host arrays.
 * Workspace: a file-scope device array of 2^21 16-byte complex entries
 * (float-float, 32 MiB) that
 * every GPU loading the library holds until exit; calls with
 * nvec * V * ndof > 2^21, nvec > 64 or an aggregate of more than 24576
 * rows per chirality fail with MG_ERR_ARG before any device work.  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the
 * life of the process; make that first call before any stream capture.  A
 * device reset (cudaDeviceReset) invalidates the kept address: calls after
 * one are not supported.  All calls share the workspace and it keeps the
 * last call's contents: calls that overlap on the GPU (other streams, other
 * host threads) race.  The call synchronises `stream` to read the rank
 * test; MG_ERR_RANK as for mg_set_nullvecs.  Error text: mg_last_error(NULL). */
mg_status mg_block_orthonormalise_noalloc(const void* vecs_dev, void* out_dev, size_t bytes,
                                          const int dims[4], const int block[4], int ndof,
                                          int nvec, void* stream);

/* Number of minimal-residual sweeps the next mg_setup_nullvecs runs (the
 * learned setup starts from proposed vectors and needs fewer).             */
mg_status mg_set_setup_sweeps(mg_ctx* ctx, int sweeps);

/* ---- Learned null-vector proposer.  The paper draws the setup's starting
 * vectors x0 at random (Sec. 3.4 step 1); this addition proposes them with
 * a three-layer network whose layers are nearest-neighbour stencils on the
 * lattice: 72 link features (Re, Im of U_mu(x)) and 8 position features
 * (cos, sin of 2 pi x_mu / L_mu) -> 32 -> 32 (tanh) -> with the 8 position
 * features again -> 24 * nvec outputs = nvec complex 12-component vectors
 * per site.  FP32 parameters, flat order W1[9][32][80], b1[32],
 * W2[9][32][32], b2[32], W3[24 nvec][40], b3[24 nvec].  Training
 * minimises, per aggregate and chirality, 1 - |Q_pred^H Q_target|_F^2 /
 * nvec (the share of the target null space outside the span of the
 * proposed vectors, with a relative ridge), averaged over blocks, with
 * Adam; the loss and its gradient with respect to the outputs are formed in
 * FP64.  Vectors use the null-vector layout [vec][V][12] complex double;
 * the gauge field the mg_create layout.                                    */
typedef struct mg_cnn mg_cnn;
mg_status mg_cnn_create(int nvec, uint64_t seed, mg_cnn** out);
mg_status mg_cnn_destroy(mg_cnn* net);
mg_status mg_cnn_nparams(mg_cnn* net, int* count);
/* parameters (which = 0) or the last gradient (which = 1), FP32, device   */
mg_status mg_cnn_get_params(mg_cnn* net, void* dst_dev, size_t bytes, int which, void* stream);
mg_status mg_cnn_set_params(mg_cnn* net, const void* src_dev, size_t bytes, void* stream);
/* proposed vectors for the lattice `dims` and gauge field gauge_dev       */
mg_status mg_cnn_forward(mg_cnn* net, const int dims[4], const void* gauge_dev, void* vecs_dev,
                         void* stream);
/* loss and gradient against target_dev (block-orthonormal null vectors of
 * the same lattice, aggregates `block`); synchronises when loss != NULL    */
mg_status mg_cnn_loss_grad(mg_cnn* net, const int dims[4], const int block[4],
                           const void* gauge_dev, const void* target_dev, double* loss,
                           void* stream);
/* one Adam step (beta 0.9 / 0.999) with the last gradient                 */
mg_status mg_cnn_adam_step(mg_cnn* net, float lr, void* stream);

/* ---- Domain decomposition of a coarse level with a one-site halo (Sec.
 * 6.5: a coarse spinor halo one site deep on every face, one pack kernel
 * for all dimensions, then the exchange).  The level's lattice is cut into
 * procs[0] x .. x procs[3] equal sub-domains, "ranks" numbered
 * lexicographically (x fastest); rank r owns the sites whose coordinates
 * lie in its block.  Every rank lives on the calling GPU (the exchange is
 * a device-to-device copy into the receiver's own halo buffer), so the
 * multi-GPU data path can be checked on one GPU.
 * Faces: f = 2 mu + s for each mu with procs[mu] > 1.  Send face 2mu holds
 * the rank's sites at local x_mu = 0 and goes to rank r - mu; send face
 * 2mu+1 the sites at x_mu = l_mu - 1, to rank r + mu; recv face f of a
 * rank receives send face f of its neighbour (recv 2mu from r + mu: the
 * +mu partners of the sites at x_mu = l_mu - 1; recv 2mu+1 from r - mu).
 * Face sites are ordered lexicographically over the other three local
 * coordinates; face f starts at site face_offset[f] of the rank's send and
 * recv buffers ([halo_sites][n] complex in the level's vector precision).*/
typedef struct mg_halo mg_halo;

/* Host-only plan of rank `rank` (no GPU is touched): for every face f the
 * rank it sends to and receives from (-1 for an inactive face), its first
 * site and its number of sites.  MG_ERR_ARG if an extent is not a multiple
 * of its rank count or rank is out of range.                               */
mg_status mg_halo_plan(const int dims[4], const int procs[4], int rank, int send_to[8],
                       int recv_from[8], int face_offset[8], int face_sites[8]);
/* Host-only: the local site index of every face site of direction mu,
 * side 0 (x_mu = 0) or 1 (x_mu = l_mu - 1), in face order; `sites` holds
 * vol(local_dims) / local_dims[mu] ints.                                   */
mg_status mg_halo_face_sites(const int local_dims[4], int mu, int side, int* sites);
/* Split the built coarse operator of `level` (1 <= level, n in 16, 32, 48,
 * 64, any link store) into the ranks' link stores and allocate every
 * rank's send and recv buffers (owned by the handle).  Synchronises.      */
mg_status mg_halo_create(mg_ctx* ctx, int level, const int procs[4], mg_halo** out,
                         void* stream);
mg_status mg_halo_destroy(mg_halo* h);
/* Number of ranks, local extents, sites and bytes of one rank's halo.     */
mg_status mg_halo_info(mg_halo* h, int* nranks, int local_dims[4], int* halo_sites,
                       size_t* halo_bytes);
/* to_global = 0: rank r's local vector [V_local][n] from a global one
 * [V][n]; to_global = 1: the reverse (rank r's sites of the global vector
 * are overwritten).  Vector precision of the level.                        */
mg_status mg_halo_scatter(mg_halo* h, int rank, void* local_dev, const void* global_dev,
                          int to_global, void* stream);
/* One kernel: every send face of rank r from its local vector.            */
mg_status mg_halo_pack(mg_halo* h, int rank, const void* local_dev, void* stream);
/* Every rank's send faces into the receivers' recv buffers (one
 * stream-ordered device-to-device copy per face); call after every rank's
 * pack and before any rank's apply.                                        */
mg_status mg_halo_exchange(mg_halo* h, void* stream);
/* Eq. (3) on the sites of rank r: y_local = (A x)_r, hops that leave the
 * sub-domain read the recv buffer.  y_local must not overlap x_local.     */
mg_status mg_halo_apply(mg_halo* h, int rank, void* y_local, const void* x_local,
                        void* stream);
/* Device addresses of rank r's send and recv buffers (for an exchange made
 * by the caller, e.g. between processes).                                 */
mg_status mg_halo_buffers(mg_halo* h, int rank, void** send_dev, void** recv_dev);
/* Kernels the handle has launched.                                         */
long long mg_halo_launch_count(mg_halo* h);

/* Synchronise `stream` and report errors that kernels recorded on the
 * device: MG_ERR_TIMEOUT if a bounded wait inside a kernel (the mbarrier
 * waits of the tensor-core multi-RHS apply, of the tiled fine operator and
 * of the Galerkin build) gave up since the last call; the record is
 * cleared.                                                                 */
mg_status mg_device_status(mg_ctx* ctx, void* stream);

/* out[0] + i out[1] = sum_k conj(a_k) b_k over one vector of `level`
 * (level_volume x level_dof complex numbers in `prec`, MG_F32 or MG_F64,
 * device memory, caller-owned), with the accumulation the solvers use
 * (Sec. 7.1; the same kernels as GCR's norms and Gram-Schmidt
 * coefficients): fp64 != 0 is the outer GCR's orthogonalisation form, FP64
 * accurate (FP32 operands: exact products summed in float-float pairs, the
 * pairs combined in FP64); fp64 = 0 the inner levels' form (FP32 operands:
 * FP32 partial sums combined in FP64).  a == b gives |a|^2.  Synchronises
 * `stream`; not concurrent with other calls on the same context.          */
mg_status mg_inner_product(mg_ctx* ctx, int level, const void* a, const void* b, mg_prec prec,
                           int fp64, double* out, void* stream);

/* Host-side fault injection for tests of the error paths (no fault of the
 * GPU is made).  what = "coarse_mma_wait": the next `count` tensor-core
 * multi-RHS launches of this context (mg_coarse_apply with nrhs > 1 on
 * 16-bit links, or mg_coarse_apply_multi with ctx first) wait, before any
 * MMA, on an mbarrier that nothing arrives at; the wait gives up after its
 * one-second budget, the launch writes no output, and the next
 * mg_device_status returns MG_ERR_TIMEOUT.  MG_ERR_ARG for another name or
 * count outside 0..1000; count = 0 cancels.                               */
mg_status mg_inject_fault(mg_ctx* ctx, const char* what, int count);

/* Measured CUDA-core peak of fused multiply-adds on the current device, in
 * TFLOP/s (2 flops per FMA): prec = MG_F32 or MG_F64.  A kernel of
 * independent FMA chains fills every SM; five launches are timed with CUDA
 * events on `stream` (synchronised).  The roofline denominator of the
 * kernels bound by the FP32 pipe (the Galerkin product) and the FP64 pipe
 * (the block Gram-Schmidt, the FP64 fine operator); the paper has no
 * counterpart.  MG_ERR_ARG for another precision or a null output.         */
mg_status mg_fma_peak(int prec, double* tflops, void* stream);

/* Number of kernels the library has launched since creation.              */
long long mg_launch_count(mg_ctx* ctx);

const char* mg_status_string(mg_status s);
const char* mg_last_error(mg_ctx* ctx);   /* ctx may be NULL (creation errors) */

#ifdef __cplusplus
}
#endif
#endif /* GBMG_H */
