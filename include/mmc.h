/*
 * mmc.h -- C ABI of the GB300 (sm_103a) Multipolynomial Monte Carlo library.
 *
 * The library estimates Tr(Theta M^-1) for the Wilson-Dirac matrix M with the
 * multipolynomial Monte Carlo method of Lashomb, Morgan, Whyte and Wilcox,
 * "Multipolynomial Monte Carlo Trace Estimation" (Lattice 2023):
 *   Sec. 1 (Eq. 1)  the trace and Hutchinson's Z(4)-noise estimator,
 *   Sec. 2 (Eq. 2)  the subtracted estimator,
 *   Sec. 3          GMRES polynomials from Leja-ordered harmonic Ritz values,
 *   Sec. 5          double (composite) polynomials,
 *   Sec. 6          the multilevel telescoping sum and exact (probed) last level,
 *   Sec. 7          deflation of the Monte Carlo levels,
 *   Sec. 8          deflated solves and the acceptance rules for eigenpairs.
 *
 * Conventions shared by every call
 *   - Every call returns MMC_OK (0) or a negative MMC_ERR_* code; nothing
 *     aborts or exits.  mmc_last_error() gives a context-owned message.
 *   - Host arrays are owned by the caller; the library copies what it keeps.
 *   - Device fields are owned by the caller (e.g. torch tensors) and passed as
 *     raw device pointers; the library never frees caller memory.  Internal
 *     work buffers are owned by the context and freed by mmc_destroy().
 *   - Complex numbers are interleaved (re, im) pairs everywhere.
 *   - Lattice: dims = {Lx, Ly, Lz, Lt}; site index s = x + Lx(y + Ly(z + Lz t)).
 *     Canonical host order of a spinor batch: [rhs][t][z][y][x][spin][colour]
 *     complex128; of the gauge field: [mu][t][z][y][x][row][col] complex128,
 *     mu = 0:x, 1:y, 2:z, 3:t.
 *   - Device field layout ("blocked"): [rb][site][c][R] complex, c = 3*spin +
 *     colour, R = mmc_rhs_block(nrhs) right-hand sides per block (at most 8
 *     on a context set by mmc_set_rhs_block_max(ctx, 8)), rb = 0 ..
 *     ceil(nrhs/R)-1; padding RHS slots are kept at zero.  Storage type per
 *     precision: MMC_F64 complex double (16 B), MMC_F32 complex float (8 B),
 *     MMC_BF16 two bfloat16 (4 B).  mmc_field_bytes() gives the size.
 *   - Precision: MMC_F64 computes in FP64; MMC_F32 and MMC_BF16 compute in
 *     FP32 (BF16 is storage only) and accumulate bilinears in FP64.
 *   - Calls taking a cudaStream_t (passed as void*) are asynchronous on that
 *     stream; all others synchronise the context's stream before returning.
 *   - Dirac matrices: chiral basis, gamma_k = [[0,-i s_k],[i s_k,0]],
 *     gamma_4 = [[0,1],[1,0]], gamma_5 = diag(1,1,-1,-1).
 *   - M psi(x) = psi(x) - kappa sum_mu [(1-gamma_mu) U_mu(x) psi(x+mu)
 *                                     + (1+gamma_mu) U_mu(x-mu)^+ psi(x-mu)],
 *     periodic in space, antiperiodic in time when requested.
 *   - Z(4) noise: Philox4x32-10, key (seed mod 2^32, seed >> 32), counter
 *     (site, noise index, level id, tag); spin-colour component c of the site
 *     takes i^((w0 >> 2c) & 3) with w0 the first output word.
 */
#ifndef MMC_H
#define MMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mmc_ctx mmc_ctx;

enum {
  MMC_OK = 0,
  MMC_ERR_ARG = -1,        /* invalid argument (null pointer, size, handle) */
  MMC_ERR_NOMEM = -2,      /* device or host allocation failed */
  MMC_ERR_CUDA = -3,       /* a CUDA runtime call failed */
  MMC_ERR_BREAKDOWN = -4,  /* Arnoldi breakdown (h_{j+1,j} ~ 0) */
  MMC_ERR_NOCONV = -5,     /* a solve or eigen iteration did not converge */
  MMC_ERR_TIMEOUT = -6,    /* a bounded device wait gave up */
  MMC_ERR_NAN = -7,        /* a NaN or Inf appeared */
  MMC_ERR_STATE = -8       /* call out of order (e.g. no gauge field loaded) */
};

enum { MMC_F64 = 0, MMC_F32 = 1, MMC_BF16 = 2 };
enum { MMC_THETA_ONE = 0, MMC_THETA_G4 = 1, MMC_THETA_G5 = 2 };
enum { MMC_EXACT_UNIT = 0, MMC_EXACT_PROBE = 1 };

#define MMC_OP_M (-1)   /* operator argument: M itself */
#define MMC_ZERO (-1)   /* level argument: the zero map */
#define MMC_INV (-2)    /* level argument: M^-1 (deflated, refined solves) */

#define MMC_TAG_NOISE 0x4E4F4953u   /* 'NOIS': Monte Carlo noise */
#define MMC_TAG_GMRES 0x474D5253u   /* 'GMRS': GMRES-polynomial start vector */
#define MMC_TAG_ARNOLDI 0x4445464Cu /* 'DEFL': PP-Arnoldi start vector */

/* Statistics of one Monte Carlo level (Sec. 4, Sec. 6, Sec. 8).
 * Samples x_j = eta_j^H Theta (A_hi - A_lo) eta_j minus the deflated part;
 * var_* are unbiased sample variances, stderr_* = sqrt(var/n);
 * corr = sum_i c_i u_i^H Theta z_i is the exact trace of the deflated part
 * (zero without deflation); value = mean + corr is the level's estimate. */
typedef struct {
  int n;
  int k_deflated;
  double mean_re, mean_im;
  double var_re, var_im, cvar;
  double stderr_re, stderr_im;
  double corr_re, corr_im;
  double value_re, value_im;
  double seconds;
  long long matvecs;       /* single-vector applications of M spent */
} mmc_level_stats;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` for a lattice dims[4] = {Lx,Ly,Lz,Lt}
 * (each >= 2) and a noise seed (Sec. 1: Z(4) noise).  *ctx is set on success. */
int mmc_create(mmc_ctx** ctx, const int dims[4], uint64_t seed, int device);
/* Free every device and host resource of the context.  NULL is accepted. */
int mmc_destroy(mmc_ctx* ctx);
/* Message describing the last error of this context (never NULL). */
const char* mmc_last_error(const mmc_ctx* ctx);
/* Noise seed of the context; may be changed between calls. */
int mmc_set_seed(mmc_ctx* ctx, uint64_t seed);

/* RHS block R used for a batch of nrhs vectors (power of two, <= 16) on a
 * context with the default layout (see mmc_set_rhs_block_max). */
int mmc_rhs_block(int nrhs);
/* Bytes of a device field of nrhs vectors in precision prec (blocked layout). */
size_t mmc_field_bytes(const mmc_ctx* ctx, int nrhs, int prec);

/* ------------------------------------------------------------- operator */

/* Load the gauge field (host, canonical complex128 [4][t][z][y][x][3][3]) and the
 * hopping parameter kappa (Sec. 4); t_antiperiodic != 0 selects antiperiodic time.
 * Keeps FP64 and FP32 device copies.  Invalidates polynomials and eigenpairs. */
int mmc_load_gauge(mmc_ctx* ctx, const double* U, double kappa, int t_antiperiodic);

/* Convert nrhs host vectors (canonical order, complex128, rhs outermost) into a
 * device field of precision prec (blocked layout), and back.  Synchronous. */
int mmc_pack(mmc_ctx* ctx, const double* host, int nrhs, int prec, void* field);
int mmc_unpack(mmc_ctx* ctx, const void* field, int nrhs, int prec, double* host);

/* dst = src element by element between storage precisions (rounding to nearest),
 * nrhs vectors in the blocked layout of both (not part of the paper: data
 * movement, e.g. FP64 solutions into an FP32 training set).  src != dst. */
int mmc_convert(mmc_ctx* ctx, const void* src, int src_prec, void* dst, int dst_prec, int nrhs, void* stream);

/* y = M x (dagger = 0) or y = M^+ x (dagger = 1) for nrhs vectors of precision
 * prec (Sec. 1, Eq. 1's Wilson-Dirac matrix).  x and y must not overlap. */
int mmc_apply_M(mmc_ctx* ctx, const void* x, void* y, int nrhs, int prec, int dagger,
                void* stream);

/* Fill a field with nrhs Z(4) noise vectors: vector r has noise index first + r,
 * level id `level` and tag `tag` (Sec. 1, "Z(4) noise"). */
int mmc_noise(mmc_ctx* ctx, uint32_t level, uint32_t first, uint32_t tag, int nrhs, int prec,
              void* field, void* stream);

/* mmc_noise without any device allocation, for callers whose device memory is
 * owned by another allocator (a framework's caching allocator holding the GPU's
 * memory, a service with a fixed memory budget that forbids allocation once it
 * runs).  The paper has no counterpart: this is an operational variant.  Same
 * arguments and output as mmc_noise; nrhs padded to the rhs block must not
 * exceed 4096 (MMC_ERR_ARG otherwise).  The (level, index) table lives in one
 * static device array per device (32 KB, held until the process exits) shared
 * by every call: calls that overlap on the GPU race on it, so the call
 * synchronises its stream before returning.  The first call on a device looks
 * up the array's device address (a runtime call that allocates nothing) and
 * should come before any stream capture.  Never calls cudaMalloc or cudaFree. */
int mmc_noise_noalloc(mmc_ctx* ctx, uint32_t level, uint32_t first, uint32_t tag, int nrhs, int prec,
                      void* field, void* stream);

/* ----------------------------------------------------------- polynomials */

/* One GMRES(m) cycle (Sec. 3) of op (MMC_OP_M, or phi_h(M) = M p_h(M) for a single
 * polynomial handle h) from the normalised Z(4) start vector (noise index 0, level
 * 0, tag MMC_TAG_GMRES), Arnoldi with CGS2 in FP64 on the device; harmonic Ritz
 * values and Leja ordering in FP64 on the host.  theta_out (2m doubles, may be
 * NULL) receives the Leja-ordered values; *handle the new polynomial
 * (MMC_OP_M: p of degree m-1 in M; else p_out in phi_h(M)). */
int mmc_gmres_poly(mmc_ctx* ctx, int m, int op_handle, double* theta_out, int* handle);

/* The GMRES(m) cycle of mmc_gmres_poly from the start vector with its components
 * along the context's deflation eigenvectors removed, b <- b - Z (U^H b)
 * (mmc_deflate or mmc_set_deflation first; MMC_ERR_STATE without eigenpairs).
 * Reading of the paper's deflated double polynomial (abstract, Sec. 7, Sec. 9:
 * named, mechanism not given): with op_handle = p_in, the outer polynomial need
 * not place roots near phi_in at the deflated eigenvalues, which the levels
 * treat exactly (mmc_trace_level with deflate = 1, also for hi = MMC_INV), so
 * the same outer degree serves the rest of the spectrum. */
int mmc_gmres_poly_deflated(mmc_ctx* ctx, int m, int op_handle, double* theta_out, int* handle);

/* Register a polynomial given by m Leja-ordered roots theta (2m doubles), p of
 * degree m-1 with pi(a) = prod (1 - a/theta_i) = 1 - a p(a) (Sec. 3). */
int mmc_poly_from_roots(mmc_ctx* ctx, int m, const double* theta, int* handle);

/* Compose the double polynomial p_double(M) = p_in(M) p_out(phi_in(M)) (Sec. 5)
 * from a single polynomial h_in in M and a polynomial h_out in phi_in(M). */
int mmc_poly_double(mmc_ctx* ctx, int h_in, int h_out, int* handle);

/* Number of M applications one vector needs for p_h (degree of p_h). */
int mmc_poly_degree(const mmc_ctx* ctx, int handle);

/* Scalar values p_h(alpha_j) for n complex points (2n doubles in and out). */
int mmc_poly_eval(const mmc_ctx* ctx, int handle, int n, const double* alpha, double* out);

/* y = p_h(M) x for nrhs vectors of precision prec (Sec. 3, Sec. 5): the Leja
 * recurrence, one fused stencil+update kernel per degree.  x, y must differ. */
int mmc_apply_poly(mmc_ctx* ctx, int handle, const void* x, void* y, int nrhs, int prec,
                   void* stream);

/* ------------------------------------------------------------- deflation */

/* PP-Arnoldi (Sec. 7): m_arnoldi FP64 Arnoldi steps on phi_h(M) = M p_h(M)
 * (poly_handle a single polynomial; MMC_OP_M for M itself) from a Z(4) start
 * vector (tag MMC_TAG_ARNOLDI); every Ritz vector z of phi is tested against M
 * (lambda = z^H M z, accepted if ||M z - lambda z|| < tol_accept, Sec. 8: 1e-3);
 * the accepted ones of smallest |lambda|, at most k, are kept with left vectors
 * u_i = gamma5 z_j (lambda_j = conj lambda_i; |Im| < 2e-4 counts as real;
 * equal eigenvalues take distinct partners; mmc_deflation_pairs) and U^H Z = I.
 * While the overlap W^H Z of the kept vectors is singular the pair of largest
 * |lambda| is dropped, and while a column of its inverse (the size of a left
 * vector u_i, which the deflated samples carry) has norm above the bound of
 * mmc_set_deflation_bound (100) the pair with the largest one is dropped; each
 * drop takes the gamma5 partner along (mmc_deflation_condition;
 * MMC_ERR_BREAKDOWN if none is left).  lambda_out (2k doubles, may be
 * NULL) receives the eigenvalues of the kept pairs. */
int mmc_deflate(mmc_ctx* ctx, int k, int poly_handle, int m_arnoldi, double tol_accept,
                double* lambda_out, int* k_accepted);

/* Bound of mmc_deflate's column-norm rule: pairs are dropped while a left vector
 * u_i (a column of (W^H Z)^{-H}, unit w) has norm above max_u (default 100; a
 * reading, not the paper's: it bounds the variance the deflated samples carry).
 * MMC_ERR_ARG unless max_u > 0. */
int mmc_set_deflation_bound(mmc_ctx* ctx, double max_u);

/* Replace the deflation data by k caller-given eigenpairs (Sec. 7): lambda (2k
 * doubles), right vectors Z and left vectors U (k vectors each, canonical host
 * order, complex128), with U^H Z = I expected (not checked).  For a deflation
 * space from elsewhere, or one saved by mmc_get_deflation (checkpoint). */
int mmc_set_deflation(mmc_ctx* ctx, int k, const double* lambda, const double* Z, const double* U);
/* Copy the current deflation data out (any pointer may be NULL; *k always set). */
int mmc_get_deflation(mmc_ctx* ctx, int* k, double* lambda, double* Z, double* U);
/* FP32 and BF16 levels project noise on the deflation vectors with tcgen05 tensor cores
 * (one BF16 GEMM, FP32 accumulation, k <= 128) when enabled (default), from BF16
 * copies of Theta z_i and u_i that also give the exact correction; otherwise on
 * CUDA cores from FP32 copies. */
int mmc_set_tensor_projections(mmc_ctx* ctx, int enable);

/* ---------------------------------------------------------------- solves */

/* Solve M x = b for nrhs FP64 fields (Sec. 1: the solves of Hutchinson's method;
 * Sec. 8: deflated, polynomial-preconditioned GMRES).  Outer loop in FP64:
 * r = b - M x, deflated correction x += Z Lambda^-1 U^H r, stop when
 * ||r|| <= rel_tol ||b|| per vector; inner right-preconditioned FGMRES(m_inner)
 * in precision prec_inner (MMC_F32 or MMC_BF16 storage with FP32 arithmetic;
 * MMC_F64 for the plain FP64 form) with
 * preconditioner p_h(M) (precond_handle, or MMC_ZERO for none).  The FP64 form
 * runs one FGMRES cycle per FP64 residual; with FP32/BF16 inner storage the
 * inner solve restarts FGMRES(m_inner) from its own FP32 residual r - M e
 * (deflated at every restart) for up to 8 cycles, until each vector's inner
 * residual is 3e-2 of its FP64 residual (or what rel_tol still needs) or stops
 * falling by 10% a cycle, so that one FP64 residual serves several cycles
 * (mmc_set_solve_refinement).
 * max_outer bounds the FP64 residuals.  x is the initial guess on entry.
 * *iters receives inner iterations (all cycles), relres_out (nrhs, may be
 * NULL) the final relative residuals. */
int mmc_solve(mmc_ctx* ctx, const void* b, void* x, int nrhs, double rel_tol, int precond_handle,
              int prec_inner, int m_inner, int max_outer, int* iters, double* relres_out);

/* ----------------------------------------------------------- estimators */

/* One Monte Carlo level (Eq. 2, Sec. 6): n_noise Z(4) vectors (noise indices
 * first_noise.., level id `level`), samples eta^H Theta (A_hi - A_lo) eta with
 * hi in {MMC_INV, polynomial handle}, lo in {polynomial handle, MMC_ZERO}.
 * deflate != 0 (polynomial operands, or hi = MMC_INV) subtracts
 * sum_i c_i (eta^H Theta z_i)(u_i^H eta) with c_i = p_hi(lambda_i) - p_lo(lambda_i)
 * (1/lambda_i in place of p_hi for MMC_INV) and reports the exact correction
 * (Sec. 7; for MMC_INV the deflated top level that goes with a deflated double
 * polynomial, see mmc_gmres_poly_deflated).  prec: storage of the polynomial chains.  For hi = MMC_INV the
 * solves use rel_tol 1e-10, preconditioner `precond` and FGMRES(m) with m from
 * mmc_set_solve_params (default 48), with an
 * FP32 inner solve, or FP64 throughout when prec = MMC_F64.
 * samples_out (2 n_noise doubles, may be NULL) receives the samples. */
int mmc_trace_level(mmc_ctx* ctx, int hi, int lo, int theta_op, int deflate, int n_noise,
                    uint32_t first_noise, uint32_t level, int prec, int precond,
                    mmc_level_stats* out, double* samples_out);

/* n_levels polynomial levels in one batch (Eq. 2, Sec. 6; the multilevel batch of
 * Sec. 7 and Sec. 8, whose levels have uneven noise counts and degrees): level l has
 * operands hi[l] (polynomial handle) and lo[l] (polynomial handle or MMC_ZERO),
 * n_noise[l] Z(4) vectors with noise indices first_noise[l].. of level id level[l].
 * Each operand gets its own slot of rhs blocks holding its level's noise, and every
 * single polynomial in M of degree >= 1 runs in one step chain over all slots: one
 * launch per degree up to the highest, each rhs block stopping after its own
 * polynomial's degree.  Double polynomials and degree-0 operands run on their slots
 * afterwards.  Samples, deflation (deflate != 0) and statistics are exactly those of
 * mmc_trace_level on the same noises (up to the summation order of the bilinears);
 * out[l].seconds is the level's share of the batch's time (the shared chain by rhs
 * steps, the noise by slots) plus its own double-polynomial and deflation time.
 * samples_out (may be NULL) holds n_levels pointers, each NULL or to 2 n_noise[l]
 * doubles.  Device memory: three fields of sum_l (slots of level l) rhs.  Errors:
 * MMC_ERR_ARG for MMC_INV or network operands (use mmc_trace_level), counts < 1 or
 * other bad arguments; those of mmc_trace_level. */
int mmc_trace_levels(mmc_ctx* ctx, int n_levels, const int* hi, const int* lo, const int* n_noise,
                     const uint32_t* first_noise, const uint32_t* level, int theta_op, int deflate, int prec,
                     mmc_level_stats* out, double* const* samples_out);

/* One level of a multilevel estimate (see mmc_estimate). */
typedef struct {
  int hi, lo;          /* level operands, as in mmc_trace_level */
  int deflate;         /* as in mmc_trace_level */
  uint32_t level;      /* level id (its noise stream) */
  int n_first;         /* noises before the first check (>= 2) */
  int n_check;         /* noises added between checks (>= 1) */
  int n_max;           /* most noises the level may use (>= n_first) */
} mmc_level_spec;

enum { MMC_ALLOC_EQUAL = 0, MMC_ALLOC_COST = 1 };

/* Multilevel Monte Carlo estimate with adaptive noise counts (Sec. 8: each
 * level's standard error is checked after a first batch of noises and again
 * after every few more; Sec. 9: cost-optimal allocation as the refinement).
 * Every level runs mmc_trace_level on consecutive noise indices first_noise,
 * first_noise + 1, ... of its level id, so the samples do not depend on the
 * batching.  alloc = MMC_ALLOC_EQUAL: level l stops at the first check where
 * its standard error is at most eps / sqrt(n_levels) (or at n_max).
 * alloc = MMC_ALLOC_COST: after the first batches, repeatedly set the targets
 * N_l = ceil(eps^-2 sqrt(V_l / C_l) sum_k sqrt(V_k C_k)) from the sample
 * variances V_l and per-sample costs C_l (cost[l] if cost != NULL, else the
 * matvecs spent per sample so far), give each level below its target the
 * shortfall rounded up to a multiple of n_check (capped at n_max), until no
 * level grows.  Variances are of the real part (imaginary for
 * MMC_THETA_G4).  out[n_levels] receives each level's statistics over all its
 * samples; total[2] (may be NULL) the sum of the level values and the
 * combined standard error sqrt(sum_l V_l / N_l).  The exact last level
 * (mmc_trace_exact) is not included.  Errors: those of mmc_trace_level;
 * MMC_ERR_ARG for bad counts, eps <= 0 or non-positive costs. */
int mmc_estimate(mmc_ctx* ctx, int n_levels, const mmc_level_spec* levels, int theta_op, int prec,
                 int precond, double eps, int alloc, const double* cost, uint32_t first_noise,
                 mmc_level_stats* out, double* total);

/* Exact Tr(Theta p_h(M)) (Sec. 6, last level): method MMC_EXACT_UNIT sums all 12V
 * unit vectors; MMC_EXACT_PROBE uses a site colouring whose equal-colour sites are
 * farther apart (periodic L1) than the degree of p_h, 12 probe vectors per colour.
 * out[2] receives the complex trace. */
int mmc_trace_exact(mmc_ctx* ctx, int handle, int theta_op, int method, int prec, double* out);

/* Number of colours of the probing colouring chosen for a reach (L1 distance). */
int mmc_probe_colours(mmc_ctx* ctx, int reach, int* n_colours);
/* The probing colouring itself (Sec. 6), pure host: for a lattice dims[4] =
 * {Lx, Ly, Lz, Lt} and a reach (periodic L1 distance), colour[V] (may be NULL;
 * site order x fastest) receives each site's colour and *n_colours their number.
 * Two distinct sites of equal colour are farther apart than reach. */
int mmc_probe_colouring(const int dims[4], int reach, int* colour, int* n_colours);

/* ------------------------------------------------- learned network (no paper section) */

/* A gauge-covariant linear stencil network N approximating M^-1: channel counts
 * 4 -> 8 -> 8 -> 4 per site (each channel a colour 3-vector, so 12 -> 24 -> 24
 * -> 12 complex), three layers out(x) = W0 in(x) + sum_mu [Wf_mu U_mu(x) in(x+mu)
 * + Wb_mu U_mu(x-mu)^+ in(x-mu)] (antiperiodic time phase as in M), no
 * nonlinearity, so Tr(Theta N) exists and a subtraction with N keeps Eq. 2's
 * estimator unbiased.  Weights: 1152 complex numbers (2304 doubles), layer
 * by layer, each [9][C_out][C_in] with index 0 = W0, 1+mu = Wf_mu, 5+mu = Wb_mu.
 * A network handle (>= MMC_NET_BASE) is accepted as mmc_solve's preconditioner,
 * as hi or lo of mmc_trace_level (without deflation) and by mmc_trace_exact
 * (probing with reach 3).  Fields given to the network are MMC_F32. */
#define MMC_NET_BASE 0x100000
#define MMC_NET_WEIGHTS 1152

/* Create a network with the given weights (NULL: near the channel embedding of
 * the identity plus seeded N(0, 0.05^2) entries). */
int mmc_net_create(mmc_ctx* ctx, const double* weights, uint64_t seed, int* handle);
int mmc_net_set_weights(mmc_ctx* ctx, int handle, const double* weights);
int mmc_net_get_weights(mmc_ctx* ctx, int handle, double* weights);
/* Storage of the network's weights and hidden activations (the reduced-precision
 * form; not in the paper): MMC_F32 (default) or MMC_BF16 (weights rounded to BF16 from the FP64
 * master copy, the 24-component hidden activations stored in BF16; FP32
 * arithmetic and accumulation; the input and output fields stay MMC_F32).  Both
 * inference and training use it; training keeps FP64 master weights (Adam on the
 * host) and FP32 gradients of the BF16 forward pass. */
int mmc_net_set_precision(mmc_ctx* ctx, int handle, int prec);
/* y = N x for nrhs MMC_F32 vectors (inference kernels, FP32 arithmetic). */
int mmc_net_apply(mmc_ctx* ctx, int handle, const void* x, void* y, int nrhs, void* stream);
/* Loss L = (1/B) sum_b ||N eta_b - x_b||^2 / ||x_b||^2 on one batch of B = nrhs
 * MMC_F32 pairs, and grad = dL/dRe W + i dL/dIm W (2304 doubles, may be NULL),
 * by the training kernels (forward, backward data, weight gradients). */
int mmc_net_loss_grad(mmc_ctx* ctx, int handle, const void* eta, const void* xs, int nrhs, double* loss,
                      double* grad);
/* Train with Adam (lr; betas 0.9, 0.999) for iters steps over mini-batches of
 * `batch` consecutive pairs (batch divides npairs and is a multiple of the rhs
 * block); loss_history (iters doubles, may be NULL) receives each step's loss. */
int mmc_net_train(mmc_ctx* ctx, int handle, const void* eta, const void* xs, int npairs, int batch, int iters,
                  double lr, double* loss_history);

/* ------------------------------------------------------------ profiling */

/* Counters of the fused step kernel (the stencil / polynomial-step hot loop):
 * launches, summed CUDA-event time of those launches, algorithmic bytes (each
 * input, output, aux and accumulator element once, the 4 links of a site once
 * per launch, 72 B each in FP32 and 144 B in FP64; the Z(4) noise of a code
 * bilinear is not counted, since it could be regenerated from the counter-based
 * generator instead of read) and flops (1368 per site and active
 * rhs for a hop, 48 more per epilogue term), plus the number of every kernel
 * the library launched.  Not part of the paper: bookkeeping for measurement. */
typedef struct {
  long long step_launches;
  double step_ms;
  double step_bytes;
  double step_flops;
  long long all_launches;
  long long graph_launches; /* step chains replayed from a CUDA graph (mmc_set_graphs) */
  long long graph_captures; /* of which captured (and instantiated) first */
} mmc_profile_stats;

/* The same counters per launch class: the step chains of one kind (with a
 * bilinear epilogue, accumulating into a field, with an aux operand such as the
 * Horner chains of the solves' preconditioner, or plain M) at one precision and
 * padded rhs count.  The time of a chain replayed from its CUDA graph is that
 * of the whole replay; launches, bytes and flops count its steps. */
enum { MMC_PROF_PLAIN = 0, MMC_PROF_BILINEAR = 1, MMC_PROF_ACCUMULATE = 2, MMC_PROF_AUX = 3 };
typedef struct {
  int kind;          /* MMC_PROF_* */
  int prec;          /* storage precision of the chain */
  int nrhs_padded;   /* right-hand sides per launch, padded to the rhs block */
  long long launches;
  double ms, bytes, flops;
} mmc_profile_class;

/* enable != 0 starts recording (counters reset); 0 stops.  While enabled every
 * step launch is bracketed by CUDA events on its stream. */
int mmc_profile(mmc_ctx* ctx, int enable);
/* Synchronise the context's work and read the counters. */
int mmc_profile_read(mmc_ctx* ctx, mmc_profile_stats* out);
/* Synchronise and copy up to max_classes per-class counters (in order of first
 * use since profiling was enabled) to out; *n_classes receives how many exist. */
int mmc_profile_classes(mmc_ctx* ctx, int max_classes, mmc_profile_class* out, int* n_classes);

/* Inner FGMRES length and outer-cycle limit of the solves inside mmc_trace_level
 * (Sec. 1 and Sec. 8: the solves of the M^-1 level; defaults 48 and 400).
 * Values <= 0 keep the current setting. */
int mmc_set_solve_params(mmc_ctx* ctx, int m_inner, int max_outer);
/* Schedule of the FP32/BF16 stage of the refined solves (mmc_solve and the solves of
 * mmc_trace_level): after each FP64 residual, up to inner_cycles FGMRES cycles, each
 * later one restarted from the stage's own FP32 residual (deflated), until every
 * vector's inner residual is inner_reduction (in (0, 1]) of its FP64 residual or stops
 * falling by 10% a cycle.  inner_cycles = 1 returns to FP64 after every cycle.
 * Defaults 3e-2 and 8.  MMC_ERR_ARG outside 1..64 cycles or (0, 1]. */
int mmc_set_solve_refinement(mmc_ctx* ctx, double inner_reduction, int inner_cycles);
/* Gram-Schmidt passes of the Arnoldi process in the FP32/BF16 stage of the refined
 * solves: 1 (classical Gram-Schmidt once, the default: the FP64 residual of the
 * refinement corrects what a less orthogonal basis leaves, and on the 24^4 workload
 * the matvecs are the same as with 2) or 2 (twice).  The Arnoldi runs of
 * mmc_gmres_poly, mmc_deflate and the plain FP64 form always take 2.  MMC_ERR_ARG
 * for other values. */
int mmc_set_gram_schmidt(mmc_ctx* ctx, int passes);
/* Field layout of the Horner chains of the polynomial preconditioner (Sec. 8: FGMRES
 * right-preconditioned by p_in) in the FP32 stage of 8-rhs solves: 0 keeps the blocked
 * layout [site][c][rhs]; 1 moves the input into a paired-component layout
 * [site][c/2][rhs][c%2] for the chain and the result back (two extra field passes per
 * application), so that the step kernel's lanes load and store two components of
 * their rhs in one 16-byte access and a site's 8 lanes read whole 128-byte lines.
 * Used only where the 8-rhs FP32 variant is the fourth kernel form (at 168
 * registers: minb 4 or 5 run as 3); the arithmetic is the same, so results are
 * bit-identical to layout 0.  Default 1 (on the 24^4 workload 0.189 against 0.213 ms
 * per Horner step).  MMC_ERR_ARG for other values. */
int mmc_set_horner_layout(mmc_ctx* ctx, int paired);
/* Storage of the inner FGMRES stage (its preconditioner chain included) in the
 * solves of the M^-1 level of a reduced-precision mmc_trace_level (Sec. 1,
 * Sec. 8; the prec_inner of mmc_solve): MMC_F32 (default) or MMC_BF16.  The FP64
 * outer loop still refines every solve to a relative residual of 1e-10, so the
 * level's samples differ only within that tolerance; the flexible inner
 * iteration tolerates the less accurate preconditioner at the cost of more
 * iterations.  MMC_ERR_ARG for any other value. */
int mmc_set_solve_storage(mmc_ctx* ctx, int prec_inner);
/* Rounding of BF16 chain storage (the reduced-precision form; not in the paper):
 * mode 0 rounds every stored element to nearest (default); mode 1 rounds it up or
 * down with probability given by its discarded bits, with random bits from a
 * counter-based hash of (element, step, a per-chain salt held in device memory and
 * advanced by each chain's first launch, so graph replays get fresh bits too),
 * which makes every stored iterate an unbiased estimate of the exact one and, the
 * chains and bilinears being linear, keeps each BF16 level unbiased.  seed sets the
 * salt sequence (results are reproducible for the same seed and call sequence).
 * The staged kernel form (version 3) is replaced by version 2 in mode 1.
 * MMC_ERR_ARG for other modes. */
enum { MMC_ROUND_NEAREST = 0, MMC_ROUND_STOCHASTIC = 1 };
int mmc_set_rounding(mmc_ctx* ctx, int mode, uint64_t seed);

/* Not part of the paper (data layout): largest right-hand-side block R of the
 * blocked field layout [rb][site][c][R] (8 or 16, default 16).  A batch of N vectors uses R = min(rmax, next power of
 * two >= N).  It changes the layout of every field sized or interpreted after
 * the call (mmc_field_bytes, mmc_pack, mmc_unpack), so set it before creating
 * fields; smaller blocks halve the L2 footprint of a site at the price of more
 * link reads per vector.  MMC_ERR_ARG for other values. */
int mmc_set_rhs_block_max(mmc_ctx* ctx, int rmax);
/* Fault injection for tests of the failure path (not part of the method):
 * enable != 0 makes the producer of the staged step kernel (version 3) issue no
 * copies, so every wait of its compute warps runs out; each wait is bounded by
 * wait_iters polls (0: the kernel's default, well over a second).  The kernel
 * then raises its error flag and returns, and the next synchronising call
 * (a level, a solve, a reduction) returns MMC_ERR_TIMEOUT with the context
 * still usable.  enable = 0 restores normal operation.  (Should the producer's
 * own bounded wait for its copies in flight ever give up, a copy might land
 * after its CTA exited: that call also returns MMC_ERR_TIMEOUT, and the context
 * is retired, every later call on it returning MMC_ERR_STATE until it is
 * destroyed.) */
int mmc_test_stall_staged(mmc_ctx* ctx, int enable, long long wait_iters);

/* Not part of the paper (launch tuning of the a1/a5 step kernel, Sec. 1 and
 * Sec. 3).  Launch variant of the fused step kernel for precision prec, for both rhs-block
 * classes (R < 16 and R = 16; mmc_set_step_variant_class sets one): rpt right-hand
 * sides per lane (1, 2; F64 uses 1), minb = minimum resident CTAs per SM asked
 * of the compiler for the generic kernel (1: no register cap; 3 or 4: capped;
 * for version 4, 3 gives 168 registers and 4 gives 128), or 100 + v to select
 * kernel version v (1: generic; 2: rhs block and epilogue fixed at compile
 * time, for F32/BF16 batches with R = 8 or 16; 3: as 2, with the lattice rows
 * staged in shared memory by bulk asynchronous copies issued by a producer
 * warp, for Lx * R up to 384, falling back to 2 otherwise; 4: as 2 with one
 * rhs per lane, a persistent grid whose CTAs take (rhs block, pass of sites)
 * items round-robin so that the sites in flight form one compact front, and
 * the loads of each hop issued while the previous hop computes (minb 3: 168
 * registers, 4: 128, 5: 128 with each pass's links staged in shared memory, 6: 168 with
 * each link's third row rebuilt from its first two, used when mmc_load_gauge found every
 * link special unitary and as minb 3 otherwise); 5: as 4 with
 * the operands of the hops staged in shared memory by per-lane asynchronous
 * copies several hops ahead, the depth set by 300 + n, FP32 3 or 4 (default 4),
 * BF16 4 (default) or 6), or 200 + b
 * for the site traversal of versions 2 and 4 (b = 0 lexicographic, 1 4 x 4 x 2
 * x 2 blocks when the extents are divisible, 2 z-half by z-half with t outermost
 * within a half when Lz is even), or 300 + n to give version 3 n ring slots
 * (2..6; 300: as many as fit) and version 5 its pipeline depth, or 400 + h for the store hint of version 4 (h =
 * 1: results stored with an L2 evict-first policy, 0: default); spc = sites per
 * CTA (16..1024, power of two).  Values <= 0 keep the current setting.  Version 3 bounds every
 * wait for its staged rows; a wait that gives up makes the next call that
 * synchronises (a level, a solve, a reduction) return MMC_ERR_TIMEOUT. */
int mmc_set_step_variant(mmc_ctx* ctx, int prec, int rpt, int minb, int spc);
/* The whole variant of one rhs-block class at once: rhs_class 0 for batches
 * whose block R is below 16 (up to 8 vectors, e.g. the solves of the M^-1
 * level), 1 for R = 16; version 1..5 (F64: 1), rpt 1 or 2, minb 1..8, spc as
 * above, blocked = traversal 0..2, ns 0 or 2..6 (version 5: its depth, 0 for
 * 4).  MMC_ERR_ARG on any value out of range.  The store hint of version 4 is
 * set by mmc_set_step_variant. */
int mmc_set_step_variant_class(mmc_ctx* ctx, int prec, int rhs_class, int version, int rpt, int minb, int spc,
                               int blocked, int ns);
/* Step chains (the degrees of a polynomial applied to a batch, Sec. 3, Sec. 5) run
 * as CUDA graphs: the first run of a chain with given operands, coefficients and
 * kernel variant captures its launches (on a private stream of the context),
 * later runs replay the graph on the caller's stream (one launch for all
 * degrees).  enable = 0 launches every degree directly (and drops the graphs);
 * results are identical either way.  Default: enabled.  While the caller's
 * stream is itself capturing, chains are launched degree by degree.  Returns
 * MMC_ERR_ARG for a NULL context. */
int mmc_set_graphs(mmc_ctx* ctx, int enable);
/* "" while chain graphs work; otherwise why the context switched to direct
 * launches (a capture the driver refused).  Context-owned string. */
const char* mmc_graph_note(const mmc_ctx* ctx);
/* Not part of the paper (launch tuning).  Autotuner: time every step-kernel
 * variant on one degree of a polynomial level chain (M applied with the step
 * update and the Z(4)-code bilinear epilogue, the form the Monte Carlo levels
 * run) over an nrhs-vector noise field of precision prec (CUDA events, median
 * of 3 after a warm-up), keep the fastest for that precision and the rhs-block
 * class of nrhs and return it (best[6] = rpt, minb, spc, kernel version,
 * traversal, ring slots of version 3) with its time per launch in ms. */
int mmc_autotune(mmc_ctx* ctx, int nrhs, int prec, int* best, double* ms);

/* Replace the device links by a new host field (same layout as mmc_load_gauge)
 * keeping kappa, polynomials and eigenpairs: for a caller that streams the same
 * configuration, or accepts them as fixed approximations (any fixed polynomial
 * keeps the estimator of Eq. 2 unbiased). */
int mmc_update_gauge(mmc_ctx* ctx, const double* U);

/* ---------------------------------------------------- host-only helpers */

/* Harmonic Ritz values of a GMRES(m) cycle (Sec. 3) from its (m+1) x m Hessenberg
 * matrix H (complex, column-major, leading dimension ldh >= m+1), Leja ordered
 * into theta_out (2m doubles).  Pure host FP64. */
int mmc_harmonic_ritz(int m, const double* H, int ldh, double* theta_out);
/* Leja ordering (Sec. 3) of m complex points: first the largest modulus, then
 * the maximiser of the product of distances (sum of logs), ties to lowest index. */
int mmc_leja_order(int m, const double* theta_in, double* theta_out);
/* Kept set of the deflation eigenpairs (Sec. 8: acceptance of Ritz pairs with
 * residual below tol_accept; left vectors from gamma_5-hermiticity), the host
 * rule mmc_deflate applies to its m candidates: lambda (2m doubles) and residual
 * norms res (m).  The accepted ones, ordered by |lambda| (stable), the first k,
 * are taken in that order: a real one (|Im| < 2e-4) is its own gamma_5 partner; a
 * complex one takes the nearest candidate to its conjugate that is neither itself
 * nor already taken, if closer than 10 max(2e-4, 1e-6 |lambda|), and is dropped
 * otherwise.  keep, partner (m ints each, caller-owned) receive candidate indices,
 * *n_keep their number.  Pure host. */
int mmc_deflation_pairs(int m, const double* lambda, const double* res, double tol_accept, int k, int* keep,
                        int* partner, int* n_keep);
/* Drop rules of mmc_deflate on the q x q overlap S(i, j) = w_i^H z_j of the kept
 * pairs (complex, column-major, leading dimension lds >= q), mates[i] = position
 * of pair i's gamma_5 partner (i for a real eigenvalue): while S restricted to the
 * selection is singular the last position is dropped, while a column of its
 * inverse conjugate transpose (the size of a left vector u_i) has norm above
 * max_u (mmc_deflate: 100) the position of the largest column is dropped; each
 * drop takes the partner along.  sel (q ints) receives the kept positions in
 * increasing order, *n_sel their number (0: nothing left).  Pure host. */
int mmc_deflation_condition(int q, const double* S, int lds, const int* mates, double max_u, int* sel,
                            int* n_sel);
/* Eigenvalues (and right eigenvectors, column-major, if vr != NULL) of a complex
 * n x n matrix A (column-major, lda >= n); pure host FP64 (Hessenberg reduction
 * + shifted QR).  Used for the Ritz values of Sec. 3 and Sec. 7. */
int mmc_eig(int n, const double* A, int lda, double* w, double* vr);

#ifdef __cplusplus
}
#endif
#endif /* MMC_H */
