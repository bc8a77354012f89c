/*
 * stag.h -- C ABI of libstag: even-odd preconditioned staggered operator and
 * mixed-precision conjugate gradient on one GB300 (sm_103a).
 *
 * Method.  Sec. 3 of the paper ("CG Performance") runs a mixed-precision
 * conjugate-gradient inverter for HYP-smeared staggered quarks on 20^3 x 64
 * lattices, single precision dominant with a double-precision part.  The paper
 * does not write the operator; this library implements the standard one-link
 * staggered operator with these conventions:
 *
 *   dims = {Lx, Ly, Lz, Lt}, all even and >= 2; V = Lx Ly Lz Lt, Ve = V / 2;
 *   lexicographic site index lex = x + Lx (y + Ly (z + Lz t));
 *   parity (x+y+z+t) mod 2, even = 0; checkerboard index of a site = lex / 2;
 *   eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}), mu = 0..3 = x, y, z, t;
 *   b_mu(x) = -1 for mu = t, x_t = Lt - 1 when STAG_ANTIPERIODIC_T is set;
 *   (D psi)(x) = sum_mu [ eta_mu(x) b_mu(x) U_mu(x) psi(x+mu)
 *                       - eta_mu(x) b_mu(x-mu) U_mu(x-mu)^dag psi(x-mu) ];
 *   D_oe: even -> odd sites, D_eo: odd -> even sites;
 *   A = M^dag M on even sites = 4 m^2 - D_eo D_oe (Hermitian positive definite).
 *
 * Data layouts at the ABI (FP64, complex numbers as interleaved (re, im)):
 *   links:  [4][Lt][Lz][Ly][Lx][3][3][2]  (direction, site, row, column, re/im)
 *   vector: [Ve][3][2] over the checkerboard index of one parity.
 * Every pointer argument may be host memory (pageable or pinned) or device
 * memory of the context's GPU; the library finds out with
 * cudaPointerGetAttributes and copies host data itself.  The caller owns all
 * memory it passes; the library never keeps a caller pointer past the call.
 *
 * Errors.  Every function returns a status (STAG_OK = 0, STAG_NOT_CONVERGED =
 * 1, negative = error) and never throws.  stag_last_error() gives a message.
 * Work is ordered on the context's CUDA stream; each call returns after its
 * results are in the caller's buffers.  A context is not thread-safe.
 */
#ifndef STAG_H
#define STAG_H

#ifdef __cplusplus
extern "C" {
#endif

#define STAG_ABI_VERSION 1

/* status codes */
#define STAG_OK 0
#define STAG_NOT_CONVERGED 1 /* x = last iterate, true_res filled */
#define STAG_ERR_ARG (-1)    /* bad dims, NULL pointer, bad count/tolerance/precision */
#define STAG_ERR_CUDA (-2)   /* a CUDA runtime call failed */
#define STAG_ERR_OOM (-3)    /* device allocation failed */
#define STAG_ERR_NOT_SU3 (-4) /* reconstruct-12 requested on links that are not SU(3) */
#define STAG_ERR_BREAKDOWN (-5) /* <p, A p> <= 0 or a non-finite residual in CG */
#define STAG_ERR_TIMEOUT (-6) /* a bounded device-side wait gave up; the results are void */
#define STAG_ERR_STATE (-7)  /* operator used before stag_links_upload */

/* arithmetic/storage precision of the inner (Krylov) iteration */
#define STAG_FP64 0 /* FP64 storage and arithmetic */
#define STAG_FP32 1 /* FP32 storage and arithmetic */
#define STAG_FP16 2 /* FP16 storage (per-site scale for vectors), FP32 arithmetic */
#define STAG_BF16 3 /* BF16 storage (per-site scale for vectors), FP32 arithmetic */

/* OR-ed into the precision of stag_dslash_oe/eo and stag_mdagm: hold every
 * vector at the storage precision and round the output to it, exactly as the
 * solver's inner iteration does (FP16/BF16: per-site scaled). */
#define STAG_ROUND_OUTPUT 0x100

/* OR-ed into the precision of stag_cg_solve / stag_time_dslash with STAG_FP16
 * or STAG_BF16: also store the Krylov vectors (p, A p and the intermediate
 * D_oe p) at that precision with a per-site scale.  Without it only the links
 * are stored at FP16/BF16 and the Krylov vectors stay FP32. */
#define STAG_HALF_VECTORS 0x200

/* OR-ed into the precision of stag_cg_solve / stag_time_cg_kernel with
 * STAG_FP32 links (or links of the same half format): store the Krylov
 * vectors p and D_oe p at FP16 / BF16 with a per-site FP32 scale (value =
 * code x scale, scale = max |component| of the site), independently of the
 * links.  The iterated residual and the partial solution stay FP32, the
 * arithmetic FP32, the reliable updates FP64.  Links rounded to FP16/BF16
 * change A itself; rounded vectors only perturb each A p, by D_eo applied to
 * the rounding of D_oe p. */
#define STAG_VEC_FP16 0x400
#define STAG_VEC_BF16 0x800

/* context flags */
#define STAG_ANTIPERIODIC_T 1 /* antiperiodic boundary in t (the sign b_mu above) */
#define STAG_RECON12 2 /* reduced-precision links keep rows 0,1; row 2 = conj(row0 x row1) */

typedef struct stag_ctx stag_ctx;

/*
 * Create a context for one lattice on the current CUDA device.
 *   dims[4]     {Lx, Ly, Lz, Lt}: each even and >= 2, V/2 < 2^31.
 *   flags       STAG_ANTIPERIODIC_T | STAG_RECON12.
 *   cuda_stream cudaStream_t to order all work on (NULL = legacy default stream).
 *   out         receives the context.
 * Errors: STAG_ERR_ARG (dims, out == NULL), STAG_ERR_CUDA, STAG_ERR_OOM.
 */
int stag_create(const int dims[4], int flags, void *cuda_stream, stag_ctx **out);

/* Free every device buffer of the context.  NULL is accepted. */
int stag_destroy(stag_ctx *ctx);

/*
 * Copy a gauge field into the context's own device layouts (Sec. 3: the
 * operator's one-link smeared SU(3) field).  `links` is [4][V][3][3][2] FP64,
 * host or device.  The FP64 copy is always kept (true residual, FP64 solves);
 * FP32/FP16/BF16 copies are made on first use.  Staggered phases and the
 * boundary sign are applied inside the kernels, never folded into the links.
 * With STAG_RECON12 the links must be SU(3): a unitarity or determinant
 * defect above 1e-12 returns STAG_ERR_NOT_SU3.
 */
int stag_links_upload(stag_ctx *ctx, const double *links);

/*
 * out_odd = D_oe in_even (the even -> odd half of the operator).
 * `precision` selects the storage/arithmetic of the computation: the FP64
 * input is rounded to it (FP16/BF16: per-site scaled vector, unscaled links),
 * the operator applied, and the result returned in FP64 without further
 * rounding (with STAG_ROUND_OUTPUT: rounded to the storage precision, as the
 * solver stores it).  in_even and out_odd are [Ve][3][2] FP64, host or device, and must
 * not overlap.  Errors: STAG_ERR_ARG, STAG_ERR_STATE, STAG_ERR_CUDA.
 */
int stag_dslash_oe(stag_ctx *ctx, int precision, const double *in_even, double *out_odd);

/* out_even = D_eo in_odd; as stag_dslash_oe with the parities exchanged. */
int stag_dslash_eo(stag_ctx *ctx, int precision, const double *in_odd, double *out_even);

/*
 * out_even = (4 m^2 - D_eo D_oe) in_even, the even-site normal operator M^dag M
 * that the CG of Sec. 3 inverts.  Same conventions as stag_dslash_oe.
 */
int stag_mdagm(stag_ctx *ctx, int precision, double mass, const double *in_even,
               double *out_even);

/*
 * Solve (4 m^2 - D_eo D_oe) x = b for every source in src[] and every mass in
 * masses[] (Sec. 3: the mixed-precision CG inverter).  nrhs * nmass systems;
 * system (r, k) has source src[r], mass masses[k] and solution x[r * nmass + k].
 *   precision  STAG_FP64: plain FP64 CG.  STAG_FP32/FP16/BF16: the inner
 *              iteration runs with links stored at that precision (FP32
 *              arithmetic; Krylov vectors FP32, or FP16/BF16 per-site scaled
 *              with STAG_VEC_FP16 / STAG_VEC_BF16 / STAG_HALF_VECTORS), the
 *              solution is accumulated and the residual recomputed in FP64
 *              whenever the iterated residual has dropped by 10x since the last
 *              recomputation ("reliable update"), and at convergence.
 *   tol        stop when ||b - A x|| / ||b|| <= tol, with the residual
 *              recomputed in FP64 on the GPU (tol > 0).
 *   maxiter    iteration cap per system (>= 1).
 *   iters[]    (may be NULL) iterations taken per system.
 *   true_res[] (may be NULL) final ||b - A x|| / ||b|| recomputed in FP64.
 * A zero source gives x = 0, 0 iterations, true_res = 0.
 * Returns STAG_OK when every system converged, STAG_NOT_CONVERGED when some
 * system hit maxiter (its x is the last iterate), STAG_ERR_BREAKDOWN on a
 * non-positive <p, A p> or a non-finite residual, STAG_ERR_TIMEOUT when a
 * kernel's bounded wait for its staged links gave up (only with the
 * shared-memory link path, STAG_TMA=1), STAG_ERR_ARG / _STATE / _CUDA.
 */
int stag_cg_solve(stag_ctx *ctx, const double *const src[], int nrhs, const double masses[],
                  int nmass, double tol, int maxiter, int precision, double *const x[],
                  int iters[], double true_res[]);

/*
 * The one-colour-trace four-fermion contraction of the NPR (RI-MOM) workload
 * (Sec. 4, Eq. (ffop): FP64, 97 % of that code's time), on every hypercube z
 * of the lattice (sites z_A = 2z + A, corners A in {0,1}^4):
 *   O(z) = sum_{A,B,C,D} [chibar1(z_A) (g_S1 x x_F1)_AB chi2(z_B)]
 *                        [chibar3(z_C) (g_S2 x x_F2)_CD chi4(z_D)]
 *                        [U_AD(z)]_{c1 c4} [U_CB(z)]_{c3 c2}
 * (colour c1 of chibar1 tied to c4 of chi4 and c3 of chibar3 to c2 of chi2
 * through the links), with the readings the paper leaves open:
 *   (g_S x x_F)_AB = (1/4) Tr(g_A^dag g_S g_B g_F^dag), g_A = g_1^A1 g_2^A2
 *   g_3^A3 g_4^A4 (Euclidean Hermitian gammas; bit mu of A = direction mu of
 *   x, y, z, t); U_AD(z) = the average over the shortest lattice paths from
 *   z_A to z_D of the link products (U_mu for a step +mu, U_mu^dag for -mu).
 *   spin_taste  (S1, F1, S2, F2), each a 4-bit corner mask 0..15;
 *   chibar1, chi2, chibar3, chi4  [V][3][2] FP64 colour-vector fields in the
 *               links' lexicographic site order (for NPR: propagator columns),
 *               host or device;
 *   O_hyp       [V/16][2] (may be NULL): O(z) at hypercube index
 *               z0 + (Lx/2)(z1 + (Ly/2)(z2 + (Lz/2) z3)), host or device;
 *   O_sum       [2] (may be NULL): sum over z, fixed-order FP64 reduction.
 * Uses the uploaded gauge field (FP64).  Errors: STAG_ERR_ARG, _STATE, _CUDA.
 */
int stag_npr_contract(stag_ctx *ctx, const int spin_taste[4], const double *chibar1, const double *chi2,
                      const double *chibar3, const double *chi4, double *O_hyp, double *O_sum);

/*
 * HYP smearing of a gauge field (Sec. 3: the quarks are "HYP-smeared"
 * staggered quarks; the paper gives no parameters): links_out = the
 * hypercubic-blocked field of links_in by Hasenfratz and Knechtli's three
 * levels of decorated staples,
 *   Vb(x,mu;e)  = P[(1-a3) U_mu(x) + a3/2 sum_{+-e} U_e U_mu U_e^dag],  e != mu,
 *   Vt(x,mu;nu) = P[(1-a2) U_mu(x) + a2/4 sum_{+-r != mu,nu} Vb(r;s) Vb(mu;s) Vb(r;s)^dag],
 *                 s = the direction outside {mu, nu, r},
 *   V(x,mu)     = P[(1-a1) U_mu(x) + a1/6 sum_{+-nu != mu} Vt(nu;mu) Vt(mu;nu) Vt(nu;mu)^dag],
 * with P(X) the unitary polar factor of X with its determinant's phase removed
 * (principal cube root), so every output link is SU(3).
 *   alpha      (a1, a2, a3); NULL = (0.75, 0.6, 0.3);
 *   links_in, links_out  [4][V][3][3][2] FP64 as stag_links_upload, host or
 *              device; they may be the same buffer.
 * FP64 throughout on the GPU; the context provides the lattice and the
 * stream (its gauge field is not touched: upload the result to use it).
 * Scratch: 2 x 12 V links of the context's device memory.
 * Errors: STAG_ERR_ARG, STAG_ERR_CUDA, STAG_ERR_OOM.
 */
int stag_hyp_smear(stag_ctx *ctx, const double alpha[3], const double *links_in, double *links_out);

/*
 * stag_cg_solve for several masses by a multi-shift CG (Sec. 3's inverter
 * with its multi-mass workloads): the systems of one source differ only by the
 * shift 4 m^2, so the masses share one Krylov space -- one operator
 * application per iteration serves them all:
 *   phase 1  the smallest mass runs the mixed-precision CG of stag_cg_solve
 *            (FP64 reliable updates) and the other masses follow its
 *            residuals as shifted systems (r_s = zeta_s r; FP32 directions and
 *            solutions), each until its estimated residual is below 1e-5;
 *   phase 2  each shifted system continues from that solution as an initial
 *            guess with the mixed-precision CG (its first step recomputes
 *            b - A x0 in FP64) to the tolerance.
 * Phase 2 is needed: FP32 shifted recurrences stall near eps_32 kappa_s of
 * their systems, and reliable updates cannot act on them (they would break
 * r_s = zeta_s r).  Arguments, layouts and statuses as stag_cg_solve;
 * iters[] counts both phases; precision must be a reduced one (not
 * STAG_FP64).  stag_solve_stats/counters/form then describe phase 2.
 */
int stag_cg_solve_multishift(stag_ctx *ctx, const double *const src[], int nrhs, const double masses[],
                             int nmass, double tol, int maxiter, int precision, double *const x[], int iters[],
                             double true_res[]);

/*
 * Solve the full-lattice staggered equation M x = b, M = 2m + D (the operator
 * at the top of this header with its mass term; Sec. 3 of the paper: the
 * equation the CG inverter serves, its even-site Schur complement being what
 * stag_cg_solve inverts), for every source and mass, by the even-odd route:
 *   b_s = 2m b_e - D_eo b_o                     (FP64, on the GPU),
 *   (4 m^2 - D_eo D_oe) x_e = b_s               (the CG of stag_cg_solve),
 *   x_o = (b_o - D_oe x_e) / (2m)               (FP64, on the GPU).
 *   src[r], x[r * nmass + k]  full-lattice vectors [V][3][2] FP64 in the
 *              lexicographic site order of the links, host or device;
 *   masses     finite and > 0;
 *   tol        stop when ||b - M x|| / ||b|| <= tol: with x_o as above the odd
 *              rows of b - M x vanish (to rounding) and the even rows are
 *              (b_s - A x_e) / (2m), so the CG holds its FP64 residual to
 *              ||b_s - A x_e|| <= tol 2m ||b||;
 *   true_res[] (may be NULL) ||b_s - A x_e|| / (2m ||b||), recomputed in FP64.
 * precision, maxiter, iters[] and the statuses as in stag_cg_solve.
 */
int stag_solve_full(stag_ctx *ctx, const double *const src[], int nrhs, const double masses[], int nmass,
                    double tol, int maxiter, int precision, double *const x[], int iters[], double true_res[]);

/*
 * Average device time of one launch of one of the two half-operator kernels
 * of the CG iteration (Sec. 3; the operator A of the top of this header, split
 * as A p = 4 m^2 p - D_eo (D_oe p)) at `precision`, measured with CUDA events
 * on the context stream over `nlaunch` pairs of the two kernels launched
 * alternately, as the iteration runs them (each starts on the cache state the
 * other leaves), on the context's own internal vectors with the solver's
 * launch configuration, including (single-system forms) the reduction of the
 * other kernel's partial sums that every block of a CG kernel finishes
 * before its own work in the solve.  With programmatic dependent launch on
 * (the default), an event between two launches would stop the overlap of a
 * kernel's launch with its predecessor's tail that the solve has, so the
 * pairs are also timed with events only around the whole sequence and each
 * kernel is given its share, from the separated timings, of that pair time:
 *   kernel 0: t = D_oe r + beta t_old (FP32/FP64 Krylov vectors) or
 *             t = D_oe (r + beta p_old) (STAG_HALF_VECTORS), with |t|^2;
 *   kernel 1: p = r + beta p_old, r -= alpha (4 m^2 p - D_eo t),
 *             x += alpha p, with |r|^2 and Re<r, p>.
 * `bytes_per_launch` (may be NULL) receives the kernel's algorithmic bytes
 * per launch: per output site its 8 links and the gathered vector once, plus
 * kernel 0: t_old (or r) read and t written; kernel 1: p, r and x read and
 * written.  Returns STAG_ERR_ARG for another `kernel` or nlaunch < 1.
 */
int stag_time_cg_kernel(stag_ctx *ctx, int precision, int kernel, int nlaunch, double *ms_per_launch,
                        double *bytes_per_launch);

/* stag_time_cg_kernel with kernel 0. */
int stag_time_dslash(stag_ctx *ctx, int precision, int nlaunch, double *ms_per_launch,
                     double *bytes_per_launch);

/* One lattice of a ragged batch: the arguments of stag_cg_solve for ctx. */
typedef struct stag_solve_desc {
  stag_ctx *ctx;
  const double *const *src; /* nrhs sources */
  int nrhs;
  const double *masses; /* nmass masses */
  int nmass;
  double *const *x;  /* nrhs * nmass solutions, slot r * nmass + k */
  int *iters;        /* nrhs * nmass, may be NULL */
  double *true_res;  /* nrhs * nmass, may be NULL */
} stag_solve_desc;

/*
 * Solve several lattices of different sizes (one context each, same device)
 * together: every lattice's solve loop is a branch of one CUDA graph, so the
 * GPU runs them concurrently (Sec. 3 workloads batched; one graph launch for
 * the whole ragged batch).  The first context's stream orders the batch.
 * tol, maxiter and precision as in stag_cg_solve, shared by all lattices.
 * Returns the worst status over the lattices (an error, else
 * STAG_NOT_CONVERGED, else STAG_OK); per-system results in each entry.
 */
int stag_cg_solve_ragged(const stag_solve_desc *descs, int ndesc, double tol, int maxiter, int precision);

/*
 * Statistics of system `sys` (0 <= sys < nrhs * nmass) of the most recent
 * stag_cg_solve on this context: iterations, FP64 reliable updates (the
 * recomputations of the residual, including the final one) and the final true
 * residual.  Any output pointer may be NULL.  STAG_ERR_ARG for a bad index or
 * before the first solve.
 */
int stag_solve_stats(const stag_ctx *ctx, int sys, int *iters, int *reliable_updates,
                     double *true_res);

/*
 * Loop counters of the most recent stag_cg_solve on this context (all its
 * systems together): passes of the solve loop (each runs up to U CG
 * iterations of every running system, U = stag_solve_form out[6]) and
 * executions of the FP64 reliable-update step (Sec. 3; each recomputes the
 * residual of every system with an update due).  From them the kernels
 * launched follow: 2 U + 1 per pass and 5 per update step (4 with
 * STAG_HALF_VECTORS).  Either pointer may be NULL.  STAG_ERR_ARG before the
 * first solve.
 */
int stag_solve_counters(const stag_ctx *ctx, int *loop_passes, int *update_steps);

/*
 * The launch form the autotuner chose for the CG kernels of the most recent
 * solve (or timing call): out[0] systems per thread, out[1] system groups,
 * out[2] / out[3] lanes per site of the first / second kernel, out[4] link
 * path (0 plane layout, 1 tiled through shared memory, 2 tiled into
 * registers), out[5] what persists in L2 during the solve (0 nothing, 1 the
 * links, 2 the Krylov vectors), out[6]
 * CG iterations per pass of the solve loop, out[7] 1 when the CG kernels
 * share each chunk's links in shared memory among the out[0] systems of a
 * block (one warp per system), 2 when every block runs every system on
 * links staged once per tile in shared memory (out[0] = the systems,
 * out[2] = out[3] = threads per site), 3 the same with the first kernel
 * taking two systems per pass through each thread.  Implementation detail of this
 * library (the paper has no counterpart), for reports.  STAG_ERR_ARG before
 * the first solve.
 */
int stag_solve_form(const stag_ctx *ctx, int out[8]);

/*
 * out_even = (4 m^2 - D_eo D_oe) in_even in FP64, with tmp_odd = D_oe in_even
 * and *dot = Re<in_even, out_even> (FP64, fixed-order reduction), for callers
 * that cannot allocate device memory (their memory is owned by another
 * allocator, or they must not allocate once set up).  The paper has no
 * counterpart of this entry point; it is an interface convenience.
 * It allocates nothing: every pointer is caller-owned device memory in the
 * layouts above (dot: one double, may be NULL), and the reduction scratch is a
 * fixed file-scope device array (512 KiB + 256 B per GPU, held until exit).
 *   - lattices with more than 8 388 608 sites per parity: STAG_ERR_ARG;
 *   - the first call on a device looks up that array's address (once per
 *     device); make it before any stream capture;
 *   - all calls share the array: calls that overlap on the GPU race;
 *   - asynchronous: results are ready when the context's stream reaches them.
 * Errors: STAG_ERR_ARG (size, NULL pointer, host memory or another GPU's
 * memory; managed memory is accepted), STAG_ERR_STATE (no links),
 * STAG_ERR_CUDA.
 */
int stag_mdagm_dot_noalloc(stag_ctx *ctx, double mass, const double *in_even, double *tmp_odd,
                           double *out_even, double *dot);

/*
 * Fermion force of the action S = phi^dag A^{-1} phi, A = 4 m^2 - D_eo D_oe,
 * given the solution x_even = A^{-1} phi (e.g. from stag_cg_solve in FP64).
 * The derivative of S with respect to the gauge field (the molecular-dynamics
 * force of the HYP-smeared staggered quarks of Sec. 3, computed on the
 * one-link field the operator uses):
 *   grad_links [4][V][3][3][2] (may be NULL): dS/dRe U + i dS/dIm U per link
 *              (the torch convention), = K^dag with dS = Re Tr(K dU);
 *   lie_force  [4][V][8] (may be NULL): f_a = Re Tr(i T_a U K), T_a =
 *              lambda_a / 2, the derivative along U -> exp(i w T_a) U.
 * One FP64 half operator (Y = D_oe X) plus one pass over the links; FP64.
 * Host or device pointers.  Errors: STAG_ERR_ARG, STAG_ERR_STATE, _CUDA.
 */
int stag_force(stag_ctx *ctx, const double *x_even, double *grad_links, double *lie_force);

/*
 * The fermion action S = phi^dag A^{-1} phi (A = 4 m^2 - D_eo D_oe; the
 * molecular-dynamics action of the staggered quarks whose inverter is Sec. 3's
 * CG) at an approximate solution x of A x = phi, in the stationary form
 *   S = 2 Re<phi, x> - Re<x, A x>,
 * exact at the exact solution and with an error second order in the residual
 * phi - A x (Re<phi, x> alone is first order).  A x in FP64; every site's term
 * summed in double-word (two-sum) FP64 arithmetic in a fixed order, so S
 * carries a few units of FP64 rounding and repeats bit for bit.  phi_even and
 * x_even are [Ve][3][2] FP64, host or device; *S is host memory.
 * Errors: STAG_ERR_ARG, STAG_ERR_STATE, STAG_ERR_CUDA.
 */
int stag_action(stag_ctx *ctx, double mass, const double *phi_even, const double *x_even, double *S);

/*
 * Backward pass of the action for an autograd engine: given x_even = A^{-1}
 * phi and the upstream factor gS = dL/dS,
 *   grad_links [4][V][3][3][2] (may be NULL) = gS K^dag (as stag_force),
 *   grad_phi   [Ve][3][2]      (may be NULL) = 2 gS x  (dS/dphi in the torch
 *              convention dS/dRe phi + i dS/dIm phi, S being real).
 * Host or device pointers.  Errors: STAG_ERR_ARG, STAG_ERR_STATE, _CUDA.
 */
int stag_action_backward(stag_ctx *ctx, const double *x_even, double gS, double *grad_links, double *grad_phi);

/* Message of the last error on this context ("" when none). */
const char *stag_last_error(const stag_ctx *ctx);

/* Static name of a status code. */
const char *stag_status_string(int status);

/* STAG_ABI_VERSION of the loaded library. */
int stag_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* STAG_H */
