/*
 * mahi.h — C ABI of the GB300 (sm_103a) implementation of Multipole-Accelerated
 * Hamiltonian Interpolation (MAHI), arxiv 2410.01754.
 *
 * One call to mahi_eval performs one periodic Fast Multipole Method evaluation of
 * the lambda-charge-scaled system (Sec. "Fast Multipole Method", Fig. "fmm_scheme":
 * P2M, M2M, M2L, L2L, L2P and the P2P near field; periodic part split as in Eq.
 * "approx_nbody_periodic": first image shell in the tree, lattice operator for the
 * far images, dipole/background term in closed form) and then the per-site
 * outputs of Hamiltonian interpolation for two-form sites (Sec. "Multipole-
 * Accelerated Hamiltonian Interpolation", Eqs. "correction_scheme",
 * "DeltaFQIHI", "Udiff"):
 *
 *   E          = E(q~) + sum_s 1/2 lambda_s (1 - lambda_s) k_s
 *   dE/dlam_s  = sum_{i in s} (qB_i - qA_i) phi~_i + (1/2 - lambda_s) k_s
 *   F_i        = -q~_i grad phi~_i - lambda_s(1-lambda_s) f sum_{j in s, j!=i} D_i D_j grad A(r_ij)
 *
 * with q~_i = qA_i + lambda_{s(i)} (qB_i - qA_i), D = qB - qA, phi~ the periodic
 * potential of q~ (tin-foil boundary, uniform neutralising background, self-image
 * term included) and k_s = f sum_{i,j in s} D_i D_j A(r_ij) the intra-site
 * (form-form) term.
 *
 * Units: nm, elementary charges, kJ/mol; f = 138.935457644382 kJ mol^-1 nm e^-2.
 * Conventions common to all calls:
 *   - Return value 0 = success, negative = error (see MAHI_ERR_*); no exception
 *     crosses this boundary.  mahi_error_string() gives a static message.
 *   - The handle is not thread-safe; one handle per host thread.
 *   - "device" pointers are CUDA device (or managed) memory of the current device.
 */
#ifndef MAHI_H
#define MAHI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mahi_ctx *mahi_t;

/* Arithmetic of the evaluation.
 *   MAHI_FP64  every stage in FP64 (the reference GPU path).
 *   MAHI_MIXED FP32 particle stages (P2M, L2P, P2P), M2L on the tensor cores as
 *              three TF32 products with FP32 accumulation, FP32 M2M/L2L; FP64
 *              lattice operator, dipole/background term, energy reduction and
 *              per-site corrections.
 *   MAHI_MIXED_SIMT  as MAHI_MIXED but M2L on FP32 CUDA cores (no tensor cores). */
enum { MAHI_FP64 = 0, MAHI_MIXED = 1, MAHI_MIXED_SIMT = 2 };

enum {
  MAHI_OK = 0,
  MAHI_ERR_INVALID_ARG = -1, /* bad size, order, depth, box, null pointer      */
  MAHI_ERR_BAD_SITE_MAP = -2,/* site index >= S, empty site, qA != qB off-site  */
  MAHI_ERR_NON_CUBIC = -3,   /* reserved: only cubic boxes (paper, Sec. FMM)    */
  MAHI_ERR_CUDA = -4,        /* a CUDA call failed; see mahi_last_cuda_error    */
  MAHI_ERR_TIMEOUT = -5,     /* a bounded device wait gave up                   */
  MAHI_ERR_NO_DEVICE = -6,   /* no usable sm_100-class device                   */
  MAHI_ERR_STATE = -7,       /* call order: charges not set                     */
  MAHI_ERR_SITE_OVERFLOW = -8/* a site's traversal lists outgrew their capacity */
};

/* Device-side failures.  Two conditions are detected inside the kernels of an
 * evaluation and recorded in a status word of the handle (host-mapped memory,
 * written by the device only on failure):
 *   MAHI_ERR_TIMEOUT        a bounded wait of the tensor-core M2L or of the
 *                           site-atom potential gave up (the kernel then
 *                           drains its copies, frees its tensor memory and
 *                           returns; the local expansions or site potentials
 *                           of that evaluation are incomplete);
 *   MAHI_ERR_SITE_OVERFLOW  the separation-controlled traversal of a site (the
 *                           refined site-atom potential) had more boxes at one
 *                           level than its list capacity (MAHI_OPT_SITE_LIST_CAP);
 *                           that site's dE/dlambda is incomplete.
 * Outputs of an evaluation that failed this way are not valid.  Because
 * mahi_eval returns once work is enqueued, such a failure is reported by the
 * next call that sees it: mahi_get_status (which synchronises), mahi_eval_host
 * (which synchronises), or the next mahi_eval, which then returns the code
 * without enqueueing anything.  Reporting clears the status word. */
int mahi_get_status(mahi_t h);

/* Create a solver for n_atoms atoms in a cubic periodic box of edge box_L_nm,
 * n_sites two-form titratable sites, multipole order order_p (expansions have
 * (p+1)^2 real coefficients) and octree depth (8^depth leaves).
 * Limits: 1 <= order_p <= 24 (MAHI_FP64), <= 16 (MAHI_MIXED_SIMT) or <= 15
 * (MAHI_MIXED: the tensor-core tile holds at most 256 coefficients), 0 <= depth <= 6,
 * n_atoms >= 1, n_sites >= 0, box_L_nm > 0.
 * cuda_stream: cudaStream_t on which all later work is enqueued (NULL = legacy
 * default stream).  Allocates all device workspaces (the library owns them) and
 * builds the translation operators and lattice coefficients on the host.
 * Returns MAHI_ERR_NO_DEVICE if no CUDA device is present. */
int mahi_create(double box_L_nm, int64_t n_atoms, int32_t n_sites, int32_t order_p, int32_t depth,
                int32_t precision, void *cuda_stream, mahi_t *out);

/* Release every resource of the handle.  Accepts NULL. */
int mahi_destroy(mahi_t h);

/* Change the stream later calls enqueue on. */
int mahi_set_stream(mahi_t h, void *cuda_stream);

/* Charges of the two forms and the site map (Sec. "Hamiltonian Interpolation
 * Formulation": sites, forms).  Arrays of length n_atoms, each in host or
 * device memory (detected per pointer): qA, qB (float64, e) and site_of_atom
 * (int32, -1 = environment, else 0..n_sites-1).  Environment atoms must have
 * qA == qB and every site must own 1 to 64 atoms, else MAHI_ERR_BAD_SITE_MAP.
 * The library copies the data; the call synchronises the handle's stream (the
 * site map is validated and indexed on the host). */
int mahi_set_charges(mahi_t h, const double *qA, const double *qB, const int32_t *site_of_atom);

/* New charges for the same site map, without a host round trip (for loops that
 * change the charges every step, e.g. charge gradients through autograd).
 * qA, qB: DEVICE arrays of n_atoms float64 (e).  Enqueued on the handle's
 * stream (one kernel, no synchronisation); the arrays may be reused once the
 * stream reaches the next evaluation.  Environment atoms carry qA only (their
 * qB is ignored, as the two forms of an environment atom are the same charge).
 * MAHI_ERR_STATE before mahi_set_charges; MAHI_ERR_INVALID_ARG for sites with
 * more than two forms (mahi_set_forms). */
int mahi_update_charges(mahi_t h, const double *qA, const double *qB);

/* Sites with more than two forms (general formulation, Eq. "iter_ham_lambda";
 * Appendix, Eqs. "lambda_list", "one_site_lambda").  Instead of
 * mahi_set_charges: HOST arrays
 *   q_env           n_atoms charges (e) of the environment atoms (entries of
 *                   site atoms are ignored)
 *   site_of_atom    n_atoms, -1 = environment, else the site (1 to 32 atoms)
 *   forms_per_site  n_sites values F_s in {2, 4, 8, 16}; site s then has
 *                   m_s = log2(F_s) lambdas
 *   q_forms         for each site in order, F_s rows (forms) of its atoms'
 *                   charges, atoms in increasing index: sum_s F_s n_s doubles
 * Form rho has weight prod_l (bit l of rho ? lambda_l : 1 - lambda_l) and the
 * site atoms the scaled charge sum_rho weight_rho q^rho.  mahi_eval then takes
 * lambda as sum_s m_s values (site 0's lambdas first, lambda_0 first) and
 * writes dE/dlambda in the same order; E adds per site
 *   C = f/2 [sum_rho w_rho G_rho,rho - w^T G w],  G = form-form matrix of the
 *   periodic kernel over the site's atoms (self term included),
 * and the forces its gradient.  mahi_n_lambdas gives the count.  A later
 * mahi_set_charges returns the handle to two-form sites.  Their backward pass
 * is mahi_backward_forms (mahi_backward returns MAHI_ERR_INVALID_ARG for
 * them).  Errors as for mahi_set_charges, and MAHI_ERR_INVALID_ARG for an F_s
 * outside the set. */
int mahi_set_forms(mahi_t h, const double *q_env, const int32_t *site_of_atom, const int32_t *forms_per_site,
                   const double *q_forms);
int mahi_n_lambdas(mahi_t h);

/* One MAHI evaluation, enqueued on the handle's stream; returns after enqueueing.
 * Its chain of kernels runs on an internal stream of the greatest priority and
 * its independent parts (the sites' pair terms, the box moments, the traversal
 * lists, the site-atom potential) on a second internal stream; both are forked
 * from and joined back to the handle's stream with events inside the call, so
 * the outputs are complete in the handle's stream order, work queued on that
 * stream before the call is seen, and the call can be captured in a CUDA graph.
 *   x          device, n_atoms x 3 row-major positions in nm (float64 if
 *              x_is_fp64 else float32); any real values (wrapped into the box).
 *   lambda     device, n_sites float64 in [0, 1].
 *   energy     device, 1 float64 (kJ/mol), HI energy.
 *   forces     device, n_atoms x 3 (same dtype as x), HI forces (kJ/mol/nm).
 *   dEdlambda  device, n_sites float64 (kJ/mol).
 * Outputs may be NULL to skip writing them (the work is still done). */
int mahi_eval(mahi_t h, const void *x, int32_t x_is_fp64, const double *lambda, double *energy,
              void *forces, double *dEdlambda);

/* The same evaluation from HOST buffers: copies x and lambda host->device,
 * evaluates, copies energy, forces and dE/dlambda device->host and synchronises
 * the stream before returning.  Pinned host memory gives the fastest copies. */
int mahi_eval_host(mahi_t h, const void *x_host, int32_t x_is_fp64, const double *lambda_host,
                   double *energy_host, void *forces_host, double *dEdlambda_host);

/* Backward pass of the HI energy of the LAST mahi_eval on this handle (for
 * reverse-mode differentiation, e.g. a torch.autograd.Function).  With
 * g = dLoss/dE (device, 1 float64) it writes, each output optional (NULL):
 *   dx       device, n_atoms x 3 (x dtype):  -g F   (F = the forces output of
 *            that evaluation, passed back in `forces`; dE/dx = -F)
 *   dlambda  device, n_sites float64:        g dE/dlambda (passed back in
 *            `dEdlambda`)
 *   dEdqA, dEdqB  device, n_atoms float64:   g dE/dqA_i, g dE/dqB_i with
 *       dE/dqA_i = (1 - l) phi~_i - l (1 - l) psi_i,  dE/dqB_i = l phi~_i + l (1 - l) psi_i
 *   for an atom of a site with lambda l (`lambda`: the same device array as in
 *   that evaluation), psi_i = f sum_{j in s} D_j A(x_i - x_j) (self term
 *   included), and dE/dqA_i = phi~_i, dE/dqB_i = 0 for environment atoms
 *   (they carry qA only).  These follow from E = E(q~) + sum_s 1/2 l_s (1 - l_s) k_s
 *   (Eqs. "DeltaFQIHI", "Udiff") with q~ = (1 - l) qA + l qB.
 * One kernel, enqueued on the handle's stream.  The potentials it uses are
 * overwritten by the next mahi_eval.  MAHI_ERR_INVALID_ARG if an output is
 * requested without its input; MAHI_ERR_STATE before mahi_set_charges. */
int mahi_backward(mahi_t h, const double *grad_energy, const void *forces, const double *dEdlambda,
                  const double *lambda, int32_t x_is_fp64, void *dx, double *dlambda, double *dEdqA, double *dEdqB);

/* Solver options (each has a default; value 0 restores it, except for
 * MAHI_OPT_M2L_SPLIT_DEGREE, whose default is 2).
 *   MAHI_OPT_SITE_THETA     separation ratio theta of the site-atom traversal:
 *       a box of circumradius a is used through its multipole at a site of
 *       radius R at distance D only if a < theta (D - R), so each multipole
 *       term converges at least like theta^(p+1).  Default
 *       theta(p) = 0.4^(13/(p+1)) clamped to [0.25, 0.4]: the truncation bound
 *       of p = 12 at theta = 0.4 held at orders 8 and up.  Range (0, 0.7].
 *   MAHI_OPT_SITE_LIST_CAP  boxes per level of one site's traversal (list
 *       capacity, 64 to 8192).  Default: 1536 at theta >= 0.4, else grown
 *       with the number of boxes a theta-ball holds.  A site that needs more
 *       fails with MAHI_ERR_SITE_OVERFLOW.  The traversal lists of compact
 *       sites are built once per evaluation in device buffers sized for this
 *       capacity: raising it after mahi_set_charges (directly, or by a smaller
 *       theta) reallocates them and synchronises the handle's streams.
 *   MAHI_OPT_WAIT_LIMIT_MS  limit of every bounded device wait of the
 *       tensor-core M2L and the site-atom potential (default 2000 ms, range 1
 *       to 60000).
 *   MAHI_OPT_WATCHDOG_SELFTEST  1: every following evaluation's tensor-core
 *       M2L makes its first wait on a barrier that nothing completes, so that
 *       the wait runs out after the wait limit and the evaluation reports
 *       MAHI_ERR_TIMEOUT (a test of the watchdog path; no fault is caused).
 *       0: off (default).
 *   MAHI_OPT_M2L_SPLIT_DEGREE  MAHI_MIXED only: the tensor-core M2L forms the
 *       products of the multipole coefficients in the K chunks (8 coefficients
 *       each) that hold input degrees l <= this value as three TF32 products
 *       (hi*hi + hi*lo + lo*hi, FP32-level operands), the rest as one (TF32
 *       operands rounded to nearest, relative rounding 2^-11 per term, on
 *       terms scaled by (a/R)^l).  Range -1..p: -1 = one product for every
 *       degree, p = three products throughout, default 2 (the first two
 *       chunks).  The products accumulate in FP32 in tensor memory, whose
 *       round-toward-zero additions (about -1 ulp each) bias the locals; fewer
 *       products per term means fewer additions.  The low degrees carry the
 *       charge and dipole of the sources, which set the far-field energy of
 *       charged configurations: one product there gives 1.8e-4 relative energy
 *       error on the 3,000-charge random system, three give 1.6e-5.
 * Launch shapes (results change only in the order of floating-point sums;
 * mahi_autotune sets them):
 *   MAHI_OPT_M2L_SINGLE_TILE  1: the tensor-core M2L uses single 128-row tiles
 *       per unit even where two fit (more, smaller units: better balance on
 *       small trees); 0: pairs where they fit (default).  Synchronises the
 *       handle's stream when it changes.
 *   MAHI_OPT_M2L_B_STAGES     operator stages of the tensor-core M2L: 2, 3 or 4
 *       (at most what fits in shared memory); 0 = as many as fit (default).
 *   MAHI_OPT_P2P_THREADS      threads per target leaf of the near field: 64,
 *       128 or 256 (0 = 128, the default).
 *   MAHI_OPT_SITE_BLOCKS      blocks per site of the site-atom traversal, 1 to
 *       16 (0 = about 3 per SM over all sites, one wave: the default).
 *   MAHI_OPT_P2P_TARGETS      near-field scheme of the single-precision paths:
 *       4 or 8 = every unordered pair of neighbouring atoms evaluated once
 *       (Newton's third law over the forward half shell of 13 neighbour
 *       leaves), with that many targets held per thread; -1 = every directed
 *       pair over all 27 neighbour leaves (block size MAHI_OPT_P2P_THREADS).
 *       0 = 8, the default.  The FP64 path always takes every directed pair.
 * MAHI_ERR_INVALID_ARG for an unknown option or a value out of range. */
enum {
  MAHI_OPT_SITE_THETA = 1,
  MAHI_OPT_SITE_LIST_CAP = 2,
  MAHI_OPT_WAIT_LIMIT_MS = 3,
  MAHI_OPT_WATCHDOG_SELFTEST = 4,
  MAHI_OPT_M2L_SPLIT_DEGREE = 5,
  MAHI_OPT_M2L_SINGLE_TILE = 6,
  MAHI_OPT_M2L_B_STAGES = 7,
  MAHI_OPT_P2P_THREADS = 8,
  MAHI_OPT_SITE_BLOCKS = 9,
  MAHI_OPT_P2P_TARGETS = 10
};
int mahi_set_option(mahi_t h, int32_t option, double value);
/* Current value of an option (the effective one for defaults). */
double mahi_get_option(mahi_t h, int32_t option);

/* Backward pass for sites with 2^m forms (mahi_set_forms), the counterpart of
 * mahi_backward.  dx and dlambda as there (dlambda has mahi_n_lambdas entries);
 * the charge gradients follow the mahi_set_forms layout:
 *   dEdq_env    device, n_atoms float64: g phi~_i for environment atoms, 0 for
 *               site atoms (their q_env entries are not used)
 *   dEdq_forms  device, sum_s F_s n_s float64 (site by site, F_s rows of its
 *               atoms' entries, as q_forms): g w_r (phi~_i + psi^r_i - sum_r' w_r' psi^r'_i)
 * with w_r the form weights prod_l (bit l of r ? lambda_l : 1 - lambda_l) and
 * psi^r_i = f sum_{j in s} A(x_i - x_j) q^r_j (self term included), from
 * E = E(q~) + sum_s f/2 [sum_r w_r G_rr - w^T G w], G_rr' = q^r^T A q^r'
 * (Eq. "iter_ham_lambda", Eq. "one_site_lambda").  Uses the last evaluation's
 * potentials; MAHI_ERR_INVALID_ARG on a two-form handle or an output without
 * its input; MAHI_ERR_STATE before the charges are set. */
int mahi_backward_forms(mahi_t h, const double *grad_energy, const void *forces, const double *dEdlambda,
                        const double *lambda, int32_t x_is_fp64, void *dx, double *dlambda, double *dEdq_env,
                        double *dEdq_forms);

/* Charge-scaled potential phi~ (kJ/mol/e, float64, original atom order) of the
 * last evaluation into a device buffer of n_atoms doubles (enqueued). */
int mahi_get_potential(mahi_t h, double *phi_device);

/* Stage timing (CUDA events).  mahi_set_timing(h, 1) turns recording on;
 * mahi_stage_times fills up to n floats (ms) of the last evaluation in the
 * order of mahi_stage_name(i) and returns the stage count.  The first ten are
 * consecutive intervals of the evaluation's chain (bin, sort, p2m, m2m, lattice,
 * m2l, l2l, near_pairs, far_near_out, site): near_pairs is the half-shell
 * near-field pair kernel and far_near_out the far field (L2P) fused with the
 * near-field sums and the outputs; in the directed near-field scheme
 * (MAHI_OPT_P2P_TARGETS = -1, and the FP64 path) they are L2P and the 27-leaf
 * near field with the outputs.  The last two are the internal side stream's work,
 * which overlaps them: side_site_pairs (the sites' FP64 pair terms, from the
 * start of the evaluation) and side_site_potential (the refined site-atom
 * potential, after the M2L), 0 when there are no sites.  It synchronises the
 * streams.  Timing is meant for eager evaluations, not for captured ones. */
int mahi_set_timing(mahi_t h, int32_t on);
int mahi_stage_times(mahi_t h, float *ms, int32_t n);
const char *mahi_stage_name(int32_t i);

/* Number of kernels the last evaluation launched. */
int mahi_launch_count(mahi_t h);

/* ---- host-only helpers (no device needed) ---------------------------------
 * Far-image lattice functions of the periodic kernel A (Eq. "approx_nbody_periodic",
 * lattice part L(omega)):
 *   H_K(r) = A(r) - sum_{|n|_inf<=K} 1/|r + nL| - (2 pi/3V)|r|^2,  harmonic for |r| < (K+1)L.
 * shell K = 1 is the paper's split (first image shell direct); K = 3 is the
 * function this library's root lattice operator uses (images 2..3 by M2L).
 * mahi_lattice_coeffs writes the solid-harmonic Taylor coefficients of H_K for
 * the unit box up to degree 2*order_p (real layout, (2*order_p+1)^2 doubles,
 * index l*l for m = 0, l*l + 2m - 1 / l*l + 2m for Re/Im of m > 0;
 * H(r) = sum_lm c_lm conj(R_lm(r)) with the scaled regular solid harmonics
 * R_00 = 1, R_mm = -(x+iy)/(2m) R_{m-1,m-1}, R_lm = ((2l-1) z R_{l-1,m} - r^2 R_{l-2,m})/((l+m)(l-m))).
 * mahi_lattice_eval evaluates H_K at n points r (n x 3, host, nm) for box edge L
 * with that degree into H (n, host, 1/nm).  K must be 1 or 3.  Deterministic. */
int mahi_lattice_coeffs(int32_t order_p, int32_t shell, double *coeffs);
int mahi_lattice_eval(double box_L_nm, int32_t order_p, int32_t shell, int64_t n, const double *r, double *H);

/* Per-site HI terms without any device allocation.  The paper has no
 * counterpart to this entry point: it is for callers that cannot allocate
 * device memory at the point where they need the terms (code running while a
 * stream is captured, programs whose device memory belongs to another
 * runtime or a fixed pool, or MD engines that compute the charge-scaled
 * potential phi~ with their own solver).  It runs the per-site stage of
 * mahi_eval (k_s, dE/dlambda, energy and force corrections) on
 * caller-provided inputs; its only scratch is a file-scope device array.
 *   n_atoms     length of the per-atom arrays below (>= 1 when n_sites > 0)
 *   site_ptr    device, n_sites + 1 int32 (CSR offsets into site_atoms)
 *   site_atoms  device, site_ptr[n_sites] int32 atom indices; every site has
 *               1..64 atoms with indices in [0, n_atoms).  A malformed site
 *               (offsets out of order or beyond site_ptr[n_sites], a size
 *               outside 1..64, an atom index out of range) is checked before
 *               any per-atom array is read: its dE/dlambda and its energy
 *               slot become NaN and none of its atoms is touched.
 *   x           device, positions (float64 if x_is_fp64 else float32), n_atoms x 3
 *   qA, qB      device float64 charges of the two forms (indexed by atom)
 *   lambda      device, n_sites float64
 *   phi         device float64 charge-scaled potential phi~ (kJ/mol/e) per atom,
 *               e.g. from mahi_get_potential after mahi_eval
 *   dEdlambda   device, n_sites float64 (out; may be NULL)
 *   energy_correction  device, 1 float64 (out; sum_s 1/2 lam(1-lam) k_s; may be NULL)
 *   forces      device, n x 3 in the x dtype: the intra-site force corrections are
 *               ADDED to the values already there for site atoms (may be NULL)
 * Limits: n_sites <= 4096 (the scratch holds one energy slot per site, 32 KiB),
 * else MAHI_ERR_INVALID_ARG.  The first call on a device (with that device
 * current) resolves the scratch address and fills its lattice tables
 * synchronously; make it before any stream capture.  Later calls only enqueue
 * kernels on cuda_stream.  Calls share the scratch: calls that overlap on the
 * GPU race. */
int mahi_site_terms_static(double box_L_nm, int64_t n_atoms, int32_t n_sites, const int32_t *site_ptr,
                           const int32_t *site_atoms,
                           const void *x, int32_t x_is_fp64, const double *qA, const double *qB,
                           const double *lambda, const double *phi, double *dEdlambda, double *energy_correction,
                           void *forces, void *cuda_stream);

/* ---- batched replicas and launch-shape tuning -------------------------------
 * Independent constant-pH replicas (each its own handle: box, atoms, sites,
 * lambdas) evaluated as ONE CUDA graph.  mahi_batch_create sets every handle's
 * stream to cuda_stream (which must not be the legacy NULL stream), runs one
 * ordinary evaluation per replica, then captures the n evaluations into a
 * graph with the given device buffers (arrays of n pointers, same meaning as
 * in mahi_eval), each replica on its own branch forked from and joined back
 * into cuda_stream, so the replicas' kernels run side by side.  mahi_batch_launch enqueues the graph on that
 * stream (one host call for all replicas); results equal n mahi_eval calls.
 * The graph keeps the captured pointers: update positions and lambdas in place
 * between launches; changing charges or tuning needs a new batch.  The batch
 * does not own the handles (destroy it before them).  The paper has no
 * counterpart (its benchmarks run one system per process). */
typedef struct mahi_batch_ctx *mahi_batch_t;
int mahi_batch_create(const mahi_t *handles, int32_t n, void *cuda_stream, const void *const *x,
                      const int32_t *x_is_fp64, const double *const *lambda, double *const *energy,
                      void *const *forces, double *const *dEdlambda, mahi_batch_t *out);
int mahi_batch_launch(mahi_batch_t b);
int mahi_batch_destroy(mahi_batch_t b);

/* Launch-shape autotuner: times reps evaluations (outputs discarded) for each
 * candidate shape on the given input and keeps the fastest in the handle:
 * first the near-field kernel (64, 128 or 256 threads per target leaf) with
 * the site-potential traversal (default blocks per site, half, double), then,
 * for MAHI_MIXED, the tensor-core M2L's tiling (paired or single 128-row tiles)
 * with its operator stage count (as many as fit, 3, 2).  Synchronises the
 * handle's stream.  Results change only in the order of floating-point sums.
 * mahi_get_tuning reports the first two choices (site_blocks 0 = the default
 * count); mahi_get_option reports all of them (MAHI_OPT_M2L_SINGLE_TILE, ...). */
int mahi_autotune(mahi_t h, const void *x, int32_t x_is_fp64, const double *lambda, int32_t reps);
int mahi_get_tuning(mahi_t h, int32_t *p2p_threads, int32_t *site_blocks);

/* Coulomb constant used by the library (kJ mol^-1 nm e^-2). */
double mahi_coulomb_constant(void);

const char *mahi_error_string(int code);
/* Text of the last CUDA error seen by any handle in this process. */
const char *mahi_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MAHI_H */
