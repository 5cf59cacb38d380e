/*
 * tm.h -- C ABI of the GB300 (sm_103a) library for the one-flavour Wilson
 * twisted-mass Dirac operator and its even/odd-preconditioned CG solve,
 * following Jansen & Urbach, "tmLQCD: a program suite to simulate Wilson
 * twisted mass lattice QCD" (arXiv:0905.3331).
 *
 * The operator (eq. eo0, App. B.1, hopping-parameter form, Wilson r = 1):
 *
 *   (M psi)(x) = [1 + i f mu~ gamma5] psi(x)
 *                - kappa sum_{mu=t,x,y,z} [ U_mu(x) (1 + gamma_mu) psi(x + mu^)
 *                                          + U_mu(x - mu^)^dag (1 - gamma_mu) psi(x - mu^) ]
 *
 * with mu~ = 2 kappa mu (mu = bare twisted mass mu_q), flavour sign f = +1
 * ("up", tau3 = +1) or -1, gamma matrices of App. A (chiral basis,
 * gamma5 = diag(1, 1, -1, -1)).  M relates to D_tm of eq. Dtm by
 * D_tm = M / (2 kappa) with m0 = 1/(2 kappa) - 4.  Gauge links are periodic;
 * fermions are antiperiodic in time and periodic in space (Sec. 2.4 with
 * theta = (1, 0, 0, 0)): the whole phase -1 sits on the hop across t = T-1 <-> 0.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * Lattice   T x L^3, T and L even and >= 2.  Site index lex = ((t L + z) L + y) L + x
 *           (index order t, z, y, x, spin, colour of Sec. 4.7.2).  Direction mu = 0:t,
 *           1:x, 2:y, 3:z.  Parity (t + x + y + z) mod 2, even = 0.  V = T L^3, h = V/2.
 * Canonical full field   V x 4 x 3 complex FP64 (24 doubles per site, re then im),
 *           [lex][spin][colour].  nrhs fields are stacked back to back.
 * Canonical gauge field  V x 4 x 3 x 3 complex FP64, [lex][mu][row][col] (72 doubles/site).
 * Half field (device layout) -- one parity p, site index cb = lex / 2 over the
 *           sites of parity p in lexicographic order (0 <= cb < h):
 *   TM_F64  double2 blocks [12][h]: block k = complex component 3*spin + colour.   192 h bytes
 *   TM_F32  float4  blocks [6][h]: block j = components 2j, 2j+1 (re, im, re, im). 96 h bytes
 *   TM_F16  uint4   blocks [3][h]: block j = components 4j..4j+3 as 8 IEEE halves
 *           (re, im, ...), then float norm[h]; value = half * norm[cb], where norm is
 *           the site's largest |re| or |im|.                                     52 h bytes
 *   TM_DF64 float4  blocks [12][h]: block k = (re.hi, re.lo, im.hi, im.lo) of component k,
 *           value = hi + lo.                                                   192 h bytes
 *   nrhs half fields are stacked back to back (stride tm_half_field_bytes()).
 * Pointers  "device" pointers are CUDA device (or managed) memory of the current
 *           device.  Arguments named "host or device" are classified with
 *           cudaPointerGetAttributes: host memory (pinned or pageable) is staged through
 *           lattice-owned device buffers, with both copies ordered on `stream`.
 * Streams   `stream` is a cudaStream_t (NULL = legacy default stream).  Every call is
 *           ordered on it; calls return once the work is enqueued unless stated
 *           otherwise.  The caller owns every buffer it passes; the lattice owns its
 *           gauge copies and work space.  One lattice must not be used from two host
 *           threads or two streams at the same time.
 * Errors    Every call returns a tm_status and never aborts or exits; on failure
 *           tm_last_error() gives a message (per host thread).  Device-side conditions
 *           (non-finite values, a solver that did not converge, a device wait that ran
 *           out) are reported through status words that the library reads back.
 */
#ifndef TM_H
#define TM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tm_lattice_s *tm_lattice;

typedef enum {
  TM_OK = 0,
  TM_ERR_ARG = 1,           /* invalid argument (null pointer, bad enum, aliasing, ...) */
  TM_ERR_ODD_EXTENT = 2,    /* T or L odd or < 2 */
  TM_ERR_NO_GAUGE = 3,      /* operator requested before tm_set_gauge */
  TM_ERR_NOT_SU3 = 4,       /* a link fails |U^dag U - 1| or |det U - 1| <= 1e-10 */
  TM_ERR_NONFINITE = 5,     /* NaN or Inf in an input */
  TM_ERR_CUDA = 6,          /* a CUDA runtime call failed */
  TM_ERR_NOT_CONVERGED = 7, /* max_iter reached; the last iterate is returned */
  TM_ERR_TIMEOUT = 8,       /* a bounded device-side wait gave up */
  TM_ERR_OOM = 9,           /* device allocation failed */
  TM_ERR_UNSUPPORTED = 10   /* a precision / link-format combination that is not built */
} tm_status;

/* Spinor storage precision.  TM_DF64 ("double-float") stores each real as two FP32 numbers
 * hi + lo and computes in double-word arithmetic on the FP32 units (about 48 significant
 * bits); a form of this library with no counterpart in the paper.  (Measured on GB300 the
 * double-word kernel is not faster than native FP64: 226 vs 173 us on 16^3 x 32.) */
typedef enum { TM_F64 = 0, TM_F32 = 1, TM_F16 = 2, TM_DF64 = 3 } tm_prec;

/* Gauge-link storage: 18 reals, 12 (rows 1-2; row 3 = conj(row1 x row2)) or 8
 * (a 2-row/column parametrisation of SU(3), reconstructed in registers).  Links
 * are stored in the precision of the spinors they act on (FP64, FP32, FP16, double-float;
 * double-float supports 18 reals only, with one thread per site). */
typedef enum { TM_LINK18 = 18, TM_LINK12 = 12, TM_LINK8 = 8 } tm_link;

/* ---------------------------------------------------------------- lattice --- */

/* Creates a T x L^3 lattice with hopping parameter kappa and bare twisted mass mu
 * (mu~ = 2 kappa mu; eq. eo0).  No gauge field yet.  Errors: TM_ERR_ODD_EXTENT,
 * TM_ERR_ARG (out == NULL, non-finite kappa/mu), TM_ERR_CUDA. */
tm_status tm_lattice_create(int T, int L, double kappa, double mu, tm_lattice *out);

/* Frees every device buffer of the lattice (synchronises the device first). NULL is a no-op. */
tm_status tm_lattice_destroy(tm_lattice lat);

/* Changes kappa and mu (the gauge copies stay valid). */
tm_status tm_lattice_set_params(tm_lattice lat, double kappa, double mu);

/* Sizes: V, and the bytes of one half field of precision `prec` (see the layout above). */
size_t tm_volume(tm_lattice lat);
size_t tm_half_field_bytes(tm_lattice lat, tm_prec prec);

/* Launch configuration of the hopping kernel for one storage form (a tuning knob; no paper
 * counterpart).  Each output site's 8 hops are shared by 1, 2 or 4 threads (the partial sums
 * are added in a fixed order); more threads per site keep more memory requests in flight on
 * lattices too small to fill the GPU.  The value 3 (TM_HOP_PIPELINED, FP32 and FP16 storage
 * only) selects one thread per site whose loads of the next hop are issued before the current
 * hop's arithmetic.  The value 5 (TM_HOP_PAIRED, FP32 and FP16 storage only) selects one thread
 * per TWO sites whose FP32 arithmetic runs on packed pairs (one instruction for both sites).
 * By default the library times the choices when the form's gauge copy is first built and keeps
 * the fastest, for the rest of the process, for every lattice of the same extents on the same
 * device (the environment variable TM_HOP_TPS=1|2|3|4|5 overrides that for every form).
 * tm_set_hop_threads fixes the choice (0 = time again if the form's gauge copy exists, and
 * keep the new choice for later lattices of these extents); tm_get_hop_threads reports it.
 * Results for different choices agree to rounding; for one fixed choice they are bitwise
 * reproducible.  Errors: TM_ERR_ARG, TM_ERR_UNSUPPORTED (3 or 5 with FP64 or double-float
 * storage, 2 or 4 with double-float). */
#define TM_HOP_PIPELINED 3
#define TM_HOP_PAIRED 5
tm_status tm_set_hop_threads(tm_lattice lat, tm_prec prec, tm_link link, int threads_per_site);
int tm_get_hop_threads(tm_lattice lat, tm_prec prec, tm_link link);

/* Copies the canonical FP64 gauge field U (host or device; 72 V doubles) into the
 * lattice, checks that every link is SU(3) (|U^dag U - 1|_max and |det U - 1| <= 1e-10,
 * all entries finite) and builds the parity-split "gauge copy" of Sec. 4.1 in device
 * memory: per parity and direction, the links U_mu(x) of the sites of that parity in the
 * order the hopping kernel reads them (the backward hop reads U_mu(x - mu^) of the
 * neighbour, of the other parity, and applies its adjoint).  Reduced-precision and
 * compressed copies are built on first use.  Synchronises `stream`.
 * Errors: TM_ERR_NOT_SU3 (nothing is changed), TM_ERR_NONFINITE, TM_ERR_ARG, TM_ERR_CUDA, TM_ERR_OOM. */
tm_status tm_set_gauge(tm_lattice lat, const double *U, void *stream);

/* ------------------------------------------------------- field conversion --- */

/* Canonical FP64 half field(s) -> device half field(s) of precision `prec`.
 * src: host or device, nrhs x h x 24 doubles, site order cb (= lex/2 over one parity).
 * dst: device, nrhs x tm_half_field_bytes(prec).  FP32 / FP16 round to nearest. */
tm_status tm_pack_half(tm_lattice lat, tm_prec prec, void *dst, const double *src, int nrhs,
                       void *stream);
/* Inverse of tm_pack_half: device half field(s) -> canonical FP64 (host or device). */
tm_status tm_unpack_half(tm_lattice lat, tm_prec prec, double *dst, const void *src, int nrhs,
                         void *stream);

/* ---------------------------------------------------------------- operator --- */

/* out = M(f) in on the full lattice (eq. eo0), or M(f)^dag in if dagger != 0
 * (M^dag = gamma5 M(-f) gamma5).  in, out: canonical full fields, host or device,
 * nrhs x 24 V doubles; out must not overlap in.  Computed in FP64 with 18-real links.
 * Errors: TM_ERR_NO_GAUGE, TM_ERR_ARG (flavour not +-1, aliasing), TM_ERR_CUDA. */
tm_status tm_apply_D(tm_lattice lat, double *out, const double *in, int flavour, int dagger,
                     int nrhs, void *stream);

/* out_p = H_{p,1-p} in: the pure hopping sum of eq. eo0 (without -kappa) onto the sites
 * of parity out_parity, from the half field of the other parity (H_eo / H_oe of eq. eo2;
 * M_eo = -kappa H_eo).  in, out: device half fields of precision `prec`, nrhs of them;
 * out must not overlap in.  Links in format `link` (built on first use).  Arithmetic is
 * FP64 for TM_F64 and FP32 otherwise.  The spin projection (1 +- gamma_mu) is applied
 * before the SU(3) multiply (Sec. 4.1), so each hop multiplies two colour vectors.
 * Errors: TM_ERR_NO_GAUGE, TM_ERR_ARG, TM_ERR_UNSUPPORTED, TM_ERR_CUDA. */
tm_status tm_apply_hopping_eo(tm_lattice lat, int out_parity, void *out, const void *in,
                              tm_prec prec, tm_link link, int nrhs, void *stream);

/* out = (M_ee^f)^{-1} in = (1 - i f mu~ gamma5) / (1 + mu~^2) in, site by site (eq. eo3).
 * in, out: device half fields of precision `prec` (either parity: M_ee = M_oo), nrhs of
 * them; in == out is allowed.  Errors: TM_ERR_ARG, TM_ERR_CUDA. */
tm_status tm_apply_Mee_inv(tm_lattice lat, void *out, const void *in, int flavour, tm_prec prec,
                           int nrhs, void *stream);

/* ------------------------------------------------------------------ solver --- */

typedef enum {
  TM_CG_FP64 = 0,     /* CG in FP64 throughout */
  TM_CG_SQRT_EPS = 1, /* Sec. 4.4: FP64 until ||r|| < sqrt(tol) ||b||, then the sloppy
                         operator; a final FP64 defect correction keeps the true residual */
  TM_CG_RELIABLE = 2  /* sloppy CG with reliable updates: FP64 true residual and FP64
                         solution accumulation whenever ||r|| falls by a factor delta */
} tm_cg_mode;

typedef struct {
  double tol;           /* relative: stop when ||b - A X|| / ||b|| < tol, b = gamma5 varphi_o */
  int max_iter;         /* total CG iterations (all precisions) */
  int mode;             /* tm_cg_mode */
  int sloppy_prec;      /* tm_prec of the sloppy operator (modes 1, 2) */
  int sloppy_link;      /* tm_link of the sloppy operator (modes 1, 2) */
  double delta;         /* reliable-update trigger (mode 2), e.g. 0.1 */
  int use_x0;           /* nonzero: x holds the initial guess (full field) */
  int flavour;          /* +1 solves M(+mu) x = b, -1 solves M(-mu) x = b; 0 means +1 */
  int update_prec;      /* modes 1, 2: arithmetic of the residual recomputations inside the
                           loop: TM_F64; TM_DF64 (double-float; about 48 bits, on the FP32
                           units); or TM_F32 (for FP16 storage): each update at delta computes
                           r = r64 - A dx with the FP32 operator, r64 the last FP64 residual and
                           dx the FP32 increment since then, and the FP64 recomputation follows
                           once ||r|| has fallen by 1e-2 since the last one.  Convergence is
                           always confirmed in FP64; if that fails the solve continues with FP64
                           recomputations. */
} tm_cg_params;

typedef struct {
  int iters;                 /* CG iterations performed (all precisions) */
  int reliable_updates;      /* FP64 residual recomputations inside the loop */
  double true_rel_residual;  /* ||b - M x|| / ||b|| on the full lattice, FP64, recomputed */
  double schur_rel_residual; /* ||b_o - A X|| / ||b_o|| of the normal equations, FP64 (mixed
                                modes: the odd part of the FP64 full-system residual, which
                                equals it up to the rounding of x_e) */
  double seconds;            /* wall time of the call */
  int status;                /* tm_status of the solve */
} tm_cg_info;

/* Solves M(f) x = b on the full lattice by even/odd preconditioning (App. B.2): source
 * preparation varphi_o = b_o - M_oe (M_ee)^{-1} b_e, CG on Qhat^f Qhat^-f X = gamma5 varphi_o
 * (eq. eo6), x_o = Qhat^-f X, x_e = (M_ee)^{-1}(b_e - M_eo x_o).  x, b: canonical full
 * fields, host or device, nrhs x 24 V doubles.  Convergence is decided by an FP64 residual:
 * in the mixed modes, once a sloppy stage reaches tol, by the FP64 residual of the full
 * system that the reconstruction computes (its odd part is ||b' - A X|| up to the rounding
 * of x_e); if that misses tol the iteration continues.  With mode TM_CG_RELIABLE, FP64
 * updates and no initial guess, nrhs > 1 systems are solved together by tm_solve_cg_batch
 * (shared launches); otherwise one after another.  Synchronises
 * `stream` to fill `info` (may be NULL; with nrhs > 1 it describes the worst system).
 * Errors: TM_ERR_NOT_CONVERGED (x holds the last iterate), TM_ERR_NO_GAUGE, TM_ERR_ARG,
 * TM_ERR_NONFINITE, TM_ERR_CUDA, TM_ERR_OOM. */
tm_status tm_solve_cg(tm_lattice lat, double *x, const double *b, int nrhs,
                      const tm_cg_params *params, tm_cg_info *info, void *stream);

/* Solves M(f) x = b like tm_solve_cg, with the stabilised bi-conjugate gradient method
 * (BiCGstab, one of the solvers of Sec. 4.4) applied directly to the non-hermitian Schur
 * system of eq. eo4 instead of CG on the normal equations:
 *   Mhat^f x_o = varphi_o,  Mhat^f = (1 + i f mu~ gamma5) - kappa^2 H_oe (M_ee^f)^{-1} H_eo,
 * varphi_o = b_o - M_oe (M_ee^f)^{-1} b_e, x_e = (M_ee^f)^{-1}(b_e - M_eo x_o) (App. B.2).
 * One iteration applies Mhat twice, the cost of one CG iteration on Qhat^f Qhat^-f.
 * Arguments, staging, nrhs and use_x0 as tm_solve_cg; params->mode TM_CG_FP64 (BiCGstab in
 * FP64, restarted from the recomputed residual if the iterated one drifted) or TM_CG_RELIABLE
 * (sloppy storage and FP32 arithmetic with FP64 reliable updates every factor delta; p and
 * the shadow residual carry across updates); max_iter counts BiCGstab iterations.  tol is
 * relative to ||varphi_o|| (info->schur_rel_residual) and the full-lattice residual is
 * reported as in tm_solve_cg.  Breakdowns (a vanishing <r^, v>, omega or rho) restart the
 * method from the FP64 residual.
 * Errors: as tm_solve_cg, plus TM_ERR_UNSUPPORTED for TM_CG_SQRT_EPS or TM_DF64 updates. */
tm_status tm_solve_bicgstab(tm_lattice lat, double *x, const double *b, int nrhs,
                            const tm_cg_params *params, tm_cg_info *info, void *stream);

/* Solves M(f) x = b like tm_solve_bicgstab with the minimal residual iteration (MR, one of the
 * solvers of Sec. 4.4) on the Schur system Mhat^f x_o = varphi_o of eq. eo4:
 *   q = Mhat r,  alpha = <q, r> / <q, q>,  x += alpha r,  r -= alpha q
 * (alpha minimises ||r - alpha q||; one Schur application per iteration).  Arguments, staging,
 * nrhs, use_x0 and info as tm_solve_cg; params->mode TM_CG_FP64 or TM_CG_RELIABLE with
 * sloppy_prec TM_F32 (18/12/8 links; r feeds the operator, so FP16 storage is not offered).
 * Like BiCGstab it needs the spectrum of Mhat on one side of the origin (see tm_solve_bicgstab).
 * Errors: as tm_solve_cg, plus TM_ERR_UNSUPPORTED for TM_CG_SQRT_EPS, TM_DF64 updates or FP16. */
tm_status tm_solve_mr(tm_lattice lat, double *x, const double *b, int nrhs, const tm_cg_params *params,
                      tm_cg_info *info, void *stream);

/* One system of a batched solve: M(f; mu) x = b on the lattice `lat` (its gauge field and
 * kappa), with this system's own bare twisted mass mu (mu~ = 2 kappa mu). */
typedef struct {
  tm_lattice lat;
  double mu;
  int flavour;     /* +1 or -1 (0 means +1) */
  double *x;       /* solution: canonical full field, device memory */
  const double *b; /* source: canonical full field, device memory */
} tm_system;

/* Solves many systems together (the paper's inversions of many sources, e.g. the 12 spin-
 * colour point sources of a propagator, Sec. 4.7.2, or sources on several lattices): the
 * mixed-precision reliable-update CG of tm_solve_cg (params->mode must be TM_CG_RELIABLE;
 * FP32 or FP16 sloppy storage; FP64 updates), with the sloppy iterations of every system in
 * the same kernel launches -- blocks of systems that share a lattice interleaved so each
 * link is read from HBM once per iteration for all of them.  The whole solve is ONE CUDA
 * graph launch: a loop over the batched iteration, each followed, when some system has reached
 * its reliable-update trigger (or its sloppy residual met tol, or it diverged or overflowed),
 * by the FP64 reliable update of those systems in batched kernels (X += x, r = b' - A X in FP64)
 * and the decision to finish or resume each.  A system is converged when that FP64 residual
 * ||b' - A X|| / ||b'|| is below tol; the full-system FP64 residual is then computed once per
 * system after the loop (true_rel_residual).  Every system keeps its own CG scalars and stops
 * on its own residual; infos[k] (may be NULL) receives system k's result (seconds = the whole
 * call).  Systems may share lattices and differ in mu, flavour and source.  The hopping
 * launches' split -- one system per thread with 1, 2 or 4 threads per site, or 2 or 4 systems
 * of one lattice per thread sharing each link -- is timed on the batch's own vectors at the
 * first call of a batch shape and cached (TM_BATCH_TPS=1|2|4 or TM_BATCH_K=2|4 in the
 * environment fixes it).  Synchronises `stream`.  Allocates its work space (about 1.9 kB per odd site per system with FP32
 * storage, plus 0.8 kB per odd site per lattice) for the duration of the call.
 * Errors: TM_ERR_NOT_CONVERGED (some systems; their x holds the last iterate), TM_ERR_ARG,
 * TM_ERR_UNSUPPORTED, TM_ERR_NO_GAUGE, TM_ERR_NONFINITE, TM_ERR_CUDA, TM_ERR_OOM. */
tm_status tm_solve_cg_batch(const tm_system *systems, int nsys, const tm_cg_params *params,
                            tm_cg_info *infos, void *stream);

/* Solves the normal equations of the odd-site Schur operator directly (eq. eo6),
 *   A X = phi,   A = Qhat^f Qhat^-f = gamma5 Mhat^f gamma5 Mhat^-f,  Qhat^f = gamma5 Mhat^f,
 * the solve that the HMC force of the twisted-mass pseudofermion needs (X = (Qhat^+ Qhat^-)^-1
 * phi, App. B.1), with the CG and the mixed-precision modes of tm_solve_cg.
 * X, phi: FP64 odd-parity half fields in DEVICE memory (the layout of tm_pack_half, TM_F64),
 * distinct.  params->use_x0 nonzero: X holds the initial guess (e.g. from tm_chrono_guess);
 * otherwise X is overwritten from zero.  params->flavour picks f (0 means +1).  tol is relative
 * to ||phi||.  info (may be NULL): iters, reliable_updates, schur_rel_residual =
 * true_rel_residual = ||phi - A X|| / ||phi||, recomputed in FP64.  Synchronises `stream`.
 * Errors: TM_ERR_NOT_CONVERGED (X holds the last iterate), TM_ERR_NO_GAUGE, TM_ERR_ARG,
 * TM_ERR_NONFINITE, TM_ERR_CUDA, TM_ERR_OOM. */
tm_status tm_solve_normal(tm_lattice lat, void *X, const void *phi, const tm_cg_params *params,
                          tm_cg_info *info, void *stream);

/* Chronological solver guess (Sec. 4.2, eq. chrono): from n earlier solutions chi_i of
 * A X = phi (A as in tm_solve_normal, flavour f), solves
 *   sum_i <chi_j, A chi_i> c_i = <chi_j, phi>    (j = 0 .. n-1; conjugate on chi_j)
 * for the c_i -- the X0 in the span of the chi_i that minimises the A-norm of the error, the
 * functional CG minimises -- and writes X0 = sum_i c_i chi_i.  The n x n system (hermitian)
 * is solved on the host in FP64 by Gaussian elimination with partial pivoting; a direction
 * whose pivot falls below 1e-13 max|G| (a linearly dependent history) gets c = 0.
 * X0, phi, chi[i]: FP64 odd half fields in DEVICE memory; chi is a HOST array of n pointers;
 * 0 <= n <= 64 (n = 0 gives X0 = 0).  X0 must not alias any chi[i].  Costs n applications
 * of A and n(n+1)/2 + n inner products.  Synchronises `stream` once (to read the n x n
 * matrix).  Errors: TM_ERR_ARG, TM_ERR_NO_GAUGE, TM_ERR_NONFINITE, TM_ERR_CUDA. */
tm_status tm_chrono_guess(tm_lattice lat, void *X0, const void *const *chi, int n, const void *phi,
                          int flavour, void *stream);

/* ------------------------------------------------ non-degenerate doublet --- */

/* The mass non-degenerate flavour doublet of eq. Dh, D_h = D_W 1_f + i mubar gamma5 tau3 +
 * epsbar tau1, in the hopping-parameter form of eq. eo0 (M_h = 2 kappa D_h, m0 = 1/(2 kappa) - 4):
 *   (M_h psi)(x) = [1 + i mb gamma5 tau3 + eb tau1] psi(x) - kappa (H psi)(x),
 *   mb = 2 kappa mubar, eb = 2 kappa epsbar (mubar, epsbar bare, like mu in tm_lattice_create),
 * H the hopping sum of eq. eo0 on each flavour; tau_k the Pauli matrices of App. A.  A doublet
 * field is two canonical full fields back to back (2 x 24 V doubles): the upper flavour
 * (tau3 = +1) first.  Uses the lattice's kappa and gauge field (its mu is ignored).
 * Requires 1 + mb^2 - eb^2 > 0 (the site term is invertible), else TM_ERR_ARG.
 * in, out: host or device, nrhs doublet fields, no overlap.  Computed in FP64 on both parities.
 * Errors: TM_ERR_NO_GAUGE, TM_ERR_ARG, TM_ERR_CUDA. */
tm_status tm_apply_Dh(tm_lattice lat, double *out, const double *in, double mubar, double epsbar,
                      int nrhs, void *stream);

/* Solves M_h x = b for one doublet field (host or device) by even/odd preconditioning (the block
 * elimination of App. B.1 with the doublet's site term D = 1 + i mb gamma5 tau3 + eb tau1,
 * D^{-1} = (1 - i mb gamma5 tau3 - eb tau1) / (1 + mb^2 - eb^2)):
 *   Mhat_h = D - kappa^2 H_oe D^{-1} H_eo (odd sites),  varphi_o = b_o + kappa H_oe D^{-1} b_e,
 *   CG on Qhat_h^2 y = gamma5 tau1 varphi_o with the hermitian Qhat_h = gamma5 tau1 Mhat_h
 *   (Mhat_h^dag = tau1 gamma5 Mhat_h gamma5 tau1, Sec. 2.3), x_o = Qhat_h y,
 *   x_e = D^{-1}(b_e + kappa H_eo x_o).
 * params: tol, max_iter, mode TM_CG_FP64 or TM_CG_RELIABLE with sloppy_prec TM_F32 (18/12/8
 * links) and FP64 reliable updates; use_x0 must be 0 (TM_ERR_UNSUPPORTED otherwise).
 * info as for tm_solve_cg (schur_rel_residual relative to ||varphi_o||, true_rel_residual the
 * full-lattice FP64 residual).  Synchronises `stream`.
 * Errors: TM_ERR_NOT_CONVERGED (x holds the last iterate), TM_ERR_NO_GAUGE, TM_ERR_ARG,
 * TM_ERR_UNSUPPORTED, TM_ERR_NONFINITE, TM_ERR_CUDA, TM_ERR_OOM. */
tm_status tm_solve_doublet(tm_lattice lat, double *x, const double *b, double mubar, double epsbar,
                           const tm_cg_params *params, tm_cg_info *info, void *stream);

/* ---------------------------------------------------------------- contractions --- */

/* Meson contraction of a point-source propagator, for the correlators of Sec. 4.3 (one-end
 * trick; gamma5-hermiticity G_u(0,x) = gamma5 G_d(x,0)^dag gamma5):
 *   C_PG(t) = sum_{x, x_t = t} tr[ G(x,0)^dag G(x,0) Gamma gamma5 ]   (Gamma on source spin),
 * with G(x,0) the d-quark propagator of a source at the origin (solutions of M(-mu) x = b).
 * props: 12 canonical full fields, host or device, back to back; field j = 3 s + c is the
 * solution for the source of spin s and colour c.  out: T x 12 x 12 complex doubles (host or
 * device), out[t][j][k] = sum_{x, x_t = t} <psi_j(x), psi_k(x)> (conjugate on psi_j); then
 * C_PG(t) = sum_{s, s', c} out[t][3s+c][3s'+c] (Gamma gamma5)[s'][s], e.g. C_PP(t) = trace.
 * FP64, deterministic; exactly hermitian (the 78 entries j <= k are summed, the others are
 * their conjugates).  Device props must be 16-byte aligned (host props are staged).
 * Errors: TM_ERR_ARG, TM_ERR_CUDA. */
tm_status tm_meson_contract(tm_lattice lat, const double *props, double *out, void *stream);

/* Correlators from the timeslice Gram matrices of tm_meson_contract (Sec. 4.3): for each of
 * ngamma 4 x 4 complex matrices X_g = Gamma_g gamma5 acting on source spin,
 *   C[g][t] = tr[ A_t (X_g (x) 1_colour) ] = sum_{s, s', c} A[t][3s+c][3s'+c] X_g[s'][s],
 * e.g. C_PP: X = 1;  C_PA (Gamma = gamma0 gamma5): X = gamma0;  C_PV (Gamma = gamma0): X = gamma0
 * gamma5 (gamma matrices of App. A).  A: T x 12 x 12 complex doubles, the output of
 * tm_meson_contract (host or device).  X: ngamma x 4 x 4 complex doubles, row-major X[s'][s]
 * (host or device), 1 <= ngamma <= 1024.  C: ngamma x T complex doubles (host or device).  FP64;
 * each entry is summed in a fixed order (deterministic).  Errors: TM_ERR_ARG, TM_ERR_CUDA. */
tm_status tm_correlator(tm_lattice lat, const double *A, const double *X, int ngamma, double *C,
                        void *stream);

/* Fills params with the defaults: tol 1e-10, max_iter 100000, TM_CG_FP64, sloppy
 * TM_F32 / TM_LINK12, delta 0.1, use_x0 0, flavour +1, update_prec TM_F64. */
void tm_cg_params_default(tm_cg_params *params);

/* ------------------------------------------------------ allocation-free variant --- */

/* The paper has no counterpart to this entry point.  Same result as tm_apply_D, for callers
 * that must not allocate device memory during the call: code running under a fixed
 * device-memory budget (a framework whose caching allocator already holds the memory, a
 * process with a hard memory limit) or in a latency-critical loop where a cudaMalloc or
 * cudaFree would synchronise the device.  tm_apply_D takes its four half-field work buffers
 * from lattice-owned memory allocated on first use; this variant takes them from one static
 * 64 MiB device array that is part of the library's device code, so the call itself calls no
 * cudaMalloc, cudaFree or other allocating routine.  Every GPU that loads the library holds
 * those 64 MiB until the process exits.
 *   Limit: 4 x 192 x V/2 bytes of scratch must fit in 64 MiB, i.e. V = T L^3 <= 174762
 *          sites (16^3 x 32 fits, 24^3 x 48 does not); larger lattices get TM_ERR_ARG.
 *   in, out: canonical full fields in DEVICE memory of the lattice's device, or managed
 *          memory (host pointers, and device memory of another GPU, get TM_ERR_ARG: staging
 *          them would need a buffer); nrhs x 24 V doubles; no overlap.
 *   Set-up: the first call on a device looks up the array's device address
 *          (cudaGetSymbolAddress, with that device current) and caches it for the rest of the
 *          process; make that first call before any stream capture.  The cached address
 *          belongs to the device's context at that time: after a cudaDeviceReset (which also
 *          frees every lattice's device memory) this entry point must not be called again in
 *          the same process.
 *   Sharing: every call uses the same array.  The array keeps the previous call's contents
 *          (each call writes every scratch byte it reads before reading it), and calls that
 *          overlap on the GPU -- on different streams, or from different host threads --
 *          race on it: order them on one stream.
 * Errors: as tm_apply_D, plus TM_ERR_ARG for the limits above. */
tm_status tm_apply_D_noalloc(tm_lattice lat, double *out, const double *in, int flavour, int dagger,
                             int nrhs, void *stream);

/* ------------------------------------------------------------------- misc --- */

/* Message of the last failed call on this host thread ("" if none). */
const char *tm_last_error(void);

/* Kernels the library has launched since tm_reset_launch_count() (all threads). */
unsigned long long tm_launch_count(void);
void tm_reset_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* TM_H */
