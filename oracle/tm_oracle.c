/*
 * tm_oracle.c -- plain FP64 CPU oracle for the one-flavour Wilson twisted-mass
 * operator and its even/odd-preconditioned CG solve (Jansen & Urbach, "tmLQCD:
 * a program suite to simulate Wilson twisted mass lattice QCD", arXiv:0905.3331).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct reference that
 * the CUDA library is checked against.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg call it.  It shares no code, header, table or
 * constant with the CUDA library, and it never calls it.
 *
 * Everything is written straight from the paper's definitions, with no
 * half-spinor trick, no blocking, no fusion and no reordering:
 *   - the operator M of eq. eo0 (App. B.1), hopping-parameter form, r = 1:
 *       (M psi)(x) = [1 + i mu~ f gamma5] psi(x)
 *                    - kappa sum_mu [ U_mu(x) (1 + gamma_mu) psi(x + mu^)
 *                                   + U_mu(x - mu^)^dag (1 - gamma_mu) psi(x - mu^) ]
 *     with mu~ = 2 kappa mu (App. B.1) and f = +1 ("up", tau3 = +1) or -1;
 *   - the gamma matrices typed in from App. A (chiral basis, gamma5 diagonal);
 *   - fermion boundary conditions psi(x + L_nu nu^) = exp(i theta_nu pi) psi(x)
 *     (Sec. 2.4).  By default the whole phase sits on the hop that wraps the
 *     boundary; the "spread" placement of Sec. 4.1.2 (a phase exp(+-i theta pi/L)
 *     on every hop) is available for the equivalence test;
 *   - the even/odd blocks of eq. eo2, the inverse of eq. eo3, the Schur operator
 *     of eq. eo4, the two inversion steps of App. B.2, and CG (Hestenes-Stiefel)
 *     on Qhat^+ Qhat^- (eq. eo6) with the relative stopping test of Sec. 4.4.
 *
 * Layout (canonical): lex = ((t*Lz + z)*Ly + y)*Lx + x, i.e. the index order
 * t, z, y, x, spin, colour of the propagator format (Sec. 4.7.2); a spinor field
 * is psi[lex][spin 4][colour 3], the gauge field U[lex][mu 4][row 3][col 3] with
 * mu = 0:t, 1:x, 2:y, 3:z.  Complex numbers are C99 double complex.  Vectors
 * that live on one parity are stored as full-lattice arrays that are zero on the
 * other parity.  Parity of a site is (t + x + y + z) mod 2, even = 0.
 *
 * Threads: the site loops of the operator are OpenMP "parallel for" loops whose
 * iterations write disjoint outputs, so results do not depend on the thread
 * count.  Every global sum runs serially in lexicographic order.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ---------------------------------------------------------------- App. A --- */
/* gamma_0 .. gamma_3 and gamma_5, typed in from App. A. */
static const cplx GAMMA[5][4][4] = {
    /* gamma_0 */
    {{0, 0, -1, 0}, {0, 0, 0, -1}, {-1, 0, 0, 0}, {0, -1, 0, 0}},
    /* gamma_1 */
    {{0, 0, 0, -I}, {0, 0, -I, 0}, {0, +I, 0, 0}, {+I, 0, 0, 0}},
    /* gamma_2 */
    {{0, 0, 0, -1}, {0, 0, +1, 0}, {0, +1, 0, 0}, {-1, 0, 0, 0}},
    /* gamma_3 */
    {{0, 0, -I, 0}, {0, 0, 0, +I}, {+I, 0, 0, 0}, {0, -I, 0, 0}},
    /* gamma_5 */
    {{+1, 0, 0, 0}, {0, +1, 0, 0}, {0, 0, -1, 0}, {0, 0, 0, -1}},
};

/* Copies gamma_k (k = 0..3, or 4 for gamma_5) into out[4][4] (row major). */
void orc_gamma(int k, cplx *out) {
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) out[4 * a + b] = GAMMA[k][a][b];
}

/* ------------------------------------------------------------- geometry --- */
typedef struct {
  int n[4]; /* extents in direction order: n[0] = T, n[1] = Lx, n[2] = Ly, n[3] = Lz */
  long V;
} geo_t;

static geo_t make_geo(const int dims[4]) {
  geo_t g;
  g.V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    g.n[mu] = dims[mu];
    g.V *= dims[mu];
  }
  return g;
}

/* c[0] = t, c[1] = x, c[2] = y, c[3] = z of site lex. */
static void coords(const geo_t *g, long lex, int c[4]) {
  c[1] = (int)(lex % g->n[1]);
  lex /= g->n[1];
  c[2] = (int)(lex % g->n[2]);
  lex /= g->n[2];
  c[3] = (int)(lex % g->n[3]);
  lex /= g->n[3];
  c[0] = (int)lex;
}

static long lex_of(const geo_t *g, const int c[4]) {
  return (((long)c[0] * g->n[3] + c[3]) * g->n[2] + c[2]) * g->n[1] + c[1];
}

static int parity_of(const int c[4]) { return (c[0] + c[1] + c[2] + c[3]) & 1; }

/* Phase exp(i theta pi) as a complex number; integer theta gives exactly +-1. */
static cplx unit_phase(double theta_pi_fraction) {
  double r = fmod(theta_pi_fraction, 2.0);
  if (r == 0.0) return 1.0;
  if (r == 1.0 || r == -1.0) return -1.0;
  return cexp(I * M_PI * theta_pi_fraction);
}

/* Phase picked up by the hop from x to x + dir mu^ (dir = +1 or -1).
 * Boundary placement: psi(x + L_mu mu^) = exp(i theta_mu pi) psi(x) (Sec. 2.4),
 * so only the hop that leaves the box carries the phase.
 * Spread placement: every hop carries exp(dir i theta_mu pi / L_mu) (Sec. 4.1.2). */
static cplx hop_phase(const geo_t *g, const double theta[4], int spread, const int c[4],
                      int mu, int dir) {
  if (spread) return cexp(I * (double)dir * theta[mu] * M_PI / (double)g->n[mu]);
  if (dir > 0 && c[mu] == g->n[mu] - 1) return unit_phase(theta[mu]);
  if (dir < 0 && c[mu] == 0) return unit_phase(-theta[mu]);
  return 1.0;
}

/* ------------------------------------------------- the hopping sum H --- */
/*
 * out(x) = sum_mu [ U_mu(x) (1 + gamma_mu) in(x + mu^) + U_mu(x - mu^)^dag (1 - gamma_mu) in(x - mu^) ]
 * (the bracket of eq. eo0 / eq. Dpsi with r = 1, without the factor -kappa), each
 * hop times its boundary phase.  If out_parity is 0 or 1 only sites of that
 * parity are computed (all their neighbours have the other parity, so this is
 * H_eo or H_oe of eq. eo2) and the other sites are set to zero; -1 computes all.
 */
static void hopping_site(const geo_t *g, const double theta[4], int spread, const cplx *U,
                         const cplx *in, long lex, cplx acc[4][3]) {
  int c[4];
  coords(g, lex, c);
  for (int s = 0; s < 4; ++s)
    for (int a = 0; a < 3; ++a) acc[s][a] = 0;
  for (int mu = 0; mu < 4; ++mu) {
    for (int dir = +1; dir >= -1; dir -= 2) {
      int cn[4] = {c[0], c[1], c[2], c[3]};
      cn[mu] = (c[mu] + dir + g->n[mu]) % g->n[mu];
      long ln = lex_of(g, cn);
      const cplx *nb = in + 12 * ln;
      /* link: U_mu(x) forward, U_mu(x - mu^)^dag backward */
      cplx link[3][3];
      if (dir > 0) {
        const cplx *u = U + 36 * lex + 9 * mu;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) link[a][b] = u[3 * a + b];
      } else {
        const cplx *u = U + 36 * ln + 9 * mu;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) link[a][b] = conj(u[3 * b + a]);
      }
      /* spin matrix (1 + dir gamma_mu), applied as a full 4x4 matrix */
      cplx P[4][4];
      for (int s = 0; s < 4; ++s)
        for (int t = 0; t < 4; ++t) P[s][t] = (s == t ? 1.0 : 0.0) + (double)dir * GAMMA[mu][s][t];
      cplx ph = hop_phase(g, theta, spread, c, mu, dir);
      for (int s = 0; s < 4; ++s) {
        cplx spin_mixed[3];
        for (int b = 0; b < 3; ++b) {
          spin_mixed[b] = 0;
          for (int t = 0; t < 4; ++t) spin_mixed[b] += P[s][t] * nb[3 * t + b];
        }
        for (int a = 0; a < 3; ++a) {
          cplx v = 0;
          for (int b = 0; b < 3; ++b) v += link[a][b] * spin_mixed[b];
          acc[s][a] += ph * v;
        }
      }
    }
  }
}

void orc_hopping(const int dims[4], const double theta[4], int spread, const cplx *U,
                 const cplx *in, cplx *out, int out_parity) {
  geo_t g = make_geo(dims);
#pragma omp parallel for schedule(static)
  for (long lex = 0; lex < g.V; ++lex) {
    int c[4];
    coords(&g, lex, c);
    cplx *o = out + 12 * lex;
    if (out_parity >= 0 && parity_of(c) != out_parity) {
      for (int k = 0; k < 12; ++k) o[k] = 0;
      continue;
    }
    cplx acc[4][3];
    hopping_site(&g, theta, spread, U, in, lex, acc);
    for (int s = 0; s < 4; ++s)
      for (int a = 0; a < 3; ++a) o[3 * s + a] = acc[s][a];
  }
}

/* ---------------------------------------------------- the operator M --- */
/* Site-diagonal term [1 + i f mu~ gamma5] of eq. eo0, applied as a 4x4 matrix. */
static void twisted_diag(double mut, int f, const cplx *in, cplx *out) {
  for (int s = 0; s < 4; ++s)
    for (int a = 0; a < 3; ++a) {
      cplx v = 0;
      for (int t = 0; t < 4; ++t) {
        cplx m = (s == t ? 1.0 : 0.0) + I * (double)f * mut * GAMMA[4][s][t];
        v += m * in[3 * t + a];
      }
      out[3 * s + a] = v;
    }
}

/* out = M psi on the full lattice, eq. eo0, mu~ = 2 kappa mu.  f = +1 or -1. */
void orc_apply_M(const int dims[4], const double theta[4], int spread, double kappa, double mu,
                 int f, const cplx *U, const cplx *in, cplx *out) {
  geo_t g = make_geo(dims);
  double mut = 2.0 * kappa * mu;
#pragma omp parallel for schedule(static)
  for (long lex = 0; lex < g.V; ++lex) {
    cplx acc[4][3], d[12];
    hopping_site(&g, theta, spread, U, in, lex, acc);
    twisted_diag(mut, f, in + 12 * lex, d);
    for (int s = 0; s < 4; ++s)
      for (int a = 0; a < 3; ++a) out[12 * lex + 3 * s + a] = d[3 * s + a] - kappa * acc[s][a];
  }
}

/* (M psi) at the listed sites only: out[k][12] = (M psi)(sites[k]).  Same
 * arithmetic as orc_apply_M, for sampled checks of very large lattices. */
void orc_apply_M_sites(const int dims[4], const double theta[4], int spread, double kappa,
                       double mu, int f, const cplx *U, const cplx *in, const long *sites,
                       long nsites, cplx *out) {
  geo_t g = make_geo(dims);
  double mut = 2.0 * kappa * mu;
#pragma omp parallel for schedule(static)
  for (long k = 0; k < nsites; ++k) {
    long lex = sites[k];
    cplx acc[4][3], d[12];
    hopping_site(&g, theta, spread, U, in, lex, acc);
    twisted_diag(mut, f, in + 12 * lex, d);
    for (int s = 0; s < 4; ++s)
      for (int a = 0; a < 3; ++a) out[12 * k + 3 * s + a] = d[3 * s + a] - kappa * acc[s][a];
  }
}

/* ----------------------------------------------- even/odd blocks (B.1) --- */
/* out = M_pp^{f} in = [1 + i f mu~ gamma5] in on the sites of the given parity,
 * zero elsewhere (eq. eo2: M_ee^+- = M_oo^+- = 1 +- i mu~ gamma5). */
void orc_apply_Mdiag(const int dims[4], double mut, int f, int parity, const cplx *in, cplx *out) {
  geo_t g = make_geo(dims);
  for (long lex = 0; lex < g.V; ++lex) {
    int c[4];
    coords(&g, lex, c);
    if (parity_of(c) != parity) {
      for (int k = 0; k < 12; ++k) out[12 * lex + k] = 0;
      continue;
    }
    twisted_diag(mut, f, in + 12 * lex, out + 12 * lex);
  }
}

/* out = (M_pp^{f})^{-1} in = (1 - i f mu~ gamma5) / (1 + mu~^2) in on the sites
 * of the given parity, zero elsewhere (eq. eo3). */
void orc_apply_Mdiag_inv(const int dims[4], double mut, int f, int parity, const cplx *in,
                         cplx *out) {
  geo_t g = make_geo(dims);
  for (long lex = 0; lex < g.V; ++lex) {
    int c[4];
    coords(&g, lex, c);
    if (parity_of(c) != parity) {
      for (int k = 0; k < 12; ++k) out[12 * lex + k] = 0;
      continue;
    }
    cplx tmp[12];
    twisted_diag(mut, -f, in + 12 * lex, tmp);
    for (int k = 0; k < 12; ++k) out[12 * lex + k] = tmp[k] / (1.0 + mut * mut);
  }
}

/* out = M_{p,1-p} in = -kappa H_{p,1-p} in (the off-diagonal blocks of eq. eo2). */
void orc_apply_Moff(const int dims[4], const double theta[4], int spread, double kappa,
                    const cplx *U, int out_parity, const cplx *in, cplx *out) {
  geo_t g = make_geo(dims);
  orc_hopping(dims, theta, spread, U, in, out, out_parity);
  for (long k = 0; k < 12 * g.V; ++k) out[k] *= -kappa;
}

static void gamma5_apply(long V, const cplx *in, cplx *out) {
  for (long lex = 0; lex < V; ++lex)
    for (int s = 0; s < 4; ++s)
      for (int a = 0; a < 3; ++a) {
        cplx v = 0;
        for (int t = 0; t < 4; ++t) v += GAMMA[4][s][t] * in[12 * lex + 3 * t + a];
        out[12 * lex + 3 * s + a] = v;
      }
}

/* Schur operator on odd sites, eq. eo2/eo4:
 *   Mhat^{f} v = M_oo^{f} v - M_oe (M_ee^{f})^{-1} M_eo v.
 * If with_gamma5 is set, returns Qhat^{f} v = gamma5 Mhat^{f} v. */
void orc_schur(const int dims[4], const double theta[4], int spread, double kappa, double mu,
               int f, const cplx *U, const cplx *v, cplx *out, int with_gamma5) {
  geo_t g = make_geo(dims);
  double mut = 2.0 * kappa * mu;
  long n = 12 * g.V;
  cplx *t1 = calloc(n, sizeof(cplx)), *t2 = calloc(n, sizeof(cplx));
  cplx *t3 = calloc(n, sizeof(cplx)), *t4 = calloc(n, sizeof(cplx));
  orc_apply_Moff(dims, theta, spread, kappa, U, 0, v, t1); /* t1 = M_eo v        */
  orc_apply_Mdiag_inv(dims, mut, f, 0, t1, t2);            /* t2 = M_ee^-1 t1    */
  orc_apply_Moff(dims, theta, spread, kappa, U, 1, t2, t3); /* t3 = M_oe t2       */
  orc_apply_Mdiag(dims, mut, f, 1, v, t4);                 /* t4 = M_oo v        */
  for (long k = 0; k < n; ++k) t4[k] -= t3[k];
  if (with_gamma5)
    gamma5_apply(g.V, t4, out);
  else
    memcpy(out, t4, n * sizeof(cplx));
  free(t1);
  free(t2);
  free(t3);
  free(t4);
}

/* out = Qhat^{f} Qhat^{-f} v, the normal operator of eq. eo6 (f = +1 gives Qhat+ Qhat-). */
void orc_normal_op(const int dims[4], const double theta[4], int spread, double kappa, double mu,
                   int f, const cplx *U, const cplx *v, cplx *out) {
  geo_t g = make_geo(dims);
  cplx *w = calloc(12 * g.V, sizeof(cplx));
  orc_schur(dims, theta, spread, kappa, mu, -f, U, v, w, 1);
  orc_schur(dims, theta, spread, kappa, mu, f, U, w, out, 1);
  free(w);
}

/* ---------------------------------------------------------- reductions --- */
static double norm2(long n, const cplx *a) {
  double s = 0;
  for (long k = 0; k < n; ++k) s += creal(a[k]) * creal(a[k]) + cimag(a[k]) * cimag(a[k]);
  return s;
}

static cplx dot(long n, const cplx *a, const cplx *b) { /* <a, b> = sum conj(a) b */
  cplx s = 0;
  for (long k = 0; k < n; ++k) s += conj(a[k]) * b[k];
  return s;
}

/* ----------------------------------------------------------------- CG --- */
/*
 * Conjugate gradient (Hestenes-Stiefel) on A = Qhat^{f} Qhat^{-f}, which is
 * Hermitian and positive definite because (Qhat^{+-})^dag = Qhat^{-+} (eq. eo6).
 * Stops when ||r||^2 / ||b||^2 < tol^2 (Sec. 4.4, relative criterion) holds for
 * the residual r = b - A x recomputed from x; if the iterated residual passes
 * but the recomputed one does not, CG restarts from the current x.
 * x holds the initial guess on entry.  Returns 0 if converged, 1 otherwise.
 */
int orc_cg(const int dims[4], const double theta[4], int spread, double kappa, double mu, int f,
           const cplx *U, const cplx *b, cplx *x, double tol, int max_iter, int *iters_out,
           double *relres_out) {
  geo_t g = make_geo(dims);
  long n = 12 * g.V;
  cplx *r = calloc(n, sizeof(cplx)), *p = calloc(n, sizeof(cplx)), *q = calloc(n, sizeof(cplx));
  double bb = norm2(n, b);
  int converged = 0, k = 0;
  double rr = 0;
  if (bb == 0.0) {
    for (long i = 0; i < n; ++i) x[i] = 0;
    converged = 1;
    goto done;
  }
  /* r = b - A x, p = r */
  orc_normal_op(dims, theta, spread, kappa, mu, f, U, x, q);
  for (long i = 0; i < n; ++i) r[i] = b[i] - q[i];
  memcpy(p, r, n * sizeof(cplx));
  rr = norm2(n, r);
  if (rr < tol * tol * bb) {
    converged = 1;
    goto done;
  }
  while (k < max_iter) {
    orc_normal_op(dims, theta, spread, kappa, mu, f, U, p, q); /* q = A p */
    double alpha = rr / creal(dot(n, p, q));
    for (long i = 0; i < n; ++i) x[i] += alpha * p[i];
    for (long i = 0; i < n; ++i) r[i] -= alpha * q[i];
    double rr_new = norm2(n, r);
    ++k;
    if (rr_new < tol * tol * bb) {
      /* recompute the true residual before stopping */
      orc_normal_op(dims, theta, spread, kappa, mu, f, U, x, q);
      for (long i = 0; i < n; ++i) r[i] = b[i] - q[i];
      rr_new = norm2(n, r);
      if (rr_new < tol * tol * bb) {
        converged = 1;
        rr = rr_new;
        break;
      }
      memcpy(p, r, n * sizeof(cplx)); /* restart */
      rr = rr_new;
      continue;
    }
    double beta = rr_new / rr;
    for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    rr = rr_new;
  }
done:
  if (iters_out) *iters_out = k;
  if (relres_out) *relres_out = bb > 0 ? sqrt(rr / bb) : 0.0;
  free(r);
  free(p);
  free(q);
  return converged ? 0 : 1;
}

/* ----------------------------------------------------------- BiCGstab --- */
/*
 * Stabilised bi-conjugate gradients (van der Vorst 1992; Saad, "Iterative Methods for
 * Sparse Linear Systems", 2003, the BiCGSTAB algorithm), one of the solvers of Sec. 4.4,
 * applied directly to the non-hermitian Schur operator Mhat^{f} of eq. eo4 (no normal
 * equations).  Shadow residual r^ = r_0; with <a, b> = sum conj(a) b:
 *   p = r
 *   repeat:  v = Mhat p;  alpha = <r^, r> / <r^, v>;  s = r - alpha v
 *            (if ||s||^2 < tol^2 ||b||^2: x += alpha p, stop)
 *            t = Mhat s;  omega = <t, s> / <t, t>
 *            x += alpha p + omega s;  r = s - omega t
 *            beta = (<r^, r_new> / <r^, r_old>) (alpha / omega);  p = r + beta (p - omega v)
 * The stopping test is the relative one of Sec. 4.4 on the iterated residual, confirmed on
 * the residual recomputed from x; if that fails, or rho or omega vanishes (breakdown), the
 * method restarts from the current x with r^ = r.  One iteration = two applications of
 * Mhat.  x holds the initial guess.  Returns 0 if converged, 1 otherwise.
 */
int orc_bicgstab(const int dims[4], const double theta[4], int spread, double kappa, double mu,
                 int f, const cplx *U, const cplx *b, cplx *x, double tol, int max_iter,
                 int *iters_out, double *relres_out) {
  geo_t g = make_geo(dims);
  long n = 12 * g.V;
  cplx *r = calloc(n, sizeof(cplx)), *rh = calloc(n, sizeof(cplx)), *p = calloc(n, sizeof(cplx));
  cplx *v = calloc(n, sizeof(cplx)), *s = calloc(n, sizeof(cplx)), *t = calloc(n, sizeof(cplx));
  double bb = norm2(n, b), stop2 = tol * tol * bb, rr = 0;
  int converged = 0, k = 0, restart = 1;
  cplx rho = 0;
  if (bb == 0.0) {
    for (long i = 0; i < n; ++i) x[i] = 0;
    converged = 1;
    goto done;
  }
  while (k < max_iter) {
    if (restart) { /* r = b - Mhat x, r^ = r, p = r */
      orc_schur(dims, theta, spread, kappa, mu, f, U, x, t, 0);
      for (long i = 0; i < n; ++i) r[i] = b[i] - t[i];
      rr = norm2(n, r);
      if (rr < stop2) {
        converged = 1;
        break;
      }
      memcpy(rh, r, n * sizeof(cplx));
      memcpy(p, r, n * sizeof(cplx));
      rho = dot(n, rh, r);
      restart = 0;
    }
    orc_schur(dims, theta, spread, kappa, mu, f, U, p, v, 0); /* v = Mhat p */
    cplx rv = dot(n, rh, v);
    if (rv == 0) {
      restart = 1;
      ++k;
      continue;
    }
    cplx alpha = rho / rv;
    for (long i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
    ++k;
    if (norm2(n, s) < stop2) {
      for (long i = 0; i < n; ++i) x[i] += alpha * p[i];
      restart = 1; /* confirm on the recomputed residual at the top of the loop */
      orc_schur(dims, theta, spread, kappa, mu, f, U, x, t, 0);
      for (long i = 0; i < n; ++i) r[i] = b[i] - t[i];
      rr = norm2(n, r);
      if (rr < stop2) {
        converged = 1;
        break;
      }
      continue;
    }
    orc_schur(dims, theta, spread, kappa, mu, f, U, s, t, 0); /* t = Mhat s */
    double tt = norm2(n, t);
    cplx omega = tt > 0 ? dot(n, t, s) / tt : 0;
    for (long i = 0; i < n; ++i) x[i] += alpha * p[i] + omega * s[i];
    for (long i = 0; i < n; ++i) r[i] = s[i] - omega * t[i];
    rr = norm2(n, r);
    if (rr < stop2) {
      orc_schur(dims, theta, spread, kappa, mu, f, U, x, t, 0);
      for (long i = 0; i < n; ++i) r[i] = b[i] - t[i];
      rr = norm2(n, r);
      if (rr < stop2) {
        converged = 1;
        break;
      }
      restart = 1;
      continue;
    }
    cplx rho_new = dot(n, rh, r);
    if (rho_new == 0 || omega == 0) {
      restart = 1;
      continue;
    }
    cplx beta = (rho_new / rho) * (alpha / omega);
    for (long i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
    rho = rho_new;
  }
done:
  if (iters_out) *iters_out = k;
  if (relres_out) *relres_out = bb > 0 ? sqrt(rr / bb) : 0.0;
  free(r);
  free(rh);
  free(p);
  free(v);
  free(s);
  free(t);
  return converged ? 0 : 1;
}

/* ------------------------------------------------------- minimal residual --- */
/*
 * Minimal residual iteration (MR; Saad 2003, the minimal residual method for general
 * matrices), one of the solvers of Sec. 4.4, on the Schur operator Mhat^{f} of eq. eo4:
 *   q = Mhat r;  alpha = <q, r> / <q, q>;  x += alpha r;  r -= alpha q
 * (alpha minimises ||r - alpha q||).  Relative stopping test of Sec. 4.4 on the iterated
 * residual, confirmed on the recomputed one (else the recursion restarts from it).  x holds
 * the initial guess.  Returns 0 if converged, 1 otherwise.
 */
int orc_mr(const int dims[4], const double theta[4], int spread, double kappa, double mu, int f,
           const cplx *U, const cplx *b, cplx *x, double tol, int max_iter, int *iters_out,
           double *relres_out) {
  geo_t g = make_geo(dims);
  long n = 12 * g.V;
  cplx *r = calloc(n, sizeof(cplx)), *q = calloc(n, sizeof(cplx));
  double bb = norm2(n, b), stop2 = tol * tol * bb, rr = 0;
  int converged = 0, k = 0;
  if (bb == 0.0) {
    for (long i = 0; i < n; ++i) x[i] = 0;
    converged = 1;
    goto done;
  }
  orc_schur(dims, theta, spread, kappa, mu, f, U, x, q, 0);
  for (long i = 0; i < n; ++i) r[i] = b[i] - q[i];
  rr = norm2(n, r);
  while (k < max_iter) {
    if (rr < stop2) { /* confirm on the recomputed residual */
      orc_schur(dims, theta, spread, kappa, mu, f, U, x, q, 0);
      for (long i = 0; i < n; ++i) r[i] = b[i] - q[i];
      rr = norm2(n, r);
      if (rr < stop2) {
        converged = 1;
        break;
      }
    }
    orc_schur(dims, theta, spread, kappa, mu, f, U, r, q, 0); /* q = Mhat r */
    double qq = norm2(n, q);
    if (qq == 0.0) break;
    cplx alpha = dot(n, q, r) / qq;
    for (long i = 0; i < n; ++i) x[i] += alpha * r[i];
    for (long i = 0; i < n; ++i) r[i] -= alpha * q[i];
    rr = norm2(n, r);
    ++k;
  }
  if (!converged && rr < stop2) { /* the last step reached the tolerance: confirm it */
    orc_schur(dims, theta, spread, kappa, mu, f, U, x, q, 0);
    for (long i = 0; i < n; ++i) r[i] = b[i] - q[i];
    rr = norm2(n, r);
    converged = rr < stop2;
  }
done:
  if (iters_out) *iters_out = k;
  if (relres_out) *relres_out = bb > 0 ? sqrt(rr / bb) : 0.0;
  free(r);
  free(q);
  return converged ? 0 : 1;
}

/* ------------------------------------------- even/odd inversion (B.2) --- */
/* Source preparation, first step of App. B.2:
 *   varphi_e = (M_ee^{f})^{-1} phi_e,   varphi_o = phi_o - M_oe varphi_e.
 * phi is a full-lattice field; varphi gets both parities. */
void orc_eo_prepare(const int dims[4], const double theta[4], int spread, double kappa, double mu,
                    int f, const cplx *U, const cplx *phi, cplx *varphi) {
  geo_t g = make_geo(dims);
  long n = 12 * g.V;
  double mut = 2.0 * kappa * mu;
  cplx *ve = calloc(n, sizeof(cplx)), *t = calloc(n, sizeof(cplx));
  orc_apply_Mdiag_inv(dims, mut, f, 0, phi, ve);       /* even part: M_ee^-1 phi_e */
  orc_apply_Moff(dims, theta, spread, kappa, U, 1, ve, t); /* t = M_oe varphi_e   */
  for (long lex = 0; lex < g.V; ++lex) {
    int c[4];
    coords(&g, lex, c);
    for (int k = 0; k < 12; ++k) {
      long i = 12 * lex + k;
      varphi[i] = parity_of(c) == 0 ? ve[i] : phi[i] - t[i];
    }
  }
  free(ve);
  free(t);
}

/* Second step of App. B.2: psi_e = varphi_e - (M_ee^{f})^{-1} M_eo psi_o,
 * given varphi (both parities) and psi_o (odd sites of psi); fills psi_e. */
void orc_eo_reconstruct(const int dims[4], const double theta[4], int spread, double kappa,
                        double mu, int f, const cplx *U, const cplx *varphi, cplx *psi) {
  geo_t g = make_geo(dims);
  long n = 12 * g.V;
  double mut = 2.0 * kappa * mu;
  cplx *t = calloc(n, sizeof(cplx)), *u = calloc(n, sizeof(cplx));
  orc_apply_Moff(dims, theta, spread, kappa, U, 0, psi, t); /* t = M_eo psi_o      */
  orc_apply_Mdiag_inv(dims, mut, f, 0, t, u);               /* u = M_ee^-1 t       */
  for (long lex = 0; lex < g.V; ++lex) {
    int c[4];
    coords(&g, lex, c);
    if (parity_of(c) != 0) continue;
    for (int k = 0; k < 12; ++k) psi[12 * lex + k] = varphi[12 * lex + k] - u[12 * lex + k];
  }
  free(t);
  free(u);
}

/*
 * Full solve of M^{f} psi = phi by even/odd preconditioning (App. B.2):
 *   1. varphi = prepare(phi);
 *   2. Mhat^{f} psi_o = varphi_o, solved as X = (Qhat^{f} Qhat^{-f})^{-1} gamma5 varphi_o,
 *      psi_o = Qhat^{-f} X (eq. eo6: Qhat^{f} psi_o = gamma5 varphi_o);
 *   3. psi_e = reconstruct(varphi, psi_o).
 * tol is the relative CG tolerance on ||b - A X|| / ||b||, b = gamma5 varphi_o.
 * Returns the CG status; iters, the normal-equation relative residual and the
 * full-lattice relative residual ||phi - M psi|| / ||phi|| are reported.
 */
int orc_solve(const int dims[4], const double theta[4], int spread, double kappa, double mu, int f,
              const cplx *U, const cplx *phi, cplx *psi, double tol, int max_iter, int *iters,
              double *relres_normal, double *relres_full) {
  geo_t g = make_geo(dims);
  long n = 12 * g.V;
  cplx *varphi = calloc(n, sizeof(cplx)), *b = calloc(n, sizeof(cplx));
  cplx *X = calloc(n, sizeof(cplx)), *t = calloc(n, sizeof(cplx));
  orc_eo_prepare(dims, theta, spread, kappa, mu, f, U, phi, varphi);
  for (long lex = 0; lex < g.V; ++lex) { /* odd part of varphi */
    int c[4];
    coords(&g, lex, c);
    for (int k = 0; k < 12; ++k) t[12 * lex + k] = parity_of(c) == 1 ? varphi[12 * lex + k] : 0;
  }
  gamma5_apply(g.V, t, b);
  int st = orc_cg(dims, theta, spread, kappa, mu, f, U, b, X, tol, max_iter, iters, relres_normal);
  orc_schur(dims, theta, spread, kappa, mu, -f, U, X, psi, 1); /* psi_o = Qhat^{-f} X */
  orc_eo_reconstruct(dims, theta, spread, kappa, mu, f, U, varphi, psi);
  if (relres_full) {
    orc_apply_M(dims, theta, spread, kappa, mu, f, U, psi, t);
    for (long i = 0; i < n; ++i) t[i] = phi[i] - t[i];
    double pp = norm2(n, phi);
    *relres_full = pp > 0 ? sqrt(norm2(n, t) / pp) : 0.0;
  }
  free(varphi);
  free(b);
  free(X);
  free(t);
  return st;
}

/* Number of OpenMP threads the site loops use (1 without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
int orc_num_threads(void) { return omp_get_max_threads(); }
#else
int orc_num_threads(void) { return 1; }
#endif

/* Pure hopping sum H at the listed sites only (same arithmetic as orc_hopping). */
void orc_hopping_sites(const int dims[4], const double theta[4], int spread, const cplx *U,
                       const cplx *in, const long *sites, long nsites, cplx *out) {
  geo_t g = make_geo(dims);
#pragma omp parallel for schedule(static)
  for (long k = 0; k < nsites; ++k) {
    cplx acc[4][3];
    hopping_site(&g, theta, spread, U, in, sites[k], acc);
    for (int s = 0; s < 4; ++s)
      for (int a = 0; a < 3; ++a) out[12 * k + 3 * s + a] = acc[s][a];
  }
}

/* ------------------------------------------- non-degenerate doublet --- */
/*
 * The mass non-degenerate flavour doublet of eq. Dh, D_h = D_W 1_f + i mubar gamma5 tau3 +
 * epsbar tau1, in the hopping-parameter form of eq. eo0 (M = 2 kappa D):
 *   (M_h psi)(x) = [1_f + i mb gamma5 tau3 + eb tau1] psi(x) - kappa (H psi)(x),
 *   mb = 2 kappa mubar, eb = 2 kappa epsbar,
 * with H the hopping sum of eq. eo0 acting on each flavour alike.  The Pauli matrices are
 * those of App. A.  A doublet field is two one-flavour fields back to back: component
 * [f][lex][spin][colour], f = 0 the upper (tau3 = +1) flavour.
 */
static const cplx PAULI[4][2][2] = {
    {{1, 0}, {0, 1}},   /* 1_f    */
    {{0, 1}, {1, 0}},   /* tau^1  */
    {{0, -I}, {I, 0}},  /* tau^2  */
    {{1, 0}, {0, -1}},  /* tau^3  */
};

void orc_pauli(int k, cplx *out) {
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) out[2 * a + b] = PAULI[k][a][b];
}

void orc_apply_Mh(const int dims[4], const double theta[4], int spread, double kappa, double mubar,
                  double epsbar, const cplx *U, const cplx *in, cplx *out) {
  geo_t g = make_geo(dims);
  long n = 12 * g.V;
  double mb = 2.0 * kappa * mubar, eb = 2.0 * kappa * epsbar;
  cplx *hop = calloc(2 * n, sizeof(cplx));
  orc_hopping(dims, theta, spread, U, in, hop, -1);         /* H psi_0 */
  orc_hopping(dims, theta, spread, U, in + n, hop + n, -1); /* H psi_1 */
#pragma omp parallel for schedule(static)
  for (long lex = 0; lex < g.V; ++lex) {
    for (int f = 0; f < 2; ++f)
      for (int s = 0; s < 4; ++s)
        for (int a = 0; a < 3; ++a) {
          /* site matrix (1_f x 1) + i mb (tau3 x gamma5) + eb (tau1 x 1), row (f, s) */
          cplx v = 0;
          for (int f2 = 0; f2 < 2; ++f2)
            for (int t = 0; t < 4; ++t) {
              cplx m = PAULI[0][f][f2] * (s == t ? 1.0 : 0.0) + I * mb * PAULI[3][f][f2] * GAMMA[4][s][t] +
                       eb * PAULI[1][f][f2] * (s == t ? 1.0 : 0.0);
              v += m * in[f2 * n + 12 * lex + 3 * t + a];
            }
          out[f * n + 12 * lex + 3 * s + a] = v - kappa * hop[f * n + 12 * lex + 3 * s + a];
        }
  }
  free(hop);
}

/* M_h^dag psi = tau1 gamma5 M_h gamma5 tau1 psi (the adjoint relation stated with the PHMC,
 * Sec. 2.3; a CPU test checks it against <chi, M_h psi> = <M_h^dag chi, psi>). */
static void apply_Mh_dag(const int dims[4], const double theta[4], int spread, double kappa,
                         double mubar, double epsbar, const cplx *U, const cplx *in, cplx *out) {
  geo_t g = make_geo(dims);
  long n = 12 * g.V;
  cplx *t1 = calloc(2 * n, sizeof(cplx)), *t2 = calloc(2 * n, sizeof(cplx));
  /* t1 = gamma5 tau1 in: flavours swapped, gamma5 on each */
  gamma5_apply(g.V, in + n, t1);
  gamma5_apply(g.V, in, t1 + n);
  orc_apply_Mh(dims, theta, spread, kappa, mubar, epsbar, U, t1, t2);
  gamma5_apply(g.V, t2 + n, out);
  gamma5_apply(g.V, t2, out + n);
  free(t1);
  free(t2);
}

void orc_apply_Mh_dag(const int dims[4], const double theta[4], int spread, double kappa, double mubar,
                      double epsbar, const cplx *U, const cplx *in, cplx *out) {
  apply_Mh_dag(dims, theta, spread, kappa, mubar, epsbar, U, in, out);
}

/*
 * Solves M_h psi = phi on the full lattice by CG on the normal equations
 * M_h^dag M_h psi = M_h^dag phi (CGNR: the residual r = phi - M_h psi is carried along and
 * tested), relative stop ||r|| / ||phi|| < tol (Sec. 4.4), confirmed on the recomputed
 * residual.  psi holds the initial guess.  Returns 0 if converged, 1 otherwise.
 */
int orc_solve_Mh(const int dims[4], const double theta[4], int spread, double kappa, double mubar,
                 double epsbar, const cplx *U, const cplx *phi, cplx *psi, double tol, int max_iter,
                 int *iters_out, double *relres_out) {
  geo_t g = make_geo(dims);
  long n = 24 * g.V;
  cplx *r = calloc(n, sizeof(cplx)), *z = calloc(n, sizeof(cplx)), *p = calloc(n, sizeof(cplx));
  cplx *w = calloc(n, sizeof(cplx));
  double bb = norm2(n, phi), rr = 0;
  int converged = 0, k = 0, restart = 1;
  double zz = 0;
  if (bb == 0.0) {
    for (long i = 0; i < n; ++i) psi[i] = 0;
    converged = 1;
    goto done;
  }
  while (k < max_iter) {
    if (restart) { /* r = phi - M psi, z = M^dag r, p = z */
      orc_apply_Mh(dims, theta, spread, kappa, mubar, epsbar, U, psi, w);
      for (long i = 0; i < n; ++i) r[i] = phi[i] - w[i];
      rr = norm2(n, r);
      if (rr < tol * tol * bb) {
        converged = 1;
        break;
      }
      apply_Mh_dag(dims, theta, spread, kappa, mubar, epsbar, U, r, z);
      memcpy(p, z, n * sizeof(cplx));
      zz = norm2(n, z);
      restart = 0;
    }
    orc_apply_Mh(dims, theta, spread, kappa, mubar, epsbar, U, p, w); /* w = M p */
    double alpha = zz / norm2(n, w);
    for (long i = 0; i < n; ++i) psi[i] += alpha * p[i];
    for (long i = 0; i < n; ++i) r[i] -= alpha * w[i];
    ++k;
    rr = norm2(n, r);
    if (rr < tol * tol * bb) {
      restart = 1; /* confirm on the recomputed residual */
      continue;
    }
    apply_Mh_dag(dims, theta, spread, kappa, mubar, epsbar, U, r, z);
    double zz_new = norm2(n, z);
    double beta = zz_new / zz;
    for (long i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    zz = zz_new;
  }
done:
  if (iters_out) *iters_out = k;
  if (relres_out) *relres_out = bb > 0 ? sqrt(rr / bb) : 0.0;
  free(r);
  free(z);
  free(p);
  free(w);
  return converged ? 0 : 1;
}
