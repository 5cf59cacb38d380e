/*
 * synth.c -- seeded synthetic inputs: random SU(3) gauge fields and Gaussian
 * spinor sources.  This file holds no arithmetic of the Dirac operator or of
 * the solver; it only draws inputs.  Both the CUDA library's tests/benchmark
 * and the CPU oracle's tests are fed from here.
 *
 * Random numbers: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used as a counter-based
 * generator: draw i of stream `seed` is mix(seed + (i + 1) * 0x9E3779B97F4A7C15),
 * which equals the i-th output of the sequential generator started at state
 * `seed`.  A uniform in [0, 1) takes the top 53 bits.  Normals come from the
 * Box-Muller transform: normal 2j uses cos, normal 2j + 1 uses sin of the pair
 * (u1, u2) = (draw 2j, draw 2j + 1), with 1 - u1 in (0, 1] under the log.
 *
 * Gauge links: U = exp(i eps H), H = sum_a h_a lambda_a / 2 with h_a ~ N(0, 1)
 * and lambda_a the Gell-Mann matrices (traceless Hermitian); the exponential is
 * a scaling-and-squaring Taylor series in FP64, followed by re-unitarisation
 * (Gram-Schmidt on rows 1 and 2, row 3 = conj(row1 x row2), so det U = 1).
 * Link number i = lex * 4 + mu (lex in t, z, y, x order, mu = t, x, y, z) uses
 * normals 8 i .. 8 i + 7.
 *
 * Gaussian source: complex component k has real part normal(2k)/sqrt(2) and
 * imaginary part normal(2k + 1)/sqrt(2), so E|z|^2 = 1.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>

typedef double complex cplx;

static const uint64_t GOLDEN = 0x9E3779B97F4A7C15ull;

uint64_t syn_splitmix64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * GOLDEN;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double syn_uniform(uint64_t seed, uint64_t i) {
  return (double)(syn_splitmix64(seed, i) >> 11) * 0x1.0p-53;
}

double syn_normal(uint64_t seed, uint64_t k) {
  uint64_t j = k >> 1;
  double u1 = 1.0 - syn_uniform(seed, 2 * j);
  double u2 = syn_uniform(seed, 2 * j + 1);
  double r = sqrt(-2.0 * log(u1));
  double ang = 2.0 * M_PI * u2;
  return (k & 1) ? r * sin(ang) : r * cos(ang);
}

void syn_normals(uint64_t seed, uint64_t start, long n, double *out) {
#pragma omp parallel for schedule(static)
  for (long k = 0; k < n; ++k) out[k] = syn_normal(seed, start + (uint64_t)k);
}

/* Gell-Mann matrices lambda_1 .. lambda_8 (standard normalisation tr l_a l_b = 2 delta_ab). */
static void hermitian_from_coeffs(const double h[8], cplx H[3][3]) {
  const double s3 = 1.0 / sqrt(3.0);
  /* H = sum_a h_a lambda_a / 2 */
  H[0][0] = 0.5 * (h[2] + s3 * h[7]);
  H[1][1] = 0.5 * (-h[2] + s3 * h[7]);
  H[2][2] = 0.5 * (-2.0 * s3 * h[7]);
  H[0][1] = 0.5 * (h[0] - I * h[1]);
  H[1][0] = 0.5 * (h[0] + I * h[1]);
  H[0][2] = 0.5 * (h[3] - I * h[4]);
  H[2][0] = 0.5 * (h[3] + I * h[4]);
  H[1][2] = 0.5 * (h[5] - I * h[6]);
  H[2][1] = 0.5 * (h[5] + I * h[6]);
}

static void mat_mul(const cplx A[3][3], const cplx B[3][3], cplx C[3][3]) {
  cplx T[3][3];
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) {
      cplx s = 0;
      for (int j = 0; j < 3; ++j) s += A[i][j] * B[j][k];
      T[i][k] = s;
    }
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) C[i][k] = T[i][k];
}

/* exp(A) for a 3x3 complex A: scale by 2^-s until ||A||_F <= 1/4, Taylor series
 * of degree 16 (Horner form), square s times. */
static void mat_exp(const cplx A_in[3][3], cplx E[3][3]) {
  double nrm = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) nrm += creal(A_in[i][j] * conj(A_in[i][j]));
  nrm = sqrt(nrm);
  int s = 0;
  while (nrm > 0.25) {
    nrm *= 0.5;
    ++s;
  }
  double scale = ldexp(1.0, -s);
  cplx A[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) A[i][j] = A_in[i][j] * scale;
  /* E = I + A/1 (I + A/2 (I + ... (I + A/16))) */
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) E[i][j] = (i == j) ? 1.0 : 0.0;
  for (int k = 16; k >= 1; --k) {
    cplx T[3][3];
    mat_mul(A, E, T);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) E[i][j] = ((i == j) ? 1.0 : 0.0) + T[i][j] / (double)k;
  }
  for (int r = 0; r < s; ++r) mat_mul(E, E, E);
}

/* Gram-Schmidt on rows 0 and 1, row 2 = conj(row0 x row1): a special unitary matrix. */
static void reunitarise(cplx U[3][3]) {
  double n0 = 0;
  for (int j = 0; j < 3; ++j) n0 += creal(U[0][j] * conj(U[0][j]));
  n0 = 1.0 / sqrt(n0);
  for (int j = 0; j < 3; ++j) U[0][j] *= n0;
  cplx d = 0;
  for (int j = 0; j < 3; ++j) d += conj(U[0][j]) * U[1][j];
  for (int j = 0; j < 3; ++j) U[1][j] -= d * U[0][j];
  double n1 = 0;
  for (int j = 0; j < 3; ++j) n1 += creal(U[1][j] * conj(U[1][j]));
  n1 = 1.0 / sqrt(n1);
  for (int j = 0; j < 3; ++j) U[1][j] *= n1;
  U[2][0] = conj(U[0][1] * U[1][2] - U[0][2] * U[1][1]);
  U[2][1] = conj(U[0][2] * U[1][0] - U[0][0] * U[1][2]);
  U[2][2] = conj(U[0][0] * U[1][1] - U[0][1] * U[1][0]);
}

/* n matrices exp(i eps H_i), H_i from normals 8 i .. 8 i + 7 of stream seed. */
void syn_su3(uint64_t seed, double eps, long n, cplx *out) {
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) {
    double h[8];
    for (int a = 0; a < 8; ++a) h[a] = syn_normal(seed, 8 * (uint64_t)i + (uint64_t)a);
    cplx H[3][3], A[3][3], U[3][3];
    hermitian_from_coeffs(h, H);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) A[r][c] = I * eps * H[r][c];
    mat_exp(A, U);
    reunitarise(U);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) out[9 * i + 3 * r + c] = U[r][c];
  }
}

/* The traceless Hermitian generators H_i themselves (for tests of the draw). */
void syn_hermitian(uint64_t seed, long n, cplx *out) {
  for (long i = 0; i < n; ++i) {
    double h[8];
    for (int a = 0; a < 8; ++a) h[a] = syn_normal(seed, 8 * (uint64_t)i + (uint64_t)a);
    cplx H[3][3];
    hermitian_from_coeffs(h, H);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) out[9 * i + 3 * r + c] = H[r][c];
  }
}

/* n complex numbers with independent N(0, 1/2) real and imaginary parts. */
void syn_gaussian(uint64_t seed, long n, cplx *out) {
  const double s = 1.0 / sqrt(2.0);
#pragma omp parallel for schedule(static)
  for (long k = 0; k < n; ++k)
    out[k] = s * syn_normal(seed, 2 * (uint64_t)k) + I * s * syn_normal(seed, 2 * (uint64_t)k + 1);
}
