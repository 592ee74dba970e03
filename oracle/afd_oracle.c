/*
 * afd_oracle.c -- plain, slow FP64 CPU oracle of 1-D (Core) AFD.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file.  Only the test suite, the smoke check and the bench's
 * CPU-baseline leg use it, to produce the values the CUDA path is compared
 * against.  It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes (Gao, Ku, Qian, "Fast algorithm of adaptive Fourier
 * series", arXiv:1711.08604):
 *   - the discretised inner product <G, e_a>~ of Sec. 3.1, Eq. (formula1) /
 *     Eq. (term81): a rectangle rule on the N points z_m = exp(2 pi i m / N),
 *       <G, e_a>~ = sum_m sqrt(1-|a|^2)/N * G(z_m) / (1 - a conj(z_m));
 *   - on the polar grid a_{s,j} = r_s exp(2 pi i j / N) of Eq. (ku1) and
 *     Sec. 3.2 (the paper writes r_s W^{-j} with W = exp(-2 pi i / N));
 *   - the maximal selection of Eq. (ak), restricted to that grid as in Step 2
 *     of the algorithm of Sec. 3.2: argmax of |<G_k, e_a>~|^2, ties going to
 *     the lowest flat index s*N + j;
 *   - the reduced-remainder (Blaschke) update of Sec. 2,
 *       G_{k+1}(z) = (G_k(z) - <G_k, e_{a_k}> e_{a_k}(z)) (1 - conj(a_k) z) / (z - a_k),
 *     with e_a(z) = sqrt(1-|a|^2) / (1 - conj(a) z);
 *   - the discrete energy E_k = (1/N) sum_m |G_k(z_m)|^2 and the relative
 *     error delta_n = ||G - S_n||^2 / ||G||^2 of Eq. (er), which equals
 *     E_{n+1} / E_1 because G - S_n = G_{n+1} times a unimodular Blaschke
 *     product on the circle (Eq. (Sn) and the remark after the energy
 *     identity in Sec. 2).
 *
 * Nothing here uses an FFT: this is the direct O(M N^2) method the paper
 * accelerates.  Loops follow the definitions; the only shared work is the
 * table of sample points z_m, computed once per call.  OpenMP splits the grid
 * loop over (s, j) pairs; each inner product is summed by one thread in order
 * m = 0..N-1, so results do not depend on the thread count.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846264338327950288

typedef double complex cplx;

/* Sample point z_m = exp(2 pi i m / N) (Sec. 3.1: t_m = 2 pi m / N). */
static cplx sample_point(int m, int N) {
  double t = 2.0 * ORACLE_PI * (double)m / (double)N;
  return cos(t) + I * sin(t);
}

/* Grid point a_{s,j} = r_s exp(2 pi i j / N) (Eq. (ku1), Sec. 3.2). */
static cplx grid_point(double r, int j, int N) {
  double t = 2.0 * ORACLE_PI * (double)j / (double)N;
  return r * cos(t) + I * (r * sin(t));
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Rectangle-rule inner product <G, e_a>~ at one point a of the disc,
 * Eq. (formula1).  G holds N complex samples, interleaved (re, im). */
static cplx inner_with_table(int N, const cplx* G, const cplx* z, cplx a) {
  double scale = sqrt(1.0 - creal(a * conj(a))) / (double)N;
  cplx acc = 0.0;
  for (int m = 0; m < N; ++m) acc += G[m] / (1.0 - a * conj(z[m]));
  return scale * acc;
}

static cplx* make_points(int N) {
  cplx* z = (cplx*)malloc(sizeof(cplx) * (size_t)N);
  if (!z) return NULL;
  for (int m = 0; m < N; ++m) z[m] = sample_point(m, N);
  return z;
}

/* out[0..1] = <G, e_a>~ for a = a_re + i a_im (|a| < 1).  Returns 0, or -1 on
 * bad arguments. */
int oracle_inner(int N, const double* G, double a_re, double a_im, double* out) {
  if (N <= 0 || !G || !out) return -1;
  cplx a = a_re + I * a_im;
  if (creal(a * conj(a)) >= 1.0) return -1;
  cplx* z = make_points(N);
  if (!z) return -1;
  cplx v = inner_with_table(N, (const cplx*)G, z, a);
  free(z);
  out[0] = creal(v);
  out[1] = cimag(v);
  return 0;
}

/* out[p] = <G, e_{a_p}>~ for n arbitrary points a_p (interleaved complex), by
 * the rectangle rule of Eq. (formula1); OpenMP over points. */
int oracle_inner_many(int N, const double* G, int n, const double* points, double* out) {
  if (N <= 0 || n <= 0 || !G || !points || !out) return -1;
  for (int p = 0; p < n; ++p) {
    cplx a = points[2 * p] + I * points[2 * p + 1];
    if (creal(a * conj(a)) >= 1.0) return -1;
  }
  cplx* z = make_points(N);
  if (!z) return -1;
#pragma omp parallel for schedule(static)
  for (int p = 0; p < n; ++p) {
    cplx a = points[2 * p] + I * points[2 * p + 1];
    cplx v = inner_with_table(N, (const cplx*)G, z, a);
    out[2 * p] = creal(v);
    out[2 * p + 1] = cimag(v);
  }
  free(z);
  return 0;
}

/* A[s*N + j] = <G, e_{a_{s,j}}>~ for the whole M x N grid (Step 1 of the
 * algorithm, evaluated directly as in Eq. (term81)).  A is 2*M*N doubles. */
int oracle_grid(int N, const double* G, int M, const double* radii, double* A) {
  if (N <= 0 || M <= 0 || !G || !radii || !A) return -1;
  for (int s = 0; s < M; ++s)
    if (!(radii[s] >= 0.0 && radii[s] < 1.0)) return -1;
  cplx* z = make_points(N);
  if (!z) return -1;
  const cplx* g = (const cplx*)G;
  cplx* out = (cplx*)A;
  long total = (long)M * (long)N;
#pragma omp parallel for schedule(static)
  for (long f = 0; f < total; ++f) {
    int s = (int)(f / N), j = (int)(f % N);
    out[f] = inner_with_table(N, g, z, grid_point(radii[s], j, N));
  }
  free(z);
  return 0;
}

/* Discrete squared norm (1/N) sum_m |e_a(z_m)|^2 of the normalised Szego
 * kernel at the grid point a = r (angle 0); by rotation it is the same at
 * every angle of the circle.  The continuous norm is 1; the discrete one
 * exceeds it when r^N is not negligible. */
double oracle_kernel_norm2(int N, double r) {
  if (N <= 0 || !(r >= 0.0 && r < 1.0)) return -1.0;
  cplx a = r;
  double na = sqrt(1.0 - r * r), acc = 0.0;
  for (int m = 0; m < N; ++m) {
    cplx e = na / (1.0 - conj(a) * sample_point(m, N));
    acc += creal(e * conj(e));
  }
  return acc / (double)N;
}

/* Maximal selection on the grid (Step 2): index of the largest objective,
 * |A|^2, or |A|^2 / ||e_a||_N^2 when norm2 (one value per radius) is given
 * (the renormalised selection), the lowest flat index winning ties.  Also
 * reports the largest value and the largest value at any other position (for
 * near-tie analysis). */
static long argmax_grid(const cplx* A, long total, int N, const double* norm2, double* best, double* second) {
  long arg = 0;
  double b = -1.0, s2 = -1.0;
  for (long f = 0; f < total; ++f) {
    double v = creal(A[f] * conj(A[f]));
    if (norm2) v /= norm2[f / N];
    if (v > b) {
      s2 = b;
      b = v;
      arg = f;
    } else if (v > s2) {
      s2 = v;
    }
  }
  *best = b;
  *second = s2;
  return arg;
}

/* Reduced-remainder update of Sec. 2:
 *   G_{k+1}(z_m) = (G_k(z_m) - c e_a(z_m)) (1 - conj(a) z_m) / (z_m - a),
 * e_a(z) = sqrt(1 - |a|^2) / (1 - conj(a) z), with c = <G_k, e_a>.  Gout may
 * alias G. */
int oracle_update(int N, const double* G, double a_re, double a_im, double c_re,
                  double c_im, double* Gout) {
  if (N <= 0 || !G || !Gout) return -1;
  cplx a = a_re + I * a_im, c = c_re + I * c_im;
  double aa = creal(a * conj(a));
  if (aa >= 1.0) return -1;
  double na = sqrt(1.0 - aa);
  const cplx* g = (const cplx*)G;
  cplx* o = (cplx*)Gout;
  for (int m = 0; m < N; ++m) {
    cplx z = sample_point(m, N);
    cplx e = na / (1.0 - conj(a) * z);
    cplx blaschke_inv = (1.0 - conj(a) * z) / (z - a);
    o[m] = (g[m] - c * e) * blaschke_inv;
  }
  return 0;
}

/*
 * Off-grid refinement of a selected point (optional; not part of the paper,
 * whose selection stays on the grid of Sec. 3.2).  The discrete objective
 * f(a) = |<G, e_a>~|^2 = (1 - |a|^2) |S(a)|^2 / N^2, S(a) = sum_m G(z_m) / (1 - a conj(z_m)),
 * is maximised over the open disc from the grid point a0 by damped Newton
 * steps on h = log f = log(1 - |a|^2) + 2 Re log S(a) + const in the real
 * coordinates (x, y) of a.  With L1 = S'/S and L2 = S''/S - L1^2 (S is
 * holomorphic, so 2 Re log S is harmonic):
 *   grad h = (2 Re L1 - 2x/rho, -2 Im L1 - 2y/rho),          rho = 1 - |a|^2,
 *   h_xx = 2 Re L2 - 2/rho - 4x^2/rho^2,  h_xy = -2 Im L2 - 4xy/rho^2,
 *   h_yy = -2 Re L2 - 2/rho - 4y^2/rho^2,
 *   S'(a) = sum G z_bar / (1 - a z_bar)^2,  S''(a) = 2 sum G z_bar^2 / (1 - a z_bar)^3.
 * Each iteration: stop unless the Hessian is negative definite; a Newton
 * step shorter than 1e-6 is taken as it is (the quadratic convergence near
 * the maximum, where f no longer resolves the gain); a longer one, shortened
 * to at most half the distance to the circle, is tried, then halved up to
 * three times, and taken at the first try that increases f (none: stop).
 * Stop after a step shorter than 1e-13.  Returns the refined a and
 * c = <G, e_a>~ = sqrt(1 - |a|^2) S(a) / N.
 */
static void refine_sums(int N, const cplx* g, const cplx* z, cplx a, cplx* S0, cplx* S1, cplx* S2) {
  cplx s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int m = 0; m < N; ++m) {
    cplx zb = conj(z[m]);
    cplx v = 1.0 / (1.0 - a * zb);
    cplx t = g[m] * v;
    cplx w = zb * v;
    s0 += t;
    s1 += t * w;
    s2 += 2.0 * t * w * w;
  }
  *S0 = s0;
  *S1 = s1;
  *S2 = s2;
}

static double refine_f(cplx a, cplx S) { return (1.0 - creal(a * conj(a))) * creal(S * conj(S)); }

static cplx refine_point(int N, const cplx* g, const cplx* z, cplx a, int iters, cplx* c_out) {
  cplx S, S1, S2;
  refine_sums(N, g, z, a, &S, &S1, &S2);
  double f = refine_f(a, S);
  for (int it = 0; it < iters; ++it) {
    if (S == 0.0) break;
    cplx L1 = S1 / S;
    cplx L2 = S2 / S - L1 * L1;
    double x = creal(a), y = cimag(a);
    double rho = 1.0 - (x * x + y * y);
    double gx = 2.0 * creal(L1) - 2.0 * x / rho;
    double gy = -2.0 * cimag(L1) - 2.0 * y / rho;
    double hxx = 2.0 * creal(L2) - 2.0 / rho - 4.0 * x * x / (rho * rho);
    double hxy = -2.0 * cimag(L2) - 4.0 * x * y / (rho * rho);
    double hyy = -2.0 * creal(L2) - 2.0 / rho - 4.0 * y * y / (rho * rho);
    double det = hxx * hyy - hxy * hxy;
    if (!(det > 0.0 && hxx < 0.0)) break;
    double dx = -(hyy * gx - hxy * gy) / det;
    double dy = -(hxx * gy - hxy * gx) / det;
    double lim = 0.5 * (1.0 - sqrt(x * x + y * y));
    double n = sqrt(dx * dx + dy * dy);
    if (n < 1e-6 && n < lim) {
      a += dx + I * dy;
      refine_sums(N, g, z, a, &S, &S1, &S2);
      f = refine_f(a, S);
      if (n < 1e-13) break;
      continue;
    }
    if (n > lim) {
      dx *= lim / n;
      dy *= lim / n;
    }
    int taken = 0;
    for (int h = 0; h < 4; ++h) {
      cplx an = a + (dx + I * dy);
      cplx T, T1, T2;
      refine_sums(N, g, z, an, &T, &T1, &T2);
      double fn = refine_f(an, T);
      if (fn > f) {
        a = an;
        S = T;
        S1 = T1;
        S2 = T2;
        f = fn;
        taken = 1;
        break;
      }
      dx *= 0.5;
      dy *= 0.5;
    }
    if (!taken) break;
    if (sqrt(dx * dx + dy * dy) < 1e-13) break;
  }
  *c_out = sqrt(1.0 - creal(a * conj(a))) * S / (double)N;
  return a;
}

int oracle_refine(int N, const double* G, double a_re, double a_im, int iters, double* a_out, double* c_out) {
  if (N <= 0 || !G || !a_out || !c_out || iters < 0) return -1;
  cplx a = a_re + I * a_im;
  if (creal(a * conj(a)) >= 1.0) return -1;
  cplx* z = make_points(N);
  if (!z) return -1;
  cplx c;
  a = refine_point(N, (const cplx*)G, z, a, iters, &c);
  free(z);
  a_out[0] = creal(a);
  a_out[1] = cimag(a);
  c_out[0] = creal(c);
  c_out[1] = cimag(c);
  return 0;
}

/* Discrete energy (1/N) sum_m |G(z_m)|^2: the rectangle rule for the norm in
 * the normalised measure dt / 2 pi used by Eq. (formula2). */
double oracle_energy(int N, const double* G) {
  const cplx* g = (const cplx*)G;
  double acc = 0.0;
  for (int m = 0; m < N; ++m) acc += creal(g[m] * conj(g[m]));
  return acc / (double)N;
}

/*
 * Core AFD, K_max greedy steps of Sec. 2 with the selection of Sec. 3.2.
 *
 * Inputs: N samples of G (interleaved complex), M ascending radii in [0, 1),
 * K_max >= 1, energy_tol (stop once delta_k <= energy_tol; 0 disables).
 * force_a1_zero != 0 sets a_1 = 0 (requires radii[0] == 0; index (0, 0)).
 * renormalise != 0 selects by |A|^2 / ||e_a||_N^2 (oracle_kernel_norm2) instead
 * of |A|^2; the coefficient is <G_k, e_a>~ either way.
 * forced_idx (2*K_max ints, (s, j) per step, s < 0 meaning "free") makes a
 * step use the given grid point instead of the argmax; compute_grid == 0
 * skips the O(M N^2) grid (allowed only when every step is forced) and takes
 * the coefficient from oracle_inner at the forced point.
 *
 * Outputs (any may be NULL):
 *   a_out[2k], coeff_out[2k]    a_k and <G_k, e_{a_k}>~ of the step used;
 *   idx_out[2k]                 (s, j) actually used;
 *   own_idx_out[2k]             the oracle's own argmax (-1 if no grid);
 *   objmax_out[k], obj2_out[k]  largest objective and largest at another point;
 *   objused_out[k]              objective at the point used;
 *   delta_out[0..K]             delta_0 = 1, delta_k = E_{k+1} / E_1;
 *   energy_out[0..K]            E_1 .. E_{K+1};
 *   G_final                     G_{k+1} after the last step (2N doubles);
 *   G_steps                     G_k at the start of every step k = 1..steps
 *                               (2N doubles per step, one after another).
 * offgrid_iters > 0 refines each step's grid point off the grid
 * (refine_point) before the coefficient and the update; idx_out then holds
 * the grid point the refinement started from.
 * Returns the number of steps done (>= 1), or -1 on bad arguments.
 */
int oracle_decompose(int N, const double* G, int M, const double* radii, int K_max,
                     double energy_tol, int force_a1_zero, int renormalise, const int* forced_idx,
                     int compute_grid, double* a_out, double* coeff_out, int* idx_out,
                     int* own_idx_out, double* objmax_out, double* obj2_out,
                     double* objused_out, double* delta_out, double* energy_out,
                     double* G_final, double* G_steps, int offgrid_iters) {
  if (N <= 0 || M <= 0 || K_max <= 0 || !G || !radii) return -1;
  for (int s = 0; s < M; ++s) {
    if (!(radii[s] >= 0.0 && radii[s] < 1.0)) return -1;
    if (s > 0 && !(radii[s] > radii[s - 1])) return -1;
  }
  if (force_a1_zero && radii[0] != 0.0) return -1;
  if (!compute_grid) {
    if (!forced_idx) return -1;
    for (int k = 0; k < K_max; ++k) {
      if (forced_idx[2 * k] < 0 && !(k == 0 && force_a1_zero)) return -1;
    }
  }
  long total = (long)M * (long)N;
  cplx* g = (cplx*)malloc(sizeof(cplx) * (size_t)N);
  cplx* A = compute_grid ? (cplx*)malloc(sizeof(cplx) * (size_t)total) : NULL;
  cplx* z = make_points(N);
  double* norm2 = renormalise ? (double*)malloc(sizeof(double) * (size_t)M) : NULL;
  if (!g || !z || (compute_grid && !A) || (renormalise && !norm2)) {
    free(g);
    free(A);
    free(z);
    free(norm2);
    return -1;
  }
  for (int s = 0; renormalise && s < M; ++s) norm2[s] = oracle_kernel_norm2(N, radii[s]);
  memcpy(g, G, sizeof(cplx) * (size_t)N);
  double E1 = oracle_energy(N, (const double*)g);
  if (delta_out) delta_out[0] = 1.0;
  if (energy_out) energy_out[0] = E1;

  int steps = 0;
  for (int k = 0; k < K_max; ++k) {
    int s_used, j_used;
    double best = -1.0, second = -1.0;
    if (G_steps) memcpy(G_steps + (size_t)2 * N * k, g, sizeof(cplx) * (size_t)N);
    long own = -1;
    if (compute_grid) {
      oracle_grid(N, (const double*)g, M, radii, (double*)A);
      own = argmax_grid(A, total, N, norm2, &best, &second);
    }
    if (k == 0 && force_a1_zero) {
      s_used = 0;
      j_used = 0;
    } else if (forced_idx && forced_idx[2 * k] >= 0) {
      s_used = forced_idx[2 * k];
      j_used = forced_idx[2 * k + 1];
      if (s_used >= M || j_used < 0 || j_used >= N) {
        free(g);
        free(A);
        free(z);
        free(norm2);
        return -1;
      }
    } else {
      s_used = (int)(own / N);
      j_used = (int)(own % N);
    }
    cplx a = grid_point(radii[s_used], j_used, N);
    cplx c = compute_grid ? A[(long)s_used * N + j_used] : inner_with_table(N, g, z, a);
    double used = creal(c * conj(c));
    if (norm2) used /= norm2[s_used];
    if (offgrid_iters > 0 && !(k == 0 && force_a1_zero)) a = refine_point(N, g, z, a, offgrid_iters, &c);

    if (a_out) { a_out[2 * k] = creal(a); a_out[2 * k + 1] = cimag(a); }
    if (coeff_out) { coeff_out[2 * k] = creal(c); coeff_out[2 * k + 1] = cimag(c); }
    if (idx_out) { idx_out[2 * k] = s_used; idx_out[2 * k + 1] = j_used; }
    if (own_idx_out) {
      own_idx_out[2 * k] = own >= 0 ? (int)(own / N) : -1;
      own_idx_out[2 * k + 1] = own >= 0 ? (int)(own % N) : -1;
    }
    if (objmax_out) objmax_out[k] = best;
    if (obj2_out) obj2_out[k] = second;
    if (objused_out) objused_out[k] = used;

    oracle_update(N, (const double*)g, creal(a), cimag(a), creal(c), cimag(c), (double*)g);
    double E = oracle_energy(N, (const double*)g);
    double delta = E1 > 0.0 ? E / E1 : 0.0;
    if (delta_out) delta_out[k + 1] = delta;
    if (energy_out) energy_out[k + 1] = E;
    steps = k + 1;
    if (energy_tol > 0.0 && delta <= energy_tol) break;
  }
  if (G_final) memcpy(G_final, g, sizeof(cplx) * (size_t)N);
  free(g);
  free(A);
  free(z);
  free(norm2);
  return steps;
}
