/*
 * afd_oracle_nu.c -- plain FP64 CPU oracle of Core AFD on non-uniform samples.
 *
 * TEST INFRASTRUCTURE ONLY (see afd_oracle.c); it shares no code with the
 * CUDA path.
 *
 * The remark after Step 2 of the algorithm of Sec. 3.2 allows non-uniform
 * sampling.  The signal is known at z_m = exp(i theta_m), m = 0..N-1, with
 * quadrature weights w_m of the normalised measure dt / 2 pi (sum w_m = 1),
 * and the rectangle rule of Eq. (formula1) becomes the weighted sum
 *     <G, e_a>~ = sqrt(1 - |a|^2) sum_m w_m G(z_m) / (1 - a conj(z_m)),
 * which is Eq. (formula1) itself when theta_m = 2 pi m / N and w_m = 1/N.
 * The dictionary grid keeps L equispaced angles, a_{s,j} = r_s exp(2 pi i j / L)
 * (Eq. (ku1) with L in place of N).  Selection, the Blaschke update of Sec. 2
 * and delta of Eq. (er) are unchanged, with the energy E = sum_m w_m |G(z_m)|^2.
 * Everything is the direct O(M L N) definition; no transform.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NU_PI 3.14159265358979323846264338327950288

typedef double complex cplx;

static int nu_check(int N, const double* theta, const double* w) {
  if (N <= 0 || !theta || !w) return -1;
  for (int m = 0; m < N; ++m) {
    if (!(theta[m] >= 0.0 && theta[m] < 2.0 * NU_PI) || !(w[m] > 0.0)) return -1;
    if (m > 0 && !(theta[m] > theta[m - 1])) return -1;
  }
  return 0;
}

static cplx nu_inner(int N, const cplx* G, const cplx* z, const double* w, cplx a) {
  double scale = sqrt(1.0 - creal(a * conj(a)));
  cplx acc = 0.0;
  for (int m = 0; m < N; ++m) acc += w[m] * G[m] / (1.0 - a * conj(z[m]));
  return scale * acc;
}

static cplx* nu_points(int N, const double* theta) {
  cplx* z = (cplx*)malloc(sizeof(cplx) * (size_t)N);
  if (!z) return NULL;
  for (int m = 0; m < N; ++m) z[m] = cos(theta[m]) + I * sin(theta[m]);
  return z;
}

/* out[0..1] = <G, e_a>~ at one point a of the disc (weighted rectangle rule). */
int oracle_nu_inner(int N, const double* G, const double* theta, const double* w, double a_re, double a_im,
                    double* out) {
  if (nu_check(N, theta, w) || !G || !out) return -1;
  cplx a = a_re + I * a_im;
  if (creal(a * conj(a)) >= 1.0) return -1;
  cplx* z = nu_points(N, theta);
  if (!z) return -1;
  cplx v = nu_inner(N, (const cplx*)G, z, w, a);
  free(z);
  out[0] = creal(v);
  out[1] = cimag(v);
  return 0;
}

/* Weighted energy sum_m w_m |G(z_m)|^2. */
double oracle_nu_energy(int N, const double* G, const double* w) {
  const cplx* g = (const cplx*)G;
  double acc = 0.0;
  for (int m = 0; m < N; ++m) acc += w[m] * creal(g[m] * conj(g[m]));
  return acc;
}

/* The Blaschke update of Sec. 2 at the points z_m (Gout may alias G). */
int oracle_nu_update(int N, const double* G, const double* theta, double a_re, double a_im, double c_re,
                     double c_im, double* Gout) {
  if (N <= 0 || !G || !theta || !Gout) return -1;
  cplx a = a_re + I * a_im, c = c_re + I * c_im;
  double aa = creal(a * conj(a));
  if (aa >= 1.0) return -1;
  double na = sqrt(1.0 - aa);
  const cplx* g = (const cplx*)G;
  cplx* o = (cplx*)Gout;
  for (int m = 0; m < N; ++m) {
    cplx z = cos(theta[m]) + I * sin(theta[m]);
    cplx e = na / (1.0 - conj(a) * z);
    o[m] = (g[m] - c * e) * (1.0 - conj(a) * z) / (z - a);
  }
  return 0;
}

/*
 * Core AFD on non-uniform samples: K_max greedy steps with the grid of L
 * angles; ties go to the lowest flat index s L + j.  Arguments and outputs as
 * oracle_decompose (flat indices use L), plus theta[N] (ascending, in
 * [0, 2 pi)), w[N] (> 0) and L >= 1.  Returns the steps done, or -1.
 */
int oracle_nu_decompose(int N, const double* G, const double* theta, const double* w, int M, const double* radii,
                        int L, int K_max, double energy_tol, const int* forced_idx, int compute_grid,
                        double* a_out, double* coeff_out, int* idx_out, int* own_idx_out, double* objmax_out,
                        double* obj2_out, double* objused_out, double* delta_out, double* energy_out,
                        double* G_final) {
  if (nu_check(N, theta, w) || !G || M <= 0 || !radii || L <= 0 || K_max <= 0) return -1;
  for (int s = 0; s < M; ++s) {
    if (!(radii[s] >= 0.0 && radii[s] < 1.0)) return -1;
    if (s > 0 && !(radii[s] > radii[s - 1])) return -1;
  }
  if (!compute_grid) {
    if (!forced_idx) return -1;
    for (int k = 0; k < K_max; ++k)
      if (forced_idx[2 * k] < 0) return -1;
  }
  long total = (long)M * (long)L;
  cplx* g = (cplx*)malloc(sizeof(cplx) * (size_t)N);
  cplx* z = nu_points(N, theta);
  cplx* A = compute_grid ? (cplx*)malloc(sizeof(cplx) * (size_t)total) : NULL;
  if (!g || !z || (compute_grid && !A)) {
    free(g);
    free(z);
    free(A);
    return -1;
  }
  memcpy(g, G, sizeof(cplx) * (size_t)N);
  double E1 = oracle_nu_energy(N, (const double*)g, w);
  if (delta_out) delta_out[0] = 1.0;
  if (energy_out) energy_out[0] = E1;
  int steps = 0;
  for (int k = 0; k < K_max; ++k) {
    long own = -1;
    double best = -1.0, second = -1.0;
    if (compute_grid) {
#pragma omp parallel for schedule(static)
      for (long f = 0; f < total; ++f) {
        int s = (int)(f / L), j = (int)(f % L);
        double t = 2.0 * NU_PI * (double)j / (double)L;
        A[f] = nu_inner(N, g, z, w, radii[s] * cos(t) + I * (radii[s] * sin(t)));
      }
      for (long f = 0; f < total; ++f) {
        double v = creal(A[f] * conj(A[f]));
        if (v > best) {
          second = best;
          best = v;
          own = f;
        } else if (v > second) {
          second = v;
        }
      }
    }
    int s_used, j_used;
    if (forced_idx && forced_idx[2 * k] >= 0) {
      s_used = forced_idx[2 * k];
      j_used = forced_idx[2 * k + 1];
      if (s_used >= M || j_used < 0 || j_used >= L) {
        free(g);
        free(z);
        free(A);
        return -1;
      }
    } else {
      s_used = (int)(own / L);
      j_used = (int)(own % L);
    }
    double t = 2.0 * NU_PI * (double)j_used / (double)L;
    cplx a = radii[s_used] * cos(t) + I * (radii[s_used] * sin(t));
    cplx c = compute_grid ? A[(long)s_used * L + j_used] : nu_inner(N, g, z, w, a);
    if (a_out) { a_out[2 * k] = creal(a); a_out[2 * k + 1] = cimag(a); }
    if (coeff_out) { coeff_out[2 * k] = creal(c); coeff_out[2 * k + 1] = cimag(c); }
    if (idx_out) { idx_out[2 * k] = s_used; idx_out[2 * k + 1] = j_used; }
    if (own_idx_out) {
      own_idx_out[2 * k] = own >= 0 ? (int)(own / L) : -1;
      own_idx_out[2 * k + 1] = own >= 0 ? (int)(own % L) : -1;
    }
    if (objmax_out) objmax_out[k] = best;
    if (obj2_out) obj2_out[k] = second;
    if (objused_out) objused_out[k] = creal(c * conj(c));
    oracle_nu_update(N, (const double*)g, theta, creal(a), cimag(a), creal(c), cimag(c), (double*)g);
    double E = oracle_nu_energy(N, (const double*)g, w);
    double delta = E1 > 0.0 ? E / E1 : 0.0;
    if (delta_out) delta_out[k + 1] = delta;
    if (energy_out) energy_out[k + 1] = E;
    steps = k + 1;
    if (energy_tol > 0.0 && delta <= energy_tol) break;
  }
  if (G_final) memcpy(G_final, g, sizeof(cplx) * (size_t)N);
  free(g);
  free(z);
  free(A);
  return steps;
}
