// Partial sums S_n of a Core AFD expansion on the N sample points, FP64.
//
// Eq. (Sn) (Sec. 2): S_n(z) = sum_{k=1..n} <G_k, e_{a_k}> B_k(z) with the
// Takenaka-Malmquist functions
//   B_k(z) = e_{a_k}(z) prod_{l<k} (z - a_l) / (1 - conj(a_l) z),
//   e_a(z) = sqrt(1 - |a|^2) / (1 - conj(a) z),
// in the normalised measure dt / 2 pi (no 1 / sqrt(2 pi) factor).  One thread
// per sample point carries the running Blaschke product.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "../../include/afd.h"
#include "afd_host.h"

using namespace afd;

namespace {

__global__ void __launch_bounds__(256)
k_synthesize(int N, const double2* __restrict__ a, const double2* __restrict__ c, int n,
             double2* __restrict__ S, int prefix_stride) {
  const int m = blockIdx.x * 256 + threadIdx.x;
  if (m >= N) return;
  double zs, zc;
  sincospi(2.0 * (double)m / (double)N, &zs, &zc);
  double pr = 1.0, pi = 0.0;  // prod_{l<k} (z - a_l) / (1 - conj(a_l) z)
  double sr = 0.0, si = 0.0;
  for (int k = 0; k < n; ++k) {
    const double2 ak = a[k], ck = c[k];
    // d = 1 - conj(a) z
    const double dr = 1.0 - (ak.x * zc + ak.y * zs);
    const double di = -(ak.x * zs - ak.y * zc);
    const double inv = 1.0 / (dr * dr + di * di);
    const double na = sqrt(fmax(0.0, 1.0 - (ak.x * ak.x + ak.y * ak.y)));
    // e = na / d = na conj(d) / |d|^2
    const double er = na * dr * inv, ei = -na * di * inv;
    // term = c e P
    const double tr = ck.x * er - ck.y * ei, ti = ck.x * ei + ck.y * er;
    sr += tr * pr - ti * pi;
    si += tr * pi + ti * pr;
    if (prefix_stride) S[(size_t)k * prefix_stride + m] = make_double2(sr, si);
    // P *= (z - a) / d
    const double nr = zc - ak.x, ni = zs - ak.y;
    const double qr = (nr * dr + ni * di) * inv, qi = (ni * dr - nr * di) * inv;
    const double p2r = pr * qr - pi * qi;
    pi = pr * qi + pi * qr;
    pr = p2r;
  }
  if (!prefix_stride) S[m] = make_double2(sr, si);
}

bool is_device(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" afd_status afd_synthesize(int N, const double* a, const double* coeff, int n, int all_prefixes,
                                     double* S_out) {
  clear_last_error();
  if (N < 1 || N > (1 << 24) || n < 1 || n > (1 << 20) || !a || !coeff || !S_out)
    return set_error(AFD_ERR_INVALID, "afd_synthesize: need 1 <= N <= 2^24, 1 <= n and non-NULL arrays");
  for (int k = 0; k < n && !is_device(a); ++k)
    if (!(a[2 * k] * a[2 * k] + a[2 * k + 1] * a[2 * k + 1] < 1.0))
      return set_error(AFD_ERR_INVALID, "afd_synthesize: |a_%d| >= 1", k);
  const size_t out_n = (size_t)N * (all_prefixes ? n : 1);
  double2 *da = nullptr, *dc = nullptr, *dS = nullptr;
  auto release = [&] {
    if (da && !is_device(a)) cudaFree(da);
    if (dc && !is_device(coeff)) cudaFree(dc);
    if (dS && !is_device(S_out)) cudaFree(dS);
  };
  cudaError_t e = cudaSuccess;
  if (is_device(a)) da = (double2*)a;
  else if ((e = cudaMalloc(&da, 16 * (size_t)n)) == cudaSuccess)
    e = cudaMemcpy(da, a, 16 * (size_t)n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    if (is_device(coeff)) dc = (double2*)coeff;
    else if ((e = cudaMalloc(&dc, 16 * (size_t)n)) == cudaSuccess)
      e = cudaMemcpy(dc, coeff, 16 * (size_t)n, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) {
    if (is_device(S_out)) dS = (double2*)S_out;
    else e = cudaMalloc(&dS, 16 * out_n);
  }
  if (e == cudaSuccess) {
    k_synthesize<<<(N + 255) / 256, 256>>>(N, da, dc, n, dS, all_prefixes ? N : 0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !is_device(S_out)) e = cudaMemcpy(S_out, dS, 16 * out_n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  release();
  if (e != cudaSuccess) return cuda_fail(e, "afd_synthesize", __LINE__);
  return AFD_OK;
}
