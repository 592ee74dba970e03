// Host-side helpers shared by the library's translation units (plans,
// batches, serving).  Not part of the public C ABI.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/afd.h"
#include "afd_internal.h"

#define CUDA_TRY(expr)                                                  \
  do {                                                                  \
    cudaError_t _e = (expr);                                            \
    if (_e != cudaSuccess) return ::afd::cuda_fail(_e, #expr, __LINE__); \
  } while (0)

#define AFD_TRY(expr)            \
  do {                           \
    afd_status _s = (expr);      \
    if (_s != AFD_OK) return _s; \
  } while (0)

namespace afd {

// Error text of the calling thread (afd_last_error).
afd_status set_error(afd_status st, const char* fmt, ...);
void clear_last_error();
const char* last_error_text();
afd_status cuda_fail(cudaError_t e, const char* what, int line);

afd_status ensure_configured(int dev);  // kernel attributes, once per device
int ilog2(int n);
bool is_pow2(int n);
inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

afd_status check_opts(const afd_plan_opts& o);
afd_status check_size(int N, int prec, bool allow_two_pass = false, bool allow_mixed = false);
afd_status check_radii(const double* radii, int M);
// opts (NULL: defaults) validated into o, with no CUDA call.
afd_status resolve_opts(const afd_plan_opts* in, afd_plan_opts& o);
// dev = the device o names (-1: the current one), checked to exist.
afd_status resolve_device(const afd_plan_opts& o, int& dev);
// resolve_opts, then resolve_device.
afd_status normalise_opts(const afd_plan_opts* in, afd_plan_opts& o, int& dev);

// Makes `dev` current for the scope and restores the caller's device.
struct DeviceScope {
  int prev = -1;
  bool ok = true;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (dev >= 0 && dev != prev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceScope() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Device tables of one (N, radii) pair (see afd_runtime.cu).
struct Tables {
  int N = 0, M = 0;  // N: grid angles (and samples, unless non-uniform)
  std::vector<double> radii;
  void* mem = nullptr;
  size_t bytes = 0;
  PlanDev dev{};
  // non-uniform samples: nN samples at exp(i theta_m), spectrum length nLc
  bool nu = false;
  int nN = 0, nLc = 0;
  void* nu_mem = nullptr;
  Tables() = default;
  Tables(const Tables&) = delete;
  Tables& operator=(const Tables&) = delete;
  ~Tables();
  int prec = 1;      // the precision the tables were built for (they differ for split sizes)
  afd_status build(int N, const double* radii, int M, int prec);
  // grid of L angles; samples theta[nN] (ascending in [0, 2 pi)) with
  // weights w[nN] (NULL: the trapezoid rule)
  afd_status build_nu(int nN, const double* theta, const double* w, int L, const double* radii, int M);
  int samples() const { return nu ? nN : N; }
  int spectrum() const { return nu ? nLc : N; }
  static size_t bytes_for(int N, int M, int prec);  // device bytes build() allocates
};

}  // namespace afd
