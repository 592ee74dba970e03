/*
 * afd.h -- C ABI of the GB300 (sm_103a) implementation of FFT-accelerated
 * 1-D (Core) adaptive Fourier decomposition, after Gao, Ku and Qian, "Fast
 * algorithm of adaptive Fourier series" (arXiv:1711.08604).
 *
 * Notation.  A signal is given by N samples G(z_m) at z_m = exp(2 pi i m / N),
 * m = 0..N-1 (Sec. 3.1: t_m = 2 pi m / N).  The dictionary grid is
 * a_{s,j} = r_s exp(2 pi i j / N) for M radii r_s and the same N angles
 * (Eq. (ku1), Sec. 3.2; the paper writes r_s W^{-j}, W = exp(-2 pi i / N)).
 * Each greedy step k picks a_k = argmax over the grid of |<G_k, e_a>~|^2
 * (Eq. (ak) restricted to the grid, Step 2 of Sec. 3.2), with <G, e_a>~ the
 * rectangle rule of Eq. (formula1) in the normalised measure dt / 2 pi, and
 * replaces G_k by the reduced remainder of Sec. 2,
 *     G_{k+1}(z) = (G_k(z) - <G_k, e_{a_k}> e_{a_k}(z)) (1 - conj(a_k) z) / (z - a_k).
 * The relative error after k steps is delta_k = ||G - S_k||^2 / ||G||^2
 * (Eq. (er)) = E_{k+1} / E_1 with E = (1/N) sum_m |G(z_m)|^2.
 *
 * Conventions for every entry point:
 *   - Complex arrays are interleaved (re, im) doubles.
 *   - Pointers to caller data may be host memory (pageable or pinned) or
 *     device memory of the plan's device; the library copies as needed.  The
 *     caller owns every buffer it passes; nothing is retained after return.
 *   - Calls are synchronous: outputs are complete when the call returns.
 *   - No exception or abort crosses the ABI; errors are returned as
 *     afd_status and described by afd_last_error() (thread-local text).
 *   - Ties in the selection go to the lowest flat index s * N + j, with the
 *     radii in the given (ascending) order.
 */
#ifndef AFD_H
#define AFD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum afd_status {
  AFD_OK = 0,
  AFD_PENDING = 1,          /* serving: request not finished yet */
  AFD_ERR_INVALID = -1,     /* bad argument (size, radius, pointer, option) */
  AFD_ERR_NOMEM = -2,       /* device or host allocation failed */
  AFD_ERR_CUDA = -3,        /* a CUDA call failed; see afd_last_error() */
  AFD_ERR_TIMEOUT = -4,     /* a bounded wait ran out */
  AFD_ERR_BUDGET = -5,      /* request larger than the serving memory budget */
  AFD_ERR_NOT_FOUND = -6,   /* unknown request id */
  AFD_ERR_NUMERIC = -7      /* non-finite objective: input holds NaN or Inf */
} afd_status;

typedef enum afd_precision {
  /* FFTs, grid and selection in FP64; coefficient taken from the FP64 grid. */
  AFD_FP64_PLAIN = 0,
  /* FFTs and grid in FP32 (twiddles and powers from FP64 tables); every grid
   * point whose FP32 objective is within guard_tau (relative) of the largest
   * is re-evaluated by the FP64 direct sum of Eq. (formula1), which decides
   * the selection and gives the coefficient.  Remainder and energy in FP64. */
  AFD_FP32_GUARDED = 1
} afd_precision;

typedef struct afd_plan_opts {
  int precision;       /* afd_precision; default AFD_FP32_GUARDED */
  double guard_tau;    /* FP32 path: relative re-evaluation window; default 1e-4 */
  int guard_cap;       /* FP32 path: most candidates re-evaluated per step, 1..64; default 16 */
  int force_a1_zero;   /* 1: a_1 = 0 (needs radii[0] == 0); default 0 */
  int device;          /* CUDA device ordinal; -1 (default): the current device */
  void* stream;        /* cudaStream_t to run on (not the legacy default stream);
                          NULL (default): a stream owned by the plan */
  int use_graph;       /* 1 (default): replay the step sequence as a CUDA graph */
  int persistent;      /* 1 (default): a single-signal FP32-path decomposition with N <= 4096
                          runs as one persistent cooperative kernel (bounded grid barriers
                          between the phases of a step), and a serving tick whose signals
                          are all FP32-path powers of two up to 16384 runs as one
                          multi-signal persistent launch (every N-class in every phase);
                          2: as 1, and a batch of such signals (mixed-radix sizes too,
                          unless N = 16384 is among them) runs as one multi-signal
                          persistent launch too (by default a batch keeps one launch per
                          kernel per N-class and step, replayed as a graph, which measures
                          faster for batches of 2 to 1024 signals); 0: one launch per
                          kernel per step everywhere.  Results are identical either way. */
  int renormalise;     /* 1: select by |<G_k, e_a>~|^2 / ||e_a||_N^2, the objective divided by
                          the discrete norm (1 + r^N)/(1 - r^N) of the kernel at a grid point
                          (the continuous norm of Sec. 2 is 1; the discrete one inflates the
                          outer circles when r^N is not negligible).  The coefficient is
                          <G_k, e_a>~ either way.  0 (default): the paper's objective. */
  int autotune;        /* batches: 1 (default) chooses, per N-class, the fastest of the grid
                          kernel's bitwise-equivalent variants (points per thread, CTA width)
                          by timing each on the batch's first step; choices are cached per
                          process.  0: the default variant. */
  int grid_variant;    /* -1 (default): as autotune decides; 0..2: use this grid-kernel variant
                          wherever it exists (plans and batches; for tests and profiling) */
  int offgrid_iters;   /* 0 (default): a_k is the grid point of Step 2 (Sec. 3.2).  n in 1..64:
                          plans (uniform samples; not with renormalise) refine each step's grid
                          winner over the open disc by at most n damped Newton steps on the
                          same discrete objective |<G_k, e_a>~|^2, then take the coefficient and
                          the update at the refined a_k (not in the paper); the step's idx
                          stays the grid starting point and flags bit 3 is set.  Batches and
                          servers reject it.  The persistent kernel is not used. */
} afd_plan_opts;

typedef struct afd_plan afd_plan;
typedef struct afd_batch afd_batch;

/* Fills *opts with the defaults above. */
void afd_plan_opts_default(afd_plan_opts* opts);

/* Text of an afd_status value (static storage). */
const char* afd_status_str(afd_status status);

/* Description of the last error raised on the calling thread ("" if none). */
const char* afd_last_error(void);

/* Library version, "major.minor.patch" (static storage). */
const char* afd_version(void);

/*
 * Creates a plan for signals of N samples and the radial grid radii[0..M-1]
 * (Sec. 3.2, Step 1: the paper precomputes and stores r_s^l and the FFT
 * twiddles; the plan holds them on the device, generated in FP64).
 *   N      a power of two, 8 <= N <= 65536, on either path (the method at every
 *          N = 2^K, Sec. 3.2 and the N-sweep of Table 9).  One CTA holds a
 *          transform of up to 16384 points (FP32) or 8192 (FP64); longer ones
 *          run as 2, 4 or 8 such transforms of decimated outputs, except
 *          FP32 N = 65536, which takes the two-pass path through HBM
 *          (single-signal plans only: batches and servers refuse it);
 *          or N = 2^a 3^b 5^c 7^d 11^e 13^f >= 9 that is not a power of two
 *          and has at least two factors, N <= 12800 (FP32 path) or 6400
 *          (FP64 path): the remark after Table 9 (Sec. 4.2) that the
 *          algorithm holds for N = p^K with p prime, taken here as mixed
 *          radices 2, 4, 8, 16 and the primes 3, 5, 7, 11, 13 (so 7^4, 11^3
 *          and 13^3 among others).  Not persistent; not served by afd_serve_*
 *          (power-of-two sizes only there).
 *   radii  host array of M ascending values in [0, 1); copied.
 *   M      1 <= M <= 4096.
 *   opts   NULL for defaults.
 * On success *out owns device memory until afd_plan_destroy.  A plan is not
 * thread-safe: use one plan per host thread.  Errors: AFD_ERR_INVALID for a
 * bad size, radius or option; AFD_ERR_NOMEM; AFD_ERR_CUDA.
 */
afd_status afd_plan_create(afd_plan** out, int N, const double* radii, int M,
                           const afd_plan_opts* opts);

/*
 * Plan for non-uniform samples (the remark after Step 2 of the algorithm of
 * Sec. 3.2: the method holds for non-uniform sampling through non-uniform
 * DFTs).  The signal is known at z_m = exp(i theta_m), m < N, with quadrature
 * weights w_m of the normalised measure dt / 2 pi, and the rectangle rule of
 * Eq. (formula1) becomes
 *     <G, e_a>~ = sqrt(1 - |a|^2) sum_m w_m G(z_m) / (1 - a conj(z_m));
 * the grid keeps L equispaced angles, a_{s,j} = r_s exp(2 pi i j / L); the
 * energy is sum_m w_m |G(z_m)|^2.
 *   N        1 <= N <= 2^20 samples.
 *   theta    host array of N angles, strictly ascending in [0, 2 pi); copied.
 *   weights  host array of N positive weights (normally summing to 1), or
 *            NULL for the trapezoid rule (theta_{m+1} - theta_{m-1}) / (4 pi),
 *            cyclic; copied.
 *   L        grid angles, a power of two, 8 <= L <= 8192.
 *   radii, M as for afd_plan_create; every radius needs r^(64 L) <= 2^-64
 *            (at most 64 folds of the non-uniform DFT onto L angles), else
 *            AFD_ERR_INVALID: use more angles.
 *   opts     the FP32-guarded precision only; force_a1_zero and renormalise
 *            are not supported; persistent is ignored.
 * afd_decompose / afd_decompose_from then take G as N samples at theta and
 * return a_k on the L-angle grid (idx: (s, j), j < L).  Errors as
 * afd_plan_create.
 */
afd_status afd_plan_create_nonuniform(afd_plan** out, int N, const double* theta, const double* weights, int L,
                                      const double* radii, int M, const afd_plan_opts* opts);

/* Frees the plan and its device memory.  NULL is accepted. */
afd_status afd_plan_destroy(afd_plan* plan);

/*
 * Core AFD of one signal: up to K_max greedy steps (Sec. 2 with the grid
 * selection of Sec. 3.2), stopping early once delta_k <= energy_tol
 * (energy_tol = 0 runs all K_max steps).
 *   G          2N doubles, G(z_m) interleaved; host or device pointer.
 *   K_max      >= 1.
 *   a_out      2*K_max doubles: a_k.                    (may be NULL)
 *   coeff_out  2*K_max doubles: <G_k, e_{a_k}>~.        (may be NULL)
 *   delta_out  K_max+1 doubles: delta_0 = 1, delta_k.   (may be NULL)
 *   idx_out    2*K_max ints: grid index (s, j) of a_k.  (may be NULL)
 *   steps_done number of steps performed.               (may be NULL)
 * Entries past *steps_done are left untouched.  Output pointers may be host
 * or device memory.  Returns AFD_ERR_NUMERIC (with the steps done so far) if
 * an objective is not finite.
 */
afd_status afd_decompose(afd_plan* plan, const double* G, int K_max, double energy_tol,
                         double* a_out, double* coeff_out, double* delta_out, int* idx_out,
                         int* steps_done);

/*
 * Checkpoint and resume.  As afd_decompose, but starting from a remainder:
 *   G       2N doubles: G itself (E1_in = 0) or a remainder G_{k+1} returned by
 *           an earlier call (E1_in = that call's E_1).
 *   E1_in   0: a fresh start (E_1 = energy of G, a_1 = 0 imposed if the plan
 *           asks for it); > 0: the reference energy of the original signal,
 *           so delta keeps its meaning across calls (delta_out[0] = E(G)/E1_in).
 *   G_final 2N doubles (host or device, may be NULL): the remainder after the
 *           last step, i.e. the state to resume from.
 *   E1_out  (may be NULL): the E_1 used.
 * A decomposition split into calls this way gives bitwise the results of one
 * call (the state between greedy steps is exactly G_{k+1} and E_1).  The step
 * records of each call are numbered from 0.
 */
afd_status afd_decompose_from(afd_plan* plan, const double* G, double E1_in, int K_max, double energy_tol,
                              double* a_out, double* coeff_out, double* delta_out, int* idx_out,
                              int* steps_done, double* G_final, double* E1_out);

/*
 * Diagnostics of the plan's last afd_decompose (host pointers, may be NULL):
 *   n_cand_out  K entries: FP64 guard candidates per step (0 on the FP64 path);
 *   flags_out   K entries: bit 0 the candidate cap ended the list, bit 1 non-finite,
 *               bit 3 the point was refined off the grid (offgrid_iters);
 *   obj32_out   K entries: largest grid objective as computed by the grid kernel.
 * K is the number of steps of that call.
 */
afd_status afd_plan_last_info(const afd_plan* plan, int* n_cand_out, int* flags_out,
                              double* obj32_out);

/*
 * Kernel accounting of a plan since creation (or the last reset): launches of
 * the library's kernels and, while profiling is on, summed device times.
 * Profiling records CUDA events on the plan's stream between consecutive
 * kernels of the step sequence (inside the CUDA graph when graphs are used,
 * as event-record nodes), so the times are those of the kernels as they run
 * in the sequence; each profiled call synchronises once more to read them.
 * afd_plan_counters: all launches, grid-kernel launches and grid-kernel ms.
 * afd_plan_kernel_times: ms[5] and launches[5] per kernel kind, in the order
 * grid, guard, update, forward, persistent (the whole-decomposition kernel;
 * initialisation launches are not included).
 * Any output pointer may be NULL.
 */
afd_status afd_plan_set_profiling(afd_plan* plan, int on);
afd_status afd_plan_counters(const afd_plan* plan, long long* kernel_launches,
                             long long* grid_launches, double* grid_ms);
afd_status afd_plan_kernel_times(const afd_plan* plan, double* ms, long long* launches);

/*
 * Phase breakdown of the persistent kernel while profiling is on: average SM
 * clock cycles per greedy step, measured by the kernel's first CTA, in the
 * order: transforms and best pairs (A), wait at barrier 1, candidates and
 * guard sums (B), barrier 2, winner and remainder update (C), barrier 3,
 * energy and stop rule (D).  steps: greedy steps averaged over.
 */
afd_status afd_plan_phase_cycles(const afd_plan* plan, double* avg_cycles, long long* steps);
afd_status afd_plan_reset_counters(afd_plan* plan);

/*
 * The CUDA stream the plan's kernels run on (cudaStream_t): opts->stream if
 * one was given, else a stream the plan owns.  A plan-owned stream is ordered
 * after work already queued on the legacy default stream at every call.
 * Useful for recording CUDA events around calls.
 */
afd_status afd_plan_get_stream(const afd_plan* plan, void** stream);

/*
 * Batched Core AFD: n_signals independent decompositions of uneven N, run
 * together: all signals' grid tiles of one N share a launch and the N
 * classes run on parallel streams, the launch sequence replayed as one CUDA
 * graph when opts->use_graph is set; with opts->persistent = 2 and FP32-path
 * powers of two up to 16384, all K steps of every signal in one cooperative
 * persistent launch instead (all N-classes share each phase; bounded grid
 * barriers between phases).
 *   N        host array, n_signals sizes (each as for afd_plan_create, but not
 *            the FP32 two-pass size 65536).
 *   radii    host array of M radii shared by all signals.
 *   K_max    steps per signal (>= 1); energy_tol as for afd_decompose.
 * afd_batch_run takes the samples packed signal after signal (signal i starts
 * at 2 * (N_0 + ... + N_{i-1}) doubles) and writes, for signal i and step k:
 *   a_out[2(i K_max + k) + {0,1}], coeff_out likewise, idx_out likewise,
 *   delta_out[i (K_max + 1) + k], steps_out[i].
 * Any output may be NULL; pointers may be host or device memory.
 */
afd_status afd_batch_create(afd_batch** out, int n_signals, const int* N, const double* radii,
                            int M, int K_max, const afd_plan_opts* opts);
afd_status afd_batch_run(afd_batch* batch, const double* G_packed, double energy_tol,
                         double* a_out, double* coeff_out, double* delta_out, int* idx_out,
                         int* steps_out);
/*
 * The autotuner's choices: *n_groups N-classes; for the first max_groups of
 * them N, the grid-kernel variant (0 default, 1: 32 points per thread,
 * 2: 512-thread CTAs) and its measured time per launch in microseconds (0 if
 * not tuned).  Output pointers may be NULL.
 */
afd_status afd_batch_tuning(const afd_batch* batch, int max_groups, int* n_groups, int* N_out, int* variant_out,
                            float* us_out);

afd_status afd_batch_counters(const afd_batch* batch, long long* kernel_launches);
afd_status afd_batch_destroy(afd_batch* batch);

/* One-shot batch: create, run and destroy. */
afd_status afd_decompose_batch(int n_signals, const int* N, const double* radii, int M,
                               const double* G_packed, int K_max, double energy_tol,
                               const afd_plan_opts* opts, double* a_out, double* coeff_out,
                               double* delta_out, int* idx_out, int* steps_out);

/*
 * Partial sums of the expansion, Eq. (Sn) (Sec. 2):
 *   S_n(z_m) = sum_{k=1..n} coeff_k B_k(z_m),
 *   B_k(z) = sqrt(1-|a_k|^2)/(1 - conj(a_k) z) prod_{l<k} (z - a_l)/(1 - conj(a_l) z),
 * at the N points z_m = exp(2 pi i m / N), in FP64 (normalised measure: no
 * 1/sqrt(2 pi) factor).  With the a_k and coefficients afd_decompose returned,
 * ||G - S_n||^2 / ||G||^2 (discrete norms) equals delta_n.
 *   a, coeff  2n doubles each (interleaved complex); host or device memory.
 *   all_prefixes  0: S_out holds S_n (2N doubles); 1: S_out holds S_1..S_n,
 *                 one after another (2 N n doubles).
 * Synchronous; allocates device staging for host pointers.
 */
afd_status afd_synthesize(int N, const double* a, const double* coeff, int n, int all_prefixes,
                          double* S_out);

/*
 * Serving: continuous batching of independent decompositions.
 *
 * A server owns a worker thread and one CUDA stream.  Requests of any N
 * (as for afd_plan_create) and their own radii, step limit and energy
 * tolerance are queued by afd_serve_submit (any host thread; the samples are
 * copied at submission).  The worker admits queued requests oldest first into
 * device slots while the memory budget allows (slot buffers and the plan
 * tables of each distinct (N, radii) count against it), then repeatedly runs
 * a tick for every admitted request at once: with opts->persistent (default)
 * and FP32-path powers of two up to 16384, four greedy steps in one
 * multi-signal launch (each request stopping at its own last step);
 * otherwise one step, launches grouped by N.  After each tick it retires the
 * requests whose stop rule fired and admits waiting ones, so
 * requests that arrive while others run share the device.  Each request gets
 * the same result as afd_decompose with the server's options would give it
 * alone.
 *   mem_budget_bytes  device memory the server may hold (>= 1 MiB).
 *   opts              precision, guard and device options as for plans
 *                     (use_graph is ignored); NULL for defaults.
 * afd_serve_submit: AFD_ERR_BUDGET if the request alone cannot fit the
 *   budget; req_id receives the id.  G may be host or device memory.
 * afd_serve_poll: AFD_PENDING while the request runs; otherwise fills *out
 *   (may be NULL) and forgets the request, returning its status (AFD_OK,
 *   AFD_ERR_NUMERIC, AFD_ERR_CUDA ...).  AFD_ERR_NOT_FOUND for unknown ids.
 * afd_serve_wait: as poll, blocking up to timeout_s seconds (AFD_ERR_TIMEOUT).
 * afd_serve_destroy: stops the worker; unfinished requests are dropped.
 */
typedef struct afd_server afd_server;

typedef struct afd_result {
  int K_cap;          /* in: capacity (steps) of the caller's arrays below */
  double* a;          /* out, host, 2*K_cap (may be NULL) */
  double* coeff;      /* out, host, 2*K_cap (may be NULL) */
  double* delta;      /* out, host, K_cap+1 (may be NULL) */
  int* idx;           /* out, host, 2*K_cap (may be NULL) */
  int steps;          /* out: steps performed */
  int status;         /* out: afd_status of the request */
  double latency_ms;  /* out: submission to completion */
} afd_result;

typedef struct afd_serve_stats {
  unsigned long long submitted, completed, failed, ticks;
  long long kernel_launches;
  int queued, active;
  size_t bytes_reserved, bytes_in_use;
  unsigned long long suspended;  /* slots moved to host memory by afd_serve_suspend */
} afd_serve_stats;

afd_status afd_serve_create(afd_server** out, size_t mem_budget_bytes, const afd_plan_opts* opts);
afd_status afd_serve_submit(afd_server* server, int N, const double* radii, int M, const double* G,
                            int K_max, double energy_tol, uint64_t* req_id);
afd_status afd_serve_poll(afd_server* server, uint64_t req_id, afd_result* out);
afd_status afd_serve_wait(afd_server* server, uint64_t req_id, double timeout_s, afd_result* out);
/*
 * Slot eviction (no counterpart in the paper, which runs one decomposition at
 * a time).  afd_serve_suspend moves a request out of the device: a queued one
 * leaves the queue; an active one leaves its slot at the next step boundary
 * (its remainder G_k, step records and E_1 are copied to host memory and the
 * slot's memory is freed for other requests); the call blocks until then, at
 * most timeout_s seconds (AFD_ERR_TIMEOUT).  AFD_ERR_INVALID if the request
 * has finished (its result stays available), AFD_ERR_NOT_FOUND if unknown.
 * afd_serve_resume queues a suspended request again; its result is bitwise
 * the one it would have had without the suspension.  Polling a suspended
 * request returns AFD_PENDING.
 */
afd_status afd_serve_suspend(afd_server* server, uint64_t req_id, double timeout_s);
afd_status afd_serve_resume(afd_server* server, uint64_t req_id);
afd_status afd_serve_get_stats(afd_server* server, afd_serve_stats* out);
afd_status afd_serve_destroy(afd_server* server);

/*
 * Allocation-free FP64 inner products (the paper has no counterpart: this is
 * an interface addition for callers that cannot allocate device memory).
 *
 * out[p] = <G, e_{a_p}>~ = sqrt(1-|a_p|^2)/N * sum_m G(z_m) / (1 - a_p conj(z_m))
 * for n_points arbitrary points a_p of the open unit disc, by the same FP64
 * rectangle rule the FP32 path uses to re-evaluate its selection candidates.
 * Some callers cannot call cudaMalloc: work being recorded into a CUDA graph
 * (allocation is not allowed during stream capture and can synchronise the
 * device), latency-critical loops, and hosts that give the library a fixed
 * pre-reserved memory pool.  This entry point allocates nothing: its scratch
 * (partial sums and a completion counter) is a static device array of
 * 128 KiB + 256 B that every GPU loading the library holds until the process
 * exits.
 *   G       2N doubles (interleaved complex), device memory; 1 <= N <= AFD_NOALLOC_MAX_N.
 *   points  2*n_points doubles, device memory; 1 <= n_points <= AFD_NOALLOC_MAX_POINTS.
 *           Each point must satisfy |a_p| < 1 and differ from every sample
 *           point z_m; the points are not read by the host, so a point
 *           outside the open disc or on a sample gives NaN or Inf in out[p]
 *           (the call still returns AFD_OK).
 *   out     2*n_points doubles, device memory.
 *   stream  cudaStream_t to run on (NULL: the legacy default stream).
 * All three buffers must belong to the current device (or be host memory
 * mapped for it).  Asynchronous: the result is ready when the stream reaches
 * that point.  Sizes beyond the limits, NULL pointers, host (unmapped)
 * pointers and memory of another device return AFD_ERR_INVALID with a
 * message in afd_last_error().  The first call on a
 * device looks up the scratch array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * All calls share the one array: calls that overlap on the GPU (different
 * streams or host threads) race and must be serialised by the caller.
 */
#define AFD_NOALLOC_MAX_N 65536
#define AFD_NOALLOC_MAX_POINTS 64
afd_status afd_inner_products_noalloc(const double* G, int N, const double* points, int n_points,
                                      double* out, void* stream);

/*
 * Self-test of the bounded waits (failure detection without a GPU fault).
 * Every spin-wait in the library's kernels gives up after a fixed number of
 * polls, flags the signal and returns, so that the host reads
 * AFD_ERR_TIMEOUT and the CUDA context stays usable.  This call makes one
 * such wait run out on purpose: it launches one CTA on `device` (-1: the
 * current device) whose wait nothing can satisfy, then reads the kernel's
 * error bits.
 *   kind 0  the grid barrier of the persistent kernel: an arrival count of 2
 *           with one CTA arriving once;
 *   kind 1  the mbarrier wait of the TMA-staged N = 65536 passes: a phase
 *           expecting 16 bytes from a copy that is never issued.
 *   status   AFD_ERR_TIMEOUT when the wait ran out (the expected outcome),
 *            AFD_OK otherwise.
 *   seconds  how long the wait polled (the GPU's global timer).
 * Returns AFD_OK, AFD_ERR_INVALID (NULL pointer, unknown kind or device) or
 * AFD_ERR_CUDA / AFD_ERR_NOMEM.  Blocks the calling thread for the length of
 * the wait (seconds); allocates and frees a few hundred bytes of device memory.
 */
afd_status afd_selftest_wait_timeout(int device, int kind, afd_status* status, double* seconds);

#ifdef __cplusplus
}
#endif

#endif /* AFD_H */
