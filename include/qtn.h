/*
 * qtn.h -- C ABI of the GB300 slice-parallel tensor-network amplitude library.
 *
 * Method (arXiv 2010.14962, "Simulation of Quantum Computing on Classical
 * Supercomputers"): a QAOA circuit is turned into an undirected-graph tensor
 * network (Sec. II.A, Fig. 1: gates/inputs/measurements are vertices, wire
 * segments are edges); k edges are cut, which splits the contraction into
 * 2^k independent subnetworks of smaller width whose scalar results add up to
 * the full contraction (Sec. III.A, Eq. 2); each subnetwork is contracted by
 * pairwise contractions (Sec. II.A, Eq. 1) along an elimination order
 * (Sec. II.B); the cut set is searched greedily or by the genetic algorithm
 * of Sec. III.B (Algorithm 1).  Edges carry dimension 2 here: the library
 * computes amplitudes <x|C|0^n>, where the paper's density-matrix form uses
 * dimension 4 and gives |<x|C|0^n>|^2.
 *
 * Circuit: C = U_B(beta_p) U_C(gamma_p) ... U_B(beta_1) U_C(gamma_1) H^n with
 *   U_C(g) = prod_{(i,j) in E} exp(-i g Z_i Z_j)  (ZZ gates in lexicographic
 *   edge order) and U_B(b) = prod_q exp(-i b X_q) = RX(2b) on every qubit.
 * Bit strings: x[q] is the measured bit of qubit q (0 or 1).
 *
 * Conventions for every entry point:
 *   - Inputs are read (and copied where kept); the caller keeps ownership.
 *   - Handles are created by qtn_build_network / qtn_plan, owned by the
 *     library, immutable for the caller and freed by the *_destroy calls.
 *     Contraction calls on one plan from several host threads at once are
 *     serialised internally.
 *   - Every call returns a qtn_status; on failure nothing is written to the
 *     outputs and qtn_last_error() (per host thread) explains why.  The
 *     library never aborts the process.
 *   - Pointers documented as "device" must be CUDA device pointers on the
 *     current device; "host" pointers are ordinary host memory.
 *   - A NULL stream means the legacy default stream.  Calls that return
 *     results to host memory synchronise the stream before returning.
 */
#ifndef QTN_H_
#define QTN_H_

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QTN_OK = 0,
  QTN_ERR_INVALID_ARG = 1,      /* bad graph, cut, order, precision, size */
  QTN_ERR_OOM = 2,              /* host or device allocation failed */
  QTN_ERR_PLAN_EXCEEDS_CAP = 3, /* plan needs more memory than allowed */
  QTN_ERR_CUDA = 4,             /* a CUDA runtime call failed */
  QTN_ERR_TIMEOUT = 5,          /* a bounded device wait gave up */
  QTN_ERR_UNSUPPORTED = 6       /* valid request this build cannot run */
} qtn_status;

/* Arithmetic of the elimination steps.  Gate phases (sincos of gamma, beta)
 * and the sum over slices are FP64 in every mode (Kahan-compensated).
 * TF32 .. BF16X6 round or split the operands as stated and accumulate in
 * FP32.  On the on-chip executors they are emulated on the FP32 pipe (the
 * products tensor cores would form); on the wide executor, TF32 and TF32X3
 * merges whose shape allows it run on the tensor cores themselves (tcgen05,
 * FP32 accumulation in tensor memory, see qtn_wide_set_kernel). */
typedef enum {
  QTN_FP64 = 0,   /* complex128 contractions (the plain FP64 GPU form) */
  QTN_FP32 = 1,   /* complex64 contractions, FP32 FMA */
  QTN_TF32 = 2,   /* operands rounded to TF32, FP32 accumulate (tensor cores on wide merges) */
  QTN_BF16X3 = 3, /* split-BF16 (hi*hi + hi*lo + lo*hi), FP32 accumulate (emulated) */
  QTN_TF32X3 = 4, /* split-TF32, 3 products, FP32 accumulate (tensor cores on wide merges) */
  QTN_BF16X6 = 5, /* 3-way split BF16, 6 products, FP32 accumulate (emulated) */
  QTN_FP32X2 = 6  /* double-float complex (hi + lo FP32 pairs), ~44-bit */
} qtn_precision;

typedef struct qtn_network qtn_network_t;
typedef struct qtn_plan qtn_plan_t;

/* Builds the network of the p-layer QAOA circuit on graph (n, edges).
 *   edges : host, m pairs (i, j), 0 <= i, j < n, i != j, no duplicates (in
 *           either orientation); every qubit must appear in an edge.
 *   gamma, beta : host, p angles each.
 * Vertices are the ZZ gates; H|0>, the mixers and <x| are absorbed into
 * their neighbouring ZZ gate (rank <= 2 tensors), so the network has p*m
 * tensors and sum_q (p*deg(q) - 1) indices (Sec. II.A, Fig. 1). */
qtn_status qtn_build_network(int n, int p, const int32_t* edges, int m, const double* gamma,
                             const double* beta, qtn_network_t** out);

/* The graphical-model form of the same circuit (the undirected graphical
 * model in which diagonal gates share indices): the ZZ gates of a layer are
 * diagonal, so a qubit keeps one basis value z_q^(l) from one mixer to the
 * next.  Indices are these n * p variables (index (l - 1) * n + q is
 * z_q^(l)); tensors are the p * m ZZ factors exp(-i gamma_l s_i s_j) (rank
 * 2) and the p * n mixer factors <z_q^(l+1)| RX(2 beta_l) |z_q^(l)> (rank 2;
 * rank 1 in the last layer, whose row is x_q).  An index is held by every
 * factor of its layer on that qubit, so eliminating it merges all of them.
 * Its width is much smaller than the gate network's; plans, slices (Sec.
 * III.A: a cut fixes one variable in every factor that holds it) and all
 * contraction entry points work on it unchanged and give the same amplitude.
 * Arguments and errors as qtn_build_network; qtn_network_index reports
 * (qubit, pos = l - 1) and two of the index's holders. */
qtn_status qtn_build_network_gm(int n, int p, const int32_t* edges, int m, const double* gamma,
                                const double* beta, qtn_network_t** out);

/* The density form of an amplitude network (Sec. II.A: vertices are the
 * gates' superoperators G (x) conj(G), every edge has dimension 4).  An edge
 * of dimension 4 is a pair of binary indices: ket index i and bra index
 * i + I (I = the amplitude network's index count), with the same endpoints.
 * Cutting both indices of an edge fixes it to one of 4 values, so m cut
 * edges give 4^m slices (Sec. III.A).  Plans of this network contract
 * <x| rho |x> = |a(x)|^2 (returned as a complex value with zero imaginary
 * part up to rounding).  *out is a new handle owned by the caller.
 * QTN_ERR_INVALID_ARG if `amplitude` is NULL or already in density form;
 * QTN_ERR_UNSUPPORTED for a graphical-model network. */
qtn_status qtn_network_density(const qtn_network_t* amplitude, qtn_network_t** out);
void qtn_network_destroy(qtn_network_t* net);

/* Counts of tensors and indices.  Index ids 0..n_indices-1 are stable. */
qtn_status qtn_network_info(const qtn_network_t* net, int* n_tensors, int* n_indices);

/* Names index `index`: it is the wire segment of qubit *qubit that enters the
 * (*pos + 1)-th ZZ gate (0-based count) acting on that qubit; *tensor_a and
 * *tensor_b are its endpoint gates (earlier first).  Any output may be NULL. */
qtn_status qtn_network_index(const qtn_network_t* net, int index, int* qubit, int* pos, int* tensor_a,
                             int* tensor_b);

/* Cut-set search used when qtn_plan gets cuts == NULL. */
typedef enum {
  QTN_SEARCH_GREEDY = 0,  /* cut the index that most lowers the width, k times */
  QTN_SEARCH_GA = 1,      /* Algorithm 1 (Sec. III.B), seeded with the greedy set;
                             fitness = width, then total flops */
  QTN_SEARCH_GA_FLOPS = 2, /* Algorithm 1 with total log2 flops as the fitness */
  QTN_SEARCH_GA_NONZERO = 3 /* Algorithm 1 with the log2 flops of the slices that are
                               not structurally zero (cut classes) as the fitness,
                               width at most the greedy set's */
} qtn_search;

typedef struct {
  qtn_search search; /* default QTN_SEARCH_GREEDY */
  int k;             /* number of cuts to search for (cuts == NULL) */
  uint64_t seed;     /* GA seed (default 1) */
  int ga_T;          /* GA maximum iteration counter (default 4) */
  int ga_N;          /* GA population size (default 11) */
  double max_slice_bytes; /* 0 = no cap; else largest per-slice working set */
  int ga_seed_greedy;     /* GA: start from the greedy set plus random sets
                             (default 1) or from random sets only (0) */
  double time_budget_s;   /* GA: stop after the generation that exceeds it
                             (0 = run all T + 1 generations) */
} qtn_plan_opts;

/* Fills `opts` with the defaults (greedy search, k = 0, T = 4, N = 11,
 * greedy seed, no time budget). */
void qtn_plan_opts_default(qtn_plan_opts* opts);

/* Plans the sliced contraction (Sec. III.A) of `net`.
 *   cuts  : host, k distinct index ids to cut (slice bit j fixes cuts[j]);
 *           NULL = search opts->k cuts with opts->search.
 *   order : host, elimination order over the non-cut indices (each exactly
 *           once); NULL = min-fill (ties: fill, bag size, lowest id).
 *   opts  : NULL = defaults.
 * Fails with QTN_ERR_PLAN_EXCEEDS_CAP when opts->max_slice_bytes is set and
 * the plan's per-slice working set is larger. */
qtn_status qtn_plan(const qtn_network_t* net, const int32_t* cuts, int k, const int32_t* order,
                    int order_len, const qtn_plan_opts* opts, qtn_plan_t** out);
void qtn_plan_destroy(qtn_plan_t* plan);

/* Runs the cut-set search alone (no plan is built).
 *   opts->k cuts are written to `cuts` (host, opts->k entries).
 *   trace (host, trace_cap doubles, may be NULL): the search's fitness after
 *     each greedy cut, or the best fitness of each GA generation (Algorithm 1
 *     Step 1, then Step 5); fitness = width + log2(total flops) / 128.
 *   *trace_len, *evaluations: entries written and fitness evaluations done. */
qtn_status qtn_search_cuts(const qtn_network_t* net, const qtn_plan_opts* opts, int32_t* cuts,
                           double* trace, int trace_cap, int* trace_len, int* evaluations);

/* Exact cost of the plan (the method's own counter, Sec. II.B):
 *   log2_flops      : log2(2^k * 8 * complex MACs per slice)
 *   log2_peak_bytes : log2 of the largest live set of one slice (complex64)
 *   width           : largest |A u B| over the pairwise contractions
 *   k               : number of cuts.  Any output may be NULL. */
qtn_status qtn_plan_cost(const qtn_plan_t* plan, double* log2_flops, double* log2_peak_bytes,
                         int* width, int* k);

/* The plan's cut index ids (k entries, host) and MACs per slice. */
qtn_status qtn_plan_cuts(const qtn_plan_t* plan, int32_t* cuts);
qtn_status qtn_plan_macs_per_slice(const qtn_plan_t* plan, double* macs);

/* One amplitude a(x) = <x|C|0^n>, host in / host out.
 *   x   : host, n bytes.   out : host, out[0] = Re a, out[1] = Im a. */
qtn_status qtn_contract_amplitude(const qtn_plan_t* plan, const uint8_t* x, qtn_precision prec,
                                  cudaStream_t stream, double out[2]);

/* nx amplitudes of one plan with device-resident data (the throughput path).
 *   d_x   : device, nx * n bytes (row j = bit string j).
 *   d_out : device, nx * 2 doubles (Re, Im per bit string).
 * Asynchronous on `stream`, except that the first call for a given (prec,
 * nx) autotunes: it times every executor the plan compiled (per-class lane
 * executor, batched executors at two shared-memory budgets) on `stream`,
 * synchronising it, and keeps the fastest -- make that first call outside any
 * stream capture.  The first call for a given (d_x, d_out, nx, prec) records
 * a CUDA graph that later calls replay. */
qtn_status qtn_contract_amplitudes_device(const qtn_plan_t* plan, const uint8_t* d_x, int nx,
                                          qtn_precision prec, cudaStream_t stream, double* d_out);

/* Allocation-free variant of qtn_contract_amplitudes_device.  The paper has
 * no counterpart: this entry point exists for callers that cannot let a
 * library call cudaMalloc -- applications whose framework already holds the
 * device memory in its own pool, or code running where allocating is not
 * allowed or would stall.  Same arguments and results as
 * qtn_contract_amplitudes_device (FP64 and FP32 precisions).
 *   Memory: a fixed scratch array of 64 MiB inside the library, which every
 *     GPU that loads the library holds until the process exits.  The plan's
 *     program, the gate tensors of the nx bit strings and the per-block
 *     partial sums must fit in it; larger requests fail with
 *     QTN_ERR_INVALID_ARG (call again with fewer bit strings).  No call makes
 *     a device allocation or frees device memory.
 *   Set-up: the first call on each device looks up the array's device
 *     address with that device current; make that first call before any
 *     stream capture.  The array's 64 MiB are reserved on a device when the
 *     library part that holds it is loaded there: with CUDA's default lazy
 *     module loading that is this first call, so a caller whose framework
 *     then reserves the rest of the device memory should make its first call
 *     before that.
 *   Errors inside the kernels (an executor that meets a merge it cannot run)
 *     write NaN into that call's d_out; the call itself has already returned
 *     QTN_OK (nothing here synchronises).
 *   Sharing: all calls use the same array, so calls that overlap on the GPU
 *     (on different streams, or from racing host threads) corrupt each
 *     other; issue them on one stream.
 *   Launches its kernels directly on `stream` (no graph is recorded). */
qtn_status qtn_contract_amplitudes_noalloc(const qtn_plan_t* plan, const uint8_t* d_x, int nx,
                                           qtn_precision prec, cudaStream_t stream, double* d_out);

/* Amplitudes of nx (bit string, angle set) pairs of the plan's graph: the
 * gate tensors depend on gamma and beta (Sec. II.A) but the network's
 * topology, cut set and elimination order (Sec. II.B, III.A) do not, so one
 * plan serves a whole QAOA parameter scan.  Same launch as
 * qtn_contract_amplitudes_device, with the leaf tables of bit string i built
 * from angle set i.
 *   d_x     : device, nx * n bytes (0/1).
 *   d_gamma : device, nx * p doubles (angle set i at i * p).
 *   d_beta  : device, nx * p doubles.
 *   d_out   : device, 2 * nx doubles (scaled amplitudes).
 * Asynchronous on `stream`; the CUDA graph is cached per (d_x, d_gamma,
 * d_beta, d_out, nx, prec), so buffers reused across calls replay it.
 * QTN_ERR_INVALID_ARG for NULL buffers or nx <= 0. */
qtn_status qtn_contract_sweep_device(const qtn_plan_t* plan, const uint8_t* d_x, const double* d_gamma,
                                     const double* d_beta, int nx, qtn_precision prec, cudaStream_t stream,
                                     double* d_out);

/* Slices [slice_lo, slice_hi) of one amplitude, e.g. to recompute the slices
 * of a lost worker (Sec. V: fault tolerance at the level of subgraphs).
 *   x         : host, n bytes.
 *   out       : host, 4 doubles: the Kahan sum (Re, Im) of the range and its
 *               compensation terms (Re, Im), NOT scaled by 2^{-n/2}.
 *   d_slices  : optional device buffer of 2 * (slice_hi - slice_lo) doubles
 *               receiving every slice's scalar (unscaled), or NULL.
 * Synchronises `stream`. */
qtn_status qtn_contract_slices(const qtn_plan_t* plan, const uint8_t* x, uint64_t slice_lo,
                               uint64_t slice_hi, qtn_precision prec, cudaStream_t stream,
                               double out[4], double* d_slices);

/* Amplitudes of njobs independent (plan, x) jobs (Sec. III.A per job: each
 * job sums its own slices; the jobs share nothing but the launch).
 *   plans : host, njobs plan handles (different networks allowed).
 *   xs    : host, njobs pointers to host bit strings (n_j bytes of 0/1).
 *   out   : host, 2 * njobs doubles (Re, Im of job j at 2j, 2j+1).
 * When every job names the same plan, the jobs run as one multi-bit-string
 * launch of that plan's tuned program.  Otherwise one launch sequence runs
 * all jobs: their leaf tables, their hoisted merges (one block per job), a
 * persistent kernel whose blocks take (job, item range) chunks from a device
 * counter -- largest jobs first -- and a fixed-order per-job sum of the chunk
 * partials, so results do not depend on the block schedule.  Each job runs
 * the level program of its plan (of this precision's width) that executes
 * the fewest multiply-adds and fits in shared memory, with as many items per
 * block as fit (1024 threads); if some job has none that fits, every job
 * runs its 48 KiB batched (else per-class) block program instead.
 * The multi-plan sequence (uploads, kernels, read-backs) is captured as a
 * CUDA graph the first time a list of plans is seen (with that precision
 * and time limit) and replayed afterwards.  Jobs whose plan has no level
 * program that fits the multi-job executor (tensors too large for shared
 * memory: the wide executor, see qtn_wide_set_kernel; or programs that fit
 * only the single-plan executors) run after that sequence, each on its
 * plan's tuned executor (as qtn_contract_amplitude); the cancel word and time
 * limit do not apply to them.
 * Errors: QTN_ERR_INVALID_ARG (NULL plan, bad x), QTN_ERR_UNSUPPORTED (a
 * job's working set exceeds shared memory), QTN_ERR_TIMEOUT (stopped, see
 * qtn_batch_cancel), QTN_ERR_CUDA.  Internal device and pinned buffers are
 * kept between calls (grow-only); calls from several host threads are
 * serialised.  Synchronises `stream`. */
qtn_status qtn_contract_batch(const qtn_plan_t* const* plans, const uint8_t* const* xs, int njobs,
                              qtn_precision prec, cudaStream_t stream, double* out);

/* Cooperative stop of multi-plan batches (jobs of several plans; Sec. V:
 * a lost or stalled part of the work is noticed and can be recomputed).  The
 * persistent executor checks, before each chunk of work, a host-mapped
 * cancel word and a time budget; nothing on the device waits.  A stopped
 * call returns QTN_ERR_TIMEOUT and no amplitudes; the library and device stay
 * usable.
 *   qtn_batch_cancel         : stops the multi-plan qtn_contract_batch call
 *                              in progress (from any host thread; a call that
 *                              starts afterwards is not affected).
 *   qtn_batch_set_time_limit : ms of executor time each block may use per
 *                              call (0: no limit, the default); applies to
 *                              later calls.  QTN_ERR_INVALID_ARG if ms < 0. */
qtn_status qtn_batch_cancel(void);
qtn_status qtn_batch_set_time_limit(double ms);

/* Device time (ms) of the most recent multi-plan qtn_contract_batch launch
 * sequence (the replayed graph: bit-string and descriptor uploads, leaf
 * tables to per-job sums, read-backs; CUDA events on its stream), and the
 * number of kernels it launched.  QTN_ERR_INVALID_ARG if none ran yet. */
qtn_status qtn_batch_last_ms(float* ms, int* kernels);

/* The program each job of the most recent qtn_contract_batch call ran (its
 * name as in qtn_plan_describe's "programs"), as a JSON array in job order;
 * measurement support (the paper has no counterpart).  Writes at most `cap`
 * bytes (NUL-terminated) to `buf` when `cap` is large enough; always sets
 * *len to the size needed ("[]" before any batch). */
qtn_status qtn_batch_last_programs(char* buf, size_t cap, size_t* len);

/* Which executor the plan runs on ("lane": one slice per GPU thread, for
 * plans with every tensor rank <= 5; "block": one slice per thread block). */
qtn_status qtn_plan_executor(const qtn_plan_t* plan, const char** name);

/* Overrides the autotuner: contraction calls of (prec, nx) use the executor
 * called `name` (one of the names in qtn_plan_describe's "programs", other
 * than the per-slice program).  "<level program>/jit" and "<level
 * program>/jit2" name the kernel generated at run time for that level
 * program and precision (fp64, fp32, fp32x2): every merge of Eq. 1 as
 * straight code; "/jit2" with the two-phase schedule (the levels of small
 * merges run on more items at once, their results parked in a device scratch
 * area the plan owns, then reloaded for the later levels).  Fails with
 * QTN_ERR_INVALID_ARG for an unknown name or one compiled for the other
 * precision, QTN_ERR_UNSUPPORTED if no run-time compiler is available or no
 * two-phase schedule fits the program. */
qtn_status qtn_plan_select_executor(const qtn_plan_t* plan, qtn_precision prec, int nx, const char* name);

/* Kernel timing for measurement: when on, qtn_contract_amplitudes_device
 * launches its three kernels directly (no graph replay) and records CUDA
 * events on the launching stream just before and after the executor kernel;
 * qtn_plan_kernel_ms returns the executor's duration in the most recent such
 * call once its stream has been synchronised. */
qtn_status qtn_plan_set_kernel_timing(const qtn_plan_t* plan, int on);
qtn_status qtn_plan_kernel_ms(const qtn_plan_t* plan, float* ms);

/* Process-wide override of the wide executor's kernel per elimination step
 * (measurement and tests; the paper has no counterpart).  The wide executor
 * runs plans whose per-slice tensors exceed shared memory with its
 * intermediates in device memory, one launch per merge (Eq. 1) and group of
 * slices; an autotuner picks, per merge shape, the SIMT kernel ("simt", one
 * output per thread; "simt4", four), or the tensor-core kernel ("tcgen05":
 * complex merges as real TF32 GEMMs with FP32 accumulation in tensor memory,
 * available to QTN_TF32 and QTN_TF32X3 where one side of the merge has at
 * least 128 entries, the other at least 8, and at least 4 entries are
 * summed).  name: "auto" (the default: autotuned), "simt", "simt4" or
 * "tcgen05" (every step that allows it; the others stay autotuned).  Takes
 * effect at each wide state's next launch outside stream capture.
 * Autotuned winners are kept per process, keyed by (ma, nb, kb, bb, items
 * per launch, arithmetic); if the environment variable QTN_WIDE_TUNE_CACHE
 * names a file, the first tuning of the process reads winners from it (one
 * JSON object per line) and every tuning writes the table back.
 * QTN_ERR_INVALID_ARG for an unknown name. */
qtn_status qtn_wide_set_kernel(const char* name);

/* Measured arithmetic peaks of the current device, the denominators of the
 * executors' roofline fractions (measurement support; the paper has no
 * counterpart).  A grid of several blocks per SM runs independent FP32 (and
 * then FP64) fused multiply-add chains; the best of `reps` timed launches
 * (CUDA events, default stream, synchronous) gives *fp32_tflops and
 * *fp64_tflops (host), counting a multiply-add as 2 flops.  Takes about
 * 50 ms per rep on a GB300.  QTN_ERR_INVALID_ARG for null outputs or
 * reps < 1; QTN_ERR_CUDA if a launch fails. */
qtn_status qtn_pipe_peaks(int reps, double* fp32_tflops, double* fp64_tflops);

/* The same measurement with packed FP32 pairs (one fma.rn.f32x2 instruction
 * is two multiply-adds; sm_100 and later), the FP32 roof of the executors
 * that use them.  *tflops (host) counts a multiply-add as 2 flops.
 * QTN_ERR_UNSUPPORTED on an older device, QTN_ERR_INVALID_ARG for a null
 * output or reps < 1, QTN_ERR_CUDA if a launch fails. */
qtn_status qtn_pipe_peak_fp32x2(int reps, double* tflops);

/* Check of the double-float (QTN_FP32X2) arithmetic on the device (test
 * support; the paper has no counterpart): `count` complex dot products of K
 * terms, a (host, count x K complex values as re, im pairs, row i = item i)
 * times b (same layout), each operand rounded to a double word.
 * out_scalar[2i..2i+1] (host) gets item i by the scalar double-float
 * sequence, out_merge by the form the contraction kernels' merge loops run
 * (packed FP32 pairs on sm_100 and later, then *packed = 1; packed may be
 * NULL).  Allocates and frees its own device buffers and synchronises.
 * QTN_ERR_INVALID_ARG for null pointers, count < 0, count > 2^24, K < 1 or
 * K > 4096; QTN_ERR_CUDA if a CUDA call fails. */
qtn_status qtn_arith_check(const double* a, const double* b, int count, int K, double* out_scalar,
                           double* out_merge, int* packed);

/* ------------------------------------------------ learned cost surrogate --
 * A small MLP predicts the exact counter's log2 total flops and log2 peak
 * bytes of cutting a set of indices (min-fill plan) from cheap features, so a
 * genetic cut search (Algorithm 1, Sec. III.B) can rank far more candidates;
 * the exact counter still scores the candidates the search keeps.  Training
 * and inference run on the device (FP32, the library's own kernels). */
typedef struct qtn_mlp qtn_mlp_t;
#define QTN_SURROGATE_FEATURES 48
#define QTN_SURROGATE_TARGETS 2

/* Features of cutting `cuts` (k index ids) out of `net` (host, 48 floats):
 * sizes, the cut pattern, the gate graph left after cutting and the bag
 * sizes of a min-degree elimination. */
qtn_status qtn_surrogate_features(const qtn_network_t* net, const int32_t* cuts, int k, float* out);
/* The exact labels of the same (host, 2 floats): log2 total flops and log2
 * peak bytes of the min-fill plan. */
qtn_status qtn_surrogate_labels(const qtn_network_t* net, const int32_t* cuts, int k, float* out);

/* `count` labelled samples (host X: count x 48, Y: count x 2 = exact log2
 * flops, log2 peak bytes) on random connected 3-regular graphs with even
 * n in [n_lo, n_hi], p in [p_lo, p_hi], k in [k_lo, k_hi]; sample i depends
 * only on (seed, i); `threads` host threads. */
qtn_status qtn_surrogate_dataset(int count, int n_lo, int n_hi, int p_lo, int p_hi, int k_lo, int k_hi,
                                 uint64_t seed, int threads, float* X, float* Y);

/* An MLP in -> hidden -> hidden -> out (ReLU), He-initialised from `seed`. */
qtn_status qtn_mlp_create(int in, int hidden, int out, uint64_t seed, qtn_mlp_t** mlp);
void qtn_mlp_destroy(qtn_mlp_t* mlp);
qtn_status qtn_mlp_num_params(const qtn_mlp_t* mlp, size_t* n);
/* Parameters (host, num_params floats: W1 b1 W2 b2 W3 b3, row-major W[out][in])
 * read (set = 0) or written (set = 1). */
qtn_status qtn_mlp_params(qtn_mlp_t* mlp, float* params, int set);
/* Input / target normalisation (mean, std per column) read or written. */
qtn_status qtn_mlp_normalisation(qtn_mlp_t* mlp, float* x_mean, float* x_std, float* y_mean, float* y_std,
                                 int set);
/* Gradients (host, num_params floats) of mean((Y_pred - Y)^2) over the n x out
 * normalised outputs for raw rows X (n x in), Y (n x out); *loss (optional)
 * receives that mean.  No parameter changes. */
qtn_status qtn_mlp_gradients(qtn_mlp_t* mlp, const float* X, const float* Y, int n, float* grads, float* loss);
/* Trains with Adam (lr, betas 0.9/0.999) on mini-batches of `batch` shuffled
 * rows for `epochs` epochs; the normalisation is set from X, Y.  epoch_loss
 * (optional, host, epochs floats) receives the mean loss of each epoch. */
qtn_status qtn_mlp_fit(qtn_mlp_t* mlp, const float* X, const float* Y, int n, int epochs, int batch, float lr,
                       uint64_t seed, float* epoch_loss);
/* Predictions (host Y: n x out) for raw feature rows (host X: n x in). */
qtn_status qtn_mlp_predict(qtn_mlp_t* mlp, const float* X, int n, float* Y);

/* Surrogate-guided genetic cut search for k cuts: population N (seeded with
 * the greedy set if seed_greedy, else random), generations t = 0..T ranked by the surrogate's predicted
 * log2 flops; each generation the `top` best are evaluated exactly and the
 * best exact set is kept.  Writes the best set by the exact counter (k
 * entries), its exact log2 total flops, the numbers of exact and surrogate
 * evaluations, and the best exact value per generation (trace). */
qtn_status qtn_search_cuts_surrogate(const qtn_network_t* net, int k, qtn_mlp_t* mlp, int T, int N, int top,
                                     uint64_t seed, int seed_greedy, int32_t* cuts, double* best_log2_flops,
                                     int* exact_evals, int* surrogate_evals, double* trace, int trace_cap,
                                     int* trace_len);

/* Introspection: a JSON description of the plan (cuts, elimination order,
 * merges, tensor index sets, both executors' step programs, gate legs), for
 * tests and tooling.  Writes at most `cap` bytes (NUL-terminated) to `buf`
 * when `cap` is large enough; always sets *len to the size needed. */
qtn_status qtn_plan_describe(const qtn_plan_t* plan, char* buf, size_t cap, size_t* len);

/* The schedule the kernel generator would give level program `program` (a
 * name from qtn_plan_describe's "programs") for precision `prec`, with
 * `smem_cap` bytes of shared memory per block, as JSON (test support for the
 * generator's host logic; no device is used): items per pass, arena stride,
 * and for two_phase != 0 the split level, the items per pass and arena
 * stride of the levels below it, and the tensors it parks ([arena offset,
 * elements, park offset] each).  Buffer convention as qtn_plan_describe.
 * QTN_ERR_INVALID_ARG for an unknown program or precision;
 * QTN_ERR_UNSUPPORTED if it is not a level program or no schedule of that
 * form fits. */
qtn_status qtn_plan_jit_schedule(const qtn_plan_t* plan, const char* program, qtn_precision prec, int two_phase,
                                 size_t smem_cap, char* buf, size_t cap, size_t* len);

/* The CUDA source the generator emits for the same program, precision and
 * schedule (test support; the run-time compiler is not called): kernels
 * "qtn_level_jit" and, for programs with hoisted merges in levels,
 * "qtn_prologue_jit".  Arguments, buffer convention and errors as
 * qtn_plan_jit_schedule; QTN_ERR_UNSUPPORTED also for a precision the
 * generator has no form for (TF32 and the split forms). */
qtn_status qtn_plan_jit_source(const qtn_plan_t* plan, const char* program, qtn_precision prec, int two_phase,
                               size_t smem_cap, char* buf, size_t cap, size_t* len);

const char* qtn_status_string(qtn_status s);
const char* qtn_last_error(void); /* per host thread; "" if none */

#ifdef __cplusplus
}
#endif
#endif /* QTN_H_ */
